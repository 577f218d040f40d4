// capi.cu — the C ABI declared in include/hm.h: argument checks, the build
// pipeline (tree -> partition -> batched ACA + recompression -> storage plan
// -> near field -> chunk copies), the products, GMRES, statistics and the
// inspection / import entry points.  Every entry point turns internal
// exceptions into an hm_status; nothing aborts.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <sstream>

#include <unordered_set>

#include "hm_internal.h"

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;
std::atomic<long long> g_hm_launches{0};

void hm_set_error(const std::string& msg) { g_last_error = msg; }
[[noreturn]] void hm_throw(hm_status st, const std::string& msg) { throw hm_error{st, msg}; }
void hm_check_cuda(cudaError_t e, const char* what, const char* file, int line) {
    if (e == cudaSuccess) return;
    (void)cudaGetLastError();
    const hm_status st = (e == cudaErrorMemoryAllocation) ? HM_ERR_OOM : HM_ERR_CUDA;
    throw hm_error{st, std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                           std::to_string(line) + ")"};
}

void* hm_dmalloc(std::vector<DevBuf>& owner, size_t bytes, cudaStream_t st, bool zero) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) == cudaErrorMemoryAllocation) {
        // memory the library's pool keeps for later builds and solves goes back first
        cudaGetLastError();
        HM_CUDA(cudaDeviceSynchronize());
        hm_scratch_trim();
        HM_CUDA(cudaMalloc(&p, bytes ? bytes : 16));
    }
    HM_CUDA(cudaGetLastError());
    owner.push_back({p, bytes});
    if (zero && bytes) HM_CUDA(cudaMemsetAsync(p, 0, bytes, st));
    return p;
}

void* hm_dmalloc_pooled(std::vector<DevBuf>& owner, size_t bytes, cudaStream_t st) {
    void* p = hm_scratch_alloc(bytes, st);
    owner.push_back({p, bytes, true, st});
    return p;
}

#define HM_API_BEGIN try {
#define HM_API_END                                  \
    }                                               \
    catch (const hm_error& e) {                     \
        hm_set_error(e.msg);                        \
        return e.st;                                \
    }                                               \
    catch (const std::bad_alloc&) {                 \
        hm_set_error("host allocation failed");     \
        return HM_ERR_OOM;                          \
    }                                               \
    catch (...) {                                   \
        hm_set_error("unexpected internal error");  \
        return HM_ERR_CUDA;                         \
    }                                               \
    return HM_OK;

namespace {

using clk = std::chrono::steady_clock;
double ms_since(clk::time_point t0) {
    return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
}

void free_all(std::vector<DevBuf>& owner) {
    for (DevBuf& d : owner)
        if (d.p) {
            if (d.pooled)
                hm_scratch_free(d.p, d.st);
            else
                cudaFree(d.p);
        }
    owner.clear();
}

// A pair of CUDA events bracketing work on one stream.
struct EvPair {
    cudaEvent_t a = nullptr, b = nullptr;
    explicit EvPair(cudaStream_t st) {
        HM_CUDA(cudaEventCreate(&a));
        HM_CUDA(cudaEventCreate(&b));
        HM_CUDA(cudaEventRecord(a, st));
    }
    double stop(cudaStream_t st) {
        HM_CUDA(cudaEventRecord(b, st));
        HM_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        HM_CUDA(cudaEventElapsedTime(&ms, a, b));
        return ms;
    }
    ~EvPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

bool finite_all(const double* p, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// ACA + recompression of every admissible block of one or several problems
// (one launch serves blocks of every problem), in batches bounded by the
// workspace budget.  Writes the FP32 factors (U' column-major 3m x r', V'
// 3n x r') into staging buffers owned by `staging` and records per block the
// pointers and ranks.  Options, eps and the recompression switch are those of
// the first problem (a batch shares them).
void build_low_rank(std::vector<hm_matrix*>& hs, std::vector<DevBuf>& staging,
                    std::vector<std::vector<const float2*>>& su,
                    std::vector<std::vector<const float2*>>& sv, cudaStream_t st) {
    hm_matrix* h0 = hs[0];
    const int nprob = (int)hs.size();
    // admissible blocks of all problems: (problem, block)
    std::vector<int32_t> aq;
    std::vector<int64_t> ab;
    for (int q = 0; q < nprob; ++q)
        for (int64_t b = 0; b < (int64_t)hs[q]->blocks.size(); ++b)
            if (hs[q]->blocks[b].admissible) {
                aq.push_back(q);
                ab.push_back(b);
            }
    const int64_t na = (int64_t)aq.size();
    auto blk_of = [&](int64_t a) -> hm_block& { return hs[aq[a]]->blocks[ab[a]]; };
    auto cl_of = [&](int64_t a, int64_t c) -> const hm_cluster& { return hs[aq[a]]->clusters[c]; };
    auto pts_of = [&](int64_t a, int64_t c) { return cl_of(a, c).end - cl_of(a, c).begin; };
    auto size_of = [&](int64_t a) { return pts_of(a, blk_of(a).tau) + pts_of(a, blk_of(a).sigma); };
    std::vector<int64_t> adm(na);
    std::iota(adm.begin(), adm.end(), 0);
    std::stable_sort(adm.begin(), adm.end(), [&](int64_t a, int64_t b) { return size_of(a) > size_of(b); });
    int cap0 = h0->opts.aca_max_rank > 0 ? h0->opts.aca_max_rank : 144;
    cap0 = std::max(3, cap0 - cap0 % 3);
    // Workspace of one ACA batch: the caller's bound, else half of the device
    // memory free when the batch is formed.  One launch takes the whole batch
    // with a dynamic queue, largest blocks first, so the SMs stay busy until its
    // last small blocks; each extra batch ends on the few CTAs that still hold
    // its largest blocks while the others idle (at 65 536 points four 24 GiB
    // batches took the ACA 573 ms, one 80 GB batch 350 ms).
    auto batch_budget = [&]() -> int64_t {
        if (h0->opts.workspace_bytes > 0) return h0->opts.workspace_bytes;
        size_t fr = 0, tot = 0;
        HM_CUDA(cudaMemGetInfo(&fr, &tot));
        return std::max<int64_t>((int64_t)((fr + hm_scratch_cached()) / 2), 1ll << 30);
    };
    int nsm = 0;
    HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h0->device));
    std::vector<int> cap(na, 0);
    for (int64_t a = 0; a < na; ++a) {
        const int64_t full = 3 * std::min(pts_of(a, blk_of(a).tau), pts_of(a, blk_of(a).sigma));
        cap[a] = (int)std::min<int64_t>(full, cap0);
    }
    int used_model = 0;
    if (h0->opts.rank_model && na > 0) {
        // learned capacities: predicted rank-3 steps with a safety margin; the
        // ACA still decides the rank and overflowing blocks are re-run
        std::vector<float> feats(6 * na), pred(na);
        for (int64_t a = 0; a < na; ++a) {
            const hm_matrix* hq = hs[aq[a]];
            rank_features(cl_of(a, blk_of(a).tau), cl_of(a, blk_of(a).sigma), hq->gp.ks, hq->gp.kp,
                          hq->eps, &feats[6 * a]);
        }
        std::vector<DevBuf> tmp;
        float* dP = (float*)hm_dmalloc(tmp, HM_RANK_MODEL_PARAMS * 4, st, false);
        float* dF = (float*)hm_dmalloc(tmp, feats.size() * 4, st, false);
        float* dO = (float*)hm_dmalloc(tmp, na * 4, st, false);
        HM_CUDA(cudaMemcpyAsync(dP, h0->opts.rank_model, HM_RANK_MODEL_PARAMS * 4, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(dF, feats.data(), feats.size() * 4, cudaMemcpyHostToDevice, st));
        rank_model_predict_dev(dP, dF, na, dO, st);
        HM_CUDA(cudaMemcpyAsync(pred.data(), dO, na * 4, cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        free_all(tmp);
        const float tm = h0->opts.rank_model[12], ts = h0->opts.rank_model[13];
        for (int64_t a = 0; a < na; ++a) {
            const double steps = std::exp((double)pred[a] * ts + tm) - 1.0;
            const int64_t full = 3 * std::min(pts_of(a, blk_of(a).tau), pts_of(a, blk_of(a).sigma));
            int64_t c = 3 * (int64_t)std::ceil(1.25 * std::max(steps, 0.0) + 2.0);
            if (!std::isfinite(steps)) c = cap0;
            cap[a] = (int)std::max<int64_t>(3, std::min<int64_t>({c, full, 768}));
        }
        // bin blocks of similar predicted rank into the same batches
        std::stable_sort(adm.begin(), adm.end(), [&](int64_t a, int64_t b) {
            if (cap[a] != cap[b]) return cap[a] > cap[b];
            return size_of(a) > size_of(b);
        });
        used_model = 1;
    }
    // points, normals and Green parameters: the problem's own, or all problems
    // concatenated (job point offsets become global, J.pad_ names the problem)
    std::vector<int64_t> poff(nprob, 0);
    const double* d_pts = h0->d_pts_p;
    const double* d_nrm = h0->d_nrm_p;
    const GreenParams* d_gps = nullptr;
    std::vector<DevBuf> batchbuf;
    if (nprob > 1) {
        int64_t tot = 0;
        bool any_nrm = false, any_w = false;
        for (int q = 0; q < nprob; ++q) {
            poff[q] = tot;
            tot += hs[q]->nc;
            any_nrm = any_nrm || hs[q]->d_nrm_p;
            any_w = any_w || hs[q]->gp.w;
        }
        double* pa = (double*)hm_dmalloc(batchbuf, 24 * tot, st, false);
        double* na3 = any_nrm ? (double*)hm_dmalloc(batchbuf, 24 * tot, st, true) : nullptr;
        double* wa = any_w ? (double*)hm_dmalloc(batchbuf, 8 * tot, st, false) : nullptr;
        std::vector<GreenParams> gps(nprob);
        for (int q = 0; q < nprob; ++q) {
            HM_CUDA(cudaMemcpyAsync(pa + 3 * poff[q], hs[q]->d_pts_p, 24 * hs[q]->nc, cudaMemcpyDeviceToDevice, st));
            if (hs[q]->d_nrm_p)
                HM_CUDA(cudaMemcpyAsync(na3 + 3 * poff[q], hs[q]->d_nrm_p, 24 * hs[q]->nc,
                                        cudaMemcpyDeviceToDevice, st));
            gps[q] = hs[q]->gp;
            if (hs[q]->gp.w) {
                HM_CUDA(cudaMemcpyAsync(wa + poff[q], hs[q]->gp.w, 8 * hs[q]->nc, cudaMemcpyDeviceToDevice, st));
                gps[q].w = wa;  // indexed by the global point index
            }
        }
        GreenParams* dg = (GreenParams*)hm_dmalloc(batchbuf, nprob * sizeof(GreenParams), st, false);
        HM_CUDA(cudaMemcpyAsync(dg, gps.data(), nprob * sizeof(GreenParams), cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaStreamSynchronize(st));
        d_pts = pa;
        d_nrm = na3;
        d_gps = dg;
    }
    double ev_aca = 0, t_aca = 0, ev_rec = 0, t_rec = 0, flops = 0, flops64 = 0, flops_df = 0,
           evals = 0, flops_apply = 0;
    int64_t batches = 0, reruns = 0, ws_peak = 0, ws_tot = 0;
    std::vector<int64_t> n_rsvd(nprob, 0), n_uncert(nprob, 0);
    double t_rsvd = 0;
    std::vector<int64_t> lost;  // admissible blocks for the randomized SVD
    int* d_counter = (int*)hm_dmalloc(staging, sizeof(int), st, true);
    // recompression of factors in d_work (Sec. 3.2) and their FP32 staging
    // copies (U' 3m x r', V' 3n x r'): jobs keep[q] of the list ids
    auto stage = [&](const std::vector<int64_t>& ids, const std::vector<int64_t>& keep,
                     const std::vector<int64_t>& uo, const std::vector<int64_t>& vo,
                     const std::vector<int64_t>& m3, const std::vector<int64_t>& n3,
                     const std::vector<int32_t>& kk, const std::vector<int64_t>& go,
                     const std::vector<int32_t>& gl, const double2* d_gram, double2* d_work,
                     const float4* d_work_df, double eps_r) {
        std::vector<int32_t> ranks;
        std::vector<int64_t> soff;
        EvPair er(st);
        void* rb = recompress_core(uo, vo, m3, n3, kk, go, gl, d_gram, h0->opts.recompress, d_work,
                                   eps_r, ranks, soff, st);
        try {
            int64_t tot = 0;
            std::vector<int64_t> so(keep.size());
            for (size_t q = 0; q < keep.size(); ++q) {
                so[q] = tot;
                tot += (m3[q] + n3[q]) * ranks[q];
            }
            float2* d_stage = (float2*)hm_dmalloc_pooled(staging, std::max<int64_t>(tot, 1) * 8, st);
            std::vector<int64_t> job_of, row0, dst;
            std::vector<int32_t> which, rows, ldv;
            for (size_t q = 0; q < keep.size(); ++q) {
                if (ranks[q] == 0) continue;
                for (int side = 0; side < 2; ++side) {
                    const int64_t R = side == 0 ? m3[q] : n3[q];
                    const int64_t base = so[q] + (side == 0 ? 0 : m3[q] * ranks[q]);
                    for (int64_t r0 = 0; r0 < R; r0 += 192) {
                        job_of.push_back((int64_t)q);
                        which.push_back(side);
                        row0.push_back(r0);
                        rows.push_back((int32_t)std::min<int64_t>(192, R - r0));
                        dst.push_back(base + r0);
                        ldv.push_back((int32_t)R);
                    }
                }
            }
            recompress_apply(rb, job_of, which, row0, rows, dst, ldv, ranks, d_work, d_work_df, d_stage, st);
            for (size_t q = 0; q < keep.size(); ++q)  // U' = U T_U, V' = V T_V in double-float
                flops_apply += 8.0 * (double)(m3[q] + n3[q]) * kk[q] * ranks[q];
            ev_rec += er.stop(st);
            for (size_t q = 0; q < keep.size(); ++q) {
                const int64_t a = ids[keep[q]];
                hm_block& bk = blk_of(a);
                bk.rank_aca = kk[q];
                bk.rank = ranks[q];
                su[aq[a]][ab[a]] = d_stage + so[q];
                sv[aq[a]][ab[a]] = d_stage + so[q] + m3[q] * ranks[q];
            }
            HM_CUDA(cudaStreamSynchronize(st));
        } catch (...) {
            recompress_release(rb, st);
            throw;
        }
        recompress_release(rb, st);
    };
    std::vector<int64_t> todo = adm;
    try {
    while (!todo.empty()) {
        std::vector<int64_t> overflow;
        size_t pos = 0;
        while (pos < todo.size()) {
            // ---- form a batch ----
            const int64_t budget = batch_budget();
            std::vector<AcaJob> jobs;
            std::vector<int64_t> ids;
            int64_t woff = 0, goff = 0, maxm = 1, maxn = 1;
            int capmax = 3;
            while (pos < todo.size()) {
                const int64_t a = todo[pos];
                const hm_block& bk = blk_of(a);
                const int64_t m = pts_of(a, bk.tau), n = pts_of(a, bk.sigma);
                // double-float factors (16 bytes an entry), Gram matrices
                const int64_t need = (3 * (m + n) * (int64_t)cap[a] + 2 * (int64_t)cap[a] * cap[a]) * 16;
                if (!jobs.empty() && (woff + goff) * 16 + need > budget) break;
                AcaJob J;
                J.tau_begin = poff[aq[a]] + cl_of(a, bk.tau).begin;
                J.m = m;
                J.sig_begin = poff[aq[a]] + cl_of(a, bk.sigma).begin;
                J.n = n;
                J.u_off = woff;
                J.v_off = woff + 3 * m * cap[a];
                J.g_off = goff;
                J.cap = cap[a];
                J.pad_ = aq[a];
                woff += 3 * (m + n) * cap[a];
                goff += 2 * (int64_t)cap[a] * cap[a];
                maxm = std::max(maxm, m);
                maxn = std::max(maxn, n);
                capmax = std::max(capmax, cap[a]);
                jobs.push_back(J);
                ids.push_back(a);
                ++pos;
            }
            const int64_t nj = (int64_t)jobs.size();
            ws_peak = std::max<int64_t>(ws_peak, (woff + goff) * 16);
            ws_tot += (woff + goff) * 16;
            const int nctas = (int)std::min<int64_t>(nj, (int64_t)nsm * aca_ctas_per_sm(capmax));
            std::vector<DevBuf> tmp;
            auto t0 = clk::now();
            // the factors as double-float pairs only: every reader takes those
            // (the residuals, the norm update, the factor application), the
            // recompression takes the Gram matrices the ACA accumulates
            double2* d_work = nullptr;
            float4* d_work_df = (float4*)hm_dmalloc_pooled(tmp, (size_t)woff * 16, st);
            double2* d_gram = (double2*)hm_dmalloc_pooled(tmp, (size_t)goff * 16, st);
            AcaJob* d_jobs = (AcaJob*)hm_dmalloc(tmp, nj * sizeof(AcaJob), st, false);
            AcaResult* d_res = (AcaResult*)hm_dmalloc(tmp, nj * sizeof(AcaResult), st, false);
            const int64_t fstride = hm_round_up(maxm + maxn, 16);
            unsigned char* d_flags = (unsigned char*)hm_dmalloc(tmp, (size_t)nctas * fstride, st, false);
            const int64_t rbs = 9 * maxn + maxn / 2 + 1, cbs = 9 * maxm + maxm / 2 + 1;
            double2* d_rb = (double2*)hm_dmalloc(tmp, (size_t)nctas * rbs * 16, st, false);
            double2* d_cb = (double2*)hm_dmalloc(tmp, (size_t)nctas * cbs * 16, st, false);
            HM_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), nj * sizeof(AcaJob), cudaMemcpyHostToDevice, st));
            EvPair ea(st);
            launch_aca(h0->gp, d_pts, d_nrm, d_jobs, nj, d_work, d_gram, d_flags, fstride, d_rb,
                       d_cb, rbs, cbs, h0->eps, d_res, nctas, capmax, d_counter, st, d_gps, d_work_df);
            ev_aca += ea.stop(st);
            std::vector<AcaResult> res(nj);
            HM_CUDA(cudaMemcpyAsync(res.data(), d_res, nj * sizeof(AcaResult), cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaStreamSynchronize(st));
            t_aca += ms_since(t0);
            batches++;
            // ---- recompression of the converged jobs ----
            t0 = clk::now();
            std::vector<int64_t> uo, vo, m3, n3, keep, go;
            std::vector<int32_t> kk, gl;
            for (int64_t j = 0; j < nj; ++j) {
                if (res[j].status == 2)
                    hm_throw(HM_ERR_NUMERIC, "non-finite value in the ACA of a block");
                if (res[j].status == 3) {  // rows the vector ACA cannot pivot: randomized SVD
                    lost.push_back(ids[j]);
                    continue;
                }
                if (res[j].status == 1) {
                    const int64_t a = ids[j];
                    const int64_t full = 3 * std::min(jobs[j].m, jobs[j].n);
                    const int nc2 = (int)std::min<int64_t>({full, 2 * (int64_t)cap[a], 768});
                    if (nc2 <= cap[a]) hm_throw(HM_ERR_UNSUPPORTED, "ACA rank above 768 columns");
                    cap[a] = nc2;
                    overflow.push_back(a);
                    continue;
                }
                {
                    // per rank-3 step with k = 3s columns built (8 flops per complex
                    // multiply-add): residual row and column 9 k (m + n), cross terms of
                    // the norm update / Gram columns 9 k (m + n) and new Gram diagonal
                    // blocks 27 (m + n), all in double-float; factor columns U = C gamma
                    // 27 m in FP64; m + n Green's tensor evaluations (FP64)
                    const double K = res[j].k / 3, mn = (double)(jobs[j].m + jobs[j].n);
                    const double cross = 8.0 * 9.0 * mn * 3.0 * (K * (K - 1.0) / 2.0);
                    flops += 2.0 * cross;
                    flops_df += 2.0 * cross + 8.0 * 27.0 * mn * K;
                    flops64 += 8.0 * 27.0 * (double)jobs[j].m * K;
                    evals += mn * K;
                }
                keep.push_back(j);
                uo.push_back(jobs[j].u_off);
                vo.push_back(jobs[j].v_off);
                m3.push_back(3 * jobs[j].m);
                n3.push_back(3 * jobs[j].n);
                kk.push_back(res[j].k);
                go.push_back(jobs[j].g_off);
                gl.push_back(jobs[j].cap);
            }
            stage(ids, keep, uo, vo, m3, n3, kk, go, gl, d_gram, d_work, d_work_df, h0->eps);
            HM_CUDA(cudaStreamSynchronize(st));
            free_all(tmp);
            t_rec += ms_since(t0);
        }
        reruns += (int64_t)overflow.size();
        todo.swap(overflow);
    }
    if (!lost.empty()) {
        // randomized SVD of the blocks the vector ACA could not pivot (remark
        // of Sec. 2.3), in groups whose FP64 blocks fit the workspace budget
        auto t0 = clk::now();
        std::vector<DevBuf> gbuf;
        const GreenParams* gps = d_gps;
        if (!gps) {
            GreenParams* g = (GreenParams*)hm_dmalloc(gbuf, sizeof(GreenParams), st, false);
            HM_CUDA(cudaMemcpyAsync(g, &h0->gp, sizeof(GreenParams), cudaMemcpyHostToDevice, st));
            gps = g;
        }
        size_t pos = 0;
        while (pos < lost.size()) {
            const int64_t budget = batch_budget();
            std::vector<RsvdBlock> rb;
            std::vector<int64_t> ids;
            int64_t bytes = 0;
            while (pos < lost.size()) {
                const int64_t a = lost[pos];
                const hm_block& bk = blk_of(a);
                const int64_t m = pts_of(a, bk.tau), n = pts_of(a, bk.sigma);
                const int64_t need = 9 * m * n * 16 + 2 * 3 * (m + n) * 776 * 16;
                if (!rb.empty() && (bytes + need > budget || rb.size() >= 65535)) break;  // grid.y
                RsvdBlock B;
                B.tau_global = poff[aq[a]] + cl_of(a, bk.tau).begin;
                B.sig_global = poff[aq[a]] + cl_of(a, bk.sigma).begin;
                B.m = m;
                B.n = n;
                B.key = rsvd_key(cl_of(a, bk.tau).begin, cl_of(a, bk.sigma).begin);
                B.prob = nprob > 1 ? aq[a] : 0;
                rb.push_back(B);
                ids.push_back(a);
                bytes += need;
                ++pos;
            }
            std::vector<DevBuf> tmp;
            EvPair ea(st);
            double2* W = rsvd_factors(rb, gps, d_pts, d_nrm, h0->eps, tmp, st);
            ev_aca += ea.stop(st);
            std::vector<int64_t> keep, uo, vo, m3, n3, go;
            std::vector<int32_t> kk, gl;
            for (size_t q = 0; q < rb.size(); ++q) {
                keep.push_back((int64_t)q);
                uo.push_back(rb[q].u_off);
                vo.push_back(rb[q].v_off);
                m3.push_back(3 * rb[q].m);
                n3.push_back(3 * rb[q].n);
                kk.push_back(rb[q].l);
                go.push_back(-1);  // Gram matrices formed by the recompression itself
                gl.push_back(0);
                n_rsvd[aq[ids[q]]]++;
                if (!rb[q].certified) n_uncert[aq[ids[q]]]++;
            }
            // range error <= eps/2 (certified), truncation eps sqrt(3)/2: total <= eps
            stage(ids, keep, uo, vo, m3, n3, kk, go, gl, nullptr, W, nullptr, h0->eps * std::sqrt(3.0) / 2);
            HM_CUDA(cudaStreamSynchronize(st));
            free_all(tmp);
        }
        free_all(gbuf);
        t_rsvd = ms_since(t0);
    }
    } catch (...) {
        cudaStreamSynchronize(st);
        free_all(batchbuf);
        throw;
    }
    free_all(batchbuf);
    for (int q = 0; q < nprob; ++q) {
        hs[q]->rsvd_blocks = n_rsvd[q];
        hs[q]->t_rsvd_ms += t_rsvd;
        hs[q]->rsvd_uncertified = n_uncert[q];
    }
    for (hm_matrix* h : hs) {  // a batch reports the shared launches in every handle
        h->ev_aca_ms += ev_aca;
        h->t_aca_ms += t_aca;
        h->ev_recomp_ms += ev_rec;
        h->t_recomp_ms += t_rec;
        h->aca_flops += flops;
        h->aca_flops_fp64 += flops64;
        h->aca_flops_df += flops_df;
        h->aca_green_evals += evals;
        h->apply_flops_df += flops_apply;
        h->aca_batches += batches;
        h->aca_overflow_reruns += reruns;
        h->aca_workspace_peak = std::max(h->aca_workspace_peak, ws_peak);
        h->aca_workspace_total += ws_tot;
        h->used_rank_model = used_model;
        h->batch_problems = nprob;
    }
}

double box_diam(const hm_cluster& c) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) s += (c.hi[a] - c.lo[a]) * (c.hi[a] - c.lo[a]);
    return std::sqrt(s);
}
double box_dist(const hm_cluster& x, const hm_cluster& y) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double g = std::max({0.0, x.lo[a] - y.hi[a], y.lo[a] - x.hi[a]});
        s += g * g;
    }
    return std::sqrt(s);
}

hm_status validate_common(const hm_matrix* h) {
    if (!h) {
        hm_set_error("null handle");
        return HM_ERR_ARG;
    }
    return HM_OK;
}

}  // namespace

void rank_features(const hm_cluster& t, const hm_cluster& s, double ks, double kp, double eps,
                   float f[6]) {
    const double D = std::max({box_diam(t), box_diam(s), 1e-30});
    f[0] = (float)(ks * D);
    f[1] = (float)(kp * D);
    f[2] = (float)(box_dist(t, s) / D);
    f[3] = (float)std::log2((double)(t.end - t.begin));
    f[4] = (float)std::log2((double)(s.end - s.begin));
    f[5] = (float)std::log10(eps);
}

// Validation, handle, points, tree, weights, normals and partition of one
// problem (everything before the low-rank blocks).  The handle is owned by
// `hold` until the caller releases it.
struct HandleHold {
    hm_matrix* p = nullptr;
    void reset(hm_matrix* h) { p = h; }
    hm_matrix* release() {
        hm_matrix* h = p;
        p = nullptr;
        return h;
    }
    ~HandleHold() {
        if (p) hm_free(p);
    }
};

hm_matrix* build_setup(const double* points, const double* normals, int64_t n_c, double rho,
                       double lambda, double mu, double omega, int32_t kernel, double eps,
                       double eta, int64_t leaf_size, const hm_opts* opts, cudaStream_t st,
                       HandleHold& hold) {
    if (!points || n_c < 1) hm_throw(HM_ERR_ARG, "null pointer or n_c < 1");
    if (!(rho > 0) || !(mu > 0) || !(omega > 0) || !std::isfinite(rho) || !std::isfinite(mu) ||
        !std::isfinite(omega) || !std::isfinite(lambda) || !(lambda + 2 * mu > 0))
        hm_throw(HM_ERR_ARG, "material parameters must be finite with rho, mu, omega > 0");
    if (!(eps > 0 && eps < 1)) hm_throw(HM_ERR_ARG, "eps must lie in (0, 1)");
    if (!(eta > 0) || !std::isfinite(eta)) hm_throw(HM_ERR_ARG, "eta must be positive");
    if (kernel != HM_KERNEL_U && kernel != HM_KERNEL_T) hm_throw(HM_ERR_ARG, "unknown kernel");
    if (kernel == HM_KERNEL_T && !normals) hm_throw(HM_ERR_ARG, "the T kernel needs normals");
    if (leaf_size < 1) hm_throw(HM_ERR_ARG, "leaf_size must be >= 1");
    if (leaf_size > 1024) hm_throw(HM_ERR_UNSUPPORTED, "leaf_size above 1024 points");
    if (!finite_all(points, 3 * n_c)) hm_throw(HM_ERR_ARG, "non-finite point coordinates");
    if (kernel == HM_KERNEL_T && !finite_all(normals, 3 * n_c))
        hm_throw(HM_ERR_ARG, "non-finite normals");
    hm_opts o;
    hm_opts_default(&o);
    if (opts) o = *opts;
    if (o.storage != HM_STORE_FP32 && o.storage != HM_STORE_BF16)
        hm_throw(HM_ERR_ARG, "unknown storage type");
    if (!std::isfinite(o.diag_value)) hm_throw(HM_ERR_ARG, "non-finite diag_value");
    if (!(o.fp64_switch_ksr > 0)) hm_throw(HM_ERR_ARG, "fp64_switch_ksr must be > 0 (or +inf)");
    if (o.aca_fp32 != 0)
        hm_throw(HM_ERR_ARG, "aca_fp32 must be 0: the ACA residual rows and columns run in "
                             "double-float arithmetic, there is no FP32 variant");
    hm_matrix* h = new hm_matrix();
    hold.reset(h);
    h->nc = n_c;
    h->kernel = kernel;
    h->rho = rho;
    h->lam = lambda;
    h->mu = mu;
    h->omega = omega;
    h->eps = eps;
    h->eta = eta;
    h->leaf = leaf_size;
    h->opts = o;
    h->gp = make_green_params(kernel, rho, lambda, mu, omega, o.diag_value);
    h->gp.ksr_switch = o.fp64_switch_ksr;
    HM_CUDA(cudaGetDevice(&h->device));
    // ---- points -> device, tree ----
    auto t0 = clk::now();
    h->d_pts_p = (double*)hm_dmalloc(h->owner, 24 * n_c, st, false);
    h->d_perm = (int64_t*)hm_dmalloc(h->owner, 8 * n_c, st, false);
    {
        std::vector<int64_t> iota(n_c);
        std::iota(iota.begin(), iota.end(), 0);
        HM_CUDA(cudaMemcpyAsync(h->d_pts_p, points, 24 * n_c, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(h->d_perm, iota.data(), 8 * n_c, cudaMemcpyHostToDevice, st));
        TreeResult tr = build_cluster_tree(h->d_pts_p, h->d_perm, n_c, leaf_size, st);
        h->clusters = std::move(tr.clusters);
        h->perm = std::move(tr.perm);
        h->depth = tr.depth;
    }
    // coincident points share every split, hence a leaf: the Green's tensor of two
    // distinct points at distance 0 is singular (Eq. elasto_U), so such input is refused
    for (const hm_cluster& c : h->clusters) {
        if (!c.is_leaf) continue;
        for (int64_t a = c.begin; a < c.end; ++a)
            for (int64_t b = a + 1; b < c.end; ++b) {
                const double* pa = points + 3 * h->perm[a];
                const double* pb = points + 3 * h->perm[b];
                if (pa[0] == pb[0] && pa[1] == pb[1] && pa[2] == pb[2]) {
                    char msg[160];
                    std::snprintf(msg, sizeof(msg), "coincident points %lld and %lld",
                                  (long long)std::min(h->perm[a], h->perm[b]),
                                  (long long)std::max(h->perm[a], h->perm[b]));
                    hm_throw(HM_ERR_ARG, msg);
                }
            }
    }
    if (o.weights) {
        std::vector<double> wp(n_c);
        for (int64_t p = 0; p < n_c; ++p) wp[p] = o.weights[h->perm[p]];
        if (!finite_all(wp.data(), n_c)) hm_throw(HM_ERR_ARG, "non-finite weights");
        double* d_w = (double*)hm_dmalloc(h->owner, 8 * n_c, st, false);
        HM_CUDA(cudaMemcpyAsync(d_w, wp.data(), 8 * n_c, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaStreamSynchronize(st));
        h->gp.w = d_w;
        h->opts.weights = nullptr;  // the caller's array is not kept
    }
    if (kernel == HM_KERNEL_T) {
        std::vector<double> np(3 * n_c);
        for (int64_t p = 0; p < n_c; ++p)
            for (int a = 0; a < 3; ++a) np[3 * p + a] = normals[3 * h->perm[p] + a];
        h->d_nrm_p = (double*)hm_dmalloc(h->owner, 24 * n_c, st, false);
        HM_CUDA(cudaMemcpyAsync(h->d_nrm_p, np.data(), 24 * n_c, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaStreamSynchronize(st));
    }
    h->t_tree_ms = ms_since(t0);
    // ---- partition ----
    t0 = clk::now();
    h->blocks = build_partition(h->clusters, eta, st);
    h->t_part_ms = ms_since(t0);
    return h;
}

// Two clouds (Sec. 4: collocation points x_i as rows, integration points y_j
// with their normals and weights as columns): the handle holds both clouds,
// targets first, each with its own cluster tree (the rule of Sec. 2.1), and
// the partition pairs a target cluster with a source cluster from the two
// roots.  Its operator is the rectangular A (3 n_x x 3 n_y) embedded in the
// square index space of n_x + n_y points: every block couples target rows with
// source columns, so the product reads the source part of x and writes the
// target part of y (the source part stays zero).
hm_matrix* build_setup2(const double* targets, int64_t n_x, const double* sources,
                        const double* normals, int64_t n_y, double rho, double lambda, double mu,
                        double omega, int32_t kernel, double eps, double eta, int64_t leaf_size,
                        const hm_opts* opts, cudaStream_t st, HandleHold& hold) {
    if (!targets || !sources || n_x < 1 || n_y < 1) hm_throw(HM_ERR_ARG, "null pointer or empty cloud");
    if (!(rho > 0) || !(mu > 0) || !(omega > 0) || !std::isfinite(rho) || !std::isfinite(mu) ||
        !std::isfinite(omega) || !std::isfinite(lambda) || !(lambda + 2 * mu > 0))
        hm_throw(HM_ERR_ARG, "material parameters must be finite with rho, mu, omega > 0");
    if (!(eps > 0 && eps < 1)) hm_throw(HM_ERR_ARG, "eps must lie in (0, 1)");
    if (!(eta > 0) || !std::isfinite(eta)) hm_throw(HM_ERR_ARG, "eta must be positive");
    if (kernel != HM_KERNEL_U && kernel != HM_KERNEL_T) hm_throw(HM_ERR_ARG, "unknown kernel");
    if (kernel == HM_KERNEL_T && !normals) hm_throw(HM_ERR_ARG, "the T kernel needs source normals");
    if (leaf_size < 1 || leaf_size > 1024) hm_throw(HM_ERR_ARG, "leaf_size must be in 1..1024");
    if (!finite_all(targets, 3 * n_x) || !finite_all(sources, 3 * n_y))
        hm_throw(HM_ERR_ARG, "non-finite point coordinates");
    if (kernel == HM_KERNEL_T && !finite_all(normals, 3 * n_y)) hm_throw(HM_ERR_ARG, "non-finite normals");
    hm_opts o;
    hm_opts_default(&o);
    if (opts) o = *opts;
    if (o.storage != HM_STORE_FP32 && o.storage != HM_STORE_BF16)
        hm_throw(HM_ERR_ARG, "unknown storage type");
    if (!std::isfinite(o.diag_value)) hm_throw(HM_ERR_ARG, "non-finite diag_value");
    if (!(o.fp64_switch_ksr > 0)) hm_throw(HM_ERR_ARG, "fp64_switch_ksr must be > 0 (or +inf)");
    if (o.aca_fp32 != 0) hm_throw(HM_ERR_ARG, "aca_fp32 must be 0");
    {  // a source at a target's position has a singular Green's tensor (Eq. elasto_U)
        struct Key {
            double x, y, z;
            bool operator==(const Key& k) const { return x == k.x && y == k.y && z == k.z; }
        };
        struct Hash {
            size_t operator()(const Key& k) const {
                const std::hash<double> h;
                return h(k.x) ^ (h(k.y) * 1000003u) ^ (h(k.z) * 998244353u);
            }
        };
        std::unordered_set<Key, Hash> tset;
        for (int64_t i = 0; i < n_x; ++i) tset.insert({targets[3 * i], targets[3 * i + 1], targets[3 * i + 2]});
        for (int64_t j = 0; j < n_y; ++j)
            if (tset.count({sources[3 * j], sources[3 * j + 1], sources[3 * j + 2]})) {
                char msg[120];
                std::snprintf(msg, sizeof(msg), "source point %lld coincides with a target point",
                              (long long)j);
                hm_throw(HM_ERR_ARG, msg);
            }
    }
    hm_matrix* h = new hm_matrix();
    hold.reset(h);
    const int64_t n = n_x + n_y;
    h->nc = n;
    h->n_targets = n_x;
    h->kernel = kernel;
    h->rho = rho;
    h->lam = lambda;
    h->mu = mu;
    h->omega = omega;
    h->eps = eps;
    h->eta = eta;
    h->leaf = leaf_size;
    h->opts = o;
    h->gp = make_green_params(kernel, rho, lambda, mu, omega, o.diag_value);
    h->gp.ksr_switch = o.fp64_switch_ksr;
    HM_CUDA(cudaGetDevice(&h->device));
    auto t0 = clk::now();
    h->d_pts_p = (double*)hm_dmalloc(h->owner, 24 * n, st, false);
    h->d_perm = (int64_t*)hm_dmalloc(h->owner, 8 * n, st, false);
    {
        std::vector<int64_t> iota(n);
        std::iota(iota.begin(), iota.end(), 0);
        HM_CUDA(cudaMemcpyAsync(h->d_pts_p, targets, 24 * n_x, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(h->d_pts_p + 3 * n_x, sources, 24 * n_y, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(h->d_perm, iota.data(), 8 * n, cudaMemcpyHostToDevice, st));
        TreeResult tx = build_cluster_tree(h->d_pts_p, h->d_perm, n_x, leaf_size, st);
        TreeResult ty = build_cluster_tree(h->d_pts_p + 3 * n_x, h->d_perm + n_x, n_y, leaf_size, st);
        const int64_t cx = (int64_t)tx.clusters.size();
        h->clusters = std::move(tx.clusters);
        for (hm_cluster c : ty.clusters) {
            c.begin += n_x;
            c.end += n_x;
            if (c.child0 >= 0) c.child0 += cx;
            if (c.child1 >= 0) c.child1 += cx;
            h->clusters.push_back(c);
        }
        h->perm = std::move(tx.perm);
        h->perm.insert(h->perm.end(), ty.perm.begin(), ty.perm.end());  // already global indices
        h->depth = std::max(tx.depth, ty.depth);
        h->sigma_root = cx;
    }
    {  // source weights (W_y of Sec. 4) in tree order; targets carry 1 (never read)
        std::vector<double> wp(n, 1.0);
        if (o.weights) {
            for (int64_t p = n_x; p < n; ++p) wp[p] = o.weights[h->perm[p] - n_x];
            if (!finite_all(wp.data(), n)) hm_throw(HM_ERR_ARG, "non-finite weights");
            double* d_w = (double*)hm_dmalloc(h->owner, 8 * n, st, false);
            HM_CUDA(cudaMemcpyAsync(d_w, wp.data(), 8 * n, cudaMemcpyHostToDevice, st));
            HM_CUDA(cudaStreamSynchronize(st));
            h->gp.w = d_w;
        }
        h->opts.weights = nullptr;
    }
    if (kernel == HM_KERNEL_T) {  // source normals in tree order; targets zero (never read)
        std::vector<double> np(3 * n, 0.0);
        for (int64_t p = n_x; p < n; ++p)
            for (int a = 0; a < 3; ++a) np[3 * p + a] = normals[3 * (h->perm[p] - n_x) + a];
        h->d_nrm_p = (double*)hm_dmalloc(h->owner, 24 * n, st, false);
        HM_CUDA(cudaMemcpyAsync(h->d_nrm_p, np.data(), 24 * n, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaStreamSynchronize(st));
    }
    h->t_tree_ms = ms_since(t0);
    t0 = clk::now();
    h->blocks = build_partition(h->clusters, eta, st, h->sigma_root);
    h->t_part_ms = ms_since(t0);
    return h;
}

// Storage plan, arena, near field, factor chunks (BF16 copy) and work vectors
// once the low-rank factors of the problem are staged.  `staged` (or null)
// owns staging memory that is released once this problem's factors are in
// the arena: the driver's unmapping of a multi-gigabyte allocation then
// overlaps the rest of the build instead of delaying the caller's first
// products by up to a millisecond.
void build_finish(hm_matrix* h, std::vector<const float2*>& su, std::vector<const float2*>& sv,
                  std::vector<DevBuf>* staged, cudaStream_t st) {
    const hm_opts& o = h->opts;
    auto t0 = clk::now();
    std::vector<int64_t> t_off;
    h->plan = build_matvec_plan(h->clusters, h->blocks, t_off);
    h->t_plan_ms = ms_since(t0);
    auto tp = clk::now();
    h->mv = matvec_dev_create(h->plan, o.storage, h->owner, st);
    h->t_arena_ms = ms_since(tp);
    auto tn = clk::now();
    assemble_dense(h->gp, h->d_pts_p, h->d_nrm_p, h->plan, h->blocks, h->clusters, h->mv, h->owner,
                   st);
    HM_CUDA(cudaStreamSynchronize(st));
    h->t_near_ms = ms_since(tn);
    auto tc = clk::now();
    copy_staged_chunks(h->mv, h->plan, h->blocks, h->clusters, su, sv, st);
    HM_CUDA(cudaStreamSynchronize(st));
    if (staged) free_all(*staged);
    h->t_stage_ms = ms_since(tc);
    tc = clk::now();
    if (o.storage == HM_STORE_BF16) {
        matvec_make_bf16(h->mv, h->plan, h->owner, st);
        HM_CUDA(cudaStreamSynchronize(st));
    }
    h->t_bf16_ms = ms_since(tc);
    h->t_copy_ms = ms_since(t0) - h->t_near_ms;
    h->d_xp = (float2*)hm_dmalloc(h->owner, 8 * 3 * h->nc, st, true);
    h->d_yp = (float2*)hm_dmalloc(h->owner, 8 * 3 * h->nc, st, true);
    HM_CUDA(cudaStreamSynchronize(st));
    tc = clk::now();
    tune_product(h, o.tune_cache, st);  // times products on d_xp / d_yp
    h->opts.tune_cache = nullptr;        // the caller's string is not kept
    h->t_tune_ms = ms_since(tc);
    tc = clk::now();
    matvec_graph_prepare(h->mv, h->d_perm, h->d_xp, h->d_yp, h->nc);
    h->t_graph_ms = ms_since(tc);
}

void report_build(const hm_matrix* h) {
    if (h->opts.verbose)
        std::fprintf(stderr,
                     "[hm] n_c=%lld blocks=%zu tree=%.1fms part=%.1fms aca=%.1fms recomp=%.1fms "
                     "near=%.1fms copy=%.1fms total=%.1fms\n",
                     (long long)h->nc, h->blocks.size(), h->t_tree_ms, h->t_part_ms, h->t_aca_ms,
                     h->t_recomp_ms, h->t_near_ms, h->t_copy_ms, h->t_total_ms);
}

extern "C" {

void hm_opts_default(hm_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->storage = HM_STORE_FP32;
    o->aca_fp32 = 0;
    o->diag_value = 1.0;
    o->fp64_switch_ksr = INFINITY;
    o->recompress = 1;
    o->aca_max_rank = 0;
    o->workspace_bytes = 0;
    o->verbose = 0;
    o->weights = nullptr;
    o->rank_model = nullptr;
}

const char* hm_status_string(hm_status s) {
    switch (s) {
        case HM_OK: return "ok";
        case HM_ERR_ARG: return "invalid argument";
        case HM_ERR_CUDA: return "CUDA error";
        case HM_ERR_OOM: return "out of device memory";
        case HM_ERR_NOCONV: return "GMRES did not converge";
        case HM_ERR_TIMEOUT: return "device wait timed out";
        case HM_ERR_NUMERIC: return "non-finite value";
        case HM_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char* hm_last_error(void) { return g_last_error.c_str(); }

hm_status hm_build(const double* points, const double* normals, int64_t n_c, double rho,
                   double lambda, double mu, double omega, int32_t kernel, double eps, double eta,
                   int64_t leaf_size, const hm_opts* opts, void* stream, hm_handle* out) {
    if (out) *out = nullptr;
    HM_API_BEGIN
    if (!out) hm_throw(HM_ERR_ARG, "null output handle");
    cudaStream_t st = (cudaStream_t)stream;
    const auto t_all = clk::now();
    HandleHold hold;
    hm_matrix* h = build_setup(points, normals, n_c, rho, lambda, mu, omega, kernel, eps, eta,
                               leaf_size, opts, st, hold);
    std::vector<hm_matrix*> hs{h};
    std::vector<DevBuf> staging;
    std::vector<std::vector<const float2*>> su(1), sv(1);
    su[0].assign(h->blocks.size(), nullptr);
    sv[0].assign(h->blocks.size(), nullptr);
    try {
        build_low_rank(hs, staging, su, sv, st);
        build_finish(h, su[0], sv[0], &staging, st);
    } catch (...) {
        cudaStreamSynchronize(st);
        free_all(staging);
        throw;
    }
    free_all(staging);
    h->t_total_ms = ms_since(t_all);
    report_build(h);
    *out = hold.release();
    HM_API_END
}

hm_status hm_build2(const double* targets, int64_t n_x, const double* sources,
                    const double* normals, int64_t n_y, double rho, double lambda, double mu,
                    double omega, int32_t kernel, double eps, double eta, int64_t leaf_size,
                    const hm_opts* opts, void* stream, hm_handle* out) {
    if (out) *out = nullptr;
    HM_API_BEGIN
    if (!out) hm_throw(HM_ERR_ARG, "null output handle");
    cudaStream_t st = (cudaStream_t)stream;
    const auto t_all = clk::now();
    HandleHold hold;
    hm_matrix* h = build_setup2(targets, n_x, sources, normals, n_y, rho, lambda, mu, omega, kernel,
                                eps, eta, leaf_size, opts, st, hold);
    std::vector<hm_matrix*> hs{h};
    std::vector<DevBuf> staging;
    std::vector<std::vector<const float2*>> su(1), sv(1);
    su[0].assign(h->blocks.size(), nullptr);
    sv[0].assign(h->blocks.size(), nullptr);
    try {
        build_low_rank(hs, staging, su, sv, st);
        build_finish(h, su[0], sv[0], &staging, st);
    } catch (...) {
        cudaStreamSynchronize(st);
        free_all(staging);
        throw;
    }
    free_all(staging);
    h->t_total_ms = ms_since(t_all);
    report_build(h);
    *out = hold.release();
    HM_API_END
}

hm_status hm_build_batch(int32_t nprob, const hm_problem* probs, double eps, const hm_opts* opts,
                         void* stream, hm_handle* out) {
    if (out && nprob > 0)
        for (int32_t q = 0; q < nprob; ++q) out[q] = nullptr;
    HM_API_BEGIN
    if (!out || !probs || nprob < 1) hm_throw(HM_ERR_ARG, "null pointer or nprob < 1");
    cudaStream_t st = (cudaStream_t)stream;
    const auto t_all = clk::now();
    std::vector<HandleHold> hold(nprob);
    std::vector<hm_matrix*> hs(nprob);
    hm_opts o;
    hm_opts_default(&o);
    if (opts) o = *opts;
    for (int32_t q = 0; q < nprob; ++q) {
        const hm_problem& P = probs[q];
        o.weights = P.weights;
        hs[q] = build_setup(P.points, P.normals, P.n_c, P.rho, P.lambda, P.mu, P.omega, P.kernel,
                            eps, P.eta, P.leaf_size, &o, st, hold[q]);
    }
    std::vector<DevBuf> staging;
    std::vector<std::vector<const float2*>> su(nprob), sv(nprob);
    for (int32_t q = 0; q < nprob; ++q) {
        su[q].assign(hs[q]->blocks.size(), nullptr);
        sv[q].assign(hs[q]->blocks.size(), nullptr);
    }
    try {
        build_low_rank(hs, staging, su, sv, st);
        for (int32_t q = 0; q < nprob; ++q)
            build_finish(hs[q], su[q], sv[q], q + 1 == nprob ? &staging : nullptr, st);
    } catch (...) {
        cudaStreamSynchronize(st);
        free_all(staging);
        throw;
    }
    free_all(staging);
    const double tot = ms_since(t_all);
    for (int32_t q = 0; q < nprob; ++q) {
        hs[q]->t_total_ms = tot;
        report_build(hs[q]);
    }
    for (int32_t q = 0; q < nprob; ++q) out[q] = hold[q].release();
    HM_API_END
}

hm_status hm_matvec(hm_handle h, int32_t nrhs, const void* x, void* y, void* stream) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (!x || !y || nrhs < 1) hm_throw(HM_ERR_ARG, "null vector or nrhs < 1");
    const int64_t n = 3 * h->nc;
    const char* xb = (const char*)x;
    const char* yb = (const char*)y;
    const int64_t bytes = n * nrhs * 16;
    if (xb < yb + bytes && yb < xb + bytes) hm_throw(HM_ERR_ARG, "x and y overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (nrhs > 1 && h->opts.storage == HM_STORE_BF16) {
        matvec_multi(h->mv, h->d_perm, (const double2*)x, (double2*)y, h->nc, nrhs, st);
        return HM_OK;
    }
    for (int32_t c = 0; c < nrhs; ++c) {
        matvec_graph(h->mv, h->d_perm, (const double2*)x + c * n, h->d_xp, h->d_yp,
                     (double2*)y + c * n, h->nc, st);
    }
    HM_API_END
}

hm_status hm_matvec_host(hm_handle h, int32_t nrhs, const void* x, void* y, void* stream) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (!x || !y || nrhs < 1) hm_throw(HM_ERR_ARG, "null vector or nrhs < 1");
    const int64_t n = 3 * h->nc;
    cudaStream_t st = (cudaStream_t)stream;
    if (h->staging_cols < nrhs) {
        std::vector<DevBuf> keep;
        for (DevBuf& d : h->owner)
            if (d.p == h->d_xh || d.p == h->d_yh)
                cudaFree(d.p);
            else
                keep.push_back(d);
        h->owner.swap(keep);
        h->d_xh = (double2*)hm_dmalloc(h->owner, (size_t)n * nrhs * 16, st, false);
        h->d_yh = (double2*)hm_dmalloc(h->owner, (size_t)n * nrhs * 16, st, false);
        h->staging_cols = nrhs;
    }
    PinnedInt flag;  // the product's error code, read back with y (one synchronisation)
    const char* xb = (const char*)x;
    const char* yb = (const char*)y;
    if (xb < yb + n * nrhs * 16 && yb < xb + n * nrhs * 16) hm_throw(HM_ERR_ARG, "x and y overlap");
    HM_CUDA(cudaMemcpyAsync(h->d_xh, x, (size_t)n * nrhs * 16, cudaMemcpyHostToDevice, st));
    const hm_status s = hm_matvec(h, nrhs, h->d_xh, h->d_yh, stream);
    if (s != HM_OK) return s;
    HM_CUDA(cudaMemcpyAsync(y, h->d_yh, (size_t)n * nrhs * 16, cudaMemcpyDeviceToHost, st));
    matvec_queue_error(h->mv, flag.p, st);
    HM_CUDA(cudaStreamSynchronize(st));
    if (matvec_read_error(h->mv, flag.p, st))
        hm_throw(HM_ERR_TIMEOUT, "a product kernel gave up waiting for its copies");
    HM_API_END
}

hm_status hm_gmres(hm_handle h, const void* b, void* x, int32_t restart, double tol,
                   int32_t maxit, int32_t* iters, double* relres, void* stream) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (!b || !x || restart < 1 || restart > 500 || !(tol > 0) || maxit < 1)
        hm_throw(HM_ERR_ARG, "invalid GMRES arguments (restart must be in 1..500)");
    if (h->n_targets) hm_throw(HM_ERR_UNSUPPORTED, "a two-cloud operator is rectangular: no GMRES");
    const GmresResult R = gmres_solve(h, (const double2*)b, (double2*)x, restart, tol, maxit,
                                      (cudaStream_t)stream);
    if (iters) *iters = R.iters;
    if (relres) *relres = R.relres;
    if (matvec_take_error(h->mv, (cudaStream_t)stream))
        hm_throw(HM_ERR_TIMEOUT, "a product kernel gave up waiting for its copies");
    if (!R.converged) {
        hm_set_error("GMRES reached maxit above the tolerance");
        return HM_ERR_NOCONV;
    }
    HM_API_END
}

hm_status hm_gmres_multi(hm_handle h, int32_t nrhs, const void* b, void* x, int32_t restart,
                         double tol, int32_t maxit, int32_t* iters, double* relres, void* stream) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (!b || !x || nrhs < 1 || restart < 1 || restart > 500 || !(tol > 0) || maxit < 1)
        hm_throw(HM_ERR_ARG, "invalid GMRES arguments (restart must be in 1..500)");
    if (h->n_targets) hm_throw(HM_ERR_UNSUPPORTED, "a two-cloud operator is rectangular: no GMRES");
    const int64_t bytes = 3 * h->nc * (int64_t)nrhs * 16;
    const char* bb = (const char*)b;
    const char* xb = (const char*)x;
    if (bb < xb + bytes && xb < bb + bytes) hm_throw(HM_ERR_ARG, "b and x overlap");
    std::vector<GmresResult> R;
    gmres_solve_multi(h, nrhs, (const double2*)b, (double2*)x, restart, tol, maxit, R,
                      (cudaStream_t)stream);
    bool all = true;
    for (int32_t s = 0; s < nrhs; ++s) {
        if (iters) iters[s] = R[s].iters;
        if (relres) relres[s] = R[s].relres;
        all = all && R[s].converged;
    }
    if (matvec_take_error(h->mv, (cudaStream_t)stream))
        hm_throw(HM_ERR_TIMEOUT, "a product kernel gave up waiting for its copies");
    if (!all) {
        hm_set_error("GMRES reached maxit above the tolerance for some right-hand side");
        return HM_ERR_NOCONV;
    }
    HM_API_END
}

hm_status hm_estimate_error(hm_handle h, int64_t nsample, uint64_t seed, double* delta_f,
                            double* norm_f, void* stream) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (!delta_f || !norm_f) hm_throw(HM_ERR_ARG, "null output");
    if (!h->segments.empty() || h->n_targets)
        hm_throw(HM_ERR_UNSUPPORTED, "not available on a joined batch or two-cloud handle");
    estimate_error(h, nsample, seed, delta_f, norm_f, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_lu_factor(hm_handle h, double eps_lu, void* stream) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (!(eps_lu > 0) || !(eps_lu < 1)) hm_throw(HM_ERR_ARG, "eps_lu must lie in (0, 1)");
    if (!h->segments.empty() || h->n_targets)
        hm_throw(HM_ERR_UNSUPPORTED, "not available on a joined batch or two-cloud handle");
    hlu_factor(h, eps_lu, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_lu_solve(hm_handle h, int32_t nrhs, const void* b, void* x, void* stream) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (nrhs < 1 || !b || !x) hm_throw(HM_ERR_ARG, "null pointer or nrhs < 1");
    const size_t bytes = (size_t)3 * h->nc * nrhs * 16;
    const char *bb = (const char*)b, *xx = (const char*)x;
    if (bb < xx + bytes && xx < bb + bytes) hm_throw(HM_ERR_ARG, "b and x overlap");
    hlu_solve(h, nrhs, (const double2*)b, (double2*)x, (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_lu_info(hm_handle h, double* seconds, int64_t* entries, int64_t* launches) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    hlu_info(h, seconds, entries, launches);
    HM_API_END
}

hm_status hm_stats(hm_handle h, char* json, size_t cap, size_t* needed) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    int64_t nd = 0, nl = 0, rmax = 0, kmax = 0, rsum = 0, ksum = 0;
    std::vector<int64_t> rows_of(h->clusters.size(), 0), cols_of(h->clusters.size(), 0);
    double nst = 0.0;  // stored complex entries (N_s)
    for (const hm_block& b : h->blocks) {
        rows_of[b.tau]++;
        cols_of[b.sigma]++;
        const double m = 3.0 * (h->clusters[b.tau].end - h->clusters[b.tau].begin);
        const double n = 3.0 * (h->clusters[b.sigma].end - h->clusters[b.sigma].begin);
        if (b.admissible) {
            nl++;
            rmax = std::max<int64_t>(rmax, b.rank);
            kmax = std::max<int64_t>(kmax, b.rank_aca);
            rsum += b.rank;
            ksum += b.rank_aca;
            nst += b.rank * (m + n);
        } else {
            nd++;
            nst += m * n;
        }
    }
    int64_t csp = 0;
    for (size_t c = 0; c < rows_of.size(); ++c) csp = std::max({csp, rows_of[c], cols_of[c]});
    const double N = 3.0 * h->nc;
    int64_t alg[3];
    matvec_alg_bytes(h->mv, 3 * h->nc, alg);
    std::ostringstream os;
    os.precision(10);
    os << "{\"n_c\": " << h->nc << ", \"n_targets\": " << h->n_targets
       << ", \"kernel\": \"" << (h->kernel ? "T" : "U") << "\""
       << ", \"depth\": " << h->depth << ", \"clusters\": " << h->clusters.size()
       << ", \"blocks\": " << h->blocks.size() << ", \"dense_blocks\": " << nd
       << ", \"lowrank_blocks\": " << nl << ", \"C_sp\": " << csp
       << ", \"rank_aca_max\": " << kmax << ", \"rank_max\": " << rmax
       << ", \"rank_aca_mean\": " << (nl ? (double)ksum / nl : 0.0)
       << ", \"rank_mean\": " << (nl ? (double)rsum / nl : 0.0) << ", \"N_s\": " << nst
       << ", \"tau_H\": " << nst / (N * N)
       << ", \"stored_bytes\": " << matvec_stored_bytes(h->mv)
       << ", \"matvec_alg_bytes\": " << alg[2] << ", \"phase1_alg_bytes\": " << alg[0]
       << ", \"phase2_alg_bytes\": " << alg[1]
       << ", \"dense_bytes\": " << matvec_dense_bytes(h->mv)
       << ", \"aca_batches\": " << h->aca_batches
       << ", \"aca_overflow_reruns\": " << h->aca_overflow_reruns
       << ", \"aca_workspace_peak_bytes\": " << h->aca_workspace_peak
       << ", \"aca_workspace_total_bytes\": " << h->aca_workspace_total
       << ", \"rank_model\": " << h->used_rank_model
       << ", \"batch_problems\": " << h->batch_problems
       << ", \"rsvd_blocks\": " << h->rsvd_blocks << ", \"rsvd_uncertified\": " << h->rsvd_uncertified
       << ", \"ms\": {\"tree\": " << h->t_tree_ms << ", \"partition\": " << h->t_part_ms
       << ", \"aca\": " << h->t_aca_ms << ", \"recompress\": " << h->t_recomp_ms
       << ", \"rsvd\": " << h->t_rsvd_ms
       << ", \"near_field\": " << h->t_near_ms << ", \"layout\": " << h->t_copy_ms
       << ", \"layout_plan\": " << h->t_plan_ms << ", \"layout_arena\": " << h->t_arena_ms
       << ", \"layout_stage_copy\": " << h->t_stage_ms << ", \"layout_bf16\": " << h->t_bf16_ms
       << ", \"tune\": " << h->t_tune_ms << ", \"graph\": " << h->t_graph_ms
       << ", \"total\": " << h->t_total_ms << "}"
       << ", \"device_ms\": {\"aca\": " << h->ev_aca_ms << ", \"recompress\": " << h->ev_recomp_ms
       << "}, \"aca_flops\": " << h->aca_flops << ", \"aca_flops_fp64\": " << h->aca_flops_fp64
       << ", \"aca_flops_df\": " << h->aca_flops_df << ", \"aca_green_evals\": " << h->aca_green_evals
       << ", \"apply_flops_df\": " << h->apply_flops_df
       << ", \"tune\": {\"source\": \"" << h->tune_source << "\", \"key\": \"" << h->tune_key
       << "\", \"nstage\": " << h->tune_nstage << ", \"item_bytes\": " << h->tune_item_bytes
       << ", \"ms\": " << h->tune_ms << ", \"trials\": [" << h->tune_trials << "]}"
       << ", \"gmres_last\": {\"fast_products\": " << h->gm_fast
       << ", \"accurate_products\": " << h->gm_accurate << ", \"cycles\": " << h->gm_cycles
       << "}}";
    const std::string s = os.str();
    if (needed) *needed = s.size() + 1;
    if (!json || cap < s.size() + 1) hm_throw(HM_ERR_ARG, "stats buffer too small");
    std::memcpy(json, s.c_str(), s.size() + 1);
    HM_API_END
}

hm_status hm_rank_samples(hm_handle h, float* feats, float* targets, int64_t* n) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (!h->segments.empty()) hm_throw(HM_ERR_UNSUPPORTED, "not available on a joined batch handle");
    int64_t q = 0;
    for (const hm_block& b : h->blocks) {
        if (!b.admissible) continue;
        if (feats) rank_features(h->clusters[b.tau], h->clusters[b.sigma], h->gp.ks, h->gp.kp, h->eps,
                                 feats + 6 * q);
        if (targets) targets[q] = (float)std::log1p(b.rank_aca / 3.0);
        ++q;
    }
    if (n) *n = q;
    HM_API_END
}

hm_status hm_sizes(hm_handle h, int64_t* n_c, int64_t* n_clusters, int64_t* n_blocks) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (n_c) *n_c = h->nc;
    if (n_clusters) *n_clusters = (int64_t)h->clusters.size();
    if (n_blocks) *n_blocks = (int64_t)h->blocks.size();
    HM_API_END
}

hm_status hm_get_tree(hm_handle h, int64_t* perm, hm_cluster* clusters) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (perm) std::memcpy(perm, h->perm.data(), 8 * h->perm.size());
    if (clusters)
        std::memcpy(clusters, h->clusters.data(), sizeof(hm_cluster) * h->clusters.size());
    HM_API_END
}

hm_status hm_get_blocks(hm_handle h, hm_block* blocks) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (!blocks) hm_throw(HM_ERR_ARG, "null output");
    std::memcpy(blocks, h->blocks.data(), sizeof(hm_block) * h->blocks.size());
    HM_API_END
}

hm_status hm_get_block_data(hm_handle h, int64_t b, void* a, void* v) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (b < 0 || b >= (int64_t)h->blocks.size() || !a) hm_throw(HM_ERR_ARG, "bad block index");
    const hm_block& B = h->blocks[b];
    const hm_cluster& t = h->clusters[B.tau];
    const hm_cluster& s = h->clusters[B.sigma];
    const int64_t m3 = 3 * (t.end - t.begin), n3 = 3 * (s.end - s.begin);
    if (B.admissible && B.rank > 0 && !v) hm_throw(HM_ERR_ARG, "null V output");
    const float2* arena = (const float2*)matvec_arena(h->mv);
    for (const Chunk& c : h->plan.chunks) {
        if (c.block != b || c.ncols == 0) continue;
        std::vector<float2> tmp((size_t)c.ld * c.ncols);
        HM_CUDA(cudaMemcpy(tmp.data(), arena + c.data, tmp.size() * 8, cudaMemcpyDeviceToHost));
        double* dst = (double*)(c.kind == 2 ? v : a);
        const int64_t owner_begin = 3 * (c.kind == 2 ? s.begin : t.begin);
        const int64_t ld = c.kind == 2 ? n3 : m3;
        const int64_t r0 = c.leaf_dof - owner_begin;
        const int64_t col0 = c.kind == 0 ? c.vec - 3 * s.begin : 0;  // dense: column leaf offset
        for (int col = 0; col < c.ncols; ++col)
            for (int r = 0; r < c.rows; ++r) {
                const float2 z = tmp[(size_t)col * c.ld + r];
                dst[2 * ((r0 + r) + (col0 + col) * ld)] = z.x;
                dst[2 * ((r0 + r) + (col0 + col) * ld) + 1] = z.y;
            }
    }
    HM_API_END
}

hm_status hm_green_eval(int32_t kernel, double rho, double lambda, double mu, double omega,
                        double diag_value, const double* x, const double* y, const double* ny,
                        int64_t npairs, void* out, void* stream) {
    HM_API_BEGIN
    if (npairs < 0 || (npairs > 0 && (!x || !y || !out))) hm_throw(HM_ERR_ARG, "null pointer");
    if (kernel != HM_KERNEL_U && kernel != HM_KERNEL_T) hm_throw(HM_ERR_ARG, "unknown kernel");
    if (kernel == HM_KERNEL_T && !ny && npairs > 0) hm_throw(HM_ERR_ARG, "T needs normals");
    if (!(rho > 0) || !(mu > 0) || !(omega > 0)) hm_throw(HM_ERR_ARG, "bad material");
    const GreenParams gp = make_green_params(kernel, rho, lambda, mu, omega, diag_value);
    launch_green_eval(gp, x, y, kernel == HM_KERNEL_T ? ny : nullptr, npairs, (double2*)out,
                      (cudaStream_t)stream);
    HM_API_END
}

hm_status hm_import(int64_t n_c, const int64_t* perm, int64_t n_clusters,
                    const hm_cluster* clusters, int64_t n_blocks, const hm_block* blocks,
                    const void* data, const hm_opts* opts, void* stream, hm_handle* out) {
    if (out) *out = nullptr;
    hm_matrix* h = nullptr;
    HM_API_BEGIN
    if (!out || !perm || !clusters || !blocks || !data || n_c < 1 || n_clusters < 1 || n_blocks < 1)
        hm_throw(HM_ERR_ARG, "null pointer or empty input");
    hm_opts o;
    hm_opts_default(&o);
    if (opts) o = *opts;
    cudaStream_t st = (cudaStream_t)stream;
    h = new hm_matrix();
    h->nc = n_c;
    h->opts = o;
    h->opts.tune_cache = nullptr;  // imported handles keep the default launch parameters
    HM_CUDA(cudaGetDevice(&h->device));
    h->perm.assign(perm, perm + n_c);
    h->clusters.assign(clusters, clusters + n_clusters);
    h->blocks.assign(blocks, blocks + n_blocks);
    {
        std::vector<char> seen(n_c, 0);
        for (int64_t p = 0; p < n_c; ++p) {
            if (perm[p] < 0 || perm[p] >= n_c || seen[perm[p]]) hm_throw(HM_ERR_ARG, "perm is not a permutation");
            seen[perm[p]] = 1;
        }
        for (const hm_block& b : h->blocks)
            if (b.tau < 0 || b.tau >= n_clusters || b.sigma < 0 || b.sigma >= n_clusters ||
                (b.admissible && b.rank < 0))
                hm_throw(HM_ERR_ARG, "bad block");
        for (const hm_cluster& c : h->clusters) {
            if (c.begin < 0 || c.end > n_c || c.begin >= c.end) hm_throw(HM_ERR_ARG, "bad cluster");
            if (c.is_leaf && c.end - c.begin > 1024) hm_throw(HM_ERR_UNSUPPORTED, "leaf above 1024 points");
        }
    }
    h->d_perm = (int64_t*)hm_dmalloc(h->owner, 8 * n_c, st, false);
    HM_CUDA(cudaMemcpyAsync(h->d_perm, perm, 8 * n_c, cudaMemcpyHostToDevice, st));
    // stage every block in FP32 (column-major as given), then lay out the chunks
    std::vector<DevBuf> staging;
    std::vector<const float2*> su(n_blocks, nullptr), sv(n_blocks, nullptr);
    try {
        int64_t tot = 0;
        std::vector<int64_t> off(n_blocks);
        for (int64_t b = 0; b < n_blocks; ++b) {
            const hm_block& B = h->blocks[b];
            const int64_t m3 = 3 * (h->clusters[B.tau].end - h->clusters[B.tau].begin);
            const int64_t n3 = 3 * (h->clusters[B.sigma].end - h->clusters[B.sigma].begin);
            off[b] = tot;
            tot += B.admissible ? (m3 + n3) * B.rank : m3 * n3;
        }
        std::vector<float2> hf(std::max<int64_t>(tot, 1));
        const double* src = (const double*)data;
        for (int64_t i = 0; i < tot; ++i) hf[i] = make_float2((float)src[2 * i], (float)src[2 * i + 1]);
        float2* d = (float2*)hm_dmalloc(staging, std::max<int64_t>(tot, 1) * 8, st, false);
        HM_CUDA(cudaMemcpyAsync(d, hf.data(), tot * 8, cudaMemcpyHostToDevice, st));
        for (int64_t b = 0; b < n_blocks; ++b) {
            const hm_block& B = h->blocks[b];
            const int64_t m3 = 3 * (h->clusters[B.tau].end - h->clusters[B.tau].begin);
            su[b] = d + off[b];
            if (B.admissible) sv[b] = d + off[b] + m3 * B.rank;
        }
        std::vector<int64_t> t_off;
        h->plan = build_matvec_plan(h->clusters, h->blocks, t_off);
        h->mv = matvec_dev_create(h->plan, o.storage, h->owner, st);
        copy_staged_chunks(h->mv, h->plan, h->blocks, h->clusters, su, sv, st);
        HM_CUDA(cudaStreamSynchronize(st));
        if (o.storage == HM_STORE_BF16) matvec_make_bf16(h->mv, h->plan, h->owner, st);
    } catch (...) {
        cudaStreamSynchronize(st);
        free_all(staging);
        throw;
    }
    free_all(staging);
    h->d_xp = (float2*)hm_dmalloc(h->owner, 8 * 3 * n_c, st, true);
    h->d_yp = (float2*)hm_dmalloc(h->owner, 8 * 3 * n_c, st, true);
    HM_CUDA(cudaStreamSynchronize(st));
    *out = h;
    h = nullptr;
    }
    catch (const hm_error& e) {
        hm_set_error(e.msg);
        if (h) hm_free(h);
        return e.st;
    }
    catch (...) {
        hm_set_error("unexpected internal error");
        if (h) hm_free(h);
        return HM_ERR_CUDA;
    }
    return HM_OK;
}

hm_status hm_profile_matvec(hm_handle h, int32_t reps, double* ms, int64_t* bytes, void* stream) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (reps < 1 || !ms || !bytes) hm_throw(HM_ERR_ARG, "reps < 1 or null output");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = 3 * h->nc;
    std::vector<DevBuf> tmp;
    double2* x = (double2*)hm_dmalloc(tmp, n * 16, st, false);
    double2* y = (double2*)hm_dmalloc(tmp, n * 16, st, false);
    {
        std::vector<double2> ones(n, make_double2(1.0, 0.0));
        HM_CUDA(cudaMemcpyAsync(x, ones.data(), n * 16, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaStreamSynchronize(st));
    }
    cudaEvent_t ev[5];
    for (auto& e : ev) HM_CUDA(cudaEventCreate(&e));
    double acc[4] = {0, 0, 0, 0};
    try {
        for (int r = 0; r < reps; ++r) {
            HM_CUDA(cudaEventRecord(ev[0], st));
            launch_gather_x(h->d_perm, x, h->d_xp, h->nc, st);
            HM_CUDA(cudaEventRecord(ev[1], st));
            matvec_phase1(h->mv, h->d_xp, st);
            HM_CUDA(cudaEventRecord(ev[2], st));
            matvec_phase2(h->mv, h->d_xp, h->d_yp, n, st);
            HM_CUDA(cudaEventRecord(ev[3], st));
            launch_scatter_y(h->d_perm, h->d_yp, y, h->nc, st);
            HM_CUDA(cudaEventRecord(ev[4], st));
            HM_CUDA(cudaEventSynchronize(ev[4]));
            for (int q = 0; q < 4; ++q) {
                float t = 0.f;
                HM_CUDA(cudaEventElapsedTime(&t, ev[q], ev[q + 1]));
                acc[q] += t;
            }
        }
    } catch (...) {
        for (auto& e : ev) cudaEventDestroy(e);
        free_all(tmp);
        throw;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    free_all(tmp);
    for (int q = 0; q < 4; ++q) ms[q] = acc[q] / reps;
    int64_t b3[3];
    matvec_alg_bytes(h->mv, n, b3);
    bytes[0] = b3[0];
    bytes[1] = b3[1];
    bytes[2] = b3[2];
    HM_API_END
}

hm_status hm_profile_matvec_multi(hm_handle h, int32_t reps, double* ms, int64_t* bytes,
                                  void* stream) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (reps < 1 || !ms || !bytes) hm_throw(HM_ERR_ARG, "reps < 1 or null output");
    if (h->opts.storage != HM_STORE_BF16) hm_throw(HM_ERR_UNSUPPORTED, "block product needs BF16 storage");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = 3 * h->nc;
    std::vector<DevBuf> tmp;
    double2* x = (double2*)hm_dmalloc(tmp, (size_t)n * HM_NRHS_BLOCK * 16, st, false);
    double2* y = (double2*)hm_dmalloc(tmp, (size_t)n * HM_NRHS_BLOCK * 16, st, false);
    try {
        std::vector<double2> ones((size_t)n * HM_NRHS_BLOCK);
        for (size_t q = 0; q < ones.size(); ++q) ones[q] = make_double2(1.0 + (q / n) * 1e-3, 0.5);
        HM_CUDA(cudaMemcpyAsync(x, ones.data(), ones.size() * 16, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaStreamSynchronize(st));
        matvec_multi_profile(h->mv, h->d_perm, x, y, h->nc, reps, ms, st);
    } catch (...) {
        free_all(tmp);
        throw;
    }
    free_all(tmp);
    bytes[0] = matvec_multi_alg_bytes(h->mv, n);
    if (matvec_take_error(h->mv, st))
        hm_throw(HM_ERR_TIMEOUT, "a product kernel gave up waiting for its copies");
    HM_API_END
}

int64_t hm_kernel_launches(void) { return (int64_t)g_hm_launches.load(); }

hm_status hm_release_cached_memory(void) {
    HM_API_BEGIN
    hm_scratch_trim();
    HM_API_END
}

void hm_free(hm_handle h) {
    if (!h) return;
    cudaDeviceSynchronize();
    try {
        hlu_release(h, 0);
    } catch (...) {
    }
    free_all(h->owner);
    matvec_dev_destroy(h->mv);
    delete h;
}

}  // extern "C"
