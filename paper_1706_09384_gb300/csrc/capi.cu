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
    HM_CUDA(cudaMalloc(&p, bytes ? bytes : 16));
    owner.push_back({p, bytes});
    if (zero && bytes) HM_CUDA(cudaMemsetAsync(p, 0, bytes, st));
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
        if (d.p) cudaFree(d.p);
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

// ACA + recompression of every admissible block, in batches bounded by the
// workspace budget.  Writes the FP32 factors (U' column-major 3m x r', V'
// 3n x r') into staging buffers owned by `staging` and records per block the
// pointers and ranks.
void build_low_rank(hm_matrix* h, std::vector<DevBuf>& staging, std::vector<const float2*>& su,
                    std::vector<const float2*>& sv, cudaStream_t st) {
    const std::vector<hm_cluster>& cl = h->clusters;
    std::vector<hm_block>& blk = h->blocks;
    std::vector<int64_t> adm;
    for (int64_t b = 0; b < (int64_t)blk.size(); ++b)
        if (blk[b].admissible) adm.push_back(b);
    auto pts_of = [&](int64_t c) { return cl[c].end - cl[c].begin; };
    std::stable_sort(adm.begin(), adm.end(), [&](int64_t a, int64_t b) {
        return pts_of(blk[a].tau) + pts_of(blk[a].sigma) > pts_of(blk[b].tau) + pts_of(blk[b].sigma);
    });
    int cap0 = h->opts.aca_max_rank > 0 ? h->opts.aca_max_rank : 144;
    cap0 = std::max(3, cap0 - cap0 % 3);
    const int64_t budget = h->opts.workspace_bytes > 0 ? h->opts.workspace_bytes : (24ll << 30);
    int nsm = 0;
    HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    std::vector<int> cap(blk.size(), 0);
    for (int64_t b : adm) {
        const int64_t full = 3 * std::min(pts_of(blk[b].tau), pts_of(blk[b].sigma));
        cap[b] = (int)std::min<int64_t>(full, cap0);
    }
    if (h->opts.rank_model && !adm.empty()) {
        // learned capacities: predicted rank-3 steps with a safety margin; the
        // ACA still decides the rank and overflowing blocks are re-run
        const int64_t na = (int64_t)adm.size();
        std::vector<float> feats(6 * na), pred(na);
        for (int64_t q = 0; q < na; ++q)
            rank_features(cl[blk[adm[q]].tau], cl[blk[adm[q]].sigma], h->gp.ks, h->gp.kp, h->eps,
                          &feats[6 * q]);
        std::vector<DevBuf> tmp;
        float* dP = (float*)hm_dmalloc(tmp, HM_RANK_MODEL_PARAMS * 4, st, false);
        float* dF = (float*)hm_dmalloc(tmp, feats.size() * 4, st, false);
        float* dO = (float*)hm_dmalloc(tmp, na * 4, st, false);
        HM_CUDA(cudaMemcpyAsync(dP, h->opts.rank_model, HM_RANK_MODEL_PARAMS * 4, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(dF, feats.data(), feats.size() * 4, cudaMemcpyHostToDevice, st));
        rank_model_predict_dev(dP, dF, na, dO, st);
        HM_CUDA(cudaMemcpyAsync(pred.data(), dO, na * 4, cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        free_all(tmp);
        const float tm = h->opts.rank_model[12], ts = h->opts.rank_model[13];
        for (int64_t q = 0; q < na; ++q) {
            const int64_t b = adm[q];
            const double steps = std::exp((double)pred[q] * ts + tm) - 1.0;
            const int64_t full = 3 * std::min(pts_of(blk[b].tau), pts_of(blk[b].sigma));
            int64_t c = 3 * (int64_t)std::ceil(1.25 * std::max(steps, 0.0) + 2.0);
            if (!std::isfinite(steps)) c = cap0;
            cap[b] = (int)std::max<int64_t>(3, std::min<int64_t>({c, full, 768}));
        }
        // bin blocks of similar predicted rank into the same batches
        std::stable_sort(adm.begin(), adm.end(), [&](int64_t a, int64_t b) {
            if (cap[a] != cap[b]) return cap[a] > cap[b];
            return pts_of(blk[a].tau) + pts_of(blk[a].sigma) > pts_of(blk[b].tau) + pts_of(blk[b].sigma);
        });
        h->used_rank_model = 1;
    }
    int* d_counter = (int*)hm_dmalloc(staging, sizeof(int), st, true);
    std::vector<int64_t> todo = adm;
    while (!todo.empty()) {
        std::vector<int64_t> overflow;
        size_t pos = 0;
        while (pos < todo.size()) {
            // ---- form a batch ----
            std::vector<AcaJob> jobs;
            std::vector<int64_t> ids;
            int64_t woff = 0, goff = 0, maxm = 1, maxn = 1;
            int capmax = 3;
            while (pos < todo.size()) {
                const int64_t b = todo[pos];
                const int64_t m = pts_of(blk[b].tau), n = pts_of(blk[b].sigma);
                const int64_t need = (3 * (m + n) * (int64_t)cap[b] + 2 * (int64_t)cap[b] * cap[b]) * 16;
                if (!jobs.empty() && (woff + goff) * 16 + need > budget) break;
                AcaJob J;
                J.tau_begin = cl[blk[b].tau].begin;
                J.m = m;
                J.sig_begin = cl[blk[b].sigma].begin;
                J.n = n;
                J.u_off = woff;
                J.v_off = woff + 3 * m * cap[b];
                J.g_off = goff;
                J.cap = cap[b];
                J.pad_ = 0;
                woff += 3 * (m + n) * cap[b];
                goff += 2 * (int64_t)cap[b] * cap[b];
                maxm = std::max(maxm, m);
                maxn = std::max(maxn, n);
                capmax = std::max(capmax, cap[b]);
                jobs.push_back(J);
                ids.push_back(b);
                ++pos;
            }
            const int64_t nj = (int64_t)jobs.size();
            h->aca_workspace_peak = std::max<int64_t>(h->aca_workspace_peak, (woff + goff) * 16);
            h->aca_workspace_total += (woff + goff) * 16;
            const int nctas = (int)std::min<int64_t>(nj, (int64_t)nsm * aca_ctas_per_sm(capmax));
            std::vector<DevBuf> tmp;
            auto t0 = clk::now();
            double2* d_work = (double2*)hm_dmalloc(tmp, (size_t)woff * 16, st, false);
            double2* d_gram = (double2*)hm_dmalloc(tmp, (size_t)goff * 16, st, false);
            AcaJob* d_jobs = (AcaJob*)hm_dmalloc(tmp, nj * sizeof(AcaJob), st, false);
            AcaResult* d_res = (AcaResult*)hm_dmalloc(tmp, nj * sizeof(AcaResult), st, false);
            const int64_t fstride = hm_round_up(maxm + maxn, 16);
            unsigned char* d_flags = (unsigned char*)hm_dmalloc(tmp, (size_t)nctas * fstride, st, false);
            const int64_t rbs = 9 * maxn + maxn / 2 + 1, cbs = 9 * maxm + maxm / 2 + 1;
            double2* d_rb = (double2*)hm_dmalloc(tmp, (size_t)nctas * rbs * 16, st, false);
            double2* d_cb = (double2*)hm_dmalloc(tmp, (size_t)nctas * cbs * 16, st, false);
            HM_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), nj * sizeof(AcaJob), cudaMemcpyHostToDevice, st));
            EvPair ea(st);
            launch_aca(h->gp, h->d_pts_p, h->d_nrm_p, d_jobs, nj, d_work, d_gram, d_flags, fstride, d_rb,
                       d_cb, rbs, cbs, h->eps, d_res, nctas, capmax, d_counter, st);
            h->ev_aca_ms += ea.stop(st);
            std::vector<AcaResult> res(nj);
            HM_CUDA(cudaMemcpyAsync(res.data(), d_res, nj * sizeof(AcaResult), cudaMemcpyDeviceToHost, st));
            HM_CUDA(cudaStreamSynchronize(st));
            h->t_aca_ms += ms_since(t0);
            h->aca_batches++;
            // ---- recompression of the converged jobs ----
            t0 = clk::now();
            std::vector<int64_t> uo, vo, m3, n3, keep, go;
            std::vector<int32_t> kk, gl;
            for (int64_t j = 0; j < nj; ++j) {
                if (res[j].status == 2)
                    hm_throw(HM_ERR_NUMERIC, "non-finite value in the ACA of a block");
                if (res[j].status == 1) {
                    const int64_t b = ids[j];
                    const int64_t full = 3 * std::min(jobs[j].m, jobs[j].n);
                    const int nc2 = (int)std::min<int64_t>({full, 2 * (int64_t)cap[b], 768});
                    if (nc2 <= cap[b]) hm_throw(HM_ERR_UNSUPPORTED, "ACA rank above 768 columns");
                    cap[b] = nc2;
                    overflow.push_back(b);
                    continue;
                }
                {
                    const double K = res[j].k / 3, mn = (double)(jobs[j].m + jobs[j].n);
                    h->aca_flops += 8.0 * 18.0 * mn * 3.0 * (K * (K - 1.0) / 2.0);
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
            std::vector<int32_t> ranks;
            std::vector<int64_t> soff;
            EvPair er(st);
            void* rb = recompress_core(uo, vo, m3, n3, kk, go, gl, d_gram, h->opts.recompress,
                                       d_work, h->eps, ranks, soff, st);
            try {
                // staging for this batch: FP32 U' (3m x r'), V' (3n x r')
                int64_t tot = 0;
                std::vector<int64_t> so(keep.size());
                for (size_t q = 0; q < keep.size(); ++q) {
                    so[q] = tot;
                    tot += (m3[q] + n3[q]) * ranks[q];
                }
                float2* d_stage = (float2*)hm_dmalloc(staging, std::max<int64_t>(tot, 1) * 8, st, false);
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
                recompress_apply(rb, job_of, which, row0, rows, dst, ldv, ranks, d_work, d_stage, st);
                h->ev_recomp_ms += er.stop(st);
                for (size_t q = 0; q < keep.size(); ++q) {
                    const int64_t b = ids[keep[q]];
                    blk[b].rank_aca = kk[q];
                    blk[b].rank = ranks[q];
                    su[b] = d_stage + so[q];
                    sv[b] = d_stage + so[q] + m3[q] * ranks[q];
                }
                HM_CUDA(cudaStreamSynchronize(st));
            } catch (...) {
                recompress_release(rb, st);
                throw;
            }
            recompress_release(rb, st);
            HM_CUDA(cudaStreamSynchronize(st));
            free_all(tmp);
            h->t_recomp_ms += ms_since(t0);
        }
        h->aca_overflow_reruns += (int64_t)overflow.size();
        todo.swap(overflow);
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
    hm_matrix* h = nullptr;
    HM_API_BEGIN
    if (!out || !points || n_c < 1) hm_throw(HM_ERR_ARG, "null pointer or n_c < 1");
    if (!(rho > 0) || !(mu > 0) || !(omega > 0) || !std::isfinite(rho) || !std::isfinite(mu) ||
        !std::isfinite(omega) || !std::isfinite(lambda) || !(lambda + 2 * mu > 0))
        hm_throw(HM_ERR_ARG, "material parameters must be finite with rho, mu, omega > 0");
    if (!(eps > 0 && eps < 1)) hm_throw(HM_ERR_ARG, "eps must lie in (0, 1)");
    if (!(eta > 0) || !std::isfinite(eta)) hm_throw(HM_ERR_ARG, "eta must be positive");
    if (kernel != HM_KERNEL_U && kernel != HM_KERNEL_T) hm_throw(HM_ERR_ARG, "unknown kernel");
    if (kernel == HM_KERNEL_T && !normals) hm_throw(HM_ERR_ARG, "the T kernel needs normals");
    if (leaf_size < 1) hm_throw(HM_ERR_ARG, "leaf_size must be >= 1");
    if (leaf_size > 64) hm_throw(HM_ERR_UNSUPPORTED, "leaf_size above 64 points");
    if (!finite_all(points, 3 * n_c)) hm_throw(HM_ERR_ARG, "non-finite point coordinates");
    if (kernel == HM_KERNEL_T && !finite_all(normals, 3 * n_c))
        hm_throw(HM_ERR_ARG, "non-finite normals");
    hm_opts o;
    hm_opts_default(&o);
    if (opts) o = *opts;
    if (o.storage != HM_STORE_FP32 && o.storage != HM_STORE_BF16)
        hm_throw(HM_ERR_ARG, "unknown storage type");
    if (!std::isfinite(o.diag_value)) hm_throw(HM_ERR_ARG, "non-finite diag_value");
    cudaStream_t st = (cudaStream_t)stream;
    const auto t_all = clk::now();
    h = new hm_matrix();
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
    // ---- low-rank blocks ----
    std::vector<DevBuf> staging;
    std::vector<const float2*> su(h->blocks.size(), nullptr), sv(h->blocks.size(), nullptr);
    try {
        build_low_rank(h, staging, su, sv, st);
        // ---- storage plan, arena, near field, factor chunks ----
        t0 = clk::now();
        std::vector<int64_t> t_off;
        h->plan = build_matvec_plan(h->clusters, h->blocks, t_off);
        h->mv = matvec_dev_create(h->plan, o.storage, h->owner, st);
        auto tn = clk::now();
        assemble_dense(h->gp, h->d_pts_p, h->d_nrm_p, h->plan, h->blocks, h->clusters, h->mv,
                       h->owner, st);
        HM_CUDA(cudaStreamSynchronize(st));
        h->t_near_ms = ms_since(tn);
        copy_staged_chunks(h->mv, h->plan, h->blocks, h->clusters, su, sv, st);
        HM_CUDA(cudaStreamSynchronize(st));
        if (o.storage == HM_STORE_BF16) matvec_make_bf16(h->mv, h->plan, h->owner, st);
        h->t_copy_ms = ms_since(t0) - h->t_near_ms;
    } catch (...) {
        cudaStreamSynchronize(st);
        free_all(staging);
        throw;
    }
    free_all(staging);
    h->d_xp = (float2*)hm_dmalloc(h->owner, 8 * 3 * n_c, st, true);
    h->d_yp = (float2*)hm_dmalloc(h->owner, 8 * 3 * n_c, st, true);
    HM_CUDA(cudaStreamSynchronize(st));
    h->t_total_ms = ms_since(t_all);
    if (o.verbose)
        std::fprintf(stderr,
                     "[hm] n_c=%lld blocks=%zu tree=%.1fms part=%.1fms aca=%.1fms recomp=%.1fms "
                     "near=%.1fms copy=%.1fms total=%.1fms\n",
                     (long long)n_c, h->blocks.size(), h->t_tree_ms, h->t_part_ms, h->t_aca_ms,
                     h->t_recomp_ms, h->t_near_ms, h->t_copy_ms, h->t_total_ms);
    *out = h;
    h = nullptr;
    }
    catch (const hm_error& e) {
        hm_set_error(e.msg);
        if (h) hm_free(h);
        return e.st;
    }
    catch (const std::bad_alloc&) {
        hm_set_error("host allocation failed");
        if (h) hm_free(h);
        return HM_ERR_OOM;
    }
    catch (...) {
        hm_set_error("unexpected internal error");
        if (h) hm_free(h);
        return HM_ERR_CUDA;
    }
    return HM_OK;
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
    HM_CUDA(cudaMemcpyAsync(h->d_xh, x, (size_t)n * nrhs * 16, cudaMemcpyHostToDevice, st));
    const hm_status s = hm_matvec(h, nrhs, h->d_xh, h->d_yh, stream);
    if (s != HM_OK) return s;
    HM_CUDA(cudaMemcpyAsync(y, h->d_yh, (size_t)n * nrhs * 16, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (matvec_take_error(h->mv, st))
        hm_throw(HM_ERR_TIMEOUT, "a product kernel gave up waiting for its copies");
    HM_API_END
}

hm_status hm_gmres(hm_handle h, const void* b, void* x, int32_t restart, double tol,
                   int32_t maxit, int32_t* iters, double* relres, void* stream) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
    if (!b || !x || restart < 1 || restart > 500 || !(tol > 0) || maxit < 1)
        hm_throw(HM_ERR_ARG, "invalid GMRES arguments (restart must be in 1..500)");
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
    os << "{\"n_c\": " << h->nc << ", \"kernel\": \"" << (h->kernel ? "T" : "U") << "\""
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
       << ", \"ms\": {\"tree\": " << h->t_tree_ms << ", \"partition\": " << h->t_part_ms
       << ", \"aca\": " << h->t_aca_ms << ", \"recompress\": " << h->t_recomp_ms
       << ", \"near_field\": " << h->t_near_ms << ", \"layout\": " << h->t_copy_ms
       << ", \"total\": " << h->t_total_ms << "}"
       << ", \"device_ms\": {\"aca\": " << h->ev_aca_ms << ", \"recompress\": " << h->ev_recomp_ms
       << "}, \"aca_flops\": " << h->aca_flops << "}";
    const std::string s = os.str();
    if (needed) *needed = s.size() + 1;
    if (!json || cap < s.size() + 1) hm_throw(HM_ERR_ARG, "stats buffer too small");
    std::memcpy(json, s.c_str(), s.size() + 1);
    HM_API_END
}

hm_status hm_rank_samples(hm_handle h, float* feats, float* targets, int64_t* n) {
    HM_API_BEGIN
    if (validate_common(h) != HM_OK) return HM_ERR_ARG;
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
        for (int col = 0; col < c.ncols; ++col)
            for (int r = 0; r < c.rows; ++r) {
                const float2 z = tmp[(size_t)col * c.ld + r];
                dst[2 * ((r0 + r) + col * ld)] = z.x;
                dst[2 * ((r0 + r) + col * ld) + 1] = z.y;
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
            if (c.is_leaf && c.end - c.begin > 64) hm_throw(HM_ERR_UNSUPPORTED, "leaf above 64 points");
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

void hm_free(hm_handle h) {
    if (!h) return;
    cudaDeviceSynchronize();
    free_all(h->owner);
    matvec_dev_destroy(h->mv);
    delete h;
}

}  // extern "C"
