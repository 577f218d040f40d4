// batch.cu — independent problems as one block-diagonal operator (no paper
// counterpart: batching of independent problems).
//
// hm_batch_join concatenates the H-matrices of several built handles into one
// handle whose operator is diag(A_1, ..., A_n): the point sets, trees and
// block partitions are concatenated (cluster and point indices shifted), the
// storage plan is laid out for the joined partition, and every problem's
// stored chunks are copied into the joined arena (runs of consecutive chunks
// become one device copy).  One H-matvec of the joined handle then applies
// every problem's operator in the same launches, and hm_gmres_batch runs one
// restarted GMRES per problem in lockstep with one such product per Arnoldi
// step (gmres.cu, segments).
#include <algorithm>
#include <chrono>

#include "hm_internal.h"
#include "matvec_dev.cuh"


extern "C" {

hm_status hm_batch_join(int32_t nprob, const hm_handle* hs, void* stream, hm_handle* out) {
    if (out) *out = nullptr;
    hm_matrix* J = nullptr;
    try {
        if (!out || !hs || nprob < 1) hm_throw(HM_ERR_ARG, "null pointer or nprob < 1");
        cudaStream_t st = (cudaStream_t)stream;
        const auto t0 = std::chrono::steady_clock::now();
        int dev = 0;
        HM_CUDA(cudaGetDevice(&dev));
        for (int32_t q = 0; q < nprob; ++q) {
            if (!hs[q] || !hs[q]->mv) hm_throw(HM_ERR_ARG, "null or empty handle");
            if (hs[q]->device != dev) hm_throw(HM_ERR_ARG, "handles on another device");
            if (hs[q]->opts.storage != hs[0]->opts.storage)
                hm_throw(HM_ERR_ARG, "handles with different storage");
            if (!hs[q]->segments.empty()) hm_throw(HM_ERR_ARG, "a joined handle cannot be joined again");
            if (hs[q]->n_targets) hm_throw(HM_ERR_ARG, "two-cloud handles cannot be joined");
        }
        J = new hm_matrix();
        J->device = dev;
        J->kernel = hs[0]->kernel;
        J->opts = hs[0]->opts;
        J->opts.weights = nullptr;
        J->opts.rank_model = nullptr;
        J->opts.tune_cache = nullptr;
        J->eps = hs[0]->eps;
        J->eta = hs[0]->eta;
        J->leaf = hs[0]->leaf;
        J->batch_problems = nprob;
        std::vector<int64_t> pofs(nprob + 1, 0), cofs(nprob + 1, 0), bofs(nprob + 1, 0);
        for (int32_t q = 0; q < nprob; ++q) {
            pofs[q + 1] = pofs[q] + hs[q]->nc;
            cofs[q + 1] = cofs[q] + (int64_t)hs[q]->clusters.size();
            bofs[q + 1] = bofs[q] + (int64_t)hs[q]->blocks.size();
            J->segments.push_back(hs[q]->nc);
            J->depth = std::max(J->depth, hs[q]->depth);
        }
        J->nc = pofs[nprob];
        for (int32_t q = 0; q < nprob; ++q) {
            const hm_matrix* h = hs[q];
            for (int64_t p : h->perm) J->perm.push_back(p + pofs[q]);
            for (hm_cluster c : h->clusters) {
                c.begin += pofs[q];
                c.end += pofs[q];
                if (c.child0 >= 0) c.child0 += cofs[q];
                if (c.child1 >= 0) c.child1 += cofs[q];
                J->clusters.push_back(c);
            }
            for (hm_block b : h->blocks) {
                b.tau += cofs[q];
                b.sigma += cofs[q];
                J->blocks.push_back(b);
            }
        }
        J->d_perm = (int64_t*)hm_dmalloc(J->owner, 8 * J->nc, st, false);
        HM_CUDA(cudaMemcpyAsync(J->d_perm, J->perm.data(), 8 * J->nc, cudaMemcpyHostToDevice, st));
        std::vector<int64_t> t_off;
        J->plan = build_matvec_plan(J->clusters, J->blocks, t_off);
        J->mv = matvec_dev_create(J->plan, J->opts.storage, J->owner, st);
        // copy every chunk from its problem's FP32 arena.  The plan creates chunks
        // block by block, so the joined plan's chunks are the problems' chunks in
        // problem order: chunk base[q] + i is chunk i of problem q (checked).
        // Walking the joined arena in order merges contiguous runs into one copy.
        std::vector<int64_t> base(nprob + 1, 0);
        for (int32_t q = 0; q < nprob; ++q) base[q + 1] = base[q] + (int64_t)hs[q]->plan.chunks.size();
        if (base[nprob] != (int64_t)J->plan.chunks.size()) hm_throw(HM_ERR_CUDA, "batch join: chunk count");
        struct Run {
            int32_t q;
            int64_t src, dst, n;
        };
        std::vector<Run> runs;
        auto add = [&](int32_t id) {
            const Chunk& c = J->plan.chunks[id];
            const int32_t q = (int32_t)(std::upper_bound(base.begin(), base.end(), (int64_t)id) - base.begin() - 1);
            const Chunk& o = hs[q]->plan.chunks[id - base[q]];
            if (o.block != c.block - bofs[q] || o.leaf_dof != c.leaf_dof - 3 * pofs[q] || o.kind != c.kind ||
                o.ld != c.ld || o.ncols != c.ncols || (c.kind == 0 && o.vec != c.vec - 3 * pofs[q]))
                hm_throw(HM_ERR_CUDA, "batch join: chunk layout mismatch");
            const int64_t n = (int64_t)c.ld * c.ncols;
            if (n == 0) return;
            if (!runs.empty() && runs.back().q == q && runs.back().src + runs.back().n == o.data &&
                runs.back().dst + runs.back().n == c.data)
                runs.back().n += n;
            else
                runs.push_back({q, o.data, c.data, n});
        };
        for (int32_t id : J->plan.row_items) add(id);
        for (int32_t id : J->plan.col_items) add(id);
        float2* dst = (float2*)matvec_arena(J->mv);
        for (const Run& r : runs)
            HM_CUDA(cudaMemcpyAsync(dst + r.dst, (const float2*)matvec_arena(hs[r.q]->mv) + r.src,
                                    r.n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        HM_CUDA(cudaStreamSynchronize(st));
        if (J->opts.storage == HM_STORE_BF16) matvec_make_bf16(J->mv, J->plan, J->owner, st);
        J->d_xp = (float2*)hm_dmalloc(J->owner, 8 * 3 * J->nc, st, true);
        J->d_yp = (float2*)hm_dmalloc(J->owner, 8 * 3 * J->nc, st, true);
        HM_CUDA(cudaStreamSynchronize(st));
        J->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        J->t_copy_ms = J->t_total_ms;
        *out = J;
    } catch (const hm_error& e) {
        if (J) hm_free(J);
        hm_set_error(e.msg);
        return e.st;
    } catch (const std::bad_alloc&) {
        if (J) hm_free(J);
        hm_set_error("host allocation failed");
        return HM_ERR_OOM;
    } catch (...) {
        if (J) hm_free(J);
        hm_set_error("unexpected internal error");
        return HM_ERR_CUDA;
    }
    return HM_OK;
}

hm_status hm_gmres_batch(hm_handle h, const void* b, void* x, int32_t restart, double tol,
                         int32_t maxit, int32_t* iters, double* relres, void* stream) {
    try {
        if (!h || h->segments.empty()) hm_throw(HM_ERR_ARG, "not a joined batch handle");
        if (!b || !x || restart < 1 || restart > 500 || !(tol > 0) || maxit < 1)
            hm_throw(HM_ERR_ARG, "invalid GMRES arguments (restart must be in 1..500)");
        const int64_t bytes = 3 * h->nc * 16;
        const char* bb = (const char*)b;
        const char* xb = (const char*)x;
        if (bb < xb + bytes && xb < bb + bytes) hm_throw(HM_ERR_ARG, "b and x overlap");
        std::vector<GmresResult> R;
        gmres_solve_segments(h, h->segments, (const double2*)b, (double2*)x, restart, tol, maxit, R,
                             (cudaStream_t)stream);
        bool all = true;
        for (size_t s = 0; s < R.size(); ++s) {
            if (iters) iters[s] = R[s].iters;
            if (relres) relres[s] = R[s].relres;
            all = all && R[s].converged;
        }
        if (matvec_take_error(h->mv, (cudaStream_t)stream))
            hm_throw(HM_ERR_TIMEOUT, "a product kernel gave up waiting for its copies");
        if (!all) {
            hm_set_error("GMRES reached maxit above the tolerance for some problem");
            return HM_ERR_NOCONV;
        }
    } catch (const hm_error& e) {
        hm_set_error(e.msg);
        return e.st;
    } catch (...) {
        hm_set_error("unexpected internal error");
        return HM_ERR_CUDA;
    }
    return HM_OK;
}

}  // extern "C"
