// estimate.cu — the H-matrix approximation error ||A - A_H||_F and ||A||_F
// for the a-posteriori bound of Sec. 3.3 (Eq. est_direct):
//     ||b - A x|| <= ||b - A_H x|| + ||A - A_H||_F ||x||,
// A = the exact collocation matrix (3x3 Green's tensors, weights, diagonal
// blocks), A_H = the stored H-matrix (FP32 arena; U'V'^H on admissible
// blocks, the dense block elsewhere).
//
// Both squared norms are sums over the N_c^2 point pairs (i, j) of the 3x3
// blocks' squared entries.  Every pair is evaluated (exact mode), or S pairs
// drawn uniformly with a counter-based generator estimate the sums without
// bias: (N_c^2 / S) sum_s |.|^2.  The host locates each pair's block, chunks
// and rows in the storage plan; the kernel evaluates the exact tensor in FP64
// and the stored one from the arena.
#include <algorithm>
#include <cmath>
#include <vector>

#include "green.cuh"
#include "hm_internal.h"

namespace {

struct EstSample {
    int64_t i, j;      // tree-order point indices
    int64_t u_off;     // arena offset of row 3 (i - leaf begin) in the dense or U chunk
    int64_t v_off;     // dense: first column 3 (j - sigma begin); low rank: V chunk row offset
    int32_t u_ld, v_ld;
    int32_t rank;      // -1: dense block
    int32_t pad_;
};

__global__ void estimate_kernel(GreenParams gp, const double* __restrict__ pts,
                                const double* __restrict__ nrm, const float2* __restrict__ arena,
                                const EstSample* __restrict__ smp, int64_t ns, double* sums) {
    __shared__ double red[2][8];
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double d2 = 0.0, a2 = 0.0;
    if (q < ns) {
        const EstSample S = smp[q];
        double2 G[9];
        entry_block(gp, pts, nrm, S.i, S.j, G);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double2 h = make_double2(0.0, 0.0);
                if (S.rank < 0) {
                    const float2 v = arena[S.u_off + a + (S.v_off + c) * (int64_t)S.u_ld];
                    h = make_double2(v.x, v.y);
                } else {
                    for (int p = 0; p < S.rank; ++p) {  // U'(row, p) conj(V'(col, p))
                        const float2 u = arena[S.u_off + a + (int64_t)p * S.u_ld];
                        const float2 v = arena[S.v_off + c + (int64_t)p * S.v_ld];
                        h.x += (double)u.x * v.x + (double)u.y * v.y;
                        h.y += (double)u.y * v.x - (double)u.x * v.y;
                    }
                }
                const double2 g = G[3 * a + c];
                d2 += (g.x - h.x) * (g.x - h.x) + (g.y - h.y) * (g.y - h.y);
                a2 += g.x * g.x + g.y * g.y;
            }
    }
    d2 = warp_sum(d2);
    a2 = warp_sum(a2);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][w] = d2;
        red[1][w] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            s0 += red[0][k];
            s1 += red[1][k];
        }
        atomicAdd(sums, s0);
        atomicAdd(sums + 1, s1);
    }
}

uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

void estimate_error(hm_matrix* h, int64_t nsample, uint64_t seed, double* delta_f, double* norm_f,
                    cudaStream_t st) {
    const MatvecPlan& P = h->plan;
    const std::vector<hm_cluster>& cl = h->clusters;
    const std::vector<hm_block>& blk = h->blocks;
    const int64_t nc = h->nc;
    const int64_t nleaf = (int64_t)P.leaf_dof_begin.size();
    // leaf of each point, and the V chunk of (block, column leaf)
    std::vector<int32_t> leaf_of(nc);
    for (int64_t l = 0; l < nleaf; ++l)
        for (int64_t p = P.leaf_dof_begin[l] / 3; p < P.leaf_dof_begin[l] / 3 + P.leaf_rows[l] / 3; ++p)
            leaf_of[p] = (int32_t)l;
    auto locate = [&](int64_t i, int64_t j, EstSample& S) {
        S.i = i;
        S.j = j;
        S.pad_ = 0;
        const int64_t li = leaf_of[i], lj = leaf_of[j];
        for (int64_t q = P.row_leaf_begin[li]; q < P.row_leaf_begin[li + 1]; ++q) {
            const Chunk& c = P.chunks[P.row_items[q]];
            const hm_block& b = blk[c.block];
            const hm_cluster& s = cl[b.sigma];
            if (j < s.begin || j >= s.end) continue;
            // a dense block is stored as one chunk per column leaf
            if (c.kind == 0 && (3 * j < c.vec || 3 * j >= c.vec + c.ncols)) continue;
            S.u_off = c.data + 3 * i - c.leaf_dof;
            S.u_ld = c.ld;
            if (c.kind == 0) {
                S.rank = -1;
                S.v_off = 3 * j - c.vec;
                S.v_ld = 0;
                return;
            }
            S.rank = c.ncols;
            S.v_off = -1;
            for (int64_t r = P.col_leaf_begin[lj]; r < P.col_leaf_begin[lj + 1]; ++r) {
                const Chunk& v = P.chunks[P.col_items[r]];
                if (v.block == c.block) {
                    S.v_off = v.data + 3 * j - v.leaf_dof;
                    S.v_ld = v.ld;
                    break;
                }
            }
            if (S.v_off < 0) hm_throw(HM_ERR_CUDA, "estimate: V chunk not found");
            return;
        }
        hm_throw(HM_ERR_CUDA, "estimate: block of a point pair not found");
    };
    std::vector<EstSample> smp;
    double scale = 1.0;
    if (nsample <= 0) {  // every pair
        if (nc > 2048) hm_throw(HM_ERR_ARG, "every-pair evaluation is limited to n_c <= 2048");
        smp.resize((size_t)nc * nc);
        for (int64_t i = 0; i < nc; ++i)
            for (int64_t j = 0; j < nc; ++j) locate(i, j, smp[(size_t)i * nc + j]);
    } else {
        smp.resize(nsample);
        for (int64_t q = 0; q < nsample; ++q) {
            const uint64_t r = splitmix64(seed ^ splitmix64((uint64_t)q));
            const int64_t i = (int64_t)((r >> 32) % (uint64_t)nc);
            const int64_t j = (int64_t)((r & 0xffffffffull) % (uint64_t)nc);
            locate(i, j, smp[q]);
        }
        scale = (double)nc * (double)nc / (double)nsample;
    }
    std::vector<DevBuf> tmp;
    try {
        EstSample* d_s = (EstSample*)hm_dmalloc(tmp, smp.size() * sizeof(EstSample), st, false);
        double* d_sum = (double*)hm_dmalloc(tmp, 2 * sizeof(double), st, true);
        HM_CUDA(cudaMemcpyAsync(d_s, smp.data(), smp.size() * sizeof(EstSample), cudaMemcpyHostToDevice, st));
        const int64_t ns = (int64_t)smp.size();
        GreenParams exact = h->gp;  // the exact matrix: FP64 tensors at every distance
        exact.ksr_switch = INFINITY;
        estimate_kernel<<<(unsigned)hm_cdiv(ns, 256), 256, 0, st>>>(
            exact, h->d_pts_p, h->d_nrm_p, (const float2*)matvec_arena(h->mv), d_s, ns, d_sum);
        HM_LAUNCHED();
        HM_CUDA(cudaGetLastError());
        double sums[2] = {0.0, 0.0};
        HM_CUDA(cudaMemcpyAsync(sums, d_sum, sizeof(sums), cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        *delta_f = std::sqrt(sums[0] * scale);
        *norm_f = std::sqrt(sums[1] * scale);
    } catch (...) {
        cudaStreamSynchronize(st);
        for (DevBuf& d : tmp) cudaFree(d.p);
        throw;
    }
    for (DevBuf& d : tmp) cudaFree(d.p);
}
