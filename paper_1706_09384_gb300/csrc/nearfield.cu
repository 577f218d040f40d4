// nearfield.cu — dense near-field blocks A_{tau x sigma} of P^non-ad
// (Sec. 2.1, Sec. 5.1: N_st = |tau||sigma| entries per block) evaluated from
// the Green's tensors (green.cuh) in FP64 and stored as complex64 in the
// matvec's chunk layout, and the direct pairwise evaluation entry point.
#include <algorithm>

#include "hm_internal.h"

namespace {

struct DenseJob {
    int64_t data;       // arena offset of the chunk
    int64_t row_begin;  // tree-order point range of the leaf (rows)
    int64_t col_begin;  // tree-order point range of the column leaf
    int32_t m, n;       // points
    int32_t ld;
    int32_t pad_;
};

__global__ void __launch_bounds__(256) dense_assemble_kernel(GreenParams gp, const double* pts,
                                                             const double* nrm,
                                                             const DenseJob* jobs,
                                                             float2* arena) {
    const DenseJob J = jobs[blockIdx.x];
    const int64_t npair = (int64_t)J.m * J.n;
    for (int64_t q = threadIdx.x; q < npair; q += blockDim.x) {
        const int64_t i = q % J.m, j = q / J.m;
        double2 G[9];
        entry_block(gp, pts, nrm, J.row_begin + i, J.col_begin + j, G);
        float2* dst = arena + J.data;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int a = 0; a < 3; ++a)
                dst[(3 * j + c) * J.ld + 3 * i + a] =
                    make_float2((float)G[3 * a + c].x, (float)G[3 * a + c].y);
    }
}

__global__ void green_eval_kernel(GreenParams gp, const double* x, const double* y,
                                  const double* ny, int64_t n, double2* out) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n) return;
    double2 G[9];
    const double* xq = x + 3 * q;
    const double* yq = y + 3 * q;
    if (xq[0] == yq[0] && xq[1] == yq[1] && xq[2] == yq[2]) {
        for (int k = 0; k < 9; ++k) G[k] = make_double2((k % 4 == 0) ? gp.diag : 0.0, 0.0);
    } else {
        green_tensor(gp, xq, yq, ny ? ny + 3 * q : nullptr, G);
    }
    for (int k = 0; k < 9; ++k) out[9 * q + k] = G[k];
}

}  // namespace

void assemble_dense(const GreenParams& gp, const double* d_pts_p, const double* d_nrm_p,
                    const MatvecPlan& plan, const std::vector<hm_block>& blocks,
                    const std::vector<hm_cluster>& cl, MatvecDev* mv, std::vector<DevBuf>& owner,
                    cudaStream_t st) {
    std::vector<DenseJob> jobs;
    for (const Chunk& c : plan.chunks) {
        if (c.kind != 0) continue;
        DenseJob J;  // one (row leaf, column leaf) piece of a dense block
        J.data = c.data;
        J.row_begin = c.leaf_dof / 3;
        J.col_begin = c.vec / 3;
        J.m = c.rows / 3;
        J.n = c.ncols / 3;
        J.ld = c.ld;
        J.pad_ = 0;
        jobs.push_back(J);
    }
    if (jobs.empty()) return;
    DenseJob* d_jobs = nullptr;
    HM_CUDA(cudaMallocAsync((void**)&d_jobs, jobs.size() * sizeof(DenseJob), st));
    HM_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(DenseJob),
                            cudaMemcpyHostToDevice, st));
    dense_assemble_kernel<<<(unsigned)jobs.size(), 256, 0, st>>>(gp, d_pts_p, d_nrm_p, d_jobs,
                                                                 (float2*)matvec_arena(mv));
                                                                 HM_LAUNCHED();
    HM_CUDA(cudaGetLastError());
    HM_CUDA(cudaFreeAsync(d_jobs, st));
    (void)owner;
}

void launch_green_eval(const GreenParams& gp, const double* x, const double* y,
                       const double* ny, int64_t npairs, double2* out, cudaStream_t st) {
    if (npairs <= 0) return;
    green_eval_kernel<<<(unsigned)hm_cdiv(npairs, 128), 128, 0, st>>>(gp, x, y, ny, npairs, out);
    HM_LAUNCHED();
    HM_CUDA(cudaGetLastError());
}
