// tree.cu — cluster tree T_I (Sec. 2.1, "Clustering of the unknowns") and
// block partition P (Sec. 2.1, "Subdivision of the matrix") on the GPU.
//
// Tree: level by level, one CTA per cluster of the level computes the tight
// bounding box, splits it at the midpoint of its largest extent (ties ->
// lowest axis) and stably partitions its points (coordinate < midpoint goes
// left).  A cluster with <= N_leaf points, a zero-extent box, or a split that
// leaves one side empty is a leaf.  Every comparison is exact, so the tree
// is the same as any exact restatement of the rule.
//
// Partition: level-synchronous traversal of T_I x T_I from (root, root); a
// pair is low rank if min(diam_box) < eta dist_box (Eq. admissibility_cond_bis,
// Sec. 6.1, with the per-axis positive part in dist_box), dense if not and one
// side is a leaf, otherwise it is replaced by its 4 child pairs.  The
// admissibility arithmetic uses explicitly rounded operations (no fused
// multiply-add) so its decision is reproducible across compilers.
#include <algorithm>
#include <cfloat>

#include "hm_internal.h"

namespace {

constexpr int TB = 512;

__device__ int block_exscan(int v, int& total) {
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    const int pre = (wid > 0 ? ws[wid - 1] : 0) + x - v;
    total = ws[nw - 1];
    __syncthreads();
    return pre;
}

struct DevTree {
    int64_t* begin;
    int64_t* end;
    double* lo;      // 3 per cluster
    double* hi;
    int32_t* level;
    int32_t* is_leaf;
    int64_t* child0;
    int64_t* child1;
    int64_t* nleft;  // size of the left child when split
};

__global__ void __launch_bounds__(TB) tree_level_kernel(const int64_t* ids, DevTree T,
                                                        double* pts, int64_t* perm,
                                                        double* tmp_pts, int64_t* tmp_perm,
                                                        int64_t leaf, int32_t* split) {
    __shared__ double red[6][TB / 32];
    __shared__ double box[6];
    __shared__ int64_t cnt_w[TB / 32];
    const int64_t c = ids[blockIdx.x];
    const int64_t b = T.begin[c], e = T.end[c];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int64_t p = b + tid; p < e; p += TB)
        for (int a = 0; a < 3; ++a) {
            const double v = pts[3 * p + a];
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            red[a][wid] = lo[a];
            red[3 + a][wid] = hi[a];
        }
    __syncthreads();
    if (tid < 6) {
        double v = red[tid][0];
        for (int w = 1; w < TB / 32; ++w) v = tid < 3 ? fmin(v, red[tid][w]) : fmax(v, red[tid][w]);
        box[tid] = v;
    }
    __syncthreads();
    if (tid < 3) {
        T.lo[3 * c + tid] = box[tid];
        T.hi[3 * c + tid] = box[3 + tid];
    }
    split[blockIdx.x] = 0;
    if (e - b <= leaf) return;
    int axis = 0;
    double ext = box[3] - box[0];
    for (int a = 1; a < 3; ++a)
        if (box[3 + a] - box[a] > ext) {
            ext = box[3 + a] - box[a];
            axis = a;
        }
    if (!(ext > 0.0)) return;
    const double mid = __dmul_rn(__dadd_rn(box[axis], box[3 + axis]), 0.5);
    int64_t nl = 0;
    for (int64_t p = b + tid; p < e; p += TB) nl += (pts[3 * p + axis] < mid) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) nl += __shfl_xor_sync(0xffffffffu, nl, o);
    if (lane == 0) cnt_w[wid] = nl;
    __syncthreads();
    nl = 0;
    for (int w = 0; w < TB / 32; ++w) nl += cnt_w[w];
    if (nl == 0 || nl == e - b) return;
    int64_t lbase = 0, rbase = 0;
    for (int64_t s = b; s < e; s += TB) {
        const int64_t p = s + tid;
        const int f = (p < e) && (pts[3 * p + axis] < mid);
        int tot;
        const int ex = block_exscan(f, tot);
        if (p < e) {
            const int64_t dst = f ? b + lbase + ex : b + nl + rbase + (tid - ex);
            tmp_pts[3 * dst + 0] = pts[3 * p + 0];
            tmp_pts[3 * dst + 1] = pts[3 * p + 1];
            tmp_pts[3 * dst + 2] = pts[3 * p + 2];
            tmp_perm[dst] = perm[p];
        }
        const int64_t chunk = (e - s) < TB ? (e - s) : TB;
        lbase += tot;
        rbase += chunk - tot;
    }
    __syncthreads();
    for (int64_t p = b + tid; p < e; p += TB) {
        pts[3 * p + 0] = tmp_pts[3 * p + 0];
        pts[3 * p + 1] = tmp_pts[3 * p + 1];
        pts[3 * p + 2] = tmp_pts[3 * p + 2];
        perm[p] = tmp_perm[p];
    }
    if (tid == 0) {
        T.is_leaf[c] = 0;
        T.nleft[c] = nl;
        split[blockIdx.x] = 1;
    }
}

// Creates the children of the clusters split at this level (ids in order),
// numbering them base, base+1, ... in the order of their parents.
__global__ void __launch_bounds__(1024) tree_children_kernel(const int64_t* ids, int64_t n,
                                                             DevTree T, const int32_t* split,
                                                             int64_t* next_ids, int64_t base,
                                                             int64_t* count) {
    int64_t run = 0;
    for (int64_t s = 0; s < n; s += blockDim.x) {
        const int64_t q = s + threadIdx.x;
        const int f = (q < n) ? split[q] : 0;
        int tot;
        const int ex = block_exscan(f, tot);
        if (f) {
            const int64_t c = ids[q];
            const int64_t k = run + ex;
            const int64_t c0 = base + 2 * k, c1 = c0 + 1;
            const int64_t b = T.begin[c], e = T.end[c], nl = T.nleft[c];
            T.child0[c] = c0;
            T.child1[c] = c1;
            const int lv = T.level[c] + 1;
            T.begin[c0] = b;
            T.end[c0] = b + nl;
            T.begin[c1] = b + nl;
            T.end[c1] = e;
            for (int64_t cc = c0; cc <= c1; ++cc) {
                T.level[cc] = lv;
                T.is_leaf[cc] = 1;
                T.child0[cc] = -1;
                T.child1[cc] = -1;
            }
            next_ids[2 * k] = c0;
            next_ids[2 * k + 1] = c1;
        }
        run += tot;
    }
    if (threadIdx.x == 0) *count = 2 * run;
}

// ---- partition ----
__device__ __forceinline__ double diam_box(const double* lo, const double* hi) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double e = __dsub_rn(hi[a], lo[a]);
        s = __dadd_rn(s, __dmul_rn(e, e));
    }
    return __dsqrt_rn(s);
}
__device__ __forceinline__ double dist_box(const double* lo1, const double* hi1,
                                           const double* lo2, const double* hi2) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        double g = 0.0;
        const double g1 = __dsub_rn(lo1[a], hi2[a]);
        const double g2 = __dsub_rn(lo2[a], hi1[a]);
        if (g1 > g) g = g1;
        if (g2 > g) g = g2;
        s = __dadd_rn(s, __dmul_rn(g, g));
    }
    return __dsqrt_rn(s);
}

// type: 0 low rank, 1 dense, 2 split
__global__ void part_classify_kernel(const int2* pairs, int64_t n, const double* lo,
                                     const double* hi, const int32_t* is_leaf, double eta,
                                     int8_t* type, unsigned long long* counts) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int t = pairs[q].x, s = pairs[q].y;
    const double d1 = diam_box(lo + 3 * t, hi + 3 * t), d2 = diam_box(lo + 3 * s, hi + 3 * s);
    const double dm = d1 < d2 ? d1 : d2;
    const double dist = dist_box(lo + 3 * t, hi + 3 * t, lo + 3 * s, hi + 3 * s);
    int8_t ty;
    if (dm < __dmul_rn(eta, dist))
        ty = 0;
    else if (is_leaf[t] || is_leaf[s])
        ty = 1;
    else
        ty = 2;
    type[q] = ty;
    atomicAdd(&counts[ty == 2 ? 1 : 0], 1ull);
}

__global__ void __launch_bounds__(1024) part_emit_kernel(const int2* pairs, int64_t n,
                                                         const int8_t* type,
                                                         const int64_t* child0,
                                                         const int64_t* child1, int2* out_blk,
                                                         int8_t* out_adm, int64_t blk_base,
                                                         int2* next) {
    int64_t rb = 0, rs = 0;
    for (int64_t s0 = 0; s0 < n; s0 += blockDim.x) {
        const int64_t q = s0 + threadIdx.x;
        const int ty = q < n ? type[q] : -1;
        int tb, ts;
        const int eb = block_exscan(ty == 0 || ty == 1, tb);
        const int es = block_exscan(ty == 2, ts);
        if (ty == 0 || ty == 1) {
            out_blk[blk_base + rb + eb] = pairs[q];
            out_adm[blk_base + rb + eb] = ty == 0 ? 1 : 0;
        } else if (ty == 2) {
            const int t = pairs[q].x, s = pairs[q].y;
            const int tc[2] = {(int)child0[t], (int)child1[t]};
            const int sc[2] = {(int)child0[s], (int)child1[s]};
            const int64_t o = 4 * (rs + es);
            next[o + 0] = make_int2(tc[0], sc[0]);
            next[o + 1] = make_int2(tc[0], sc[1]);
            next[o + 2] = make_int2(tc[1], sc[0]);
            next[o + 3] = make_int2(tc[1], sc[1]);
        }
        rb += tb;
        rs += ts;
    }
}

template <class T>
T* dalloc(size_t n, cudaStream_t st) {
    void* p = nullptr;
    HM_CUDA(cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), st));
    return (T*)p;
}

}  // namespace

TreeResult build_cluster_tree(double* d_pts, int64_t* d_perm, int64_t nc, int64_t leaf,
                              cudaStream_t st) {
    TreeResult R;
    const int64_t cap = 2 * nc + 1;
    DevTree T;
    T.begin = dalloc<int64_t>(cap, st);
    T.end = dalloc<int64_t>(cap, st);
    T.lo = dalloc<double>(3 * cap, st);
    T.hi = dalloc<double>(3 * cap, st);
    T.level = dalloc<int32_t>(cap, st);
    T.is_leaf = dalloc<int32_t>(cap, st);
    T.child0 = dalloc<int64_t>(cap, st);
    T.child1 = dalloc<int64_t>(cap, st);
    T.nleft = dalloc<int64_t>(cap, st);
    double* tmp_pts = dalloc<double>(3 * nc, st);
    int64_t* tmp_perm = dalloc<int64_t>(nc, st);
    int64_t* ids = dalloc<int64_t>(nc + 1, st);
    int64_t* next = dalloc<int64_t>(nc + 1, st);
    int32_t* split = dalloc<int32_t>(nc + 1, st);
    int64_t* d_count = dalloc<int64_t>(1, st);
    {
        const int64_t zero = 0, one_leaf = 1, minus1 = -1;
        const int32_t lvl0 = 0, leaf1 = 1;
        HM_CUDA(cudaMemcpyAsync(T.begin, &zero, 8, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(T.end, &nc, 8, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(T.level, &lvl0, 4, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(T.is_leaf, &leaf1, 4, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(T.child0, &minus1, 8, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(T.child1, &minus1, 8, cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaMemcpyAsync(ids, &zero, 8, cudaMemcpyHostToDevice, st));
        (void)one_leaf;
    }
    int64_t n = 1, ncl = 1;
    int level = 0;
    while (n > 0) {
        tree_level_kernel<<<(unsigned)n, TB, 0, st>>>(ids, T, d_pts, d_perm, tmp_pts, tmp_perm,
                                                      leaf, split);
                                                      HM_LAUNCHED();
        HM_CUDA(cudaGetLastError());
        tree_children_kernel<<<1, 1024, 0, st>>>(ids, n, T, split, next, ncl, d_count);
        HM_LAUNCHED();
        HM_CUDA(cudaGetLastError());
        int64_t cnt = 0;
        HM_CUDA(cudaMemcpyAsync(&cnt, d_count, 8, cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        if (cnt > 0) level++;
        ncl += cnt;
        std::swap(ids, next);
        n = cnt;
    }
    R.depth = level;
    std::vector<int64_t> b(ncl), e(ncl), c0(ncl), c1(ncl);
    std::vector<double> lo(3 * ncl), hi(3 * ncl);
    std::vector<int32_t> lv(ncl), il(ncl);
    HM_CUDA(cudaMemcpyAsync(b.data(), T.begin, 8 * ncl, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(e.data(), T.end, 8 * ncl, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(c0.data(), T.child0, 8 * ncl, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(c1.data(), T.child1, 8 * ncl, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(lo.data(), T.lo, 24 * ncl, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(hi.data(), T.hi, 24 * ncl, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(lv.data(), T.level, 4 * ncl, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(il.data(), T.is_leaf, 4 * ncl, cudaMemcpyDeviceToHost, st));
    R.perm.resize(nc);
    HM_CUDA(cudaMemcpyAsync(R.perm.data(), d_perm, 8 * nc, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    R.clusters.resize(ncl);
    for (int64_t c = 0; c < ncl; ++c) {
        hm_cluster& h = R.clusters[c];
        h.begin = b[c];
        h.end = e[c];
        h.child0 = il[c] ? -1 : c0[c];
        h.child1 = il[c] ? -1 : c1[c];
        h.level = lv[c];
        h.is_leaf = il[c];
        for (int a = 0; a < 3; ++a) {
            h.lo[a] = lo[3 * c + a];
            h.hi[a] = hi[3 * c + a];
        }
    }
    for (void* p : {(void*)T.begin, (void*)T.end, (void*)T.lo, (void*)T.hi, (void*)T.level,
                    (void*)T.is_leaf, (void*)T.child0, (void*)T.child1, (void*)T.nleft,
                    (void*)tmp_pts, (void*)tmp_perm, (void*)ids, (void*)next, (void*)split,
                    (void*)d_count})
        HM_CUDA(cudaFreeAsync(p, st));
    return R;
}

std::vector<hm_block> build_partition(const std::vector<hm_cluster>& cl, double eta,
                                      cudaStream_t st, int64_t sigma_root) {
    const int64_t ncl = (int64_t)cl.size();
    std::vector<double> lo(3 * ncl), hi(3 * ncl);
    std::vector<int32_t> il(ncl);
    std::vector<int64_t> c0(ncl), c1(ncl);
    for (int64_t c = 0; c < ncl; ++c) {
        for (int a = 0; a < 3; ++a) {
            lo[3 * c + a] = cl[c].lo[a];
            hi[3 * c + a] = cl[c].hi[a];
        }
        il[c] = cl[c].is_leaf;
        c0[c] = cl[c].child0;
        c1[c] = cl[c].child1;
    }
    double* d_lo = dalloc<double>(3 * ncl, st);
    double* d_hi = dalloc<double>(3 * ncl, st);
    int32_t* d_il = dalloc<int32_t>(ncl, st);
    int64_t* d_c0 = dalloc<int64_t>(ncl, st);
    int64_t* d_c1 = dalloc<int64_t>(ncl, st);
    HM_CUDA(cudaMemcpyAsync(d_lo, lo.data(), 24 * ncl, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(d_hi, hi.data(), 24 * ncl, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(d_il, il.data(), 4 * ncl, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(d_c0, c0.data(), 8 * ncl, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(d_c1, c1.data(), 8 * ncl, cudaMemcpyHostToDevice, st));

    int64_t fcap = 1024, bcap = 4096;
    int2* front = dalloc<int2>(fcap, st);
    int2* next = dalloc<int2>(fcap, st);
    int8_t* type = dalloc<int8_t>(fcap, st);
    int2* blk = dalloc<int2>(bcap, st);
    int8_t* adm = dalloc<int8_t>(bcap, st);
    unsigned long long* d_counts = dalloc<unsigned long long>(2, st);
    const int2 root = make_int2(0, (int)sigma_root);
    HM_CUDA(cudaMemcpyAsync(front, &root, sizeof(int2), cudaMemcpyHostToDevice, st));
    int64_t n = 1, nb = 0;
    while (n > 0) {
        HM_CUDA(cudaMemsetAsync(d_counts, 0, 16, st));
        part_classify_kernel<<<(unsigned)hm_cdiv(n, 256), 256, 0, st>>>(
            front, n, d_lo, d_hi, d_il, eta, type, d_counts);
            HM_LAUNCHED();
        HM_CUDA(cudaGetLastError());
        unsigned long long cnt[2];
        HM_CUDA(cudaMemcpyAsync(cnt, d_counts, 16, cudaMemcpyDeviceToHost, st));
        HM_CUDA(cudaStreamSynchronize(st));
        const int64_t nblk = (int64_t)cnt[0], nnext = 4 * (int64_t)cnt[1];
        if (nb + nblk > bcap) {  // grow the block list
            int64_t nc2 = std::max(2 * bcap, nb + nblk);
            int2* b2 = dalloc<int2>(nc2, st);
            int8_t* a2 = dalloc<int8_t>(nc2, st);
            HM_CUDA(cudaMemcpyAsync(b2, blk, nb * sizeof(int2), cudaMemcpyDeviceToDevice, st));
            HM_CUDA(cudaMemcpyAsync(a2, adm, nb, cudaMemcpyDeviceToDevice, st));
            HM_CUDA(cudaFreeAsync(blk, st));
            HM_CUDA(cudaFreeAsync(adm, st));
            blk = b2;
            adm = a2;
            bcap = nc2;
        }
        if (nnext > fcap) {
            HM_CUDA(cudaFreeAsync(next, st));
            next = dalloc<int2>(nnext, st);
            // front must also fit the next level when swapped
            int2* f2 = dalloc<int2>(nnext, st);
            HM_CUDA(cudaMemcpyAsync(f2, front, n * sizeof(int2), cudaMemcpyDeviceToDevice, st));
            HM_CUDA(cudaFreeAsync(front, st));
            front = f2;
            int8_t* t2 = dalloc<int8_t>(nnext, st);
            HM_CUDA(cudaMemcpyAsync(t2, type, n, cudaMemcpyDeviceToDevice, st));
            HM_CUDA(cudaFreeAsync(type, st));
            type = t2;
            fcap = nnext;
        }
        part_emit_kernel<<<1, 1024, 0, st>>>(front, n, type, d_c0, d_c1, blk, adm, nb, next);
        HM_LAUNCHED();
        HM_CUDA(cudaGetLastError());
        nb += nblk;
        std::swap(front, next);
        n = nnext;
    }
    std::vector<int2> hb(nb);
    std::vector<int8_t> ha(nb);
    HM_CUDA(cudaMemcpyAsync(hb.data(), blk, nb * sizeof(int2), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaMemcpyAsync(ha.data(), adm, nb, cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    for (void* p : {(void*)d_lo, (void*)d_hi, (void*)d_il, (void*)d_c0, (void*)d_c1,
                    (void*)front, (void*)next, (void*)type, (void*)blk, (void*)adm,
                    (void*)d_counts})
        HM_CUDA(cudaFreeAsync(p, st));
    std::vector<hm_block> out(nb);
    for (int64_t q = 0; q < nb; ++q) {
        out[q].tau = hb[q].x;
        out[q].sigma = hb[q].y;
        out[q].admissible = ha[q];
        out[q].rank_aca = 0;
        out[q].rank = 0;
        out[q].pad_ = 0;
    }
    return out;
}
