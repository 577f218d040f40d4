// matvec_multi.cu — the H-matrix product (Sec. 3.1) for a block of
// NRHS_BLOCK = 32 right-hand sides on the tcgen05 tensor cores, BF16 storage.
//
// With 32 right-hand sides every stored complex entry meets 32 vector
// entries: D X and U (V^H X) become dense contractions, run as real BF16 MMAs
// (kind::f16, FP32 accumulators in TMEM).  A complex entry a = (a_r, a_i) is
// one bf16 pair; the right-hand side s occupies the real columns n = 2s
// (real part) and n = 2s + 1 (imaginary part) of the MMA's N = 64.
//
//  phase 1, t = s_U s_V V^H x per V column j (M = columns, K = 2 rows):
//     A[j][2r + c] = component c of V[r][j] (the stored column, K-major),
//     B[2r][n]     = (x_r, x_i) of right-hand side n / 2    (row 2r of XB),
//     B[2r + 1][n] = (x_i, -x_r), i.e. -i x               (row 2r + 1 of XB),
//     so D[j][2s] + i D[j][2s + 1] = sum_r conj(V[r][j]) x_s[r].
//  phase 2, y += M w over the item's columns j (M = 2 rows, K = columns):
//     A[2r + c][j] = component c of M[r][j] (the stored column, MN-major),
//     B[j][n]      = the bf16 row of w_j: T16 row t_j (U columns) or XB row
//                    2 dof_j (dense columns),
//     so y_r(s) = D[2r][2s] - D[2r+1][2s+1] + i (D[2r][2s+1] + D[2r+1][2s]).
//
// The BF16 arena is viewed, per leading dimension ld16, as a 2-D tensor whose
// rows are the stored columns (2 ld16 bf16 each, 4 ld16 bytes apart); every
// work item (the chunks of one leaf, stored back to back) starts on a row of
// that view.  TMA loads 128-byte-swizzled tiles of it (and of XB) straight
// into the operand layout the MMA reads, so no thread touches the stored
// entries.  One CTA per item: warp 0 issues the TMA loads, warp 1 the MMAs
// (it owns the TMEM allocation), warps 2-5 copy the phase-2 weight rows and
// move the accumulators out (FP32 atomics: several items share T rows and Y
// rows).  Every wait is bounded; a timeout sets the error word and the CTA
// drains its own copies and MMAs before it retires.
//
// Vectors (tree order, right-hand side fastest, complex): XB[2 dof + c][32]
// bf16 pairs, T[t][32] FP32 (accumulated), T16[t][32] bf16 pairs, Y[dof][32]
// FP32.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "matvec_dev.cuh"
#include "pipeline.cuh"

namespace {

constexpr int NR = NRHS_BLOCK;
static_assert(NR == 32 && NR == HM_NRHS_BLOCK, "N = 64 real columns: 32 right-hand sides");
constexpr int MV_ERR_TIMEOUT = 1;

constexpr int TC_KBMAX = 2 * MAX_LD / 64;             // 64-wide K boxes of a column (6)
// phase 1: warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int P1_THREADS = 192;
constexpr int P1_NS = 8;                              // A stages
constexpr int P1_BOX = 16;                            // row granularity of the A boxes
constexpr int P1_NZ = 4;                              // A box heights 128, 64, 32, 16 (map sets)
constexpr bool P1_SPLIT_TAIL = true;                  // last tile of an item: boxes cover its rows
constexpr int P1_MT = 4;                              // M tiles of an item (512 columns)
constexpr int P1_ABYTES = 128 * 128;                  // 128 columns x 64 bf16 of K
constexpr int P1_BBYTES = 64 * 128;                   // 64 K rows of XB
constexpr uint32_t P1_TMEM_COLS = 512;                // two sets of four 128 x 64 accumulators
// phase 2: warp 0 TMA, warp 1 MMA, P2_WW weight-row warps, four epilogue warps
constexpr int P2_WW = 4;                              // weight-row warps
constexpr int P2_WT = 32 * P2_WW;                     // weight-row threads
constexpr int P2_THREADS = 32 * (2 + P2_WW + 4);
constexpr int P2_NS = 6;
constexpr int P2_ABYTES = TC_KBMAX * 4096;            // up to six 64 x 32 boxes
constexpr int P2_WBYTES = 32 * 128;                   // 32 weight rows
constexpr uint32_t P2_TMEM_COLS = 512;                // two sets of up to three 128 x 64
// kind::f16 instruction descriptor: FP32 accumulate (bit 4), A and B BF16
// (bits 7, 10), A MN-major (bit 15), B MN-major (bit 16), N >> 3 at bit 17,
// M >> 4 at bit 24; M = 128, N = 64
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(64 >> 3) << 17) |
                              (uint32_t(128 >> 4) << 24);
constexpr uint32_t TC_A_MN = 1u << 15;
constexpr uint32_t TC_B_MN = 1u << 16;

struct P1Smem {
    unsigned char a[P1_NS][P1_ABYTES];         // 1024-byte aligned (swizzle atoms)
    unsigned char b[2][TC_KBMAX][P1_BBYTES];   // XB rows of two segments (all K boxes)
    int32_t abort;
    uint32_t tmem;
    alignas(8) uint64_t full[P1_NS];
    uint64_t empty[P1_NS];
    uint64_t bfull[2];
    uint64_t bempty[2];
    uint64_t accf[2];
    uint64_t acce[2];
};
struct P2Smem {
    unsigned char a[P2_NS][P2_ABYTES];
    unsigned char w[P2_NS][P2_WBYTES];
    uint32_t code[2][MAX_ITEM_COLS];  // column codes of two items (weight-row warps)
    int32_t abort;
    uint32_t tmem;
    alignas(8) uint64_t full[P2_NS];
    uint64_t wfull[P2_NS];
    uint64_t empty[P2_NS];
    uint64_t accf[2];
    uint64_t acce[2];
};
// one CTA per SM (persistent): all of TMEM is available, shared memory within
// 227 KB including the 1 KB alignment slack
static_assert(sizeof(P1Smem) + 1024 <= 227 * 1024, "phase 1 shared memory");
static_assert(sizeof(P2Smem) + 1024 <= 227 * 1024, "phase 2 shared memory");
static_assert(P2_WT % 8 == 0 && 256 % P2_WT == 0 && MAX_ITEM_COLS % P2_WT == 0, "weight-row threads");
static_assert(TC_KBMAX <= 6 && P2_ABYTES == 6 * 4096, "phase-2 stages: at most three M tiles");
static_assert(P1_NZ == TMAP_PHASE2 && (128 >> (P1_NZ - 1)) == P1_BOX, "phase-1 map sets");
static_assert(P1_ABYTES % 1024 == 0 && P1_BBYTES % 1024 == 0 && P2_ABYTES % 1024 == 0 &&
                  (P1_BOX * 128) % 1024 == 0 && 128 % P1_BOX == 0 &&
                  P2_WBYTES % 1024 == 0,
              "swizzle atoms stay aligned");

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return l | (h << 16);
}

// Slot and phase parity of a ring of n stages, advanced stage by stage (no
// divisions in the issue loops).
struct Ring {
    uint32_t q = 0, ph = 0;
    __device__ __forceinline__ void next(int n) {
        if (++q == (uint32_t)n) {
            q = 0;
            ph ^= 1u;
        }
    }
};

// Rows of M tile mt of an item of ncol columns as the phase-1 copies load them:
// 128 (one box) or the tile's columns rounded up to 16.
__device__ __forceinline__ int tile_rows(int ncol, int mt) {
    return P1_SPLIT_TAIL ? (min(128, ncol - 128 * mt) + P1_BOX - 1) / P1_BOX * P1_BOX : 128;
}

// Shared-memory matrix descriptor, 128-byte swizzle: start >> 4, leading byte
// offset >> 4 (MN-major: between 64-element atoms along M/N), stride byte
// offset >> 4 (between 8-row groups), version 1, layout 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Issue helpers of a role that a whole warp runs with warp-uniform control
// flow and operands: elect.sync picks the one lane that issues, so the
// operands need not move out of the uniform datapath for every instruction.
__device__ __forceinline__ void w_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t}" ::"r"(smem_u32(b)),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ void w_tma_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar,
                                         uint64_t policy) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;\n\t}" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void w_tma_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                         uint64_t* bar, uint64_t policy) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;\n\t}" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void w_umma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void w_commit(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void tmap_acquire(const CUtensorMap* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
// the 64 accumulator columns [col, col + 64) of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld64(uint32_t tmem, int lane_quarter, int col, uint32_t (&v)[64]) {
    const uint32_t base = tmem + ((uint32_t)(lane_quarter * 32) << 16) + (uint32_t)col;
    tmem_ld16(base, v);
    tmem_ld16(base + 16, v + 16);
    tmem_ld16(base + 32, v + 32);
    tmem_ld16(base + 48, v + 48);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// y[0..3] += v without a return value (a reduction, not an atomic round trip)
__device__ __forceinline__ void red_add_v4(float* y, float a, float b, float c, float d) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(y), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// The kernel's shared-memory struct at the first 1024-byte boundary of the
// dynamic allocation (which carries 1024 bytes of slack).
template <typename Smem>
__device__ __forceinline__ Smem& tc_smem(unsigned char* raw) {
    return *reinterpret_cast<Smem*>(raw + ((1024u - (smem_u32(raw) & 1023u)) & 1023u));
}

// The items of this CTA (blockIdx.x, + gridDim.x, ...), the record of the
// next one fetched an item ahead.
template <typename Item>
struct ItemIter {
    const Item* items;
    int nitems, item;
    Item cur, nxt;
    __device__ ItemIter(const Item* it, int n) : items(it), nitems(n), item(blockIdx.x) {
        if (item < n) cur = it[item];
        if (item + (int)gridDim.x < n) nxt = it[item + gridDim.x];
    }
    __device__ bool valid() const { return item < nitems; }
    __device__ bool has_next() const { return item + (int)gridDim.x < nitems; }
    __device__ void advance() {
        item += gridDim.x;
        cur = nxt;
        if (has_next()) nxt = items[item + gridDim.x];
    }
};

// TMEM allocation by warp 1 and the abort flag; ends past a block barrier
// (barriers are initialised by thread 0 before).
template <typename Smem>
__device__ __forceinline__ void tc_setup(Smem& S, uint32_t cols) {
    if ((threadIdx.x >> 5) == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) S.abort = 0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}
template <typename Smem>
__device__ __forceinline__ void tc_teardown(Smem& S, uint32_t cols) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"(cols));
}

// 16-byte asynchronous copy global -> shared (bytes = 16, or 0 to zero-fill)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes)
                 : "memory");
}
// A wait of one role: on a timeout the error word and the abort flag are set
// and false is returned; once the flag is set no role waits for a phase that
// has not completed.
template <typename Smem>
__device__ __forceinline__ bool tc_wait(Smem& S, uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*(volatile int32_t*)&S.abort) return false;
    if (mbar_wait_slow(bar, parity)) return true;
    atomicExch(err, MV_ERR_TIMEOUT);
    *(volatile int32_t*)&S.abort = 1;
    return false;
}
// Item and segment records as warp-uniform values (lane 0's copy): the loop
// bounds of the issuing roles then stay on the uniform datapath.
__device__ __forceinline__ int uni(int v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ int64_t uni(int64_t v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ TcGroup uni(const TcGroup& x) {
    return {uni(x.t0), uni(x.ncol), uni(x.seg0), uni(x.seg1), uni(x.red)};
}
__device__ __forceinline__ TcSeg uni(const TcSeg& x) { return {uni(x.dof), uni(x.row0), uni(x.ld16)}; }
__device__ __forceinline__ TcItem uni(const TcItem& x) {
    return {uni(x.dof), uni(x.col0), uni(x.row0), uni(x.ld16), uni(x.ncol), uni(x.rows)};
}
// The same wait taken by a whole warp, with one result for all its lanes.
template <typename Smem>
__device__ __forceinline__ bool w_wait(Smem& S, uint64_t* bar, uint32_t parity, int* err) {
    return __all_sync(0xffffffffu, tc_wait(S, bar, parity, err));
}
template <typename Smem>
__device__ __forceinline__ bool tc_aborted(Smem& S) {
    return *(volatile int32_t*)&S.abort != 0;
}

// Phase 1 (persistent, items blockIdx.x, + gridDim.x, ...): T[t0 + j] =
// s_V s_U D[j] for the columns j of one column-cluster group: the V columns of
// every block that shares the column cluster sigma are one run of rows of
// each segment of sigma, in the same order, so one set of TMEM accumulators
// (up to four 128 x 64 M tiles) sums over all segments of sigma (K) and the
// t rows are written once.  Stages run over (item, segment, M tile, 64-wide K
// box), so the K boxes of a stored column are read back to back; the XB rows
// of a segment (the B operand, all its K boxes) go to one of two buffers; an
// A tile is one 128-row TMA box, or for the last tile of an item boxes of 64,
// 32 and 16 rows that cover its columns rounded up to 16.  Two
// accumulator sets let the epilogue of an item trail the MMAs of the next.
// Items of a group cut along K add into zeroed t rows.
__global__ void __launch_bounds__(P1_THREADS, 1) mvc_phase1(const TcGroup* items, int nitems,
                                                           const TcSeg* __restrict__ segs,
                                                           const float* __restrict__ tscale,
                                                           const CUtensorMap* maps,
                                                           const CUtensorMap* map_xb, float2* T,
                                                           int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    P1Smem& S = tc_smem<P1Smem>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    if (tid == 0) {
        for (int q = 0; q < P1_NS; ++q) {
            mbar_init(&S.full[q], 1);
            mbar_init(&S.empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&S.bfull[q], 1);
            mbar_init(&S.bempty[q], 1);
            mbar_init(&S.accf[q], 1);
            mbar_init(&S.acce[q], 4);
        }
        mbar_fence_init();
    }
    tc_setup(S, P1_TMEM_COLS);
    const uint32_t tmem = S.tmem;
    if (warp == 0) {  // ---- TMA producer ----
        {  // the whole warp: one lane issues (elect.sync)
            tmap_acquire(map_xb);
            const uint64_t pol_stream = l2_policy_evict_first(), pol_keep = l2_policy_evict_last();
            int g = 0, gs = 0;  // A stages and segments issued
            Ring ra;            // A ring slot of stage g
            uint64_t acquired[P1_NZ] = {0, 0, 0, 0};
            bool ok = true;
            for (ItemIter<TcGroup> X(items, nitems); ok && X.valid() && !tc_aborted(S); X.advance()) {
                const TcGroup I = uni(X.cur);
                const int nmt = (I.ncol + 127) >> 7;
                TcSeg nx = uni(segs[I.seg0]);
                for (int s = I.seg0; ok && s < I.seg1; ++s) {
                    const TcSeg sg = nx;
                    if (s + 1 < I.seg1) nx = uni(segs[s + 1]);  // read one segment ahead
                    const int li = sg.ld16 >> 2;
                    const int nkb = (2 * sg.ld16 + 63) >> 6, bs = gs & 1;
                    if (gs >= 2 && !w_wait(S, &S.bempty[bs], ((gs >> 1) - 1) & 1, err)) break;
                    // B: XB rows 2 dof + k, k < 64 nkb (beyond 2 R they meet zero A entries)
                    w_expect_tx(&S.bfull[bs], (uint32_t)nkb * P1_BBYTES);
                    for (int kb = 0; kb < nkb; ++kb)
                        w_tma_2d(S.b[bs][kb], map_xb, 0, (int)(2 * sg.dof) + 64 * kb, &S.bfull[bs], pol_keep);
                    ++gs;
                    for (int mt = 0; mt < nmt; ++mt) {
                        const int rr = tile_rows(I.ncol, mt);
                        for (int z = 0; z < P1_NZ; ++z)
                            if ((rr == 128) == (z == 0) && (z == 0 || (rr & (128 >> z))) &&
                                !((acquired[z] >> li) & 1)) {  // each descriptor once
                                tmap_acquire(maps + z * TMAP_PER_PHASE + li);
                                acquired[z] |= 1ull << li;
                            }
                    }
                    const CUtensorMap* map0 = maps + li;
                    for (int mt = 0; ok && mt < nmt; ++mt) {
                        const int rr = tile_rows(I.ncol, mt), y = sg.row0 + 128 * mt;
                        for (int kb = 0; kb < nkb; ++kb) {
                            if (g >= P1_NS && !w_wait(S, &S.empty[ra.q], ra.ph ^ 1u, err)) {
                                ok = false;
                                break;
                            }
                            unsigned char* dst = S.a[ra.q];
                            uint64_t* bar = &S.full[ra.q];
                            w_expect_tx(bar, (uint32_t)(rr * 128));
                            if (rr == 128) {
                                w_tma_2d(dst, map0, kb * 64, y, bar, pol_stream);
                            } else {
                                int off = 0;
#pragma unroll
                                for (int z = 1; z < P1_NZ; ++z)
                                    if (rr & (128 >> z)) {
                                        w_tma_2d(dst + off * 128, map0 + z * TMAP_PER_PHASE, kb * 64, y + off,
                                                    bar, pol_stream);
                                        off += 128 >> z;
                                    }
                            }
                            ++g;
                            ra.next(P1_NS);
                        }
                    }
                }
            }
            // own copies land before the block can retire (an abort may leave
            // the count one short of a stage: waiting on it only times out)
            for (int k = max(0, gs - 2); k < gs; ++k)
                if (!mbar_wait(&S.bfull[k & 1], (k >> 1) & 1)) atomicExch(err, MV_ERR_TIMEOUT);
            for (int k = max(0, g - P1_NS); k < g; ++k)
                if (!mbar_wait(&S.full[k % P1_NS], (k / P1_NS) & 1)) atomicExch(err, MV_ERR_TIMEOUT);
        }
        __syncwarp();
    } else if (warp == 1) {  // ---- MMA issue ----
        {  // the whole warp: one lane issues (elect.sync)
            int g = 0, gs = 0, ii = 0;  // A stages, segments, items
            Ring ra;
            bool ok = true;
            // descriptors of A stage 0 and B buffer 0; the others are offsets
            // in the 16-byte address field (no carry: shared memory < 256 KB)
            const uint64_t da0 = desc_sw128(smem_u32(S.a[0]), 16, 1024);
            const uint64_t db0 = desc_sw128(smem_u32(S.b[0][0]), 8192, 1024);
            for (ItemIter<TcGroup> X(items, nitems); ok && X.valid(); X.advance(), ++ii) {
                const TcGroup I = uni(X.cur);
                const int nmt = (I.ncol + 127) >> 7, set = ii & 1;
                if (ii >= 2 && !w_wait(S, &S.acce[set], ((ii >> 1) - 1) & 1, err)) break;
                tc_fence_after();
                const uint32_t dacc = tmem + (uint32_t)(set * 256);
                int nkb_next = (2 * uni(segs[I.seg0].ld16) + 63) >> 6;
                for (int s = I.seg0; ok && s < I.seg1; ++s) {
                    const int nkb = nkb_next, bs = gs & 1;
                    if (s + 1 < I.seg1) nkb_next = (2 * uni(segs[s + 1].ld16) + 63) >> 6;
                    if (!w_wait(S, &S.bfull[bs], (gs >> 1) & 1, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t dbs = db0 + (uint64_t)((bs * TC_KBMAX * P1_BBYTES) >> 4);
                    for (int mt = 0; ok && mt < nmt; ++mt) {
                        const uint32_t d = dacc + (uint32_t)(mt * 64);
                        for (int kb = 0; kb < nkb; ++kb) {
                            if (!w_wait(S, &S.full[ra.q], ra.ph, err)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint64_t da = da0 + (uint64_t)((ra.q * P1_ABYTES) >> 4);
                            const uint64_t db = dbs + (uint64_t)((kb * P1_BBYTES) >> 4);
                            // K = 16 per MMA: 32 bytes along A's rows, two 8-row groups of B
                            w_umma(d, da, db, TC_IDESC | TC_B_MN, (s > I.seg0 || kb > 0) ? 1u : 0u);
                            w_umma(d, da + 2, db + 128, TC_IDESC | TC_B_MN, 1u);
                            w_umma(d, da + 4, db + 256, TC_IDESC | TC_B_MN, 1u);
                            w_umma(d, da + 6, db + 384, TC_IDESC | TC_B_MN, 1u);
                            w_commit(&S.empty[ra.q]);
                            ++g;
                            ra.next(P1_NS);
                        }
                    }
                    if (!ok) break;
                    w_commit(&S.bempty[bs]);
                    ++gs;
                }
                if (ok) w_commit(&S.accf[set]);
            }
            if (g > 0) {  // the MMAs finish before shared memory and TMEM go
                const int k = g - 1;
                if (!mbar_wait(&S.empty[k % P1_NS], (k / P1_NS) & 1)) atomicExch(err, MV_ERR_TIMEOUT);
            }
        }
        __syncwarp();
    } else {  // ---- accumulators into T ----
        const int lq = warp & 3;  // TMEM lane quarter this warp may read
        int ii = 0;
        for (ItemIter<TcGroup> X(items, nitems); X.valid(); X.advance(), ++ii) {
            const TcGroup I = X.cur;
            const int nmt = (I.ncol + 127) >> 7, set = ii & 1;
            float sc[P1_MT];
#pragma unroll
            for (int mt = 0; mt < P1_MT; ++mt) {
                const int j = 128 * mt + 32 * lq + lane;
                sc[mt] = j < I.ncol ? __ldg(tscale + I.t0 + j) : 0.f;
            }
            if (!__all_sync(0xffffffffu, tc_wait(S, &S.accf[set], (ii >> 1) & 1, err))) break;
            tc_fence_after();
#pragma unroll
            for (int mt = 0; mt < P1_MT; ++mt) {
                if (mt < nmt) {
                    uint32_t v[64];
                    tmem_ld64(tmem, lq, set * 256 + mt * 64, v);
                    const int j = 128 * mt + 32 * lq + lane;
                    if (j < I.ncol) {
                        float* dst = reinterpret_cast<float*>(T + (I.t0 + j) * NR);
                        const float c = sc[mt];
                        if (I.red) {
#pragma unroll
                            for (int q = 0; q < 16; ++q)
                                red_add_v4(dst + 4 * q, c * __uint_as_float(v[4 * q]),
                                           c * __uint_as_float(v[4 * q + 1]), c * __uint_as_float(v[4 * q + 2]),
                                           c * __uint_as_float(v[4 * q + 3]));
                        } else {
#pragma unroll
                            for (int q = 0; q < 16; ++q)
                                reinterpret_cast<float4*>(dst)[q] =
                                    make_float4(c * __uint_as_float(v[4 * q]), c * __uint_as_float(v[4 * q + 1]),
                                                c * __uint_as_float(v[4 * q + 2]), c * __uint_as_float(v[4 * q + 3]));
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.acce[set]);
        }
    }
    tc_teardown(S, P1_TMEM_COLS);
}

// Phase 2 (persistent): Y[dof + r] += sum_j M[r][j] w_j over the columns j of
// each item (the dense and U chunks of one row leaf).  Stages of 32 columns
// run across items: the A boxes by TMA, the 32 weight rows (128 bytes each)
// copied by the weight-row warps (cp.async) into the swizzled B layout.  Two sets of TMEM
// accumulators (one item each) let the epilogue of an item overlap the next.
__global__ void __launch_bounds__(P2_THREADS, 1) mvc_phase2(const TcItem* items, int nitems,
                                                           const uint32_t* __restrict__ colcode,
                                                           const CUtensorMap* maps,
                                                           const uint32_t* __restrict__ XB,
                                                           const uint32_t* __restrict__ T16,
                                                           float2* Y, int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    P2Smem& S = tc_smem<P2Smem>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    if (tid == 0) {
        for (int q = 0; q < P2_NS; ++q) {
            mbar_init(&S.full[q], 1);
            mbar_init(&S.wfull[q], P2_WT);  // one arrival per weight-row thread
            mbar_init(&S.empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&S.accf[q], 1);
            mbar_init(&S.acce[q], 4);
        }
        mbar_fence_init();
    }
    tc_setup(S, P2_TMEM_COLS);
    const uint32_t tmem = S.tmem;
    if (warp == 0) {  // ---- TMA producer ----
        {  // the whole warp: one lane issues (elect.sync)
            const uint64_t pol = l2_policy_evict_first();
            int g = 0;
            Ring ra;
            uint64_t acquired = 0;
            for (ItemIter<TcItem> X(items, nitems); X.valid() && !tc_aborted(S); X.advance()) {
                const TcItem I = uni(X.cur);
                const CUtensorMap* map = maps + (I.ld16 >> 2);
                if (!((acquired >> (I.ld16 >> 2)) & 1)) {  // each descriptor once
                    tmap_acquire(map);
                    acquired |= 1ull << (I.ld16 >> 2);
                }
                const int nbox = (2 * I.ld16 + 63) >> 6;  // 64-row m-blocks along m = 2r + re/im
                const int nst = (I.ncol + 31) >> 5;
                for (int k = 0; k < nst; ++k, ++g, ra.next(P2_NS)) {
                    if (g >= P2_NS && !w_wait(S, &S.empty[ra.q], ra.ph ^ 1u, err)) break;
                    // one copy: 32 stored columns x all m-blocks, m-block b at 4096 b
                    w_expect_tx(&S.full[ra.q], (uint32_t)nbox * 4096u);
                    w_tma_3d(S.a[ra.q], map, 0, I.row0 + k * 32, 0, &S.full[ra.q], pol);
                }
            }
            for (int k = max(0, g - P2_NS); k < g; ++k)
                if (!mbar_wait(&S.full[k % P2_NS], (k / P2_NS) & 1)) atomicExch(err, MV_ERR_TIMEOUT);
        }
        __syncwarp();
    } else if (warp == 1) {  // ---- MMA issue ----
        {  // the whole warp: one lane issues (elect.sync)
            int g = 0, ii = 0;
            Ring ra;
            bool ok = true;
            // descriptors of A stage 0 and weight stage 0 (others: address-field offsets)
            const uint64_t da0 = desc_sw128(smem_u32(S.a[0]), 4096, 1024);
            const uint64_t dw0 = desc_sw128(smem_u32(S.w[0]), 8192, 1024);
            for (ItemIter<TcItem> X(items, nitems); ok && X.valid(); X.advance(), ++ii) {
                const TcItem I = uni(X.cur);
                const int nmt = (((2 * I.ld16 + 63) >> 6) + 1) >> 1;  // 128-row M tiles
                const int nst = (I.ncol + 31) >> 5;
                const int set = ii & 1;
                if (ii >= 2 && !w_wait(S, &S.acce[set], ((ii >> 1) - 1) & 1, err)) break;
                tc_fence_after();
                const uint32_t dacc = tmem + (uint32_t)(set * 256);
                for (int k = 0; k < nst; ++k, ++g, ra.next(P2_NS)) {
                    if (!w_wait(S, &S.full[ra.q], ra.ph, err) || !w_wait(S, &S.wfull[ra.q], ra.ph, err)) {
                        ok = false;
                        break;
                    }
                    // the weight rows were written by cp.async (generic proxy): order
                    // them before the tensor core's reads
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tc_fence_after();
                    const uint64_t da = da0 + (uint64_t)((ra.q * P2_ABYTES) >> 4);
                    const uint64_t dw = dw0 + (uint64_t)((ra.q * P2_WBYTES) >> 4);
                    const uint32_t en = k > 0 ? 1u : 0u;
#pragma unroll
                    for (int t = 0; t < 3; ++t)  // K = 16 per MMA: two 8-row groups of both operands
                        if (t < nmt) {
                            w_umma(dacc + (uint32_t)(t * 64), da + (uint64_t)(t * 512), dw,
                                 TC_IDESC | TC_A_MN | TC_B_MN, en);
                            w_umma(dacc + (uint32_t)(t * 64), da + (uint64_t)(t * 512 + 128), dw + 128,
                                 TC_IDESC | TC_A_MN | TC_B_MN, 1u);
                        }
                    w_commit(&S.empty[ra.q]);
                }
                if (ok) w_commit(&S.accf[set]);  // also for an empty item: keeps the phases in step
            }
            if (g > 0) {
                const int k = g - 1;
                if (!mbar_wait(&S.empty[k % P2_NS], (k / P2_NS) & 1)) atomicExch(err, MV_ERR_TIMEOUT);
            }
        }
        __syncwarp();
    } else if (warp < 2 + P2_WW) {  // ---- weight rows into B ----
        // thread: 16-byte chunk c of rows jr + (P2_WT / 8) h of a stage
        constexpr int RSTEP = P2_WT / 8, RPT = 32 / RSTEP;  // row step, rows per thread
        const int wt = tid - 64, c = wt & 7, jr = wt >> 3;
        // the warps pass the same named barriers: after an abort they keep
        // walking the items (every wait then returns at once) instead of leaving;
        // each thread holds its share of the next item's column codes
        constexpr int NPC = MAX_ITEM_COLS / P2_WT;
        uint32_t pc[NPC];
        auto fetch = [&](const TcItem& J, bool valid) {
#pragma unroll
            for (int i = 0; i < NPC; ++i) {
                const int idx = wt + P2_WT * i;
                pc[i] = (valid && idx < J.ncol) ? __ldg(colcode + J.col0 + idx) : 0u;
            }
        };
        int g = 0, ii = 0;
        ItemIter<TcItem> X(items, nitems);
        fetch(X.cur, X.valid());
        for (; X.valid(); X.advance(), ++ii) {
            const TcItem I = X.cur;
            const int nst = (I.ncol + 31) >> 5;
            uint32_t* tab = S.code[ii & 1];
#pragma unroll
            for (int i = 0; i < NPC; ++i)
                if (wt + P2_WT * i < I.ncol) tab[wt + P2_WT * i] = pc[i];
            named_sync<1, P2_WT>();  // the table is complete (the other buffer may be refilled)
            fetch(X.nxt, X.has_next());
            for (int k = 0; k < nst; ++k, ++g) {
                const int q = g % P2_NS;
                bool ok = g < P2_NS || tc_wait(S, &S.empty[q], ((g / P2_NS) - 1) & 1, err);
                ok = __all_sync(0xffffffffu, ok && !tc_aborted(S));
                if (!ok) break;
#pragma unroll
                for (int h = 0; h < RPT; ++h) {  // row j: 128 bytes, chunks XOR-swizzled by j mod 8
                    const int jj = jr + RSTEP * h, j = k * 32 + jj;
                    const uint32_t* row = XB;
                    uint32_t bytes = 0;  // 0: zero fill
                    if (j < I.ncol) {
                        const uint32_t code = tab[j];
                        row = (code & 0x80000000u) ? T16 + (int64_t)(code & 0x7fffffffu) * NR
                                                   : XB + (int64_t)code * NR;
                        bytes = 16;
                    }
                    cp_async16(S.w[q] + jj * 128 + ((c ^ (jj & 7)) << 4), row + 4 * c, bytes);
                }
                // the stage's barrier counts this thread once its copies have landed
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&S.wfull[q]))
                             : "memory");
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");  // no copy outlives the block
    } else {  // ---- accumulators into Y ----
        const int lq = warp & 3;
        const bool odd = lane & 1;
        int ii = 0;
        for (ItemIter<TcItem> X(items, nitems); X.valid(); X.advance(), ++ii) {
            const TcItem I = X.cur;
            const int nmt = (((2 * I.ld16 + 63) >> 6) + 1) >> 1;
            const int set = ii & 1;
            if (!__all_sync(0xffffffffu, tc_wait(S, &S.accf[set], (ii >> 1) & 1, err))) break;
            tc_fence_after();
            for (int t = 0; I.ncol > 0 && t < nmt; ++t) {
                uint32_t v[64];
                tmem_ld64(tmem, lq, set * 256 + t * 64, v);
                // even lane: row m = 2r (real parts of M), odd lane: m = 2r + 1;
                // the even lane forms y_r(s) for s < 16, the odd lane for s >= 16
                float o[32];  // even: D_odd[cc]; odd: D_even[32 + cc]
#pragma unroll
                for (int cc = 0; cc < 32; ++cc)
                    o[cc] = __uint_as_float(__shfl_xor_sync(0xffffffffu, odd ? v[cc] : v[32 + cc], 1));
                const int r = (t * 128 + lq * 32 + lane) >> 1;
                if (r < I.rows) {
                    float* dst = reinterpret_cast<float*>(Y + (I.dof + r) * NR + (odd ? 16 : 0));
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float out[4];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int cc = 4 * q + 2 * h;  // 2 x (local right-hand side)
                            if (!odd) {
                                out[2 * h] = __uint_as_float(v[cc]) - o[cc + 1];
                                out[2 * h + 1] = __uint_as_float(v[cc + 1]) + o[cc];
                            } else {
                                out[2 * h] = o[cc] - __uint_as_float(v[32 + cc + 1]);
                                out[2 * h + 1] = o[cc + 1] + __uint_as_float(v[32 + cc]);
                            }
                        }
                        red_add_v4(dst + 4 * q, out[0], out[1], out[2], out[3]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.acce[set]);
        }
    }
    tc_teardown(S, P2_TMEM_COLS);
}

// Scale of every t row (s_V s_U of its block) from the uploaded V chunk
// headers; the chunks of a block in different segments write the same value.
__global__ void tscale_kernel(const DevChunk16* hdr, int64_t nchunk, float* tscale) {
    const int64_t q = blockIdx.x;
    if (q >= nchunk) return;
    const DevChunk16 ch = hdr[q];
    for (int c = threadIdx.x; c < ch.ncols; c += blockDim.x) tscale[ch.vec + c] = ch.scale * ch.fold;
}

// The gather and scatter of the block product transpose between the caller's
// column-major vectors (input order, one column per right-hand side) and the
// tree-order DOF rows of 32 right-hand sides, through a shared-memory tile of
// GS_Q consecutive input-order DOFs: each warp reads (or writes) one column
// contiguously, and each DOF's row moves whole to its tree position.
constexpr int GS_Q = 64;        // input-order DOFs per CTA
constexpr int GS_THREADS = 256;

// XB rows 2q and 2q + 1 of tree-order DOF q: (x_r, x_i) and (x_i, -x_r) of each
// right-hand side s (zero for s >= nrhs); x is column-major n x nrhs, input order.
__global__ void __launch_bounds__(GS_THREADS) gather_xb_kernel(const int64_t* iperm, const double2* x,
                                                               int64_t n, int nrhs, uint32_t* XB) {
    __shared__ float2 tile[NR][GS_Q + 1];
    const int64_t i0 = blockIdx.x * (int64_t)GS_Q;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // columns: warp w reads right-hand sides w, w + 8, ...; lanes the tile's DOFs
    for (int s = wid; s < NR; s += GS_THREADS / 32)
        for (int il = lane; il < GS_Q; il += 32) {
            const int64_t i = i0 + il;
            float2 v = make_float2(0.f, 0.f);
            if (s < nrhs && i < n) {
                const double2 u = x[(int64_t)s * n + i];
                v = make_float2((float)u.x, (float)u.y);
            }
            tile[s][il] = v;
        }
    __syncthreads();
    // rows: 32 consecutive threads write one 128-byte XB row
    for (int e = tid; e < 2 * GS_Q * NR; e += GS_THREADS) {
        const int s = e % NR, r = e / NR, il = r >> 1;
        const int64_t i = i0 + il;
        if (i >= n) continue;
        const int64_t q = tree_dof(iperm, i);
        const float2 v = tile[s][il];
        XB[(2 * q + (r & 1)) * NR + s] = (r & 1) ? pack_bf16(v.y, -v.x) : pack_bf16(v.x, v.y);
    }
}

// T16 = T rounded to bf16 pairs (the phase-2 weights of the U columns).
__global__ void t16_kernel(const float4* T, uint2* T16, int64_t npair) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npair) return;
    const float4 v = T[i];
    T16[i] = make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
}

// y (column-major n x nrhs, input order) from the tree-order rows Y[q][32].
__global__ void __launch_bounds__(GS_THREADS) scatter_multi_kernel(const int64_t* iperm, const float2* Y,
                                                                   int64_t n, int nrhs, double2* y) {
    __shared__ float2 tile[NR][GS_Q + 1];
    const int64_t i0 = blockIdx.x * (int64_t)GS_Q;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int e = tid; e < GS_Q * NR; e += GS_THREADS) {  // whole 256-byte rows
        const int s = e % NR, il = e / NR;
        const int64_t i = i0 + il;
        tile[s][il] = i < n ? Y[tree_dof(iperm, i) * NR + s] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int s = wid; s < nrhs; s += GS_THREADS / 32)
        for (int il = lane; il < GS_Q; il += 32) {
            const int64_t i = i0 + il;
            if (i >= n) continue;
            const float2 v = tile[s][il];
            y[(int64_t)s * n + i] = make_double2(v.x, v.y);
        }
}

typedef CUresult (*TmapEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TmapEncodeFn tmap_encoder() {
    static TmapEncodeFn enc = nullptr;
    if (!enc) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            hm_throw(HM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        enc = (TmapEncodeFn)fn;
    }
    return enc;
}

// 2-D BF16 view (inner extent, rows, row pitch in bytes) with 128-byte swizzle.
void encode_tmap(CUtensorMap* out, const void* base, uint64_t inner, uint64_t rows, uint64_t pitch,
                 uint32_t box_inner, uint32_t box_rows) {
    TmapEncodeFn enc = tmap_encoder();
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {box_inner, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) hm_throw(HM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
}

// The phase-2 view of the BF16 arena with leading dimension ld (complex
// entries): element (i, c, b) = bf16 64 b + i of stored column c, i.e. the
// column's 128-byte m-blocks as the outer dimension (stride 128 bytes) and the
// columns in between (stride 4 ld bytes), so that one box of 64 x 32 x nmb
// lands in shared memory as nmb blocks of 32 columns x 128 bytes (the
// MN-major operand layout).  The last m-block of a column whose 2 ld is not a
// multiple of 64 runs into the next column: those rows m >= 2 ld of A only
// reach accumulator rows that are never read.  The arena carries 256 bytes of
// slack so the last column's block stays inside the allocation.
void encode_tmap_mblocks(CUtensorMap* out, const void* base, uint64_t ld, uint64_t cols) {
    TmapEncodeFn enc = tmap_encoder();
    const uint64_t nmb = (2 * ld + 63) / 64;
    const cuuint64_t dims[3] = {64, (cuuint64_t)cols, (cuuint64_t)nmb};
    const cuuint64_t strides[2] = {(cuuint64_t)(4 * ld), 128};
    const cuuint32_t box[3] = {64, 32, (cuuint32_t)nmb};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) hm_throw(HM_ERR_CUDA, "cuTensorMapEncodeTiled failed (phase-2 view)");
}

}  // namespace

void make_block_tmaps(void* d_maps, const uint32_t* arena16, int64_t words,
                      const std::vector<int32_t>& lds, cudaStream_t st) {
    std::vector<CUtensorMap> maps(TMAP_SETS * TMAP_PER_PHASE);
    std::memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
    std::vector<char> done(TMAP_PER_PHASE, 0);
    for (const int32_t ld : lds) {
        if (ld % 4 || ld < 32 || ld > MAX_LD) hm_throw(HM_ERR_UNSUPPORTED, "BF16 leading dimension");
        if (done[ld / 4]) continue;
        done[ld / 4] = 1;
        // phase 1: 64 K x 128, 64, 32 or 16 columns; phase 2: 64 m x 32 columns x all m-blocks
        for (int z = 0; z < P1_NZ; ++z)
            encode_tmap(&maps[z * TMAP_PER_PHASE + ld / 4], arena16, 2 * ld, words / ld, 4 * ld, 64, 128 >> z);
        encode_tmap_mblocks(&maps[TMAP_PHASE2 * TMAP_PER_PHASE + ld / 4], arena16, ld, words / ld);
    }
    HM_CUDA(cudaMemcpyAsync(d_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                            cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaStreamSynchronize(st));
}

// Algorithmic bytes of one block product: the stored BF16 entries and scales,
// plus X, T and Y for NRHS_BLOCK right-hand sides (complex64 each way).
int64_t matvec_multi_alg_bytes(const MatvecDev* m, int64_t ndof) {
    if (!m->arena16) return 0;
    return 4 * (m->alg_v + m->alg_du) + 4 * (m->nchunks_v + m->nchunks_du) +
           (int64_t)NR * 8 * (2 * ndof + 2 * m->t_elems);
}

static int device_sms() {
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        HM_CUDA(cudaGetDevice(&dev));
        HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    return nsm;
}

// Phase-1 groups: per segment, the runs of V chunks that share a column
// cluster (the plan stores them contiguously, in block order); the runs of
// one cluster must agree on width and t range in every segment.  Each group
// is cut into items of at most P1_MT M tiles and, along its segments, into
// pieces of about `target` stored bytes so that the persistent CTAs get
// similar loads; items are ordered largest first.
static void make_groups(const MatvecPlan& plan, const std::vector<DevChunk16>& c16,
                        std::vector<TcGroup>& items, std::vector<TcSeg>& segs) {
    struct Run {
        int64_t sigma, seg, row, t0;
        int32_t ld16, w;
    };
    std::vector<Run> runs;
    const int64_t nseg = (int64_t)plan.col_leaf_begin.size() - 1;
    for (int64_t l = 0; l < nseg; ++l) {
        int64_t end_data = -1;
        for (int64_t q = plan.col_leaf_begin[l]; q < plan.col_leaf_begin[l + 1]; ++q) {
            const int32_t id = plan.col_items[q];
            const DevChunk16& c = c16[id];
            if (c.ncols == 0) continue;
            const int64_t sig = plan.chunks[id].sigma;
            if (!runs.empty() && runs.back().seg == l && runs.back().sigma == sig) {
                Run& r = runs.back();
                if (c.data != end_data || c.vec != r.t0 + r.w || c.ld != r.ld16)
                    hm_throw(HM_ERR_UNSUPPORTED, "column group not contiguous in the BF16 arena");
                r.w += c.ncols;
            } else {
                if (c.data % c.ld) hm_throw(HM_ERR_UNSUPPORTED, "column group not on a row of its ld view");
                runs.push_back({sig, l, c.data / c.ld, c.vec, c.ld, c.ncols});
            }
            end_data = c.data + (int64_t)c.ld * c.ncols;
        }
    }
    std::stable_sort(runs.begin(), runs.end(), [](const Run& a, const Run& b) { return a.sigma < b.sigma; });
    int64_t total = 0;
    for (const Run& r : runs) {
        if (r.row > INT32_MAX - 4096) hm_throw(HM_ERR_UNSUPPORTED, "BF16 arena above 2^31 rows of its ld view");
        total += hm_round_up(r.w, P1_BOX) * 4 * r.ld16;
    }
    const int64_t target = std::max<int64_t>(128 * 1024, total / (4 * device_sms()));
    std::vector<std::pair<int64_t, int32_t>> cost;  // (bytes, item)
    for (size_t g0 = 0; g0 < runs.size();) {
        size_t g1 = g0;
        while (g1 < runs.size() && runs[g1].sigma == runs[g0].sigma) ++g1;
        const int32_t w = runs[g0].w;
        for (size_t q = g0; q < g1; ++q)
            if (runs[q].w != w || runs[q].t0 != runs[g0].t0)
                hm_throw(HM_ERR_UNSUPPORTED, "column group differs between segments");
        for (int32_t c0 = 0; c0 < w; c0 += 128 * P1_MT) {
            const int32_t wc = std::min<int32_t>(128 * P1_MT, w - c0);
            const int64_t wpad = hm_round_up(wc, P1_BOX);
            std::vector<std::pair<size_t, size_t>> pieces;
            int64_t acc = 0;
            size_t p0 = g0;
            for (size_t q = g0; q < g1; ++q) {
                const int64_t b = wpad * 4 * runs[q].ld16;
                if (q > p0 && acc + b > target) {
                    pieces.push_back({p0, q});
                    p0 = q;
                    acc = 0;
                }
                acc += b;
            }
            pieces.push_back({p0, g1});
            for (const auto& pc : pieces) {
                TcGroup it;
                it.t0 = runs[g0].t0 + c0;
                it.ncol = wc;
                it.seg0 = (int32_t)segs.size();
                it.red = pieces.size() > 1 ? 1 : 0;
                int64_t bytes = 0;
                for (size_t q = pc.first; q < pc.second; ++q) {
                    segs.push_back({plan.leaf_dof_begin[runs[q].seg], (int32_t)(runs[q].row + c0), runs[q].ld16});
                    bytes += wpad * 4 * runs[q].ld16;
                }
                it.seg1 = (int32_t)segs.size();
                cost.push_back({bytes, (int32_t)items.size()});
                items.push_back(it);
            }
        }
        g0 = g1;
    }
    if (segs.size() > (size_t)INT32_MAX) hm_throw(HM_ERR_UNSUPPORTED, "phase-1 segment table");
    std::stable_sort(cost.begin(), cost.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<TcGroup> sorted;
    sorted.reserve(items.size());
    for (const auto& c : cost) sorted.push_back(items[c.second]);
    items.swap(sorted);
}

void make_block_items(MatvecDev* m, const MatvecPlan& plan, const std::vector<DevChunk16>& c16,
                      std::vector<DevBuf>& owner, cudaStream_t st) {
    std::vector<TcItem> t2;
    t2.reserve(m->h_items2.size());
    int64_t ncodes = 0;  // one code per phase-2 column (millions): sized once
    for (const WorkItem& w : m->h_items2)
        for (int32_t q = w.first; q < w.last; ++q) ncodes += c16[m->h_order2[q]].ncols;
    std::vector<uint32_t> codes((size_t)ncodes);
    int64_t col = 0;
    for (const WorkItem& w : m->h_items2) {
        const DevChunk16& a = c16[m->h_order2[w.first]];
        TcItem t;
        t.dof = w.dof;
        t.col0 = col;
        t.row0 = (int32_t)(a.data / a.ld);
        t.ld16 = a.ld;
        t.rows = w.rows;
        for (int32_t q = w.first; q < w.last; ++q) {
            const DevChunk16& c = c16[m->h_order2[q]];
            uint32_t* dst = codes.data() + col;
            if (c.kind != 0)
                for (int32_t j = 0; j < c.ncols; ++j) dst[j] = (uint32_t)(c.vec + j) | 0x80000000u;
            else
                for (int32_t j = 0; j < c.ncols; ++j) dst[j] = (uint32_t)(2 * (c.vec + j));
            col += c.ncols;
        }
        t.ncol = (int32_t)(col - t.col0);
        t2.push_back(t);
    }
    std::vector<TcGroup> g1;
    std::vector<TcSeg> s1;
    make_groups(plan, c16, g1, s1);
    m->ngroups1 = (int64_t)g1.size();
    m->tgroups1 = (TcGroup*)hm_dmalloc(owner, std::max<size_t>(g1.size(), 1) * sizeof(TcGroup), st, false);
    m->tsegs1 = (TcSeg*)hm_dmalloc(owner, std::max<size_t>(s1.size(), 1) * sizeof(TcSeg), st, false);
    m->tscale1 = (float*)hm_dmalloc(owner, std::max<int64_t>(m->t_elems, 1) * sizeof(float), st, false);
    m->titems2 = (TcItem*)hm_dmalloc(owner, std::max<size_t>(t2.size(), 1) * sizeof(TcItem), st, false);
    m->colcode2 = (uint32_t*)hm_dmalloc(owner, std::max<size_t>(codes.size(), 1) * 4, st, false);
    HM_CUDA(cudaMemcpyAsync(m->tgroups1, g1.data(), g1.size() * sizeof(TcGroup), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(m->tsegs1, s1.data(), s1.size() * sizeof(TcSeg), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(m->titems2, t2.data(), t2.size() * sizeof(TcItem), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemcpyAsync(m->colcode2, codes.data(), codes.size() * 4, cudaMemcpyHostToDevice, st));
    if (m->n_o1) {
        tscale_kernel<<<(unsigned)m->n_o1, 128, 0, st>>>(m->hdr16_1, m->n_o1, m->tscale1);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
    HM_CUDA(cudaStreamSynchronize(st));  // host vectors go out of scope
}

static int multi_grid(int64_t nitems) { return (int)std::min<int64_t>(nitems, device_sms()); }

static void multi_setup(MatvecDev* m, const int64_t* d_perm, int64_t n, cudaStream_t st) {
    if (m->xb) return;
    matvec_ensure_iperm(m, d_perm, n / 3, st);
    HM_CUDA(cudaFuncSetAttribute(mvc_phase1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(P1Smem) + 1024));
    HM_CUDA(cudaFuncSetAttribute(mvc_phase2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(P2Smem) + 1024));
    const int64_t nt = std::max<int64_t>(m->t_elems, 1);
    HM_CUDA(cudaMalloc((void**)&m->xb, (size_t)2 * n * NR * 4));
    HM_CUDA(cudaMalloc((void**)&m->ym, (size_t)n * NR * sizeof(float2)));
    HM_CUDA(cudaMalloc((void**)&m->tm, (size_t)nt * NR * sizeof(float2)));
    HM_CUDA(cudaMalloc((void**)&m->t16, (size_t)nt * NR * 4));
    HM_CUDA(cudaMalloc(&m->tmap_xb, sizeof(CUtensorMap)));
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    encode_tmap(&map, m->xb, 2 * NR, 2 * n, 4 * NR, 64, 64);  // 64 K rows of XB per box
    HM_CUDA(cudaMemcpyAsync(m->tmap_xb, &map, sizeof(map), cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaStreamSynchronize(st));
}

// The kernels of one block product after the gather (zeroing, both phases,
// the T16 rounding in between); events e1, e2 (may be null) mark the phases.
static void multi_phases(MatvecDev* m, int64_t n, cudaStream_t st, cudaEvent_t e1, cudaEvent_t e2) {
    if (m->t_elems) HM_CUDA(cudaMemsetAsync(m->tm, 0, (size_t)m->t_elems * NR * sizeof(float2), st));
    HM_CUDA(cudaMemsetAsync(m->ym, 0, (size_t)n * NR * sizeof(float2), st));
    if (e1) HM_CUDA(cudaEventRecord(e1, st));
    if (m->ngroups1) {
        mvc_phase1<<<multi_grid(m->ngroups1), P1_THREADS, sizeof(P1Smem) + 1024, st>>>(
            m->tgroups1, (int)m->ngroups1, m->tsegs1, m->tscale1, (const CUtensorMap*)m->tmaps,
            (const CUtensorMap*)m->tmap_xb, m->tm, m->d_err);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
    if (e2) HM_CUDA(cudaEventRecord(e2, st));
    if (m->t_elems) {
        const int64_t npair = m->t_elems * NR / 2;
        t16_kernel<<<(unsigned)hm_cdiv(npair, 256), 256, 0, st>>>((const float4*)m->tm, (uint2*)m->t16,
                                                                   npair);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
    if (m->n2) {
        mvc_phase2<<<multi_grid(m->n2), P2_THREADS, sizeof(P2Smem) + 1024, st>>>(
            m->titems2, (int)m->n2, m->colcode2, (const CUtensorMap*)m->tmaps + TMAP_PHASE2 * TMAP_PER_PHASE, m->xb,
            m->t16, m->ym, m->d_err);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
}

void matvec_multi(MatvecDev* m, const int64_t* d_perm, const double2* x, double2* y, int64_t nc,
                  int32_t nrhs, cudaStream_t st) {
    if (!m->arena16) hm_throw(HM_ERR_UNSUPPORTED, "tensor-core block product needs BF16 storage");
    const int64_t n = 3 * nc;
    multi_setup(m, d_perm, n, st);
    const unsigned nbv = (unsigned)hm_cdiv(n, GS_Q);
    for (int32_t c0 = 0; c0 < nrhs; c0 += NR) {
        const int ng = std::min<int32_t>(NR, nrhs - c0);
        gather_xb_kernel<<<nbv, GS_THREADS, 0, st>>>(m->iperm, x + (int64_t)c0 * n, n, ng, m->xb);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
        multi_phases(m, n, st, nullptr, nullptr);
        scatter_multi_kernel<<<nbv, GS_THREADS, 0, st>>>(m->iperm, m->ym, n, ng, y + (int64_t)c0 * n);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
}

// Per-kernel device times of one block product (ms: gather and zeroing,
// phase 1, T16 rounding and phase 2, scatter), averaged over reps, for the
// roofline report.
void matvec_multi_profile(MatvecDev* m, const int64_t* d_perm, const double2* x, double2* y,
                          int64_t nc, int32_t reps, double ms[4], cudaStream_t st) {
    matvec_multi(m, d_perm, x, y, nc, NR, st);  // allocations and attributes
    const int64_t n = 3 * nc;
    const unsigned nbv = (unsigned)hm_cdiv(n, GS_Q);
    cudaEvent_t ev[5];
    for (auto& e : ev) HM_CUDA(cudaEventCreate(&e));
    for (int q = 0; q < 4; ++q) ms[q] = 0.0;
    for (int r = 0; r < reps; ++r) {
        HM_CUDA(cudaEventRecord(ev[0], st));
        gather_xb_kernel<<<nbv, GS_THREADS, 0, st>>>(m->iperm, x, n, NR, m->xb);
        HM_LAUNCHED();
        multi_phases(m, n, st, ev[1], ev[2]);
        HM_CUDA(cudaEventRecord(ev[3], st));
        scatter_multi_kernel<<<nbv, GS_THREADS, 0, st>>>(m->iperm, m->ym, n, NR, y);
        HM_LAUNCHED();
        HM_CUDA(cudaEventRecord(ev[4], st));
        HM_CUDA(cudaGetLastError());
        HM_CUDA(cudaEventSynchronize(ev[4]));
        for (int q = 0; q < 4; ++q) {
            float tq = 0.f;
            HM_CUDA(cudaEventElapsedTime(&tq, ev[q], ev[q + 1]));
            ms[q] += tq / reps;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
}
