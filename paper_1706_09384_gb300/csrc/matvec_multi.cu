// matvec_multi.cu — the H-matrix product (Sec. 3.1) for a block of
// NRHS_BLOCK = 32 right-hand sides on the tensor cores, BF16 storage only.
//
// With 32 right-hand sides every stored complex entry meets 32 vector
// entries: D X and U (V^H X) become dense contractions (64 flops per stored
// byte), so the complex products run as real BF16 MMAs (mma.sync m16n8k16,
// FP32 accumulation).  A stored complex entry a = (a_r, a_i) is one bf16 pair,
// i.e. two consecutive K elements of the MMA's A operand.  The B operand
// supplies, for right-hand side s, two real columns whose K-pairs are
//   phase 2 (Y += M W):   column 2s: (w_r, -w_i)   column 2s+1: (w_i,  w_r)
//   phase 1 (T = V^H X):  column 2s: (x_r,  x_i)   column 2s+1: (x_i, -x_r)
// so the FP32 accumulators of columns 2s and 2s+1 are the real and imaginary
// parts of the complex result for right-hand side s (phase 1 conjugates V).
//
// Both phases stream the items of the BF16 arena (the chunks of one leaf, one
// contiguous column-major matrix) through a ring of shared-memory stages with
// bulk asynchronous copies, one copy per column into a padded slot so the
// fragment loads hit distinct banks.  Shared-memory traffic per stored byte
// is kept low by register blocking:
//   phase 1: K = rows of the column leaf (<= 192) is short and X is fixed per
//            item, so each consumer warp keeps its B fragments (two n-tiles,
//            all k-steps) in registers; the A tiles (16 columns of V) are read
//            with ldmatrix by the four consumer warps.
//   phase 2: M = rows of the row leaf (<= 192, 12 m-tiles), N = 64; eight
//            consumer warps each own 3 m-tiles x 4 n-tiles of the item's
//            accumulators; the per-column weights w_j = scale_j v_j of each
//            stage are converted once into a shared table.
// Vectors (tree order, right-hand side fastest): X[dof][32], T[t][32],
// Y[dof][32], complex FP32.
#include <cuda_bf16.h>

#include <algorithm>

#include "matvec_dev.cuh"
#include "pipeline.cuh"

namespace {

constexpr int NR = NRHS_BLOCK;
static_assert(NR == 32 && NR == HM_NRHS_BLOCK, "the fragment maps below assume 32 right-hand sides (8 n-tiles)");

constexpr int P1_CONS = 4;
constexpr int P1_THREADS = 32 * (P1_CONS + 1);
constexpr int P1_G = 16;               // V columns per stage: one m16 tile
constexpr int P1_NSTAGE = 3;
constexpr int P1_LDP = 196;            // largest slot stride (words): >= 192, = 4 mod 8
constexpr int P1_KMAX = MAX_LD / 8;    // k-steps of 8 complex rows

constexpr int P2_CONS = 8;
constexpr int P2_THREADS = 32 * (P2_CONS + 1);
constexpr int P2_G = 32;               // columns per stage: 4 k-steps
constexpr int P2_NSTAGE = 3;
constexpr int P2_LDP = 200;            // largest slot stride (words): >= 192, = 8 mod 16
constexpr int P2_WLD = 72;             // weight-table row stride (words), = 8 mod 32

constexpr int MV_ERR_TIMEOUT = 1;

struct P1Smem {
    alignas(128) uint32_t stage[P1_NSTAGE][P1_G * P1_LDP];
    float2 cinfo[MAX_ITEM_COLS];  // (t index bits, chunk scale)
    DevChunk16 hdr[MAX_ITEM_CHUNKS];
    int32_t colstart[MAX_ITEM_CHUNKS + 1];
    int32_t ncol;
    alignas(8) uint64_t full[P1_NSTAGE];
    uint64_t empty[P1_NSTAGE];
};
struct P2Smem {
    alignas(128) uint32_t stage[P2_NSTAGE][P2_G * P2_LDP];
    alignas(16) uint32_t wt[2][P2_G * P2_WLD];  // per-stage weights, double-buffered
    float2 cinfo[MAX_ITEM_COLS];  // (source index | kind << 31, chunk scale)
    DevChunk16 hdr[MAX_ITEM_CHUNKS];
    int32_t colstart[MAX_ITEM_CHUNKS + 1];
    int32_t ncol;
    int32_t abort;  // a consumer's wait gave up: all consumers leave after the next barrier
    alignas(8) uint64_t full[P2_NSTAGE];
    uint64_t empty[P2_NSTAGE];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return l | (h << 16);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t& r0, uint32_t& r1,
                                            uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// Headers of the item into shared memory, barriers initialised, column
// offsets of the chunks (exclusive scan), stages zeroed (slot padding is
// never written by the copies and must read as zero).
template <typename Smem, int NSTAGE, int NCONS, int THREADS>
__device__ __forceinline__ void item_prologue(Smem& S, const WorkItem& it, const DevChunk16* hdr) {
    const int nch = it.last - it.first;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < nch; i += THREADS) S.hdr[i] = hdr[it.first + i];
    uint32_t* st = &S.stage[0][0];
    constexpr int NW = (int)(sizeof(S.stage) / 4);
    for (int i = tid; i < NW; i += THREADS) st[i] = 0u;
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], NCONS);
        }
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == 0) {
        const int a0 = 2 * lane < nch ? S.hdr[2 * lane].ncols : 0;
        const int a1 = 2 * lane + 1 < nch ? S.hdr[2 * lane + 1].ncols : 0;
        int inc = a0 + a1;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const int exc = inc - a0 - a1;
        S.colstart[2 * lane] = exc;
        S.colstart[2 * lane + 1] = exc + a0;
        if (lane == 31) {
            S.colstart[MAX_ITEM_CHUNKS] = inc;
            S.ncol = inc;
        }
    }
    __syncthreads();
}

// Producer (one lane): the item's columns, G per stage, each into a slot of
// ldp words; waits for a stage to be released before refilling it and for
// its own copies before returning.
template <typename Smem, int NSTAGE, int G>
__device__ __forceinline__ void item_producer(Smem& S, const uint32_t* arena, int ldp, int* err) {
    const int ncol = S.ncol;
    const int ld16 = S.hdr[0].ld;
    const uint32_t colb = (uint32_t)ld16 * 4u;
    const int nst = (ncol + G - 1) / G;
    const uint32_t* src0 = arena + S.hdr[0].data;
    int issued = 0;
    for (int k = 0; k < nst; ++k) {
        const int s = k % NSTAGE;
        if (k >= NSTAGE && !mbar_wait(&S.empty[s], ((k / NSTAGE) - 1) & 1)) {
            atomicExch(err, MV_ERR_TIMEOUT);
            break;
        }
        const int g = min(G, ncol - k * G);
        mbar_arrive_expect_tx(&S.full[s], (uint32_t)g * colb);
        for (int c = 0; c < g; ++c)
            bulk_g2s(&S.stage[s][c * ldp], src0 + (size_t)(k * G + c) * ld16, colb, &S.full[s]);
        ++issued;
    }
    for (int k = max(0, issued - NSTAGE); k < issued; ++k)
        if (!mbar_wait(&S.full[k % NSTAGE], (k / NSTAGE) & 1)) atomicExch(err, MV_ERR_TIMEOUT);
}

// ---- phase 1: T[t_j][s] += scale_j * sum_r conj(V[r][j]) X[dof + r][s] ----
__global__ void __launch_bounds__(P1_THREADS, 3) mvm_phase1(const WorkItem* items,
                                                           const DevChunk16* hdr,
                                                           const uint32_t* __restrict__ arena,
                                                           const float2* __restrict__ X,
                                                           float2* T, int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    P1Smem& S = *reinterpret_cast<P1Smem*>(smem_raw);
    const WorkItem it = items[blockIdx.x];
    item_prologue<P1Smem, P1_NSTAGE, P1_CONS, P1_THREADS>(S, it, hdr);
    const int R = it.rows;
    const int ldp = ((R + 7) & ~7) + 4;  // = 4 mod 8: ldmatrix rows on distinct banks
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == P1_CONS) {
        if (lane == 0) item_producer<P1Smem, P1_NSTAGE, P1_G>(S, arena, ldp, err);
        return;
    }
    const int nch = it.last - it.first;
    for (int ci = warp; ci < nch; ci += P1_CONS) {
        const DevChunk16 ch = S.hdr[ci];
        for (int c = lane; c < ch.ncols; c += 32)
            S.cinfo[S.colstart[ci] + c] = make_float2(__int_as_float((int)(ch.vec + c)), ch.scale);
    }
    // B fragments of this warp's two n-tiles for every k-step, from X of the leaf
    const int g = lane >> 2, t = lane & 3;
    const int nks = (R + 7) >> 3;
    uint32_t breg[P1_KMAX][2][2];
#pragma unroll
    for (int ks = 0; ks < P1_KMAX; ++ks)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int s = (2 * warp + q) * 4 + (g >> 1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = ks * 8 + t + 4 * h;
                float2 x = make_float2(0.f, 0.f);
                if (ks < nks && r < R) x = __ldg(X + (it.dof + r) * NR + s);
                breg[ks][q][h] = (g & 1) ? pack_bf16(x.y, -x.x) : pack_bf16(x.x, x.y);
            }
        }
    named_sync<1, 32 * P1_CONS>();  // column table complete
    const int ncol = S.ncol;
    const int nst = (ncol + P1_G - 1) / P1_G;
    // ldmatrix row addresses: lanes 0-15 rows 0-15 (k 0-7), lanes 16-31 rows 0-15 (k 8-15)
    const uint32_t lane_off = (uint32_t)(((lane & 15) * ldp + 4 * (lane >> 4)) * 4);
    for (int k = 0; k < nst; ++k) {
        const int s = k % P1_NSTAGE;
        if (!mbar_wait(&S.full[s], (k / P1_NSTAGE) & 1)) {
            atomicExch(err, MV_ERR_TIMEOUT);
            break;
        }
        const uint32_t abase = smem_u32(S.stage[s]) + lane_off;
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int ks = 0; ks < P1_KMAX; ++ks) {
            if (ks < nks) {
                uint32_t a0, a1, a2, a3;
                ldmatrix_x4(abase + ks * 32, a0, a1, a2, a3);
                mma_bf16(acc[0], a0, a1, a2, a3, breg[ks][0][0], breg[ks][0][1]);
                mma_bf16(acc[1], a0, a1, a2, a3, breg[ks][1][0], breg[ks][1][1]);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[s]);
        const int jb = k * P1_G;
        const int gk = min(P1_G, ncol - jb);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int sr = (2 * warp + q) * 4 + t;
            if (g < gk) {
                const float2 ci = S.cinfo[jb + g];
                atomicAdd(T + (int64_t)__float_as_int(ci.x) * NR + sr,
                          make_float2(acc[q][0] * ci.y, acc[q][1] * ci.y));
            }
            if (g + 8 < gk) {
                const float2 ci = S.cinfo[jb + g + 8];
                atomicAdd(T + (int64_t)__float_as_int(ci.x) * NR + sr,
                          make_float2(acc[q][2] * ci.y, acc[q][3] * ci.y));
            }
        }
    }
}

// ---- phase 2: Y[dof + r][s] += sum_j M[r][j] scale_j v_j[s] ----
__global__ void __launch_bounds__(P2_THREADS, 2) mvm_phase2(const WorkItem* items,
                                                           const DevChunk16* hdr,
                                                           const uint32_t* __restrict__ arena,
                                                           const float2* __restrict__ X,
                                                           const float2* __restrict__ T,
                                                           float2* Y, int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    P2Smem& S = *reinterpret_cast<P2Smem*>(smem_raw);
    const WorkItem it = items[blockIdx.x];
    if (threadIdx.x == 0) S.abort = 0;
    item_prologue<P2Smem, P2_NSTAGE, P2_CONS, P2_THREADS>(S, it, hdr);
    const int R = it.rows;
    const int ldp = ((R + 15) & ~15) + 8;  // = 8 mod 16: fragment loads on distinct banks
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == P2_CONS) {
        if (lane == 0) item_producer<P2Smem, P2_NSTAGE, P2_G>(S, arena, ldp, err);
        return;
    }
    const int nch = it.last - it.first;
    for (int ci = warp; ci < nch; ci += P2_CONS) {
        const DevChunk16 ch = S.hdr[ci];
        const uint32_t kind = ch.kind == 0 ? 0u : 0x80000000u;
        for (int c = lane; c < ch.ncols; c += 32)
            S.cinfo[S.colstart[ci] + c] =
                make_float2(__uint_as_float((uint32_t)(ch.vec + c) | kind), ch.scale);
    }
    named_sync<1, 32 * P2_CONS>();
    const int g = lane >> 2, t = lane & 3;
    const int mt0 = warp >> 1, nt0 = 4 * (warp & 1);
    const int MT = (R + 15) >> 4;
    float acc[3][4][4];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][q][e] = 0.f;
    const int ncol = S.ncol;
    const int nst = (ncol + P2_G - 1) / P2_G;
    // weights of stage k: loaded into registers one stage ahead (the L2
    // latency hides behind the MMAs of the stage before), converted and stored
    // into the double-buffered table after those MMAs
    constexpr int WPW = P2_G / P2_CONS;  // columns per warp per stage
    float2 wv[WPW];
    float wsc[WPW];
    auto load_w = [&](int k) {
#pragma unroll
        for (int c = 0; c < WPW; ++c) {
            const int jj = warp + c * P2_CONS;
            const int j = k * P2_G + jj;
            wv[c] = make_float2(0.f, 0.f);
            wsc[c] = 0.f;
            if (k < nst && j < ncol) {
                const float2 ci = S.cinfo[j];
                const uint32_t code = __float_as_uint(ci.x);
                const float2* src = (code & 0x80000000u) ? T : X;
                wv[c] = __ldg(src + (int64_t)(code & 0x7fffffffu) * NR + lane);
                wsc[c] = ci.y;
            }
        }
    };
    auto store_w = [&](int k) {
        uint32_t* wt = S.wt[k & 1];
#pragma unroll
        for (int c = 0; c < WPW; ++c) {
            const int jj = warp + c * P2_CONS;
            const float wr = wv[c].x * wsc[c], wi = wv[c].y * wsc[c];
            *reinterpret_cast<uint2*>(wt + jj * P2_WLD + 2 * lane) =
                make_uint2(pack_bf16(wr, -wi), pack_bf16(wi, wr));
        }
    };
    load_w(0);
    store_w(0);
    for (int k = 0; k < nst; ++k) {
        const int s = k % P2_NSTAGE;
        const int jb = k * P2_G;
        const int gk = min(P2_G, ncol - jb);
        if (!mbar_wait(&S.full[s], (k / P2_NSTAGE) & 1)) {
            atomicExch(err, MV_ERR_TIMEOUT);
            *(volatile int32_t*)&S.abort = 1;
        }
        named_sync<1, 32 * P2_CONS>();  // weights of stage k visible; stage k-1 done everywhere
        if (*(volatile int32_t*)&S.abort) break;  // same decision in every consumer warp
        load_w(k + 1);
        const uint32_t* wt = S.wt[k & 1];
        const uint32_t* sb = S.stage[s];
#pragma unroll
        for (int ks = 0; ks < P2_G / 8; ++ks) {
            const int j0 = ks * 8;
            if (j0 < gk) {
                uint32_t b[4][2];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int n = (nt0 + q) * 8 + g;
                    b[q][0] = wt[(j0 + t) * P2_WLD + n];
                    b[q][1] = wt[(j0 + t + 4) * P2_WLD + n];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int mt = mt0 + 4 * i;
                    if (mt < MT) {
                        const int r = mt * 16 + g;
                        const uint32_t a0 = sb[(j0 + t) * ldp + r];
                        const uint32_t a1 = sb[(j0 + t) * ldp + r + 8];
                        const uint32_t a2 = sb[(j0 + t + 4) * ldp + r];
                        const uint32_t a3 = sb[(j0 + t + 4) * ldp + r + 8];
#pragma unroll
                        for (int q = 0; q < 4; ++q) mma_bf16(acc[i][q], a0, a1, a2, a3, b[q][0], b[q][1]);
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[s]);
        if (k + 1 < nst) store_w(k + 1);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int mt = mt0 + 4 * i;
        if (mt >= MT) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int sr = (nt0 + q) * 4 + t;
            const int r0 = mt * 16 + g;
            if (r0 < R) atomicAdd(Y + (it.dof + r0) * NR + sr, make_float2(acc[i][q][0], acc[i][q][1]));
            if (r0 + 8 < R)
                atomicAdd(Y + (it.dof + r0 + 8) * NR + sr, make_float2(acc[i][q][2], acc[i][q][3]));
        }
    }
}

// ---- phase 2 on the tcgen05 tensor cores (accumulators in TMEM) ----
// The item's rows are the MMA's M (up to two tiles of 128), the 64 real output
// columns its N, the complex columns (as bf16 pairs) its K.  Per stage of 16
// complex columns (K = 32) the consumer warps load the BF16 columns from the
// arena (16-byte loads, four columns by four rows per thread) and store them
// transposed into K-major core matrices (8 rows x 16 bytes, no swizzle; core
// groups 16 bytes apart beyond their 4 x 128 bytes so the 16-byte stores of
// one warp hit distinct banks), build the weights w_j = scale_j v_j as the B
// operand in the same layout, and signal the MMA warp; one thread issues the
// tcgen05.mma instructions into two TMEM accumulator tiles and commits each
// stage to an mbarrier that releases its buffers.  At the end the consumers
// read the accumulators back with tcgen05.ld.  Shared-memory descriptors:
// start >> 4, leading (K-direction core) byte offset 128, stride (8-row
// group) byte offset T2_SBO, version 1, no swizzle.
constexpr int T2_CONS = 8;
constexpr int T2_THREADS = 32 * (T2_CONS + 1);  // + the MMA warp
constexpr int T2_KC = 16;                        // complex columns per stage
constexpr int T2_SBO = 4 * 128 + 16;             // bytes between 8-row core groups
constexpr int T2_ATILE = 16 * T2_SBO;            // 128 rows
constexpr int T2_BBYTES = 8 * T2_SBO;            // 64 rows (real output columns)
constexpr uint32_t T2_TMEM_COLS = 128;           // two 128 x 64 FP32 accumulators
// kind::f16: FP32 accumulate (bit 4), A and B BF16 (bits 7, 10), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t T2_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(64 >> 3) << 17) |
                              (uint32_t(128 >> 4) << 24);

struct T2Smem {
    alignas(128) unsigned char a[2][2][T2_ATILE];  // [slot][m tile]
    alignas(128) unsigned char b[2][T2_BBYTES];    // [slot]
    float2 cinfo[MAX_ITEM_COLS];                    // (source index | kind << 31, chunk scale)
    DevChunk16 hdr[MAX_ITEM_CHUNKS];
    int32_t colstart[MAX_ITEM_CHUNKS + 1];
    int32_t ncol;
    int32_t abort;
    uint32_t tmem;
    alignas(8) uint64_t ready[2];  // consumer warps -> MMA thread: slot filled
    uint64_t done[2];              // MMA thread (tcgen05.commit) -> consumers: slot consumed
};
static_assert(sizeof(T2Smem) <= 56 * 1024, "four CTAs per SM");

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(T2_SBO >> 4) << 32) | ((uint64_t)1 << 46);
}

__global__ void __launch_bounds__(T2_THREADS, 4) mvt_phase2(const WorkItem* items,
                                                           const DevChunk16* hdr,
                                                           const uint32_t* __restrict__ arena,
                                                           const float2* __restrict__ X,
                                                           const float2* __restrict__ T,
                                                           float2* Y, int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T2Smem& S = *reinterpret_cast<T2Smem*>(smem_raw);
    const WorkItem it = items[blockIdx.x];
    const int nch = it.last - it.first;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < nch; i += T2_THREADS) S.hdr[i] = hdr[it.first + i];
    if (tid == 0) {
        S.abort = 0;
        for (int q = 0; q < 2; ++q) {
            mbar_init(&S.ready[q], T2_CONS);
            mbar_init(&S.done[q], 1);
        }
        mbar_fence_init();
    }
    if (warp == T2_CONS) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem)),
                     "r"(T2_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) {  // column offsets of the chunks (exclusive scan)
        const int a0 = 2 * lane < nch ? S.hdr[2 * lane].ncols : 0;
        const int a1 = 2 * lane + 1 < nch ? S.hdr[2 * lane + 1].ncols : 0;
        int inc = a0 + a1;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const int exc = inc - a0 - a1;
        S.colstart[2 * lane] = exc;
        S.colstart[2 * lane + 1] = exc + a0;
        if (lane == 31) {
            S.colstart[MAX_ITEM_CHUNKS] = inc;
            S.ncol = inc;
        }
    }
    __syncthreads();
    for (int ci = warp; ci < nch; ci += T2_CONS + 1) {
        const DevChunk16 ch = S.hdr[ci];
        const uint32_t kind = ch.kind == 0 ? 0u : 0x80000000u;
        for (int c = lane; c < ch.ncols; c += 32)
            S.cinfo[S.colstart[ci] + c] =
                make_float2(__uint_as_float((uint32_t)(ch.vec + c) | kind), ch.scale);
    }
    __syncthreads();
    const int R = it.rows;
    const int MT = R > 128 ? 2 : 1;
    const int ncol = S.ncol;
    const int nst = (ncol + T2_KC - 1) / T2_KC;
    const uint32_t tmem = S.tmem;
    if (warp == T2_CONS) {  // ---- MMA issue ----
        if (lane == 0) {
            int issued = -1;
            for (int k = 0; k < nst; ++k) {
                const int slot = k & 1;
                if (!mbar_wait(&S.ready[slot], (k >> 1) & 1)) {
                    atomicExch(err, MV_ERR_TIMEOUT);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sb = smem_u32(S.b[slot]);
                for (int t = 0; t < MT; ++t) {
                    const uint32_t sa = smem_u32(S.a[slot][t]);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t da = umma_desc(sa + kk * 256), db = umma_desc(sb + kk * 256);
                        const uint32_t acc = (k > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                tmem + (uint32_t)(t * 64)),
                            "l"(da), "l"(db), "r"(T2_IDESC), "r"(acc));
                    }
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&S.done[slot]))
                    : "memory");
                issued = k;
            }
            if (issued >= 0 && !mbar_wait(&S.done[issued & 1], (issued >> 1) & 1))
                atomicExch(err, MV_ERR_TIMEOUT);  // own MMAs complete before the buffers go
        }
        __syncwarp();
    } else {  // ---- consumers: operands in, accumulators out ----
        const int RQ = (R + 3) >> 2;  // row quads (ld16 = 4 RQ)
        const int ld16 = S.hdr[0].ld;
        const uint32_t* src0 = arena + S.hdr[0].data;
        const int task = tid;  // (column group cg, row quad q), q fastest
        const int cg = task / RQ, q = task - cg * RQ;
        const bool has_task = task < 4 * RQ;
        uint4 u[4];
        auto load_a = [&](int k) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = k * T2_KC + 4 * cg + c;
                u[c] = (has_task && k < nst && j < ncol)
                           ? __ldcs(reinterpret_cast<const uint4*>(src0 + (size_t)j * ld16) + q)
                           : make_uint4(0, 0, 0, 0);
            }
        };
        float2 wv[2];
        float wsc[2];
        auto load_w = [&](int k) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int j = k * T2_KC + warp + c * T2_CONS;
                wv[c] = make_float2(0.f, 0.f);
                wsc[c] = 0.f;
                if (k < nst && j < ncol) {
                    const float2 ci = S.cinfo[j];
                    const uint32_t code = __float_as_uint(ci.x);
                    const float2* src = (code & 0x80000000u) ? T : X;
                    wv[c] = __ldg(src + (int64_t)(code & 0x7fffffffu) * NR + lane);
                    wsc[c] = ci.y;
                }
            }
        };
        load_a(0);
        load_w(0);
        for (int k = 0; k < nst; ++k) {
            const int slot = k & 1;
            if (k >= 2 && !mbar_wait(&S.done[slot], ((k >> 1) - 1) & 1)) {
                atomicExch(err, MV_ERR_TIMEOUT);
                *(volatile int32_t*)&S.abort = 1;
            }
            if (__any_sync(0xffffffffu, *(volatile int32_t*)&S.abort)) break;  // warp-uniform
            // A: rows 4q..4q+3 of columns 4cg..4cg+3, transposed into four 16-byte rows
            if (has_task) {
                const uint32_t* w = reinterpret_cast<const uint32_t*>(u);  // w[4 c + i]: column c, row i
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = 4 * q + i;
                    const int t = r >> 7, rr = r & 127;
                    if (t < MT) {
                        unsigned char* dst = S.a[slot][t] + (rr >> 3) * T2_SBO + cg * 128 + (rr & 7) * 16;
                        *reinterpret_cast<uint4*>(dst) = make_uint4(w[i], w[4 + i], w[8 + i], w[12 + i]);
                    }
                }
            }
            // B: w_j as (w_r, -w_i) for real column 2s and (w_i, w_r) for 2s + 1
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int j = warp + c * T2_CONS;  // stage-local column
                const float wr = wv[c].x * wsc[c], wi = wv[c].y * wsc[c];
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    const int n = 2 * lane + v;
                    const uint32_t word = v == 0 ? pack_bf16(wr, -wi) : pack_bf16(wi, wr);
                    *reinterpret_cast<uint32_t*>(S.b[slot] + (n >> 3) * T2_SBO + (j >> 2) * 128 +
                                                 (n & 7) * 16 + (j & 3) * 4) = word;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.ready[slot]);
            load_a(k + 1);
            load_w(k + 1);
        }
        // every stage's MMAs done: accumulators to Y
        const int last = nst - 1;
        bool ok = last >= 0 && !*(volatile int32_t*)&S.abort;
        if (ok && !mbar_wait(&S.done[last & 1], (last >> 1) & 1)) {
            atomicExch(err, MV_ERR_TIMEOUT);
            ok = false;
        }
        ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int t = warp >> 2, lg = warp & 3;
        if (ok && t < MT) {
            const int r = t * 128 + lg * 32 + lane;
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                      "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                      "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(t * 64 + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (r < R) {
#pragma unroll
                    for (int e = 0; e < 16; e += 2)  // real columns 2s, 2s + 1: RHS s
                        atomicAdd(Y + (it.dof + r) * NR + (c0 + e) / 2,
                                  make_float2(__uint_as_float(v[e]), __uint_as_float(v[e + 1])));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == T2_CONS)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(T2_TMEM_COLS));
}

// X[(3p + a) * 32 + s] = x_s[3 perm[p] + a]  (zero for s >= nrhs)
__global__ void gather_multi_kernel(const int64_t* perm, const double2* x, int64_t n, int nrhs,
                                    float2* X, int64_t nc) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= 3 * nc * NR) return;
    const int64_t q = idx / NR;
    const int s = (int)(idx - q * NR);
    float2 v = make_float2(0.f, 0.f);
    if (s < nrhs) {
        const int64_t p = q / 3, a = q - 3 * p;
        const double2 u = x[(int64_t)s * n + 3 * perm[p] + a];
        v = make_float2((float)u.x, (float)u.y);
    }
    X[idx] = v;
}

__global__ void scatter_multi_kernel(const int64_t* perm, const float2* Y, int64_t n, int nrhs,
                                     double2* y, int64_t nc) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= 3 * nc * NR) return;
    const int64_t q = idx / NR;
    const int s = (int)(idx - q * NR);
    if (s >= nrhs) return;
    const int64_t p = q / 3, a = q - 3 * p;
    const float2 v = Y[idx];
    y[(int64_t)s * n + 3 * perm[p] + a] = make_double2(v.x, v.y);
}

static_assert(sizeof(P1Smem) <= 113 * 1024, "phase 1: two CTAs per SM");
static_assert(sizeof(P2Smem) <= 113 * 1024, "phase 2: two CTAs per SM");

}  // namespace

static void launch_phase2(MatvecDev* m, cudaStream_t st) {
    if (m->phase2_tc)
        mvt_phase2<<<(unsigned)m->n2, T2_THREADS, sizeof(T2Smem), st>>>(
            m->items2, m->hdr16_2, m->arena16, m->xm, m->tm, m->ym, m->d_err);
    else
        mvm_phase2<<<(unsigned)m->n2, P2_THREADS, sizeof(P2Smem), st>>>(
            m->items2, m->hdr16_2, m->arena16, m->xm, m->tm, m->ym, m->d_err);
}

// Algorithmic bytes of one block product: the stored BF16 entries and scales,
// plus X, T and Y for NRHS_BLOCK right-hand sides (complex64 each way).
int64_t matvec_multi_alg_bytes(const MatvecDev* m, int64_t ndof) {
    if (!m->arena16) return 0;
    return 4 * (m->alg_v + m->alg_du) + 4 * (m->nchunks_v + m->nchunks_du) +
           (int64_t)NR * 8 * (2 * ndof + 2 * m->t_elems);
}

void matvec_multi(MatvecDev* m, const int64_t* d_perm, const double2* x, double2* y, int64_t nc,
                  int32_t nrhs, cudaStream_t st) {
    if (!m->arena16) hm_throw(HM_ERR_UNSUPPORTED, "tensor-core block product needs BF16 storage");
    const int64_t n = 3 * nc;
    if (!m->xm) {
        HM_CUDA(cudaFuncSetAttribute(mvm_phase1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(P1Smem)));
        HM_CUDA(cudaFuncSetAttribute(mvm_phase2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(P2Smem)));
        HM_CUDA(cudaFuncSetAttribute(mvt_phase2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(T2Smem)));
        // phase 2 on tcgen05 unless HM_BLOCK_PHASE2=mma asks for the mma.sync kernel
        const char* e = getenv("HM_BLOCK_PHASE2");
        m->phase2_tc = (e && e[0] == 'm') ? 0 : 1;
        HM_CUDA(cudaMalloc((void**)&m->xm, (size_t)n * NR * sizeof(float2)));
        HM_CUDA(cudaMalloc((void**)&m->ym, (size_t)n * NR * sizeof(float2)));
        HM_CUDA(cudaMalloc((void**)&m->tm, (size_t)std::max<int64_t>(m->t_elems, 1) * NR * sizeof(float2)));
    }
    const unsigned nbv = (unsigned)hm_cdiv(n * NR, 256);
    for (int32_t c0 = 0; c0 < nrhs; c0 += NR) {
        const int ng = std::min<int32_t>(NR, nrhs - c0);
        gather_multi_kernel<<<nbv, 256, 0, st>>>(d_perm, x + (int64_t)c0 * n, n, ng, m->xm, nc);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
        if (m->t_elems) HM_CUDA(cudaMemsetAsync(m->tm, 0, (size_t)m->t_elems * NR * sizeof(float2), st));
        HM_CUDA(cudaMemsetAsync(m->ym, 0, (size_t)n * NR * sizeof(float2), st));
        if (m->n1) {
            mvm_phase1<<<(unsigned)m->n1, P1_THREADS, sizeof(P1Smem), st>>>(
                m->items1, m->hdr16_1, m->arena16, m->xm, m->tm, m->d_err);
            HM_CUDA(cudaGetLastError());
            HM_LAUNCHED();
        }
        if (m->n2) {
            launch_phase2(m, st);
            HM_CUDA(cudaGetLastError());
            HM_LAUNCHED();
        }
        scatter_multi_kernel<<<nbv, 256, 0, st>>>(d_perm, m->ym, n, ng, y + (int64_t)c0 * n, nc);
        HM_CUDA(cudaGetLastError());
        HM_LAUNCHED();
    }
}

// Per-kernel device times of one block product (ms: gather, phase 1, phase 2,
// scatter), averaged over reps, for the roofline report.
void matvec_multi_profile(MatvecDev* m, const int64_t* d_perm, const double2* x, double2* y,
                          int64_t nc, int32_t reps, double ms[4], cudaStream_t st) {
    matvec_multi(m, d_perm, x, y, nc, NR, st);  // allocations and attributes
    const int64_t n = 3 * nc;
    const unsigned nbv = (unsigned)hm_cdiv(n * NR, 256);
    cudaEvent_t ev[5];
    for (auto& e : ev) HM_CUDA(cudaEventCreate(&e));
    for (int q = 0; q < 4; ++q) ms[q] = 0.0;
    for (int r = 0; r < reps; ++r) {
        HM_CUDA(cudaEventRecord(ev[0], st));
        gather_multi_kernel<<<nbv, 256, 0, st>>>(d_perm, x, n, NR, m->xm, nc);
        HM_LAUNCHED();
        if (m->t_elems) HM_CUDA(cudaMemsetAsync(m->tm, 0, (size_t)m->t_elems * NR * sizeof(float2), st));
        HM_CUDA(cudaMemsetAsync(m->ym, 0, (size_t)n * NR * sizeof(float2), st));
        HM_CUDA(cudaEventRecord(ev[1], st));
        if (m->n1) {
            mvm_phase1<<<(unsigned)m->n1, P1_THREADS, sizeof(P1Smem), st>>>(
                m->items1, m->hdr16_1, m->arena16, m->xm, m->tm, m->d_err);
            HM_LAUNCHED();
        }
        HM_CUDA(cudaEventRecord(ev[2], st));
        if (m->n2) {
            launch_phase2(m, st);
            HM_LAUNCHED();
        }
        HM_CUDA(cudaEventRecord(ev[3], st));
        scatter_multi_kernel<<<nbv, 256, 0, st>>>(d_perm, m->ym, n, NR, y, nc);
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
