// matvec_dev.cuh — device-side layout of the stored H-matrix shared by the
// product kernels (matvec.cu: one right-hand side; matvec_multi.cu: blocks of
// right-hand sides on the tensor cores).
#pragma once
#include <vector>

#include "hm_internal.h"

constexpr int MAX_LD = 192;               // 3 * 64 rows: storage segments of up to 64 points
constexpr int MAX_ITEM_CHUNKS = 64;       // chunk headers staged in shared memory per item
constexpr int MAX_ITEM_COLS = 1024;       // columns of one item (per-column table in smem)

struct DevChunk {
    int64_t data;   // arena element offset
    int64_t vec;    // x (kind 0) or t (kind 1/2) element offset
    int32_t ld;
    int32_t ncols;
    int32_t kind;
    int32_t rows;
};
// Chunk of the BF16 arena: complex entries as two bf16 (4 bytes), to be
// multiplied by an FP32 scale (one per block and factor for U and V, 1 for
// dense blocks); rows padded to a multiple of 4 (16-byte columns), at least 32.
struct DevChunk16 {
    int64_t data;   // element offset in arena16
    int64_t vec;
    int32_t ld;
    int32_t ncols;
    int32_t kind;
    int32_t rows;
    float scale;
    float fold;     // V chunks: the U scale of the same block; otherwise 1
};
struct WorkItem {
    int64_t dof;      // first tree-order DOF of the segment
    int32_t rows;     // 3 |segment|
    int32_t ld;
    int32_t first;    // chunk ids [first, last)
    int32_t last;
};

// Work item of the tensor-core block product (one segment's chunks, contiguous
// in the BF16 arena, starting on a row of the arena's ld16 view).
struct TcItem {
    int64_t dof;    // first tree-order DOF of the segment
    int64_t col0;   // first entry of the item in the per-column table
    int32_t row0;   // first row of the item in the ld16 view (data / ld16)
    int32_t ld16;
    int32_t ncol;
    int32_t rows;   // 3 |segment|
};

// Phase-1 work item of the tensor-core block product: columns [c0, c0 + ncol)
// of one column-cluster group (the V columns of every block that shares the
// column cluster sigma, t rows t0 - c0 ...) over the segments [seg0, seg1) of
// sigma (all of them unless the group is cut along K; red then says that
// other items add into the same t rows).
struct TcGroup {
    int64_t t0;     // t row of column c0
    int32_t ncol;   // <= 512 (four 128-column M tiles)
    int32_t seg0;   // entries [seg0, seg1) of the segment table
    int32_t seg1;
    int32_t red;    // 1: add into T (zeroed before), 0: store
};
// One segment of a phase-1 item: row of the item's first column in the
// segment's ld16 view of the BF16 arena, its ld16, and its first DOF.
struct TcSeg {
    int64_t dof;
    int32_t row0;
    int32_t ld16;
};

struct MatvecDev {
    int storage = 0;
    int s16_nstage = 3;                 // stages of the streamed BF16 kernels (2, 3 or 4; the
                                        // autotuner may change it)
    int64_t item_bytes = 256 * 1024;    // target FP32 bytes of a work item (set from the
                                        // operator's size at creation)
    std::vector<DevChunk> dc;           // chunk headers in plan order (host)
    std::vector<DevBuf> tile_bufs;      // items, orders and headers of the current tiling
    // the full item lists of the tiling, and buffers for a subset of them (a
    // joined batch whose converged problems are left out of the products)
    WorkItem* items1_full = nullptr;
    WorkItem* items2_full = nullptr;
    int64_t n1_full = 0, n2_full = 0;
    WorkItem* sel1 = nullptr;
    WorkItem* sel2 = nullptr;
    float2* arena = nullptr;
    int64_t arena_elems = 0;
    DevChunk* chunks = nullptr;
    WorkItem* items1 = nullptr;   // phase 1 (V)
    WorkItem* items2 = nullptr;   // phase 2 (dense + U)
    int32_t* order1 = nullptr;    // chunk ids referenced by items, phase 1
    int32_t* order2 = nullptr;
    DevChunk* hdr1 = nullptr;     // chunk headers in item order (phase 1, phase 2)
    DevChunk* hdr2 = nullptr;
    DevChunk16* hdr16_1 = nullptr;
    DevChunk16* hdr16_2 = nullptr;
    int64_t n_o1 = 0, n_o2 = 0;
    int64_t n1 = 0, n2 = 0;
    float2* t = nullptr;
    double2* t64 = nullptr;       // accurate product: t in FP64
    int64_t t_elems = 0;
    int64_t dense_elems = 0;
    int64_t lr_elems = 0;
    int64_t alg_v = 0;      // stored entries (rows x cols, no padding) of V chunks
    int64_t alg_du = 0;     // ... of dense and U chunks
    // BF16 copy of the arena (HM_STORE_BF16): the fast product reads it; the
    // FP32 arena stays for the accurate product
    uint32_t* arena16 = nullptr;
    int64_t arena16_elems = 0;
    DevChunk16* chunks16 = nullptr;
    int64_t nchunks = 0;
    int64_t nchunks_v = 0, nchunks_du = 0;  // scale counts for the byte model
    // CUDA graph of one whole product (gather, both phases, scatter), captured
    // on first use; x and y are re-pointed in the instantiated graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t g_gather = nullptr, g_scatter = nullptr;
    const double2* g_x = nullptr;
    double2* g_y = nullptr;
    long long g_kernels = 0;
    int* d_err = nullptr;             // error code written by the streamed kernels
    std::vector<WorkItem> h_items1, h_items2;
    std::vector<int32_t> h_order1, h_order2;
    // block of NRHS_BLOCK right-hand sides (tensor-core product), allocated on
    // first use: XB bf16 rows (x, -i x) per DOF, Y and T in FP32, T16 = bf16(T)
    uint32_t* xb = nullptr;
    float2* ym = nullptr;
    int64_t* iperm = nullptr;  // tree position of each input-order point
    float2* tm = nullptr;
    uint32_t* t16 = nullptr;
    // TMA descriptors (CUtensorMap, 128 bytes each): the BF16 arena viewed as
    // rows of 2 ld16 bf16, [set][ld16 / 4] (TMAP_SETS sets); and XB
    void* tmaps = nullptr;
    void* tmap_xb = nullptr;
    // tensor-core items and tables: phase 1 groups, their segments and the
    // scale s_V s_U of every t row; phase 2 items and per-column codes
    // (T16 row | 1 << 31 for U columns, XB row 2 dof for dense ones)
    TcGroup* tgroups1 = nullptr;
    int64_t ngroups1 = 0;
    TcSeg* tsegs1 = nullptr;
    float* tscale1 = nullptr;
    TcItem* titems2 = nullptr;
    uint32_t* colcode2 = nullptr;
};
constexpr int TMAP_PER_PHASE = MAX_LD / 4 + 1;
// descriptor sets: phase 1 with boxes of 128, 64, 32 and 16 rows, then phase 2
constexpr int TMAP_PHASE2 = 4;
constexpr int TMAP_SETS = 5;
// Items and per-column tables of the tensor-core block product (after the
// BF16 chunks, headers and scales exist on the device); c16 as uploaded.
void make_block_items(MatvecDev* m, const MatvecPlan& plan, const std::vector<DevChunk16>& c16,
                      std::vector<DevBuf>& owner, cudaStream_t st);
// Encodes the descriptors for the leading dimensions in lds (device copy at
// d_maps, TMAP_SETS * TMAP_PER_PHASE entries); defined with the block product.
void make_block_tmaps(void* d_maps, const uint32_t* arena16, int64_t words,
                      const std::vector<int32_t>& lds, cudaStream_t st);

// Block of NRHS_BLOCK right-hand sides for the tensor-core product (created on
// first use; tree-order vectors, right-hand side fastest: v[dof * NRHS_BLOCK + s]).
constexpr int NRHS_BLOCK = 32;

// m->iperm (the tree position of each input-order point) from the handle's
// permutation, computed on first use.
void matvec_ensure_iperm(MatvecDev* m, const int64_t* d_perm, int64_t nc, cudaStream_t st);
// Tree-order DOF of input-order DOF i.
__device__ __forceinline__ int64_t tree_dof(const int64_t* iperm, int64_t i) {
    const int64_t p = i / 3;
    return 3 * iperm[p] + (i - 3 * p);
}
