// spnn_internal.cuh -- launch parameter blocks shared by the surrogate's GEMM
// kernels (spnn_gemm.cu) and its C ABI / runtime (spnn_api.cu).
//
// Activation layout ("chunk planes"): BF16 [C/8][B][D][H][W][8].  One plane
// holds 8 channels of every voxel, 16 bytes per voxel, so a run of voxels
// along x is contiguous and a TMA box row spans up to 32 voxels (512 bytes);
// in shared memory a box lands as rows of 16 bytes, the no-swizzle core
// matrix layout the tensor cores read.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace spnn {

enum { KIND_CONV3 = 0, KIND_DOWN = 1, KIND_UP = 2 };
// How the row-GEMM producer finds the A chunk for (tap, channel chunk):
//   TAP_SHIFT3 conv3 taps: coordinates shifted by the tap, map 0 / 1 = the two
//              concatenated sources;
//   TAP_MAP    one map per tap (strided views), no shift;
//   TAP_NONE   a single tap, no shift, maps 0 / 1 as for TAP_SHIFT3.
enum { TAP_SHIFT3 = 0, TAP_MAP = 1, TAP_NONE = 2 };
enum { ERR_TIMEOUT = 1 };

constexpr int kRows = 128;                 // GEMM rows per CTA (MMA M)
constexpr int kThreads = 192;              // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Tiles of a voxel grid: boxes of bx * by * bz * bb voxels (x fastest), nx *
// ny * nz boxes per sample block; tile t -> box origin, row r -> voxel.
struct TileGrid {
    int B, D, H, W;
    int bx, by, bz, bb;
    int nx, ny, nz;
};

__host__ __device__ inline void tile_origin(const TileGrid& g, long long t, int& x0, int& y0, int& z0, int& b0) {
    x0 = (int)(t % g.nx) * g.bx;
    t /= g.nx;
    y0 = (int)(t % g.ny) * g.by;
    t /= g.ny;
    z0 = (int)(t % g.nz) * g.bz;
    b0 = (int)(t / g.nz) * g.bb;
}

// Linear voxel index ((b D + z) H + y) W + x of row r of the tile at (x0, y0, z0, b0).
__host__ __device__ inline long long row_voxel(const TileGrid& g, int x0, int y0, int z0, int b0, int r,
                                               int* vx, int* vy, int* vz, int* vb) {
    const int x = x0 + r % g.bx;
    r /= g.bx;
    const int y = y0 + r % g.by;
    r /= g.by;
    const int z = z0 + r % g.bz;
    const int b = b0 + r / g.bz;
    *vx = x, *vy = y, *vz = z, *vb = b;
    return (((long long)b * g.D + z) * g.H + y) * g.W + x;
}

struct EpiDest {
    __nv_bfloat16* out;             // BF16 chunk-plane destination (may be null)
    const __nv_bfloat16* addend;    // added before the activation (same addressing), or null
    const __nv_bfloat16* mask;      // result zeroed where mask <= 0 (same addressing), or null
    const float* bias;              // per destination channel, or null
    long long plane;                // elements per chunk plane of the destination (voxels * 8)
    int col0;                       // first GEMM column that lands in this destination
    int relu;
};

// Rows GEMM: D[row, n] = sum_k A[row, k] B[n, k]; rows are the 128 voxels of
// one box of the row grid, k = (tap, channel), A gathered by TMA boxes from
// chunk-plane maps (coordinates 8x, y, z, b, c8) or, for TAP_MAP, stride-2
// views (coordinates 0, x, y, z, c8 * B + b).
//
// conv3 (TAP_SHIFT3) K-steps are (x-shift dx, block of E chunk planes): with
// `halo` set the tile is one z-plane and a single box of (bx, by + 2, 3)
// voxels holds all nine (dz, dy) taps, each a descriptor offset into it;
// otherwise nine boxes of the tile's own shape are loaded.  Other modes step
// over (tap, kc_step chunk planes).
struct RowsParams {
    CUtensorMap maps[8];
    const __nv_bfloat16* wpack;     // packed operand, layout per kind (see the packing kernel)
    int n_taps, kc_total, kc0, kc_step, tap_mode;
    int halo, E;                    // conv3 only: halo 0 per-tap boxes, 1 one box per x-shift,
                                    // 2 one box for all 27 taps (bx = 8 tiles)
    uint32_t halo_plane;            // bytes of one chunk plane of the halo box
    int mt;                         // 128-row subtiles per CTA, stacked along y (halo mode), else 1
    TileGrid g;                     // CTA boxes: 128 * mt voxels each
    int n_tile, n_total, ksteps, stages;
    int tiles;                      // CTA boxes of the grid; persistent CTAs claim them in order
    int* tile_ctr;                  // [grid_n] claim counters, zero at launch
    int persistent;                 // k >= 1: k x SMs x resident CTAs; 0: one CTA per tile
    int nbuf;                       // TMEM accumulator buffers (2: epilogue overlaps the next tile)
    uint32_t a_stage_bytes, b_stage_bytes, stage_bytes;
    uint32_t idesc;
    int scatter_up, cout_up, split;
    EpiDest d[2];
    float* head_out;                // fused one-channel head: out = head_b + sum_c y_c head_w[c]
    const float* head_w;
    const float* head_b;
    int* err;
};

// Weight-gradient GEMM: D[(group, r), n] = sum_v A_group[v, r] B[v, n] over a
// range of 64-voxel K-steps (boxes of the V grid); rows are 16 groups of 8
// input channels (one tap each), both operands MN-major, results added to
// FP32 dW with atomics.  A maps are stride-2 views for KIND_DOWN, B maps for
// KIND_UP; all others are chunk-plane maps.
struct WgradParams {
    CUtensorMap amaps[8];
    CUtensorMap bmaps[8];
    int mode;                       // KIND_*
    int kc_total, kc0, n_groups, ones_group;
    int kv;                         // voxels per K-step (64 or 128): a group's block is kv * 16 bytes
    int ea, eb;                     // chunk planes per A / B box (1 for stride-2 views)
    TileGrid g;
    int ksteps_total, ksteps_per_cta, n, stages;
    uint32_t a_stage_bytes, b_stage_bytes, stage_bytes;
    uint32_t idesc;
    float* dw;                      // [taps][kc_total * 8][n]
    float* db;                      // [n]
    int* err;
};

// conv3 weight gradient with halo K-steps: dW[tap][ci][co] = sum_v
// X[v + tap][ci] dY[v][co], summed as sum_u X[u][ci] dY[u - d][co].  Each
// K-step is one x-run of rl (16 or 32) voxels u.  A (MN-major): one TMA box of
// the input, (rl x 3 x 3) voxels of npc chunk planes laid out [plane][dz][dy][x],
// so the row groups (plane, dz, dy) sit one run (16 rl bytes) apart; row group
// 9 npc is a row of ones (bias gradient).  B (MN-major): three boxes of dY, at x - dx for dx =
// -1, 0, 1, side by side, so one MMA has N = 3 n columns (dx, co) and no
// operand needs an x-halo.  blockIdx.y splits the planes (npc per CTA, within
// one source; ceil((9 npc + 1) / 16) 128-row tiles each), blockIdx.x the K-steps, which walk
// x-runs, then z within a slab of zs planes, then y, then slabs, then samples.
struct WgradHaloParams {
    CUtensorMap amaps[2];           // chunk-plane maps of the sources, box (8 rl, 3, 3, 1, npc0 / npc1)
    CUtensorMap bmap;               // output gradient, box (8 rl, 1, 1, 1, n/8)
    int rl;                         // voxels per x-run (K-step)
    int kc0, kc1, n;
    int npc0, npc1;                 // planes per CTA of source 0 / 1
    int splits0;                    // plane splits over source 0 (the rest cover source 1)
    int ones_split;                 // split whose ones row gives the bias gradient (-1: none)
    int nx, zs, nzs;                // x-runs per row, z slab depth, slabs per sample
    TileGrid g;                     // B, D, H, W of the layer
    int ksteps_total, ksteps_per_cta, stages;
    int ksub;                       // K-steps per stage (each its own a_region + B block, sub_bytes apart)
    uint32_t a_region, b_stage_bytes, sub_bytes, stage_bytes;
    uint32_t idesc;
    float* dw;                      // [27][8 * (kc0 + kc1)][n]
    float* db;                      // [n] or null
    int* err;
};

// Persistent launch: min(tiles, persistent x SMs x resident CTAs) x grid_n CTAs.
constexpr int kMaxGridN = 16;               // N tiles of one rows GEMM (claim counters per launch)
cudaError_t launch_rows(const RowsParams& p, int grid_n, size_t smem, cudaStream_t s);
cudaError_t launch_wgrad_halo(const WgradHaloParams& p, dim3 grid, size_t smem, cudaStream_t s);
cudaError_t launch_wgrad(const WgradParams& p, dim3 grid, size_t smem, cudaStream_t s);
// TMEM columns to allocate for n FP32 accumulator columns (a power of two >= 32).
__host__ __device__ inline uint32_t tmem_cols(int n) {
    uint32_t c = 32;
    while (c < (uint32_t)n) c <<= 1;
    return c;
}

}  // namespace spnn
