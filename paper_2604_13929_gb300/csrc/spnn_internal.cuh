// spnn_internal.cuh -- launch parameter blocks shared by the surrogate's GEMM
// kernels (spnn_gemm.cu) and its C ABI / runtime (spnn_api.cu).
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
constexpr int kWgradK = 64;                // voxels per wgrad K-step
constexpr int kThreads = 192;              // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr uint64_t kWaitLimitNs = 2000000000ull;

struct EpiDest {
    __nv_bfloat16* out;             // bf16 channels-last destination (may be null)
    const __nv_bfloat16* addend;    // added before the activation (same addressing), or null
    const __nv_bfloat16* mask;      // result zeroed where mask <= 0 (same addressing), or null
    const float* bias;              // per destination channel, or null
    int ld;                         // channels of the destination tensor
    int col0;                       // first GEMM column that lands in this destination
    int relu;
};

// Rows GEMM: D[row, n] = sum_k A[row, k] B[n, k]; rows are 128 consecutive
// voxels of the row grid, k = (tap, channel), A gathered by TMA boxes.
struct RowsParams {
    CUtensorMap maps[8];
    const __nv_bfloat16* wpack;     // [n tiles][taps][kc_total][n_tile][8]
    int n_taps, kc_total, kc0, kc_step, tap_mode;
    int R_B, R_D, R_H, R_W;
    int n_tile, n_total, ksteps, stages;
    uint32_t a_stage_bytes, b_stage_bytes, stage_bytes;
    uint32_t idesc, lbo_a, sbo_a, lbo_b, sbo_b;
    int scatter_up, cout_up, split;
    EpiDest d[2];
    float* head_out;                // fused one-channel head: out = head_b + sum_c y_c head_w[c]
    const float* head_w;
    const float* head_b;
    int* err;
};

// Weight-gradient GEMM: D[(group, r), n] = sum_v A_group[v, r] B[v, n] over a
// range of 64-voxel K-steps; rows are 16 groups of 8 input channels (one tap
// each), both operands MN-major, results added to fp32 dW with atomics.
struct WgradParams {
    CUtensorMap amaps[8];
    CUtensorMap bmaps[8];
    int mode;                       // KIND_*
    int kc_total, kc0, n_groups, ones_group;
    int V_B, V_D, V_H, V_W;
    int ksteps_total, ksteps_per_cta, n, stages;
    uint32_t a_stage_bytes, b_stage_bytes, stage_bytes;
    uint32_t idesc, lbo, sbo;
    float* dw;                      // [taps][kc_total * 8][n]
    float* db;                      // [n]
    int* err;
};

cudaError_t launch_rows(const RowsParams& p, int grid_m, int grid_n, size_t smem, cudaStream_t s);
cudaError_t launch_wgrad(const WgradParams& p, dim3 grid, size_t smem, cudaStream_t s);
// TMEM columns to allocate for n FP32 accumulator columns (a power of two >= 32).
__host__ __device__ inline uint32_t tmem_cols(int n) {
    uint32_t c = 32;
    while (c < (uint32_t)n) c <<= 1;
    return c;
}

}  // namespace spnn
