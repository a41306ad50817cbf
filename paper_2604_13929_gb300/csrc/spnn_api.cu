// spnn_api.cu -- C ABI of the fluence surrogate (include/spnn.h): tensor-map
// construction, layer calls on the tensor-core GEMM kernels, weight packing,
// data kernels and the U-Net runtime (buffers, forward, backward, Adam).
#include <atomic>
#include <cudaTypedefs.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <utility>
#include <vector>

#include "spnn.h"
#include "spnn_internal.cuh"
#include "spnn_umma.cuh"

using namespace spnn;

namespace {

thread_local std::string g_error;
__device__ int g_err_flag;
// Tile claim counters of the persistent rows GEMM: each launch takes the next
// of kCtrSlots rows and zeroes it on its stream first, so up to kCtrSlots
// launches may be in flight on different streams at once.
constexpr int kCtrSlots = 64;
__device__ int g_tile_ctr[kCtrSlots][spnn::kMaxGridN];

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(SPNN_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CU(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

int* err_ptr() {
    static int* p = nullptr;
    if (!p) {
        void* q = nullptr;
        if (cudaGetSymbolAddress(&q, g_err_flag) != cudaSuccess) return nullptr;
        p = static_cast<int*>(q);
    }
    return p;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// ------------------------------------------------------------ tensor maps --
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tiles of `rows` voxels over a (B, D, H, W) grid with power-of-two extents:
// x-runs of at most 32 voxels (a 512-byte TMA box row), then y, z, samples.
bool make_grid(int rows, int B, int D, int H, int W, TileGrid* g) {
    int rem = rows;
    g->B = B, g->D = D, g->H = H, g->W = W;
    g->bx = W < 32 ? W : 32;
    if (g->bx > rem) g->bx = rem;
    rem /= g->bx;
    g->by = H < rem ? H : rem;
    rem /= g->by;
    g->bz = D < rem ? D : rem;
    rem /= g->bz;
    g->bb = rem;
    if ((long long)g->bx * g->by * g->bz * g->bb != rows || g->bb > B || B % g->bb) return false;
    g->nx = W / g->bx;
    g->ny = H / g->by;
    g->nz = D / g->bz;
    return true;
}

long long n_tiles(const TileGrid& g) { return (long long)g.nx * g.ny * g.nz * (g.B / g.bb); }
long long n_voxels(const TileGrid& g) { return (long long)g.B * g.D * g.H * g.W; }

int encode(CUtensorMap* m, const void* base, const cuuint64_t dims[5], const cuuint64_t strides[4],
           const cuuint32_t box[5]) {
    auto fn = encode_fn();
    if (!fn) return fail(SPNN_ECUDA, "cuTensorMapEncodeTiled unavailable");
    if (reinterpret_cast<uintptr_t>(base) % 16) return fail(SPNN_EINVAL, "tensor base not 16-byte aligned");
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SPNN_EINVAL, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return SPNN_OK;
}

// Chunk-plane tensor [C/8][B][D][H][W][8] on grid g: dims (8W, H, D, B, C/8);
// coordinates (8x, y, z, b, c8).  Default box (8 bx, by, bz, bb, planes); the
// conv3 halo box is (8 bx, by + 2, 3, 1, planes).
int map_planes(CUtensorMap* m, const void* p, int C, const TileGrid& g, int planes = 1, int halo = 0) {
    const cuuint64_t row = 16ull * g.W;
    cuuint64_t dims[5] = {8ull * g.W, (cuuint64_t)g.H, (cuuint64_t)g.D, (cuuint64_t)g.B, (cuuint64_t)(C / 8)};
    cuuint64_t strides[4] = {row, row * g.H, row * g.H * g.D, row * g.H * g.D * g.B};
    cuuint32_t box[5] = {8u * g.bx, (cuuint32_t)g.by, (cuuint32_t)g.bz, (cuuint32_t)g.bb, (cuuint32_t)planes};
    if (halo) {
        if (halo == 2) box[0] = 8u * (g.bx + 2);   // x-halo too: all 27 taps in one box
        box[1] = g.by + 2;
        box[2] = 3;
        box[3] = 1;
    }
    return encode(m, p, dims, strides, box);
}

// Stride-2 view at offset o = (oz, oy, ox) of a fine chunk-plane tensor of grid
// (B, 2D, 2H, 2W), indexed by the coarse grid g: dims (8, W, H, D, C/8 * B),
// box (8, bx, by, bz, bb); coordinates (0, x, y, z, c8 B + b).
int map_strided(CUtensorMap* m, const void* p, int C, const TileGrid& g, int o) {
    const long long Wf = 2LL * g.W, Hf = 2LL * g.H, Df = 2LL * g.D;
    const int oz = o >> 2, oy = (o >> 1) & 1, ox = o & 1;
    const __nv_bfloat16* base = static_cast<const __nv_bfloat16*>(p) + ((oz * Hf + oy) * Wf + ox) * 8;
    cuuint64_t dims[5] = {8, (cuuint64_t)g.W, (cuuint64_t)g.H, (cuuint64_t)g.D, (cuuint64_t)(C / 8) * g.B};
    cuuint64_t strides[4] = {32, (cuuint64_t)(32 * Wf), (cuuint64_t)(32 * Wf * Hf), (cuuint64_t)(16 * Wf * Hf * Df)};
    cuuint32_t box[5] = {8, (cuuint32_t)g.bx, (cuuint32_t)g.by, (cuuint32_t)g.bz, (cuuint32_t)g.bb};
    return encode(m, base, dims, strides, box);
}

int n_taps_of(int kind) { return kind == KIND_CONV3 ? 27 : 8; }


// ------------------------------------------------------------ rows GEMM --
// Choose the K-step geometry of a rows GEMM (maps already hold their boxes).
// N-tile width of a rows GEMM and of its packed operand: up to 256 columns;
// 128 for a GEMM with a scatter epilogue (up forward, down input gradient)
// and N >= 256, which the epilogue bounds: two CTAs (eight epilogue warps)
// then share an SM.  Measured 1.3 - 1.6x faster on the U-Net's up layers.
int gemm_n_tile(bool scatter, int n_total) {
    if (scatter && n_total >= 256) return 128;
    return n_total <= 256 ? n_total : 256;
}

void rows_geometry(RowsParams& p) {
    p.n_tile = gemm_n_tile(p.scatter_up, p.n_total);
    if (p.tap_mode == TAP_SHIFT3 && p.halo == 2) {
        const uint32_t nrow = (uint32_t)p.n_tile * 16u;
        p.halo_plane = (uint32_t)((p.g.bx + 2) * (p.g.by + 2) * 3 * 16);
        p.a_stage_bytes = p.E * p.halo_plane;
        p.b_stage_bytes = 27u * p.E * nrow;
        p.ksteps = p.kc_total / p.E;
    } else if (p.tap_mode == TAP_SHIFT3) {
        const uint32_t nrow = (uint32_t)p.n_tile * 16u;
        p.halo_plane = (uint32_t)(p.g.bx * (p.g.by + 2) * 3 * 16);
        p.a_stage_bytes = p.halo ? p.E * p.halo_plane : 9u * p.E * 2048u;
        p.b_stage_bytes = 9u * p.E * nrow;
        p.ksteps = 3 * (p.kc_total / p.E);
    } else {
        p.ksteps = p.n_taps * (p.kc_total / p.kc_step);
        p.a_stage_bytes = 2048u * p.kc_step;
        p.b_stage_bytes = (uint32_t)(p.kc_step * p.n_tile * 16);
    }
    p.stage_bytes = (p.a_stage_bytes + p.b_stage_bytes + 1023u) & ~1023u;
}

// Launch tuning (spnn_set_option): conv3 subtiles per CTA, chunk planes per
// K-step, and the shared-memory budget of the stage ring; 0 = automatic.
int g_opt_mt = 0, g_opt_planes = 0, g_opt_stage_kb = 0, g_opt_wgrad_halo = 1, g_opt_full_halo = 0,
    g_opt_rows_persistent = 2, g_opt_loss_fluence = 0;

int stage_budget() { return (g_opt_stage_kb > 0 ? g_opt_stage_kb : 110) * 1024; }

// conv3 tiling: mt 128-row subtiles per CTA (stacked along y, sharing one halo
// box and one weight copy) and E chunk planes per K-step.  Prefers the most
// subtiles, then the most planes, whose stage fits half the ring budget.
// Returns false if the grid does not tile.
bool conv_tiling_with(int opt_mt, int opt_planes, int B, int D, int H, int W, int kc0, int kc1, int n_total,
                      TileGrid* g, int* mt, int* E, int* halo);

// Full-halo tiling: CTA boxes of 8 x (16 mt) voxels in one z-plane, all 27 taps
// from one (10, 16 mt + 2, 3) box per block of E planes.
bool full_halo_tiling(int B, int D, int H, int W, int kc0, int kc1, int n_total, TileGrid* g, int* mt, int* E) {
    const long long n_tile = n_total <= 256 ? n_total : 256;
    if (W % 8 || H % 16) return false;
    for (int m : {2, 1}) {
        if (g_opt_mt > 0 && m != g_opt_mt) continue;
        if (H % (16 * m) || m * n_tile > 512) continue;
        for (int e : {4, 2}) {
            if (g_opt_planes > 0 && e != g_opt_planes) continue;
            if (kc0 % e || kc1 % e) continue;
            const long long a = (long long)e * 10 * (16 * m + 2) * 3 * 16;
            const long long b = 27LL * e * n_tile * 16;
            if (2 * (a + b) > stage_budget()) continue;
            g->B = B, g->D = D, g->H = H, g->W = W;
            g->bx = 8, g->by = 16 * m, g->bz = 1, g->bb = 1;
            g->nx = W / 8, g->ny = H / (16 * m), g->nz = D;
            *mt = m, *E = e;
            return true;
        }
    }
    return false;
}

bool conv_tiling(int B, int D, int H, int W, int kc0, int kc1, int n_total, TileGrid* g, int* mt, int* E,
                 int* halo) {
    if (g_opt_full_halo && full_halo_tiling(B, D, H, W, kc0, kc1, n_total, g, mt, E)) {
        *halo = 2;
        return true;
    }
    // options that do not fit this layer fall back to the automatic choice
    return conv_tiling_with(g_opt_mt, g_opt_planes, B, D, H, W, kc0, kc1, n_total, g, mt, E, halo) ||
           conv_tiling_with(0, 0, B, D, H, W, kc0, kc1, n_total, g, mt, E, halo);
}

bool conv_tiling_with(int opt_mt, int opt_planes, int B, int D, int H, int W, int kc0, int kc1, int n_total,
                      TileGrid* g, int* mt, int* E, int* halo) {
    const long long n_tile = n_total <= 256 ? n_total : 256;
    const int mts[3] = {4, 2, 1};
    for (int mi = 0; mi < 3; ++mi) {
        const int m = mts[mi];
        if (opt_mt > 0 && m != opt_mt) continue;
        TileGrid t;
        if (!make_grid(kRows * m, B, D, H, W, &t)) continue;
        const bool h = t.bz == 1 && t.bb == 1;
        if (m > 1 && !h) continue;
        if (m * n_tile > 512) continue;
        for (int e : {4, 2}) {
            if (opt_planes > 0 && e != opt_planes) continue;
            if (kc0 % e || kc1 % e) continue;
            const long long a = h ? (long long)e * t.bx * (t.by + 2) * 3 * 16 : 9LL * e * 2048;
            const long long b = 9LL * e * n_tile * 16;
            if (2 * (a + b) > stage_budget() && !(m == 1 && e == 2)) continue;
            *g = t, *mt = m, *E = e, *halo = h ? 1 : 0;
            return true;
        }
    }
    return false;
}

// Chunk planes per K-step for the other modes: the largest even divisor of kc_total up to 8.
int plain_kc_step(int kc_total) {
    int ks = kc_total < 8 ? kc_total : 8;
    while (kc_total % ks) ks -= 2;
    return ks;
}

int rows_gemm(RowsParams& p, cudaStream_t st) {
    if (p.n_total <= 0 || p.n_total % 16) return fail(SPNN_EINVAL, "GEMM N %d not a multiple of 16", p.n_total);
    if (p.n_total > 256 && p.n_total % 256) return fail(SPNN_EINVAL, "GEMM N %d > 256 not a multiple of 256", p.n_total);
    if (p.kc_total < 2 || p.kc_total % 2) return fail(SPNN_EINVAL, "input channels not a multiple of 16");
    rows_geometry(p);
    if (p.mt < 1) p.mt = 1;
    // two accumulator buffers where they fit in TMEM; a CTA whose buffers take
    // all 512 columns runs alone on its SM, so its ring may use twice the budget
    p.nbuf = 2 * p.mt * p.n_tile <= 512 ? 2 : 1;
    const bool alone = tmem_cols(p.nbuf * p.mt * p.n_tile) > 256;
    const uint32_t budget = (uint32_t)stage_budget() * (alone && g_opt_stage_kb <= 0 ? 2u : 1u);
    int S = (int)(budget / p.stage_bytes);
    p.stages = S < 2 ? 2 : (S > 8 ? 8 : S);
    p.tiles = (int)n_tiles(p.g);
    p.persistent = g_opt_rows_persistent;
    // K-major no-swizzle operands: leading-dimension offset = step between
    // 16-byte chunk planes along K, stride-dimension offset = step between
    // 8-row groups (128 bytes); the kernel builds the descriptors.
    p.idesc = idesc_bf16(128, p.n_tile, 0, 0);
    p.err = err_ptr();
    if (!p.err) return fail(SPNN_ECUDA, "no device");
    const int grid_n = p.n_total / p.n_tile;
    if (grid_n > kMaxGridN) return fail(SPNN_EINVAL, "GEMM N %d: more than %d N tiles", p.n_total, kMaxGridN);
    static std::atomic<unsigned> ctr_next{0};   // launches may come from several host threads
    void* ctr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ctr, g_tile_ctr);
    if (e != cudaSuccess) return cuda_fail(e, "tile counters");
    p.tile_ctr = static_cast<int*>(ctr) + (size_t)(ctr_next.fetch_add(1) % kCtrSlots) * kMaxGridN;
    e = cudaMemsetAsync(p.tile_ctr, 0, sizeof(int) * grid_n, st);
    if (e != cudaSuccess) return cuda_fail(e, "tile counter reset");
    // stages, alignment slack, 2 S + 12 mbarriers, four tile slots and the TMEM address slot
    size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + (2 * p.stages + 15) * 8;
    if (smem > 227 * 1024) return fail(SPNN_EINVAL, "stage of %u bytes does not fit", p.stage_bytes);
    e = launch_rows(p, grid_n, smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "rows_kernel launch");
    return SPNN_OK;
}

// ----------------------------------------------------------- wgrad GEMM --
int wgrad_gemm(WgradParams& p, int btaps, cudaStream_t st) {
    if (p.n <= 0 || p.n % 16 || p.n > 256) return fail(SPNN_EINVAL, "wgrad N %d must be 16..256, step 16", p.n);
    p.ksteps_total = (int)n_tiles(p.g);
    const int groups_all = p.n_groups + (p.ones_group >= 0 ? 1 : 0);
    const int m_tiles = (groups_all + 15) / 16;
    int splits = (4 * 152 + m_tiles * btaps - 1) / (m_tiles * btaps);
    if (splits < 1) splits = 1;
    if (splits > p.ksteps_total) splits = p.ksteps_total;
    p.ksteps_per_cta = (p.ksteps_total + splits - 1) / splits;
    splits = (p.ksteps_total + p.ksteps_per_cta - 1) / p.ksteps_per_cta;
    const uint32_t gbytes = (uint32_t)p.kv * 16u;
    p.a_stage_bytes = 16u * gbytes;
    p.b_stage_bytes = (uint32_t)(p.n / 8) * gbytes;
    p.stage_bytes = p.a_stage_bytes + p.b_stage_bytes;
    int S = (int)((100u * 1024u) / p.stage_bytes);
    p.stages = S < 2 ? 2 : (S > 6 ? 6 : S);
    // MN-major no-swizzle operands (descriptors built in the kernel):
    // leading-dimension offset = step between 8-voxel core matrices along K
    // (128 bytes), stride-dimension offset = step between 8-channel groups
    // along M / N (one group block, kv * 16 bytes).
    p.idesc = idesc_bf16(128, p.n, 1, 1);
    p.err = err_ptr();
    if (!p.err) return fail(SPNN_ECUDA, "no device");
    size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + (2 * p.stages + 2) * 8;
    cudaError_t e = launch_wgrad(p, dim3(splits, m_tiles, btaps), smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "wgrad_kernel launch");
    return SPNN_OK;
}

}  // namespace

namespace {

// ------------------------------------------------------------- packing --
// Packed operand B[n][k] of one GEMM, n = output column, k = (tap, input
// channel), BF16, grouped in 16-byte chunks of 8 consecutive k:
//   conv3     [n tiles][dx + 1][kc][(dz + 1) * 3 + (dy + 1)][n_tile][8]
//             (the nine taps of one x-shift and one 8-channel chunk kc are
//             adjacent, so a K-step over (x-shift, chunk block) is one copy);
//   down / up [n tiles][taps][kc][n_tile][8].
// The source is the FP32 master W[t][ci][co], t = (dz+1)*9 + (dy+1)*3 + (dx+1).
__global__ void pack_kernel(int kind, int which, int cin, int cout, int taps_p, int kc_total, int n_tile,
                            const float* __restrict__ w, __nv_bfloat16* __restrict__ out, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        long long r = i;
        const int e = (int)(r % 8);
        r /= 8;
        const int nn = (int)(r % n_tile);
        r /= n_tile;
        int tap, kc, tile;
        if (kind == KIND_CONV3) {
            const int t9 = (int)(r % 9);
            r /= 9;
            kc = (int)(r % kc_total);
            r /= kc_total;
            const int dxi = (int)(r % 3);
            tile = (int)(r / 3);
            tap = t9 * 3 + dxi;      // (dz+1)*9 + (dy+1)*3 + (dx+1)
        } else {
            kc = (int)(r % kc_total);
            r /= kc_total;
            tap = (int)(r % taps_p);
            tile = (int)(r / taps_p);
        }
        const int n = tile * n_tile + nn, k = kc * 8 + e;
        int t, ci, co;
        if (which == SPNN_PACK_FWD) {
            if (kind == KIND_UP) {         // n = (o, co), k = ci
                t = n / cout;
                co = n % cout;
                ci = k;
            } else {                       // n = co, k = ci
                t = tap;
                ci = k;
                co = n;
            }
        } else {
            if (kind == KIND_CONV3) {      // n = ci, k = co, flipped taps
                t = 26 - tap;
                ci = n;
                co = k;
            } else if (kind == KIND_DOWN) {  // n = (o, ci), k = co
                t = n / cin;
                ci = n % cin;
                co = k;
            } else {                       // n = ci, k = (o, co)
                t = tap;
                ci = n;
                co = k;
            }
        }
        out[i] = __float2bfloat16_rn(w[((size_t)t * cin + ci) * cout + co]);
    }
}

// GEMM geometry of a packed operand: taps in the pack, K chunks, N.
void pack_geometry(int kind, int which, int cin, int cout, int* taps_p, int* kc_total, int* n_total) {
    if (which == SPNN_PACK_FWD) {
        *taps_p = kind == KIND_UP ? 1 : n_taps_of(kind);
        *kc_total = cin / 8;
        *n_total = kind == KIND_UP ? 8 * cout : cout;
    } else {
        *taps_p = kind == KIND_DOWN ? 1 : n_taps_of(kind);
        *kc_total = cout / 8;
        *n_total = kind == KIND_DOWN ? 8 * cin : cin;
    }
}

int check_kind(int kind, int cin, int cout) {
    if (kind < KIND_CONV3 || kind > KIND_UP) return fail(SPNN_EINVAL, "unknown layer kind %d", kind);
    if (cin <= 0 || cout <= 0 || cin % 16 || cout % 16)
        return fail(SPNN_EINVAL, "channels (%d, %d) must be positive multiples of 16", cin, cout);
    return SPNN_OK;
}

int grid_ok(int B, int D, int H, int W) {
    if (B <= 0 || !pow2(D) || !pow2(H) || !pow2(W))
        return fail(SPNN_EINVAL, "grid (%d, %d, %d, %d): D, H, W must be powers of two", B, D, H, W);
    return SPNN_OK;
}

EpiDest dest(void* out, long long plane, int col0, const void* addend, const void* mask, const float* bias,
             int relu) {
    EpiDest d;
    d.out = static_cast<__nv_bfloat16*>(out);
    d.addend = static_cast<const __nv_bfloat16*>(addend);
    d.mask = static_cast<const __nv_bfloat16*>(mask);
    d.bias = bias;
    d.plane = plane;
    d.col0 = col0;
    d.relu = relu;
    return d;
}

int bad_grid(int rows, const TileGrid&) {
    return fail(SPNN_EINVAL, "grid does not tile into %d-voxel boxes", rows);
}

int layer_forward(int kind, int B, int D, int H, int W, const void* x0, int c0, const void* x1, int c1,
                  const void* packed, const float* bias, int cout, int relu, void* y, const float* head_w,
                  const float* head_b, float* head_out, cudaStream_t st) {
    int rc;
    if ((rc = check_kind(kind, c0 + c1, cout)) || (rc = grid_ok(B, D, H, W))) return rc;
    if (!x0 || !packed || !y || (c1 && !x1)) return fail(SPNN_EINVAL, "null tensor");
    if (c1 && kind != KIND_CONV3) return fail(SPNN_EINVAL, "concatenated input only for conv3");
    if (c0 % 8 || c1 % 8) return fail(SPNN_EINVAL, "source channels must be multiples of 8");
    if (kind == KIND_DOWN && (D < 2 || H < 2 || W < 2)) return fail(SPNN_EINVAL, "down needs D, H, W >= 2");
    if (head_out && (kind != KIND_CONV3 || cout > 256 || !head_w || !head_b))
        return fail(SPNN_EINVAL, "fused head needs conv3, cout <= 256, head_w and head_b");
    RowsParams p;
    memset(&p, 0, sizeof p);
    const int s = kind == KIND_DOWN ? 2 : 1;
    p.mt = 1;
    if (kind == KIND_CONV3) {
        int halo = 0;
        if (!conv_tiling(B, D, H, W, c0 / 8, c1 / 8, cout, &p.g, &p.mt, &p.E, &halo)) return bad_grid(kRows, p.g);
        p.halo = halo;
    } else if (!make_grid(kRows, B, D / s, H / s, W / s, &p.g)) {
        return bad_grid(kRows, p.g);
    }
    p.kc_total = (c0 + c1) / 8;
    p.kc0 = c0 / 8;
    if (kind == KIND_CONV3) {
        p.tap_mode = TAP_SHIFT3;
        p.n_taps = 27;
        if ((rc = map_planes(&p.maps[0], x0, c0, p.g, p.E, p.halo))) return rc;
        if (c1 && (rc = map_planes(&p.maps[1], x1, c1, p.g, p.E, p.halo))) return rc;
    } else if (kind == KIND_DOWN) {
        p.tap_mode = TAP_MAP;
        p.n_taps = 8;
        p.kc_step = plain_kc_step(p.kc_total);
        for (int o = 0; o < 8; ++o)
            if ((rc = map_strided(&p.maps[o], x0, c0, p.g, o))) return rc;
    } else {
        p.tap_mode = TAP_NONE;
        p.n_taps = 1;
        p.kc_step = plain_kc_step(p.kc_total);
        if ((rc = map_planes(&p.maps[0], x0, c0, p.g, p.kc_step))) return rc;
    }
    p.wpack = static_cast<const __nv_bfloat16*>(packed);
    p.n_total = kind == KIND_UP ? 8 * cout : cout;
    p.scatter_up = kind == KIND_UP;
    p.cout_up = cout;
    p.split = p.n_total;
    const long long out_vox = n_voxels(p.g) * (kind == KIND_UP ? 8 : 1);
    p.d[0] = dest(y, out_vox * 8, 0, nullptr, nullptr, bias, relu);
    p.d[1] = p.d[0];
    p.head_out = head_out;
    p.head_w = head_w;
    p.head_b = head_b;
    return rows_gemm(p, st);
}

int layer_dgrad(int kind, int B, int D, int H, int W, const void* dy, int cout, const void* packed, int c0,
                int c1, void* dx0, const void* add0, const void* mask0, void* dx1, const void* add1,
                const void* mask1, cudaStream_t st) {
    int rc;
    if ((rc = check_kind(kind, c0 + c1, cout)) || (rc = grid_ok(B, D, H, W))) return rc;
    if (!dy || !packed || !dx0 || (c1 && !dx1)) return fail(SPNN_EINVAL, "null tensor");
    if (c1 && kind != KIND_CONV3) return fail(SPNN_EINVAL, "split input gradient only for conv3");
    if (c0 % 16 || c1 % 16) return fail(SPNN_EINVAL, "input-gradient destinations need multiples of 16 channels");
    RowsParams p;
    memset(&p, 0, sizeof p);
    const long long in_vox = (long long)B * D * H * W;
    p.kc_total = cout / 8;
    p.kc0 = p.kc_total;
    p.mt = 1;
    if (kind == KIND_CONV3) {
        int halo = 0;
        if (!conv_tiling(B, D, H, W, p.kc_total, 0, c0 + c1, &p.g, &p.mt, &p.E, &halo))
            return bad_grid(kRows, p.g);
        p.halo = halo;
        if ((rc = map_planes(&p.maps[0], dy, cout, p.g, p.E, p.halo))) return rc;
        p.tap_mode = TAP_SHIFT3;
        p.n_taps = 27;
        p.n_total = c0 + c1;
        p.split = c0;
        p.d[0] = dest(dx0, in_vox * 8, 0, add0, mask0, nullptr, 0);
        p.d[1] = c1 ? dest(dx1, in_vox * 8, c0, add1, mask1, nullptr, 0) : p.d[0];
    } else if (kind == KIND_DOWN) {
        if (!make_grid(kRows, B, D / 2, H / 2, W / 2, &p.g)) return bad_grid(kRows, p.g);
        p.kc_step = plain_kc_step(p.kc_total);
        if ((rc = map_planes(&p.maps[0], dy, cout, p.g, p.kc_step))) return rc;
        p.tap_mode = TAP_NONE;
        p.n_taps = 1;
        p.n_total = 8 * c0;
        p.split = p.n_total;
        p.scatter_up = 1;
        p.cout_up = c0;
        p.d[0] = dest(dx0, in_vox * 8, 0, add0, mask0, nullptr, 0);
        p.d[1] = p.d[0];
    } else {
        if (!make_grid(kRows, B, D, H, W, &p.g)) return bad_grid(kRows, p.g);
        p.kc_step = plain_kc_step(p.kc_total);
        for (int o = 0; o < 8; ++o)
            if ((rc = map_strided(&p.maps[o], dy, cout, p.g, o))) return rc;
        p.tap_mode = TAP_MAP;
        p.n_taps = 8;
        p.n_total = c0;
        p.split = c0;
        p.d[0] = dest(dx0, in_vox * 8, 0, add0, mask0, nullptr, 0);
        p.d[1] = p.d[0];
    }
    p.wpack = static_cast<const __nv_bfloat16*>(packed);
    return rows_gemm(p, st);
}

// conv3 weight gradient on halo K-steps (see WgradHaloParams).  Returns
// SPNN_OK, or 1 when the layer does not fit the halo scheme (caller falls back).
int wgrad_halo(int B, int D, int H, int W, const void* x0, int c0, const void* x1, int c1, const void* dy,
               int cout, float* dw, float* db, cudaStream_t st) {
    const int kc0 = c0 / 8, kc1 = c1 / 8;
    // x-runs of 16 or 32 voxels; one MMA of N = 3 cout <= 256; a CTA's planes np give
    // 9 np + 1 row groups in nM tiles of 16 with nM * 3 cout <= 512 TMEM columns
    if (W < 16 || W % 16 || 3 * cout > 256) return 1;
    // automatic use only where it measured faster than the per-tap kernel
    // (cout 32: 1.2 - 1.6x; cout 64: 0.8x); SPNN_OPT_WGRAD_HALO 2 forces it
    if (g_opt_wgrad_halo < 2 && cout > 32) return 1;
    // at most two 128-row tiles per CTA where that keeps its accumulators
    // within 256 TMEM columns: two CTAs per SM keep twice the loads in flight
    // (the kernel is latency-bound; 1.25x faster on the 64^3 32-channel layers
    // than three tiles and one CTA per SM, despite the extra padded rows)
    int nm_max = 512 / (3 * cout);
    if (2 * 3 * cout <= 256 && nm_max > 2) nm_max = 2;
    const int np_max = (16 * nm_max - 1) / 9;
    if (np_max < 1) return 1;
    WgradHaloParams p;
    memset(&p, 0, sizeof p);
    p.kc0 = kc0;
    p.kc1 = kc1;
    p.n = cout;
    p.dw = dw;
    p.db = db;
    // per source: the fewest splits of at most np_max planes, balanced
    const int sp0 = (kc0 + np_max - 1) / np_max, sp1 = kc1 ? (kc1 + np_max - 1) / np_max : 0;
    p.npc0 = (kc0 + sp0 - 1) / sp0;
    p.npc1 = kc1 ? (kc1 + sp1 - 1) / sp1 : 0;
    p.splits0 = sp0;
    const int splits = sp0 + sp1;
    p.ones_split = db ? splits - 1 : -1;
    const int np_big = p.npc0 > p.npc1 ? p.npc0 : p.npc1;
    const int nM = (9 * np_big + 16) / 16;
    p.g.B = B, p.g.D = D, p.g.H = H, p.g.W = W;
    // resident CTAs per SM by TMEM columns; runs of 32 voxels (512-byte TMA
    // rows, the longest a box row holds) when two share an SM (measured faster
    // there, slower with one CTA per SM)
    const int per_sm = 512 / (int)tmem_cols(nM * 3 * cout);
    p.rl = per_sm > 1 && W % 32 == 0 ? 32 : 16;
    p.nx = W / p.rl;
    p.zs = D % 8 == 0 ? 8 : (D % 4 == 0 ? 4 : (D % 2 == 0 ? 2 : 1));
    p.nzs = D / p.zs;
    int rc;
    const cuuint64_t row = 16ull * W;
    auto halo_map = [&](CUtensorMap* m, const void* ptr, int C, int planes) {
        cuuint64_t dims[5] = {8ull * W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B, (cuuint64_t)(C / 8)};
        cuuint64_t strides[4] = {row, row * H, row * H * D, row * H * D * B};
        cuuint32_t box[5] = {8u * p.rl, 3, 3, 1, (cuuint32_t)planes};
        return encode(m, ptr, dims, strides, box);
    };
    if ((rc = halo_map(&p.amaps[0], x0, c0, p.npc0))) return rc;
    if (c1 && (rc = halo_map(&p.amaps[1], x1, c1, p.npc1))) return rc;
    {
        cuuint64_t dims[5] = {8ull * W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B, (cuuint64_t)(cout / 8)};
        cuuint64_t strides[4] = {row, row * H, row * H * D, row * H * D * B};
        cuuint32_t box[5] = {8u * p.rl, 1, 1, 1, (cuuint32_t)(cout / 8)};
        if ((rc = encode(&p.bmap, dy, dims, strides, box))) return rc;
    }
    p.ksteps_total = B * D * H * p.nx;
    // A region: the rows of nM tiles (one run per row group), then three dY boxes
    const uint32_t run = 16u * (uint32_t)p.rl;
    p.a_region = ((uint32_t)(16 * nM) * run + 1023u) & ~1023u;
    p.b_stage_bytes = 3u * (uint32_t)(cout / 8) * run;
    // with one CTA per SM two K-steps per stage halve the barrier handshakes
    p.ksub = per_sm > 1 ? 1 : 2;
    p.sub_bytes = (p.a_region + p.b_stage_bytes + 1023u) & ~1023u;
    p.stage_bytes = (uint32_t)p.ksub * p.sub_bytes;
    int S = (int)((uint32_t)(per_sm > 1 ? 100 : 200) * 1024u / p.stage_bytes);
    p.stages = S < 2 ? 2 : (S > 8 ? 8 : S);
    p.idesc = idesc_bf16(128, 3 * cout, 1, 1);
    p.err = err_ptr();
    if (!p.err) return fail(SPNN_ECUDA, "no device");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device attributes");
    // K splits: about one CTA per resident slot over all plane splits
    int gx = (sms * per_sm + splits - 1) / splits;
    if (gx > p.ksteps_total) gx = p.ksteps_total;
    p.ksteps_per_cta = (p.ksteps_total + gx - 1) / gx;
    gx = (p.ksteps_total + p.ksteps_per_cta - 1) / p.ksteps_per_cta;
    const size_t smem = (size_t)p.stages * p.stage_bytes + 1024 + (2 * p.stages + 2) * 8;
    e = launch_wgrad_halo(p, dim3(gx, splits), smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "wgrad_halo_kernel launch");
    return SPNN_OK;
}

int layer_wgrad(int kind, int B, int D, int H, int W, const void* x0, int c0, const void* x1, int c1,
                const void* dy, int cout, float* dw, float* db, cudaStream_t st) {
    int rc;
    if ((rc = check_kind(kind, c0 + c1, cout)) || (rc = grid_ok(B, D, H, W))) return rc;
    if (!x0 || !dy || !dw || (c1 && !x1)) return fail(SPNN_EINVAL, "null tensor");
    if (c1 && kind != KIND_CONV3) return fail(SPNN_EINVAL, "concatenated input only for conv3");
    if (c0 % 8 || c1 % 8) return fail(SPNN_EINVAL, "source channels must be multiples of 8");
    if (kind == KIND_CONV3 && g_opt_wgrad_halo) {
        const int h = wgrad_halo(B, D, H, W, x0, c0, x1, c1, dy, cout, dw, db, st);
        if (h != 1) return h;
    }
    WgradParams p;
    memset(&p, 0, sizeof p);
    p.mode = kind;
    p.kc_total = (c0 + c1) / 8;
    p.kc0 = c0 / 8;
    p.n = cout;
    p.dw = dw;
    p.db = db;
    int btaps = 1;
    const int s = kind == KIND_DOWN ? 2 : 1;
    // 128-voxel K-steps while the stage stays small, else 64
    p.kv = cout <= 64 ? 128 : 64;
    if (!make_grid(p.kv, B, D / s, H / s, W / s, &p.g)) {
        p.kv = 64;
        if (!make_grid(p.kv, B, D / s, H / s, W / s, &p.g)) return bad_grid(p.kv, p.g);
    }
    // planes per box: runs of consecutive chunks of one tap and one source,
    // aligned to the 16-group M tiles
    auto run = [](int a, int b) {
        int e = 16;
        while (e > 1 && ((a % e) || (b % e))) e /= 2;
        return e;
    };
    p.eb = kind == KIND_UP ? 1 : run(cout / 8, cout / 8);
    if (kind == KIND_CONV3) {
        p.ea = run(c0 / 8, c1 ? c1 / 8 : c0 / 8);
        if ((rc = map_planes(&p.amaps[0], x0, c0, p.g, p.ea))) return rc;
        if (c1 && (rc = map_planes(&p.amaps[1], x1, c1, p.g, p.ea))) return rc;
        if ((rc = map_planes(&p.bmaps[0], dy, cout, p.g, p.eb))) return rc;
        p.n_groups = 27 * p.kc_total;
    } else if (kind == KIND_DOWN) {
        p.ea = 1;
        for (int o = 0; o < 8; ++o)
            if ((rc = map_strided(&p.amaps[o], x0, c0, p.g, o))) return rc;
        if ((rc = map_planes(&p.bmaps[0], dy, cout, p.g, p.eb))) return rc;
        p.n_groups = 8 * p.kc_total;
    } else {
        p.ea = run(c0 / 8, c0 / 8);
        if ((rc = map_planes(&p.amaps[0], x0, c0, p.g, p.ea))) return rc;
        for (int o = 0; o < 8; ++o)
            if ((rc = map_strided(&p.bmaps[o], dy, cout, p.g, o))) return rc;
        p.n_groups = p.kc_total;
        btaps = 8;
    }
    p.ones_group = db ? p.n_groups : -1;
    return wgrad_gemm(p, btaps, st);
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// --------------------------------------------------------- data kernels --
// Pore fraction of each sample's mask: one block per sample.
__global__ void porosity_kernel(const uint8_t* __restrict__ mask, long long vox_per_sample, float* __restrict__ phi) {
    const uint8_t* m = mask + (long long)blockIdx.x * vox_per_sample;
    unsigned long long c = 0;
    for (long long i = threadIdx.x; i < vox_per_sample; i += blockDim.x) c += m[i] ? 1 : 0;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ unsigned long long part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        phi[blockIdx.x] = (float)((double)t / (double)vox_per_sample);
    }
}

// Input features in chunk planes: plane 0 holds channels 0-7, plane 1 channels 8-15 (zero).
// Channel 6 is the diffusion-theory attenuation exponent -mu_eff (z + 1/2) / 8 of the
// medium scaled to its solid fraction (mu' = (1 - phi) mu), channel 7 the porosity phi.
__global__ void pack_input_kernel(const uint8_t* __restrict__ mask, const float* __restrict__ optics,
                                  const float* __restrict__ phi, int D, long long vox_per_sample,
                                  long long total, __nv_bfloat16* __restrict__ x, int HW) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / vox_per_sample;
        const int z = (int)((i % vox_per_sample) / HW);
        const float pore = mask[i] ? 1.f : 0.f;
        const float mus = optics[3 * b], mua = optics[3 * b + 1], g = optics[3 * b + 2], ph = phi[b];
        const float ma = (1.f - ph) * mua, msp = (1.f - ph) * mus * (1.f - g);
        const float mu_eff = sqrtf(3.f * ma * (ma + msp));
        const float zc = z + 0.5f;
        const float f[8] = {pore, 1.f - pore, logf(mus), 0.25f * logf(mua), g, zc / (float)D,
                            -mu_eff * zc * 0.125f, ph};
        uint4 w;
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
        *reinterpret_cast<uint4*>(x + i * 8) = w;
        *reinterpret_cast<uint4*>(x + (total + i) * 8) = make_uint4(0, 0, 0, 0);
    }
}

__global__ void log_fluence_kernel(const uint64_t* __restrict__ raw, const double* __restrict__ n_photons,
                                   long long vox_per_sample, long long total, double area, float floor_,
                                   float* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double n = n_photons[i / vox_per_sample];
        const double phi = (double)raw[i] * (area / (n * 4294967296.0));
        out[i] = logf(fmaxf((float)phi, floor_));
    }
}

// one block per (sample, z layer): sums of exp(log_phi) per phase
__global__ void phase_profile_kernel(const float* __restrict__ log_phi, const uint8_t* __restrict__ mask, int HW,
                                     float* __restrict__ prof, int D) {
    const long long base = (long long)blockIdx.x * HW;
    float s[2] = {0.f, 0.f};
    int c[2] = {0, 0};
    for (int i = threadIdx.x; i < HW; i += blockDim.x) {
        const int ph = mask[base + i] ? 1 : 0;
        s[ph] += expf(log_phi[base + i]);
        c[ph] += 1;
    }
    __shared__ float ss[2][32];
    __shared__ int cc[2][32];
    for (int ph = 0; ph < 2; ++ph) {
        for (int o = 16; o; o >>= 1) {
            s[ph] += __shfl_xor_sync(0xffffffffu, s[ph], o);
            c[ph] += __shfl_xor_sync(0xffffffffu, c[ph], o);
        }
        if ((threadIdx.x & 31) == 0) {
            ss[ph][threadIdx.x >> 5] = s[ph];
            cc[ph][threadIdx.x >> 5] = c[ph];
        }
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int ph = threadIdx.x;
        float t = 0.f;
        int n = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t += ss[ph][w];
            n += cc[ph][w];
        }
        const int b = blockIdx.x / D, z = blockIdx.x % D;
        prof[((long long)b * 2 + ph) * D + z] = n ? t / n : __int_as_float(0x7fc00000);
    }
}

// Fluence-weighted loss: norm[b] = voxels / sum over sample b of exp(target),
// one block per sample (FP64 sum).
__global__ void loss_norm_kernel(const float* __restrict__ target, long long per_sample, float* __restrict__ norm) {
    __shared__ double part[8];
    const float* t = target + (long long)blockIdx.x * per_sample;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < per_sample; i += blockDim.x) acc += (double)expf(t[i]);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += part[w];
        norm[blockIdx.x] = (float)((double)per_sample / sum);
    }
}

// Loss and head backward, one thread per voxel: d = pred - target, weight
// w = 1 or (norm given) exp(target) norm[sample]; loss += w d^2 / n,
// dp = 2 w d / n; g[v, c] = dp h[c] (a[v, c] > 0); dh[c] += dp a[v, c]; dc += dp.
template <int C>
__global__ void loss_head_kernel(const float* __restrict__ pred, const float* __restrict__ target,
                                 const __nv_bfloat16* __restrict__ act, const float* __restrict__ hw,
                                 long long total, double inv_n, const float* __restrict__ norm,
                                 long long per_sample, double* loss, __nv_bfloat16* __restrict__ g,
                                 float* __restrict__ dhw, float* __restrict__ dhb) {
    __shared__ float sh[C + 1];
    __shared__ double sl;
    if (threadIdx.x <= C) sh[threadIdx.x] = 0.f;
    if (threadIdx.x == 0) sl = 0.0;
    __syncthreads();
    float acc[C + 1];
#pragma unroll
    for (int c = 0; c <= C; ++c) acc[c] = 0.f;
    double l = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = (double)pred[i] - (double)target[i];
        const double wv = norm ? (double)(expf(target[i]) * norm[i / per_sample]) : 1.0;
        l += wv * d * d;
        const float dp = (float)(2.0 * wv * d * inv_n);
        acc[C] += dp;
#pragma unroll
        for (int c0 = 0; c0 < C; c0 += 8) {
            const long long off = (c0 / 8) * total * 8 + i * 8;   // chunk plane c0 / 8, voxel i
            const uint4 u = *reinterpret_cast<const uint4*>(act + off);
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
            uint4 o;
            __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 a = __bfloat1622float2(h[k]);
                const int c = c0 + 2 * k;
                acc[c] += dp * a.x;
                acc[c + 1] += dp * a.y;
                oh[k] = __floats2bfloat162_rn(a.x > 0.f ? dp * hw[c] : 0.f, a.y > 0.f ? dp * hw[c + 1] : 0.f);
            }
            *reinterpret_cast<uint4*>(g + off) = o;
        }
    }
#pragma unroll
    for (int c = 0; c <= C; ++c) {
        float v = acc[c];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sh[c], v);
    }
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sl, l);
    __syncthreads();
    if (threadIdx.x < C) atomicAdd(&dhw[threadIdx.x], sh[threadIdx.x]);
    if (threadIdx.x == C) atomicAdd(dhb, sh[C]);
    if (threadIdx.x == 0 && loss) atomicAdd(loss, sl * inv_n);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

int grid_for(long long n, int threads = 256) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

int pack(int kind, int cin, int cout, int which, const float* w, void* packed, cudaStream_t st) {
    int rc;
    if ((rc = check_kind(kind, cin, cout))) return rc;
    if (!w || !packed) return fail(SPNN_EINVAL, "null tensor");
    int taps_p, kc, n_total;
    pack_geometry(kind, which, cin, cout, &taps_p, &kc, &n_total);
    // the GEMMs with a scatter epilogue: up forward and down input gradient
    const bool scatter = which == SPNN_PACK_FWD ? kind == KIND_UP : kind == KIND_DOWN;
    const int n_tile = gemm_n_tile(scatter, n_total);
    if (n_total % n_tile) return fail(SPNN_EINVAL, "packed N %d > 256 not a multiple of 256", n_total);
    const long long total = (long long)taps_p * kc * 8 * n_total;
    pack_kernel<<<grid_for(total), 256, 0, st>>>(kind, which, cin, cout, taps_p, kc, n_tile, w,
                                                  static_cast<__nv_bfloat16*>(packed), total);
    CU(cudaGetLastError());
    return SPNN_OK;
}

}  // namespace

// ================================================================ U-Net ==
struct spnn_unet {
    struct Layer {
        int kind, cin, cout, relu, src0, src1, edge_in, edge_out, taps;
        size_t woff, boff;
        __nv_bfloat16 *pk_fwd = nullptr, *pk_dgrad = nullptr;
        __nv_bfloat16 *act = nullptr, *grad = nullptr;
    };
    int c0 = 0, n = 0, max_batch = 0, adam_t = 0;
    std::vector<Layer> L;
    size_t nparam = 0, head_w = 0, head_b = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    float* loss_norm = nullptr;      // [max_batch]: per-sample 1 / mean exp(target) (fluence-weighted loss)
    const void* last_x = nullptr;
    float* last_pred = nullptr;
    int last_batch = 0;
};

namespace {

constexpr int kLayers = 20;
// source layer indices (-1 = network input), decoder "a" layers read [up, skip]
const int kSrc0[kLayers] = {-1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18};
const int kSrc1[kLayers] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 7, -1, -1, 4, -1, -1, 1, -1};
const int kKind[kLayers] = {0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 2, 0, 0, 2, 0, 0, 2, 0, 0};
const int kLevel[kLayers] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0};  // of the input
const int kCoutMul[kLayers] = {1, 1, 2, 2, 2, 4, 4, 4, 8, 8, 8, 4, 4, 4, 2, 2, 2, 1, 1, 1};

void free_net(spnn_unet* net) {
    if (!net) return;
    for (auto& l : net->L) {
        cudaFree(l.pk_fwd);
        cudaFree(l.pk_dgrad);
        cudaFree(l.act);
        cudaFree(l.grad);
    }
    cudaFree(net->params);
    cudaFree(net->loss_norm);
    cudaFree(net->grads);
    cudaFree(net->m);
    cudaFree(net->v);
    delete net;
}

int repack(spnn_unet* net, cudaStream_t st) {
    int rc;
    for (auto& l : net->L) {
        if ((rc = pack(l.kind, l.cin, l.cout, SPNN_PACK_FWD, net->params + l.woff, l.pk_fwd, st))) return rc;
        if ((rc = pack(l.kind, l.cin, l.cout, SPNN_PACK_DGRAD, net->params + l.woff, l.pk_dgrad, st))) return rc;
    }
    return SPNN_OK;
}

int src_channels(const spnn_unet* net, int s) { return s < 0 ? 16 : net->L[s].cout; }

}  // namespace

// ============================================================ C ABI ==
extern "C" {

const char* spnn_last_error(void) { return g_error.c_str(); }
int spnn_version(void) { return 1; }

int spnn_status(void* stream) {
    CU(cudaStreamSynchronize(as_stream(stream)));
    int* e = err_ptr();
    if (!e) return fail(SPNN_ECUDA, "no device");
    int h = 0;
    CU(cudaMemcpy(&h, e, sizeof h, cudaMemcpyDeviceToHost));
    if (h) {
        CU(cudaMemset(e, 0, sizeof h));
        return fail(SPNN_ECUDA, "a kernel gave up on a bounded wait (flag %d)", h);
    }
    return SPNN_OK;
}

int spnn_set_option(int key, int value) {
    if (value < 0) return fail(SPNN_EINVAL, "option values are >= 0");
    switch (key) {
    case SPNN_OPT_CONV_SUBTILES:
        if (value != 0 && value != 1 && value != 2 && value != 4) return fail(SPNN_EINVAL, "subtiles: 0, 1, 2 or 4");
        g_opt_mt = value;
        return SPNN_OK;
    case SPNN_OPT_CONV_PLANES:
        if (value != 0 && value != 2 && value != 4) return fail(SPNN_EINVAL, "planes: 0, 2 or 4");
        g_opt_planes = value;
        return SPNN_OK;
    case SPNN_OPT_STAGE_KB:
        if (value > 220) return fail(SPNN_EINVAL, "stage budget above 220 KB");
        g_opt_stage_kb = value;
        return SPNN_OK;
    case SPNN_OPT_WGRAD_HALO:
        if (value < 0 || value > 2) return fail(SPNN_EINVAL, "halo weight-gradient setting %d not in 0..2", value);
        g_opt_wgrad_halo = value;
        return SPNN_OK;
    case SPNN_OPT_CONV_FULL_HALO:
        g_opt_full_halo = value != 0;
        return SPNN_OK;
    case SPNN_OPT_LOSS_FLUENCE_WEIGHT:
        if (value != 0 && value != 1) return fail(SPNN_EINVAL, "loss weighting must be 0 or 1");
        g_opt_loss_fluence = value;
        return SPNN_OK;
    case SPNN_OPT_ROWS_PERSISTENT:
        if (value < 0 || value > 16) return fail(SPNN_EINVAL, "persistent grid multiple %d not in 0..16", value);
        g_opt_rows_persistent = value;
        return SPNN_OK;
    default:
        return fail(SPNN_EINVAL, "unknown option %d", key);
    }
}

size_t spnn_packed_elems(int kind, int cin, int cout) {
    return (size_t)(kind == KIND_CONV3 ? 27 : 8) * cin * cout;
}

int spnn_pack_weights(int kind, int cin, int cout, int which, const float* w, void* packed, void* stream) {
    return pack(kind, cin, cout, which, w, packed, as_stream(stream));
}

int spnn_layer_forward(int kind, int B, int D, int H, int W, const void* x0, int c0, const void* x1, int c1,
                       const void* packed, const float* bias, int cout, int relu, void* y, const float* head_w,
                       const float* head_b, float* head_out, void* stream) {
    return layer_forward(kind, B, D, H, W, x0, c0, x1, c1, packed, bias, cout, relu, y, head_w, head_b, head_out,
                         as_stream(stream));
}

int spnn_layer_dgrad(int kind, int B, int D, int H, int W, const void* dy, int cout, const void* packed, int c0,
                     int c1, void* dx0, const void* addend0, const void* mask0, void* dx1, const void* addend1,
                     const void* mask1, void* stream) {
    return layer_dgrad(kind, B, D, H, W, dy, cout, packed, c0, c1, dx0, addend0, mask0, dx1, addend1, mask1,
                       as_stream(stream));
}

int spnn_layer_wgrad(int kind, int B, int D, int H, int W, const void* x0, int c0, const void* x1, int c1,
                     const void* dy, int cout, float* dw, float* db, void* stream) {
    return layer_wgrad(kind, B, D, H, W, x0, c0, x1, c1, dy, cout, dw, db, as_stream(stream));
}

int spnn_pack_input(const uint8_t* mask, const float* optics, int B, int D, int H, int W, void* x, void* stream) {
    if (!mask || !optics || !x || B <= 0 || D <= 0 || H <= 0 || W <= 0) return fail(SPNN_EINVAL, "bad arguments");
    const long long vps = (long long)D * H * W, total = vps * B;
    cudaStream_t st = as_stream(stream);
    float* phi = nullptr;
    CU(cudaMallocAsync(reinterpret_cast<void**>(&phi), sizeof(float) * B, st));
    porosity_kernel<<<B, 256, 0, st>>>(mask, vps, phi);
    pack_input_kernel<<<grid_for(total), 256, 0, st>>>(mask, optics, phi, D, vps, total,
                                                        static_cast<__nv_bfloat16*>(x), H * W);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(phi, st);
    if (e != cudaSuccess) return cuda_fail(e, "pack_input launch");
    return SPNN_OK;
}

int spnn_log_fluence(const uint64_t* raw, const double* n_photons, int B, int D, int H, int W, float floor_,
                     float* out, void* stream) {
    if (!raw || !n_photons || !out || B <= 0 || D <= 0 || H <= 0 || W <= 0 || !(floor_ > 0.f))
        return fail(SPNN_EINVAL, "bad arguments");
    const long long vps = (long long)D * H * W, total = vps * B;
    log_fluence_kernel<<<grid_for(total), 256, 0, as_stream(stream)>>>(raw, n_photons, vps, total,
                                                                        (double)W * H, floor_, out);
    CU(cudaGetLastError());
    return SPNN_OK;
}

int spnn_phase_profiles(const float* log_phi, const uint8_t* mask, int B, int D, int H, int W, float* prof,
                        void* stream) {
    if (!log_phi || !mask || !prof || B <= 0 || D <= 0 || H <= 0 || W <= 0) return fail(SPNN_EINVAL, "bad arguments");
    phase_profile_kernel<<<B * D, 256, 0, as_stream(stream)>>>(log_phi, mask, H * W, prof, D);
    CU(cudaGetLastError());
    return SPNN_OK;
}

spnn_unet_t* spnn_unet_create(int c0, int n, int max_batch) {
    if ((c0 != 16 && c0 != 32) || !pow2(n) || n < 16 || max_batch <= 0) {
        fail(SPNN_EINVAL, "c0 must be 16 or 32, n a power of two >= 16, max_batch > 0");
        return nullptr;
    }
    auto* net = new spnn_unet;
    net->c0 = c0;
    net->n = n;
    net->max_batch = max_batch;
    size_t off = 0;
    for (int i = 0; i < kLayers; ++i) {
        spnn_unet::Layer l;
        l.kind = kKind[i];
        l.src0 = kSrc0[i];
        l.src1 = kSrc1[i];
        l.cout = kCoutMul[i] * c0;
        l.cin = (l.src0 < 0 ? 16 : net->L[l.src0].cout) + (l.src1 < 0 ? 0 : net->L[l.src1].cout);
        l.relu = l.kind != KIND_UP;
        l.edge_in = n >> kLevel[i];
        l.edge_out = l.kind == KIND_DOWN ? l.edge_in / 2 : (l.kind == KIND_UP ? l.edge_in * 2 : l.edge_in);
        l.taps = n_taps_of(l.kind);
        l.woff = off;
        off += (size_t)l.taps * l.cin * l.cout;
        l.boff = off;
        off += l.cout;
        net->L.push_back(l);
    }
    net->head_w = off;
    off += c0;
    net->head_b = off;
    off += 1;
    net->nparam = off;
    bool ok = cudaMalloc(&net->params, off * 4) == cudaSuccess && cudaMalloc(&net->grads, off * 4) == cudaSuccess &&
              cudaMalloc(&net->m, off * 4) == cudaSuccess && cudaMalloc(&net->v, off * 4) == cudaSuccess &&
              cudaMalloc(&net->loss_norm, (size_t)max_batch * 4) == cudaSuccess;
    for (auto& l : net->L) {
        if (!ok) break;
        const size_t pe = spnn_packed_elems(l.kind, l.cin, l.cout) * 2;
        const size_t ae = (size_t)max_batch * l.edge_out * l.edge_out * l.edge_out * l.cout * 2;
        ok = cudaMalloc(&l.pk_fwd, pe) == cudaSuccess && cudaMalloc(&l.pk_dgrad, pe) == cudaSuccess &&
             cudaMalloc(&l.act, ae) == cudaSuccess && cudaMalloc(&l.grad, ae) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        free_net(net);
        fail(SPNN_ENOMEM, "device allocation failed");
        return nullptr;
    }
    cudaMemset(net->params, 0, off * 4);
    cudaMemset(net->grads, 0, off * 4);
    cudaMemset(net->m, 0, off * 4);
    cudaMemset(net->v, 0, off * 4);
    return net;
}

void spnn_unet_destroy(spnn_unet_t* net) { free_net(net); }

size_t spnn_unet_param_count(const spnn_unet_t* net) { return net ? net->nparam : 0; }

int spnn_unet_set_params(spnn_unet_t* net, const float* params) {
    if (!net || !params) return fail(SPNN_EINVAL, "null argument");
    CU(cudaMemcpy(net->params, params, net->nparam * 4, cudaMemcpyHostToDevice));
    CU(cudaMemset(net->m, 0, net->nparam * 4));
    CU(cudaMemset(net->v, 0, net->nparam * 4));
    net->adam_t = 0;
    int rc = repack(net, nullptr);
    if (rc) return rc;
    CU(cudaDeviceSynchronize());
    return SPNN_OK;
}

int spnn_unet_get_params(spnn_unet_t* net, float* params) {
    if (!net || !params) return fail(SPNN_EINVAL, "null argument");
    CU(cudaDeviceSynchronize());
    CU(cudaMemcpy(params, net->params, net->nparam * 4, cudaMemcpyDeviceToHost));
    return SPNN_OK;
}

int spnn_unet_get_grads(spnn_unet_t* net, float* grads) {
    if (!net || !grads) return fail(SPNN_EINVAL, "null argument");
    CU(cudaDeviceSynchronize());
    CU(cudaMemcpy(grads, net->grads, net->nparam * 4, cudaMemcpyDeviceToHost));
    return SPNN_OK;
}

int spnn_unet_copy_activation(spnn_unet_t* net, int layer, int batch, void* dst, void* stream) {
    if (!net || !dst || layer < 0 || layer >= kLayers || batch <= 0 || batch > net->max_batch)
        return fail(SPNN_EINVAL, "bad arguments");
    const auto& l = net->L[layer];
    const size_t bytes = (size_t)batch * l.edge_out * l.edge_out * l.edge_out * l.cout * 2;
    CU(cudaMemcpyAsync(dst, l.act, bytes, cudaMemcpyDeviceToDevice, as_stream(stream)));
    return SPNN_OK;
}

int spnn_unet_layer_shape(const spnn_unet_t* net, int layer, int* edge, int* channels) {
    if (!net || !edge || !channels || layer < 0 || layer >= kLayers) return fail(SPNN_EINVAL, "bad arguments");
    *edge = net->L[layer].edge_out;
    *channels = net->L[layer].cout;
    return SPNN_OK;
}

int spnn_unet_forward(spnn_unet_t* net, const void* x, int batch, float* pred, void* stream) {
    if (!net || !x || !pred || batch <= 0 || batch > net->max_batch) return fail(SPNN_EINVAL, "bad arguments");
    cudaStream_t st = as_stream(stream);
    for (int i = 0; i < kLayers; ++i) {
        auto& l = net->L[i];
        const void* x0 = l.src0 < 0 ? x : net->L[l.src0].act;
        const void* x1 = l.src1 < 0 ? nullptr : net->L[l.src1].act;
        const int c0 = src_channels(net, l.src0), c1 = l.src1 < 0 ? 0 : net->L[l.src1].cout;
        const bool last = i == kLayers - 1;
        const int e = l.edge_in;
        int rc = layer_forward(l.kind, batch, e, e, e, x0, c0, x1, c1, l.pk_fwd, net->params + l.boff, l.cout,
                               l.relu, l.act, last ? net->params + net->head_w : nullptr,
                               last ? net->params + net->head_b : nullptr, last ? pred : nullptr, st);
        if (rc) return rc;
    }
    net->last_x = x;
    net->last_pred = pred;
    net->last_batch = batch;
    return SPNN_OK;
}

int spnn_unet_backward(spnn_unet_t* net, const float* target, int batch, double* loss, void* stream) {
    if (!net || !target || batch != net->last_batch || !net->last_pred)
        return fail(SPNN_EINVAL, "backward needs the forward of the same batch first");
    cudaStream_t st = as_stream(stream);
    CU(cudaMemsetAsync(net->grads, 0, net->nparam * 4, st));
    auto& last = net->L[kLayers - 1];
    const long long per_sample = (long long)net->n * net->n * net->n;
    const long long vox = (long long)batch * per_sample;
    const double inv_n = 1.0 / (double)vox;
    const int blocks = grid_for(vox, 256);
    const float* norm = nullptr;
    if (g_opt_loss_fluence) {
        loss_norm_kernel<<<batch, 256, 0, st>>>(target, per_sample, net->loss_norm);
        norm = net->loss_norm;
    }
    if (net->c0 == 16)
        loss_head_kernel<16><<<blocks, 256, 0, st>>>(net->last_pred, target, last.act, net->params + net->head_w,
                                                     vox, inv_n, norm, per_sample, loss, last.grad,
                                                     net->grads + net->head_w, net->grads + net->head_b);
    else
        loss_head_kernel<32><<<blocks, 256, 0, st>>>(net->last_pred, target, last.act, net->params + net->head_w,
                                                     vox, inv_n, norm, per_sample, loss, last.grad,
                                                     net->grads + net->head_w, net->grads + net->head_b);
    CU(cudaGetLastError());
    for (int i = kLayers - 1; i >= 0; --i) {
        auto& l = net->L[i];
        const int e = l.edge_in;
        const void* x0 = l.src0 < 0 ? net->last_x : net->L[l.src0].act;
        const void* x1 = l.src1 < 0 ? nullptr : net->L[l.src1].act;
        const int c0 = src_channels(net, l.src0), c1 = l.src1 < 0 ? 0 : net->L[l.src1].cout;
        int rc = layer_wgrad(l.kind, batch, e, e, e, x0, c0, x1, c1, l.grad, l.cout, net->grads + l.woff,
                             net->grads + l.boff, st);
        if (rc) return rc;
        if (i == 0) continue;
        if (l.src1 >= 0) {
            // [up, skip]: raw gradient of the up output; partial gradient of the skip
            rc = layer_dgrad(l.kind, batch, e, e, e, l.grad, l.cout, l.pk_dgrad, c0, c1, net->L[l.src0].grad,
                             nullptr, nullptr, net->L[l.src1].grad, nullptr, nullptr, st);
        } else {
            auto& s = net->L[l.src0];
            // a down layer reading a skip completes the skip's gradient in place
            const bool skip = l.kind == KIND_DOWN && (l.src0 == 1 || l.src0 == 4 || l.src0 == 7);
            rc = layer_dgrad(l.kind, batch, e, e, e, l.grad, l.cout, l.pk_dgrad, c0, 0, s.grad,
                             skip ? s.grad : nullptr, s.relu ? s.act : nullptr, nullptr, nullptr, nullptr, st);
        }
        if (rc) return rc;
    }
    return SPNN_OK;
}

int spnn_unet_adam(spnn_unet_t* net, float lr, float beta1, float beta2, float eps, void* stream) {
    if (!net) return fail(SPNN_EINVAL, "null network");
    cudaStream_t st = as_stream(stream);
    net->adam_t += 1;
    const double c1 = 1.0 / (1.0 - pow((double)beta1, net->adam_t));
    const double c2 = 1.0 / (1.0 - pow((double)beta2, net->adam_t));
    adam_kernel<<<grid_for((long long)net->nparam), 256, 0, st>>>(net->params, net->grads, net->m, net->v,
                                                                   net->nparam, lr, beta1, beta2, eps, (float)c1,
                                                                   (float)c2);
    CU(cudaGetLastError());
    return repack(net, st);
}

}  // extern "C"
