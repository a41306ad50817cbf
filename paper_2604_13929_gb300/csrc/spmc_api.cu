// spmc_api.cu -- C ABI of libspmc: handle life cycle, mask bit-packing,
// launches, and the FP64 normalisation of the integer tallies on the GPU.
//
// Normalisation (arXiv 2604.13929): R, T, A from independent counters
// (Eq. RTA) with the closure of Eq. closure; fluence per unit incident flux
// Phi/S0 = F nx ny / N (Eq. Phi_norm, steady source); <Phi>_3D over solid
// voxels (Eq. Phi_MC3D), <Phi>_1D over all voxels (Eq. Phi_MC1D), the pore
// mean, r (Eq. r_def), the concentration ratio and the residual of the
// dilution identity (Eq. dilution); depth profiles per phase (App. B); the
// exit-weighted pore-path statistics of Sec. 3.5(c).  Sums over voxels are
// exact 128-bit integers; only the final divisions are floating point.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "spmc.h"
#include "spmc_internal.cuh"

using namespace spmc;

// ------------------------------------------------------------ errors ----

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? SP_ENOMEM : SP_ECUDA,         \
                        "%s: %s", #expr, cudaGetErrorString(e_));                       \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// ------------------------------------------------------------ handle ----

struct sp_mc {
    int device = 0, sm_count = 0;
    int nx = 0, ny = 0, nz = 0, nbx = 0, nby = 0, nbz = 0;
    double voxel_h = 0, mus = 0, mua = 0, g = 0;   // mus, mua per voxel
    u64 n_vox = 0, n_pore = 0;
    u64 n_field = 0;        // padded voxels of the brick-layout field: 64 per brick
    double porosity = 0;
    // options
    double path_cap_opt = 0, rr_weight = 1e-4, rr_mult = 10.0;
    int field = 1, precision = 32, blocks_opt = 0, threads = 256, smem_bricks_opt = 0;
    u64 n_rec = 0, iter_limit_opt = 0, pid_offset = 0;
    int compact_k = 8;
    int mirror = 0;         // lateral faces: 0 periodic, 1 mirrors
    int variant = 1;        // FP32 kernel: 0 generic template, 1 streamlined
    int steps_per_pass = 8; // streamlined FP32 kernel: voxel steps per warp pass
    u32 bin_mul = 0;        // depth bin by multiply-high, when exact for this nz
    int bin_exact = 0;
    // device memory
    u64 *d_bricks = nullptr, *d_field = nullptr, *d_layer = nullptr, *d_bin_count = nullptr;
    DevTallies *d_tal = nullptr;
    sp_mc_result_t *d_result = nullptr;
    double *d_rec_sites = nullptr, *d_rec_vals = nullptr;
    long long *d_rec_ints = nullptr;
    u64 photons_done = 0;
};

static double default_path_cap(const sp_mc *h) {
    // Eq. tend with n = 1 as a path length in voxels, EMA-scaled optics.
    const double L = h->nz, solid = 1.0 - h->porosity;
    const double s_abs = h->mua > 0 ? 5.0 / h->mua : 0.0;
    const double s_diff = 18.0 * L * L * (h->mua + h->mus * (1.0 - h->g)) * solid;
    return std::fmax(std::fmax(s_abs, s_diff), 4.0 * L);
}

static double path_cap(const sp_mc *h) {
    return h->path_cap_opt > 0 ? h->path_cap_opt : default_path_cap(h);
}

static u64 iter_limit(const sp_mc *h) {
    if (h->iter_limit_opt) return h->iter_limit_opt;
    // face crossings per unit path <= sqrt(3) (plus ties), interactions ~ mu_s
    const double s = path_cap(h);
    const double lim = (3.0 * 1.7320508075688772 + 4.0 * h->mus + 1.0) * s + 1.0e4;
    return lim > 4.0e9 ? 0xffffffffull : (u64)lim;
}

// Depth bin floor(64 iz / nz) as umulhi(64 iz, ceil(2^32 / nz)); used only
// when that is exact for every layer of the volume, which is checked here.
static void set_bin_mul(sp_mc *h) {
    h->bin_mul = 0;
    h->bin_exact = 0;
    const int nz = h->nz;
    if (nz < 2 || (u64)nz * 64 >= (1ull << 32)) return;
    const u64 m = ((1ull << 32) + (u64)nz - 1) / (u64)nz;
    if (m >= (1ull << 32)) return;
    for (int z = 0; z < nz; ++z)
        if ((int)((((u64)z * 64) * m) >> 32) != (int)(((long long)z * kNBin) / nz)) return;
    h->bin_mul = (u32)m;
    h->bin_exact = 1;
}

// FP32 copies of the optics and limits of a launch (computed on the host so
// FP32 kernels never convert doubles inside their loop).
static void fill_f32(const sp_mc *h, double s_max, TransportParams::F32 &f, int &hg_iso,
                     int &small_x) {
    hg_iso = std::fabs(h->g) < 1e-6;
    small_x = h->mua * 1.7320508075688772 <= 0.1;
    f.mus = (float)h->mus;
    f.mua = (float)h->mua;
    f.inv_mus = h->mus > 0 ? (float)(1.0 / h->mus) : 0.0f;
    f.inv_mua = h->mua > 0 ? (float)(1.0 / h->mua) : 0.0f;
    const float gf = (float)h->g;           // the FP32 kernel's g, expressions in FP32
    f.one_m_g2 = 1.0f - gf * gf;
    f.one_p_g2 = 1.0f + gf * gf;
    f.one_m_g = 1.0f - gf;
    f.two_g = 2.0f * gf;
    f.inv_2g = hg_iso ? 0.0f : (float)(1.0 / (2.0 * h->g));
    f.s_max = (float)s_max;
    f.rr_weight = (float)h->rr_weight;
    f.rr_mult = (float)h->rr_mult;
    f.rr_p = (float)(1.0 / h->rr_mult);
    f.rr_gain = (float)(h->rr_mult - 1.0);
    f.hist_scale = (float)(256.0 / (4.0 * (double)h->nz));
}

// --------------------------------------------------------- kernels ------

// One thread per 4x4x4 brick: bit (lz*4+ly)*4+lx set for pore voxels;
// bricks are z-major so the entry slab comes first.
__global__ void pack_bricks_kernel(const uint8_t *__restrict__ mask, u64 *__restrict__ bricks,
                                   int nx, int ny, int nz, int nbx, int nby, int nbz) {
    const long long nb = (long long)nbx * nby * nbz;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((long long)nbx * nby));
        u64 word = 0;
        for (int lz = 0; lz < 4; ++lz) {
            const int z = bz * 4 + lz;
            if (z >= nz) break;
            for (int ly = 0; ly < 4; ++ly) {
                const int y = by * 4 + ly;
                if (y >= ny) break;
                const uint8_t *row = mask + ((size_t)z * ny + y) * (size_t)nx;
                for (int lx = 0; lx < 4; ++lx) {
                    const int x = bx * 4 + lx;
                    if (x >= nx) break;
                    if (row[x]) word |= 1ull << ((lz << 4) | (ly << 2) | lx);
                }
            }
        }
        bricks[b] = word;
    }
}

__device__ __forceinline__ bool is_pore(const u64 *bricks, int nbx, int nby, int x, int y, int z) {
    const u64 w = bricks[((size_t)(z >> 2) * nby + (y >> 2)) * nbx + (x >> 2)];
    return (w >> (((z & 3) << 4) | ((y & 3) << 2) | (x & 3))) & 1ull;
}

// Offset of voxel (x, y, z) in the brick-layout field: 64 consecutive words
// per 4x4x4 brick, bricks z-major, the same bit order as the mask bricks.
__device__ __forceinline__ u64 field_index(int nbx, int nby, int x, int y, int z) {
    const u64 b = ((u64)(z >> 2) * (u64)nby + (u64)(y >> 2)) * (u64)nbx + (u64)(x >> 2);
    return (b << 6) | (u64)(((z & 3) << 4) | ((y & 3) << 2) | (x & 3));
}

__device__ __forceinline__ void add_u128(u64 &lo, u64 &hi, u64 vlo, u64 vhi) {
    lo += vlo;
    hi += vhi + (lo < vlo ? 1ull : 0ull);
}

// Exact per-layer sums of the Q32.32 field per phase: layer[z][phase][lo,hi].
__global__ void layer_sums_kernel(const u64 *__restrict__ field, const u64 *__restrict__ bricks,
                                  int nx, int ny, int nbx, int nby, u64 *__restrict__ layer,
                                  DevTallies *tal) {
    const int z = blockIdx.x;
    const size_t nxy = (size_t)nx * ny;
    u64 lo[2] = {0, 0}, hi[2] = {0, 0};
    bool big = false;
    for (size_t i = threadIdx.x; i < nxy; i += blockDim.x) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        const u64 val = field[field_index(nbx, nby, x, y, z)];
        const int p = is_pore(bricks, nbx, nby, x, y, z) ? 1 : 0;
        add_u128(lo[p], hi[p], val, 0);
        big |= (val >> 62) != 0;
    }
    if (__syncthreads_or(big) && threadIdx.x == 0) atomicOr(&tal->flags, (u32)F_OVERFLOW);
    __shared__ u64 s[32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int p = 0; p < 2; ++p) {
        for (int o = 16; o > 0; o >>= 1) {
            const u64 ol = __shfl_down_sync(0xffffffffu, lo[p], o);
            const u64 oh = __shfl_down_sync(0xffffffffu, hi[p], o);
            add_u128(lo[p], hi[p], ol, oh);
        }
    }
    if (lane == 0) { s[wid][0] = lo[0]; s[wid][1] = hi[0]; s[wid][2] = lo[1]; s[wid][3] = hi[1]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 a[4] = {0, 0, 0, 0};
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            add_u128(a[0], a[1], s[k][0], s[k][1]);
            add_u128(a[2], a[3], s[k][2], s[k][3]);
        }
        for (int k = 0; k < 4; ++k) layer[(size_t)z * 4 + k] = a[k];
    }
}

__device__ __forceinline__ double u128_to_double(u64 lo, u64 hi) {
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

// FP64 normalisation and estimators; one block of 64 threads (one per bin).
__global__ void finalize_kernel(const DevTallies *__restrict__ tal, const u64 *__restrict__ layer,
                                const u64 *__restrict__ bin_count, int nx, int ny, int nz,
                                double porosity, sp_mc_result_t *out) {
    __shared__ u64 s_sum[2][kNBin][2];
    const int b = threadIdx.x;
    const double Q32 = 4294967296.0, Q16 = 65536.0;
    double N = 0;
    for (int k = 0; k < kNBatch; ++k) N += (double)tal->batch[k][B_PHOTONS];
    const double scale = (double)nx * (double)ny / (N * Q32);

    if (b < kNBin) {
        u64 a[2][2] = {{0, 0}, {0, 0}};
        if (layer) {
            for (int z = 0; z < nz; ++z) {
                if ((int)(((long long)z * kNBin) / nz) != b) continue;
                add_u128(a[0][0], a[0][1], layer[(size_t)z * 4 + 0], layer[(size_t)z * 4 + 1]);
                add_u128(a[1][0], a[1][1], layer[(size_t)z * 4 + 2], layer[(size_t)z * 4 + 3]);
            }
        } else {
            for (int p = 0; p < 2; ++p) { a[p][0] = tal->depth[p][b][0]; a[p][1] = tal->depth[p][b][1]; }
        }
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        u64 cnt_all = 0;
        for (int p = 0; p < 2; ++p) {
            s_sum[p][b][0] = a[p][0];
            s_sum[p][b][1] = a[p][1];
            out->raw_depth[p][b][0] = a[p][0];
            out->raw_depth[p][b][1] = a[p][1];
            const u64 c = bin_count[p * kNBin + b];
            out->depth_count[p][b] = c;
            cnt_all += c;
            out->depth[p][b] = c ? u128_to_double(a[p][0], a[p][1]) * scale / (double)c : nan;
        }
        u64 lo = a[0][0], hi = a[0][1];
        add_u128(lo, hi, a[1][0], a[1][1]);
        out->depth[2][b] = cnt_all ? u128_to_double(lo, hi) * scale / (double)cnt_all : nan;
    }
    for (int i = b; i < kNHist; i += blockDim.x) {
        out->raw_hist[i] = tal->hist[i];
        out->pore_hist[i] = (double)tal->hist[i] / Q32 / N;
    }
    __syncthreads();
    if (b != 0) return;

    // weight budget and batch-means standard errors
    const int slots[6] = {B_R, B_T, B_A, B_GATED, B_LOST, B_GAIN};
    double tot[6];
    double se[3];
    for (int q = 0; q < 6; ++q) {
        unsigned __int128 s = 0;
        double m = 0, m2 = 0;
        int nb = 0;
        for (int k = 0; k < kNBatch; ++k) {
            const u64 x = tal->batch[k][slots[q]];
            s += x;
            if (tal->batch[k][B_PHOTONS]) {
                const double v = (double)x / Q32 / (double)tal->batch[k][B_PHOTONS];
                m += v; m2 += v * v; ++nb;
            }
        }
        tot[q] = u128_to_double((u64)s, (u64)(s >> 64)) / Q32 / N;
        if (q < 3) {
            const double mean = m / nb;
            const double var = nb > 1 ? (m2 - nb * mean * mean) / (nb - 1) : 0.0 / 0.0;
            se[q] = sqrt(fmax(var, 0.0) / nb);
        }
    }
    out->R = tot[0]; out->T = tot[1]; out->A = tot[2];
    out->gated = tot[3]; out->lost = tot[4]; out->gain = tot[5];
    out->closure = tot[0] + tot[1] + tot[2] + tot[3] + tot[4] - tot[5];
    out->R_se = se[0]; out->T_se = se[1]; out->A_se = se[2];
    for (int k = 0; k < kNBatch; ++k) {
        out->raw_R[k] = tal->batch[k][B_R];
        out->raw_T[k] = tal->batch[k][B_T];
        out->raw_A[k] = tal->batch[k][B_A];
        out->raw_gated[k] = tal->batch[k][B_GATED];
        out->raw_lost[k] = tal->batch[k][B_LOST];
        out->raw_gain[k] = tal->batch[k][B_GAIN];
        out->batch_photons[k] = tal->batch[k][B_PHOTONS];
    }

    // phase means (exact 128-bit totals, then FP64)
    unsigned __int128 ts = 0, tp = 0;
    u64 cs = 0, cp = 0;
    for (int k = 0; k < kNBin; ++k) {
        ts += ((unsigned __int128)s_sum[0][k][1] << 64) | s_sum[0][k][0];
        tp += ((unsigned __int128)s_sum[1][k][1] << 64) | s_sum[1][k][0];
        cs += bin_count[k];
        cp += bin_count[kNBin + k];
    }
    const double sum_s = u128_to_double((u64)ts, (u64)(ts >> 64)) * scale;
    const double sum_p = u128_to_double((u64)tp, (u64)(tp >> 64)) * scale;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    out->phi_3d = cs ? sum_s / (double)cs : nan;
    out->phi_pore = cp ? sum_p / (double)cp : nan;
    out->phi_1d = (sum_s + sum_p) / (double)(cs + cp);
    out->r = out->phi_pore / out->phi_3d;
    out->ratio = out->phi_3d / out->phi_1d;
    out->identity_residual = out->ratio * (porosity * out->r + (1.0 - porosity)) - 1.0;

    // exit-weighted pore path
    const double sw = u128_to_double(tal->sums[0], tal->sums[1]);
    const double swp = u128_to_double(tal->sums[2], tal->sums[3]);
    const double swp2 = u128_to_double(tal->sums[4], tal->sums[5]);
    out->escape_weight = sw / Q32 / N;
    out->pore_path_mean = sw > 0 ? swp / sw : nan;
    out->pore_path_m2 = sw > 0 ? (swp2 / Q16) / (sw / Q32) : nan;
    double h_all = 0, h_gt = 0;
    for (int k = 0; k < kNHist; ++k) {
        h_all += (double)tal->hist[k];
        if (k >= 64) h_gt += (double)tal->hist[k];
    }
    out->p_pore_gt_L = h_all > 0 ? h_gt / h_all : nan;
    for (int k = 0; k < 2; ++k) {
        out->raw_sum_w[k] = tal->sums[k];
        out->raw_sum_wP[k] = tal->sums[2 + k];
        out->raw_sum_wP2[k] = tal->sums[4 + k];
    }
    out->launched = tal->counts[C_LAUNCHED];
    out->interactions = tal->counts[C_INTERACT];
    out->scatters = tal->counts[C_SCATTER];
    out->rr_survive = tal->counts[C_RR_SURV];
    out->rr_kill = tal->counts[C_RR_KILL];
    out->exit_R = tal->counts[C_EXIT_R];
    out->exit_T = tal->counts[C_EXIT_T];
    out->gated_n = tal->counts[C_GATED];
    out->steps = tal->counts[C_STEPS];
    out->solid_steps = tal->counts[C_SOLID_STEPS];
}

// Field in x-fastest order: Phi/S0 as float/double, or the raw Q32.32 words
// (T = u64, no scaling).
template <typename T>
__global__ void fluence_kernel(const u64 *__restrict__ field, T *__restrict__ out, int nx, int ny,
                               int nz, int nbx, int nby, const DevTallies *__restrict__ tal) {
    double scale = 1.0;
    if constexpr (!std::is_same<T, u64>::value) {
        double N = 0;
        for (int k = 0; k < kNBatch; ++k) N += (double)tal->batch[k][B_PHOTONS];
        scale = (double)nx * (double)ny / (N * 4294967296.0);
    }
    const size_t n = (size_t)nx * ny * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const u64 val = field[field_index(nbx, nby, x, y, z)];
        if constexpr (std::is_same<T, u64>::value) out[i] = val;
        else out[i] = (T)((double)val * scale);
    }
}

// ------------------------------------------------------------ helpers ---

static void free_all(sp_mc *h) {
    cudaFree(h->d_bricks);
    cudaFree(h->d_field);
    cudaFree(h->d_layer);
    cudaFree(h->d_bin_count);
    cudaFree(h->d_tal);
    cudaFree(h->d_result);
    cudaFree(h->d_rec_sites);
    cudaFree(h->d_rec_ints);
    cudaFree(h->d_rec_vals);
    h->d_bricks = h->d_field = h->d_layer = h->d_bin_count = nullptr;
    h->d_tal = nullptr;
    h->d_result = nullptr;
    h->d_rec_sites = h->d_rec_vals = nullptr;
    h->d_rec_ints = nullptr;
}

static int alloc_field(sp_mc *h) {
    if (!h->field || h->d_field) return SP_OK;
    CUDA_TRY(cudaMalloc(&h->d_field, h->n_field * sizeof(u64)));
    CUDA_TRY(cudaMemset(h->d_field, 0, h->n_field * sizeof(u64)));
    return SP_OK;
}

static int alloc_records(sp_mc *h, u64 n) {
    cudaFree(h->d_rec_sites);
    cudaFree(h->d_rec_ints);
    cudaFree(h->d_rec_vals);
    h->d_rec_sites = h->d_rec_vals = nullptr;
    h->d_rec_ints = nullptr;
    h->n_rec = 0;
    if (!n) return SP_OK;
    CUDA_TRY(cudaMalloc(&h->d_rec_sites, n * 24 * sizeof(double)));
    CUDA_TRY(cudaMalloc(&h->d_rec_ints, n * 4 * sizeof(long long)));
    CUDA_TRY(cudaMalloc(&h->d_rec_vals, n * 4 * sizeof(double)));
    CUDA_TRY(cudaMemset(h->d_rec_sites, 0xff, n * 24 * sizeof(double)));   // NaN
    CUDA_TRY(cudaMemset(h->d_rec_ints, 0, n * 4 * sizeof(long long)));
    CUDA_TRY(cudaMemset(h->d_rec_vals, 0, n * 4 * sizeof(double)));
    h->n_rec = n;
    return SP_OK;
}

static int check_handle(const sp_mc *h) {
    if (!h) return fail(SP_EINVAL, "null handle");
    return SP_OK;
}

// --------------------------------------------------------------- ABI ----

extern "C" {

const char *sp_mc_last_error(void) { return g_err.c_str(); }

const char *sp_mc_version(void) { return "spmc 0.1.0 sm_103a"; }

size_t sp_mc_result_size(void) { return sizeof(sp_mc_result_t); }

sp_mc_t *sp_mc_create(const uint8_t *mask, int nx, int ny, int nz, double voxel_h, double mu_s,
                      double mu_a, double g) {
    g_err.clear();
    if (!mask) { fail(SP_EINVAL, "mask is NULL"); return nullptr; }
    if (nx < 1 || ny < 1 || nz < 1) { fail(SP_EINVAL, "dimensions must be >= 1"); return nullptr; }
    const u64 n_vox = (u64)nx * (u64)ny * (u64)nz;
    const u64 n_bricks_req = (u64)((nx + 3) / 4) * (u64)((ny + 3) / 4) * (u64)((nz + 3) / 4);
    if (n_bricks_req >= (1ull << 31)) { fail(SP_EINVAL, "the volume must have fewer than 2^31 4x4x4 bricks (about 2^37 voxels)"); return nullptr; }
    if (!(voxel_h > 0) || !std::isfinite(voxel_h)) { fail(SP_EINVAL, "voxel_h must be > 0"); return nullptr; }
    if (!(mu_s >= 0) || !(mu_a >= 0) || !std::isfinite(mu_s) || !std::isfinite(mu_a)) {
        fail(SP_EINVAL, "mu_s and mu_a must be finite and >= 0");
        return nullptr;
    }
    if (!(g > -1.0 && g < 1.0)) { fail(SP_EINVAL, "g must lie in (-1, 1)"); return nullptr; }

    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1 || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        fail(SP_ECUDA, "no CUDA device available");
        return nullptr;
    }
    sp_mc *h = new (std::nothrow) sp_mc();
    if (!h) { fail(SP_ENOMEM, "host allocation failed"); return nullptr; }
    h->device = dev;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
    h->nx = nx; h->ny = ny; h->nz = nz;
    h->nbx = (nx + 3) / 4; h->nby = (ny + 3) / 4; h->nbz = (nz + 3) / 4;
    h->voxel_h = voxel_h;
    h->mus = mu_s * voxel_h;
    h->mua = mu_a * voxel_h;
    h->g = g;
    h->n_vox = n_vox;
    h->n_field = (u64)h->nbx * h->nby * h->nbz * 64;

    // voxel counts per (phase, depth bin), exact, on the host
    std::vector<u64> cnt(2 * kNBin, 0);
    u64 n_pore = 0;
    for (int z = 0; z < nz; ++z) {
        const uint8_t *layer = mask + (size_t)z * nx * ny;
        u64 p = 0;
        for (size_t i = 0; i < (size_t)nx * ny; ++i) p += layer[i] != 0;
        const int b = (int)(((long long)z * kNBin) / nz);
        cnt[kNBin + b] += p;
        cnt[b] += (u64)nx * ny - p;
        n_pore += p;
    }
    h->n_pore = n_pore;
    h->porosity = (double)n_pore / (double)n_vox;
    set_bin_mul(h);

    auto bail = [&](int code) -> sp_mc_t * {
        (void)code;
        free_all(h);
        delete h;
        return nullptr;
    };
    const u64 n_bricks = (u64)h->nbx * h->nby * h->nbz;
    uint8_t *d_mask = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&d_mask, n_vox)) != cudaSuccess ||
        (e = cudaMalloc(&h->d_bricks, n_bricks * sizeof(u64))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_tal, sizeof(DevTallies))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_result, sizeof(sp_mc_result_t))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_layer, (size_t)nz * 4 * sizeof(u64))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_bin_count, 2 * kNBin * sizeof(u64))) != cudaSuccess) {
        cudaFree(d_mask);
        fail(e == cudaErrorMemoryAllocation ? SP_ENOMEM : SP_ECUDA, "allocation: %s", cudaGetErrorString(e));
        return bail(0);
    }
    // a1: upload and bit-pack the mask on the device
    if ((e = cudaMemcpy(d_mask, mask, n_vox, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_bin_count, cnt.data(), cnt.size() * sizeof(u64), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(h->d_tal, 0, sizeof(DevTallies))) != cudaSuccess) {
        cudaFree(d_mask);
        fail(SP_ECUDA, "upload: %s", cudaGetErrorString(e));
        return bail(0);
    }
    const int pack_blocks = (int)std::min<u64>((n_bricks + 255) / 256, 65535ull * 8);
    pack_bricks_kernel<<<pack_blocks, 256>>>(d_mask, h->d_bricks, nx, ny, nz, h->nbx, h->nby, h->nbz);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
        cudaFree(d_mask);
        fail(SP_ECUDA, "mask packing: %s", cudaGetErrorString(e));
        return bail(0);
    }
    cudaFree(d_mask);
    if (alloc_field(h) != SP_OK) return bail(0);
    return h;
}

void sp_mc_destroy(sp_mc_t *h) {
    if (!h) return;
    DeviceGuard guard(h->device);
    free_all(h);
    delete h;
}

int sp_mc_set_option(sp_mc_t *h, int key, double value) {
    if (check_handle(h)) return SP_EINVAL;
    DeviceGuard guard(h->device);
    if (!std::isfinite(value)) return fail(SP_EINVAL, "option value must be finite");
    switch (key) {
    case SP_OPT_PATH_CAP: h->path_cap_opt = value; return SP_OK;
    case SP_OPT_RR_WEIGHT:
        if (value < 0) return fail(SP_EINVAL, "roulette threshold must be >= 0");
        h->rr_weight = value; return SP_OK;
    case SP_OPT_RR_MULT:
        if (value < 1) return fail(SP_EINVAL, "roulette multiplier must be >= 1");
        h->rr_mult = value; return SP_OK;
    case SP_OPT_TALLY_FIELD: {
        const int f = value != 0;
        if (f == h->field) return SP_OK;
        if (h->photons_done) return fail(SP_EINVAL, "tally mode can only change before the first run");
        h->field = f;
        if (!f) { cudaFree(h->d_field); h->d_field = nullptr; return SP_OK; }
        return alloc_field(h);
    }
    case SP_OPT_PRECISION: {
        const int p = (int)value;
        if (p != 32 && p != 64) return fail(SP_EINVAL, "precision must be 32 or 64");
        if (p != h->precision && h->photons_done)
            return fail(SP_EINVAL, "precision can only change before the first run");
        h->precision = p; return SP_OK;
    }
    case SP_OPT_RECORDS:
        if (value < 0 || value > 1e8) return fail(SP_EINVAL, "records must be in [0, 1e8]");
        if (h->photons_done) return fail(SP_EINVAL, "records can only be set before the first run");
        return alloc_records(h, (u64)value);
    case SP_OPT_BLOCKS:
        if (value < 0 || value > 1e6) return fail(SP_EINVAL, "blocks out of range");
        h->blocks_opt = (int)value; return SP_OK;
    case SP_OPT_THREADS: {
        const int t = (int)value;
        if (t < 32 || t > 256 || t % 32) return fail(SP_EINVAL, "threads must be a multiple of 32 in [32, 256]");
        h->threads = t; return SP_OK;
    }
    case SP_OPT_ITER_LIMIT:
        if (value < 0) return fail(SP_EINVAL, "iteration limit must be >= 0");
        h->iter_limit_opt = (u64)value; return SP_OK;
    case SP_OPT_SMEM_BRICKS:
        if (value < -1 || value > 1e7) return fail(SP_EINVAL, "smem bricks out of range");
        h->smem_bricks_opt = (int)value; return SP_OK;
    case SP_OPT_COMPACT:
        if (value < 1 || value > 32) return fail(SP_EINVAL, "compaction threshold must be in [1, 32]");
        h->compact_k = (int)value; return SP_OK;
    case SP_OPT_LATERAL_BC:
        if (value != 0 && value != 1) return fail(SP_EINVAL, "lateral BC must be 0 (periodic) or 1 (mirror)");
        h->mirror = (int)value; return SP_OK;
    case SP_OPT_PID_OFFSET:
        if (value < 0 || value > 1.8e19) return fail(SP_EINVAL, "photon id offset out of range");
        if (h->photons_done) return fail(SP_EINVAL, "the photon id offset can only be set before the first run");
        h->pid_offset = (u64)value; return SP_OK;
    case SP_OPT_KERNEL:
        if (value != 0 && value != 1) return fail(SP_EINVAL, "kernel variant must be 0 or 1");
        h->variant = (int)value; return SP_OK;
    case SP_OPT_STEPS_PER_PASS:
        if (value < 1 || value > 64) return fail(SP_EINVAL, "steps per pass must be in [1, 64]");
        h->steps_per_pass = (int)value; return SP_OK;
    default: return fail(SP_EINVAL, "unknown option %d", key);
    }
}

int sp_mc_get_option(const sp_mc_t *h, int key, double *value) {
    if (check_handle(h)) return SP_EINVAL;
    if (!value) return fail(SP_EINVAL, "value is NULL");
    switch (key) {
    case SP_OPT_PATH_CAP: *value = path_cap(h); return SP_OK;
    case SP_OPT_RR_WEIGHT: *value = h->rr_weight; return SP_OK;
    case SP_OPT_RR_MULT: *value = h->rr_mult; return SP_OK;
    case SP_OPT_TALLY_FIELD: *value = h->field; return SP_OK;
    case SP_OPT_PRECISION: *value = h->precision; return SP_OK;
    case SP_OPT_RECORDS: *value = (double)h->n_rec; return SP_OK;
    case SP_OPT_BLOCKS: *value = h->blocks_opt; return SP_OK;
    case SP_OPT_THREADS: *value = h->threads; return SP_OK;
    case SP_OPT_ITER_LIMIT: *value = (double)iter_limit(h); return SP_OK;
    case SP_OPT_SMEM_BRICKS: *value = h->smem_bricks_opt; return SP_OK;
    case SP_OPT_PID_OFFSET: *value = (double)h->pid_offset; return SP_OK;
    case SP_OPT_COMPACT: *value = h->compact_k; return SP_OK;
    case SP_OPT_LATERAL_BC: *value = h->mirror; return SP_OK;
    case SP_OPT_KERNEL: *value = h->variant; return SP_OK;
    case SP_OPT_STEPS_PER_PASS: *value = h->steps_per_pass; return SP_OK;
    default: return fail(SP_EINVAL, "unknown option %d", key);
    }
}

// One single-problem transport launch of n_photons from photon id pid_begin
// (or from *pid_begin_dev when it is set), stream-ordered and capturable.
static int launch_run(sp_mc *h, u64 n_photons, u64 seed, u64 pid_begin, const u64 *pid_begin_dev,
                      cudaStream_t s) {

    const u64 n_bricks = (u64)h->nbx * h->nby * h->nbz;
    int smem_bricks = h->smem_bricks_opt;
    if (smem_bricks < 0) smem_bricks = (int)std::min<u64>(n_bricks, 12288);   // auto: 96 KiB
    smem_bricks = (int)std::min<u64>((u64)smem_bricks, n_bricks);
    const size_t smem = (size_t)smem_bricks * sizeof(u64);
    const bool f64 = h->precision == 64;
    const bool field = h->field != 0;
    if (smem > 48 * 1024) {
        CUDA_TRY(cudaFuncSetAttribute(f64 ? kernel_f64(field, h->mirror != 0)
                                          : kernel_f32(field, h->mirror != 0, h->variant),
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    int blocks = h->blocks_opt;
    if (blocks <= 0) {
        int per_sm = 0;
        CUDA_TRY(f64 ? occupancy_f64(field, h->mirror != 0, h->threads, smem, &per_sm)
                     : occupancy_f32(field, h->mirror != 0, h->variant, h->threads, smem, &per_sm));
        if (per_sm < 1) return fail(SP_ECUDA, "transport kernel cannot be resident with %zu B smem", smem);
        blocks = per_sm * h->sm_count;
    }

    TransportParams p{};
    p.bricks = h->d_bricks;
    p.field = field ? h->d_field : nullptr;
    p.tal = h->d_tal;
    p.rec_sites = h->d_rec_sites;
    p.rec_ints = h->d_rec_ints;
    p.rec_vals = h->d_rec_vals;
    p.n_rec = h->n_rec;
    p.nx = h->nx; p.ny = h->ny; p.nz = h->nz;
    p.nbx = h->nbx; p.nby = h->nby; p.nbz = h->nbz;
    p.smem_bricks = smem_bricks;
    p.key0 = (u32)seed;
    p.key1 = (u32)(seed >> 32);
    p.pid_begin = pid_begin;
    p.pid_begin_dev = pid_begin_dev;
    p.rec_base = h->pid_offset;
    p.n_photons = n_photons;
    p.mus = h->mus; p.mua = h->mua; p.g = h->g;
    p.s_max = path_cap(h);
    p.rr_weight = h->rr_weight;
    p.rr_mult = h->rr_mult;
    p.iter_limit = iter_limit(h);
    p.compact_k = h->compact_k;
    p.mirror = h->mirror;
    p.steps_per_pass = h->steps_per_pass;
    p.bin_mul = h->bin_mul;
    p.bin_exact = h->bin_exact;
    fill_f32(h, p.s_max, p.f32, p.hg_iso, p.small_x);

    LaunchExtras ex;
    ex.variant = h->variant;
    CUDA_TRY(cudaMemsetAsync(&h->d_tal->next, 0, sizeof(u64), s));
    CUDA_TRY(f64 ? launch_transport_f64(p, field, blocks, h->threads, smem, s)
                 : launch_transport_f32(p, field, blocks, h->threads, smem, s, ex));
    return SP_OK;
}

int sp_mc_run(sp_mc_t *h, uint64_t n_photons, uint64_t seed, void *stream) {
    if (check_handle(h)) return SP_EINVAL;
    if (n_photons == 0) return SP_OK;
    if (h->pid_offset + h->photons_done + n_photons < h->pid_offset + h->photons_done)
        return fail(SP_EINVAL, "photon id overflow");
    DeviceGuard guard(h->device);
    if (!guard.ok) return fail(SP_ECUDA, "cannot select device %d", h->device);
    const int rc = launch_run(h, n_photons, seed, h->pid_offset + h->photons_done, nullptr,
                              reinterpret_cast<cudaStream_t>(stream));
    if (rc) return rc;
    h->photons_done += n_photons;
    return SP_OK;
}

int sp_mc_tallies(sp_mc_t *h, sp_mc_result_t *out, void *stream) {
    if (check_handle(h)) return SP_EINVAL;
    if (!out) return fail(SP_EINVAL, "out is NULL");
    DeviceGuard guard(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (h->field) {
        layer_sums_kernel<<<h->nz, 256, 0, s>>>(h->d_field, h->d_bricks, h->nx, h->ny, h->nbx, h->nby,
                                                h->d_layer, h->d_tal);
        CUDA_TRY(cudaGetLastError());
    }
    finalize_kernel<<<1, kNBin, 0, s>>>(h->d_tal, h->field ? h->d_layer : nullptr, h->d_bin_count,
                                        h->nx, h->ny, h->nz, h->porosity, h->d_result);
    CUDA_TRY(cudaGetLastError());
    u32 flags = 0;
    CUDA_TRY(cudaMemcpyAsync(out, h->d_result, sizeof(sp_mc_result_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&flags, &h->d_tal->flags, sizeof(u32), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    out->photons = h->photons_done;
    out->precision = h->precision;
    out->s_max = path_cap(h);
    out->porosity = h->porosity;
    out->status = SP_OK;
    if (flags & F_ITER_LIMIT) out->status = SP_ESTEPLIMIT;
    else if (flags & F_OVERFLOW) out->status = SP_EOVERFLOW;
    if (out->status != SP_OK)
        return fail(out->status, out->status == SP_ESTEPLIMIT ? "a photon hit the iteration limit"
                                                              : "a voxel tally neared 2^62");
    return SP_OK;
}

static int field_out(sp_mc *h, void *dst, int dtype, int on_device, cudaStream_t s) {
    // dtype 0 f64, 1 f32, 2 raw u64
    const size_t esz = dtype == 1 ? 4 : 8;
    const size_t bytes = h->n_vox * esz;
    void *d_out = dst;
    if (!on_device) CUDA_TRY(cudaMalloc(&d_out, bytes));
    const int blocks = h->sm_count * 8;
    if (dtype == 0)
        fluence_kernel<double><<<blocks, 256, 0, s>>>(h->d_field, (double *)d_out, h->nx, h->ny, h->nz, h->nbx, h->nby, h->d_tal);
    else if (dtype == 1)
        fluence_kernel<float><<<blocks, 256, 0, s>>>(h->d_field, (float *)d_out, h->nx, h->ny, h->nz, h->nbx, h->nby, h->d_tal);
    else
        fluence_kernel<u64><<<blocks, 256, 0, s>>>(h->d_field, (u64 *)d_out, h->nx, h->ny, h->nz, h->nbx, h->nby, h->d_tal);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !on_device) {
        e = cudaMemcpyAsync(dst, d_out, bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (!on_device) cudaFree(d_out);
    if (e != cudaSuccess) return fail(SP_ECUDA, "field output: %s", cudaGetErrorString(e));
    return SP_OK;
}

int sp_mc_fluence(sp_mc_t *h, void *dst, int dtype, int on_device, void *stream) {
    if (check_handle(h)) return SP_EINVAL;
    if (!dst) return fail(SP_EINVAL, "dst is NULL");
    if (!h->field) return fail(SP_EINVAL, "the voxel field tally is disabled");
    if (dtype != 0 && dtype != 1) return fail(SP_EINVAL, "dtype must be 0 (f64) or 1 (f32)");
    if (!h->photons_done) return fail(SP_EINVAL, "no photons have been run");
    DeviceGuard guard(h->device);
    return field_out(h, dst, dtype, on_device, reinterpret_cast<cudaStream_t>(stream));
}

int sp_mc_raw_field(sp_mc_t *h, uint64_t *dst, int on_device, void *stream) {
    if (check_handle(h)) return SP_EINVAL;
    if (!dst) return fail(SP_EINVAL, "dst is NULL");
    if (!h->field) return fail(SP_EINVAL, "the voxel field tally is disabled");
    DeviceGuard guard(h->device);
    return field_out(h, dst, 2, on_device, reinterpret_cast<cudaStream_t>(stream));
}

int sp_mc_records(sp_mc_t *h, uint64_t n, double *sites, int64_t *ints, double *vals, void *stream) {
    if (check_handle(h)) return SP_EINVAL;
    if (n > h->n_rec) return fail(SP_EINVAL, "only %llu photons are recorded", (unsigned long long)h->n_rec);
    if (!n) return SP_OK;
    DeviceGuard guard(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (sites) CUDA_TRY(cudaMemcpyAsync(sites, h->d_rec_sites, n * 24 * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (ints) CUDA_TRY(cudaMemcpyAsync(ints, h->d_rec_ints, n * 4 * sizeof(long long), cudaMemcpyDeviceToHost, s));
    if (vals) CUDA_TRY(cudaMemcpyAsync(vals, h->d_rec_vals, n * 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SP_OK;
}

int sp_mc_reset(sp_mc_t *h, void *stream) {
    if (check_handle(h)) return SP_EINVAL;
    DeviceGuard guard(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(h->d_tal, 0, sizeof(DevTallies), s));
    if (h->d_field) CUDA_TRY(cudaMemsetAsync(h->d_field, 0, h->n_field * sizeof(u64), s));
    if (h->n_rec) {
        CUDA_TRY(cudaMemsetAsync(h->d_rec_sites, 0xff, h->n_rec * 24 * sizeof(double), s));
        CUDA_TRY(cudaMemsetAsync(h->d_rec_ints, 0, h->n_rec * 4 * sizeof(long long), s));
        CUDA_TRY(cudaMemsetAsync(h->d_rec_vals, 0, h->n_rec * 4 * sizeof(double), s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    h->photons_done = 0;
    return SP_OK;
}

// Checkpoint layout: header (magic, version, nx, ny, nz, field, photons_done),
// the DevTallies block, then the Q32.32 field when enabled.
struct CkptHeader {
    u64 magic, version, nx, ny, nz, field, photons_done, tal_bytes;
};
static const u64 kMagic = 0x54504b43434d5053ull;   // "SPMCCKPT"

size_t sp_mc_checkpoint_size(const sp_mc_t *h) {
    if (!h) return 0;
    return sizeof(CkptHeader) + sizeof(DevTallies) + (h->field ? h->n_field * sizeof(u64) : 0);
}

int sp_mc_checkpoint(sp_mc_t *h, void *buf, size_t size, void *stream) {
    if (check_handle(h)) return SP_EINVAL;
    if (!buf || size < sp_mc_checkpoint_size(h)) return fail(SP_EINVAL, "checkpoint buffer too small");
    DeviceGuard guard(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CkptHeader hd{kMagic, 2, (u64)h->nx, (u64)h->ny, (u64)h->nz, (u64)h->field, h->photons_done,
                  sizeof(DevTallies)};
    std::memcpy(buf, &hd, sizeof hd);
    char *p = static_cast<char *>(buf) + sizeof hd;
    CUDA_TRY(cudaMemcpyAsync(p, h->d_tal, sizeof(DevTallies), cudaMemcpyDeviceToHost, s));
    if (h->field)
        CUDA_TRY(cudaMemcpyAsync(p + sizeof(DevTallies), h->d_field, h->n_field * sizeof(u64),
                                 cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SP_OK;
}

int sp_mc_restore(sp_mc_t *h, const void *buf, size_t size, void *stream) {
    if (check_handle(h)) return SP_EINVAL;
    if (!buf || size < sizeof(CkptHeader)) return fail(SP_EINVAL, "checkpoint too small");
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (hd.magic != kMagic || hd.version != 2 || hd.tal_bytes != sizeof(DevTallies))
        return fail(SP_EINVAL, "not a compatible checkpoint");
    if (hd.nx != (u64)h->nx || hd.ny != (u64)h->ny || hd.nz != (u64)h->nz || hd.field != (u64)h->field)
        return fail(SP_EINVAL, "checkpoint was taken on a different geometry or tally mode");
    if (size < sp_mc_checkpoint_size(h)) return fail(SP_EINVAL, "checkpoint truncated");
    DeviceGuard guard(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const char *p = static_cast<const char *>(buf) + sizeof hd;
    CUDA_TRY(cudaMemcpyAsync(h->d_tal, p, sizeof(DevTallies), cudaMemcpyHostToDevice, s));
    if (h->field)
        CUDA_TRY(cudaMemcpyAsync(h->d_field, p + sizeof(DevTallies), h->n_field * sizeof(u64),
                                 cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    h->photons_done = hd.photons_done;
    return SP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Allocation-free entry point.
//
// For callers that may not allocate device memory themselves, e.g. code
// embedded in a host application whose own allocator owns all device memory,
// or latency-critical loops that cannot afford an allocator call.  Its
// working memory is the fixed array below, which every GPU that loads this
// library keeps until the process exits.  The paper has no counterpart to
// this; it is an interface convenience around the same transport kernel.
// ------------------------------------------------------------------------

namespace {

constexpr u64 kNoAllocMaxBricks = 1ull << 18;     // 262144 bricks = 2^24 voxels (256^3)
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffBricks = 0;
constexpr size_t kOffTal = align_up(kOffBricks + kNoAllocMaxBricks * sizeof(u64));
constexpr size_t kOffCount = align_up(kOffTal + sizeof(DevTallies));
constexpr size_t kOffResult = align_up(kOffCount + 2 * kNBin * sizeof(u64));
constexpr size_t kScratchBytes = align_up(kOffResult + sizeof(sp_mc_result_t));

}  // namespace

// The scratch array (about 2.03 MiB).  Host code must not pass its name to a
// kernel: on the host it is only a stand-in symbol, so its device address is
// looked up with cudaGetSymbolAddress on the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Pore voxels per depth bin (phase 1) and solid voxels (phase 0).
__global__ void noalloc_count_kernel(const uint8_t *__restrict__ mask, int nx, int ny, int nz,
                                     u64 *__restrict__ bin_count) {
    __shared__ u64 s_cnt[2 * kNBin];
    for (int i = threadIdx.x; i < 2 * kNBin; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    const size_t nxy = (size_t)nx * ny, n = nxy * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(i / nxy);
        const int b = (int)(((long long)z * kNBin) / nz);
        atomicAdd(&s_cnt[(mask[i] != 0 ? kNBin : 0) + b], 1ull);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kNBin; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(&bin_count[i], s_cnt[i]);
}

extern "C" int sp_mc_simulate_noalloc(const uint8_t *d_mask, int nx, int ny, int nz,
                                      double voxel_h, double mu_s, double mu_a, double g,
                                      uint64_t n_photons, uint64_t seed, sp_mc_result_t *out,
                                      void *stream) {
    // Messages here stay within the short-string capacity, so reporting a
    // failure does not allocate either.
    if (!d_mask || !out) return fail(SP_EINVAL, "null pointer");
    if (nx < 1 || ny < 1 || nz < 1 || !(voxel_h > 0) || !std::isfinite(voxel_h) ||
        !(mu_s >= 0) || !(mu_a >= 0) || !std::isfinite(mu_s) || !std::isfinite(mu_a) ||
        !(g > -1.0 && g < 1.0))
        return fail(SP_EINVAL, "bad argument");
    const u64 nbx = (u64)(nx + 3) / 4, nby = (u64)(ny + 3) / 4, nbz = (u64)(nz + 3) / 4;
    if (nbx * nby * nbz > kNoAllocMaxBricks) return fail(SP_EINVAL, "size too large");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(SP_ECUDA, "no CUDA device");
    }
    // Set-up, repeated on every call with the caller's device current: the
    // array's device address.  The lookup allocates nothing, and doing it
    // each time keeps the address right after a device reset or a new
    // context, where the module (and the array) may have moved.
    void *sym = nullptr;
    if (cudaGetSymbolAddress(&sym, g_noalloc_scratch) != cudaSuccess || !sym) {
        cudaGetLastError();
        return fail(SP_ECUDA, "symbol lookup");
    }
    unsigned char *base = static_cast<unsigned char *>(sym);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    u64 *bricks = reinterpret_cast<u64 *>(base + kOffBricks);
    DevTallies *tal = reinterpret_cast<DevTallies *>(base + kOffTal);
    u64 *bin_count = reinterpret_cast<u64 *>(base + kOffCount);
    sp_mc_result_t *d_result = reinterpret_cast<sp_mc_result_t *>(base + kOffResult);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(SP_ECUDA, "CUDA error");

    // The array keeps the previous call's contents: clear the tallies and
    // counts, repack the mask.
    const u64 n_bricks = nbx * nby * nbz;
    if (cudaMemsetAsync(tal, 0, sizeof(DevTallies), s) != cudaSuccess ||
        cudaMemsetAsync(bin_count, 0, 2 * kNBin * sizeof(u64), s) != cudaSuccess)
        return fail(SP_ECUDA, "CUDA error");
    pack_bricks_kernel<<<(int)((n_bricks + 255) / 256), 256, 0, s>>>(d_mask, bricks, nx, ny, nz,
                                                                       (int)nbx, (int)nby, (int)nbz);
    noalloc_count_kernel<<<2 * sms, 256, 0, s>>>(d_mask, nx, ny, nz, bin_count);
    u64 cnt[2 * kNBin];
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(cnt, bin_count, sizeof cnt, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SP_ECUDA, "CUDA error");
    u64 n_pore = 0;
    for (int b = 0; b < kNBin; ++b) n_pore += cnt[kNBin + b];
    const double porosity = (double)n_pore / ((double)nx * (double)ny * (double)nz);

    // Default options of a fresh handle, profile-only tally (no voxel field);
    // the launch constants come from the same helpers as sp_mc_run's.
    sp_mc tmp;
    tmp.nx = nx; tmp.ny = ny; tmp.nz = nz;
    tmp.mus = mu_s * voxel_h; tmp.mua = mu_a * voxel_h; tmp.g = g;
    tmp.porosity = porosity;
    set_bin_mul(&tmp);
    int per_sm = 0;
    if (occupancy_f32(false, false, tmp.variant, tmp.threads, 0, &per_sm) != cudaSuccess || per_sm < 1)
        return fail(SP_ECUDA, "CUDA error");

    TransportParams p{};
    p.bricks = bricks;
    p.field = nullptr;
    p.tal = tal;
    p.nx = nx; p.ny = ny; p.nz = nz;
    p.nbx = (int)nbx; p.nby = (int)nby; p.nbz = (int)nbz;
    p.smem_bricks = 0;
    p.key0 = (u32)seed;
    p.key1 = (u32)(seed >> 32);
    p.pid_begin = 0;
    p.n_photons = n_photons;
    p.mus = tmp.mus; p.mua = tmp.mua; p.g = g;
    p.s_max = path_cap(&tmp);
    p.rr_weight = tmp.rr_weight;
    p.rr_mult = tmp.rr_mult;
    p.iter_limit = iter_limit(&tmp);
    p.compact_k = tmp.compact_k;
    p.mirror = 0;
    p.steps_per_pass = tmp.steps_per_pass;
    p.bin_mul = tmp.bin_mul;
    p.bin_exact = tmp.bin_exact;
    fill_f32(&tmp, p.s_max, p.f32, p.hg_iso, p.small_x);
    LaunchExtras ex;
    ex.variant = tmp.variant;

    if (n_photons > 0 && launch_transport_f32(p, false, per_sm * sms, tmp.threads, 0, s, ex) != cudaSuccess)
        return fail(SP_ECUDA, "CUDA error");
    finalize_kernel<<<1, kNBin, 0, s>>>(tal, nullptr, bin_count, nx, ny, nz, porosity, d_result);
    u32 flags = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(out, d_result, sizeof(sp_mc_result_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&flags, &tal->flags, sizeof flags, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SP_ECUDA, "CUDA error");
    out->photons = n_photons;
    out->precision = 32;
    out->s_max = p.s_max;
    out->porosity = porosity;
    out->status = (flags & F_ITER_LIMIT) ? SP_ESTEPLIMIT : SP_OK;
    if (out->status != SP_OK) return fail(out->status, "step limit");
    return SP_OK;
}

// ------------------------------------------------------------------------
// Batched launches: many masks of uneven size and optics in one persistent
// launch (a device table of problems, one shared photon-claim counter), an
// optional CUDA graph of {counter reset, transport, photon-id advance} that
// later runs replay, and a host autotuner over threads per CTA, CTAs per SM
// and the warp compaction threshold.
// ------------------------------------------------------------------------

// After a batched launch, every problem's next photon ids start past the
// photons just run (lets a captured graph be replayed as further runs).
__global__ void batch_advance_kernel(BatchProblem *table, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) table[i].pid_begin += table[i].n_photons;
}

struct sp_mc_batch {
    int device = 0, sm_count = 0, n = 0;
    std::vector<sp_mc *> h;
    std::vector<BatchProblem> table;
    BatchProblem *d_table = nullptr;
    u64 *d_next = nullptr;
    int threads = 128, blocks_per_sm = 0, compact_k = 8, use_graph = 1, mode = 0;
    int variant = 1, steps_per_pass = 8;   // one-launch kernel and its steps per pass
    u32 chunk = 128;                       // photons per warp claim (streamlined kernel): small
                                           // claims keep the problems in flight, and so the
                                           // voxel fields written, few (L2)
    u64 total_chunks = 0;
    bool any_mirror = false;
    bool table_valid = false;              // device table matches table[]
    std::vector<u64> cfg_n;                // configuration of the device table / graph
    u64 cfg_seed = 0;
    cudaStream_t cap = nullptr;            // private stream for graph capture
    cudaGraphExec_t exec = nullptr;
    int graph_threads = 0, graph_blocks = 0, graph_compact = 0, graph_mode = 0, graph_variant = 0,
        graph_spp = 0;
    // per-problem mode: launches fork over side streams so one problem's tail
    // overlaps the next problem's start (graph branches when captured)
    static constexpr int kSide = 4;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {};
};

static void batch_free(sp_mc_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int k = 0; k < sp_mc_batch::kSide; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->d_table);
    cudaFree(b->d_next);
    for (sp_mc *x : b->h) {
        if (x) { free_all(x); delete x; }
    }
    b->h.clear();
}

extern "C" sp_mc_batch_t *sp_mc_batch_create(int n, const uint8_t *const *masks, const int *dims,
                                             const double *optics) {
    g_err.clear();
    if (n < 1 || !masks || !dims || !optics) { fail(SP_EINVAL, "bad batch arguments"); return nullptr; }
    sp_mc_batch *b = new (std::nothrow) sp_mc_batch();
    if (!b) { fail(SP_ENOMEM, "host allocation failed"); return nullptr; }
    b->n = n;
    for (int i = 0; i < n; ++i) {
        sp_mc *h = sp_mc_create(masks[i], dims[3 * i], dims[3 * i + 1], dims[3 * i + 2],
                                optics[4 * i], optics[4 * i + 1], optics[4 * i + 2], optics[4 * i + 3]);
        if (!h) {
            const std::string msg = std::string("problem ") + std::to_string(i) + ": " + g_err;
            batch_free(b);
            delete b;
            fail(SP_EINVAL, "%s", msg.c_str());
            return nullptr;
        }
        b->h.push_back(h);
    }
    b->device = b->h[0]->device;
    b->sm_count = b->h[0]->sm_count;
    b->table.resize(n);
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_table, n * sizeof(BatchProblem))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_next, sizeof(u64))) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) {
        batch_free(b);
        delete b;
        fail(SP_ENOMEM, "batch allocation: %s", cudaGetErrorString(e));
        return nullptr;
    }
    return b;
}

extern "C" void sp_mc_batch_destroy(sp_mc_batch_t *b) {
    if (!b) return;
    DeviceGuard guard(b->device);
    batch_free(b);
    delete b;
}

extern "C" int sp_mc_batch_set_option(sp_mc_batch_t *b, int key, double value) {
    if (!b) return fail(SP_EINVAL, "null batch");
    if (!std::isfinite(value)) return fail(SP_EINVAL, "option value must be finite");
    switch (key) {
    case SP_OPT_THREADS: {
        const int t = (int)value;
        if (t < 32 || t > 256 || t % 32) return fail(SP_EINVAL, "threads must be a multiple of 32 in [32, 256]");
        b->threads = t; return SP_OK;
    }
    case SP_OPT_BLOCKS:     // CTAs per SM for batched launches; 0 = as many as fit
        if (value < 0 || value > 32) return fail(SP_EINVAL, "CTAs per SM must be in [0, 32]");
        b->blocks_per_sm = (int)value; return SP_OK;
    case SP_OPT_COMPACT:
        if (value < 1 || value > 32) return fail(SP_EINVAL, "compaction threshold must be in [1, 32]");
        b->compact_k = (int)value; return SP_OK;
    case SP_OPT_GRAPH:
        b->use_graph = value != 0; return SP_OK;
    case SP_OPT_BATCH_MODE:
        if (value != 0 && value != 1) return fail(SP_EINVAL, "batch mode must be 0 or 1");
        b->mode = (int)value; return SP_OK;
    case SP_OPT_BATCH_CHUNK:
        if (value < 32 || value > (double)(1 << 24)) return fail(SP_EINVAL, "batch chunk must be in [32, 2^24]");
        if ((u32)value != b->chunk) {
            b->chunk = (u32)value;
            b->table_valid = false;          // chunk indices of the problem table change
        }
        return SP_OK;
    case SP_OPT_KERNEL:
    case SP_OPT_STEPS_PER_PASS: {
        // the one-launch kernel's own setting, and every problem's for mode 1
        if (key == SP_OPT_KERNEL && value != 0 && value != 1)
            return fail(SP_EINVAL, "kernel variant must be 0 or 1");
        if (key == SP_OPT_STEPS_PER_PASS && (value < 1 || value > 64))
            return fail(SP_EINVAL, "steps per pass must be in [1, 64]");
        if (key == SP_OPT_KERNEL) b->variant = (int)value; else b->steps_per_pass = (int)value;
        for (sp_mc *h : b->h) {
            const int rc = sp_mc_set_option(h, key, value);
            if (rc) return rc;
        }
        return SP_OK;
    }
    default: {
        // optics-independent per-problem options apply to every problem
        if (key == SP_OPT_TALLY_FIELD || key == SP_OPT_PRECISION || key == SP_OPT_RECORDS ||
            key == SP_OPT_PID_OFFSET)
            return fail(SP_EINVAL, "option %d is fixed for batched launches", key);
        for (sp_mc *h : b->h) {
            const int rc = sp_mc_set_option(h, key, value);
            if (rc) return rc;
        }
        b->table_valid = false;
        return SP_OK;
    }
    }
}

extern "C" int sp_mc_batch_get_option(const sp_mc_batch_t *b, int key, double *value) {
    if (!b || !value) return fail(SP_EINVAL, "null argument");
    switch (key) {
    case SP_OPT_THREADS: *value = b->threads; return SP_OK;
    case SP_OPT_BLOCKS: *value = b->blocks_per_sm; return SP_OK;
    case SP_OPT_COMPACT: *value = b->compact_k; return SP_OK;
    case SP_OPT_GRAPH: *value = b->use_graph; return SP_OK;
    case SP_OPT_BATCH_MODE: *value = b->mode; return SP_OK;
    case SP_OPT_BATCH_CHUNK: *value = b->chunk; return SP_OK;
    case SP_OPT_KERNEL: *value = b->variant; return SP_OK;
    case SP_OPT_STEPS_PER_PASS: *value = b->steps_per_pass; return SP_OK;
    default: return sp_mc_get_option(b->h[0], key, value);
    }
}

// Side streams and events of the per-problem mode, made before any capture.
static int ensure_side(sp_mc_batch *b) {
    if (b->fork) return SP_OK;
    CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    for (int k = 0; k < sp_mc_batch::kSide; ++k) {
        CUDA_TRY(cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming));
    }
    return SP_OK;
}

static int batch_launch(sp_mc_batch *b, u64 total, cudaStream_t s) {
    if (b->mode == 1) {
        // one single-problem launch per problem; photon ids come from the
        // device table, which the advance kernel moves on after each run
        if (!b->fork) return fail(SP_ECUDA, "side streams not created");
        CUDA_TRY(cudaEventRecord(b->fork, s));
        for (int k = 0; k < sp_mc_batch::kSide; ++k) CUDA_TRY(cudaStreamWaitEvent(b->side[k], b->fork, 0));
        for (int i = 0, j = 0; i < b->n; ++i) {
            if (b->cfg_n[i] == 0) continue;
            const int rc = launch_run(b->h[i], b->cfg_n[i], b->cfg_seed, 0, &b->d_table[i].pid_begin,
                                      b->side[j++ % sp_mc_batch::kSide]);
            if (rc) return rc;
        }
        for (int k = 0; k < sp_mc_batch::kSide; ++k) {
            CUDA_TRY(cudaEventRecord(b->join[k], b->side[k]));
            CUDA_TRY(cudaStreamWaitEvent(s, b->join[k], 0));
        }
        batch_advance_kernel<<<(b->n + 127) / 128, 128, 0, s>>>(b->d_table, b->n);
        CUDA_TRY(cudaGetLastError());
        b->graph_mode = 1;
        return SP_OK;
    }
    int per_sm = 0;
    CUDA_TRY(occupancy_batch(b->variant, b->any_mirror, b->threads, &per_sm));
    if (per_sm < 1) return fail(SP_ECUDA, "batched transport cannot be resident with %d threads", b->threads);
    if (b->blocks_per_sm > 0 && b->blocks_per_sm < per_sm) per_sm = b->blocks_per_sm;
    BatchParams bp{};
    bp.problems = b->d_table;
    bp.n_problems = b->n;
    bp.total_photons = total;
    bp.total_chunks = b->total_chunks;
    bp.chunk = b->chunk;
    bp.next = b->d_next;
    bp.key0 = (u32)b->cfg_seed;
    bp.key1 = (u32)(b->cfg_seed >> 32);
    bp.compact_k = b->compact_k;
    bp.steps_per_pass = b->steps_per_pass;
    CUDA_TRY(cudaMemsetAsync(b->d_next, 0, sizeof(u64), s));
    CUDA_TRY(launch_transport_batch(bp, b->variant, b->any_mirror, per_sm * b->sm_count, b->threads, s));
    batch_advance_kernel<<<(b->n + 127) / 128, 128, 0, s>>>(b->d_table, b->n);
    CUDA_TRY(cudaGetLastError());
    b->graph_threads = b->threads;
    b->graph_blocks = per_sm;
    b->graph_compact = b->compact_k;
    b->graph_variant = b->variant;
    b->graph_spp = b->steps_per_pass;
    b->graph_mode = 0;
    return SP_OK;
}

// Whether any problem has mirror lateral faces (selects the batched kernel).
static void refresh_mirror(sp_mc_batch *b) {
    b->any_mirror = false;
    for (const sp_mc *h : b->h) b->any_mirror = b->any_mirror || h->mirror != 0;
}

extern "C" int sp_mc_batch_run(sp_mc_batch_t *b, const uint64_t *n_photons, uint64_t seed,
                               void *stream) {
    if (!b || !n_photons) return fail(SP_EINVAL, "null argument");
    DeviceGuard guard(b->device);
    refresh_mirror(b);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    u64 total = 0;
    for (int i = 0; i < b->n; ++i) total += n_photons[i];
    if (total == 0) return SP_OK;
    if (b->mode == 1) {
        const int rc = ensure_side(b);
        if (rc) return rc;
    }
    const std::vector<u64> want(n_photons, n_photons + b->n);
    const bool same_cfg = b->table_valid && want == b->cfg_n && seed == b->cfg_seed;
    if (!same_cfg) {
        // (re)build the device table from the handles' photon counters
        u64 offset = 0, chunk_begin = 0;
        for (int i = 0; i < b->n; ++i) {
            sp_mc *h = b->h[i];
            BatchProblem &t = b->table[i];
            t = BatchProblem{};
            t.bricks = h->d_bricks;
            t.field = h->d_field;
            t.tal = h->d_tal;
            t.nx = h->nx; t.ny = h->ny; t.nz = h->nz;
            t.nbx = h->nbx; t.nby = h->nby; t.nbz = h->nbz;
            t.pid_begin = h->pid_offset + h->photons_done;
            t.n_photons = n_photons[i];
            t.offset = offset;
            offset += n_photons[i];
            t.chunk_begin = chunk_begin;
            chunk_begin += (n_photons[i] + b->chunk - 1) / b->chunk;
            const u64 lim = iter_limit(h);
            t.iter_limit = lim > 0xffffffffull ? 0xffffffffu : (u32)lim;
            fill_f32(h, path_cap(h), t.f32, t.hg_iso, t.small_x);
            t.mirror = h->mirror;
            CUDA_TRY(cudaMemsetAsync(&h->d_tal->next, 0, sizeof(u64), s));
        }
        CUDA_TRY(cudaMemcpyAsync(b->d_table, b->table.data(), b->n * sizeof(BatchProblem),
                                 cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaStreamSynchronize(s));     // the host table may change after return
        b->total_chunks = chunk_begin;
        b->cfg_n = want;
        b->cfg_seed = seed;
        b->table_valid = true;
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    }
    if (b->use_graph) {
        int per_sm = 0;
        CUDA_TRY(occupancy_batch(b->variant, b->any_mirror, b->threads, &per_sm));
        if (b->blocks_per_sm > 0 && b->blocks_per_sm < per_sm) per_sm = b->blocks_per_sm;
        if (b->exec && (b->graph_mode != b->mode ||
                        (b->mode == 0 && (b->graph_threads != b->threads || b->graph_blocks != per_sm ||
                                          b->graph_compact != b->compact_k ||
                                          b->graph_variant != b->variant ||
                                          b->graph_spp != b->steps_per_pass)))) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        if (!b->exec) {
            // capture {counter reset, transport, id advance} once; later runs replay it
            CUDA_TRY(cudaStreamSynchronize(s));
            cudaGraph_t graph = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            const int rc = batch_launch(b, total, b->cap);
            const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
            if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
            if (e != cudaSuccess) return fail(SP_ECUDA, "graph capture: %s", cudaGetErrorString(e));
            const cudaError_t e2 = cudaGraphInstantiate(&b->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e2 != cudaSuccess) { b->exec = nullptr; return fail(SP_ECUDA, "graph instantiate: %s", cudaGetErrorString(e2)); }
        }
        CUDA_TRY(cudaGraphLaunch(b->exec, s));
    } else {
        const int rc = batch_launch(b, total, s);
        if (rc) return rc;
    }
    for (int i = 0; i < b->n; ++i) b->h[i]->photons_done += n_photons[i];
    return SP_OK;
}

extern "C" int sp_mc_batch_tallies(sp_mc_batch_t *b, int i, sp_mc_result_t *out, void *stream) {
    if (!b || i < 0 || i >= b->n) return fail(SP_EINVAL, "problem index out of range");
    return sp_mc_tallies(b->h[i], out, stream);
}

extern "C" int sp_mc_batch_raw_field(sp_mc_batch_t *b, int i, uint64_t *dst, int on_device,
                                     void *stream) {
    if (!b || i < 0 || i >= b->n) return fail(SP_EINVAL, "problem index out of range");
    return sp_mc_raw_field(b->h[i], dst, on_device, stream);
}

extern "C" int sp_mc_batch_reset(sp_mc_batch_t *b, void *stream) {
    if (!b) return fail(SP_EINVAL, "null batch");
    for (sp_mc *h : b->h) {
        const int rc = sp_mc_reset(h, stream);
        if (rc) return rc;
    }
    b->table_valid = false;
    return SP_OK;
}

extern "C" int sp_mc_batch_autotune(sp_mc_batch_t *b, const uint64_t *n_photons, uint64_t seed,
                                    double *photons_per_s, void *stream) {
    if (!b || !n_photons) return fail(SP_EINVAL, "null argument");
    DeviceGuard guard(b->device);
    refresh_mirror(b);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int saved_graph = b->use_graph;
    b->use_graph = 0;
    u64 total = 0;
    for (int i = 0; i < b->n; ++i) total += n_photons[i];
    if (total == 0) return fail(SP_EINVAL, "autotuning needs photons");
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // one-launch candidates: threads per CTA, all or half the resident CTAs,
    // compaction threshold and (streamlined kernel) steps per pass
    const int threads_c[] = {64, 128, 256};
    const int compact_c[] = {4, 8, 12, 16};
    const int spp_c[] = {8, 16};
    double best = -1.0;
    int best_t = b->threads, best_b = b->blocks_per_sm, best_k = b->compact_k, best_mode = 0;
    int best_spp = b->steps_per_pass;
    b->mode = 0;
    int rc = SP_OK;
    for (int t : threads_c) {
        int per_sm = 0;
        if (occupancy_batch(b->variant, b->any_mirror, t, &per_sm) != cudaSuccess || per_sm < 1) continue;
        for (int bps : {per_sm, (per_sm + 1) / 2}) {
            for (int k : compact_c) {
                for (int spp : spp_c) {
                    if (b->variant == 0 && spp != spp_c[0]) continue;
                    b->threads = t;
                    b->blocks_per_sm = bps;
                    b->compact_k = k;
                    b->steps_per_pass = spp;
                    cudaEventRecord(e0, s);
                    if ((rc = sp_mc_batch_run(b, n_photons, seed, stream)) != SP_OK) goto done;
                    cudaEventRecord(e1, s);
                    float ms = 0;
                    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        rc = fail(SP_ECUDA, "autotune timing failed");
                        goto done;
                    }
                    const double rate = (double)total / (ms * 1e-3);
                    if (rate > best) { best = rate; best_t = t; best_b = bps; best_k = k; best_spp = spp; }
                }
            }
        }
    }
    {   // the per-problem mode (each problem's own launch shape)
        b->mode = 1;
        cudaEventRecord(e0, s);
        if ((rc = sp_mc_batch_run(b, n_photons, seed, stream)) != SP_OK) goto done;
        cudaEventRecord(e1, s);
        float ms = 0;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = fail(SP_ECUDA, "autotune timing failed");
            goto done;
        }
        const double rate = (double)total / (ms * 1e-3);
        if (rate > best) { best = rate; best_mode = 1; }
        b->mode = 0;
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->threads = best_t;
    b->blocks_per_sm = best_b;
    b->compact_k = best_k;
    b->steps_per_pass = best_spp;
    b->mode = best_mode;
    b->use_graph = saved_graph;
    if (rc) return rc;
    if (photons_per_s) *photons_per_s = best;
    return sp_mc_batch_reset(b, stream);     // the calibration runs leave no tallies behind
}
