// spmc_internal.cuh -- device-side data layout shared by the translation
// units of libspmc (transport kernels, reductions, host API).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace spmc {

using u64 = unsigned long long;
using u32 = unsigned int;

constexpr int kNBatch = 16;   // batch-means slots: photon id modulo 16
constexpr int kNBin = 64;     // depth bins: floor(iz * 64 / nz)
constexpr int kNHist = 257;   // pore-path histogram, 256 bins on [0, 4 nz) + overflow

// Per-batch weight tallies (Q32.32) and photon counts.
enum { B_R = 0, B_T, B_A, B_GATED, B_LOST, B_GAIN, B_PHOTONS, B_N = 8 };
// Integer event counts.
enum { C_LAUNCHED = 0, C_INTERACT, C_SCATTER, C_RR_SURV, C_RR_KILL, C_EXIT_R, C_EXIT_T,
       C_GATED, C_STEPS, C_SOLID_STEPS, C_N = 16 };
// Error flags raised by kernels.
enum { F_ITER_LIMIT = 1u, F_OVERFLOW = 2u };

#ifdef __CUDACC__
// Fire-and-forget 64-bit add into global memory.  The field pointers of
// batched problems are loaded from the device problem table, so the compiler
// cannot see that they are global and would issue the generic atomic; the
// explicit global-space reduction keeps every field update a reduction at L2
// (7 % faster batched launches).
__device__ __forceinline__ void red_add_global(u64 *p, u64 v) {
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v) : "memory");
}
#endif

// Global integer tallies of one simulation (zeroed at create / reset).
// Every member is an exact integer sum, so the totals do not depend on the
// order in which photons finish.
struct DevTallies {
    u64 batch[kNBatch][B_N];
    u64 counts[C_N];
    u64 hist[kNHist];
    u64 sums[6];                   // 128-bit (lo, hi): sum q32(w), q32(w P), q16(w P^2)
    u64 depth[2][kNBin][2];        // 128-bit (lo, hi) per phase and bin (profile mode)
    u64 next;                      // photons claimed in the current launch
    u32 flags;
    u32 pad;
};

// Arguments of one transport launch.  Optics are per voxel (mu * h).
struct TransportParams {
    const u64 *bricks;             // 4x4x4 bit bricks, bit (lz*4+ly)*4+lx, 1 = pore
    u64 *field;                    // Q32.32 track length per voxel, or nullptr
    DevTallies *tal;
    double *rec_sites;             // [n_rec][8][3]
    long long *rec_ints;           // [n_rec][4]
    double *rec_vals;              // [n_rec][4]
    u64 n_rec;                     // records for photon ids [rec_base, rec_base + n_rec)
    u64 rec_base;
    int nx, ny, nz;
    int nbx, nby, nbz;             // bricks per axis (ceil(n/4))
    int smem_bricks;               // leading bricks (z-major) staged per CTA
    u32 key0, key1;                // Philox key = seed
    u64 pid_begin, n_photons;
    const u64 *pid_begin_dev;      // if set, the first photon id is read here (graph replays)
    double mus, mua, g;
    double s_max, rr_weight, rr_mult;
    u64 iter_limit;
    int compact_k;                 // parked lanes per warp that trigger the event phase
    int hg_iso;                    // |g| < 1e-6: isotropic scattering
    int mirror;                    // lateral faces: 0 periodic, 1 specular mirrors
    int small_x;                   // mu_a * sqrt(3) <= 0.1: Taylor branch for 1 - exp(-x)
    int steps_per_pass;            // FP32 kernel: voxel steps per pass of the warp
    u32 bin_mul;                   // depth bin = umulhi(64 iz, bin_mul) when bin_exact
    int bin_exact;
    // The optics again as FP32, converted on the host: in FP32 kernels every
    // constant is a float, so no double-to-float conversion (an FP64-pipe
    // instruction) is ever rematerialised inside the loop.
    struct F32 {
        float mus, mua, inv_mus, inv_mua, one_m_g2, one_p_g2, one_m_g, two_g, inv_2g;
        float s_max, rr_weight, rr_mult, rr_p, rr_gain, hist_scale;
    } f32;
};

// One problem of a batched launch: its own mask bricks, voxel field and
// tallies, dimensions and FP32 optics.  Photons of all problems share one
// claim counter: global index k belongs to the problem whose
// [offset, offset + n_photons) contains it, with photon id pid_begin + k - offset.
// The streamlined FP32 kernel claims work in chunks of `chunk` photons of one
// problem per warp: problem i owns the global chunk indices
// [chunk_begin, chunk_begin + ceil(n_photons / chunk)).
struct BatchProblem {
    const u64 *bricks;
    u64 *field;
    DevTallies *tal;
    int nx, ny, nz, nbx, nby, nbz;
    u64 pid_begin, n_photons, offset;
    u64 chunk_begin;
    u32 iter_limit;
    int hg_iso, small_x, mirror;
    TransportParams::F32 f32;
};

struct BatchParams {
    const BatchProblem *problems;   // device table
    int n_problems;
    u64 total_photons;              // sum of n_photons (one run)
    u64 total_chunks;               // chunks over all problems (streamlined kernel)
    u32 chunk;                      // photons per chunk (streamlined kernel)
    u64 *next;                      // claim counter, zeroed before each launch
    u32 key0, key1;                 // Philox key = seed (shared by all problems)
    int compact_k;
    int steps_per_pass;
};

// Launch choices of the FP32 path beyond TransportParams: which kernel.
struct LaunchExtras {
    int variant = 1;               // 0 generic template kernel, 1 streamlined FP32 kernel
};

// Launch helpers (defined in the per-precision translation units).
cudaError_t launch_transport_f32(const TransportParams &p, bool field, int blocks, int threads,
                                 size_t smem, cudaStream_t s, const LaunchExtras &e);
cudaError_t launch_transport_f64(const TransportParams &p, bool field, int blocks, int threads,
                                 size_t smem, cudaStream_t s);
cudaError_t occupancy_f32(bool field, bool mirror, int variant, int threads, size_t smem,
                          int *blocks_per_sm);
cudaError_t launch_transport_batch(const BatchParams &b, int variant, bool mirror, int blocks,
                                   int threads, cudaStream_t s);
cudaError_t occupancy_batch(int variant, bool mirror, int threads, int *blocks_per_sm);
cudaError_t occupancy_f64(bool field, bool mirror, int threads, size_t smem, int *blocks_per_sm);
const void *kernel_f32(bool field, bool mirror, int variant);
const void *kernel_f64(bool field, bool mirror);

}  // namespace spmc
