/*
 * spmc.h -- C ABI of libspmc: voxel Monte Carlo photon migration through a
 * 3D binary pore mask on one GB300 GPU (sm_103a).
 *
 * Method (arXiv 2604.13929, Sec. 2.5 "Three-dimensional Monte Carlo
 * simulation", Sec. 2.6 "Fluence estimators and the phase-contrast
 * identity", App. B "Monte Carlo solver configuration", Sec. 3.5(c)):
 * a planar collimated source covers the whole z = 0 face; pore voxels are
 * void (mu_a = mu_s = 0) and are crossed ballistically; solid voxels scatter
 * (Henyey-Greenstein) and absorb (continuous weight decay); the remaining
 * optical depth of a photon is carried across pores; photons leaving through
 * z < 0 count as reflectance R, through z > L as transmittance T; lateral
 * faces are periodic; Russian roulette removes low-weight photons; a path
 * cap plays the part of the time gate (Eq. tend).  Track-length tallies give
 * the voxel fluence, from which the solid-weighted mean <Phi>_3D (Eq.
 * Phi_MC3D), the volume mean <Phi>_1D (Eq. Phi_MC1D), the pore mean, the
 * phase contrast r (Eq. r_def) and the concentration ratio with its dilution
 * identity (Eq. dilution) follow, together with R, T, A (Eq. RTA) and the
 * exit-weighted pore-path distribution (Sec. 3.5(c)).
 *
 * Units: lengths in the caller's unit L; mu_s, mu_a in 1/L; the library
 * works in voxel units (mu * voxel_h per voxel).  Fluence is reported per
 * unit incident flux, Phi/S0 = F * nx * ny / N with F the weighted track
 * length per voxel (Eq. Phi_norm for a steady source, without t_end).
 *
 * Threading: a handle may be used from one host thread at a time.  All
 * entry points return SP_OK (0) or a negative SP_E* code; the message of
 * the last failure on the calling thread is returned by sp_mc_last_error().
 * There is no CPU fallback: without a usable CUDA device every call that
 * needs one fails with SP_ECUDA.
 */
#ifndef SPMC_H
#define SPMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ errors --- */
#define SP_OK          0
#define SP_EINVAL     -1   /* invalid argument or state                     */
#define SP_ENOMEM     -2   /* device or host allocation failed              */
#define SP_ECUDA      -3   /* CUDA runtime error / no device                */
#define SP_ESTEPLIMIT -4   /* a photon hit the per-photon iteration limit   */
#define SP_EOVERFLOW  -5   /* a fixed-point tally left its headroom         */

#define SP_NBATCH 16       /* batch-means slots (photon id modulo 16)       */
#define SP_NBIN   64       /* depth bins, b = floor(iz * 64 / nz)           */
#define SP_NHIST  257      /* pore-path histogram: 256 bins on [0,4 nz) + 1 */

/* ----------------------------------------------------------- options --- */
enum sp_option {
    SP_OPT_PATH_CAP    = 1,  /* path cap in voxel units; <= 0 restores the
                                default max[5/mu_a', 18 nz^2 (mu_a'+mu_s'(1-g))(1-phi)],
                                at least 4 nz (Eq. tend with n = 1)       */
    SP_OPT_RR_WEIGHT   = 2,  /* roulette threshold on the weight (1e-4)   */
    SP_OPT_RR_MULT     = 3,  /* survivors are multiplied by this; survival
                                probability is its inverse (10)           */
    SP_OPT_TALLY_FIELD = 4,  /* 1 (default): full voxel fluence field;
                                0: depth profiles per phase only          */
    SP_OPT_PRECISION   = 5,  /* 32 (default): FP32 transport; 64: FP64    */
    SP_OPT_RECORDS     = 6,  /* record the first n photon ids (debug)     */
    SP_OPT_BLOCKS      = 7,  /* persistent CTAs; 0 = SMs x resident CTAs  */
    SP_OPT_THREADS     = 8,  /* threads per CTA (multiple of 32, <= 256)  */
    SP_OPT_ITER_LIMIT  = 9,  /* per-photon loop limit (< 2^32); 0 = derived */
    SP_OPT_SMEM_BRICKS = 10, /* mask bricks staged in shared memory per
                                CTA (entry slab); -1 = auto, 0 = none     */
    SP_OPT_PID_OFFSET  = 11, /* first photon id of this handle (default 0);
                                lets ranks run disjoint id ranges whose
                                integer tallies sum to one larger run.
                                Only before the first run.                */
    SP_OPT_COMPACT     = 12, /* warp compaction threshold in [1, 32]: lanes
                                needing an interaction or a new photon wait
                                until this many of their warp do (8)      */
    SP_OPT_GRAPH       = 13, /* batched launches only: 1 (default) captures
                                the launch in a CUDA graph and replays it
                                while photon counts and seed are unchanged */
    SP_OPT_LATERAL_BC  = 14, /* 0 (default): periodic x and y; 1: specular
                                mirrors on the lateral faces (the paper's
                                bc = "mmamma", Sec. 2.5)                  */
    SP_OPT_BATCH_MODE  = 15, /* batched launches only: 0 (default) one
                                persistent launch over all problems; 1 one
                                single-problem launch per problem (shared-
                                memory mask slab and tallies), still one
                                graph replay per run                      */
    SP_OPT_KERNEL      = 16, /* FP32 transport kernel: 1 (default) the
                                streamlined kernel (several voxel steps per
                                warp vote, branch-free phases, all events in
                                the compacted event phase); 0 the generic
                                template kernel (same photons, same method) */
    SP_OPT_STEPS_PER_PASS = 17,/* streamlined kernel: voxel steps a lane
                                takes per pass of its warp, [1, 64] (8);
                                results do not depend on it                */
    SP_OPT_BATCH_CHUNK = 18   /* batched one-launch mode, streamlined kernel:
                                photons per warp claim, [32, 2^24] (128);
                                results do not depend on it                */
};

typedef struct sp_mc sp_mc_t;   /* opaque, owned by the library */

/* Results of sp_mc_tallies().  All fluences are Phi/S0 (dimensionless). */
typedef struct {
    uint64_t photons;               /* photons run since create/reset       */
    int32_t  status;                /* SP_OK, or SP_ESTEPLIMIT/SP_EOVERFLOW */
    int32_t  precision;             /* 32 or 64                             */
    double   s_max;                 /* path cap used (voxel units)          */
    double   porosity;              /* pore voxels / all voxels             */
    /* weight budget per launched photon (Eq. RTA and Eq. closure) */
    double   R, T, A, gated, lost, gain;
    double   closure;               /* R + T + A + gated + lost - gain      */
    double   R_se, T_se, A_se;      /* batch-means standard errors          */
    /* estimators (Sec. 2.6) */
    double   phi_3d, phi_1d, phi_pore, r, ratio, identity_residual;
    /* depth profiles: [0] solid, [1] pore, [2] all voxels; NaN when empty */
    double   depth[3][SP_NBIN];
    uint64_t depth_count[2][SP_NBIN];
    /* exit-weighted pore path of escaping photons (Sec. 3.5(c)) */
    double   escape_weight;         /* sum of exit weights / N              */
    double   pore_path_mean;        /* sum w P / sum w (voxel units)        */
    double   pore_path_m2;          /* sum w P^2 / sum w                    */
    double   p_pore_gt_L;           /* weight fraction with P > nz          */
    double   pore_hist[SP_NHIST];   /* exit weight per bin / N              */
    /* integer event counts */
    uint64_t launched, interactions, scatters, rr_survive, rr_kill;
    uint64_t exit_R, exit_T, gated_n, steps;
    uint64_t solid_steps;           /* voxel steps inside solid voxels      */
    /* raw Q32.32 tallies (exact), per batch slot pid % 16 */
    uint64_t raw_R[SP_NBATCH], raw_T[SP_NBATCH], raw_A[SP_NBATCH];
    uint64_t raw_gated[SP_NBATCH], raw_lost[SP_NBATCH], raw_gain[SP_NBATCH];
    uint64_t batch_photons[SP_NBATCH];
    /* exact 128-bit track-length sums per phase and depth bin (lo, hi) */
    uint64_t raw_depth[2][SP_NBIN][2];
    uint64_t raw_hist[SP_NHIST];
    uint64_t raw_sum_w[2], raw_sum_wP[2];  /* Q32.32, 128-bit (lo, hi)      */
    uint64_t raw_sum_wP2[2];               /* Q48.16, 128-bit (lo, hi)      */
} sp_mc_result_t;

/*
 * Create a simulation over a binary mask.
 *   mask      host pointer, nz*ny*nx bytes, x fastest ([iz][iy][ix]);
 *             nonzero = pore (void), 0 = solid.  Copied; the caller keeps it.
 *   nx,ny,nz  >= 1 each, fewer than 2^31 4x4x4 bricks (about 2^37 voxels).
 *   voxel_h   voxel edge (> 0) in the length unit of mu_s, mu_a.
 *   mu_s,mu_a solid scattering / absorption coefficients (>= 0, finite).
 *   g         HG anisotropy, -1 < g < 1.
 * Uses the current CUDA device.  Returns NULL on failure (see
 * sp_mc_last_error()).  Device memory: the bit-packed mask (1 bit/voxel),
 * the voxel fluence field (8 bytes/voxel over the volume padded to
 * multiples of 4, when enabled) and a few KiB.
 */
sp_mc_t *sp_mc_create(const uint8_t *mask, int nx, int ny, int nz, double voxel_h,
                      double mu_s, double mu_a, double g);

/* Set / get an option (enum sp_option).  SP_OPT_TALLY_FIELD and
 * SP_OPT_PRECISION may only change while no photons have been run. */
int sp_mc_set_option(sp_mc_t *h, int key, double value);
int sp_mc_get_option(const sp_mc_t *h, int key, double *value);

/*
 * Run n_photons photons, asynchronously on `stream` (a cudaStream_t; NULL is
 * the legacy default stream).  Tallies ACCUMULATE: photon ids continue from
 * SP_OPT_PID_OFFSET plus the number already run, so run(N1) then run(N2)
 * equals run(N1 + N2) bit for bit with the same seed.  Photon id p draws Philox4x32-10 blocks
 * with key (seed lo, seed hi) and counter (event, 0, p lo, p hi).
 * Returns SP_OK once the launch is queued.
 */
int sp_mc_run(sp_mc_t *h, uint64_t n_photons, uint64_t seed, void *stream);

/*
 * Normalise on the GPU in FP64 and copy the results into *out (caller-owned
 * host memory).  Synchronises `stream`.  Returns SP_OK, or SP_ESTEPLIMIT /
 * SP_EOVERFLOW (out is still filled) when a run reported that condition.
 */
int sp_mc_tallies(sp_mc_t *h, sp_mc_result_t *out, void *stream);

/*
 * Normalised voxel fluence Phi/S0 into dst[nz*ny*nx] (x fastest).
 *   dtype      0 = float64, 1 = float32
 *   on_device  nonzero if dst is device memory (written in stream order),
 *              zero for host memory (the call synchronises `stream`).
 * SP_EINVAL when the field tally is disabled.
 */
int sp_mc_fluence(sp_mc_t *h, void *dst, int dtype, int on_device, void *stream);

/* Raw Q32.32 voxel track-length field into dst[nz*ny*nx] (uint64). */
int sp_mc_raw_field(sp_mc_t *h, uint64_t *dst, int on_device, void *stream);

/*
 * Debug records of the first n photon ids of the handle (ids PID_OFFSET ..
 * PID_OFFSET + n - 1, n <= SP_OPT_RECORDS), host buffers:
 *   sites[n][8][3]  unwrapped positions (voxel units) of the first 8
 *                   interaction events (NaN when fewer)
 *   ints[n][4]      interaction events, voxel steps, exit kind
 *                   (1 R, 2 T, 3 roulette, 4 path cap), roulette survivals
 *   vals[n][4]      exit weight, pore path, total path, absorbed weight
 * Any pointer may be NULL.  Synchronises `stream`.
 */
int sp_mc_records(sp_mc_t *h, uint64_t n, double *sites, int64_t *ints, double *vals,
                  void *stream);

/* Zero all tallies and the photon counter (mask and options kept). */
int sp_mc_reset(sp_mc_t *h, void *stream);

/* Checkpoint of the raw integer tallies and the photon counter: size in
 * bytes, save into a host buffer of that size, restore from one.  A
 * restored run continues bit for bit. */
size_t sp_mc_checkpoint_size(const sp_mc_t *h);
int sp_mc_checkpoint(sp_mc_t *h, void *buf, size_t size, void *stream);
int sp_mc_restore(sp_mc_t *h, const void *buf, size_t size, void *stream);

/* Free the handle and its device memory (NULL is ignored). */
void sp_mc_destroy(sp_mc_t *h);

/* Message of the last failure on this host thread ("" if none). */
const char *sp_mc_last_error(void);

/* Library version, e.g. "spmc 0.1.0 sm_103a". */
const char *sp_mc_version(void);

/*
 * Measurement helper with no counterpart in the paper: the throughput ceiling
 * of the transport kernel's memory pattern on this GPU.  Straight rays step
 * face by face through an all-pore n^3 volume (n a multiple of 4 in
 * [16, 1024]) with the transport kernel's traversal arithmetic and mask-brick
 * fetches, and, when red != 0, one Q32.32 RED.ADD.U64 per step into an n^3
 * brick-layout field (8 n^3 bytes, allocated and freed by the call).  One
 * timed launch of steps_per_thread steps per thread on the current device;
 * *ms gets its CUDA-event time and *steps_per_s the step rate.
 */
int sp_mc_probe_step_ceiling(int n, int red, long long steps_per_thread, double *ms,
                             double *steps_per_s);

/* sizeof(sp_mc_result_t) as compiled into the library, so bindings can
 * verify their copy of the layout. */
size_t sp_mc_result_size(void);

/* ---------------------------------------------------------- batches --- */
/*
 * Many masks of uneven size and optics transported in ONE persistent launch
 * (the batched pattern of the design sweeps; the paper runs its cases one at
 * a time).  Each problem has its own bit-packed mask, Q32.32 voxel field and
 * integer tallies, exactly as an sp_mc_create handle.  With the streamlined
 * kernel (SP_OPT_KERNEL = 1, default) every warp claims chunks of
 * SP_OPT_BATCH_CHUNK (128) photons of one problem from a shared counter and keeps that problem's
 * tallies in shared memory until it moves on; with the generic kernel (0)
 * photons of all problems are claimed one by one, so lanes of a warp carry
 * different problems.  With the same seed and photon counts every problem's
 * tallies equal those of a separate sp_mc_run on its own handle (same kernel
 * variant), bit for bit.
 */
typedef struct sp_mc_batch sp_mc_batch_t;

/* masks[i]: host pointer to problem i's mask (as sp_mc_create);
 * dims[3i..3i+2] = nx, ny, nz; optics[4i..4i+3] = voxel_h, mu_s, mu_a, g.
 * Returns NULL on failure (sp_mc_last_error names the problem). */
sp_mc_batch_t *sp_mc_batch_create(int n, const uint8_t *const *masks, const int *dims,
                                  const double *optics);
/* SP_OPT_THREADS (threads per CTA, default 128), SP_OPT_BLOCKS (CTAs per SM,
 * 0 = as many as fit), SP_OPT_COMPACT, SP_OPT_GRAPH and SP_OPT_BATCH_MODE
 * apply to the launch (in mode 1 every problem uses its own launch options);
 * SP_OPT_KERNEL and SP_OPT_STEPS_PER_PASS apply to the one launch and to
 * every problem's own launches; the
 * path-cap, roulette and iteration-limit options apply to every problem;
 * tally mode, precision, records and photon-id offset are fixed (field,
 * FP32, none, 0). */
int sp_mc_batch_set_option(sp_mc_batch_t *b, int key, double value);
int sp_mc_batch_get_option(const sp_mc_batch_t *b, int key, double *value);
/* Run n_photons[i] photons of every problem i in one launch on `stream`;
 * tallies accumulate and photon ids continue per problem as in sp_mc_run.
 * With SP_OPT_GRAPH the first run of a given (n_photons, seed, launch shape)
 * is captured as a CUDA graph {counter reset, transport, id advance} and
 * later runs replay it. */
int sp_mc_batch_run(sp_mc_batch_t *b, const uint64_t *n_photons, uint64_t seed, void *stream);
/* Results / raw field of problem i (as sp_mc_tallies / sp_mc_raw_field). */
int sp_mc_batch_tallies(sp_mc_batch_t *b, int i, sp_mc_result_t *out, void *stream);
int sp_mc_batch_raw_field(sp_mc_batch_t *b, int i, uint64_t *dst, int on_device, void *stream);
/* Zero every problem's tallies and photon counter. */
int sp_mc_batch_reset(sp_mc_batch_t *b, void *stream);
/* Autotuner: times one batched run of n_photons[] for each candidate launch
 * shape of the one-launch mode (threads per CTA 64/128/256, all or half the
 * resident CTAs per SM, compaction threshold 4/8/12/16, and for the
 * streamlined kernel 8 or 16 steps per pass) and for the per-problem mode,
 * keeps the fastest, stores its rate in *photons_per_s (may be NULL), then
 * resets the tallies. */
int sp_mc_batch_autotune(sp_mc_batch_t *b, const uint64_t *n_photons, uint64_t seed,
                         double *photons_per_s, void *stream);
void sp_mc_batch_destroy(sp_mc_batch_t *b);

/*
 * One complete simulation that allocates nothing.  The paper has no
 * counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc or any allocating routine: for instance code embedded in an
 * application whose own allocator owns all device memory, or
 * latency-critical loops that cannot afford an allocator call.
 *
 *   d_mask     DEVICE pointer, nz*ny*nx bytes, x fastest, nonzero = pore;
 *              read only, owned by the caller.
 *   nx,ny,nz   >= 1, at most 2^18 4x4x4 bricks (e.g. 256^3 voxels);
 *              larger volumes are rejected with SP_EINVAL ("size too large").
 *   voxel_h, mu_s, mu_a, g   as for sp_mc_create.
 *   n_photons, seed          photon ids 0 .. n_photons-1, Philox key = seed.
 *   out        HOST pointer to the caller's result struct (filled).
 *   stream     cudaStream_t or NULL.  The call synchronises it twice: once
 *              to read the per-bin voxel counts back (they give the
 *              porosity, which sets the path cap) and once for the result.
 * Runs with the default options of a fresh handle in the depth-profile tally
 * mode (SP_OPT_TALLY_FIELD = 0): R/T/A, estimators, depth profiles and the
 * pore-path statistics are produced, the voxel field is not.  Results equal
 * those of sp_mc_create/sp_mc_run/sp_mc_tallies with that option.
 *
 * Working memory is one fixed array of about 2.03 MiB inside the library,
 * held by every GPU that loads it until the process exits.  Every call looks
 * up that array's device address on the current device (which allocates
 * nothing), so the address stays right across a device reset.  Every call
 * reuses the array and clears what must start at zero, so calls whose GPU
 * work overlaps (other streams, other host threads) race and must be
 * serialised by the caller.  Returns SP_OK or a negative SP_E* code.
 */
int sp_mc_simulate_noalloc(const uint8_t *d_mask, int nx, int ny, int nz, double voxel_h,
                           double mu_s, double mu_a, double g, uint64_t n_photons,
                           uint64_t seed, sp_mc_result_t *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SPMC_H */
