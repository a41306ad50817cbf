/*
 * spmc_oracle.h -- plain, slow FP64 CPU oracle for voxel Monte Carlo photon
 * migration through a binary pore mask (arXiv 2604.13929, Sec. 2.5-2.6 and
 * App. B).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * library (libspmc) shares no code, header, table or helper with it.
 *
 * Conventions (voxel units throughout):
 *   mask[(iz*ny + iy)*nx + ix], x fastest, 1 = pore (void), 0 = solid.
 *   mus, mua  = solid scattering / absorption coefficients times the voxel
 *               edge (dimensionless per voxel); pores have mus = mua = 0.
 *   Every tally contribution c >= 0 is quantised as round-to-nearest(c*2^32)
 *   into an unsigned 64-bit integer ("Q32.32"), so sums are exact.
 */
#ifndef SPMC_ORACLE_H
#define SPMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NBATCH 16   /* batch-means slots: photon id modulo 16            */
#define OR_NBIN   64   /* depth bins: b = floor(iz*64/nz)                    */
#define OR_NHIST  257  /* pore-path histogram: 256 bins over [0,4nz) + over  */

/* counts[] slots */
enum {
    OR_C_LAUNCHED = 0, OR_C_INTERACT, OR_C_SCATTER, OR_C_RR_SURVIVE,
    OR_C_RR_KILL, OR_C_EXIT_R, OR_C_EXIT_T, OR_C_GATED, OR_C_STEPS,
    OR_C_SOLID_STEPS,       /* voxel steps (l > 0) inside solid voxels       */
    OR_NCOUNT
};

/* per-photon record exit kinds */
enum { OR_EXIT_R = 1, OR_EXIT_T = 2, OR_EXIT_RR = 3, OR_EXIT_GATE = 4 };

typedef struct {
    int nx, ny, nz;
    const uint8_t *mask;
    double mus, mua, g;     /* solid optics per voxel                        */
    double s_max;           /* path cap in voxel units (the time gate)       */
    double rr_weight;       /* Russian roulette threshold on w               */
    double rr_mult;         /* survivors are multiplied by this (1/p_survive) */
    uint64_t seed;          /* Philox key = (seed lo, seed hi)               */
    int lateral_bc;         /* 0 periodic x/y; 1 specular mirrors on x/y     */
} or_problem_t;

typedef struct {
    /* weight tallies per batch slot, Q32.32 */
    uint64_t R[OR_NBATCH], T[OR_NBATCH], A[OR_NBATCH];
    uint64_t gated[OR_NBATCH], lost[OR_NBATCH], gain[OR_NBATCH];
    uint64_t photons[OR_NBATCH];
    /* depth-resolved track length per batch, phase (0 solid, 1 pore), bin */
    uint64_t depth[OR_NBATCH][2][OR_NBIN];
    /* exit-weighted pore-path histogram (escaping photons only) */
    uint64_t hist[OR_NHIST];
    /* exact 128-bit sums (lo, hi) of q(w), q(w*P), q(w*P^2) over escapes */
    uint64_t sum_w[2], sum_wP[2], sum_wP2[2];
    uint64_t counts[OR_NCOUNT];
} or_tallies_t;

/* Philox4x32-10 block (Salmon et al., SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* u = (2*(r >> 9) + 1) * 2^-24, in (0,1). */
double or_uniform(uint32_t r);
/* Henyey-Greenstein cosine from one uniform. */
double or_hg_cos(double u, double g);
/* Rotate direction dir[3] by polar cosine cost and azimuth phi. */
void or_rotate(double dir[3], double cost, double phi);
/* Default path cap from the diffusion-aware time gate (Eq. tend), n = 1. */
double or_default_path_cap(int nz, double porosity, double mus, double mua, double g);

/*
 * Run photons with ids [pid_begin, pid_end).  Tallies are ADDED into *t and
 * (when non-NULL) into field[nz*ny*nx] (Q32.32 track length per voxel).
 * Records (when non-NULL) for photons pid_begin + k, k < n_rec:
 *   sites[k][8][3]  unwrapped positions of the first 8 interaction events
 *   ints[k][4]      (interaction events, voxel steps, exit kind, RR survivals)
 *   vals[k][4]      (exit weight, pore path, total path, absorbed weight)
 * Returns 0, or -1 on invalid arguments.
 */
int or_run(const or_problem_t *pb, uint64_t pid_begin, uint64_t pid_end,
           int n_threads, or_tallies_t *t, uint64_t *field,
           double *sites, int64_t *ints, double *vals, uint64_t n_rec);

#ifdef __cplusplus
}
#endif
#endif
