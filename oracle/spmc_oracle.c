/*
 * spmc_oracle.c -- plain FP64 CPU oracle for voxel Monte Carlo photon
 * migration through a binary pore mask.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg.  It shares no code with the CUDA library.
 *
 * What it follows (arXiv 2604.13929):
 *   Sec. 2.5 / App. B  planar collimated source over the whole z = 0 face,
 *                      open axial faces (z < 0 -> R, z > L -> T), weighted
 *                      photons with Russian roulette, the time gate (Eq. tend),
 *                      independent R, T and absorbed-energy counters (Eq. RTA);
 *   Sec. 2.5 media     pore voxels void (mu_a = mu_s = 0), solid voxels scatter
 *                      and absorb;
 *   Sec. 3.5(c)        per-photon cumulative pore path of escaping photons.
 * The lateral faces are periodic (the benchmark configuration) or specular
 * mirrors (the paper's bc = "mmamma"); the phase function is Henyey-Greenstein;
 * n = 1 everywhere (no Fresnel terms).
 *
 * The method is a stochastic algorithm, so this file restates its steps in
 * their natural order with the obvious data structures: unwrapped FP64
 * positions, authoritative integer voxel indices, one face crossing per loop
 * iteration.  No blocking, fusion or reordering.
 */
#include "spmc_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ---------------------------------------------------------------- RNG ---- */

/* Philox4x32-10: ten rounds of two 32x32->64 multiplications with the
 * published multipliers, the key bumped by the published Weyl constants
 * between rounds (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double or_uniform(uint32_t r)
{
    return (double)(2u * (r >> 9) + 1u) * 0x1p-24;
}

/* Event j of photon pid: counter (j, 0, pid lo, pid hi). */
static void draw(const uint32_t key[2], uint64_t pid, uint32_t j, uint32_t out[4])
{
    uint32_t ctr[4] = {j, 0u, (uint32_t)pid, (uint32_t)(pid >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------ phase function -- */

/* Inverse CDF of the Henyey-Greenstein phase function; uniform in cos for
 * g -> 0. */
double or_hg_cos(double u, double g)
{
    double c;
    if (fabs(g) < 1e-6) {
        c = 2.0 * u - 1.0;
    } else {
        double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
        c = (1.0 + g * g - t * t) / (2.0 * g);
    }
    if (c < -1.0) c = -1.0;
    if (c > 1.0) c = 1.0;
    return c;
}

/* New direction at polar cosine cost and azimuth phi about the old one
 * (spherical rotation as in MCML, Wang, Jacques & Zheng 1995), renormalised. */
void or_rotate(double d[3], double cost, double phi)
{
    double sint = sqrt(1.0 - cost * cost);
    double cosp = cos(phi), sinp = sin(phi);
    double ux = d[0], uy = d[1], uz = d[2];
    double vx, vy, vz;
    if (fabs(uz) > 0.99999) {
        vx = sint * cosp;
        vy = sint * sinp;
        vz = (uz >= 0.0) ? cost : -cost;
    } else {
        double tmp = sqrt(1.0 - uz * uz);
        vx = sint * (ux * uz * cosp - uy * sinp) / tmp + ux * cost;
        vy = sint * (uy * uz * cosp + ux * sinp) / tmp + uy * cost;
        vz = -sint * cosp * tmp + uz * cost;
    }
    double n = sqrt(vx * vx + vy * vy + vz * vz);
    d[0] = vx / n;
    d[1] = vy / n;
    d[2] = vz / n;
}

/* ------------------------------------------------------------ time gate -- */

/* Eq. tend with n = 1, written as a path length c*t_end in voxel units:
 * max[5/mu_a, 6 L^2 / D], D = 1/(3 (mu_a,eff + mu_s',eff)), EMA scaling
 * mu_eff = mu (1 - porosity) (Eq. EMA_scaling), mu_s' = mu_s (1 - g).
 * The absorption term is dropped when mu_a = 0; never below 4 L. */
double or_default_path_cap(int nz, double porosity, double mus, double mua, double g)
{
    double L = (double)nz;
    double solid = 1.0 - porosity;
    double s_abs = (mua > 0.0) ? 5.0 / mua : 0.0;
    double s_diff = 18.0 * L * L * (mua * solid + mus * (1.0 - g) * solid);
    double s = (s_abs > s_diff) ? s_abs : s_diff;
    if (s < 4.0 * L) s = 4.0 * L;
    return s;
}

/* ------------------------------------------------------------- tallies --- */

static uint64_t q32(double c)          /* Q32.32, round to nearest */
{
    return (uint64_t)llrint(c * 4294967296.0);
}

static uint64_t q16(double c)          /* Q48.16 for the second moment */
{
    return (uint64_t)llrint(c * 65536.0);
}

static void add128(uint64_t s[2], uint64_t v)
{
    unsigned __int128 a = ((unsigned __int128)s[1] << 64) | s[0];
    a += v;
    s[0] = (uint64_t)a;
    s[1] = (uint64_t)(a >> 64);
}

static long pmod(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

enum { EV_CROSS = 0, EV_INTERACT = 1, EV_GATE = 2 };

/* ------------------------------------------------------- one photon ----- */

static void run_photon(const or_problem_t *pb, uint64_t pid, or_tallies_t *t,
                       uint64_t *field, double *site, int64_t *ri, double *rv)
{
    const long nx = pb->nx, ny = pb->ny, nz = pb->nz;
    const uint32_t key[2] = {(uint32_t)pb->seed, (uint32_t)(pb->seed >> 32)};
    const int b = (int)(pid % OR_NBATCH);
    uint32_t r[4];

    /* launch: event 0 = (x, y, free path, unused) */
    draw(key, pid, 0u, r);
    double p[3] = {or_uniform(r[0]) * (double)nx, or_uniform(r[1]) * (double)ny, 0.0};
    double u[3] = {0.0, 0.0, 1.0};
    long iv[3] = {(long)floor(p[0]), (long)floor(p[1]), 0};
    if (iv[0] >= nx) iv[0] = nx - 1;
    if (iv[1] >= ny) iv[1] = ny - 1;
    double w = 1.0, tau = -log(or_uniform(r[2]));
    double s = 0.0, P = 0.0, A = 0.0;
    uint32_t event = 1u;
    int64_t n_int = 0, n_steps = 0, n_surv = 0, n_solid = 0;
    int kind = 0;

    t->photons[b] += 1;
    t->counts[OR_C_LAUNCHED] += 1;

    for (;;) {
        const long xw = pmod(iv[0], nx), yw = pmod(iv[1], ny), z = iv[2];
        const size_t v = ((size_t)z * (size_t)ny + (size_t)yw) * (size_t)nx + (size_t)xw;
        const int pore = pb->mask[v] != 0;

        /* distance to the next face along each axis */
        double d[3];
        for (int a = 0; a < 3; ++a) {
            if (u[a] > 0.0)      d[a] = ((double)(iv[a] + 1) - p[a]) / u[a];
            else if (u[a] < 0.0) d[a] = ((double)iv[a] - p[a]) / u[a];
            else                 d[a] = INFINITY;
            if (d[a] < 0.0) d[a] = 0.0;
        }
        int ax = 2;                       /* ties: z, then y, then x */
        if (d[1] < d[ax]) ax = 1;
        if (d[0] < d[ax]) ax = 0;

        double l = d[ax];
        int ev = EV_CROSS;
        /* optical depth is consumed only in the solid and carried across pores */
        if (!pore && pb->mus > 0.0 && tau < pb->mus * l) {
            l = tau / pb->mus;
            ev = EV_INTERACT;
        }
        if (s + l >= pb->s_max) {
            l = pb->s_max - s;
            if (l < 0.0) l = 0.0;
            ev = EV_GATE;
        }

        /* track-length tally of this segment */
        if (l > 0.0) {
            double dep;
            if (pore) {
                dep = w * l;
                P += l;
            } else if (pb->mua > 0.0) {
                double x = pb->mua * l;
                double f = -expm1(-x);           /* 1 - exp(-mua l) */
                dep = w * f / pb->mua;           /* integral of w exp(-mua s) ds */
                A += w * f;
                w = w * exp(-x);
            } else {
                dep = w * l;
            }
            const uint64_t qd = q32(dep);
            if (field) __atomic_fetch_add(&field[v], qd, __ATOMIC_RELAXED);
            t->depth[b][pore][(z * OR_NBIN) / nz] += qd;
            s += l;
            n_steps += 1;
            if (!pore) n_solid += 1;
        }
        if (!pore && ev == EV_CROSS) tau -= pb->mus * l;
        for (int a = 0; a < 3; ++a) p[a] += l * u[a];

        if (ev == EV_GATE) {
            t->gated[b] += q32(w);
            t->counts[OR_C_GATED] += 1;
            kind = OR_EXIT_GATE;
            break;
        }
        if (ev == EV_INTERACT) {
            if (site && n_int < 8) {
                site[n_int * 3 + 0] = p[0];
                site[n_int * 3 + 1] = p[1];
                site[n_int * 3 + 2] = p[2];
            }
            n_int += 1;
            t->counts[OR_C_INTERACT] += 1;
            draw(key, pid, event, r);   /* (cos, azimuth, free path, roulette) */
            event += 1u;
            if (w < pb->rr_weight) {
                if (or_uniform(r[3]) < 1.0 / pb->rr_mult) {
                    t->gain[b] += q32(w * (pb->rr_mult - 1.0));
                    w = w * pb->rr_mult;
                    n_surv += 1;
                    t->counts[OR_C_RR_SURVIVE] += 1;
                } else {
                    t->lost[b] += q32(w);
                    t->counts[OR_C_RR_KILL] += 1;
                    kind = OR_EXIT_RR;
                    break;
                }
            }
            double cost = or_hg_cos(or_uniform(r[0]), pb->g);
            or_rotate(u, cost, 2.0 * OR_PI * or_uniform(r[1]));
            tau = -log(or_uniform(r[2]));
            t->counts[OR_C_SCATTER] += 1;
            continue;
        }

        /* cross the face on axis ax */
        p[ax] = (u[ax] > 0.0) ? (double)(iv[ax] + 1) : (double)iv[ax];
        if (ax < 2 && pb->lateral_bc == 1) {
            /* mirror lateral faces (Sec. 2.5, bc = "mmamma"): at the domain
             * edge the direction component is reversed and the photon stays
             * in its voxel */
            const long ni = iv[ax] + ((u[ax] > 0.0) ? 1 : -1);
            if (ni < 0 || ni >= (ax == 0 ? nx : ny)) {
                u[ax] = -u[ax];
                continue;
            }
        }
        iv[ax] += (u[ax] > 0.0) ? 1 : -1;
        if (ax == 2 && (iv[2] < 0 || iv[2] >= nz)) {
            kind = (iv[2] < 0) ? OR_EXIT_R : OR_EXIT_T;
            break;
        }
    }

    if (kind == OR_EXIT_R || kind == OR_EXIT_T) {
        const uint64_t qw = q32(w);
        if (kind == OR_EXIT_R) { t->R[b] += qw; t->counts[OR_C_EXIT_R] += 1; }
        else                   { t->T[b] += qw; t->counts[OR_C_EXIT_T] += 1; }
        long hb = (long)floor(P / (4.0 * (double)nz) * 256.0);
        if (hb > 256) hb = 256;
        t->hist[hb] += qw;
        add128(t->sum_w, qw);
        add128(t->sum_wP, q32(w * P));
        add128(t->sum_wP2, q16(w * P * P));
    }
    t->A[b] += q32(A);
    t->counts[OR_C_STEPS] += (uint64_t)n_steps;
    t->counts[OR_C_SOLID_STEPS] += (uint64_t)n_solid;

    if (ri) {
        ri[0] = n_int; ri[1] = n_steps; ri[2] = kind; ri[3] = n_surv;
    }
    if (rv) {
        rv[0] = w; rv[1] = P; rv[2] = s; rv[3] = A;
    }
}

/* ------------------------------------------------------------- driver --- */

static void merge(or_tallies_t *dst, const or_tallies_t *src)
{
    const uint64_t *s = (const uint64_t *)src;
    uint64_t *d = (uint64_t *)dst;
    /* all-u64 struct except the three 128-bit sums, merged with carries */
    size_t n = sizeof(or_tallies_t) / sizeof(uint64_t);
    size_t o_w = offsetof(or_tallies_t, sum_w) / sizeof(uint64_t);
    size_t o_p = offsetof(or_tallies_t, sum_wP) / sizeof(uint64_t);
    size_t o_q = offsetof(or_tallies_t, sum_wP2) / sizeof(uint64_t);
    for (size_t i = 0; i < n; ++i) {
        if (i == o_w || i == o_w + 1 || i == o_p || i == o_p + 1 || i == o_q || i == o_q + 1)
            continue;
        d[i] += s[i];
    }
    const uint64_t *pairs[3] = {src->sum_w, src->sum_wP, src->sum_wP2};
    uint64_t *dp[3] = {dst->sum_w, dst->sum_wP, dst->sum_wP2};
    for (int k = 0; k < 3; ++k) {
        unsigned __int128 a = ((unsigned __int128)dp[k][1] << 64) | dp[k][0];
        unsigned __int128 c = ((unsigned __int128)pairs[k][1] << 64) | pairs[k][0];
        a += c;
        dp[k][0] = (uint64_t)a;
        dp[k][1] = (uint64_t)(a >> 64);
    }
}

int or_run(const or_problem_t *pb, uint64_t pid_begin, uint64_t pid_end,
           int n_threads, or_tallies_t *t, uint64_t *field,
           double *sites, int64_t *ints, double *vals, uint64_t n_rec)
{
    if (!pb || !t || !pb->mask || pb->nx < 1 || pb->ny < 1 || pb->nz < 1) return -1;
    if (!(pb->mus >= 0.0) || !(pb->mua >= 0.0) || !(fabs(pb->g) < 1.0)) return -1;
    if (!(pb->s_max > 0.0) || !isfinite(pb->s_max) || !(pb->rr_mult >= 1.0)) return -1;
    if (pb->lateral_bc != 0 && pb->lateral_bc != 1) return -1;
    if (pid_end < pid_begin) return -1;

    int nt = 1;
#ifdef _OPENMP
    nt = (n_threads > 0) ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
#endif
    or_tallies_t *part = (or_tallies_t *)calloc((size_t)nt, sizeof(or_tallies_t));
    if (!part) return -1;
    const int64_t n = (int64_t)(pid_end - pid_begin);

#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(dynamic, 64)
#endif
    for (int64_t k = 0; k < n; ++k) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        const int rec = (uint64_t)k < n_rec;
        run_photon(pb, pid_begin + (uint64_t)k, &part[tid], field,
                   (rec && sites) ? sites + (size_t)k * 24 : NULL,
                   (rec && ints) ? ints + (size_t)k * 4 : NULL,
                   (rec && vals) ? vals + (size_t)k * 4 : NULL);
    }
    for (int i = 0; i < nt; ++i) merge(t, &part[i]);
    free(part);
    return 0;
}
