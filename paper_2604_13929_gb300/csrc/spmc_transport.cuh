// spmc_transport.cuh -- persistent photon-transport kernel (sm_103a).
//
// One photon per thread.  A thread whose photon has ended immediately claims
// the next photon id (one warp-aggregated atomic per claim), so lanes are
// refilled instead of idling; the grid is SMs x resident CTAs and lives for
// the whole run.
//
// Per photon (arXiv 2604.13929, Sec. 2.5 and App. B; periodic lateral faces
// and HG scattering as configured):
//   launch   uniform over the z = 0 face, direction +z, weight 1, optical
//            depth tau = -ln u (Philox event 0);
//   step     Amanatides-Woo traversal: one voxel face per iteration, the
//            ray parameter of the next x/y/z face kept per axis; in solid
//            voxels tau is consumed at rate mu_s, in pores it is carried
//            unchanged; the weight decays continuously as exp(-mu_a l);
//   tally    the segment's weighted track length int w ds is added to the
//            voxel as a Q32.32 integer (RED.ADD.U64), so sums are exact and
//            independent of photon order;
//   interact roulette (w < threshold: survive with 1/M, w *= M), HG polar
//            cosine, uniform azimuth, spherical rotation, new tau
//            (Philox event j);
//   exit     z < 0 -> R, z >= nz -> T; x and y wrap; path cap -> gated.
// Block-local integer tallies live in shared memory and are flushed with
// 64-bit integer atomics when the CTA retires.
#pragma once

#include <cooperative_groups.h>

#include "spmc_internal.cuh"

namespace spmc {

namespace cg = cooperative_groups;

// ------------------------------------------------------------------ RNG --

// Philox4x32-10 (Salmon et al., SC'11): two 32x32 -> 64-bit products per
// round (each one wide multiply giving both halves), key bumped by the Weyl
// constants between rounds.
__device__ __forceinline__ void philox4x32_10(u32 c0, u32 c1, u32 c2, u32 c3, u32 k0, u32 k1,
                                              u32 out[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const u64 p0 = (u64)0xD2511F53u * c0, p1 = (u64)0xCD9E8D57u * c2;
        const u32 lo0 = (u32)p0, hi0 = (u32)(p0 >> 32);
        const u32 lo1 = (u32)p1, hi1 = (u32)(p1 >> 32);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// --------------------------------------------------- precision policies --

template <typename Real> struct Ops;

template <> struct Ops<float> {
    __device__ static float inf() { return __int_as_float(0x7f800000); }
    // (2 (r>>9) + 1) 2^-24, exact: the float 1 + (r>>9) 2^-23 built from its
    // bit pattern, minus 1 - 2^-24 (both multiples of 2^-24, the difference
    // has at most 24 significant bits, so the subtraction is exact)
    __device__ static float uniform(u32 r) {
        return __uint_as_float(0x3f800000u | (r >> 9)) - 0.999999940395355225f;
    }
    __device__ static float neg_log(float u) { return -__logf(u); }
    __device__ static void sincos_2pi(float u, float *s, float *c) { sincospif(2.0f * u, s, c); }
    __device__ static float rsqrt(float x) { return rsqrtf(x); }
    __device__ static float rcp(float x) { return __frcp_rn(x); }
    __device__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ static u64 q32(float c) { return __float2ull_rn(c * 4294967296.0f); }
    __device__ static u64 q16(float c) { return __float2ull_rn(c * 65536.0f); }
    // 1 - exp(-x) for 0 <= x <= 0.1 by its Taylor series to x^5 (relative
    // truncation error below x^5/720 < 2e-8), with no special-function op.
    __device__ static float one_minus_exp_small(float x) {
        float p = fmaf(-x, 1.0f / 5.0f, 1.0f);
        p = fmaf(-x * (1.0f / 4.0f), p, 1.0f);
        p = fmaf(-x * (1.0f / 3.0f), p, 1.0f);
        p = fmaf(-x * 0.5f, p, 1.0f);
        return x * p;
    }
    __device__ static float one_minus_exp(float x) { return -expm1f(-x); }
};

template <> struct Ops<double> {
    __device__ static double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    __device__ static double uniform(u32 r) {
        return (double)(((r >> 9) << 1) | 1u) * 5.9604644775390625e-8;
    }
    __device__ static double neg_log(double u) { return -log(u); }
    __device__ static void sincos_2pi(double u, double *s, double *c) {
        const double phi = 2.0 * 3.14159265358979323846 * u;
        *s = sin(phi);
        *c = cos(phi);
    }
    __device__ static double rsqrt(double x) { return 1.0 / sqrt(x); }
    __device__ static double rcp(double x) { return 1.0 / x; }
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static u64 q32(double c) { return __double2ull_rn(c * 4294967296.0); }
    __device__ static u64 q16(double c) { return __double2ull_rn(c * 65536.0); }
    __device__ static double one_minus_exp(double x) { return -expm1(-x); }
};

// 128-bit accumulation with 64-bit atomics: carry into the high word.
__device__ __forceinline__ void atomic_add_u128(u64 *lohi, u64 v) {
    const u64 old = atomicAdd(lohi, v);
    if (old + v < old) atomicAdd(lohi + 1, 1ull);
}

// -------------------------------------------------------------- kernel --

struct SmemTallies {
    u64 batch[kNBatch][B_N];
    u64 counts[C_N];
    u64 hist[kNHist];
    u64 sums[6];
    u64 depth[2][kNBin];
};

// Q32.32 quantisation, round to nearest even, of a float 0 <= c < 2^13, with
// FP32 arithmetic only (no conversion instruction, no branch).  c is split
// exactly into k1 2^-9 + r with integer k1 = rint(c 2^9) and |r| <= 2^-10,
// each part rounded by adding 1.5 2^23 (the sum's low mantissa bits are then
// the rounded integer): c 2^32 = k1 2^23 + r 2^32, and rint(r 2^32) rounds
// only the fraction, so q = k1 2^23 + rint(r 2^32) = rint(c 2^32).
__device__ __forceinline__ u64 q32_bits(float c) {
    const float magic = 12582912.0f;                       // 1.5 * 2^23
    const float t1 = fmaf(c, 512.0f, magic);               // k1 in the low bits
    const int k1 = (int)(__float_as_uint(t1) - 0x4B400000u);
    const float r = fmaf(t1 - magic, -1.0f / 512.0f, c);   // exact remainder
    const float t2 = fmaf(r, 4294967296.0f, magic);        // |r 2^32| <= 2^22
    const int k2 = (int)(__float_as_uint(t2) - 0x4B400000u);
    return ((u64)(u32)k1 << 23) + (u64)(long long)k2;
}

// Lane modes of the persistent loop.
enum { M_STEP = 0, M_EVENT = 1, M_NEW = 2, M_DONE = 3 };

// Two traversal formulations share the kernel:
//  * FP32 (production): Amanatides-Woo.  Per axis the ray parameter of the
//    next face (tm) and the spacing of faces (dt = 1/|u|); a step picks the
//    smallest tm.  Parameters are rebased to the current point once the ray
//    parameter exceeds 4 voxels, so FP32 rounding does not accumulate along
//    long pore flights.  Sines from sqrt((1-c)(1+c)) and sincospif keep
//    forward scattering accurate.
//  * FP64 (exact variant): unwrapped absolute positions, the distance to
//    each next face recomputed every step by division, the same formulas in
//    the same order as the plain definition (compiled without FMA
//    contraction), so the FP64 transport reproduces a plain FP64 evaluation
//    of the method up to the last ulp of the transcendental functions.
//
// Warp-level compaction: a lane whose photon needs a random-number event (an
// interaction, or the launch of a new photon) parks until at least
// `compact_k` lanes of its warp are parked or none can step; the warp then
// runs the Philox block and the event code for all parked lanes at once.
// Each photon's history depends only on its id, so the order of events
// across lanes changes nothing in the results.
// Launch-shape tuning knobs (compile time): voxel steps per pass of the
// warp-level event check, and the minimum resident CTAs per SM requested
// from the register allocator.
#ifndef SPMC_STEPS_PER_PASS
#define SPMC_STEPS_PER_PASS 1
#endif
#ifndef SPMC_MIN_BLOCKS
#define SPMC_MIN_BLOCKS 1
#endif

// Batched launches (kBatch): many problems (masks, sizes, optics) in one
// persistent launch.  A lane loads its problem's dimensions, optics and
// pointers when it claims a photon, so one warp can carry photons of
// different problems; per-photon tallies go straight to the problem's global
// integer tallies.
// Batched launches carry per-lane problem constants; three resident CTAs of
// 256 threads need <= 85 registers, which the bound below asks for.  kMirror
// compiles the specular lateral faces in (per lane in batched launches);
// without it the periodic kernel carries no mirror code.
template <typename Real, bool kField, bool kBatch, bool kMirror>
__global__ void __launch_bounds__(256, kBatch ? 3 : SPMC_MIN_BLOCKS) transport_kernel(const TransportParams p,
                                                                                      const BatchParams bp) {
    using O = Ops<Real>;
    constexpr bool kExact = sizeof(Real) == 8;
    extern __shared__ u64 s_bricks[];
    __shared__ SmemTallies st;

    {   // zero the block tallies, stage the entry slab of the mask
        u64 *z = reinterpret_cast<u64 *>(&st);
        for (int i = threadIdx.x; i < (int)(sizeof(SmemTallies) / 8); i += blockDim.x) z[i] = 0;
        if constexpr (!kBatch)
            for (int i = threadIdx.x; i < p.smem_bricks; i += blockDim.x) s_bricks[i] = __ldg(p.bricks + i);
    }
    __syncthreads();

    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    int nx = p.nx, ny = p.ny, nz = p.nz;
    int nbx = p.nbx, nby = p.nby;
    const u64 *bricks_ptr = p.bricks;            // per lane in batched launches
    u64 *field_ptr = p.field;
    DevTallies *tal_ptr = p.tal;
    const u32 key0 = kBatch ? bp.key0 : p.key0, key1 = kBatch ? bp.key1 : p.key1;
    int prob = 0;
    bool mirror = kMirror && p.mirror != 0;      // per lane in batched launches
    Real mus, mua, inv_mus, inv_mua, one_m_g2, one_p_g2, one_m_g, two_g, inv_2g, g;
    Real s_max, rr_w, rr_m, rr_p, rr_gain, hist_scale;
    if constexpr (kExact) {
        mus = p.mus; mua = p.mua;
        inv_mus = p.mus > 0 ? 1.0 / p.mus : 0.0;
        inv_mua = p.mua > 0 ? 1.0 / p.mua : 0.0;
        g = p.g;
        one_m_g2 = 1.0 - g * g; one_p_g2 = 1.0 + g * g; one_m_g = 1.0 - g; two_g = 2.0 * g;
        inv_2g = p.hg_iso ? 0.0 : 1.0 / (2.0 * p.g);
        s_max = p.s_max; rr_w = p.rr_weight; rr_m = p.rr_mult;
        rr_p = 1.0 / p.rr_mult; rr_gain = p.rr_mult - 1.0;
        hist_scale = 256.0 / (4.0 * (double)nz);
    } else {
        mus = p.f32.mus; mua = p.f32.mua; inv_mus = p.f32.inv_mus; inv_mua = p.f32.inv_mua;
        g = 0;
        one_m_g2 = p.f32.one_m_g2; one_p_g2 = p.f32.one_p_g2; one_m_g = p.f32.one_m_g;
        two_g = p.f32.two_g; inv_2g = p.f32.inv_2g;
        s_max = p.f32.s_max; rr_w = p.f32.rr_weight; rr_m = p.f32.rr_mult;
        rr_p = p.f32.rr_p; rr_gain = p.f32.rr_gain; hist_scale = p.f32.hist_scale;
    }
    bool absorb_on = mua > 0;
    bool small_x = p.small_x != 0;
    bool hg_iso = p.hg_iso != 0;
    const Real kInf = O::inf();
    u32 iter_limit = p.iter_limit > 0xffffffffull ? 0xffffffffu : (u32)p.iter_limit;
    const int ck = kBatch ? bp.compact_k : p.compact_k;
    const u64 pid0 = (!kBatch && p.pid_begin_dev) ? *p.pid_begin_dev : p.pid_begin;
    const int compact_k = ck < 1 ? 1 : (ck > 32 ? 32 : ck);

    // photon state
    int mode = M_NEW;
    u64 pid = 0;
    int ix = 0, iy = 0, iz = 0, kx = 0, ky = 0, bin = 0, batch = 0;
    int sx = 1, sy = 1, sz = 1;                  // step direction per axis along the ray
    u32 brick = 0, bit = 0;                      // current voxel = field[brick * 64 + bit]
    u64 word = 0;                                // mask bits of the current brick
    Real ux = 0, uy = 0, uz = 1;
    Real w = 1, tau = 0, s = 0, P = 0, A = 0;
    u32 event = 1, n_int = 0, n_surv = 0, n_scat = 0, n_steps = 0, n_solid = 0, iters = 0;
    // FP32 traversal: face parameters along the current ray, origin fractions
    Real tmx = kInf, tmy = kInf, tmz = 1, dtx = kInf, dty = kInf, dtz = 1, t = 0;
    Real fx = 0, fy = 0, fz = 0;
    // FP64 traversal: unwrapped absolute position
    Real px = 0, py = 0, pz = 0;

    const u32 nbxy = (u32)nbx * (u32)nby;
    auto brick_of = [&](int x, int y, int z) -> u32 {
        return ((u32)(z >> 2) * (u32)nby + (u32)(y >> 2)) * (u32)nbx + (u32)(x >> 2);
    };
    auto bit_of = [&](int x, int y, int z) -> u32 {
        return (u32)(((z & 3) << 4) | ((y & 3) << 2) | (x & 3));
    };
    auto fetch = [&](u32 b) -> u64 {
        if constexpr (kBatch) return __ldg(bricks_ptr + b);
        else return ((int)b < p.smem_bricks) ? s_bricks[b] : __ldg(p.bricks + b);
    };
    (void)nbxy;
    auto q32 = [&](Real c) -> u64 {
        if constexpr (kExact) return O::q32(c);
        else return q32_bits(c);
    };

    auto finish = [&](int kind) {
        // kind: 1 R, 2 T, 3 roulette, 4 path cap
        u64 (*tb)[B_N] = st.batch;
        u64 *tc = st.counts, *th = st.hist, *ts = st.sums;
        if constexpr (kBatch) {
            tb = tal_ptr->batch; tc = tal_ptr->counts; th = tal_ptr->hist; ts = tal_ptr->sums;
            hist_scale = bp.problems[prob].f32.hist_scale;
        }
        if (kind == 1 || kind == 2) {
            const u64 qw = q32(w);
            atomicAdd(&tb[batch][kind == 1 ? B_R : B_T], qw);
            int hb = (int)(P * hist_scale);
            hb = hb > 256 ? 256 : (hb < 0 ? 0 : hb);
            atomicAdd(&th[hb], qw);
            atomic_add_u128(&ts[0], qw);
            atomic_add_u128(&ts[2], O::q32(w * P));
            atomic_add_u128(&ts[4], O::q16(w * P * P));
            atomicAdd(&tc[kind == 1 ? C_EXIT_R : C_EXIT_T], 1ull);
        } else if (kind == 3) {
            atomicAdd(&tb[batch][B_LOST], q32(w));
            atomicAdd(&tc[C_RR_KILL], 1ull);
        } else {
            atomicAdd(&tb[batch][B_GATED], q32(w));
            atomicAdd(&tc[C_GATED], 1ull);
        }
        atomicAdd(&tb[batch][B_A], q32(A));
        atomicAdd(&tb[batch][B_PHOTONS], 1ull);
        atomicAdd(&tc[C_INTERACT], (u64)n_int);
        atomicAdd(&tc[C_SCATTER], (u64)n_scat);
        atomicAdd(&tc[C_RR_SURV], (u64)n_surv);
        atomicAdd(&tc[C_STEPS], (u64)n_steps);
        atomicAdd(&tc[C_SOLID_STEPS], (u64)n_solid);
        if (pid - p.rec_base < p.n_rec) {
            long long *ri = p.rec_ints + (pid - p.rec_base) * 4;
            double *rv = p.rec_vals + (pid - p.rec_base) * 4;
            ri[0] = n_int; ri[1] = (long long)n_steps; ri[2] = kind; ri[3] = n_surv;
            rv[0] = (double)w; rv[1] = (double)P; rv[2] = (double)s; rv[3] = (double)A;
        }
        mode = M_NEW;
    };

    // ---- one voxel step of a lane in M_STEP ------------------------------
    auto step = [&]() {
        // ---- one voxel step ------------------------------------------------
        // The face the ray leaves through does not depend on the phase, so the
        // next voxel and its mask brick are computed first and the brick load
        // is in flight while the current voxel is tallied.
        int ax = 2;                                   // ties: z, then y, then x
        Real seg, tn = 0;
        if constexpr (kExact) {
            const long long jx = ix + (long long)kx * nx, jy = iy + (long long)ky * ny;
            Real d0, d1, d2;
            if (ux > 0) d0 = ((Real)(jx + 1) - px) / ux;
            else if (ux < 0) d0 = ((Real)jx - px) / ux;
            else d0 = kInf;
            if (uy > 0) d1 = ((Real)(jy + 1) - py) / uy;
            else if (uy < 0) d1 = ((Real)jy - py) / uy;
            else d1 = kInf;
            if (uz > 0) d2 = ((Real)(iz + 1) - pz) / uz;
            else if (uz < 0) d2 = ((Real)iz - pz) / uz;
            else d2 = kInf;
            if (d0 < 0) d0 = 0;
            if (d1 < 0) d1 = 0;
            if (d2 < 0) d2 = 0;
            seg = d2;
            if (d1 < seg) { seg = d1; ax = 1; }
            if (d0 < seg) { seg = d0; ax = 0; }
        } else {
            tn = tmz;
            if (tmy < tn) { tn = tmy; ax = 1; }
            if (tmx < tn) { tn = tmx; ax = 0; }
            seg = fmaxf(tn - t, 0.0f);
        }
        // next voxel, branch-free: step the crossed axis, wrap x and y
        int nix = ix + (ax == 0 ? sx : 0);
        int niy = iy + (ax == 1 ? sy : 0);
        const int niz = iz + (ax == 2 ? sz : 0);
        const int wx = (nix >= nx) - (nix < 0), wy = (niy >= ny) - (niy < 0);
        // mirror lateral faces: at the domain edge the photon stays in its
        // voxel and the crossing component of its direction reverses
        const bool rx = kMirror && mirror && wx != 0, ry = kMirror && mirror && wy != 0;
        nix = rx ? ix : (wx > 0 ? 0 : (wx < 0 ? nx - 1 : nix));
        niy = ry ? iy : (wy > 0 ? 0 : (wy < 0 ? ny - 1 : niy));
        const bool leaves = niz < 0 || niz >= nz;
        const u32 nbrick = leaves ? brick : brick_of(nix, niy, niz);
        const u64 nword = (nbrick != brick) ? fetch(nbrick) : word;
        const bool pore = (word >> bit) & 1ull;
        int ev = 0;                                   // 0 cross, 1 interact, 2 gate
        Real need = 0;
        if (!pore) {
            need = mus * seg;                         // tau > 0, so mu_s = 0 never interacts
            if (tau < need) {
                if constexpr (kExact) seg = tau / mus;
                else seg = tau * inv_mus;
                ev = 1;
            }
        }
        if (!(s + seg < s_max)) {                     // NaN-safe: a NaN path is gated
            seg = s_max - s;
            if (!(seg > 0)) seg = 0;
            ev = 2;
        }
        if (++iters > iter_limit) { ev = 2; atomicOr(&tal_ptr->flags, (u32)F_ITER_LIMIT); }

        if (seg > 0) {
            Real dep;
            if (pore) {
                dep = w * seg;
                P += seg;
            } else if (absorb_on) {
                const Real x = mua * seg;
                if constexpr (kExact) {
                    const Real f = O::one_minus_exp(x);
                    dep = w * f / mua;
                    A += w * f;
                    w = w * exp(-x);
                } else {
                    const Real f = small_x ? O::one_minus_exp_small(x) : O::one_minus_exp(x);
                    const Real dA = w * f;
                    dep = dA * inv_mua;
                    A += dA;
                    w = w - dA;
                }
            } else {
                dep = w * seg;
            }
            const u64 q = q32(dep);
            if constexpr (kField) {
                if (q) atomicAdd(field_ptr + (((u64)brick << 6) | bit), q);
            } else {
                atomicAdd(&st.depth[pore ? 1 : 0][bin], q);
            }
            s += seg;
            ++n_steps;
            n_solid += pore ? 0u : 1u;
        }
        if (ev == 0) tau -= need;
        if constexpr (kExact) {
            px += seg * ux;
            py += seg * uy;
            pz += seg * uz;
        }

        if (ev == 2) { finish(4); return; }
        if (ev == 1) {
            if constexpr (!kExact) t += seg;
            mode = M_EVENT;
            return;
        }

        // ---- face crossing: commit the next voxel ----------------------------
        if constexpr (kExact) {
            if (ax == 0) px = ux > 0 ? (Real)(ix + (long long)kx * nx + 1) : (Real)(ix + (long long)kx * nx);
            else if (ax == 1) py = uy > 0 ? (Real)(iy + (long long)ky * ny + 1) : (Real)(iy + (long long)ky * ny);
            else pz = uz > 0 ? (Real)(iz + 1) : (Real)iz;
        } else {
            t = tn;
            if (ax == 0) tmx += dtx;
            if (ax == 1) tmy += dty;
            if (ax == 2) tmz += dtz;
            if (t > 4.0f) {             // rebase the ray parameters at the current point
                tmx -= t; tmy -= t; tmz -= t;
                t = 0;
            }
        }
        if (leaves) { finish(niz < 0 ? 1 : 2); return; }
        ix = nix; iy = niy; iz = niz;
        if (rx) { ux = -ux; sx = -sx; } else kx += wx;
        if (ry) { uy = -uy; sy = -sy; } else ky += wy;
        brick = nbrick;
        word = nword;
        bit = bit_of(ix, iy, iz);
        if constexpr (!kField) bin = (int)(((long long)iz * kNBin) / nz);
    };


    for (;;) {
        // ---- event phase: claims, launches and interactions, compacted ---
        const unsigned parked = __ballot_sync(kFull, mode == M_EVENT || mode == M_NEW);
        const unsigned stepping = __ballot_sync(kFull, mode == M_STEP);
        if (!parked && !stepping) break;                  // warp finished
        if (__popc(parked) >= compact_k || !stepping) {
            // claim photon ids for lanes that need a new photon
            const unsigned want = __ballot_sync(kFull, mode == M_NEW);
            if (want) {
                const int leader = __ffs(want) - 1;
                u64 base = 0;
                if (lane == leader) base = atomicAdd(kBatch ? bp.next : &p.tal->next, (u64)__popc(want));
                base = __shfl_sync(kFull, base, leader);
                if (mode == M_NEW) {
                    const u64 k = base + (u64)__popc(want & lt_mask);
                    if (k >= (kBatch ? bp.total_photons : p.n_photons)) {
                        mode = M_DONE;
                    } else {
                        if constexpr (kBatch) {
                            // the problem owning global index k (last offset <= k)
                            int lo = 0, hi = bp.n_problems - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (bp.problems[mid].offset <= k) lo = mid; else hi = mid - 1;
                            }
                            prob = lo;
                            const BatchProblem &pr = bp.problems[prob];
                            pid = pr.pid_begin + (k - pr.offset);
                            nx = pr.nx; ny = pr.ny; nz = pr.nz; nbx = pr.nbx; nby = pr.nby;
                            bricks_ptr = pr.bricks; field_ptr = pr.field; tal_ptr = pr.tal;
                            mus = pr.f32.mus; mua = pr.f32.mua;
                            inv_mus = pr.f32.inv_mus; inv_mua = pr.f32.inv_mua;
                            s_max = pr.f32.s_max;
                            absorb_on = mua > 0;
                            small_x = pr.small_x != 0;
                            iter_limit = pr.iter_limit;
                            mirror = pr.mirror != 0;
                        } else {
                            pid = pid0 + k;
                        }
                        event = 0;
                        mode = M_EVENT;
                    }
                }
            }
            if (mode == M_EVENT) {
                if constexpr (kBatch) {   // event-time optics of this lane's problem
                    const TransportParams::F32 &f = bp.problems[prob].f32;
                    one_m_g2 = f.one_m_g2; one_p_g2 = f.one_p_g2; one_m_g = f.one_m_g;
                    two_g = f.two_g; inv_2g = f.inv_2g;
                    rr_w = f.rr_weight; rr_m = f.rr_mult; rr_p = f.rr_p; rr_gain = f.rr_gain;
                    hg_iso = bp.problems[prob].hg_iso != 0;
                }
                u32 r[4];
                philox4x32_10(event, 0u, (u32)pid, (u32)(pid >> 32), key0, key1, r);
                if (event == 0) {
                    // ---- launch: uniform over the z = 0 face, +z ----------
                    const Real xr = O::uniform(r[0]) * (Real)nx;
                    const Real yr = O::uniform(r[1]) * (Real)ny;
                    ix = (int)xr; if (ix >= nx) ix = nx - 1;
                    iy = (int)yr; if (iy >= ny) iy = ny - 1;
                    iz = 0;
                    kx = ky = 0;
                    ux = 0; uy = 0; uz = 1;
                    sx = 1; sy = 1; sz = 1;
                    if constexpr (kExact) {
                        px = xr; py = yr; pz = 0;
                    } else {
                        fx = xr - (Real)ix; fy = yr - (Real)iy; fz = 0;
                        tmx = kInf; tmy = kInf; dtx = kInf; dty = kInf; tmz = 1; dtz = 1; t = 0;
                    }
                    w = 1; tau = O::neg_log(O::uniform(r[2])); s = 0; P = 0; A = 0;
                    event = 1; n_int = 0; n_surv = 0; n_scat = 0; n_steps = 0; n_solid = 0; iters = 0;
                    batch = (int)(pid & (kNBatch - 1));
                    brick = brick_of(ix, iy, 0);
                    bit = bit_of(ix, iy, 0);
                    bin = 0;
                    word = fetch(brick);
                    if constexpr (kBatch) atomicAdd(&tal_ptr->counts[C_LAUNCHED], 1ull);
                    else atomicAdd(&st.counts[C_LAUNCHED], 1ull);
                    mode = M_STEP;
                    if (pid - p.rec_base < p.n_rec) {
                        double *site = p.rec_sites + (pid - p.rec_base) * 24;
                        for (int i = 0; i < 24; ++i) site[i] = __longlong_as_double(0x7ff8000000000000ll);
                    }
                } else {
                    // ---- interaction ---------------------------------------
                    ++event;
                    if constexpr (!kExact) {
                        if (ux != 0) { const Real d = (tmx - t) * fabsf(ux); fx = ux > 0 ? 1.0f - d : d; }
                        if (uy != 0) { const Real d = (tmy - t) * fabsf(uy); fy = uy > 0 ? 1.0f - d : d; }
                        if (uz != 0) { const Real d = (tmz - t) * fabsf(uz); fz = uz > 0 ? 1.0f - d : d; }
                        fx = fminf(fmaxf(fx, 0.0f), 1.0f);
                        fy = fminf(fmaxf(fy, 0.0f), 1.0f);
                        fz = fminf(fmaxf(fz, 0.0f), 1.0f);
                    }
                    if (pid - p.rec_base < p.n_rec && n_int < 8) {
                        double *site = p.rec_sites + (pid - p.rec_base) * 24 + n_int * 3;
                        if constexpr (kExact) {
                            site[0] = px; site[1] = py; site[2] = pz;
                        } else {
                            site[0] = (double)(ix + (long long)kx * nx) + (double)fx;
                            site[1] = (double)(iy + (long long)ky * ny) + (double)fy;
                            site[2] = (double)iz + (double)fz;
                        }
                    }
                    ++n_int;
                    bool alive = true;
                    if (w < rr_w) {
                        if (O::uniform(r[3]) < rr_p) {
                            if constexpr (kBatch) atomicAdd(&tal_ptr->batch[batch][B_GAIN], q32(w * rr_gain));
                            else atomicAdd(&st.batch[batch][B_GAIN], q32(w * rr_gain));
                            w = w * rr_m;
                            ++n_surv;
                        } else {
                            finish(3);
                            alive = false;
                        }
                    }
                    if (alive) {
                        // Henyey-Greenstein polar cosine
                        const Real u0 = O::uniform(r[0]);
                        Real cost;
                        if (hg_iso) {
                            cost = (Real)2 * u0 - (Real)1;
                        } else if constexpr (kExact) {
                            const Real tq = one_m_g2 / (one_m_g + two_g * u0);
                            cost = (one_p_g2 - tq * tq) / ((Real)2 * g);
                        } else {
                            const Real tq = one_m_g2 * O::rcp(one_m_g + two_g * u0);
                            cost = (one_p_g2 - tq * tq) * inv_2g;
                        }
                        if (cost < (Real)-1) cost = -1;
                        if (cost > (Real)1) cost = 1;
                        Real sint, sinp, cosp;
                        if constexpr (kExact) sint = sqrt((Real)1 - cost * cost);
                        else sint = sqrtf(fmaxf((1.0f - cost) * (1.0f + cost), 0.0f));
                        O::sincos_2pi(O::uniform(r[1]), &sinp, &cosp);
                        Real vx, vy, vz;
                        if (fabs(uz) > (Real)0.99999) {
                            vx = sint * cosp;
                            vy = sint * sinp;
                            vz = uz >= 0 ? cost : -cost;
                        } else if constexpr (kExact) {
                            const Real tmp = sqrt((Real)1 - uz * uz);
                            vx = sint * (ux * uz * cosp - uy * sinp) / tmp + ux * cost;
                            vy = sint * (uy * uz * cosp + ux * sinp) / tmp + uy * cost;
                            vz = -sint * cosp * tmp + uz * cost;
                        } else {
                            const Real tmp2 = (Real)1 - uz * uz;
                            const Real itmp = O::rsqrt(tmp2);
                            const Real tmp = tmp2 * itmp;
                            vx = sint * (ux * uz * cosp - uy * sinp) * itmp + ux * cost;
                            vy = sint * (uy * uz * cosp + ux * sinp) * itmp + uy * cost;
                            vz = -sint * cosp * tmp + uz * cost;
                        }
                        if constexpr (kExact) {
                            const Real nrm = sqrt(vx * vx + vy * vy + vz * vz);
                            ux = vx / nrm; uy = vy / nrm; uz = vz / nrm;
                        } else {
                            const Real inrm = O::rsqrt(vx * vx + vy * vy + vz * vz);
                            ux = vx * inrm; uy = vy * inrm; uz = vz * inrm;
                        }
                        tau = O::neg_log(O::uniform(r[2]));
                        ++n_scat;
                        sx = ux > 0 ? 1 : -1;
                        sy = uy > 0 ? 1 : -1;
                        sz = uz > 0 ? 1 : -1;
                        if constexpr (!kExact) {   // new ray from (fx, fy, fz)
                            if (ux > 0)      { dtx = O::rcp(ux);  tmx = (1.0f - fx) * dtx; }
                            else if (ux < 0) { dtx = O::rcp(-ux); tmx = fx * dtx; }
                            else             { dtx = kInf; tmx = kInf; }
                            if (uy > 0)      { dty = O::rcp(uy);  tmy = (1.0f - fy) * dty; }
                            else if (uy < 0) { dty = O::rcp(-uy); tmy = fy * dty; }
                            else             { dty = kInf; tmy = kInf; }
                            if (uz > 0)      { dtz = O::rcp(uz);  tmz = (1.0f - fz) * dtz; }
                            else if (uz < 0) { dtz = O::rcp(-uz); tmz = fz * dtz; }
                            else             { dtz = kInf; tmz = kInf; }
                            t = 0;
                        }
                        mode = M_STEP;
                    }
                }
            }
        }
        if (mode != M_STEP) continue;
#pragma unroll 1
        for (int k = 0; k < SPMC_STEPS_PER_PASS; ++k) {   // voxel steps per pass of
            if (mode != M_STEP) break;                     // the warp-level event check
            step();
        }
    }

    // ---- retire: flush the block tallies with integer atomics -----------
    if constexpr (kBatch) return;
    __syncthreads();
    DevTallies *g_t = p.tal;
    for (int i = threadIdx.x; i < kNBatch * B_N; i += blockDim.x) {
        const u64 x = (&st.batch[0][0])[i];
        if (x) atomicAdd(&g_t->batch[0][0] + i, x);
    }
    for (int i = threadIdx.x; i < C_N; i += blockDim.x)
        if (st.counts[i]) atomicAdd(&g_t->counts[i], st.counts[i]);
    for (int i = threadIdx.x; i < kNHist; i += blockDim.x)
        if (st.hist[i]) atomicAdd(&g_t->hist[i], st.hist[i]);
    if (threadIdx.x < 3) {
        const u64 lo = st.sums[2 * threadIdx.x], hi = st.sums[2 * threadIdx.x + 1];
        atomic_add_u128(&g_t->sums[2 * threadIdx.x], lo);
        if (hi) atomicAdd(&g_t->sums[2 * threadIdx.x + 1], hi);
    }
    if constexpr (!kField) {
        for (int i = threadIdx.x; i < 2 * kNBin; i += blockDim.x) {
            const u64 x = (&st.depth[0][0])[i];
            if (x) atomic_add_u128(&g_t->depth[i / kNBin][i % kNBin][0], x);
        }
    }
}

template <typename Real>
cudaError_t launch_transport(const TransportParams &p, bool field, int blocks, int threads,
                             size_t smem, cudaStream_t s) {
    const BatchParams none{};
    if (p.mirror) {
        if (field) transport_kernel<Real, true, false, true><<<blocks, threads, smem, s>>>(p, none);
        else transport_kernel<Real, false, false, true><<<blocks, threads, smem, s>>>(p, none);
    } else {
        if (field) transport_kernel<Real, true, false, false><<<blocks, threads, smem, s>>>(p, none);
        else transport_kernel<Real, false, false, false><<<blocks, threads, smem, s>>>(p, none);
    }
    return cudaGetLastError();
}

template <typename Real>
const void *kernel_ptr(bool field, bool mirror) {
    if (mirror)
        return field ? reinterpret_cast<const void *>(&transport_kernel<Real, true, false, true>)
                     : reinterpret_cast<const void *>(&transport_kernel<Real, false, false, true>);
    return field ? reinterpret_cast<const void *>(&transport_kernel<Real, true, false, false>)
                 : reinterpret_cast<const void *>(&transport_kernel<Real, false, false, false>);
}

template <typename Real>
cudaError_t occupancy(bool field, bool mirror, int threads, size_t smem, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel_ptr<Real>(field, mirror), threads,
                                                         smem);
}

}  // namespace spmc
