// spmc_transport_f32.cuh -- the FP32 production transport kernel (sm_103a).
//
// Same method and same per-photon random streams as the generic kernel in
// spmc_transport.cuh (arXiv 2604.13929, Sec. 2.5, App. B; HG scattering,
// periodic or mirror lateral faces), written for issue-slot economy:
//
//  * a pass of the warp takes up to `steps_per_pass` voxel steps per lane
//    without any warp vote; a lane whose photon needs an event (interaction,
//    exit, path cap, new photon) leaves the pass and parks;
//  * pore and solid voxels share one branch-free step: the phase only picks
//    the coefficients (mu_s, mu_a are zero in pores), and the deposit uses
//    g(x) = (1 - e^-x)/x, which is 1 in pores, so no lane diverges on the
//    phase of its voxel;
//  * every event -- launch, interaction, roulette, exit and path-cap
//    tallies -- runs in the compacted event phase, where the warp serves
//    all parked lanes at once; the stepping loop carries none of that code;
//  * in the depth-profile tally mode a lane sums its deposits of the current
//    depth bin per phase in registers (exact integers) and adds them to the
//    block's shared-memory bins only when the photon changes bin or ends.
//
// Batched launches (kBatch) run many problems (masks, sizes, optics) in one
// persistent launch: a warp claims chunks of photons of ONE problem at a
// time, so the problem's constants are uniform across the warp and its block
// tallies stay in shared memory (one set per warp, flushed to the problem's
// global tallies when the warp moves on to another problem).  A warp changes
// problem only once every photon it carries has finished.
//
// Per photon the arithmetic depends only on its id, its problem and the mask,
// never on the warp it runs in, so the integer tallies are bit-identical
// across launch shapes, compaction thresholds, steps per pass, run splits and
// batched versus separate launches.
#pragma once

#include "spmc_transport.cuh"

namespace spmc {

// Resident 256-thread CTAs per SM requested from the register allocator for
// the voxel-field kernels (the depth-profile kernels ask for 4: without the
// field REDs they gain from the extra warps, the field kernels did not).
#ifndef SPMC_F32_MIN_BLOCKS
#define SPMC_F32_MIN_BLOCKS 3
#endif

// Lane modes.  L_WAIT: a lane that needs a new photon while its warp drains
// the photons of the current problem before moving on to the next one.
enum { L_STEP = 0, L_INTERACT = 1, L_FINISH = 2, L_NEW = 3, L_WAIT = 4, L_DONE = 5 };

template <bool kField, bool kMirror, bool kBatch>
__global__ void __launch_bounds__(256, kBatch ? 3 : (kField ? SPMC_F32_MIN_BLOCKS : 4))
transport_f32_kernel(const TransportParams p, const BatchParams bp) {
    // dynamic shared memory: the staged entry slab of mask bricks, or
    // (batched) one SmemTallies per warp
    extern __shared__ u64 s_bricks[];
    __shared__ SmemTallies st_one;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    SmemTallies &st = kBatch ? reinterpret_cast<SmemTallies *>(s_bricks)[warp] : st_one;
    {
        u64 *z = kBatch ? s_bricks : reinterpret_cast<u64 *>(&st_one);
        const int n = (int)(sizeof(SmemTallies) / 8) * (kBatch ? (int)(blockDim.x >> 5) : 1);
        for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = 0;
        if constexpr (!kBatch)
            for (int i = threadIdx.x; i < p.smem_bricks; i += blockDim.x) s_bricks[i] = __ldg(p.bricks + i);
    }
    __syncthreads();

    using O = Ops<float>;
    const unsigned kFull = 0xffffffffu;
    const unsigned lt_mask = (1u << lane) - 1u;
    const float kInf = O::inf();
    const int ck_opt = kBatch ? bp.compact_k : p.compact_k;
    const int compact_k = ck_opt < 1 ? 1 : (ck_opt > 32 ? 32 : ck_opt);
    const int spp_opt = kBatch ? bp.steps_per_pass : p.steps_per_pass;
    const int spp = spp_opt < 1 ? 1 : spp_opt;
    const u32 key0 = kBatch ? bp.key0 : p.key0, key1 = kBatch ? bp.key1 : p.key1;

    // ---- problem constants: kernel parameters, or (batched) the warp's
    // current problem, reloaded when the warp moves to another problem ----
    int nx = p.nx, ny = p.ny, nz = p.nz, nbx = p.nbx, nby = p.nby;
    const u64 *bricks = p.bricks;
    u64 *field = p.field;
    DevTallies *tal = p.tal;
    float mus = p.f32.mus, mua = p.f32.mua, inv_mus = p.f32.inv_mus, s_max = p.f32.s_max;
    u32 iter_limit = p.iter_limit > 0xffffffffull ? 0xffffffffu : (u32)p.iter_limit;
    bool small_x = p.small_x != 0;
    bool mirror = kMirror && p.mirror != 0;
    int prob = -1;                      // batched: the warp's current problem
    u64 ck_next = 0, ck_end = 0;        // batched: photon indices left in its chunk
    long long pend = -1;                // batched: a claimed chunk not yet started
    const u64 pid0 = kBatch ? 0 : (p.pid_begin_dev ? *p.pid_begin_dev : p.pid_begin);

    auto brick_of = [&](int ix, int iy, int iz) -> u32 {
        return ((u32)(iz >> 2) * (u32)nby + (u32)(iy >> 2)) * (u32)nbx + (u32)(ix >> 2);
    };
    auto bit_of = [&](int ix, int iy, int iz) -> u32 {
        return (u32)(((iz & 3) << 4) | ((iy & 3) << 2) | (ix & 3));
    };
    auto fetch = [&](u32 b) -> u64 {
        if constexpr (kBatch) return __ldg(bricks + b);
        else return ((int)b < p.smem_bricks) ? s_bricks[b] : __ldg(p.bricks + b);
    };
    auto bin_of = [&](int iz) -> int {
        return p.bin_exact ? (int)__umulhi((u32)iz * 64u, p.bin_mul) : (int)(((long long)iz * kNBin) / nz);
    };
    // event-time constants (HG, roulette, histogram) of the current problem
    auto ev = [&]() -> const TransportParams::F32 & {
        if constexpr (kBatch) return bp.problems[prob].f32;
        else return p.f32;
    };
    // batched: add the warp's shared-memory tallies to problem q's global
    // tallies and clear them (all 32 lanes, converged)
    auto flush_warp = [&](int q) {
        DevTallies *g_t = bp.problems[q].tal;
        for (int i = lane; i < kNBatch * B_N; i += 32) {
            u64 *x = &st.batch[0][0] + i;
            if (*x) atomicAdd(&g_t->batch[0][0] + i, *x);
            *x = 0;
        }
        for (int i = lane; i < C_N; i += 32) {
            if (st.counts[i]) atomicAdd(&g_t->counts[i], st.counts[i]);
            st.counts[i] = 0;
        }
        for (int i = lane; i < kNHist; i += 32) {
            if (st.hist[i]) atomicAdd(&g_t->hist[i], st.hist[i]);
            st.hist[i] = 0;
        }
        if (lane < 3) {
            const u64 lo = st.sums[2 * lane], hi = st.sums[2 * lane + 1];
            atomic_add_u128(&g_t->sums[2 * lane], lo);
            if (hi) atomicAdd(&g_t->sums[2 * lane + 1], hi);
            st.sums[2 * lane] = 0;
            st.sums[2 * lane + 1] = 0;
        }
        __syncwarp();
    };

    // ---- lane state ----------------------------------------------------
    int mode = L_NEW, kind = 0;
    u64 pid = 0;
    int ix = 0, iy = 0, iz = 0, kx = 0, ky = 0, bin = 0;
    int sx = 1, sy = 1, sz = 1;
    u32 brick = 0, bit = 0;
    u64 word = 0;
    float ux = 0, uy = 0, uz = 1;
    float w = 1, tau = 0, s = 0, P = 0, A = 0;
    float tmx = kInf, tmy = kInf, tmz = 1, dtx = kInf, dty = kInf, dtz = 1, t = 0;
    float fx = 0, fy = 0, fz = 0;
    u32 event = 1, n_int = 0, n_surv = 0, n_steps = 0, n_solid = 0, iters = 0;
    u64 acc_s = 0, acc_p = 0;           // profile mode: current bin's solid / pore sums
    auto flush_bin = [&]() {
        if constexpr (!kField) {
            if (acc_s) atomicAdd(&st.depth[0][bin], acc_s);
            if (acc_p) atomicAdd(&st.depth[1][bin], acc_p);
            acc_s = 0;
            acc_p = 0;
        }
    };

    for (;;) {
        // ---- event phase: exits, claims, launches, interactions ------------
        const unsigned parked = __ballot_sync(kFull, mode == L_INTERACT || mode == L_FINISH || mode == L_NEW);
        const unsigned stepping = __ballot_sync(kFull, mode == L_STEP);
        if (!parked && !stepping) break;
        if (__popc(parked) >= compact_k || !stepping) {
            if (mode == L_FINISH) {
                // kind: 1 R, 2 T, 3 roulette, 4 path cap
                flush_bin();
                const int b = (int)(pid & (kNBatch - 1));
                if (kind <= 2) {
                    const u64 qw = q32_bits(w);
                    atomicAdd(&st.batch[b][kind == 1 ? B_R : B_T], qw);
                    int hb = (int)(P * ev().hist_scale);
                    hb = hb > 256 ? 256 : (hb < 0 ? 0 : hb);
                    atomicAdd(&st.hist[hb], qw);
                    atomic_add_u128(&st.sums[0], qw);
                    atomic_add_u128(&st.sums[2], O::q32(w * P));
                    atomic_add_u128(&st.sums[4], O::q16(w * P * P));
                    atomicAdd(&st.counts[kind == 1 ? C_EXIT_R : C_EXIT_T], 1ull);
                } else if (kind == 3) {
                    atomicAdd(&st.batch[b][B_LOST], q32_bits(w));
                    atomicAdd(&st.counts[C_RR_KILL], 1ull);
                } else {
                    atomicAdd(&st.batch[b][B_GATED], q32_bits(w));
                    atomicAdd(&st.counts[C_GATED], 1ull);
                }
                atomicAdd(&st.batch[b][B_A], q32_bits(A));
                atomicAdd(&st.batch[b][B_PHOTONS], 1ull);
                atomicAdd(&st.counts[C_INTERACT], (u64)n_int);
                atomicAdd(&st.counts[C_SCATTER], (u64)(n_int - (kind == 3 ? 1u : 0u)));
                atomicAdd(&st.counts[C_RR_SURV], (u64)n_surv);
                atomicAdd(&st.counts[C_STEPS], (u64)n_steps);
                atomicAdd(&st.counts[C_SOLID_STEPS], (u64)n_solid);
                if (!kBatch && pid - p.rec_base < p.n_rec) {
                    long long *ri = p.rec_ints + (pid - p.rec_base) * 4;
                    double *rv = p.rec_vals + (pid - p.rec_base) * 4;
                    ri[0] = n_int; ri[1] = (long long)n_steps; ri[2] = kind; ri[3] = n_surv;
                    rv[0] = (double)w; rv[1] = (double)P; rv[2] = (double)s; rv[3] = (double)A;
                }
                mode = L_NEW;
            }
            // ---- claim photon ids for lanes that need a new photon ----------
            if constexpr (!kBatch) {
                const unsigned want = __ballot_sync(kFull, mode == L_NEW);
                if (want) {
                    const int leader = __ffs(want) - 1;
                    u64 base = 0;
                    if (lane == leader) base = atomicAdd(&p.tal->next, (u64)__popc(want));
                    base = __shfl_sync(kFull, base, leader);
                    if (mode == L_NEW) {
                        const u64 k = base + (u64)__popc(want & lt_mask);
                        if (k >= p.n_photons) {
                            mode = L_DONE;
                        } else {
                            pid = pid0 + k;
                            event = 0;
                            mode = L_INTERACT;       // event 0 is the launch
                        }
                    }
                }
            } else {
                // photons come from the warp's chunk of its current problem;
                // a chunk of another problem starts only after the warp drained
                if (mode == L_WAIT) mode = L_NEW;
                unsigned want = __ballot_sync(kFull, mode == L_NEW);
                while (want) {                       // warp-uniform loop
                    if (ck_next < ck_end) {
                        const u64 give = ck_end - ck_next, n_want = (u64)__popc(want);
                        const u64 rank = (u64)__popc(want & lt_mask);
                        if (mode == L_NEW && rank < give) {
                            pid = bp.problems[prob].pid_begin + ck_next + rank;
                            event = 0;
                            mode = L_INTERACT;
                        }
                        ck_next += give < n_want ? give : n_want;
                        want = __ballot_sync(kFull, mode == L_NEW);
                        continue;
                    }
                    if (pend < 0) {
                        u64 c = 0;
                        if (lane == 0) c = atomicAdd(bp.next, 1ull);
                        pend = (long long)__shfl_sync(kFull, c, 0);
                    }
                    if ((u64)pend >= bp.total_chunks) {
                        if (mode == L_NEW) mode = L_DONE;
                        break;
                    }
                    // the problem owning chunk pend (last chunk_begin <= pend)
                    int lo = 0, hi = bp.n_problems - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (bp.problems[mid].chunk_begin <= (u64)pend) lo = mid; else hi = mid - 1;
                    }
                    if (lo != prob) {
                        const unsigned busy = __ballot_sync(kFull, mode == L_STEP || mode == L_INTERACT ||
                                                                       mode == L_FINISH);
                        if (busy) {
                            if (mode == L_NEW) mode = L_WAIT;
                            break;
                        }
                        if (prob >= 0) flush_warp(prob);
                        prob = lo;
                        const BatchProblem &pr = bp.problems[prob];
                        nx = pr.nx; ny = pr.ny; nz = pr.nz; nbx = pr.nbx; nby = pr.nby;
                        bricks = pr.bricks; field = pr.field; tal = pr.tal;
                        mus = pr.f32.mus; mua = pr.f32.mua; inv_mus = pr.f32.inv_mus; s_max = pr.f32.s_max;
                        iter_limit = pr.iter_limit;
                        small_x = pr.small_x != 0;
                        mirror = kMirror && pr.mirror != 0;
                    }
                    const BatchProblem &pr = bp.problems[prob];
                    ck_next = ((u64)pend - pr.chunk_begin) * (u64)bp.chunk;
                    ck_end = ck_next + (u64)bp.chunk < pr.n_photons ? ck_next + (u64)bp.chunk : pr.n_photons;
                    pend = -1;
                }
            }
            if (mode == L_INTERACT) {
                u32 r[4];
                philox4x32_10(event, 0u, (u32)pid, (u32)(pid >> 32), key0, key1, r);
                if (event == 0) {
                    // ---- launch: uniform over the z = 0 face, direction +z
                    const float xr = O::uniform(r[0]) * (float)nx;
                    const float yr = O::uniform(r[1]) * (float)ny;
                    ix = (int)xr; if (ix >= nx) ix = nx - 1;
                    iy = (int)yr; if (iy >= ny) iy = ny - 1;
                    iz = 0; kx = ky = 0;
                    ux = 0; uy = 0; uz = 1;
                    sx = 1; sy = 1; sz = 1;
                    fx = xr - (float)ix; fy = yr - (float)iy; fz = 0;
                    tmx = kInf; tmy = kInf; dtx = kInf; dty = kInf; tmz = 1; dtz = 1; t = 0;
                    w = 1; tau = O::neg_log(O::uniform(r[2])); s = 0; P = 0; A = 0;
                    event = 1; n_int = 0; n_surv = 0; n_steps = 0; n_solid = 0; iters = 0;
                    brick = brick_of(ix, iy, 0);
                    bit = bit_of(ix, iy, 0);
                    bin = 0;
                    word = fetch(brick);
                    atomicAdd(&st.counts[C_LAUNCHED], 1ull);
                    mode = L_STEP;
                    if (!kBatch && pid - p.rec_base < p.n_rec) {
                        double *site = p.rec_sites + (pid - p.rec_base) * 24;
                        for (int i = 0; i < 24; ++i) site[i] = __longlong_as_double(0x7ff8000000000000ll);
                    }
                } else {
                    // ---- interaction: position within the voxel, record, roulette
                    const TransportParams::F32 &c = ev();
                    ++event;
                    if (ux != 0) { const float d = (tmx - t) * fabsf(ux); fx = ux > 0 ? 1.0f - d : d; }
                    if (uy != 0) { const float d = (tmy - t) * fabsf(uy); fy = uy > 0 ? 1.0f - d : d; }
                    if (uz != 0) { const float d = (tmz - t) * fabsf(uz); fz = uz > 0 ? 1.0f - d : d; }
                    fx = fminf(fmaxf(fx, 0.0f), 1.0f);
                    fy = fminf(fmaxf(fy, 0.0f), 1.0f);
                    fz = fminf(fmaxf(fz, 0.0f), 1.0f);
                    if (!kBatch && pid - p.rec_base < p.n_rec && n_int < 8) {
                        double *site = p.rec_sites + (pid - p.rec_base) * 24 + n_int * 3;
                        site[0] = (double)(ix + (long long)kx * nx) + (double)fx;
                        site[1] = (double)(iy + (long long)ky * ny) + (double)fy;
                        site[2] = (double)iz + (double)fz;
                    }
                    ++n_int;
                    mode = L_STEP;
                    if (w < c.rr_weight) {
                        if (O::uniform(r[3]) < c.rr_p) {
                            atomicAdd(&st.batch[pid & (kNBatch - 1)][B_GAIN], q32_bits(w * c.rr_gain));
                            w = w * c.rr_mult;
                            ++n_surv;
                        } else {
                            mode = L_FINISH;
                            kind = 3;
                        }
                    }
                    if (mode == L_STEP) {
                        // Henyey-Greenstein polar cosine, uniform azimuth
                        const float u0 = O::uniform(r[0]);
                        float cost;
                        if (kBatch ? bp.problems[prob].hg_iso != 0 : p.hg_iso != 0) {
                            cost = 2.0f * u0 - 1.0f;
                        } else {
                            const float tq = c.one_m_g2 * O::rcp(c.one_m_g + c.two_g * u0);
                            cost = (c.one_p_g2 - tq * tq) * c.inv_2g;
                        }
                        cost = fminf(fmaxf(cost, -1.0f), 1.0f);
                        const float sint = sqrtf(fmaxf((1.0f - cost) * (1.0f + cost), 0.0f));
                        // azimuth 2 pi u, evaluated as 2 pi u - pi in (-pi, pi)
                        // where the SFU sine and cosine are accurate; both
                        // change sign under the shift
                        float sinp, cosp;
                        __sincosf(fmaf(O::uniform(r[1]), 6.28318530717958648f, -3.14159265358979324f),
                                  &sinp, &cosp);
                        sinp = -sinp;
                        cosp = -cosp;
                        float vx, vy, vz;
                        if (fabsf(uz) > 0.99999f) {
                            vx = sint * cosp;
                            vy = sint * sinp;
                            vz = uz >= 0 ? cost : -cost;
                        } else {
                            const float tmp2 = 1.0f - uz * uz;
                            const float itmp = rsqrtf(tmp2);
                            const float tmp = tmp2 * itmp;
                            vx = sint * (ux * uz * cosp - uy * sinp) * itmp + ux * cost;
                            vy = sint * (uy * uz * cosp + ux * sinp) * itmp + uy * cost;
                            vz = -sint * cosp * tmp + uz * cost;
                        }
                        const float inrm = rsqrtf(vx * vx + vy * vy + vz * vz);
                        ux = vx * inrm; uy = vy * inrm; uz = vz * inrm;
                        tau = O::neg_log(O::uniform(r[2]));
                        sx = ux > 0 ? 1 : -1;
                        sy = uy > 0 ? 1 : -1;
                        sz = uz > 0 ? 1 : -1;
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
                }
            }
        }
        if (mode != L_STEP) continue;

        // ---- stepping: up to spp voxel steps, no warp vote ------------------
#pragma unroll 1
        for (int k = 0; k < spp; ++k) {
            // next face: ties resolve to z, then y, then x
            float tn = tmz;
            const bool ylt = tmy < tn;
            tn = ylt ? tmy : tn;
            const bool xlt = tmx < tn;
            tn = xlt ? tmx : tn;
            const bool ax_x = xlt, ax_y = !xlt && ylt, ax_z = !xlt && !ylt;
            float seg = fmaxf(tn - t, 0.0f);

            // the voxel behind that face, and its mask brick (load in flight
            // while this voxel is tallied)
            int nix = ax_x ? ix + sx : ix;
            int niy = ax_y ? iy + sy : iy;
            const int niz = ax_z ? iz + sz : iz;
            const bool wx = (unsigned)nix >= (unsigned)nx, wy = (unsigned)niy >= (unsigned)ny;
            const bool rx = mirror && wx, ry = mirror && wy;
            nix = rx ? ix : (wx ? (nix < 0 ? nx - 1 : 0) : nix);
            niy = ry ? iy : (wy ? (niy < 0 ? ny - 1 : 0) : niy);
            const bool leaves = (unsigned)niz >= (unsigned)nz;
            const u32 nbrick = leaves ? brick : brick_of(nix, niy, niz);
            const u64 nword = (nbrick != brick) ? fetch(nbrick) : word;

            // this voxel: optical depth, path cap, deposit
            const bool pore = (word >> bit) & 1ull;
            const float mus_v = pore ? 0.0f : mus;
            const float mua_v = pore ? 0.0f : mua;
            const float need = mus_v * seg;
            const bool inter = tau < need;           // never in pores (tau > 0)
            seg = inter ? tau * inv_mus : seg;
            bool gate = !(s + seg < s_max);          // NaN-safe: a NaN path is gated
            if (gate) seg = fmaxf(s_max - s, 0.0f);
            if (++iters > iter_limit) { gate = true; atomicOr(&tal->flags, (u32)F_ITER_LIMIT); }
            const float xa = mua_v * seg;
            float gx;                                // (1 - e^-x)/x, 1 at x = 0
            if (small_x) {
                gx = fmaf(-xa, 1.0f / 120.0f, 1.0f / 24.0f);
                gx = fmaf(-xa, gx, 1.0f / 6.0f);
                gx = fmaf(-xa, gx, 0.5f);
                gx = fmaf(-xa, gx, 1.0f);
            } else {
                gx = xa > 0.0f ? __fdividef(-expm1f(-xa), xa) : 1.0f;
            }
            const float dep = (w * seg) * gx;        // integral of w e^(-mu_a s) ds
            const float dA = dep * mua_v;
            A += dA;
            w -= dA;
            P += pore ? seg : 0.0f;
            s += seg;
            n_steps += seg > 0.0f ? 1u : 0u;
            n_solid += (seg > 0.0f && !pore) ? 1u : 0u;
            const u64 q = q32_bits(dep);
            if constexpr (kField) {
                if constexpr (kBatch) {   // field pointer from the problem table: say it is global
                    if (q) red_add_global(field + (((u64)brick << 6) | bit), q);
                } else {
                    if (q) atomicAdd(field + (((u64)brick << 6) | bit), q);
                }
            } else {
                if (pore) acc_p += q; else acc_s += q;
            }
            if (gate || inter || leaves) {           // the photon leaves the pass
                if (gate) { mode = L_FINISH; kind = 4; }
                else if (inter) { t += seg; mode = L_INTERACT; }
                else { mode = L_FINISH; kind = niz < 0 ? 1 : 2; }
                break;
            }
            tau -= need;

            // face crossing: commit the next voxel
            t = tn;
            if (ax_x) tmx += dtx;
            if (ax_y) tmy += dty;
            if (ax_z) tmz += dtz;
            if (t > 4.0f) {          // rebase the ray parameters at the current point
                tmx -= t; tmy -= t; tmz -= t;
                t = 0;
            }
            if (rx) { ux = -ux; sx = -sx; } else if (wx) kx += sx;
            if (ry) { uy = -uy; sy = -sy; } else if (wy) ky += sy;
            ix = nix; iy = niy; iz = niz;
            brick = nbrick;
            word = nword;
            bit = bit_of(ix, iy, iz);
            if constexpr (!kField) {
                if (ax_z) {
                    const int nb = bin_of(iz);
                    if (nb != bin) { flush_bin(); bin = nb; }
                }
            }
        }
    }

    // ---- retire: flush the block tallies with integer atomics -----------
    if constexpr (kBatch) {
        if (prob >= 0) flush_warp(prob);
        return;
    }
    __syncthreads();
    DevTallies *g_t = p.tal;
    for (int i = threadIdx.x; i < kNBatch * B_N; i += blockDim.x) {
        const u64 v = (&st.batch[0][0])[i];
        if (v) atomicAdd(&g_t->batch[0][0] + i, v);
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
            const u64 v = (&st.depth[0][0])[i];
            if (v) atomic_add_u128(&g_t->depth[i / kNBin][i % kNBin][0], v);
        }
    }
}

}  // namespace spmc
