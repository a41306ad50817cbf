// spnn_gemm.cu -- the tensor-core GEMM kernels of the surrogate: rows_kernel
// (forward and input-gradient layers), wgrad_kernel and wgrad_halo_kernel
// (weight gradients).
//
// All are warp-specialised, 192 threads:
//   warp 0      TMA producer: fills a ring of shared-memory stages,
//   warp 1      allocates TMEM and issues tcgen05.mma,
//   warps 2..5  epilogue: tcgen05.ld of the FP32 accumulators, fused
//               bias / residual / ReLU / ReLU-derivative mask, BF16 stores
//               (FP32 atomics for weight gradients).
// The MMA warp (and the weight-gradient producers) walk their K loop with all
// 32 lanes so that descriptor and coordinate arithmetic stays warp-uniform; one
// elected lane issues.  K loops carry their stage index and tile origin as
// running values: integer division per step costs a lone thread hundreds of
// cycles.  Stages hand over with mbarriers: "full" completes when TMA bytes
// land, "empty" when the MMAs that read the stage retire (tcgen05.commit).
// Every wait is bounded by kWaitLimitNs; a timeout sets an error flag, and the
// CTA still releases its TMEM and exits.
#include "spnn_internal.cuh"
#include "spnn_umma.cuh"

namespace spnn {

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// Stage index and wrap count of a ring of S stages, advanced once per K-step
// (the K loops avoid integer division, which costs a lone thread hundreds of
// cycles per step).
struct Ring {
    int s = 0;
    uint32_t r = 0;
    __device__ __forceinline__ void next(int S) {
        if (++s == S) {
            s = 0;
            ++r;
        }
    }
};

// Origin of the tile after (x0, y0, z0, b0): the increment of tile_origin.
__device__ __forceinline__ void tile_next(const TileGrid& g, int& x0, int& y0, int& z0, int& b0) {
    if ((x0 += g.bx) < g.nx * g.bx) return;
    x0 = 0;
    if ((y0 += g.by) < g.ny * g.by) return;
    y0 = 0;
    if ((z0 += g.bz) < g.nz * g.bz) return;
    z0 = 0;
    b0 += g.bb;
}

// 16 channels of one voxel: 8 at p[0..7] and 8 one chunk plane further.
__device__ __forceinline__ void load16_planes(const __nv_bfloat16* p, long long plane, float (&f)[16]) {
    uint4 u[2] = {*reinterpret_cast<const uint4*>(p), *reinterpret_cast<const uint4*>(p + plane)};
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(u);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}

// TMA box of chunk plane c8: chunk-plane map (8x, y, z, b, c8) or stride-2 view (0, x, y, z, c8 B + b).
__device__ __forceinline__ void load_box(uint32_t dst, const CUtensorMap* m, uint32_t bar, bool strided, int c8,
                                         int x, int y, int z, int b, int B) {
    if (strided)
        tma_load_5d(dst, m, bar, 0, x, y, z, c8 * B + b);
    else
        tma_load_5d(dst, m, bar, 8 * x, y, z, b, c8);
}

// The MMAs of one conv3 K-step: nine (dz, dy) taps x EH K-slices of 16
// channels x MT subtiles.  Descriptors are the step's base descriptors plus
// start-address offsets in 16-byte units (no carry: every address is inside
// shared memory): tap_off[t9] for the tap, a_koff per K-slice, 128 (2048
// bytes) per subtile; B holds [slice][tap] blocks of n_tile rows.  Unrolled so
// that one instruction stream issues every MMA back to back.
template <int MT, int EH>
__device__ __forceinline__ void issue_conv_step(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                                const uint32_t (&tap_off)[9], uint32_t a_koff, uint32_t n_tile,
                                                uint32_t idesc, bool first) {
#pragma unroll
    for (int t9 = 0; t9 < 9; ++t9)
#pragma unroll
        for (int i = 0; i < EH; ++i) {
            const uint64_t bd = bdesc + (uint64_t)((uint32_t)(2 * i * 9 + t9) * n_tile);
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const uint64_t ad = adesc + (uint64_t)(tap_off[t9] + (uint32_t)i * a_koff + 128u * m);
                umma_bf16(tmem + (uint32_t)m * n_tile, ad, bd, idesc, (first && t9 == 0 && i == 0) ? 0u : 1u);
            }
        }
}

__device__ __forceinline__ void issue_conv_step(int mt, int eh, uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                                const uint32_t (&tap_off)[9], uint32_t a_koff, uint32_t n_tile,
                                                uint32_t idesc, bool first) {
    if (mt == 4 && eh == 2)
        issue_conv_step<4, 2>(tmem, adesc, bdesc, tap_off, a_koff, n_tile, idesc, first);
    else if (mt == 4)
        issue_conv_step<4, 1>(tmem, adesc, bdesc, tap_off, a_koff, n_tile, idesc, first);
    else if (mt == 2 && eh == 2)
        issue_conv_step<2, 2>(tmem, adesc, bdesc, tap_off, a_koff, n_tile, idesc, first);
    else if (mt == 2)
        issue_conv_step<2, 1>(tmem, adesc, bdesc, tap_off, a_koff, n_tile, idesc, first);
    else if (eh == 2)
        issue_conv_step<1, 2>(tmem, adesc, bdesc, tap_off, a_koff, n_tile, idesc, first);
    else
        issue_conv_step<1, 1>(tmem, adesc, bdesc, tap_off, a_koff, n_tile, idesc, first);
}

// ------------------------------------------------------------------------
// Rows GEMM (forward, input-gradient and transposed-conv layers).
// A tile: kc_step chunk planes of 128 rows x 16 bytes (2 KB each), K-major;
// B tile: kc_step planes of n_tile rows x 16 bytes, K-major.
//
// Persistent, dynamically scheduled: the producer claims the next tile from a
// global counter (so any grid size is safe: a CTA that becomes resident only
// after the others have claimed every tile finds none and exits; tiles are
// claimed in grid order) and hands its index to the MMA and epilogue warps
// through a ring of four shared slots (tile_full / tile_empty; index -1 ends
// the CTA).  The stage ring runs on
// across tiles, so the next tile's operands load while the current one
// multiplies.  The accumulators of consecutive tiles alternate
// between two TMEM buffers (nbuf = 2 when they fit in 512 columns): the
// epilogue of tile i reads one buffer while the MMAs of tile i + 1 fill the
// other.  acc_full[b] completes when the MMAs of a tile retire
// (tcgen05.commit), acc_empty[b] when the four epilogue warps have read it.
// ------------------------------------------------------------------------

// Origin of tile t (32-bit: a lone thread divides once per tile).
__device__ __forceinline__ void tile_origin_u32(const TileGrid& g, uint32_t t, int& x0, int& y0, int& z0,
                                                int& b0) {
    uint32_t q = t / (uint32_t)g.nx;
    x0 = (int)(t - q * (uint32_t)g.nx) * g.bx;
    t = q;
    q = t / (uint32_t)g.ny;
    y0 = (int)(t - q * (uint32_t)g.ny) * g.by;
    t = q;
    q = t / (uint32_t)g.nz;
    z0 = (int)(t - q * (uint32_t)g.nz) * g.bz;
    b0 = (int)q * g.bb;
}

__global__ void __launch_bounds__(kThreads, 1) rows_kernel(const __grid_constant__ RowsParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    const int S = p.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * p.stage_bytes);
    volatile int* tile_slot = reinterpret_cast<volatile int*>(bars + 2 * S + 12);   // [4]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 14);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = smem_u32(bars);
    const uint32_t acc_full = bar0 + 16u * S, acc_empty = acc_full + 16u;   // [2] each
    const uint32_t tile_full = acc_empty + 16u, tile_empty = tile_full + 32u;   // [4] each
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t acc_cols = (uint32_t)(p.mt * p.n_tile);   // one accumulator per subtile
    const uint32_t ncols = tmem_cols(p.nbuf * (int)acc_cols);

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(bar0 + 8u * s, 1);
            mbar_init(bar0 + 8u * (S + s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full + 8u * b, 1);
            mbar_init(acc_empty + 8u * b, 4);
        }
        for (int b = 0; b < 4; ++b) {
            mbar_init(tile_full + 8u * b, 1);
            mbar_init(tile_empty + 8u * b, 5);   // the MMA warp and the four epilogue warps
        }
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    int* const tile_ctr = p.tile_ctr + blockIdx.y;

    const bool conv = p.tap_mode == TAP_SHIFT3;
    if (warp == 0) {
        if (lane == 0) {
            const int gpt = conv ? p.kc_total / p.E : p.kc_total / p.kc_step;
            const uint32_t tx = p.a_stage_bytes + p.b_stage_bytes;
            Ring q;
            bool ok = true;
            int claimed = atomicAdd(tile_ctr, 1);
            for (uint32_t it = 0; ok; ++it) {
                // publish the claimed tile's index (-1: none left) in slot it % 4
                const uint32_t ts = it & 3u, tu = it >> 2;
                if (tu > 0 && !mbar_wait(tile_empty + 8u * ts, (tu - 1) & 1u, kWaitLimitNs)) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    break;
                }
                const int t = claimed < p.tiles ? claimed : -1;
                tile_slot[ts] = t;
                mbar_arrive(tile_full + 8u * ts);
                if (t < 0) break;
                // claim the following tile now: the atomic's latency hides behind this tile's loads
                claimed = atomicAdd(tile_ctr, 1);
                int x0, y0, z0, b0;
                tile_origin_u32(p.g, (uint32_t)t, x0, y0, z0, b0);
                int tap = 0, g = 0;   // K-step k = tap * gpt + g
                for (int k = 0; k < p.ksteps; ++k, q.next(S), g = (g + 1 < gpt) ? g + 1 : 0, tap += (g == 0)) {
                    const int s = q.s;
                    const uint32_t r = q.r;
                    const uint32_t full = bar0 + 8u * s, empty = bar0 + 8u * (S + s);
                    if (r > 0 && !mbar_wait(empty, (r - 1) & 1u, kWaitLimitNs)) {
                        atomicOr(p.err, ERR_TIMEOUT);
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(full, tx);
                    const uint32_t a_dst = sbase + (uint32_t)s * p.stage_bytes;
                    if (conv && p.halo == 2) {
                        // full halo: one box of (bx + 2, by + 2, 3) voxels per block of E planes
                        // holds all 27 taps; the weights of the three x-shifts follow
                        const int kc = k * p.E;
                        const int mi = kc < p.kc0 ? 0 : 1, c8 = kc < p.kc0 ? kc : kc - p.kc0;
                        tma_load_5d(a_dst, &p.maps[mi], full, 8 * (x0 - 1), y0 - 1, z0 - 1, b0, c8);
                        const uint32_t bsz = 9u * p.E * p.n_tile * 16u;
                        for (int dxi = 0; dxi < 3; ++dxi) {
                            const __nv_bfloat16* src =
                                p.wpack + ((size_t)(blockIdx.y * 3 + dxi) * p.kc_total + kc) * 9 * p.n_tile * 8;
                            bulk_load(a_dst + p.a_stage_bytes + bsz * dxi, src, bsz, full);
                        }
                    } else if (conv) {
                        // tap = x-shift index, g = block of E chunk planes
                        const int dx = tap - 1, kc = g * p.E;
                        const int mi = kc < p.kc0 ? 0 : 1, c8 = kc < p.kc0 ? kc : kc - p.kc0;
                        if (p.halo) {
                            tma_load_5d(a_dst, &p.maps[mi], full, 8 * (x0 + dx), y0 - 1, z0 - 1, b0, c8);
                        } else {
                            for (int t9 = 0; t9 < 9; ++t9)
                                tma_load_5d(a_dst + (uint32_t)(t9 * p.E) * 2048u, &p.maps[mi], full, 8 * (x0 + dx),
                                            y0 + (t9 % 3) - 1, z0 + (t9 / 3) - 1, b0, c8);
                        }
                        const __nv_bfloat16* src =
                            p.wpack + ((size_t)(blockIdx.y * 3 + tap) * p.kc_total + kc) * 9 * p.n_tile * 8;
                        bulk_load(a_dst + p.a_stage_bytes, src, p.b_stage_bytes, full);
                    } else {
                        if (p.tap_mode == TAP_MAP) {
                            for (int j = 0; j < p.kc_step; ++j)
                                load_box(a_dst + 2048u * j, &p.maps[tap], full, true, g * p.kc_step + j, x0, y0, z0,
                                         b0, p.g.B);
                        } else {
                            // TAP_NONE: one box of kc_step chunk planes
                            tma_load_5d(a_dst, &p.maps[0], full, 8 * x0, y0, z0, b0, g * p.kc_step);
                        }
                        const __nv_bfloat16* src =
                            p.wpack + ((size_t)(blockIdx.y * p.n_taps + tap) * p.kc_total + (size_t)g * p.kc_step) *
                                          p.n_tile * 8;
                        bulk_load(a_dst + p.a_stage_bytes, src, p.b_stage_bytes, full);
                    }
                }
            }
        }
    } else if (warp == 1) {
        // The whole warp walks the K-steps, so the descriptor arithmetic stays
        // warp-uniform; one elected lane issues every MMA and commit.
        const bool leader = elect_one();
        const uint32_t nrow = (uint32_t)p.n_tile * 16u;   // bytes of one packed chunk of B
        // conv3 with halo 0 / 1: start offsets (16-byte units) of the nine (dz, dy)
        // taps and the A operand's K-direction core-matrix stride
        const uint32_t a_lbo = p.halo == 1 ? p.halo_plane : 2048u;
        uint32_t tap_off[9];
#pragma unroll
        for (int t9 = 0; t9 < 9; ++t9)
            tap_off[t9] = p.halo == 1 ? (uint32_t)(((t9 / 3) * (p.g.by + 2) + (t9 % 3)) * p.g.bx)
                                      : (uint32_t)(t9 * p.E) * 128u;
        Ring q;
        bool ok = true;
        for (uint32_t it = 0; ok; ++it) {
            const uint32_t ts = it & 3u, tu = it >> 2;
            if (!__all_sync(0xffffffffu, mbar_wait(tile_full + 8u * ts, tu & 1u, kWaitLimitNs))) {
                if (leader) atomicOr(p.err, ERR_TIMEOUT);
                break;
            }
            const int t = tile_slot[ts];
            __syncwarp();
            if (leader) mbar_arrive(tile_empty + 8u * ts);
            if (t < 0) break;
            // accumulator buffer of this tile and how often it was filled before
            const uint32_t buf = p.nbuf == 2 ? (it & 1u) : 0u, use = p.nbuf == 2 ? (it >> 1) : it;
            if (use > 0 && !__all_sync(0xffffffffu, mbar_wait(acc_empty + 8u * buf, (use - 1) & 1u, kWaitLimitNs))) {
                if (leader) atomicOr(p.err, ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const uint32_t acc = tmem + buf * acc_cols;
            for (int k = 0; k < p.ksteps; ++k, q.next(S)) {
                const int s = q.s;
                const uint32_t r = q.r;
                if (!__all_sync(0xffffffffu, mbar_wait(bar0 + 8u * s, r & 1u, kWaitLimitNs))) {
                    if (leader) atomicOr(p.err, ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = sbase + (uint32_t)s * p.stage_bytes;
                const uint32_t b0s = a0 + p.a_stage_bytes;
                if (conv && p.halo == 2) {
                    if (leader) {
                        // rows of a subtile are y-runs of bx = 8 voxels: one core-matrix group
                        // each, (bx + 2) * 16 bytes apart in the halo box; every tap is a
                        // start offset ((dz, dy) rows, dx * 16 bytes)
                        const uint32_t rowb = (uint32_t)(p.g.bx + 2) * 16u;
                        const uint32_t sub = (uint32_t)(kRows / p.g.bx) * rowb;
                        const uint32_t bsz = 9u * p.E * nrow;
                        for (int dxi = 0; dxi < 3; ++dxi)
                            for (int t9 = 0; t9 < 9; ++t9) {
                                const uint32_t a_tap =
                                    a0 + (uint32_t)((t9 / 3) * (p.g.by + 2) + (t9 % 3)) * rowb + 16u * dxi;
                                for (int i = 0; i < p.E / 2; ++i) {
                                    const uint64_t bd =
                                        smem_desc(b0s + bsz * dxi + (uint32_t)(2 * i * 9 + t9) * nrow, 9u * nrow, 128);
                                    for (int m = 0; m < p.mt; ++m) {
                                        const uint64_t ad =
                                            smem_desc(a_tap + sub * m + 2u * i * p.halo_plane, p.halo_plane, rowb);
                                        umma_bf16(acc + (uint32_t)(m * p.n_tile), ad, bd, p.idesc,
                                                  (k > 0 || dxi > 0 || t9 > 0 || i > 0) ? 1u : 0u);
                                    }
                                }
                            }
                    }
                } else if (conv) {
                    const uint64_t ad = smem_desc(a0, a_lbo, 128), bd = smem_desc(b0s, 9u * nrow, 128);
                    if (leader)
                        issue_conv_step(p.mt, p.E / 2, acc, ad, bd, tap_off, a_lbo / 8u, (uint32_t)p.n_tile, p.idesc,
                                        k == 0);
                } else if (leader) {
                    for (int i = 0; i < p.kc_step / 2; ++i) {
                        const uint64_t ad = smem_desc(a0 + 4096u * i, 2048u, 128);
                        const uint64_t bd = smem_desc(b0s + 2u * i * nrow, nrow, 128);
                        umma_bf16(acc, ad, bd, p.idesc, (k > 0 || i > 0) ? 1u : 0u);
                    }
                }
                if (leader) umma_commit(bar0 + 8u * (S + s));
                __syncwarp();
            }
            if (!ok) break;
            if (leader) umma_commit(acc_full + 8u * buf);
            __syncwarp();
        }
    } else {
        const int q = warp & 3;
        const int r = q * 32 + lane;
        for (uint32_t it = 0;; ++it) {
            const uint32_t ts = it & 3u, tu = it >> 2;
            if (!__all_sync(0xffffffffu, mbar_wait(tile_full + 8u * ts, tu & 1u, kWaitLimitNs))) {
                if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
                break;
            }
            const int t = tile_slot[ts];
            __syncwarp();
            if (lane == 0) mbar_arrive(tile_empty + 8u * ts);
            if (t < 0) break;
            const uint32_t buf = p.nbuf == 2 ? (it & 1u) : 0u, use = p.nbuf == 2 ? (it >> 1) : it;
            if (!__all_sync(0xffffffffu, mbar_wait(acc_full + 8u * buf, use & 1u, kWaitLimitNs))) {
                if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
                break;
            }
            {
                tc_fence_after();
                const uint32_t acc = tmem + buf * acc_cols;
                int x0, y0, z0, b0;
                tile_origin_u32(p.g, (uint32_t)t, x0, y0, z0, b0);
                const uint32_t lane_base = (uint32_t)(q * 32) << 16;
                const int nch = p.n_tile / 16;
                // up layers: column n = o n_up + channel, o = (oz, oy, ox) the fine offset
                const long long fW = 2LL * p.g.W, fHW = fW * (2LL * p.g.H);
                for (int m = 0; m < p.mt; ++m) {
                    int vx, vy, vz, vb;
                    const long long vox = row_voxel(p.g, x0, y0, z0, b0, m * kRows + r, &vx, &vy, &vz, &vb);
                    // fine voxel (2 vx, 2 vy, 2 vz) of sample vb (up layers)
                    const long long fine0 = ((long long)vb * (2 * p.g.D) + 2 * vz) * fHW + 2LL * vy * fW + 2 * vx;
                    float head_acc = 0.f;
                    // epilogue of accumulator chunk j (16 columns)
                    auto emit = [&](int j, const uint32_t (&v)[16]) {
                        const int n0 = blockIdx.y * p.n_tile + j * 16;
                        const EpiDest& d = (n0 < p.split) ? p.d[0] : p.d[1];
                        if (d.out == nullptr) return;
                        int ch0;
                        long long off;
                        if (p.scatter_up) {
                            const int o = n0 / p.cout_up;
                            ch0 = n0 - o * p.cout_up;
                            const long long fine = fine0 + (o >> 2) * fHW + ((o >> 1) & 1) * fW + (o & 1);
                            off = (ch0 >> 3) * d.plane + fine * 8;
                        } else {
                            ch0 = n0 - d.col0;
                            off = (ch0 >> 3) * d.plane + vox * 8;
                        }
                        float f[16];
                        #pragma unroll
                        for (int i = 0; i < 16; ++i) f[i] = __uint_as_float(v[i]);
                        if (d.bias) {
                            #pragma unroll
                            for (int i = 0; i < 16; ++i) f[i] += d.bias[ch0 + i];
                        }
                        if (d.addend) {
                            float a[16];
                            load16_planes(d.addend + off, d.plane, a);
                            #pragma unroll
                            for (int i = 0; i < 16; ++i) f[i] += a[i];
                        }
                        if (d.relu) {
                            #pragma unroll
                            for (int i = 0; i < 16; ++i) f[i] = fmaxf(f[i], 0.f);
                        }
                        if (d.mask) {
                            float mk[16];
                            load16_planes(d.mask + off, d.plane, mk);
                            #pragma unroll
                            for (int i = 0; i < 16; ++i) f[i] = (mk[i] > 0.f) ? f[i] : 0.f;
                        }
                        uint4 w[2];
                        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(w);
                        #pragma unroll
                        for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
                        *reinterpret_cast<uint4*>(d.out + off) = w[0];
                        *reinterpret_cast<uint4*>(d.out + off + d.plane) = w[1];
                        if (p.head_out) {
                            #pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const float2 rb = __bfloat1622float2(h[i]);
                                head_acc += rb.x * p.head_w[ch0 + 2 * i] + rb.y * p.head_w[ch0 + 2 * i + 1];
                            }
                        }
                    };
                    for (int j = 0; j < nch; ++j) {
                        uint32_t v[16];
                        tmem_ld16(acc + lane_base + (uint32_t)(m * p.n_tile + j * 16), v);
                        tmem_wait_ld();
                        emit(j, v);
                    }
                    if (p.head_out) p.head_out[vox] = head_acc + *p.head_b;
                }
            }
            // this warp's reads of the buffer are complete: hand it back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty + 8u * buf);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

// ------------------------------------------------------------------------
// Weight-gradient GEMM.  Per K-step (64 voxels of the V grid) the producer
// loads, for each of the tile's 16 row groups, a 64 x 16-byte box of the
// group's (tap, 8-channel chunk) input view, and the n/8 boxes of the output
// gradient: both operands are MN-major (8 channels contiguous per voxel).
// A row group may be the bias group: constant ones, so its rows accumulate
// sum_v dY[v, n], the bias gradient.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) wgrad_kernel(const __grid_constant__ WgradParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    const int S = p.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * p.stage_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = smem_u32(bars);
    const uint32_t done = bar0 + 16u * S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncols = tmem_cols(p.n);
    const int g0 = blockIdx.y * 16;
    const int groups_all = p.n_groups + (p.ones_group >= 0 ? 1 : 0);
    const int ng = min(16, groups_all - g0);
    const int btap = blockIdx.z;
    const int kbeg = blockIdx.x * p.ksteps_per_cta;
    const int kend = min(kbeg + p.ksteps_per_cta, p.ksteps_total);

    const uint32_t gbytes = (uint32_t)p.kv * 16u;   // one group's block of a stage
    // bias group: bf16 ones in its slot of every stage (written once, never loaded over)
    const int ones_slot = (p.ones_group >= g0 && p.ones_group < g0 + 16) ? p.ones_group - g0 : -1;
    if (ones_slot >= 0) {
        for (int s = 0; s < S; ++s) {
            uint32_t* dst = reinterpret_cast<uint32_t*>(smem + (size_t)s * p.stage_bytes + gbytes * ones_slot);
            for (int i = threadIdx.x; i < (int)(gbytes / 4); i += blockDim.x) dst[i] = 0x3F803F80u;
        }
        fence_async_shared();
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(bar0 + 8u * s, 1);
            mbar_init(bar0 + 8u * (S + s), 1);
        }
        mbar_init(done, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // the whole warp walks the K-steps; one elected lane issues (see rows_kernel)
        const bool leader = elect_one();
        int real = 0;
        for (int sl = 0; sl < ng; ++sl) real += (sl != ones_slot);
        const uint32_t tx = gbytes * real + (uint32_t)(p.n / 8) * gbytes;
        // every K-step loads the same slots: lane sl decodes slot sl once (source
        // map mi, chunk plane c8, tap shift), packed mi | c8 << 4 | (dx, dy, dz) + 1
        // in bits 14, 16, 18
        int code = 0;
        if (lane < ng && lane != ones_slot) {
            const int g = g0 + lane;
            int mi = 0, c8, dx = 0, dy = 0, dz = 0;
            if (p.mode == KIND_CONV3) {
                const int tap = g / p.kc_total;
                c8 = g % p.kc_total;
                dz = tap / 9 - 1;
                dy = (tap / 3) % 3 - 1;
                dx = tap % 3 - 1;
                if (c8 >= p.kc0) {
                    mi = 1;
                    c8 -= p.kc0;
                }
            } else if (p.mode == KIND_DOWN) {
                mi = g / p.kc_total;
                c8 = g % p.kc_total;
            } else {
                c8 = g;
            }
            code = mi | (c8 << 4) | ((dx + 1) << 14) | ((dy + 1) << 16) | ((dz + 1) << 18);
        }
        Ring q;
        int x0, y0, z0, b0;
        tile_origin(p.g, kbeg, x0, y0, z0, b0);
        for (int k = kbeg; k < kend; ++k, q.next(S), tile_next(p.g, x0, y0, z0, b0)) {
            const int kk = k - kbeg;
            const int s = q.s;
            const uint32_t r = q.r;
            const uint32_t full = bar0 + 8u * s, empty = bar0 + 8u * (S + s);
            if (kk >= S && !__all_sync(0xffffffffu, mbar_wait(empty, (r - 1) & 1u, kWaitLimitNs))) {
                if (leader) atomicOr(p.err, ERR_TIMEOUT);
                break;
            }
            if (leader) mbar_expect_tx(full, tx);
            const uint32_t a_dst = sbase + (uint32_t)s * p.stage_bytes;
            for (int sl = 0; sl < ng;) {
                if (sl == ones_slot) {
                    ++sl;
                    continue;
                }
                const int c = __shfl_sync(0xffffffffu, code, sl);
                const int mi = c & 15, c8 = (c >> 4) & 1023;
                const int dx = ((c >> 14) & 3) - 1, dy = ((c >> 16) & 3) - 1, dz = ((c >> 18) & 3) - 1;
                // one box brings ea consecutive chunk planes (runs never straddle a tap or source)
                if (leader)
                    load_box(a_dst + gbytes * sl, &p.amaps[mi], full, p.mode == KIND_DOWN, c8, x0 + dx, y0 + dy,
                             z0 + dz, b0, p.g.B);
                sl += p.ea;
            }
            const CUtensorMap* bm = &p.bmaps[p.mode == KIND_UP ? btap : 0];
            for (int j = 0; j < p.n / 8; j += p.eb)
                if (leader)
                    load_box(a_dst + p.a_stage_bytes + gbytes * j, bm, full, p.mode == KIND_UP, j, x0, y0, z0, b0,
                             p.g.B);
            __syncwarp();
        }
    } else if (warp == 1) {
        // the whole warp walks the K-steps; one elected lane issues (see rows_kernel)
        const bool leader = elect_one();
        Ring q;
        for (int k = kbeg; k < kend; ++k, q.next(S)) {
            const int kk = k - kbeg;
            const int s = q.s;
            const uint32_t r = q.r;
            if (!__all_sync(0xffffffffu, mbar_wait(bar0 + 8u * s, r & 1u, kWaitLimitNs))) {
                if (leader) atomicOr(p.err, ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const uint32_t a0 = sbase + (uint32_t)s * p.stage_bytes;
            const uint32_t b0s = a0 + p.a_stage_bytes;
            // K-slice i starts 256 bytes (16 units) further in both operands
            const uint64_t ad = smem_desc(a0, 128u, gbytes), bd = smem_desc(b0s, 128u, gbytes);
            if (leader) {
                for (int i = 0; i < p.kv / 16; ++i)
                    umma_bf16(tmem, ad + 16u * i, bd + 16u * i, p.idesc, (kk > 0 || i > 0) ? 1u : 0u);
                umma_commit(bar0 + 8u * (S + s));
            }
            __syncwarp();
        }
        if (leader) umma_commit(done);
        __syncwarp();
    } else {
        const int q = warp & 3;
        const int r = q * 32 + lane;
        const int sl = r >> 3, r8 = r & 7;
        const int g = g0 + sl;
        bool ok = mbar_wait(done, 0, kWaitLimitNs);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
        } else if (kend > kbeg) {
            tc_fence_after();
            float* dst = nullptr;
            if (sl < ng) {
                if (g == p.ones_group) {
                    dst = (r8 == 0) ? p.db : nullptr;
                } else {
                    int tap, c8;
                    if (p.mode == KIND_UP) {
                        tap = btap;
                        c8 = g;
                    } else {
                        tap = g / p.kc_total;
                        c8 = g % p.kc_total;
                    }
                    dst = p.dw + ((size_t)(tap * p.kc_total + c8) * 8 + r8) * p.n;
                }
            }
            for (int j = 0; j < p.n / 16; ++j) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(j * 16), v);
                tmem_wait_ld();
                if (dst) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) atomicAdd(dst + j * 16 + i, __uint_as_float(v[i]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

cudaError_t launch_rows(const RowsParams& p, int grid_n, size_t smem, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(rows_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // resident CTAs per SM: the occupancy query's answer, at most 512 / ncols
    // by TMEM (a CTA beyond that would wait in tcgen05.alloc for a whole
    // persistent CTA).  The grid is `persistent` times that many CTAs per SM:
    // tiles are claimed dynamically, so a surplus CTA finds none and exits.
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rows_kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    const int by_tmem = 512 / (int)tmem_cols(p.nbuf * p.mt * p.n_tile);
    const int per_sm = occ < by_tmem ? occ : by_tmem;
    long long grid_m = (long long)sms * (per_sm > 0 ? per_sm : 1) * (p.persistent > 0 ? p.persistent : 1);
    if (grid_m > p.tiles || !p.persistent) grid_m = p.tiles;
    rows_kernel<<<dim3((unsigned)grid_m, grid_n), kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_wgrad(const WgradParams& p, dim3 grid, size_t smem, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    wgrad_kernel<<<grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace spnn

namespace spnn {

// K-step walk of the halo weight gradient: x-runs of rl voxels fastest, then z
// within a slab of zs planes, then y, then the slab, then the sample, so that
// the (dz, dy) halo rows a K-step loads were loaded by a recent K-step (L2).
struct HaloWalk {
    int xr, zi, y, zsl, b;
    __device__ __forceinline__ void start(const WgradHaloParams& p, int k) {
        xr = k % p.nx;
        k /= p.nx;
        zi = k % p.zs;
        k /= p.zs;
        y = k % p.g.H;
        k /= p.g.H;
        zsl = k % p.nzs;
        b = k / p.nzs;
    }
    __device__ __forceinline__ void next(const WgradHaloParams& p) {
        if (++xr < p.nx) return;
        xr = 0;
        if (++zi < p.zs) return;
        zi = 0;
        if (++y < p.g.H) return;
        y = 0;
        if (++zsl < p.nzs) return;
        zsl = 0;
        ++b;
    }
    __device__ __forceinline__ int x0(const WgradHaloParams& p) const { return p.rl * xr; }
    __device__ __forceinline__ int z0(const WgradHaloParams& p) const { return zsl * p.zs + zi; }
};

__global__ void __launch_bounds__(kThreads, 1) wgrad_halo_kernel(const __grid_constant__ WgradHaloParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    const int S = p.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * p.stage_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = smem_u32(bars);
    const uint32_t done = bar0 + 16u * S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kbeg = blockIdx.x * p.ksteps_per_cta;
    const int kend = min(kbeg + p.ksteps_per_cta, p.ksteps_total);
    // this CTA's planes: npc planes of one source from plane `first` on (planes
    // past the source's end load as zeros), `real` of them inside the source
    const int split = blockIdx.y;
    const int src = split < p.splits0 ? 0 : 1;
    const int npc = src ? p.npc1 : p.npc0;
    const int first = (src ? split - p.splits0 : split) * npc;
    const int real = min(npc, (src ? p.kc1 : p.kc0) - first);
    const int plane_off = (src ? p.kc0 : 0) + first;       // in the concatenated input
    const int groups = 9 * npc;                            // row group `groups` is the ones row
    const int nM = (groups + 16) / 16;                     // 128-row tiles holding groups + 1
    const uint32_t n3 = 3u * (uint32_t)p.n;                 // MMA N: (dx, output channel)
    const uint32_t ncols = tmem_cols(nM * (int)n3);
    const uint32_t row = 16u * (uint32_t)p.rl;             // bytes of one run of one chunk plane

    // the ones row of every K-step region of every stage (written once; TMA never writes it)
    for (int s = 0; s < S * p.ksub; ++s) {
        uint32_t* dst = reinterpret_cast<uint32_t*>(smem + (size_t)(s / p.ksub) * p.stage_bytes +
                                                    (size_t)(s % p.ksub) * p.sub_bytes + (size_t)groups * row);
        for (int i = threadIdx.x; i < (int)(row / 4); i += blockDim.x) dst[i] = 0x3F803F80u;
    }
    fence_async_shared();
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(bar0 + 8u * s, 1);
            mbar_init(bar0 + 8u * (S + s), 1);
        }
        mbar_init(done, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // the whole warp walks the K-steps; one elected lane issues (see rows_kernel)
        const bool leader = elect_one();
        const uint32_t b_box = (uint32_t)(p.n / 8) * row;   // n/8 planes of one run
        const uint32_t tx = (uint32_t)groups * row + 3u * b_box;
        Ring q;
        HaloWalk w;
        w.start(p, kbeg);
        // a stage holds ns <= ksub consecutive K-steps
        for (int k = kbeg; k < kend; q.next(S)) {
            const int ns = min(p.ksub, kend - k);
            const int s = q.s;
            const uint32_t r = q.r;
            const uint32_t full = bar0 + 8u * s, empty = bar0 + 8u * (S + s);
            if (r > 0 && !__all_sync(0xffffffffu, mbar_wait(empty, (r - 1) & 1u, kWaitLimitNs))) {
                if (leader) atomicOr(p.err, ERR_TIMEOUT);
                break;
            }
            if (leader) mbar_expect_tx(full, (uint32_t)ns * tx);
            for (int j = 0; j < ns; ++j, w.next(p)) {
                const uint32_t a_dst = sbase + (uint32_t)s * p.stage_bytes + (uint32_t)j * p.sub_bytes;
                if (leader) {
                    const int x0 = w.x0(p), z0 = w.z0(p);
                    // input: (rl, 3, 3) voxels of npc planes, rows (plane, dz, dy)
                    tma_load_5d(a_dst, &p.amaps[src], full, 8 * x0, w.y - 1, z0 - 1, w.b, first);
                    // output gradient shifted by -dx: B block dxi holds dY at x - (dxi - 1)
                    for (int dxi = 0; dxi < 3; ++dxi)
                        tma_load_5d(a_dst + p.a_region + (uint32_t)dxi * b_box, &p.bmap, full, 8 * (x0 + 1 - dxi),
                                    w.y, z0, w.b, 0);
                }
            }
            k += ns;
            __syncwarp();
        }
    } else if (warp == 1) {
        // the whole warp walks the K-steps; one elected lane issues (see rows_kernel)
        const bool leader = elect_one();
        Ring q;
        for (int k = kbeg; k < kend; q.next(S)) {
            const int ns = min(p.ksub, kend - k);
            const int s = q.s;
            const uint32_t r = q.r;
            if (!__all_sync(0xffffffffu, mbar_wait(bar0 + 8u * s, r & 1u, kWaitLimitNs))) {
                if (leader) atomicOr(p.err, ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            for (int j = 0; j < ns; ++j) {
                const uint32_t a0 = sbase + (uint32_t)s * p.stage_bytes + (uint32_t)j * p.sub_bytes;
                // MN-major operands: 8-voxel core matrices 128 bytes apart along K,
                // 8-channel groups one run apart along M / N; K-block kb = voxels
                // 16 kb .. 16 kb + 15 of the run, a 256-byte start offset
                if (leader)
                    for (int kb = 0; kb < p.rl / 16; ++kb) {
                        const uint64_t bd = smem_desc(a0 + p.a_region + 256u * kb, 128u, row);
                        for (int m = 0; m < nM; ++m)
                            umma_bf16(tmem + (uint32_t)m * n3, smem_desc(a0 + (uint32_t)m * 16u * row + 256u * kb, 128u, row),
                                      bd, p.idesc, (k > kbeg || j > 0 || kb > 0) ? 1u : 0u);
                    }
            }
            if (leader) umma_commit(bar0 + 8u * (S + s));
            k += ns;
            __syncwarp();
        }
        if (leader) umma_commit(done);
        __syncwarp();
    } else {
        const int q = warp & 3;
        const int r = q * 32 + lane;
        bool ok = mbar_wait(done, 0, kWaitLimitNs);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
        } else if (kend > kbeg) {
            tc_fence_after();
            const int ci_all = 8 * (p.kc0 + p.kc1);
            for (int m = 0; m < nM; ++m) {
                const int g = 16 * m + (r >> 3), r8 = r & 7;
                const int pl = g / 9, t9 = g % 9;             // t9 = (dz + 1) * 3 + (dy + 1)
                const bool wrow = g < groups && pl < real;
                const bool orow = g == groups && r8 == 0 && split == p.ones_split;
                for (uint32_t c = 0; c < n3; c += 16) {
                    uint32_t v[16];
                    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)m * n3 + c, v);
                    tmem_wait_ld();
                    const int dxi = (int)c / p.n, co = (int)c % p.n;
                    float* dst = nullptr;
                    if (wrow)
                        dst = p.dw + ((size_t)(t9 * 3 + dxi) * ci_all + (plane_off + pl) * 8 + r8) * p.n + co;
                    else if (orow && dxi == 1)
                        dst = p.db + co;
                    if (dst) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) atomicAdd(dst + e, __uint_as_float(v[e]));
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

cudaError_t launch_wgrad_halo(const WgradHaloParams& p, dim3 grid, size_t smem, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(wgrad_halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    wgrad_halo_kernel<<<grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace spnn
