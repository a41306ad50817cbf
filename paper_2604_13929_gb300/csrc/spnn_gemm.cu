// spnn_gemm.cu -- the two tensor-core GEMM kernels of the surrogate.
//
// Both are warp-specialised, one CTA per output tile, 192 threads:
//   warp 0      TMA producer: fills a ring of shared-memory stages,
//   warp 1      allocates TMEM and issues tcgen05.mma from one thread,
//   warps 2..5  epilogue: tcgen05.ld of the FP32 accumulators, fused
//               bias / residual / ReLU / ReLU-derivative mask, BF16 stores.
// Stages hand over with mbarriers: "full" completes when TMA bytes land,
// "empty" when the MMAs that read the stage retire (tcgen05.commit).  Every
// wait is bounded by kWaitLimitNs; a timeout sets an error flag, and the CTA
// still releases its TMEM and exits.
#include "spnn_internal.cuh"
#include "spnn_umma.cuh"

namespace spnn {

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ void load16_bf16(const __nv_bfloat16* p, float (&f)[16]) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    uint4 u[2] = {q[0], q[1]};
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(u);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}

// ------------------------------------------------------------------------
// Rows GEMM (forward, input-gradient and transposed-conv layers).
// A tile: kc_step chunk planes of 128 rows x 16 bytes (2 KB each), K-major;
// B tile: kc_step planes of n_tile rows x 16 bytes, K-major.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) rows_kernel(const __grid_constant__ RowsParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    const int S = p.stages;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * p.stage_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = smem_u32(bars);
    const uint32_t done = bar0 + 16u * S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncols = tmem_cols(p.n_tile);

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

    const long long row0 = (long long)blockIdx.x * kRows;
    const int x0 = (int)(row0 % p.R_W);
    long long t = row0 / p.R_W;
    const int y0 = (int)(t % p.R_H);
    t /= p.R_H;
    const int z0 = (int)(t % p.R_D);
    const int b0 = (int)(t / p.R_D);

    if (warp == 0) {
        if (lane == 0) {
            const int gpt = p.kc_total / p.kc_step;
            const uint32_t tx = p.a_stage_bytes + p.b_stage_bytes;
            for (int k = 0; k < p.ksteps; ++k) {
                const int s = k % S;
                const uint32_t r = (uint32_t)(k / S);
                const uint32_t full = bar0 + 8u * s, empty = bar0 + 8u * (S + s);
                if (k >= S && !mbar_wait(empty, (r - 1) & 1u, kWaitLimitNs)) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    break;
                }
                mbar_expect_tx(full, tx);
                const int tap = k / gpt, g = k % gpt;
                int dx = 0, dy = 0, dz = 0;
                if (p.tap_mode == TAP_SHIFT3) {
                    dz = tap / 9 - 1;
                    dy = (tap / 3) % 3 - 1;
                    dx = tap % 3 - 1;
                }
                const uint32_t a_dst = sbase + (uint32_t)s * p.stage_bytes;
                for (int j = 0; j < p.kc_step; ++j) {
                    const int kc = g * p.kc_step + j;
                    int mi, c;
                    if (p.tap_mode == TAP_MAP) {
                        mi = tap;
                        c = kc * 8;
                    } else if (kc < p.kc0) {
                        mi = 0;
                        c = kc * 8;
                    } else {
                        mi = 1;
                        c = (kc - p.kc0) * 8;
                    }
                    tma_load_5d(a_dst + 2048u * j, &p.maps[mi], full, c, x0 + dx, y0 + dy, z0 + dz, b0);
                }
                const __nv_bfloat16* src =
                    p.wpack + ((size_t)(blockIdx.y * p.n_taps + tap) * p.kc_total + (size_t)g * p.kc_step) *
                                  p.n_tile * 8;
                bulk_load(a_dst + p.a_stage_bytes, src, p.b_stage_bytes, full);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int k = 0; k < p.ksteps; ++k) {
                const int s = k % S;
                const uint32_t r = (uint32_t)(k / S);
                if (!mbar_wait(bar0 + 8u * s, r & 1u, kWaitLimitNs)) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = sbase + (uint32_t)s * p.stage_bytes;
                const uint32_t b0s = a0 + p.a_stage_bytes;
                for (int i = 0; i < p.kc_step / 2; ++i) {
                    const uint64_t ad = smem_desc(a0 + 4096u * i, p.lbo_a, p.sbo_a);
                    const uint64_t bd = smem_desc(b0s + (uint32_t)(2 * i * p.n_tile * 16), p.lbo_b, p.sbo_b);
                    umma_bf16(tmem, ad, bd, p.idesc, (k > 0 || i > 0) ? 1u : 0u);
                }
                umma_commit(bar0 + 8u * (S + s));
            }
            umma_commit(done);
        }
    } else {
        const int q = warp & 3;
        const int r = q * 32 + lane;
        const long long grow = row0 + r;
        bool ok = mbar_wait(done, 0, kWaitLimitNs);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
        } else {
            tc_fence_after();
            // coarse-grid coordinates of this row (for the 2x upsampling scatter)
            const int vx = (int)(grow % p.R_W);
            long long tt = grow / p.R_W;
            const int vy = (int)(tt % p.R_H);
            tt /= p.R_H;
            const int vz = (int)(tt % p.R_D);
            const long long vb = tt / p.R_D;
            float head_acc = 0.f;
            for (int j = 0; j < p.n_tile / 16; ++j) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(j * 16), v);
                tmem_wait_ld();
                const int n0 = blockIdx.y * p.n_tile + j * 16;
                const EpiDest& d = (n0 < p.split) ? p.d[0] : p.d[1];
                if (d.out == nullptr) continue;
                int ch0;
                long long off;
                if (p.scatter_up) {
                    const int o = n0 / p.cout_up;
                    ch0 = n0 % p.cout_up;
                    const int oz = o >> 2, oy = (o >> 1) & 1, ox = o & 1;
                    const long long fine =
                        ((vb * (2LL * p.R_D) + 2 * vz + oz) * (2LL * p.R_H) + 2 * vy + oy) * (2LL * p.R_W) +
                        2 * vx + ox;
                    off = fine * d.ld + ch0;
                } else {
                    ch0 = n0 - d.col0;
                    off = grow * d.ld + ch0;
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
                    load16_bf16(d.addend + off, a);
#pragma unroll
                    for (int i = 0; i < 16; ++i) f[i] += a[i];
                }
                if (d.relu) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) f[i] = fmaxf(f[i], 0.f);
                }
                if (d.mask) {
                    float m[16];
                    load16_bf16(d.mask + off, m);
#pragma unroll
                    for (int i = 0; i < 16; ++i) f[i] = (m[i] > 0.f) ? f[i] : 0.f;
                }
                uint4 w[2];
                __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(w);
#pragma unroll
                for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
                uint4* dst = reinterpret_cast<uint4*>(d.out + off);
                dst[0] = w[0];
                dst[1] = w[1];
                if (p.head_out) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float2 rb = __bfloat1622float2(h[i]);
                        head_acc += rb.x * p.head_w[ch0 + 2 * i] + rb.y * p.head_w[ch0 + 2 * i + 1];
                    }
                }
            }
            if (p.head_out) p.head_out[grow] = head_acc + *p.head_b;
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

    // bias group: bf16 ones in its slot of every stage (written once, never loaded over)
    const int ones_slot = (p.ones_group >= g0 && p.ones_group < g0 + 16) ? p.ones_group - g0 : -1;
    if (ones_slot >= 0) {
        for (int s = 0; s < S; ++s) {
            uint32_t* dst = reinterpret_cast<uint32_t*>(smem + (size_t)s * p.stage_bytes + 1024 * ones_slot);
            for (int i = threadIdx.x; i < 256; i += blockDim.x) dst[i] = 0x3F803F80u;
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
        if (lane == 0) {
            int real = 0;
            for (int sl = 0; sl < ng; ++sl) real += (sl != ones_slot);
            const uint32_t tx = 1024u * real + 128u * p.n;
            for (int k = kbeg; k < kend; ++k) {
                const int kk = k - kbeg;
                const int s = kk % S;
                const uint32_t r = (uint32_t)(kk / S);
                const uint32_t full = bar0 + 8u * s, empty = bar0 + 8u * (S + s);
                if (kk >= S && !mbar_wait(empty, (r - 1) & 1u, kWaitLimitNs)) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    break;
                }
                mbar_expect_tx(full, tx);
                const long long v0 = (long long)k * kWgradK;
                const int x0 = (int)(v0 % p.V_W);
                long long t = v0 / p.V_W;
                const int y0 = (int)(t % p.V_H);
                t /= p.V_H;
                const int z0 = (int)(t % p.V_D);
                const int b0 = (int)(t / p.V_D);
                const uint32_t a_dst = sbase + (uint32_t)s * p.stage_bytes;
                for (int sl = 0; sl < ng; ++sl) {
                    if (sl == ones_slot) continue;
                    const int g = g0 + sl;
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
                    tma_load_5d(a_dst + 1024u * sl, &p.amaps[mi], full, c8 * 8, x0 + dx, y0 + dy, z0 + dz, b0);
                }
                const CUtensorMap* bm = &p.bmaps[p.mode == KIND_UP ? btap : 0];
                for (int j = 0; j < p.n / 8; ++j)
                    tma_load_5d(a_dst + p.a_stage_bytes + 1024u * j, bm, full, j * 8, x0, y0, z0, b0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int k = kbeg; k < kend; ++k) {
                const int kk = k - kbeg;
                const int s = kk % S;
                const uint32_t r = (uint32_t)(kk / S);
                if (!mbar_wait(bar0 + 8u * s, r & 1u, kWaitLimitNs)) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = sbase + (uint32_t)s * p.stage_bytes;
                const uint32_t b0s = a0 + p.a_stage_bytes;
#pragma unroll
                for (int i = 0; i < kWgradK / 16; ++i) {
                    const uint64_t ad = smem_desc(a0 + 256u * i, p.lbo, p.sbo);
                    const uint64_t bd = smem_desc(b0s + 256u * i, p.lbo, p.sbo);
                    umma_bf16(tmem, ad, bd, p.idesc, (kk > 0 || i > 0) ? 1u : 0u);
                }
                umma_commit(bar0 + 8u * (S + s));
            }
            umma_commit(done);
        }
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

cudaError_t launch_rows(const RowsParams& p, int grid_m, int grid_n, size_t smem, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    rows_kernel<<<dim3(grid_m, grid_n), kThreads, smem, s>>>(p);
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
