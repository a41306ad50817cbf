// spmc_probe.cu -- measurement helper: the throughput ceiling of face-by-face
// stepping with one Q32.32 tally word per step on this GPU.  No counterpart
// in the paper; it gives the transport kernel's roofline a measured ceiling.
#include <cmath>

#include "spmc.h"
#include "spmc_internal.cuh"

using namespace spmc;

namespace {

__device__ __forceinline__ u64 probe_q32(float c) {    // same rounding as the transport
    const float magic = 12582912.0f;
    const float t1 = fmaf(c, 512.0f, magic);
    const int k1 = (int)(__float_as_uint(t1) - 0x4B400000u);
    const float r = fmaf(t1 - magic, -1.0f / 512.0f, c);
    const float t2 = fmaf(r, 4294967296.0f, magic);
    const int k2 = (int)(__float_as_uint(t2) - 0x4B400000u);
    return ((u64)(u32)k1 << 23) + (u64)(long long)k2;
}

// Straight rays through an all-pore n^3 volume (n a multiple of 4), periodic
// in all three axes, mask bricks fetched as in the transport kernel, and (when
// red) one RED.ADD.U64 per step into a brick-layout field.  Rays start at
// pseudo-random points with pseudo-random directions (a per-thread LCG).
// Every coordinate stays in [0, n), so brick < (n/4)^3 and the field word
// index brick * 64 + bit < n^3.
__global__ void __launch_bounds__(256) probe_kernel(u64 *field, const u64 *bricks, int n,
                                                    long long steps, int red, float *sink) {
    u32 s = 2654435761u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
    auto rnd = [&]() { s = s * 1664525u + 1013904223u; return (float)(s >> 8) * (1.0f / 16777216.0f); };
    const int nb = n >> 2;
    auto wrap = [&](int i) { return i < 0 ? n - 1 : (i >= n ? 0 : i); };
    int ix = min((int)(rnd() * n), n - 1), iy = min((int)(rnd() * n), n - 1), iz = min((int)(rnd() * n), n - 1);
    float ux = rnd() - 0.5f, uy = rnd() - 0.5f, uz = rnd() - 0.5f;
    const float inv = rsqrtf(ux * ux + uy * uy + uz * uz + 1e-12f);
    ux *= inv; uy *= inv; uz *= inv;
    const float dtx = 1.0f / fmaxf(fabsf(ux), 1e-6f), dty = 1.0f / fmaxf(fabsf(uy), 1e-6f),
                dtz = 1.0f / fmaxf(fabsf(uz), 1e-6f);
    float tmx = 0.5f * dtx, tmy = 0.5f * dty, tmz = 0.5f * dtz, t = 0.0f, acc = 0.0f;
    const int sx = ux > 0 ? 1 : -1, sy = uy > 0 ? 1 : -1, sz = uz > 0 ? 1 : -1;
    u32 brick = ((u32)(iz >> 2) * nb + (iy >> 2)) * nb + (ix >> 2);
    u32 bit = ((iz & 3) << 4) | ((iy & 3) << 2) | (ix & 3);
    u64 word = bricks[brick];
    for (long long k = 0; k < steps; ++k) {
        int ax = 2;
        float tn = tmz;
        if (tmy < tn) { tn = tmy; ax = 1; }
        if (tmx < tn) { tn = tmx; ax = 0; }
        const float seg = tn - t;
        const int nix = wrap(ix + (ax == 0 ? sx : 0)), niy = wrap(iy + (ax == 1 ? sy : 0)),
                  niz = wrap(iz + (ax == 2 ? sz : 0));
        const u32 nbk = ((u32)(niz >> 2) * nb + (niy >> 2)) * nb + (nix >> 2);
        const u64 nword = nbk != brick ? __ldg(bricks + nbk) : word;
        acc += ((word >> bit) & 1ull) ? seg : 0.0f;
        if (red) atomicAdd(field + (((u64)brick << 6) | bit), probe_q32(seg));
        t = tn;
        if (ax == 0) tmx += dtx;
        if (ax == 1) tmy += dty;
        if (ax == 2) tmz += dtz;
        if (t > 4.0f) { tmx -= t; tmy -= t; tmz -= t; t = 0.0f; }
        ix = nix; iy = niy; iz = niz; brick = nbk; word = nword;
        bit = ((iz & 3) << 4) | ((iy & 3) << 2) | (ix & 3);
    }
    if (acc == -1.0f) sink[0] = acc;        // keeps the loop's work observable
}

}  // namespace

extern "C" int sp_mc_probe_step_ceiling(int n, int red, long long steps_per_thread, double *ms,
                                        double *steps_per_s) {
    if (n < 16 || n > 1024 || (n & 3) || steps_per_thread < 1 || !ms || !steps_per_s)
        return SP_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    const size_t nvox = (size_t)n * n * n;
    u64 *field = nullptr, *bricks = nullptr;
    float *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = SP_ECUDA;
    if (cudaMalloc(&field, nvox * sizeof(u64)) == cudaSuccess &&
        cudaMalloc(&bricks, nvox / 8) == cudaSuccess && cudaMalloc(&sink, sizeof(float)) == cudaSuccess &&
        cudaMemset(field, 0, nvox * sizeof(u64)) == cudaSuccess &&
        cudaMemset(bricks, 0xff, nvox / 8) == cudaSuccess && cudaEventCreate(&a) == cudaSuccess &&
        cudaEventCreate(&b) == cudaSuccess) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_kernel, 256, 0);
        const int blocks = sms * (per_sm > 0 ? per_sm : 1);
        probe_kernel<<<blocks, 256>>>(field, bricks, n, 256, red, sink);          // warm-up
        cudaEventRecord(a);
        probe_kernel<<<blocks, 256>>>(field, bricks, n, steps_per_thread, red, sink);
        cudaEventRecord(b);
        float t = 0;
        if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&t, a, b) == cudaSuccess &&
            cudaGetLastError() == cudaSuccess) {
            *ms = t;
            *steps_per_s = (double)blocks * 256.0 * (double)steps_per_thread / (t * 1e-3);
            rc = SP_OK;
        }
    }
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(field);
    cudaFree(bricks);
    cudaFree(sink);
    return rc;
}
