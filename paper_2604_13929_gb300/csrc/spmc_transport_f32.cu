// spmc_transport_f32.cu -- FP32 transport kernels: the streamlined
// production kernel (spmc_transport_f32.cuh) and the float instantiations of
// the generic template (kept as variant 0 and for batched launches).
#include "spmc_transport_f32.cuh"

namespace spmc {

namespace {

template <bool kField, bool kMirror>
const void *fast_ptr() {
    return reinterpret_cast<const void *>(&transport_f32_kernel<kField, kMirror, false>);
}

const void *fast_kernel(bool field, bool mirror) {
    if (mirror) return field ? fast_ptr<true, true>() : fast_ptr<false, true>();
    return field ? fast_ptr<true, false>() : fast_ptr<false, false>();
}

// per-warp tallies of the streamlined batched kernel (dynamic shared memory)
size_t batch_smem(int threads) { return (size_t)(threads / 32) * sizeof(SmemTallies); }

const void *batch_kernel(int variant, bool mirror) {
    if (variant == 0) return reinterpret_cast<const void *>(&transport_kernel<float, true, true, true>);
    return mirror ? reinterpret_cast<const void *>(&transport_f32_kernel<true, true, true>)
                  : reinterpret_cast<const void *>(&transport_f32_kernel<true, false, true>);
}

}  // namespace

const void *kernel_f32(bool field, bool mirror, int variant) {
    return variant == 0 ? kernel_ptr<float>(field, mirror) : fast_kernel(field, mirror);
}

cudaError_t launch_transport_f32(const TransportParams &p, bool field, int blocks, int threads,
                                 size_t smem, cudaStream_t s, const LaunchExtras &e) {
    if (e.variant == 0) return launch_transport<float>(p, field, blocks, threads, smem, s);
    const BatchParams none{};
    if (p.mirror) {
        if (field) transport_f32_kernel<true, true, false><<<blocks, threads, smem, s>>>(p, none);
        else transport_f32_kernel<false, true, false><<<blocks, threads, smem, s>>>(p, none);
    } else {
        if (field) transport_f32_kernel<true, false, false><<<blocks, threads, smem, s>>>(p, none);
        else transport_f32_kernel<false, false, false><<<blocks, threads, smem, s>>>(p, none);
    }
    return cudaGetLastError();
}

cudaError_t occupancy_f32(bool field, bool mirror, int variant, int threads, size_t smem,
                          int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel_f32(field, mirror, variant),
                                                         threads, smem);
}

// Batched launches: variant 0 the generic kernel (lanes of a warp carry
// photons of different problems), 1 the streamlined kernel (chunks of one
// problem per warp).  mirror: some problem has mirror lateral faces.
cudaError_t launch_transport_batch(const BatchParams &b, int variant, bool mirror, int blocks,
                                   int threads, cudaStream_t s) {
    TransportParams p{};
    p.compact_k = b.compact_k;
    const size_t smem = variant == 0 ? 0 : batch_smem(threads);
    if (variant == 0) transport_kernel<float, true, true, true><<<blocks, threads, 0, s>>>(p, b);
    else if (mirror) transport_f32_kernel<true, true, true><<<blocks, threads, smem, s>>>(p, b);
    else transport_f32_kernel<true, false, true><<<blocks, threads, smem, s>>>(p, b);
    return cudaGetLastError();
}

cudaError_t occupancy_batch(int variant, bool mirror, int threads, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel(variant, mirror),
                                                         threads, variant == 0 ? 0 : batch_smem(threads));
}

}  // namespace spmc
