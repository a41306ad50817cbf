// spmc_transport_f32.cu -- float instantiation of the transport kernel.
#include "spmc_transport.cuh"

namespace spmc {

cudaError_t launch_transport_f32(const TransportParams &p, bool field, int blocks, int threads,
                                 size_t smem, cudaStream_t s) {
    return launch_transport<float>(p, field, blocks, threads, smem, s);
}

cudaError_t occupancy_f32(bool field, bool mirror, int threads, size_t smem, int *blocks_per_sm) {
    return occupancy<float>(field, mirror, threads, smem, blocks_per_sm);
}

const void *kernel_f32(bool field, bool mirror) { return kernel_ptr<float>(field, mirror); }

cudaError_t launch_transport_batch(const BatchParams &b, int blocks, int threads, cudaStream_t s) {
    TransportParams p{};
    p.compact_k = b.compact_k;
    transport_kernel<float, true, true, true><<<blocks, threads, 0, s>>>(p, b);
    return cudaGetLastError();
}

cudaError_t occupancy_batch(int threads, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                         transport_kernel<float, true, true, true>,
                                                         threads, 0);
}

}  // namespace spmc
