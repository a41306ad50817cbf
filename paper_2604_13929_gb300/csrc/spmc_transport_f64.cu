// spmc_transport_f64.cu -- double instantiation of the transport kernel.
#include "spmc_transport.cuh"

namespace spmc {

cudaError_t launch_transport_f64(const TransportParams &p, bool field, int blocks, int threads,
                                 size_t smem, cudaStream_t s) {
    return launch_transport<double>(p, field, blocks, threads, smem, s);
}

cudaError_t occupancy_f64(bool field, bool mirror, int threads, size_t smem, int *blocks_per_sm) {
    return occupancy<double>(field, mirror, threads, smem, blocks_per_sm);
}

const void *kernel_f64(bool field, bool mirror) { return kernel_ptr<double>(field, mirror); }

}  // namespace spmc
