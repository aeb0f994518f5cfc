// omni_fft_smem_c.cu -- four-step passes of 4096 points.
#include "omni_fft_smem.cuh"

namespace omni {

cudaError_t launch_smem_c(const Pass& p, const PassArgs& a, cudaStream_t st) {
    switch (p.L) {
        case 4096: return launch_smem_len<64, 64>(p, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t smem_last_occupancy_c(const Pass& p, int src_kind, int* blocks_per_sm) {
    switch (p.L) {
        case 4096: return smem_last_occupancy_len<64, 64>(p, src_kind, blocks_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t upload_twiddles_smem_c() { return upload_twiddles(); }

}  // namespace omni
