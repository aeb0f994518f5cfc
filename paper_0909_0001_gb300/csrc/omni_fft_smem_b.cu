// omni_fft_smem_b.cu -- four-step passes of 1024 and 2048 points.
#include "omni_fft_smem.cuh"

namespace omni {

cudaError_t launch_smem_b(const Pass& p, const PassArgs& a, cudaStream_t st) {
    switch (p.L) {
        case 1024: return launch_smem_len<32, 32>(p, a, st);
        case 2048: return launch_smem_len<64, 32>(p, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t smem_last_occupancy_b(const Pass& p, int src_kind, int* blocks_per_sm) {
    switch (p.L) {
        case 1024: return smem_last_occupancy_len<32, 32>(p, src_kind, blocks_per_sm);
        case 2048: return smem_last_occupancy_len<64, 32>(p, src_kind, blocks_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t upload_twiddles_smem_b() { return upload_twiddles(); }

}  // namespace omni
