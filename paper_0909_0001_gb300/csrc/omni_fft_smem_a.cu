// omni_fft_smem_a.cu -- four-step passes of 128, 256 and 512 points.
#include "omni_fft_smem.cuh"

namespace omni {

cudaError_t launch_smem_a(const Pass& p, const PassArgs& a, cudaStream_t st) {
    switch (p.L) {
        case 128: return launch_smem_len<16, 8>(p, a, st);
        case 256: return launch_smem_len<16, 16>(p, a, st);
        case 512: return launch_smem_len<32, 16>(p, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t smem_last_occupancy_a(const Pass& p, int src_kind, int* blocks_per_sm) {
    switch (p.L) {
        case 128: return smem_last_occupancy_len<16, 8>(p, src_kind, blocks_per_sm);
        case 256: return smem_last_occupancy_len<16, 16>(p, src_kind, blocks_per_sm);
        case 512: return smem_last_occupancy_len<32, 16>(p, src_kind, blocks_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t upload_twiddles_smem_a() { return upload_twiddles(); }

}  // namespace omni
