// omni_fft_reg_b.cu -- register passes of 32 and 64 points.
#include "omni_fft_reg.cuh"

namespace omni {

cudaError_t launch_reg_b(const Pass& p, const PassArgs& a, cudaStream_t st) {
    switch (p.L) {
        case 32: return launch_reg_len<32>(p, a, st);
        case 64: return launch_reg_len<64>(p, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t upload_twiddles_reg_b() { return upload_twiddles(); }

}  // namespace omni
