// omni_fft_reg_a.cu -- register passes of 4, 8 and 16 points.
#include "omni_fft_reg.cuh"

namespace omni {

cudaError_t launch_reg_a(const Pass& p, const PassArgs& a, cudaStream_t st) {
    switch (p.L) {
        case 4: return launch_reg_len<4>(p, a, st);
        case 8: return launch_reg_len<8>(p, a, st);
        case 16: return launch_reg_len<16>(p, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t upload_twiddles_reg_a() { return upload_twiddles(); }

}  // namespace omni
