// omni_fft_level_a.cu -- level passes of 4, 8, 16 points per axis.
#include "omni_fft_level.cuh"

namespace omni {

cudaError_t launch_level_a(const Pass& p, const PassArgs& a, cudaStream_t st) {
    switch (p.L) {
        case 4: return launch_level_len<4>(p, a, st);
        case 8: return launch_level_len<8>(p, a, st);
        case 16: return launch_level_len<16>(p, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t level_occupancy_a(int L, bool finest, int src_kind, int* out) {
    switch (L) {
        case 4: return level_last_blocks_per_sm<4>(finest, src_kind, out);
        case 8: return level_last_blocks_per_sm<8>(finest, src_kind, out);
        case 16: return level_last_blocks_per_sm<16>(finest, src_kind, out);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t level_stream_occupancy_a(int L, int src_kind, int* out) {
    switch (L) {
        case 4: return level_stream_blocks_per_sm<4>(src_kind, out);
        case 8: return level_stream_blocks_per_sm<8>(src_kind, out);
        case 16: return level_stream_blocks_per_sm<16>(src_kind, out);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t upload_twiddles_level_a() { return upload_twiddles(); }

}  // namespace omni
