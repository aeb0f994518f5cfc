// omni_fft_level_b.cu -- level passes of 32, 64 points per axis.
#include "omni_fft_level.cuh"

namespace omni {

cudaError_t launch_level_b(const Pass& p, const PassArgs& a, cudaStream_t st) {
    switch (p.L) {
        case 32: return launch_level_len<32>(p, a, st);
        case 64: return launch_level_len<64>(p, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t level_occupancy_b(int L, bool finest, int src_kind, int* out) {
    switch (L) {
        case 32: return level_last_blocks_per_sm<32>(finest, src_kind, out);
        case 64: return level_last_blocks_per_sm<64>(finest, src_kind, out);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t level_stream_occupancy_b(int L, int src_kind, int* out) {
    switch (L) {
        case 32: return level_stream_blocks_per_sm<32>(src_kind, out);
        case 64: return level_stream_blocks_per_sm<64>(src_kind, out);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t upload_twiddles_level_b() { return upload_twiddles(); }

}  // namespace omni
