// omni_dispatch.cpp -- routes a pass to its kernel family and sets up the
// per-device twiddle tables of every kernel translation unit.
#include "omni_internal.h"

#include <mutex>
#include <vector>

namespace omni {

cudaError_t launch_reg_a(const Pass& p, const PassArgs& a, cudaStream_t st);
cudaError_t launch_reg_b(const Pass& p, const PassArgs& a, cudaStream_t st);
cudaError_t launch_smem_a(const Pass& p, const PassArgs& a, cudaStream_t st);
cudaError_t launch_smem_b(const Pass& p, const PassArgs& a, cudaStream_t st);
cudaError_t launch_smem_c(const Pass& p, const PassArgs& a, cudaStream_t st);
cudaError_t launch_direct(const Pass& p, const PassArgs& a, cudaStream_t st);
cudaError_t launch_level_a(const Pass& p, const PassArgs& a, cudaStream_t st);
cudaError_t launch_level_b(const Pass& p, const PassArgs& a, cudaStream_t st);
cudaError_t level_occupancy_a(int L, bool finest, int src_kind, int* out);
cudaError_t smem_last_occupancy_a(const Pass& p, int src_kind, int* blocks_per_sm);
cudaError_t smem_last_occupancy_b(const Pass& p, int src_kind, int* blocks_per_sm);
cudaError_t smem_last_occupancy_c(const Pass& p, int src_kind, int* blocks_per_sm);
cudaError_t level_occupancy_b(int L, bool finest, int src_kind, int* out);
cudaError_t level_stream_occupancy_a(int L, int src_kind, int* out);
cudaError_t level_stream_occupancy_b(int L, int src_kind, int* out);
cudaError_t upload_twiddles_reg_a();
cudaError_t upload_twiddles_reg_b();
cudaError_t upload_twiddles_smem_a();
cudaError_t upload_twiddles_smem_b();
cudaError_t upload_twiddles_smem_c();
cudaError_t upload_twiddles_smem3();
cudaError_t upload_twiddles_level_a();
cudaError_t upload_twiddles_level_b();

cudaError_t launch_pass(const Pass& p, const PassArgs& a, cudaStream_t st) {
    switch (p.kind) {
        case KIND_REG: return p.L <= 16 ? launch_reg_a(p, a, st) : launch_reg_b(p, a, st);
        case KIND_SMEM:
            return p.L <= 512 ? launch_smem_a(p, a, st)
                 : p.L <= 2048 ? launch_smem_b(p, a, st) : launch_smem_c(p, a, st);
        case KIND_LEVEL: return p.L <= 16 ? launch_level_a(p, a, st) : launch_level_b(p, a, st);
        case KIND_SMEM3: return launch_smem3(p, a, st);
        case KIND_TC_A:
        case KIND_TC_B: return launch_tc(p, a, st);
        case KIND_TC5_B: return launch_tc5(p, a, st);
        case KIND_XSPEC: return launch_xspec(p, a, st);
        case KIND_XSPEC5:
        case KIND_COV5: return launch_xspec5(p, a, st);
        default: return launch_direct(p, a, st);
    }
}

cudaError_t smem_last_occupancy(const Pass& p, int src_kind, int* blocks_per_sm) {
    return p.L <= 512 ? smem_last_occupancy_a(p, src_kind, blocks_per_sm)
         : p.L <= 2048 ? smem_last_occupancy_b(p, src_kind, blocks_per_sm)
                       : smem_last_occupancy_c(p, src_kind, blocks_per_sm);
}

cudaError_t level_last_occupancy(const Pass& p, int src_kind, int* blocks_per_sm) {
    return p.L <= 16 ? level_occupancy_a(p.L, p.inner == 1, src_kind, blocks_per_sm)
                     : level_occupancy_b(p.L, p.inner == 1, src_kind, blocks_per_sm);
}

cudaError_t level_stream_occupancy(const Pass& p, int src_kind, int* blocks_per_sm) {
    return p.L <= 16 ? level_stream_occupancy_a(p.L, src_kind, blocks_per_sm)
                     : level_stream_occupancy_b(p.L, src_kind, blocks_per_sm);
}

cudaError_t init_device_tables() {
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (int d : done)
        if (d == dev) return cudaSuccess;
    for (auto up : {upload_twiddles_reg_a, upload_twiddles_reg_b, upload_twiddles_smem_a,
                    upload_twiddles_smem_b, upload_twiddles_smem_c, upload_twiddles_smem3,
                    upload_twiddles_level_a, upload_twiddles_level_b})
        if ((e = up()) != cudaSuccess) return e;
    if ((e = upload_tc_tables()) != cudaSuccess) return e;
    if ((e = upload_tc5_tables()) != cudaSuccess) return e;
    done.push_back(dev);
    return cudaSuccess;
}

}  // namespace omni
