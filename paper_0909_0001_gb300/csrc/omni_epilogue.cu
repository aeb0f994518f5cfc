// omni_epilogue.cu -- physical-baseline epilogue: sums of visibilities by
// group (coincident physical baselines, or radial bins of |dr|; Sec. II.D,
// Sec. III's radially binned baseline distribution).
//
// One pass over [C][Q] complex128 visibilities.  With few groups (radial bins)
// each CTA accumulates a private copy of its channel's group sums in shared
// memory and adds it to global memory once; with many groups (merging
// coincident baselines: nearly one group per lag) the sums go straight to
// global memory.
#include "omni.h"
#include "omni_fft_common.cuh"

#include <algorithm>

namespace omni {
namespace {

constexpr int kSumThreads = 256;
constexpr int64_t kSharedGroups = 4096;  // 64 KB of double2 per CTA

__global__ void __launch_bounds__(kSumThreads) sum_groups_shared(const double2* vis, int64_t Q,
                                                                 const int32_t* group, int64_t n_groups,
                                                                 double2* out, int64_t per_cta) {
    extern __shared__ double2 acc[];
    const int64_t c = blockIdx.y;
    for (int64_t g = threadIdx.x; g < n_groups; g += blockDim.x) acc[g] = make_double2(0.0, 0.0);
    __syncthreads();
    const int64_t q0 = (int64_t)blockIdx.x * per_cta;
    const int64_t q1 = q0 + per_cta < Q ? q0 + per_cta : Q;
    const double2* v = vis + c * Q;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        const int32_t g = group[q];
        if (g >= 0 && g < n_groups) {
            const double2 x = v[q];
            atomicAdd(&acc[g].x, x.x);
            atomicAdd(&acc[g].y, x.y);
        }
    }
    __syncthreads();
    for (int64_t g = threadIdx.x; g < n_groups; g += blockDim.x) {
        const double2 x = acc[g];
        if (x.x != 0.0 || x.y != 0.0) {
            atomicAdd(&out[c * n_groups + g].x, x.x);
            atomicAdd(&out[c * n_groups + g].y, x.y);
        }
    }
}

__global__ void __launch_bounds__(kSumThreads) sum_groups_global(const double2* vis, int64_t C, int64_t Q,
                                                                 const int32_t* group, int64_t n_groups,
                                                                 double2* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C * Q) return;
    const int64_t c = i / Q, q = i - c * Q;
    const int32_t g = group[q];
    if (g < 0 || g >= n_groups) return;
    const double2 x = vis[i];
    atomicAdd(&out[c * n_groups + g].x, x.x);
    atomicAdd(&out[c * n_groups + g].y, x.y);
}

}  // namespace
}  // namespace omni

extern "C" omni_status omni_sum_groups(const double* vis_dev, int64_t C, int64_t Q,
                                       const int32_t* group_dev, int64_t n_groups, double* out_dev,
                                       void* stream) {
    using namespace omni;
    if (!vis_dev || !group_dev || !out_dev || C < 0 || Q < 0 || n_groups < 0) {
        set_last_error("omni_sum_groups: NULL pointer or negative size");
        return OMNI_ERR_INVALID_ARG;
    }
    if ((uintptr_t)vis_dev % 16 || (uintptr_t)out_dev % 16) {
        set_last_error("omni_sum_groups: vis_dev and out_dev must be 16-byte aligned");
        return OMNI_ERR_INVALID_ARG;
    }
    if (C == 0 || n_groups == 0) return OMNI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(out_dev, 0, (size_t)C * n_groups * sizeof(double2), s);
    if (e == cudaSuccess && Q > 0) {
        const double2* v = reinterpret_cast<const double2*>(vis_dev);
        double2* o = reinterpret_cast<double2*>(out_dev);
        if (n_groups <= kSharedGroups) {
            // enough CTAs per channel to fill the GPU, each a contiguous range of lags
            const int64_t per_cta = std::max<int64_t>(8 * kSumThreads, (Q + 63) / 64);
            const int64_t ctas = (Q + per_cta - 1) / per_cta;
            const size_t smem = (size_t)n_groups * sizeof(double2);
            e = smem_limit_once((const void*)sum_groups_shared, smem);
            if (e == cudaSuccess && C <= 65535) {
                sum_groups_shared<<<dim3((unsigned)ctas, (unsigned)C), kSumThreads, smem, s>>>(
                    v, Q, group_dev, n_groups, o, per_cta);
                e = cudaGetLastError();
            } else if (e == cudaSuccess) {
                e = cudaErrorInvalidValue;
            }
        } else {
            const int64_t blocks = (C * Q + kSumThreads - 1) / kSumThreads;
            sum_groups_global<<<(unsigned)blocks, kSumThreads, 0, s>>>(v, C, Q, group_dev, n_groups, o);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return OMNI_ERR_CUDA;
    }
    return OMNI_OK;
}
