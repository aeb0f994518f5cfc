// omni_tiles.cu -- tile hybrid (Sec. III): FFT correlation within identical
// tiles placed at arbitrary offsets, brute-force correlation between them.
//
// After the forward passes each sample holds every tile's zero-padded 2-D
// spectrum Y_j(k), k = k1 + L1 k2 (the tile's "synthesized beams").  This pass
// accumulates, for every ordered tile pair (i, j) and frequency k,
//   S_ij(k) += sum over the chunk's samples of Y_i(k) conj(Y_j(k)),
// in FP32 registers over the chunk, then in an FP64 complex accumulator
// [C][n_tiles][n_tiles][K].  The inverse 2-D FFT of S_ij gives the visibility
// of every antenna pair (a in tile i, b in tile j) with intra-tile offset
// m_a - m_b = D: the convolution theorem of Sec. II.C applied to two
// different tiles, exact because of the padding.
#include "omni_fft_common.cuh"

namespace omni {
namespace {

constexpr int kXK = 32;  // frequencies per CTA (one per lane)
constexpr int kXR = 8;   // thread rows per CTA (warps)
constexpr int kXI = 16;  // tiles i per CTA: two per thread (rows r and r + 8)
constexpr int kXJ = 16;  // tiles j per CTA, all of them per thread

// CTA = (channel of the chunk, tile group i, tile chunk j, frequency tile);
// thread = (frequency, tiles i = r and r + 8), 2 x 16 complex accumulators:
// each spectrum value read from shared memory feeds two (or sixteen) products.
// 8-byte asynchronous copy global -> shared (zero-filled when !valid).
__device__ __forceinline__ void cp_async8(float2* dst, const float2* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__global__ void __launch_bounds__(kXK * kXR, 2) xspec(Pass p, PassArgs a) {
    // the next sample's tile is copied asynchronously into the other buffer
    // while the current one is multiplied (no registers held for it)
    __shared__ float2 sI[2][kXI][kXK];
    __shared__ float2 sJ[2][kXJ][kXK];
    const int NT = (int)p.outer;
    const int64_t K = p.L;
    const int64_t ktiles = (K + kXK - 1) / kXK;
    const int igroups = (NT + kXI - 1) / kXI, jchunks = (NT + kXJ - 1) / kXJ;
    int64_t b = blockIdx.x;
    const int64_t kt = b % ktiles;
    b /= ktiles;
    const int jc = (int)(b % jchunks);
    b /= jchunks;
    const int ig = (int)(b % igroups);
    const int64_t cc = b / igroups;
    const int kl = threadIdx.x % kXK, r = threadIdx.x / kXK;
    const int64_t k = kt * kXK + kl;
    const int i0 = ig * kXI, j0 = jc * kXJ;
    float ar[2][kXJ], ai[2][kXJ];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int jj = 0; jj < kXJ; ++jj) ar[h][jj] = ai[h][jj] = 0.f;
    auto issue = [&](int ts) {
        const float2* Y = reinterpret_cast<const float2*>(a.src) + src_base(a, cc * a.tc + ts);
        const bool kin = k < K;
        const int buf = ts & 1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ii = i0 + r + h * kXR, jr = j0 + r + h * kXR;
            const bool vi = ii < NT && kin, vj = jr < NT && kin;
            cp_async8(&sI[buf][r + h * kXR][kl], vi ? Y + (int64_t)ii * K + k : Y, vi);
            cp_async8(&sJ[buf][r + h * kXR][kl], vj ? Y + (int64_t)jr * K + k : Y, vj);
        }
        cp_async_commit();
    };
    if (a.tc > 0) issue(0);
    for (int ts = 0; ts < a.tc; ++ts) {
        if (ts + 1 < a.tc) {
            issue(ts + 1);
            cp_async_wait<1>();  // this sample's copies done, the next one's in flight
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int buf = ts & 1;
        const float2 y0 = sI[buf][r][kl], y1 = sI[buf][r + kXR][kl];
#pragma unroll
        for (int jj = 0; jj < kXJ; ++jj) {
            const float2 z = sJ[buf][jj][kl];
            ar[0][jj] = fmaf(y0.x, z.x, fmaf(y0.y, z.y, ar[0][jj]));   // y conj(z)
            ai[0][jj] = fmaf(y0.y, z.x, fmaf(-y0.x, z.y, ai[0][jj]));
            ar[1][jj] = fmaf(y1.x, z.x, fmaf(y1.y, z.y, ar[1][jj]));
            ai[1][jj] = fmaf(y1.y, z.x, fmaf(-y1.x, z.y, ai[1][jj]));
        }
        __syncthreads();  // the buffer is refilled two samples later
    }
    if (k >= K) return;
    double2* S = reinterpret_cast<double2*>(a.P + (a.c0 + cc) * a.P_stride);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = i0 + r + h * kXR;
        if (i >= NT) break;
#pragma unroll
        for (int jj = 0; jj < kXJ; ++jj) {
            const int j = j0 + jj;
            if (j >= NT) break;
            double2& s = S[((int64_t)i * NT + j) * K + k];
            s.x += (double)ar[h][jj];
            s.y += (double)ai[h][jj];
        }
    }
}

}  // namespace

int64_t xspec_ctas_per_channel(const Pass& p) {
    const int64_t NT = p.outer;
    return ((p.L + kXK - 1) / kXK) * ((NT + kXI - 1) / kXI) * ((NT + kXJ - 1) / kXJ);
}

cudaError_t xspec_occupancy(int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, xspec, kXK * kXR, 0);
}

cudaError_t launch_xspec(const Pass& p, const PassArgs& a, cudaStream_t st) {
    if (a.src_kind != SRC_BUF) return cudaErrorInvalidValue;
    const int64_t blocks = a.S * xspec_ctas_per_channel(p);
    if (blocks <= 0) return cudaSuccess;
    xspec<<<(unsigned)blocks, kXK * kXR, 0, st>>>(p, a);
    return cudaGetLastError();
}

}  // namespace omni
