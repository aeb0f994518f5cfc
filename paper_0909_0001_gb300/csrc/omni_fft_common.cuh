// omni_fft_common.cuh -- device helpers shared by the transform-pass kernels.
//
// Included by each kernel translation unit; the twiddle tables have internal
// linkage, so every unit owns a copy that upload_twiddles() fills.
#pragma once

#include "omni_internal.h"

#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

namespace omni {

// exp(-2 pi i k / 64): every register-FFT twiddle (spans <= 64) is one of these.
static __constant__ float2 c_tw64[64];
// exp(-2 pi i k / 4096): four-step twiddles w_L^(j2 k1) for L <= 4096.
static __device__ float2 g_tw4096[kTwiddleN];

// Fill this unit's tables on the current device (values from double-precision
// cos/sin, rounded once to float).
[[maybe_unused]] static cudaError_t upload_twiddles() {
    const double two_pi = 6.283185307179586476925286766559;
    std::vector<float2> t64(64), t4096(kTwiddleN);
    for (int k = 0; k < 64; ++k) {
        const double ang = two_pi * k / 64.0;
        t64[k] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    for (int k = 0; k < kTwiddleN; ++k) {
        const double ang = two_pi * k / (double)kTwiddleN;
        t4096[k] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    cudaError_t e = cudaMemcpyToSymbol(c_tw64, t64.data(), sizeof(float2) * 64);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_tw4096, t4096.data(), sizeof(float2) * kTwiddleN);
}

// Raise a kernel's dynamic shared-memory limit once per (kernel, device, size):
// later launches (including ones recorded into a CUDA graph) make no attribute call.
inline cudaError_t smem_limit_once(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void*, int>, size_t>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (auto& d : done)
        if (d.first.first == kernel && d.first.second == dev && d.second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.push_back({{kernel, dev}, bytes});
    return e;
}

// ---------------------------------------------------------------- complex helpers

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float cnorm(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }
__host__ __device__ constexpr int brev(int k, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((k >> b) & 1) << (bits - 1 - b);
    return r;
}

// a * exp(-2 pi i j / M) for 0 <= j < M/2, M <= 64; j and M are compile-time
// constants once the callers are unrolled, so the special angles cost no
// multiplies.
__device__ __forceinline__ float2 twiddle(float2 a, int j, int M) {
    const float h = 0.70710678118654752440f;
    if (j == 0) return a;
    if (4 * j == M) return make_float2(a.y, -a.x);
    if (8 * j == M) return make_float2((a.x + a.y) * h, (a.y - a.x) * h);
    if (8 * j == 3 * M) return make_float2((a.y - a.x) * h, -(a.x + a.y) * h);
    return cmul(a, c_tw64[j * (64 / M)]);
}

// In-place radix-2 decimation-in-frequency DFT of L (power of two <= 64)
// points held in registers: natural-order input, bit-reversed output
// (X[k] = v[brev(k)]).  PRUNED: inputs n >= L/2 are zero, so the first stage
// is twiddles only.
template <int L, bool PRUNED>
__device__ __forceinline__ void fft_dif(float2 (&v)[L]) {
    constexpr int LOG = ilog2(L);
#pragma unroll
    for (int st = 0; st < LOG; ++st) {
        const int half = L >> (st + 1);
#pragma unroll
        for (int base = 0; base < L; base += 2 * half) {
#pragma unroll
            for (int j = 0; j < half; ++j) {
                const float2 a = v[base + j];
                if (PRUNED && st == 0) {
                    v[base + j + half] = twiddle(a, j, 2 * half);
                } else {
                    const float2 b = v[base + j + half];
                    v[base + j] = cadd(a, b);
                    v[base + j + half] = twiddle(csub(a, b), j, 2 * half);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- sources

// Offset of sample s's first element in the source, in source elements.
// (Kept to one comparison per branch: a second one here raised the tensor-core
// stage-A kernel from 80 to 82 registers, past an allocation step, and cost 9%
// of the mixed path's step time through lost co-residency.)
__device__ __forceinline__ int64_t src_base(const PassArgs& a, int64_t s) {
    if (a.src_kind == SRC_CF32 || a.src_kind == SRC_CI8)
        return ((a.vc0 + s / a.tc) * a.T + a.t0 + s % a.tc) * a.N;
    if (a.src_kind >= SRC_P64) return (a.c0 + s) * a.src_stride;  // P64, PC64: per channel
    return s * a.src_stride;
}

template <int SRC>
__device__ __forceinline__ float2 ld_src(const void* p, int64_t e) {
    if constexpr (SRC == SRC_BUF || SRC == SRC_CF32) {
        return __ldg(reinterpret_cast<const float2*>(p) + e);
    } else if constexpr (SRC == SRC_CI8) {
        const char2 c = reinterpret_cast<const char2*>(p)[e];
        return make_float2((float)c.x, (float)c.y);
    } else if constexpr (SRC == SRC_PC64) {
        // conjugated on load: the inverse passes run forward (e^-) transforms and
        // conjugate at the end, IFFT(S) = conj(FFT(conj(S))) / L; a real |F|^2
        // needs no input conjugate, a complex cross-spectrum does
        const double2 d = __ldg(reinterpret_cast<const double2*>(p) + e);
        return make_float2((float)d.x, -(float)d.y);
    } else {
        return make_float2((float)__ldg(reinterpret_cast<const double*>(p) + e), 0.0f);
    }
}

// Inverse passes: output slot q of a line holds lag q - q_shift, which is FFT
// bin (q - q_shift) mod L.
__device__ __forceinline__ int inv_bin(int q, int q_shift, int L) {
    int k = q - q_shift;
    return k < 0 ? k + L : k;
}

// Source kinds a pass mode can read: forward passes read the caller's
// voltages or the scratch buffer, inverse passes the FP64 accumulator (real
// |F|^2, or complex cross-spectra of the tile hybrid) or the scratch buffer.
template <int MODE, class F>
cudaError_t dispatch_src(int src_kind, F&& f) {
    if constexpr (MODE == MODE_MID || MODE == MODE_LAST) {
        switch (src_kind) {
            case SRC_BUF: return f(std::integral_constant<int, SRC_BUF>{});
            case SRC_CF32: return f(std::integral_constant<int, SRC_CF32>{});
            case SRC_CI8: return f(std::integral_constant<int, SRC_CI8>{});
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (src_kind) {
            case SRC_BUF: return f(std::integral_constant<int, SRC_BUF>{});
            case SRC_P64: return f(std::integral_constant<int, SRC_P64>{});
            case SRC_PC64: return f(std::integral_constant<int, SRC_PC64>{});
            default: return cudaErrorInvalidValue;
        }
    }
}

template <class F>
cudaError_t dispatch_mode(int mode, F&& f) {
    switch (mode) {
        case MODE_MID: return f(std::integral_constant<int, MODE_MID>{});
        case MODE_LAST: return f(std::integral_constant<int, MODE_LAST>{});
        case MODE_INV_MID: return f(std::integral_constant<int, MODE_INV_MID>{});
        default: return f(std::integral_constant<int, MODE_INV_LAST>{});
    }
}

}  // namespace omni
