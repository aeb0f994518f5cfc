#pragma once
// omni_fft_reg.cuh -- register-resident axis transforms (kernel and launch templates).
//
// Register passes: one thread per line, the whole (power-of-two, <= 64) line
// held in registers.  A forward pass reads the n_d measured values of a line
// and produces all L_d = 2 n_d frequencies (zero padding never stored; the
// first radix-2 stage is twiddles only; a beam-space pointing axis, n_d = L_d,
// is transformed whole).  The last forward pass squares the
// modulus and sums over the chunk's samples before folding into FP64.  An
// inverse pass transforms a full line and keeps the 2 n_d - 1 lag bins.
#include "omni_fft_common.cuh"

#include <type_traits>

namespace omni {

// ---------------------------------------------------------------- register passes

// One thread per line; the whole line lives in registers.
template <int L, int MODE, int SRC>
__global__ void __launch_bounds__(256) pass_reg(Pass p, PassArgs a) {
    constexpr bool FWD = (MODE == MODE_MID || MODE == MODE_LAST);
    constexpr int LOG = ilog2(L);
    const int64_t flat = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t inner = p.inner;
    const void* src = a.src;

    if constexpr (MODE == MODE_LAST) {
        // outer == 1: thread per (channel, inner index); loop over the chunk's samples.
        if (flat >= a.S * inner) return;
        const int64_t cc = flat / inner, i = flat - cc * inner;
        float acc[L];
#pragma unroll
        for (int k = 0; k < L; ++k) acc[k] = 0.0f;
        for (int tt = 0; tt < a.tc; ++tt) {
            const int64_t s = cc * a.tc + tt;
            const int64_t base = src_base(a, s) + i;
            float2 v[L];
#pragma unroll
            for (int j = 0; j < L; ++j)
                v[j] = (j < L / 2) ? ld_src<SRC>(src, base + (int64_t)j * inner) : make_float2(0.f, 0.f);
            fft_dif<L, true>(v);
#pragma unroll
            for (int k = 0; k < L; ++k) acc[k] += cnorm(v[brev(k, LOG)]);
        }
        double* P = a.P + (a.c0 + cc) * a.P_stride + i;
#pragma unroll
        for (int k = 0; k < L; ++k) P[(int64_t)k * inner] += (double)acc[k];
        return;
    } else {
        const int64_t lines = p.outer * inner;
        if (flat >= a.S * lines) return;
        const int64_t s = flat / lines;
        const int64_t r = flat - s * lines;
        const int64_t o = r / inner, i = r - o * inner;
        const int64_t base = src_base(a, s) + o * p.n * inner + i;
        // an unpadded forward line (n == L: a beam-space pointing axis) is a full
        // transform; otherwise the upper half is the zero padding
        const bool full = !FWD || p.n == L;
        float2 v[L];
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const bool live = full || j < L / 2;
            v[j] = live ? ld_src<SRC>(src, base + (int64_t)j * inner) : make_float2(0.f, 0.f);
        }
        if (full) fft_dif<L, false>(v);
        else fft_dif<L, true>(v);
        if constexpr (MODE == MODE_MID) {
            float2* d = a.dst + s * a.dst_stride + o * (int64_t)L * inner + i;
#pragma unroll
            for (int k = 0; k < L; ++k) d[(int64_t)k * inner] = v[brev(k, LOG)];
        } else {
            // keep 2 n_d - 1 = L - 1 bins: lags -(L/2-1) .. L/2-1
            constexpr int Q = L - 1;
            constexpr int SH = L / 2 - 1;
            if constexpr (MODE == MODE_INV_MID) {
                float2* d = a.dst + s * a.dst_stride + o * (int64_t)Q * inner + i;
#pragma unroll
                for (int q = 0; q < Q; ++q) d[(int64_t)q * inner] = v[brev((q - SH + L) % L, LOG)];
            } else {
                double2* d = a.V + (a.c0 + s) * a.V_stride + o * (int64_t)Q * inner + i;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float2 x = v[brev((q - SH + L) % L, LOG)];
                    d[(int64_t)q * inner] = make_double2((double)x.x * a.scale, -(double)x.y * a.scale);
                }
            }
        }
    }
}

template <int L, int MODE, int SRC>
cudaError_t launch_reg_t(const Pass& p, const PassArgs& a, cudaStream_t st) {
    const int64_t work = (MODE == MODE_LAST) ? a.S * p.inner : a.S * p.outer * p.inner;
    if (work <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (work + threads - 1) / threads;
    pass_reg<L, MODE, SRC><<<(unsigned)blocks, threads, 0, st>>>(p, a);
    return cudaGetLastError();
}

// Every mode and source of one register-pass length.
template <int L>
cudaError_t launch_reg_len(const Pass& p, const PassArgs& a, cudaStream_t st) {
    return dispatch_mode(p.mode, [&](auto M) {
        return dispatch_src<decltype(M)::value>(a.src_kind, [&](auto S) {
            return launch_reg_t<L, decltype(M)::value, decltype(S)::value>(p, a, st);
        });
    });
}

}  // namespace omni
