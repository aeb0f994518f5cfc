// omni_fft_direct.cu -- direct-DFT axis transforms.
//
// Direct-DFT passes for axes of any length (non-powers of two, and the
// degenerate single-antenna lattice), one thread per output value.
#include "omni_fft_common.cuh"

#include <type_traits>

namespace omni {

// ---------------------------------------------------------------- direct DFT passes

// Any length: one thread per output value, X[k] = sum_j x[j] w_L^(jk mod L).
template <int MODE, int SRC>
__global__ void __launch_bounds__(256) pass_direct(Pass p, PassArgs a) {
    const int64_t flat = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t inner = p.inner;
    const int L = p.L, n = p.n, Q = p.q_out;
    if constexpr (MODE == MODE_LAST) {
        const int64_t per = (int64_t)L * inner;
        if (flat >= a.S * per) return;
        const int64_t cc = flat / per;
        const int64_t r = flat - cc * per;
        const int k = (int)(r / inner);
        const int64_t i = r - (int64_t)k * inner;
        float acc = 0.0f;
        for (int tt = 0; tt < a.tc; ++tt) {
            const int64_t base = src_base(a, cc * a.tc + tt) + i;
            float2 sum = make_float2(0.f, 0.f);
            int m = 0;
            for (int j = 0; j < n; ++j) {
                const float2 x = ld_src<SRC>(a.src, base + (int64_t)j * inner);
                const float2 w = __ldg(p.tw + m);
                sum.x = fmaf(x.x, w.x, fmaf(-x.y, w.y, sum.x));
                sum.y = fmaf(x.x, w.y, fmaf(x.y, w.x, sum.y));
                m += k;
                if (m >= L) m -= L;
            }
            acc += cnorm(sum);
        }
        a.P[(a.c0 + cc) * a.P_stride + (int64_t)k * inner + i] += (double)acc;
    } else {
        const int64_t per = p.outer * (int64_t)Q * inner;
        if (flat >= a.S * per) return;
        const int64_t s = flat / per;
        int64_t r = flat - s * per;
        const int64_t o = r / ((int64_t)Q * inner);
        r -= o * (int64_t)Q * inner;
        const int q = (int)(r / inner);
        const int64_t i = r - (int64_t)q * inner;
        const int k = (MODE == MODE_MID) ? q : inv_bin(q, p.q_shift, L);
        const int64_t base = src_base(a, s) + o * (int64_t)n * inner + i;
        float2 sum = make_float2(0.f, 0.f);
        int m = 0;
        for (int j = 0; j < n; ++j) {
            const float2 x = ld_src<SRC>(a.src, base + (int64_t)j * inner);
            const float2 w = __ldg(p.tw + m);
            sum.x = fmaf(x.x, w.x, fmaf(-x.y, w.y, sum.x));
            sum.y = fmaf(x.x, w.y, fmaf(x.y, w.x, sum.y));
            m += k;
            if (m >= L) m -= L;
        }
        const int64_t e = (o * (int64_t)Q + q) * inner + i;
        if constexpr (MODE == MODE_INV_LAST) {
            a.V[(a.c0 + s) * a.V_stride + e] = make_double2((double)sum.x * a.scale, -(double)sum.y * a.scale);
        } else {
            a.dst[s * a.dst_stride + e] = sum;
        }
    }
}


namespace {

template <int MODE, int SRC>
cudaError_t launch_direct_t(const Pass& p, const PassArgs& a, cudaStream_t st) {
    const int64_t work = (MODE == MODE_LAST) ? a.S * (int64_t)p.L * p.inner
                                             : a.S * p.outer * (int64_t)p.q_out * p.inner;
    if (work <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (work + threads - 1) / threads;
    pass_direct<MODE, SRC><<<(unsigned)blocks, threads, 0, st>>>(p, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_direct(const Pass& p, const PassArgs& a, cudaStream_t st) {
    return dispatch_mode(p.mode, [&](auto M) {
        return dispatch_src<decltype(M)::value>(a.src_kind, [&](auto S) {
            return launch_direct_t<decltype(M)::value, decltype(S)::value>(p, a, st);
        });
    });
}

}  // namespace omni
