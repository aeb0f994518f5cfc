// omni_fengine.cu -- F-engine (Appendix A, step 2): each antenna's samples are
// Fourier transformed in time into frequency channels and calibrated, and the
// channel voltages are written in the correlator's input layout [F][T][N].
//
// Frame t of antenna a (frame length 2F, P taps):
//   u_t(n) = sum_p w(p 2F + n) r_a((t + p) 2F + n)         (polyphase sum)
//   X_t(f) = sum_n u_t(n) exp(-2 pi i f n / 2F), f < F     (real FFT, Nyquist dropped)
//   y_t(f) = scale g(f, a) X_t(f)                          (calibration)
// Kernel 1 packs the real frame as F complex points z(m) = u(2m) + i u(2m+1),
// runs an F-point radix-2 FFT in shared memory and unpacks the real spectrum;
// kernel 2 applies gains and scale, quantises (round half to even, clip to
// +-127) or keeps FP32, and transposes [N][T][F] -> [F][T][N] through
// shared-memory tiles so that both sides are coalesced.
#include "omni_fft_common.cuh"
#include "omni.h"

#include <algorithm>

namespace omni {
namespace {

constexpr int kFThreads = 256;
constexpr int kFPoints = 512;  // complex points in shared memory per round (>= F)

// CTA = (antenna, run of frames); each round transforms FR = kFPoints / F
// frames at once (one F-point FFT each) so that small F still fills the CTA.
__global__ void __launch_bounds__(kFThreads) fengine_fft(const int8_t* __restrict__ raw, int64_t N,
                                                         int64_t S, int F, int logF, int P,
                                                         const float* __restrict__ w, int64_t T,
                                                         int frames_per_cta, float2* __restrict__ inter) {
    extern __shared__ float2 z[];  // FR frames x F complex points
    const int FR = max(1, kFPoints / F);
    const int64_t chunks = (T + frames_per_cta - 1) / frames_per_cta;
    const int64_t a = blockIdx.x / chunks;
    const int64_t t0 = (blockIdx.x - a * chunks) * frames_per_cta;
    const int64_t M = 2 * (int64_t)F;
    const int8_t* ra = raw + a * S;
    const int n = FR * F;
    for (int64_t tr = t0; tr < t0 + frames_per_cta && tr < T; tr += FR) {
        // polyphase sum, packed (even, odd), bit-reversed within each frame
        for (int idx = threadIdx.x; idx < n; idx += kFThreads) {
            const int fr = idx / F, m = idx - fr * F;
            const int64_t t = tr + fr;
            float ue = 0.f, uo = 0.f;
            if (t < T)
                for (int p = 0; p < P; ++p) {
                    const int8_t* r = ra + (t + p) * M + 2 * m;  // byte loads: rows need no alignment
                    const float we = w ? __ldg(w + p * M + 2 * m) : 1.f;
                    const float wo = w ? __ldg(w + p * M + 2 * m + 1) : 1.f;
                    ue = fmaf(we, (float)r[0], ue);
                    uo = fmaf(wo, (float)r[1], uo);
                }
            z[fr * F + (int)(__brev((unsigned)m) >> (32 - logF))] = make_float2(ue, uo);
        }
        __syncthreads();
        // radix-2 decimation-in-time stages, all frames of the round together
        for (int half = 1; half < F; half <<= 1) {
            for (int jt = threadIdx.x; jt < n / 2; jt += kFThreads) {
                const int fr = jt / (F / 2), j = jt - fr * (F / 2);
                const int pos = j & (half - 1);
                const int i0 = fr * F + ((j - pos) << 1) + pos, i1 = i0 + half;
                float s, c;
                sincospif(-(float)pos / (float)half, &s, &c);
                const float2 b = cmul(z[i1], make_float2(c, s));
                const float2 x0 = z[i0];
                z[i0] = cadd(x0, b);
                z[i1] = csub(x0, b);
            }
            __syncthreads();
        }
        // real spectrum: X_f = E_f + e^{-i pi f / F} O_f with
        // E_f = (Z_f + conj Z_{F-f}) / 2, O_f = (Z_f - conj Z_{F-f}) / (2i)
        for (int idx = threadIdx.x; idx < n; idx += kFThreads) {
            const int fr = idx / F, f = idx - fr * F;
            const int64_t t = tr + fr;
            if (t >= T) continue;
            const float2 zf = z[fr * F + f], zc = z[fr * F + ((F - f) & (F - 1))];
            const float2 e = make_float2(0.5f * (zf.x + zc.x), 0.5f * (zf.y - zc.y));
            const float2 o = make_float2(0.5f * (zf.y + zc.y), -0.5f * (zf.x - zc.x));
            float s, c;
            sincospif(-(float)f / (float)F, &s, &c);
            inter[(a * T + t) * F + f] = cadd(e, cmul(o, make_float2(c, s)));
        }
        __syncthreads();
    }
}

// y = scale * g * X with no contraction, so that the float and the int8 output
// modes compute the same float (the quantiser decides on exactly that value)
__device__ __forceinline__ float2 calibrate(float2 x, float2 g, float scale) {
    const float yr = __fsub_rn(__fmul_rn(g.x, x.x), __fmul_rn(g.y, x.y));
    const float yi = __fadd_rn(__fmul_rn(g.x, x.y), __fmul_rn(g.y, x.x));
    return make_float2(__fmul_rn(scale, yr), __fmul_rn(scale, yi));
}

__device__ __forceinline__ int8_t quantize8(float v) {
    const int q = __float2int_rn(v);  // round half to even
    return (int8_t)max(-127, min(127, q));
}

// CTA = 32 channels x 32 antennas of one frame; 32 x 8 threads.
template <bool I8>
__global__ void __launch_bounds__(256) fengine_out(const float2* __restrict__ inter, int64_t N, int64_t T,
                                                   int F, const float2* __restrict__ gains, float scale,
                                                   void* __restrict__ out) {
    __shared__ float2 tile[32][33];
    const int64_t ftiles = (F + 31) / 32, atiles = (N + 31) / 32;
    int64_t b = blockIdx.x;
    const int64_t ft = b % ftiles;
    b /= ftiles;
    const int64_t at = b % atiles;
    const int64_t t = b / atiles;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {  // rows: antennas; columns: channels
        const int64_t a = at * 32 + r, f = ft * 32 + tx;
        tile[r][tx] = (a < N && f < F) ? __ldg(inter + (a * T + t) * F + f) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {  // rows: channels; columns: antennas
        const int64_t f = ft * 32 + r, a = at * 32 + tx;
        if (f >= F || a >= N) continue;
        const float2 g = gains ? __ldg(gains + f * N + a) : make_float2(1.f, 0.f);
        const float2 y = calibrate(tile[tx][r], g, scale);
        const int64_t o = (f * T + t) * N + a;
        if (I8) reinterpret_cast<char2*>(out)[o] = make_char2(quantize8(y.x), quantize8(y.y));
        else reinterpret_cast<float2*>(out)[o] = y;
    }
}

}  // namespace

int64_t fengine_frames(int64_t n_samples, int32_t F, int32_t P) {
    const int64_t M = 2 * (int64_t)F;
    return n_samples >= (int64_t)(P - 1) * M ? (n_samples - (int64_t)(P - 1) * M) / M : 0;
}

cudaError_t launch_fengine(const int8_t* raw, int64_t N, int64_t S, int32_t F, int32_t P,
                           const float* window, const float2* gains, float scale, int out_i8,
                           void* out, float2* scratch, cudaStream_t st) {
    const int64_t T = fengine_frames(S, F, P);
    if (T <= 0 || N <= 0) return cudaSuccess;
    int logF = 0;
    while ((1 << logF) < F) ++logF;
    const int FR = std::max(1, kFPoints / F);
    const int frames_per_cta = std::max(FR, 32);
    const int64_t ctas = N * ((T + frames_per_cta - 1) / frames_per_cta);
    const size_t smem = sizeof(float2) * (size_t)FR * F;
    fengine_fft<<<(unsigned)ctas, kFThreads, smem, st>>>(raw, N, S, F, logF, P, window, T, frames_per_cta,
                                                       scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t out_ctas = ((F + 31) / 32) * ((N + 31) / 32) * T;
    if (out_i8) fengine_out<true><<<(unsigned)out_ctas, 256, 0, st>>>(scratch, N, T, F, gains, scale, out);
    else fengine_out<false><<<(unsigned)out_ctas, 256, 0, st>>>(scratch, N, T, F, gains, scale, out);
    return cudaGetLastError();
}

}  // namespace omni
