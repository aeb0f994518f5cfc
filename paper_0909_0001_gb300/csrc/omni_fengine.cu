// omni_fengine.cu -- F-engine (Appendix A, step 2): each antenna's samples are
// Fourier transformed in time into frequency channels and calibrated, and the
// channel voltages are written in the correlator's input layout [F][T][N].
//
// Frame t of antenna a (frame length 2F, P taps):
//   u_t(n) = sum_p w(p 2F + n) r_a((t + p) 2F + n)         (polyphase sum)
//   X_t(f) = sum_n u_t(n) exp(-2 pi i f n / 2F), f < F     (real FFT, Nyquist dropped)
//   y_t(f) = scale g(f, a) X_t(f)                          (calibration)
// The real frame is packed as F complex points z(m) = u(2m) + i u(2m+1), run
// through an F-point radix-2 FFT in shared memory and unpacked to the real
// spectrum.  F <= 256: one fused pass per 16 antennas, outputs written as
// 16-antenna rows.  Larger F: kernel 1 writes the spectra [N][T][F] to a
// scratch buffer, kernel 2 applies gains and scale, quantises (round half to
// even, clip to +-127) or keeps FP32, and transposes to [F][T][N] through
// shared-memory tiles so that both sides are coalesced.
#include "omni_fft_common.cuh"
#include "omni.h"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

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

// e^{-2 pi i j / 8192}, j < 4096, built on the host in double: every twiddle of
// an F-point stage (e^{-i pi pos / half} = entry pos * 4096 / half) and of the
// real-spectrum unpacking (e^{-i pi f / F} = entry f * 4096 / F) for F <= 4096.
__device__ float2 g_fetw[4096];

constexpr int kFuseAnt = 16;     // antennas per CTA: 32-byte int8 output rows
constexpr int kFusePoints = 4096;  // complex points in shared memory (32 KB)
static_assert(kFuseAnt == 16 && kFusePoints / kFuseAnt == 256, "fused index shifts assume 16 x 256 points");

// Fused F-engine for F <= 256: CTA = (16 consecutive antennas, FR frames),
// FR = 256 / F; polyphase, FFT, unpacking, calibration and quantisation in
// shared memory, each output row (channel f, frame t) written as the 16
// antennas' values together, so no intermediate spectrum goes through HBM.
template <bool I8, bool VEC>
__global__ void __launch_bounds__(kFThreads) fengine_fused(const int8_t* __restrict__ raw, int64_t N,
                                                           int64_t S, int F, int logF, int P,
                                                           const float* __restrict__ w, int64_t T,
                                                           const float2* __restrict__ gains, float scale,
                                                           void* __restrict__ out) {
    // [antenna][frame][F]: each antenna's 256 points padded to 257 so that the
    // 16 antennas of an output row fall in different banks
    constexpr int kPad = kFusePoints / kFuseAnt + 1;
    __shared__ float2 z[kFuseAnt * kPad];
    // this F's twiddles, from the table into shared memory once per CTA:
    // stw[m] = e^{-2 pi i m / F} (m < F/2, the butterflies), utw[f] = e^{-i pi f / F}
    __shared__ float2 stw[128], utw[256];
    for (int j = threadIdx.x; j < F; j += kFThreads) {
        if (j < F / 2) stw[j] = g_fetw[j << (13 - logF)];
        utw[j] = g_fetw[j << (12 - logF)];
    }
    // per antenna: FR frames x F points = 256 points; all index splits below
    // are shifts and masks (F is a power of two)
    constexpr int per = kFusePoints / kFuseAnt, logPer = 8, n = kFusePoints;
    const int FR = per >> logF;
    const int64_t tchunks = (T + FR - 1) / FR;
    const int64_t a0 = (blockIdx.x / tchunks) * kFuseAnt;
    const int64_t t0 = (blockIdx.x % tchunks) * FR;
    const int64_t M = 2 * (int64_t)F;
    // polyphase sums, packed (even, odd), bit-reversed within each frame.
    // VEC (rows 16-byte aligned, F >= 8): a thread takes 8 packed points, one
    // 16-byte load of samples and four of window weights per tap
    if (VEC) {
        for (int idx = threadIdx.x; idx < n / 8; idx += kFThreads) {
            const int al = idx >> (logPer - 3), rem = idx & (per / 8 - 1), fr = rem >> (logF - 3);
            const int m0 = 8 * (rem & ((F >> 3) - 1));
            const int64_t a = a0 + al, t = t0 + fr;
            float ue[8], uo[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) ue[k] = uo[k] = 0.f;
            if (a < N && t < T) {
                const int8_t* ra = raw + a * S;
                for (int p = 0; p < P; ++p) {
                    const int4 rv = __ldg(reinterpret_cast<const int4*>(ra + (t + p) * M + 2 * m0));
                    const int8_t* r = reinterpret_cast<const int8_t*>(&rv);
                    float wv[16];
                    if (w) {
                        const float4* w4 = reinterpret_cast<const float4*>(w + p * M + 2 * m0);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 x = __ldg(w4 + q);
                            wv[4 * q] = x.x;
                            wv[4 * q + 1] = x.y;
                            wv[4 * q + 2] = x.z;
                            wv[4 * q + 3] = x.w;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) wv[q] = 1.f;
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        ue[k] = fmaf(wv[2 * k], (float)r[2 * k], ue[k]);
                        uo[k] = fmaf(wv[2 * k + 1], (float)r[2 * k + 1], uo[k]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                z[al * kPad + fr * F + (int)(__brev((unsigned)(m0 + k)) >> (32 - logF))] = make_float2(ue[k], uo[k]);
        }
    } else
    for (int idx = threadIdx.x; idx < n; idx += kFThreads) {
        const int al = idx >> logPer, rem = idx & (per - 1), fr = rem >> logF, m = rem & (F - 1);
        const int64_t a = a0 + al, t = t0 + fr;
        float ue = 0.f, uo = 0.f;
        if (a < N && t < T) {
            const int8_t* ra = raw + a * S;
            for (int p = 0; p < P; ++p) {
                const int8_t* r = ra + (t + p) * M + 2 * m;
                const float we = w ? __ldg(w + p * M + 2 * m) : 1.f;
                const float wo = w ? __ldg(w + p * M + 2 * m + 1) : 1.f;
                ue = fmaf(we, (float)r[0], ue);
                uo = fmaf(wo, (float)r[1], uo);
            }
        }
        z[al * kPad + fr * F + (int)(__brev((unsigned)m) >> (32 - logF))] = make_float2(ue, uo);
    }
    __syncthreads();
    for (int half = 1, lh = 0; half < F; half <<= 1, ++lh) {
        for (int jt = threadIdx.x; jt < n / 2; jt += kFThreads) {
            const int tr = jt >> (logF - 1), j = jt & (F / 2 - 1);  // transform = (antenna, frame)
            const int pos = j & (half - 1);
            const int base = (tr >> (logPer - logF)) * kPad + (tr & (FR - 1)) * F;
            const int i0 = base + ((j - pos) << 1) + pos, i1 = i0 + half;
            const float2 b = cmul(z[i1], stw[pos << (logF - 1 - lh)]);
            const float2 x0 = z[i0];
            z[i0] = cadd(x0, b);
            z[i1] = csub(x0, b);
        }
        __syncthreads();
    }
    // unpack, calibrate, quantise; thread index: antenna fastest so that each
    // (f, t) row of 16 antennas is one contiguous store
    for (int idx = threadIdx.x; idx < n; idx += kFThreads) {
        const int al = idx & (kFuseAnt - 1), rest = idx >> 4, fr = rest >> logF, f = rest & (F - 1);
        const int64_t a = a0 + al, t = t0 + fr;
        if (a >= N || t >= T) continue;
        const float2* zz = z + al * kPad + fr * F;
        const float2 zf = zz[f], zc = zz[(F - f) & (F - 1)];
        const float2 e = make_float2(0.5f * (zf.x + zc.x), 0.5f * (zf.y - zc.y));
        const float2 o = make_float2(0.5f * (zf.y + zc.y), -0.5f * (zf.x - zc.x));
        const float2 x = cadd(e, cmul(o, utw[f]));
        const float2 g = gains ? __ldg(gains + (int64_t)f * N + a) : make_float2(1.f, 0.f);
        const float2 y = calibrate(x, g, scale);
        const int64_t oi = ((int64_t)f * T + t) * N + a;
        if (I8) reinterpret_cast<char2*>(out)[oi] = make_char2(quantize8(y.x), quantize8(y.y));
        else reinterpret_cast<float2*>(out)[oi] = y;
    }
}

// F = 64 (128-sample frames): eight lanes per (antenna, frame) transform, the
// 64-point FFT as 8 x 8 in registers (m = l + 8 q on lane l, k = k_a + 8 k_b):
//   step 1: lane l: 8-point DFT over q, times w_64^(l k_a)
//   step 2: lane k_a: 8-point DFT over l (the 8 x 8 transpose through a per-warp
//           shared buffer, warp-synchronous: no CTA barrier inside a transform)
// then Z(64 - f) from the partner lane by shuffles, the real-spectrum unpacking and
// calibration.  CTA = 32 consecutive antennas (a warp: 4 of them) x kF64Frames
// frames; per frame the 64 x 32 spectrum is staged so that each (channel, frame)
// row of 32 antennas is one 64-byte (int8) or 256-byte (FP32) store.  Buffer index
// of point m: 9 (m / 8) + m % 8 and a transform pitch of 72: the half-warps of every
// step touch 16 different bank pairs.
constexpr int kF64Ant = 32;
constexpr int kF64Frames = 8;
constexpr int kF64MaxTaps = 8;

// (three CTAs per SM: 6.33 against 6.82 ms on the 64-channel bench leg at two)
template <bool I8>
__global__ void __launch_bounds__(256, 3) fengine64(const int8_t* __restrict__ raw, int64_t N, int64_t S, int P,
                                                 const float* __restrict__ w, int64_t T,
                                                 const float2* __restrict__ gains, float scale,
                                                 void* __restrict__ out) {
    __shared__ float2 zs[8][4 * 72];              // per warp: 4 transforms
    __shared__ float2 ys[64][kF64Ant + 1];        // one frame's spectra, [channel][antenna]
    __shared__ __align__(16) float wsm[kF64MaxTaps * 128];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tr = lane >> 3, l = lane & 7;
    for (int i = tid; i < P * 128; i += 256) wsm[i] = w ? w[i] : 1.f;
    const int64_t tchunks = (T + kF64Frames - 1) / kF64Frames;
    const int64_t a0 = (blockIdx.x / tchunks) * kF64Ant, t0 = (blockIdx.x % tchunks) * kF64Frames;
    const int al = 4 * warp + tr;  // antenna within the CTA
    const int64_t a = a0 + al;
    float2* buf = zs[warp] + 72 * tr;
    // unpacking twiddles e^{-i pi f / 64} and the gains of this lane's f = l + 8 k_b
    float2 ut[8], gl[8];
#pragma unroll
    for (int kb = 0; kb < 8; ++kb) {
        ut[kb] = g_fetw[(l + 8 * kb) * 64];
        gl[kb] = (gains && a < N) ? __ldg(gains + (int64_t)(l + 8 * kb) * N + a) : make_float2(1.f, 0.f);
    }
    __syncthreads();
    for (int64_t t = t0; t < t0 + kF64Frames && t < T; ++t) {
        // polyphase sums of samples 16 l .. 16 l + 15: z(8 l + q) = u(16 l + 2q) + i u(16 l + 2q + 1)
        float ue[8], uo[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) ue[q] = uo[q] = 0.f;
        if (a < N) {
            const int8_t* ra = raw + a * S + 16 * l;
            for (int p = 0; p < P; ++p) {
                const int4 rv = __ldg(reinterpret_cast<const int4*>(ra + (t + p) * 128));
                const int8_t* r = reinterpret_cast<const int8_t*>(&rv);
                const float4* w4 = reinterpret_cast<const float4*>(wsm + p * 128 + 16 * l);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const float4 ww = w4[h];
                    ue[2 * h] = fmaf(ww.x, (float)r[4 * h], ue[2 * h]);
                    uo[2 * h] = fmaf(ww.y, (float)r[4 * h + 1], uo[2 * h]);
                    ue[2 * h + 1] = fmaf(ww.z, (float)r[4 * h + 2], ue[2 * h + 1]);
                    uo[2 * h + 1] = fmaf(ww.w, (float)r[4 * h + 3], uo[2 * h + 1]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) buf[9 * l + q] = make_float2(ue[q], uo[q]);  // point m = 8 l + q
        __syncwarp();
        // step 1: lane l holds z(l + 8 q), q < 8 (buffer index 9 q + l)
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = buf[9 * q + l];
        fft_dif<8, false>(v);
        __syncwarp();
#pragma unroll
        for (int ka = 0; ka < 8; ++ka) {
            float2 y = v[brev(ka, 3)];
            if (l * ka) y = cmul(y, c_tw64[(l * ka) & 63]);
            buf[9 * ka + l] = y;  // Y[l][k_a]
        }
        __syncwarp();
        // step 2: lane k_a = l holds Y[0..7][k_a] -> Z(k_a + 8 k_b) = v[brev(k_b)]
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = buf[9 * l + j];
        fft_dif<8, false>(v);
        __syncwarp();
        // Z(64 - f) for f = k_a + 8 k_b lives on lane (8 - k_a) mod 8 of this transform
        float2 zp[8];
        const int src = (lane & ~7) | ((8 - l) & 7);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float2 mine = v[brev(r, 3)];
            zp[r] = make_float2(__shfl_sync(0xffffffffu, mine.x, src), __shfl_sync(0xffffffffu, mine.y, src));
        }
#pragma unroll
        for (int kb = 0; kb < 8; ++kb) {
            const int f = l + 8 * kb;
            const float2 zf = v[brev(kb, 3)];
            // 64 - f = (8 - l) + 8 (7 - k_b) for l > 0, 8 (8 - k_b) for l = 0
            const float2 zc = l ? zp[(7 - kb) & 7] : zp[(8 - kb) & 7];
            const float2 e = make_float2(0.5f * (zf.x + zc.x), 0.5f * (zf.y - zc.y));
            const float2 o = make_float2(0.5f * (zf.y + zc.y), -0.5f * (zf.x - zc.x));
            const float2 x = cadd(e, cmul(o, ut[kb]));
            ys[f][al] = calibrate(x, gl[kb], scale);
        }
        __syncthreads();
        // rows (channel f, frame t) of the CTA's 32 antennas
        if (I8) {
            const int f = tid >> 2, q = tid & 3;  // 8 antennas (16 bytes) per thread
            if (a0 + 8 * q < N) {
                char2 c[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) c[k] = make_char2(quantize8(ys[f][8 * q + k].x), quantize8(ys[f][8 * q + k].y));
                char2* o = reinterpret_cast<char2*>(out) + ((int64_t)f * T + t) * N + a0 + 8 * q;
                if (a0 + 8 * q + 8 <= N && ((uintptr_t)o % 16) == 0) {
                    *reinterpret_cast<int4*>(o) = *reinterpret_cast<const int4*>(c);
                } else {
                    for (int k = 0; k < 8 && a0 + 8 * q + k < N; ++k) o[k] = c[k];
                }
            }
        } else {
            for (int e = tid; e < 64 * kF64Ant; e += 256) {
                const int f = e / kF64Ant, k = e - f * kF64Ant;
                if (a0 + k < N) reinterpret_cast<float2*>(out)[((int64_t)f * T + t) * N + a0 + k] = ys[f][k];
            }
        }
        __syncthreads();
    }
}

cudaError_t upload_fengine_twiddles() {
    static float2 h[4096];
    for (int j = 0; j < 4096; ++j) {
        const double ang = -6.283185307179586476925286766559 * j / 8192.0;
        h[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    return cudaMemcpyToSymbol(g_fetw, h, sizeof h);
}

}  // namespace

int64_t fengine_frames(int64_t n_samples, int32_t F, int32_t P) {
    const int64_t M = 2 * (int64_t)F;
    return n_samples >= (int64_t)(P - 1) * M ? (n_samples - (int64_t)(P - 1) * M) / M : 0;
}

int64_t fengine_scratch_bytes(int64_t N, int64_t S, int32_t F, int32_t P) {
    if (F <= 256) return 0;  // the fused single pass needs no scratch
    return (int64_t)sizeof(float2) * N * fengine_frames(S, F, P) * F;
}

int64_t fengine_ctas(int64_t N, int64_t T, int32_t F) {
    if (F <= 256) {
        const int FR = kFusePoints / (kFuseAnt * F);
        return ((N + kFuseAnt - 1) / kFuseAnt) * ((T + FR - 1) / FR);
    }
    const int FR = std::max(1, kFPoints / F);
    const int64_t frames_per_cta = std::max(FR, 32);
    return std::max<int64_t>(N * ((T + frames_per_cta - 1) / frames_per_cta), ((F + 31) / 32) * ((N + 31) / 32) * T);
}

cudaError_t launch_fengine(const int8_t* raw, int64_t N, int64_t S, int32_t F, int32_t P,
                           const float* window, const float2* gains, float scale, int out_i8,
                           void* out, float2* scratch, cudaStream_t st) {
    const int64_t T = fengine_frames(S, F, P);
    if (T <= 0 || N <= 0) return cudaSuccess;
    int logF = 0;
    while ((1 << logF) < F) ++logF;
    if (F <= 256) {
        static std::mutex mu;
        static std::vector<int> done;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        {
            std::lock_guard<std::mutex> lock(mu);
            if (std::find(done.begin(), done.end(), dev) == done.end()) {
                if ((e = upload_fengine_twiddles()) != cudaSuccess) return e;
                if ((e = upload_twiddles()) != cudaSuccess) return e;  // this unit's FFT tables
                done.push_back(dev);
            }
        }
        const bool vec = F >= 8 && S % 16 == 0 && (uintptr_t)raw % 16 == 0 && (uintptr_t)window % 16 == 0;
        if (F == 64 && vec && P <= kF64MaxTaps) {
            const unsigned c64 = (unsigned)(((N + kF64Ant - 1) / kF64Ant) * ((T + kF64Frames - 1) / kF64Frames));
            if (out_i8) fengine64<true><<<c64, 256, 0, st>>>(raw, N, S, P, window, T, gains, scale, out);
            else fengine64<false><<<c64, 256, 0, st>>>(raw, N, S, P, window, T, gains, scale, out);
            return cudaGetLastError();
        }
        const unsigned ctas = (unsigned)fengine_ctas(N, T, F);
        if (out_i8 && vec)
            fengine_fused<true, true><<<ctas, kFThreads, 0, st>>>(raw, N, S, F, logF, P, window, T, gains, scale, out);
        else if (out_i8)
            fengine_fused<true, false><<<ctas, kFThreads, 0, st>>>(raw, N, S, F, logF, P, window, T, gains, scale, out);
        else if (vec)
            fengine_fused<false, true><<<ctas, kFThreads, 0, st>>>(raw, N, S, F, logF, P, window, T, gains, scale, out);
        else
            fengine_fused<false, false><<<ctas, kFThreads, 0, st>>>(raw, N, S, F, logF, P, window, T, gains, scale, out);
        return cudaGetLastError();
    }
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
