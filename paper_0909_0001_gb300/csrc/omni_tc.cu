// omni_tc.cu -- mixed-precision path: the DFT stages of a 2-level hierarchy of
// 16x16 blocks on an 8x8 grid as split-FP16 tensor-core GEMMs (mma.sync
// m16n8k16, FP32 accumulation).
//
// Each padded DFT of Sec. II.C is a dense complex matrix product.  In real
// form a complex product W x becomes [[Wr, -Wi], [Wi, Wr]] [xr; xi].  The DFT
// matrices and the data are split into FP16 hi + lo parts; the products
// hi*hi + hi*lo + lo*hi recover about 22 bits, and the FP32 accumulators keep
// the sums.  int8 voltages are exact in FP16, so the first GEMM needs only the
// two twiddle halves.
//
// Stage A (per 16x16 block, one warp, Appendix A step 4's per-block 2-D FFT):
//   GEMM 1: D0 [k1 re|im][m2] = W32(k1, m1) . X(m2, m1)^T    (64 x 32 x 16)
//   GEMM 2: D1 [k1][k2 re|im] = D0^T . V32(m2, k2)          (32 x 32 x 64)
//   The accumulator fragments of GEMM 1 are, unchanged, the A operand
//   fragments of GEMM 2 (rows k1, contraction over m2).  Output Y[k2][k1] is
//   written in FP32, scaled by 1/16 so that the level-2 FP16 operands stay in
//   range (|Y| <= 127 * 16 * sqrt 2).
// Stage B (per level-1 frequency kA, one warp; Appendix A step 5):
//   GEMM 3: D2 [k3 re|im][m4] = W16(k3, m3) . Z(m4, m3)^T   (32 x 16 x 8)
//   GEMM 4: D3 [k3][k4 re|im] = D2^T . V16(m4, k4)          (16 x 16 x 32)
//   |D3|^2 is summed over the chunk's samples in registers and folded into the
//   FP64 accumulator with the factor 16^2 that undoes the stage-A scale.
//
// mma.sync m16n8k16 fragment layouts used throughout (lane = 4g + t):
//   A: R0 = A[g][2t..2t+1], R1 = A[g+8][2t..], R2 = A[g][2t+8..], R3 = A[g+8][2t+8..]
//   B: R0 = B[2t..2t+1][g], R1 = B[2t+8..2t+9][g]
//   C: c0 = C[g][2t], c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1]
#include "omni_fft_common.cuh"

#include <cuda_fp16.h>

#include <algorithm>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace omni {
namespace {

// Constant operand fragments (per lane), hi/lo FP16 halves of the DFT matrices.
__device__ uint4 g_tcA1[4][2][2][32];  // [mt][ks][hl][lane] stage A GEMM 1, A operand
__device__ uint2 g_tcB2[2][8][2][32];  // [ks][nt][hl][lane] stage A GEMM 2, B operand
__device__ uint4 g_tcA3[2][2][32];     // [mt][hl][lane]     stage B GEMM 3, A operand
__device__ uint2 g_tcB4[4][2][32];     // [nt][hl][lane]     stage B GEMM 4, B operand

constexpr float kScaleA = 1.0f / 16.0f;   // stage A output scale
constexpr double kFoldB = 256.0;          // (1/kScaleA)^2 applied at the FP64 fold
constexpr int kStageAWarps = 8;

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    // not volatile: the product has no side effects, so the compiler may
    // interleave independent accumulators
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t h2u(__half2 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

// (x0, x1) -> hi = fp16(x), lo = fp16(x - hi), packed (x0 in the low half).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    hi = h2u(h);
    lo = h2u(__floats2half2_rn(x0 - hf.x, x1 - hf.y));
}

// two complex int8 (re0, im0, re1, im1) -> packed real pair, packed imaginary pair
__device__ __forceinline__ void ci8_pair(uint32_t w, uint32_t& re, uint32_t& im) {
    const int8_t r0 = (int8_t)(w & 0xff), i0 = (int8_t)((w >> 8) & 0xff);
    const int8_t r1 = (int8_t)((w >> 16) & 0xff), i1 = (int8_t)(w >> 24);
    re = h2u(__floats2half2_rn((float)r0, (float)r1));
    im = h2u(__floats2half2_rn((float)i0, (float)i1));
}

// ------------------------------------------------------------------ stage A

__global__ void __launch_bounds__(kStageAWarps * 32) tc_stage_a(Pass p, PassArgs a) {
    __shared__ uint4 sA1[4][2][2][32];
    __shared__ uint2 sB2[2][8][2][32];
    for (int i = threadIdx.x; i < 4 * 2 * 2 * 32; i += blockDim.x) (&sA1[0][0][0][0])[i] = (&g_tcA1[0][0][0][0])[i];
    for (int i = threadIdx.x; i < 2 * 8 * 2 * 32; i += blockDim.x) (&sB2[0][0][0][0])[i] = (&g_tcB2[0][0][0][0])[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t units = a.S * p.outer;
    const int64_t warps = (int64_t)gridDim.x * kStageAWarps;
    for (int64_t u = (int64_t)blockIdx.x * kStageAWarps + (threadIdx.x >> 5); u < units; u += warps) {
        const int64_t s = u / p.outer, o = u - s * p.outer;
        const uint8_t* xb = (const uint8_t*)a.src + 2 * (src_base(a, s) + o * 256);
        // B operand of GEMM 1: X rows m2 = g (nt 0) and g+8 (nt 1), m1 pairs 2t.., 2t+8..
        uint32_t bre[2][2], bim[2][2];  // [nt][reg]
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const uint8_t* row = xb + 2 * 16 * (8 * nt + g);
            ci8_pair(*reinterpret_cast<const uint32_t*>(row + 4 * t), bre[nt][0], bim[nt][0]);
            ci8_pair(*reinterpret_cast<const uint32_t*>(row + 4 * t + 16), bre[nt][1], bim[nt][1]);
        }
        // GEMM 1 (X exact: twiddle hi and lo terms); the 8 accumulators are
        // updated round-robin so that consecutive products are independent
        float d0[4][2][4];
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int r = 0; r < 4; ++r) d0[mt][nt][r] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
            for (int hl = 0; hl < 2; ++hl)
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                    const uint4 w = sA1[mt][ks][hl][lane];
                    const uint32_t af[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        if (ks == 0) mma16816(d0[mt][nt], af, bre[nt][0], bre[nt][1]);
                        else mma16816(d0[mt][nt], af, bim[nt][0], bim[nt][1]);
                    }
                }
        // chain: A operand of GEMM 2, [mt'][ks'] from D0 rows (ks' = 0: re, 1: im)
        uint32_t ah[2][2][4], al[2][2][4];
#pragma unroll
        for (int mp = 0; mp < 2; ++mp)
#pragma unroll
            for (int kp = 0; kp < 2; ++kp) {
                const int src = mp + 2 * kp;
                split2(d0[src][0][0], d0[src][0][1], ah[mp][kp][0], al[mp][kp][0]);
                split2(d0[src][0][2], d0[src][0][3], ah[mp][kp][1], al[mp][kp][1]);
                split2(d0[src][1][0], d0[src][1][1], ah[mp][kp][2], al[mp][kp][2]);
                split2(d0[src][1][2], d0[src][1][3], ah[mp][kp][3], al[mp][kp][3]);
            }
        float2* yb = a.dst + s * a.dst_stride + o * 1024;
        // GEMM 2 by pairs of n-tiles (real part nt, imaginary part nt + 4)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            float dre[2][4], dim[2][4];
#pragma unroll
            for (int mp = 0; mp < 2; ++mp)
#pragma unroll
                for (int r = 0; r < 4; ++r) dre[mp][r] = dim[mp][r] = 0.f;
#pragma unroll
            for (int kp = 0; kp < 2; ++kp) {
                const uint2 bhr = sB2[kp][nt][0][lane], blr = sB2[kp][nt][1][lane];
                const uint2 bhi = sB2[kp][nt + 4][0][lane], bli = sB2[kp][nt + 4][1][lane];
                // term-major: the four accumulators (re/im x mp) are independent
#pragma unroll
                for (int term = 0; term < 3; ++term)
#pragma unroll
                    for (int mp = 0; mp < 2; ++mp) {
                        const uint32_t(&aa)[4] = term == 2 ? al[mp][kp] : ah[mp][kp];
                        const uint2 br = term == 1 ? blr : bhr, bi = term == 1 ? bli : bhi;
                        mma16816(dre[mp], aa, br.x, br.y);
                        mma16816(dim[mp], aa, bi.x, bi.y);
                    }
            }
            // Y[k2][k1]: k1 = 16 mp + g (+8), k2 = 8 nt + 2t (+1)
#pragma unroll
            for (int mp = 0; mp < 2; ++mp)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int k1 = 16 * mp + g + (r >= 2 ? 8 : 0);
                    const int k2 = 8 * nt + 2 * t + (r & 1);
                    yb[k2 * 32 + k1] = make_float2(dre[mp][r] * kScaleA, dim[mp][r] * kScaleA);
                }
        }
    }
}

// ------------------------------------------------------------------ stage B (LAST)

// A warp owns (channel of the chunk, 4 consecutive level-1 frequencies kA) for
// all of the chunk's samples.  Each lane loads its two blocks' 4-kA runs (32
// bytes each, whole sectors) straight from global memory: no shared-memory
// tile and no block-wide barrier.  (A tiled form with 32 kA per CTA staged
// through shared memory, and forms with two or four kA interleaved per warp or
// with register prefetch of the next sample, all measured within 6% of this
// one: the legacy HMMA pipe, 57% busy, is the limit, not latency.)
constexpr int kB2Warps = 4;
constexpr int kB2KPW = 4;  // kA per warp

template <bool PREFETCH>
__global__ void __launch_bounds__(kB2Warps * 32, 4) tc_stage_b(Pass p, PassArgs a) {
    __shared__ uint4 sA3[2][2][32];
    __shared__ uint2 sB4[4][2][32];
    for (int i = threadIdx.x; i < 2 * 2 * 32; i += blockDim.x) (&sA3[0][0][0])[i] = (&g_tcA3[0][0][0])[i];
    for (int i = threadIdx.x; i < 4 * 2 * 32; i += blockDim.x) (&sB4[0][0][0])[i] = (&g_tcB4[0][0][0])[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t groups = p.inner / kB2KPW;
    const int64_t u = (int64_t)blockIdx.x * kB2Warps + (threadIdx.x >> 5);
    if (u >= a.S * groups) return;
    const int64_t cc = u / groups;
    const int64_t kA0 = (u - cc * groups) * kB2KPW;
    // GEMM 4 fragments: in registers, or (PREFETCH) read from shared memory at
    // each use so that the registers hold the next sample's data instead
    uint32_t b4[4][2][2];
    if (!PREFETCH)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int hl = 0; hl < 2; ++hl) {
                const uint2 w = sB4[nt][hl][lane];
                b4[nt][hl][0] = w.x;
                b4[nt][hl][1] = w.y;
            }
    float acc[kB2KPW][8];
#pragma unroll
    for (int q = 0; q < kB2KPW; ++q)
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[q][r] = 0.f;
    // blocks m3 + 8 m4 with m4 = g, m3 = 2t and 2t + 1; 4 kA each (two float4)
    const int64_t b0 = 8 * g + 2 * t;
    const int64_t step = p.inner / 2;  // one block, in float4
    auto fetch = [&](float4 (&z)[4], int64_t s) {
        const float4* base = reinterpret_cast<const float4*>(
            reinterpret_cast<const float2*>(a.src) + src_base(a, s) + b0 * p.inner + kA0);
        z[0] = __ldg(base);
        z[1] = __ldg(base + 1);
        z[2] = __ldg(base + step);
        z[3] = __ldg(base + step + 1);
    };
    float4 cur[4], nxt[4];
    if (PREFETCH) fetch(nxt, cc * a.tc);
    for (int ts = 0; ts < a.tc; ++ts) {
        if (PREFETCH) {
#pragma unroll
            for (int i = 0; i < 4; ++i) cur[i] = nxt[i];
            if (ts + 1 < a.tc) fetch(nxt, cc * a.tc + ts + 1);
        } else {
            fetch(cur, cc * a.tc + ts);
        }
#pragma unroll
        for (int q = 0; q < kB2KPW; ++q) {
            // kA0 + q of blocks b0 (z0) and b0 + 1 (z1), at the 1/16 scale stage A writes
            const float4 h0 = cur[q >> 1], h1 = cur[2 + (q >> 1)];
            float2 z0 = (q & 1) ? make_float2(h0.z, h0.w) : make_float2(h0.x, h0.y);
            float2 z1 = (q & 1) ? make_float2(h1.z, h1.w) : make_float2(h1.x, h1.y);
            if (p.unscaled_in) {  // FP32 level-1 pass: apply the scale here (exact, 2^-4)
                z0 = make_float2(z0.x * kScaleA, z0.y * kScaleA);
                z1 = make_float2(z1.x * kScaleA, z1.y * kScaleA);
            }
            uint32_t bh0, bl0, bh1, bl1;
            split2(z0.x, z1.x, bh0, bl0);  // rows re m3 = 2t, 2t+1
            split2(z0.y, z1.y, bh1, bl1);  // rows im m3
            float d2[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int r = 0; r < 4; ++r) d2[mt][r] = 0.f;
#pragma unroll
            for (int term = 0; term < 3; ++term)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const uint4 w = sA3[mt][term == 1 ? 1 : 0][lane];
                    const uint32_t af[4] = {w.x, w.y, w.z, w.w};
                    mma16816(d2[mt], af, term == 2 ? bl0 : bh0, term == 2 ? bl1 : bh1);
                }
            // chain: the GEMM 3 accumulators are the A fragments of GEMM 4
            uint32_t ah[4], al[4];
            split2(d2[0][0], d2[0][1], ah[0], al[0]);
            split2(d2[0][2], d2[0][3], ah[1], al[1]);
            split2(d2[1][0], d2[1][1], ah[2], al[2]);
            split2(d2[1][2], d2[1][3], ah[3], al[3]);
            float d3[4][4];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int r = 0; r < 4; ++r) d3[nt][r] = 0.f;
#pragma unroll
            for (int term = 0; term < 3; ++term)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    uint32_t f0, f1;
                    if (PREFETCH) {
                        const uint2 w = sB4[nt][term == 1 ? 1 : 0][lane];
                        f0 = w.x;
                        f1 = w.y;
                    } else {
                        f0 = b4[nt][term == 1 ? 1 : 0][0];
                        f1 = b4[nt][term == 1 ? 1 : 0][1];
                    }
                    mma16816(d3[nt], term == 2 ? al : ah, f0, f1);
                }
            // |F|^2: n-tiles 0, 1 real and 2, 3 imaginary parts of k4 < 8, k4 >= 8
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    acc[q][4 * nt + r] = fmaf(d3[nt][r], d3[nt][r],
                                              fmaf(d3[nt + 2][r], d3[nt + 2][r], acc[q][4 * nt + r]));
        }
    }
    // fold: fragment r = 4 nt + rr holds (k3 = g + 8 [rr >= 2], k4 = 8 nt + 2t + (rr & 1));
    // the warp's 4 kA are 32 contiguous bytes of each P row (row = 16 k4 + k3)
    double* P = a.P + (a.c0 + cc) * a.P_stride;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int nt = r >> 2, rr = r & 3;
        const int k3 = g + ((rr >= 2) ? 8 : 0), k4 = 8 * nt + 2 * t + (rr & 1);
        double2* row = reinterpret_cast<double2*>(P + (int64_t)(16 * k4 + k3) * p.inner + kA0);
        double2 v0 = row[0], v1 = row[1];
        v0.x += kFoldB * (double)acc[0][r];
        v0.y += kFoldB * (double)acc[1][r];
        v1.x += kFoldB * (double)acc[2][r];
        v1.y += kFoldB * (double)acc[3][r];
        row[0] = v0;
        row[1] = v1;
    }
}

}  // namespace

// ------------------------------------------------------------------ host side

namespace {

uint32_t pack_h2(double a, double b, bool lo_part) {
    // hi = fp16(x); lo = fp16(x - hi)
    auto h = [&](double x) {
        const __half hi = __float2half_rn((float)x);
        if (!lo_part) return hi;
        return __float2half_rn((float)(x - (double)__half2float(hi)));
    };
    const __half ha = h(a), hb = h(b);
    uint16_t ua, ub;
    memcpy(&ua, &ha, 2);
    memcpy(&ub, &hb, 2);
    return (uint32_t)ua | ((uint32_t)ub << 16);
}

// Real form of a complex matrix on the left: [[Wr, -Wi], [Wi, Wr]], W[k][m] = exp(-2 pi i k m / L).
double left_real(int L, int n, int row, int col) {
    const int k = row % L, m = col % n;
    const double ang = -6.283185307179586476925286766559 * (double)k * m / L;
    const bool im_row = row >= L, im_col = col >= n;
    if (!im_row && !im_col) return std::cos(ang);
    if (!im_row && im_col) return -std::sin(ang);
    if (im_row && !im_col) return std::sin(ang);
    return std::cos(ang);
}

// Real form of V on the right: [[Vr, Vi], [-Vi, Vr]], V[m][k] = exp(-2 pi i m k / L).
double right_real(int L, int n, int row, int col) {
    const int m = row % n, k = col % L;
    const double ang = -6.283185307179586476925286766559 * (double)k * m / L;
    const bool im_row = row >= n, im_col = col >= L;
    if (!im_row && !im_col) return std::cos(ang);
    if (!im_row && im_col) return std::sin(ang);
    if (im_row && !im_col) return -std::sin(ang);
    return std::cos(ang);
}

// A fragment (16x16 tile at (r0, c0)) of a matrix given by f(row, col).
template <class F>
uint4 frag_a(F f, int r0, int c0, int lane, bool lo) {
    const int g = lane >> 2, t = lane & 3;
    uint4 u;
    u.x = pack_h2(f(r0 + g, c0 + 2 * t), f(r0 + g, c0 + 2 * t + 1), lo);
    u.y = pack_h2(f(r0 + g + 8, c0 + 2 * t), f(r0 + g + 8, c0 + 2 * t + 1), lo);
    u.z = pack_h2(f(r0 + g, c0 + 2 * t + 8), f(r0 + g, c0 + 2 * t + 9), lo);
    u.w = pack_h2(f(r0 + g + 8, c0 + 2 * t + 8), f(r0 + g + 8, c0 + 2 * t + 9), lo);
    return u;
}

// B fragment (16x8 tile at (r0, c0)).
template <class F>
uint2 frag_b(F f, int r0, int c0, int lane, bool lo) {
    const int g = lane >> 2, t = lane & 3;
    uint2 u;
    u.x = pack_h2(f(r0 + 2 * t, c0 + g), f(r0 + 2 * t + 1, c0 + g), lo);
    u.y = pack_h2(f(r0 + 2 * t + 8, c0 + g), f(r0 + 2 * t + 9, c0 + g), lo);
    return u;
}

}  // namespace

cudaError_t upload_tc_tables() {
    static uint4 A1[4][2][2][32];
    static uint2 B2[2][8][2][32];
    static uint4 A3[2][2][32];
    static uint2 B4[4][2][32];
    auto w1 = [](int r, int c) { return left_real(32, 16, r, c); };
    auto v2 = [](int r, int c) { return right_real(32, 16, r, c); };
    auto w3 = [](int r, int c) { return left_real(16, 8, r, c); };
    auto v4 = [](int r, int c) { return right_real(16, 8, r, c); };
    for (int lane = 0; lane < 32; ++lane)
        for (int hl = 0; hl < 2; ++hl) {
            for (int mt = 0; mt < 4; ++mt)
                for (int ks = 0; ks < 2; ++ks) A1[mt][ks][hl][lane] = frag_a(w1, 16 * mt, 16 * ks, lane, hl);
            for (int ks = 0; ks < 2; ++ks)
                for (int nt = 0; nt < 8; ++nt) B2[ks][nt][hl][lane] = frag_b(v2, 16 * ks, 8 * nt, lane, hl);
            for (int mt = 0; mt < 2; ++mt) A3[mt][hl][lane] = frag_a(w3, 16 * mt, 0, lane, hl);
            for (int nt = 0; nt < 4; ++nt) B4[nt][hl][lane] = frag_b(v4, 0, 8 * nt, lane, hl);
        }
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(g_tcA1, A1, sizeof A1)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(g_tcB2, B2, sizeof B2)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(g_tcA3, A3, sizeof A3)) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_tcB4, B4, sizeof B4);
}

bool tc_supports(const int32_t* n, int D, int dtype_is_ci8) {
    return D == 4 && n[0] == 16 && n[1] == 16 && n[2] == 8 && n[3] == 8 && dtype_is_ci8;
}

int tc_stage_b_tile() { return kB2Warps * kB2KPW; }

// Stage-B form: next-sample register prefetch with shared-memory GEMM 4
// fragments (default), or OMNI_TCB_PREFETCH=0 for register fragments and
// loads at the top of each sample.
void (*stage_b_kernel())(Pass, PassArgs) {
    static const bool prefetch = [] {
        const char* env = std::getenv("OMNI_TCB_PREFETCH");
        return !(env && std::atoi(env) == 0);
    }();
    return prefetch ? tc_stage_b<true> : tc_stage_b<false>;
}

cudaError_t tc_occupancy(int kind, int* blocks_per_sm) {
    if (kind == KIND_TC_A)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tc_stage_a, kStageAWarps * 32, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, stage_b_kernel(), kB2Warps * 32, 0);
}

cudaError_t launch_tc(const Pass& p, const PassArgs& a, cudaStream_t st) {
    if (p.kind == KIND_TC_A) {
        if (a.src_kind != SRC_CI8) return cudaErrorInvalidValue;
        const int64_t units = a.S * p.outer;
        if (units <= 0) return cudaSuccess;
        const int64_t blocks = std::min<int64_t>((units + kStageAWarps - 1) / kStageAWarps,
                                                 std::max(1, p.grid_cap));
        tc_stage_a<<<(unsigned)blocks, kStageAWarps * 32, 0, st>>>(p, a);
        return cudaGetLastError();
    }
    if (a.src_kind != SRC_BUF || p.inner % kB2KPW) return cudaErrorInvalidValue;
    const int64_t warps = a.S * (p.inner / kB2KPW);
    if (warps <= 0) return cudaSuccess;
    stage_b_kernel()<<<(unsigned)((warps + kB2Warps - 1) / kB2Warps), kB2Warps * 32, 0, st>>>(p, a);
    return cudaGetLastError();
}

}  // namespace omni
