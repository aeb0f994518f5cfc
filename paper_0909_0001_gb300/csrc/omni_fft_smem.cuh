#pragma once
// omni_fft_smem.cuh -- four-step shared-memory axis transforms (kernel and launch templates).
//
// Four-step passes for power-of-two axes of 128..4096 points: each line is
// split as L = L1 x L2 and transformed as columns then rows in shared memory.
#include "omni_fft_common.cuh"

#include <type_traits>

namespace omni {

// ---------------------------------------------------------------- four-step passes

// L = L1 * L2 (powers of two, L1 >= L2, both <= 64).  A CTA holds W lines
// (W consecutive inner indices, or, for a non-LAST pass along the innermost axis,
// W consecutive outer lines) in shared memory as [w][j1][j2] (j = j2 + L2 j1,
// i.e. natural order), with odd pitches so that column and row sweeps are
// conflict-free.  Step 1: L1-point FFT down each column j2, times w_L^(j2 k1).
// Step 2: L2-point FFT along each row k1 gives X[k1 + L1 k2].  Lines along the
// innermost axis are read and written as contiguous runs: the threads take the
// points of one line first (j2, or k1, fastest) and the lines second.
template <int L1, int L2, int MODE, int SRC>
__global__ void __launch_bounds__(256) pass_smem(Pass p, PassArgs a) {
    constexpr bool FWD = (MODE == MODE_MID || MODE == MODE_LAST);
    constexpr int L = L1 * L2;
    constexpr int PITCH = L2 + 1;
    constexpr int PLANE = L1 * PITCH + 1;
    constexpr int LOG1 = ilog2(L1), LOG2 = ilog2(L2);
    constexpr int TWS = kTwiddleN / L;
    extern __shared__ float2 sm[];
    const int W = p.W;
    const int64_t inner = p.inner;
    const int n = FWD ? L / 2 : L;
    // lines along the innermost axis: W consecutive outer lines per CTA
    const bool rows = MODE != MODE_LAST && inner == 1;
    const int64_t tiles = rows ? (p.outer + W - 1) / W : (inner + W - 1) / W;

    int64_t b = blockIdx.x;
    const int64_t tile = b % tiles;
    b /= tiles;
    const int64_t i0 = rows ? 0 : tile * W;
    int64_t o = 0, s_first = 0, n_samples = 1, cc = 0;
    if constexpr (MODE == MODE_LAST) {
        cc = b;  // outer == 1
        s_first = cc * a.tc;
        n_samples = a.tc;
    } else if (rows) {
        o = tile * W;  // first of the CTA's outer lines
        s_first = b;
    } else {
        o = b % p.outer;
        s_first = b / p.outer;
    }
    auto line_ok = [&](int w) { return rows ? o + w < p.outer : i0 + w < inner; };

    // step-2 ownership (fixed across samples so LAST can keep sums in registers)
    const int u2 = threadIdx.x;
    const int w2 = rows ? u2 / L1 : u2 % W, k1 = rows ? u2 % L1 : u2 / W;
    const bool own2 = u2 < W * L1;
    float acc[L2];
#pragma unroll
    for (int k = 0; k < L2; ++k) acc[k] = 0.0f;

    for (int64_t ts = 0; ts < n_samples; ++ts) {
        const int64_t s = s_first + ts;
        const int64_t base = src_base(a, s) + o * (int64_t)n * inner + i0;
        // load n inputs of each of the W lines (coalesced over inner, or along each line)
        for (int e = threadIdx.x; e < n * W; e += blockDim.x) {
            const int j = rows ? e % n : e / W, w = rows ? e / n : e % W;
            float2 x = make_float2(0.f, 0.f);
            if (line_ok(w)) x = ld_src<SRC>(a.src, rows ? base + (int64_t)w * n + j : base + (int64_t)j * inner + w);
            sm[w * PLANE + (j / L2) * PITCH + (j % L2)] = x;
        }
        __syncthreads();
        // step 1: columns
        for (int u = threadIdx.x; u < W * L2; u += blockDim.x) {
            const int w = rows ? u / L2 : u % W, j2 = rows ? u % L2 : u / W;
            float2* col = sm + w * PLANE + j2;
            float2 v[L1];
#pragma unroll
            for (int j1 = 0; j1 < L1; ++j1)
                v[j1] = (!FWD || j1 < L1 / 2) ? col[j1 * PITCH] : make_float2(0.f, 0.f);
            fft_dif<L1, FWD>(v);
#pragma unroll
            for (int kk = 0; kk < L1; ++kk) {
                float2 y = v[brev(kk, LOG1)];
                const int e = (j2 * kk) & (L - 1);
                if (e) y = cmul(y, g_tw4096[e * TWS]);
                col[kk * PITCH] = y;
            }
        }
        __syncthreads();
        // step 2: rows
        if (own2) {
            const float2* row = sm + w2 * PLANE + k1 * PITCH;
            float2 v[L2];
#pragma unroll
            for (int j2 = 0; j2 < L2; ++j2) v[j2] = row[j2];
            fft_dif<L2, false>(v);
            const int64_t i = i0 + w2;
            if (line_ok(w2)) {
                // line (outer oo, inner ii) of this thread's outputs
                const int64_t oo = rows ? o + w2 : o, ii = rows ? 0 : i;
                if constexpr (MODE == MODE_LAST) {
#pragma unroll
                    for (int k2 = 0; k2 < L2; ++k2) acc[k2] += cnorm(v[brev(k2, LOG2)]);
                } else if constexpr (MODE == MODE_MID) {
                    float2* d = a.dst + s * a.dst_stride + oo * (int64_t)L * inner + ii;
#pragma unroll
                    for (int k2 = 0; k2 < L2; ++k2) d[(int64_t)(k1 + L1 * k2) * inner] = v[brev(k2, LOG2)];
                } else {
                    constexpr int Q = L - 1, SH = L / 2 - 1;
#pragma unroll
                    for (int k2 = 0; k2 < L2; ++k2) {
                        const int k = k1 + L1 * k2;
                        const int q = (k + SH) % L;  // lag k (k < L/2) or k - L (k > L/2)
                        if (k == L / 2) continue;    // the one padding bin no lag maps to
                        const float2 x = v[brev(k2, LOG2)];
                        if constexpr (MODE == MODE_INV_MID) {
                            a.dst[s * a.dst_stride + (oo * (int64_t)Q + q) * inner + ii] = x;
                        } else {
                            a.V[(a.c0 + s) * a.V_stride + (oo * (int64_t)Q + q) * inner + ii] =
                                make_double2((double)x.x * a.scale, -(double)x.y * a.scale);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if constexpr (MODE == MODE_LAST) {
        const int64_t i = i0 + w2;
        if (own2 && i < inner) {
            double* P = a.P + (a.c0 + cc) * a.P_stride + i;
#pragma unroll
            for (int k2 = 0; k2 < L2; ++k2) P[(int64_t)(k1 + L1 * k2) * inner] += (double)acc[k2];
        }
    }
}

template <int L1, int L2, int MODE, int SRC>
cudaError_t launch_smem_t(const Pass& p, const PassArgs& a, cudaStream_t st) {
    const bool rows = MODE != MODE_LAST && p.inner == 1;
    const int64_t tiles = rows ? (p.outer + p.W - 1) / p.W : (p.inner + p.W - 1) / p.W;
    const int64_t blocks = (MODE == MODE_LAST) ? a.S * tiles : rows ? a.S * tiles : a.S * p.outer * tiles;
    if (blocks <= 0) return cudaSuccess;
    const int threads = p.W * L1;
    const size_t smem = (size_t)p.W * (L1 * (L2 + 1) + 1) * sizeof(float2);
    auto k = pass_smem<L1, L2, MODE, SRC>;
    cudaError_t e = smem_limit_once((const void*)k, smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)blocks, threads, smem, st>>>(p, a);
    return cudaGetLastError();
}

// Resident CTAs per SM of the LAST-mode kernel of one four-step length.
template <int L1, int L2>
cudaError_t smem_last_occupancy_len(const Pass& p, int src_kind, int* blocks_per_sm) {
    const int threads = p.W * L1;
    const size_t smem = (size_t)p.W * (L1 * (L2 + 1) + 1) * sizeof(float2);
    return dispatch_src<MODE_LAST>(src_kind, [&](auto S) {
        auto k = pass_smem<L1, L2, MODE_LAST, decltype(S)::value>;
        cudaError_t e = smem_limit_once((const void*)k, smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem);
    });
}

// Every mode and source of one four-step length.
template <int L1, int L2>
cudaError_t launch_smem_len(const Pass& p, const PassArgs& a, cudaStream_t st) {
    return dispatch_mode(p.mode, [&](auto M) {
        return dispatch_src<decltype(M)::value>(a.src_kind, [&](auto S) {
            return launch_smem_t<L1, L2, decltype(M)::value, decltype(S)::value>(p, a, st);
        });
    });
}

}  // namespace omni
