#pragma once
// omni_fft_level.cuh -- level passes: both axes of one hierarchy level in one kernel.
//
// The hypercube of Eq. ProofEq2 has two axes per level.  A level pass
// transforms axes a = 2k and b = 2k+1 of level k together: per sample the data
// is [outer][n_b][n_a][inner] on input and [outer][L_b][L_a][inner] on output
// (inner = product of the padded lengths of the finer levels, outer = product
// of the sizes of the coarser ones).
//
// Tiling is fixed at compile time:
//  * the finest level (inner == 1): a CTA owns U whole n x n blocks of
//    antennas (Appendix A step 4's per-block 2-D FFT), W = 1, each block
//    contiguous in memory;
//  * a coarser level: a CTA owns W consecutive inner indices (U = 1) so that
//    every global access is a W-wide coalesced row.
// The tile is staged in shared memory as [k_b][k_a][w]; axis a is transformed
// one line per thread (pruned first stage: the upper half of every line is
// zero padding), then axis b, whose outputs go straight to global memory (MID)
// or are squared and summed over the chunk's samples in registers and folded
// into the FP64 accumulator once per chunk (LAST: the |F|^2 time integration).
// In LAST mode the next sample's inputs are loaded into registers while the
// current sample is transformed.
#include "omni_fft_common.cuh"

#include <algorithm>
#include <type_traits>

namespace omni {

// Compile-time tiling of a level pass of L points per axis.
template <int L, bool FINEST, int MODE>
struct LevelTile {
    static constexpr int N = L / 2;
    static constexpr int LPT = (MODE == MODE_LAST) ? (L >= 64 ? 1 : 2) : 1;
    static constexpr int W = FINEST ? 1 : 256 * LPT / L;
    static constexpr int U = FINEST ? ((MODE == MODE_LAST) ? 1 : (L >= 64 ? 2 : 256 / L)) : 1;
    static constexpr int RP = FINEST ? L + 1 : L;          // row pitch, odd for W == 1
    static constexpr int UPL = L * RP * W;                 // shared elements per unit
    static constexpr int IN_PER_UNIT = N * N * W;
    static constexpr int LINES_A = U * N * W;
    static constexpr int LINES_B = U * L * W;
    static constexpr int THREADS = (MODE == MODE_LAST)
        ? (LINES_B / LPT < 32 ? 32 : LINES_B / LPT)
        : (LINES_B > 256 ? 256 : (LINES_B < 32 ? 32 : LINES_B));
    static constexpr int EPT = (U * IN_PER_UNIT + THREADS - 1) / THREADS;  // loads per thread
    static constexpr size_t SMEM = (size_t)U * UPL * sizeof(float2);
};

template <int L, bool FINEST, int MODE, int SRC>
__global__ void __launch_bounds__(LevelTile<L, FINEST, MODE>::THREADS)
level_pass(Pass p, PassArgs a) {
    using T = LevelTile<L, FINEST, MODE>;
    constexpr int N = T::N, W = T::W, U = T::U, RP = T::RP, UPL = T::UPL;
    constexpr int LOG = ilog2(L);
    constexpr int NT = T::THREADS, LPT = T::LPT, EPT = T::EPT;
    extern __shared__ float2 sm[];
    const int64_t inner = p.inner;

    if constexpr (MODE == MODE_MID) {
        __shared__ int64_t unit_src[U];
        __shared__ int64_t unit_dst[U];
        // ---- per-unit base offsets (sample, outer block, inner tile)
        const int64_t tiles = FINEST ? 1 : (inner + W - 1) / W;
        const int64_t units_total = a.S * p.outer * tiles;
        if (threadIdx.x < U) {
            const int64_t ug = (int64_t)blockIdx.x * U + threadIdx.x;
            int64_t sb = -1, db = -1;
            if (ug < units_total) {
                const int64_t tile = FINEST ? 0 : ug % tiles;
                const int64_t so = FINEST ? ug : ug / tiles;
                const int64_t o = so % p.outer, s = so / p.outer;
                sb = src_base(a, s) + o * (int64_t)N * N * inner + tile * W;
                db = s * a.dst_stride + o * (int64_t)L * L * inner + tile * W;
            }
            unit_src[threadIdx.x] = sb;
            unit_dst[threadIdx.x] = db;
        }
        __syncthreads();
        // valid w of this CTA's tile (U == 1 when W > 1)
        const int64_t i_lim = FINEST ? 1 : inner - ((int64_t)blockIdx.x % tiles) * W;
        // ---- load
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int e = threadIdx.x + q * NT;
            if (e < U * T::IN_PER_UNIT) {
                const int u = e / T::IN_PER_UNIT;
                const int r = e - u * T::IN_PER_UNIT;
                const int w = r % W, ja = (r / W) % N, jb = r / (W * N);
                float2 x = make_float2(0.f, 0.f);
                if (unit_src[u] >= 0 && w < i_lim)
                    x = ld_src<SRC>(a.src, unit_src[u] + (int64_t)(jb * N + ja) * inner + w);
                sm[u * UPL + (jb * RP + ja) * W + w] = x;
            }
        }
        __syncthreads();
        // ---- axis a
        for (int l = threadIdx.x; l < T::LINES_A; l += NT) {
            const int u = l / (N * W), r = l - u * (N * W);
            const int jb = r / W, w = r % W;
            float2* row = sm + u * UPL + jb * RP * W + w;
            float2 v[L];
#pragma unroll
            for (int j = 0; j < L; ++j) v[j] = (j < N) ? row[j * W] : make_float2(0.f, 0.f);
            fft_dif<L, true>(v);
#pragma unroll
            for (int k = 0; k < L; ++k) row[k * W] = v[brev(k, LOG)];
        }
        __syncthreads();
        // ---- axis b, straight to global memory
        for (int l = threadIdx.x; l < T::LINES_B; l += NT) {
            const int u = l / (L * W), r = l - u * (L * W);
            const int ka = r / W, w = r % W;
            const float2* col = sm + u * UPL + ka * W + w;
            float2 v[L];
#pragma unroll
            for (int j = 0; j < L; ++j) v[j] = (j < N) ? col[j * RP * W] : make_float2(0.f, 0.f);
            fft_dif<L, true>(v);
            if (unit_dst[u] >= 0 && w < i_lim) {
                float2* d = a.dst + unit_dst[u] + (int64_t)ka * inner + w;
#pragma unroll
                for (int k = 0; k < L; ++k) d[(int64_t)k * L * inner] = v[brev(k, LOG)];
            }
        }
    } else {
        // ---- LAST: CTA = (channel of the chunk, inner tile); loop over samples
        const int64_t tiles = FINEST ? 1 : (inner + W - 1) / W;
        const int64_t cc = blockIdx.x / tiles;
        const int64_t tile = blockIdx.x - cc * tiles;
        const int64_t i0 = tile * W;
        const int64_t i_lim = FINEST ? 1 : inner - i0;
        float acc[LPT][L];
#pragma unroll
        for (int li = 0; li < LPT; ++li)
#pragma unroll
            for (int k = 0; k < L; ++k) acc[li][k] = 0.0f;
        // per-thread load slots: offset within a sample, shared-memory index
        int64_t goff[EPT];
        int sidx[EPT];
        bool live[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int e = threadIdx.x + q * NT;  // U == 1
            const int w = e % W, ja = (e / W) % N, jb = e / (W * N);
            live[q] = e < T::IN_PER_UNIT && w < i_lim;
            goff[q] = (int64_t)(jb * N + ja) * inner + i0 + w;
            sidx[q] = e < T::IN_PER_UNIT ? (jb * RP + ja) * W + w : -1;
        }
        float2 pre[EPT];
        auto fetch = [&](int64_t s) {
            const int64_t base = src_base(a, s);
#pragma unroll
            for (int q = 0; q < EPT; ++q)
                pre[q] = live[q] ? ld_src<SRC>(a.src, base + goff[q]) : make_float2(0.f, 0.f);
        };
        fetch(cc * a.tc);
        for (int ts = 0; ts < a.tc; ++ts) {
#pragma unroll
            for (int q = 0; q < EPT; ++q)
                if (sidx[q] >= 0) sm[sidx[q]] = pre[q];
            if (ts + 1 < a.tc) fetch(cc * a.tc + ts + 1);  // in flight during this sample
            __syncthreads();
            for (int l = threadIdx.x; l < T::LINES_A; l += NT) {
                const int jb = l / W, w = l % W;
                float2* row = sm + jb * RP * W + w;
                float2 v[L];
#pragma unroll
                for (int j = 0; j < L; ++j) v[j] = (j < N) ? row[j * W] : make_float2(0.f, 0.f);
                fft_dif<L, true>(v);
#pragma unroll
                for (int k = 0; k < L; ++k) row[k * W] = v[brev(k, LOG)];
            }
            __syncthreads();
#pragma unroll
            for (int li = 0; li < LPT; ++li) {
                const int l = threadIdx.x + li * NT;
                if (l < T::LINES_B) {
                    const int ka = l / W, w = l % W;
                    const float2* col = sm + ka * W + w;
                    float2 v[L];
#pragma unroll
                    for (int j = 0; j < L; ++j) v[j] = (j < N) ? col[j * RP * W] : make_float2(0.f, 0.f);
                    fft_dif<L, true>(v);
#pragma unroll
                    for (int k = 0; k < L; ++k) acc[li][k] += cnorm(v[brev(k, LOG)]);
                }
            }
            __syncthreads();
        }
        double* P = a.P + (a.c0 + cc) * a.P_stride;
        const double fs = a.fold_scale != 0.0 ? a.fold_scale : 1.0;
#pragma unroll
        for (int li = 0; li < LPT; ++li) {
            const int l = threadIdx.x + li * NT;
            if (l < T::LINES_B) {
                const int ka = l / W, w = l % W;
                if (w < i_lim) {
#pragma unroll
                    for (int k = 0; k < L; ++k)
                        P[((int64_t)k * L + ka) * inner + i0 + w] += fs * (double)acc[li][k];
                }
            }
        }
    }
}

// Finest-level MID pass, persistent: the CTA walks groups of U contiguous
// blocks (group g, g + gridDim.x, ...), loading the next group two elements
// per thread per load (4-byte int8 or 16-byte float loads, coalesced) into
// registers while the current group is transformed.  Requires every group to
// lie inside one sample (outer % U == 0) and 16-byte aligned group bases.
template <int L, int SRC>
__global__ void __launch_bounds__(LevelTile<L, true, MODE_MID>::THREADS)
level_finest_stream(Pass p, PassArgs a) {
    using T = LevelTile<L, true, MODE_MID>;
    constexpr int N = T::N, U = T::U, RP = T::RP, UPL = T::UPL, NT = T::THREADS;
    constexpr int LOG = ilog2(L);
    constexpr int PER_GROUP = U * N * N;
    constexpr int PAIRS = PER_GROUP / 2 / NT;  // two-element loads per thread per group
    static_assert(PER_GROUP % (2 * NT) == 0, "group must split evenly into pairs");
    using Pair = typename std::conditional<SRC == SRC_CI8, char4, float4>::type;
    extern __shared__ float2 sm[];
    const int64_t groups = a.S * p.outer / U;

    auto group_src = [&](int64_t g) -> const Pair* {
        const int64_t ug = g * U;                    // first unit: (sample, outer block)
        const int64_t s = ug / p.outer, o = ug - s * p.outer;
        return reinterpret_cast<const Pair*>(
            (SRC == SRC_CI8 ? (const char*)a.src + 2 * (src_base(a, s) + o * N * N)
                            : (const char*)a.src + 8 * (src_base(a, s) + o * N * N)));
    };
    Pair pre[PAIRS];
    auto fetch = [&](int64_t g) {
        const Pair* src = group_src(g);
#pragma unroll
        for (int q = 0; q < PAIRS; ++q) pre[q] = src[threadIdx.x + q * NT];
    };
    int64_t g = blockIdx.x;
    if (g < groups) fetch(g);
    for (; g < groups; g += gridDim.x) {
        // registers -> shared memory ([u][j_b][j_a] with odd row pitch)
#pragma unroll
        for (int q = 0; q < PAIRS; ++q) {
            const int e = 2 * (threadIdx.x + q * NT);
            const int u = e / (N * N), r = e - u * N * N;
            const int jb = r / N, ja = r - jb * N;  // ja even: both elements in one row
            float2 x0, x1;
            if constexpr (SRC == SRC_CI8) {
                x0 = make_float2((float)pre[q].x, (float)pre[q].y);
                x1 = make_float2((float)pre[q].z, (float)pre[q].w);
            } else {
                x0 = make_float2(pre[q].x, pre[q].y);
                x1 = make_float2(pre[q].z, pre[q].w);
            }
            float2* d = sm + u * UPL + jb * RP + ja;
            d[0] = x0;
            d[1] = x1;
        }
        if (g + gridDim.x < groups) fetch(g + gridDim.x);  // in flight during this group
        __syncthreads();
        for (int l = threadIdx.x; l < T::LINES_A; l += NT) {
            const int u = l / N, jb = l - u * N;
            float2* row = sm + u * UPL + jb * RP;
            float2 v[L];
#pragma unroll
            for (int j = 0; j < L; ++j) v[j] = (j < N) ? row[j] : make_float2(0.f, 0.f);
            fft_dif<L, true>(v);
#pragma unroll
            for (int k = 0; k < L; ++k) row[k] = v[brev(k, LOG)];
        }
        __syncthreads();
        const int64_t ug0 = g * U;
        const int64_t s = ug0 / p.outer, o0 = ug0 - s * p.outer;
        float2* dst0 = a.dst + s * a.dst_stride + o0 * (int64_t)L * L;
        for (int l = threadIdx.x; l < T::LINES_B; l += NT) {
            const int u = l / L, ka = l - u * L;
            const float2* col = sm + u * UPL + ka;
            float2 v[L];
#pragma unroll
            for (int j = 0; j < L; ++j) v[j] = (j < N) ? col[j * RP] : make_float2(0.f, 0.f);
            fft_dif<L, true>(v);
            float2* d = dst0 + (int64_t)u * L * L + ka;
#pragma unroll
            for (int k = 0; k < L; ++k) d[k * L] = v[brev(k, LOG)];
        }
        __syncthreads();
    }
}

template <int L, bool FINEST, int MODE, int SRC>
cudaError_t launch_level_t(const Pass& p, const PassArgs& a, cudaStream_t st) {
    using T = LevelTile<L, FINEST, MODE>;
    const int64_t tiles = FINEST ? 1 : (p.inner + T::W - 1) / T::W;
    const int64_t blocks = (MODE == MODE_LAST) ? a.S * tiles
                                               : (a.S * p.outer * tiles + T::U - 1) / T::U;
    if (blocks <= 0) return cudaSuccess;
    if constexpr (FINEST && MODE == MODE_MID && SRC != SRC_P64 && L >= 8) {
        constexpr int PER_GROUP = T::U * T::N * T::N;
        const size_t eb = SRC == SRC_CI8 ? 2 : 8;
        const bool contiguous = p.outer % T::U == 0 && PER_GROUP % (2 * T::THREADS) == 0;
        const bool aligned = (((uintptr_t)a.src) % 16 == 0) && ((PER_GROUP * eb) % 16 == 0) &&
                             ((SRC == SRC_BUF ? a.src_stride * eb : a.N * eb) % 16 == 0);
        if (contiguous && aligned && p.grid_cap > 0) {
            const int64_t groups = a.S * p.outer / T::U;
            const int64_t grid = std::min<int64_t>(groups, p.grid_cap);
            auto ks = level_finest_stream<L, SRC>;
            cudaError_t e = smem_limit_once((const void*)ks, T::SMEM);
            if (e != cudaSuccess) return e;
            ks<<<(unsigned)grid, T::THREADS, T::SMEM, st>>>(p, a);
            return cudaGetLastError();
        }
    }
    auto k = level_pass<L, FINEST, MODE, SRC>;
    cudaError_t e = smem_limit_once((const void*)k, T::SMEM);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)blocks, T::THREADS, T::SMEM, st>>>(p, a);
    return cudaGetLastError();
}

// Every forward mode and source of one square level length.
template <int L>
cudaError_t launch_level_len(const Pass& p, const PassArgs& a, cudaStream_t st) {
    return dispatch_mode(p.mode, [&](auto M) -> cudaError_t {
        constexpr int MODE = decltype(M)::value;
        if constexpr (MODE == MODE_MID || MODE == MODE_LAST) {
            return dispatch_src<MODE>(a.src_kind, [&](auto S) {
                return p.inner == 1 ? launch_level_t<L, true, MODE, decltype(S)::value>(p, a, st)
                                    : launch_level_t<L, false, MODE, decltype(S)::value>(p, a, st);
            });
        } else {
            return cudaErrorInvalidValue;
        }
    });
}

// Resident CTAs per SM of the finest-level streaming MID pass (host sizing).
template <int L>
cudaError_t level_stream_blocks_per_sm(int src_kind, int* out) {
    *out = 0;
    if constexpr (L < 8) return cudaSuccess;  // 4-point levels use level_pass
    else return dispatch_src<MODE_MID>(src_kind, [&](auto S) -> cudaError_t {
        using T = LevelTile<L, true, MODE_MID>;
        auto k = level_finest_stream<L, decltype(S)::value>;
        cudaError_t e = smem_limit_once((const void*)k, T::SMEM);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, T::THREADS, T::SMEM);
    });
}

// Resident CTAs per SM of the LAST level pass of a given shape (host sizing).
template <int L>
cudaError_t level_last_blocks_per_sm(bool finest, int src_kind, int* out) {
    return dispatch_src<MODE_LAST>(src_kind, [&](auto S) -> cudaError_t {
        constexpr int SRC = decltype(S)::value;
        if (finest) {
            using T = LevelTile<L, true, MODE_LAST>;
            auto k = level_pass<L, true, MODE_LAST, SRC>;
            cudaError_t e = smem_limit_once((const void*)k, T::SMEM);
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, T::THREADS, T::SMEM);
        }
        using T = LevelTile<L, false, MODE_LAST>;
        auto k = level_pass<L, false, MODE_LAST, SRC>;
        cudaError_t e = smem_limit_once((const void*)k, T::SMEM);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, T::THREADS, T::SMEM);
    });
}

}  // namespace omni
