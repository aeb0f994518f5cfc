// omni_fft_smem3.cu -- three-step shared-memory forward transforms of 2048 and
// 4096 points.
//
// L = L1 x L2 x L3 with L1 = L2 = 16 and L3 = 8 or 16, so that no register
// transform is longer than 16 points (a 64-point column held in registers took
// 210-255 registers and left one or two CTAs per SM).  With j = j3 + L3 j2 + M j1
// (M = L2 L3) and k = k1 + L1 (k2 + L2 k3):
//   step 1: L1-point DFTs over j1 for each j' = j3 + L3 j2, times w_L^(j' k1)
//   step 2: L2-point DFTs over j2 for each (k1, j3), times w_M^(j3 k2)
//   step 3: L3-point DFTs over j3 for each (k1, k2)
// (the factorisation of w_L^(j k) into the three DFTs and two twiddle stages).
// The inverse passes use the same transform (the inverse runs as a forward FFT)
// on all L inputs and keep the lag slots, the last one conjugated and scaled.
// A CTA transforms W lines held in shared memory as [j1][j2][j3] with a row pitch
// L3 + 1, a j1 pitch = 8 and a line pitch = 16 / W (mod 16) float2, so that each
// step's half-warps touch 16 different bank pairs; each thread reads one twiddle w^j from
// a shared-memory table (LAST: through L1) and forms the powers it needs in
// registers.  LAST runs two 256-thread CTAs per SM and, reading the scratch
// buffer, copies the next sample's inputs asynchronously (cp.async) into a staging
// buffer while the current sample runs steps 2 and 3.  Lines
// are W consecutive inner indices (strided axes), or, for an axis that is
// innermost in memory, W consecutive outer lines read and written contiguously.
// MID and the inverse passes write through shared memory in natural order; LAST keeps
// |X|^2 of the chunk's samples in registers and folds them into the FP64
// accumulator once.  The forward inputs j >= L/2 are zero (padding): step 1
// never reads them.
#include "omni_fft_common.cuh"

namespace omni {
namespace {

// threads per CTA: 512, or 256 for LAST (whose 32 FP32 |X|^2 sums per thread and
// ~120 registers would otherwise leave one CTA per SM and no overlap of one CTA's
// loads with another's transforms)
template <int MODE>
__host__ __device__ constexpr int s3_threads() { return MODE == MODE_LAST ? 256 : 512; }

template <int L1, int L2, int L3, int W>
struct S3Geom {
    static constexpr int L = L1 * L2 * L3, M = L2 * L3;
    static constexpr int P2 = L3 + 1;
    static constexpr int P1 = L2 * P2 + ((8 - (L2 * P2) % 16 + 16) % 16);
    // lines 16 / W float2 apart mod 16: the W lines x 16 / W consecutive inputs of a
    // half-warp's strided load land in 16 different bank pairs
    static constexpr int PG = (16 / W) % 16;
    static constexpr int PLANE = L1 * P1 + ((PG - (L1 * P1) % 16 + 16) % 16);
    static_assert(P1 % 16 == 8 && PLANE % 16 == PG, "pitches");
    static_assert(PLANE >= L + L / 16, "the natural-order output fits the plane");
};

__device__ __forceinline__ int out_at(int k) { return k + (k >> 4); }  // natural order, 1 pad per 16

// 16-byte asynchronous copy global -> shared (zero-filled when !valid; src must
// still be a valid address)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// w^k for k < 16 from w^1 (one shared-memory read per thread instead of a read of
// w^(j k) per k, whose stride k across the lanes conflicted): powers 1..3 and
// 4, 8, 12 by squaring, then w^(4a + b) = w^(4a) w^b (at most six roundings)
struct Pow16 {
    float2 p[4], q[4];  // w^b, w^(4a)
    __device__ __forceinline__ explicit Pow16(float2 w) {
        p[0] = make_float2(1.f, 0.f);
        p[1] = w;
        p[2] = cmul(w, w);
        p[3] = cmul(p[2], w);
        q[0] = p[0];
        q[1] = cmul(p[2], p[2]);
        q[2] = cmul(q[1], q[1]);
        q[3] = cmul(q[2], q[1]);
    }
    __device__ __forceinline__ float2 operator()(int k) const {  // k a compile-time constant after unrolling
        return (k & 3) == 0 ? q[k >> 2] : (k < 4 ? p[k] : cmul(q[k >> 2], p[k & 3]));
    }
};

// PF (LAST from the float2 scratch buffer, 16-byte aligned rows): the next
// sample's W x L/2 inputs are copied asynchronously into a staging buffer
// [j][W] while the current sample runs steps 2 and 3, and step 1 reads them there.
template <int L1, int L2, int L3, int W, bool ROWS, int MODE, int SRC, bool PF>
__global__ void __launch_bounds__(s3_threads<MODE>(), 512 / s3_threads<MODE>()) pass_smem3(Pass p, PassArgs a) {
    constexpr int kS3Threads = s3_threads<MODE>();
    using G = S3Geom<L1, L2, L3, W>;
    static_assert(!PF || (MODE == MODE_LAST && SRC == SRC_BUF && !ROWS && W % 2 == 0), "prefetch form");
    constexpr int L = G::L, M = G::M, P1 = G::P1, P2 = G::P2, PLANE = G::PLANE;
    constexpr bool FWD = MODE == MODE_MID || MODE == MODE_LAST;  // forward: inputs j >= L/2 are zero
    constexpr int LOG1 = ilog2(L1), LOG2 = ilog2(L2), LOG3 = ilog2(L3);
    constexpr int T1 = (W * M + kS3Threads - 1) / kS3Threads;       // step-1 tasks per thread
    constexpr int T2 = (W * L1 * L3 + kS3Threads - 1) / kS3Threads;  // step 2
    constexpr int T3 = (W * L1 * L2 + kS3Threads - 1) / kS3Threads;  // step 3
    // LAST reads its twiddles through L1 (its shared memory holds the lines and,
    // with PF, the staging buffer of two CTAs per SM); the others keep a table
    constexpr bool TWG = MODE == MODE_LAST;
    extern __shared__ float2 sm[];
    float2* tw = sm;                    // [L]: w_L^m (not TWG)
    float2* lines = sm + (TWG ? 0 : L); // [W][PLANE]
    float2* stage = lines + W * PLANE;  // PF: [L/2][W]
    const int tid = threadIdx.x;
    if constexpr (!TWG)
        for (int m = tid; m < L; m += kS3Threads) tw[m] = g_tw4096[m * (kTwiddleN / L)];
    auto twv = [&](int m) { return TWG ? __ldg(&g_tw4096[m * (kTwiddleN / L)]) : tw[m]; };

    const int n = p.n;  // inputs per line (<= L / 2 forward, <= L inverse)
    const int64_t inner = p.inner;
    int64_t b = blockIdx.x, o0 = 0, i0 = 0, s_first = 0, n_samples = 1, cc = 0;
    if constexpr (ROWS) {  // W consecutive outer lines (inner == 1), one sample
        const int64_t tiles = (p.outer + W - 1) / W;
        o0 = (b % tiles) * W;
        s_first = b / tiles;
    } else {
        const int64_t tiles = (inner + W - 1) / W;
        i0 = (b % tiles) * W;
        b /= tiles;
        if constexpr (MODE == MODE_LAST) {
            cc = b;  // outer == 1
            s_first = cc * a.tc;
            n_samples = a.tc;
        } else {
            o0 = b % p.outer;
            s_first = b / p.outer;
        }
    }
    // the lines this CTA has (the last tile may be short)
    auto line_ok = [&](int w) { return ROWS ? o0 + w < p.outer : i0 + w < inner; };

    float acc[T3][L3];
#pragma unroll
    for (int u = 0; u < T3; ++u)
#pragma unroll
        for (int k = 0; k < L3; ++k) acc[u][k] = 0.f;

    // PF: one sample's inputs, 16 bytes (two lines) per copy; rows j >= n and lines
    // past the axis are zero-filled
    auto prefetch = [&](int64_t s) {
        const float2* row0 = reinterpret_cast<const float2*>(a.src) + s * a.src_stride + i0;
        constexpr int CH = W / 2, NC = (L / 2) * CH / kS3Threads;
        static_assert(NC * kS3Threads == (L / 2) * CH, "copies per thread");
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const int c = tid + r * kS3Threads, j = c / CH, h = c % CH;
            const bool ok = j < n && i0 + 2 * h < inner;
            cp_async16(stage + j * W + 2 * h, ok ? row0 + (int64_t)j * inner + 2 * h : row0, ok);
        }
        cp_async_commit();
    };
    if constexpr (PF)
        if (n_samples > 0) prefetch(s_first);

    for (int64_t ts = 0; ts < n_samples; ++ts) {
        const int64_t s = s_first + ts;
        const int64_t base = src_base(a, s);
        // load: contiguous runs along the line (ROWS) or W inner indices per input,
        // each thread's loads issued together before its shared-memory stores
        auto at_j = [&](int w, int j) { return w * PLANE + (j / M) * P1 + ((j / L3) % L2) * P2 + (j % L3); };
        if constexpr (PF) {
            cp_async_wait_all();  // this sample's staging copies (the barrier below publishes them)
        } else if constexpr (ROWS) {
            constexpr int NR = (FWD ? L / 2 : L) / kS3Threads;  // loads per line and thread
            float2 x[W][NR];
#pragma unroll
            for (int w = 0; w < W; ++w)
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int j = tid + r * kS3Threads;
                    x[w][r] = (j < n && line_ok(w)) ? ld_src<SRC>(a.src, base + (o0 + w) * (int64_t)n + j)
                                                    : make_float2(0.f, 0.f);
                }
#pragma unroll
            for (int w = 0; w < W; ++w)
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int j = tid + r * kS3Threads;
                    if (j < n) lines[at_j(w, j)] = x[w][r];
                }
        } else {
            constexpr int NB = 16;  // loads in flight per thread
            const int n_in = W * n;
            const int64_t col = base + o0 * (int64_t)n * inner + i0;
            for (int e0 = 0; e0 < n_in; e0 += NB * kS3Threads) {
                float2 x[NB];
#pragma unroll
                for (int r = 0; r < NB; ++r) {
                    const int e = e0 + tid + r * kS3Threads, j = e / W, w = e % W;
                    x[r] = (e < n_in && line_ok(w)) ? ld_src<SRC>(a.src, col + (int64_t)j * inner + w)
                                                    : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int r = 0; r < NB; ++r) {
                    const int e = e0 + tid + r * kS3Threads;
                    if (e < n_in) lines[at_j(e % W, e / W)] = x[r];
                }
            }
        }
        __syncthreads();
        // step 1: j' = j3 + L3 j2 fastest across the threads
#pragma unroll
        for (int u = 0; u < T1; ++u) {
            const int t = tid + u * kS3Threads;
            if (t < W * M) {
                // PF: the W lines fastest (the half-warp reads 16 consecutive staged inputs)
                const int w = PF ? t % W : t / M, jp = PF ? t / W : t - w * M, j2 = jp / L3, j3 = jp - j2 * L3;
                float2* col = lines + w * PLANE + j2 * P2 + j3;
                float2 v[L1];
#pragma unroll
                for (int j1 = 0; j1 < L1; ++j1) {
                    if constexpr (PF)
                        v[j1] = j1 < L1 / 2 ? stage[(jp + M * j1) * W + w] : make_float2(0.f, 0.f);
                    else
                        v[j1] = (!FWD || j1 < L1 / 2) ? col[j1 * P1] : make_float2(0.f, 0.f);
                }
                fft_dif<L1, FWD>(v);
                const Pow16 pw(twv(jp));  // w_L^(j' k1)
#pragma unroll
                for (int k1 = 0; k1 < L1; ++k1) {
                    float2 y = v[brev(k1, LOG1)];
                    if (k1) y = cmul(y, pw(k1));
                    col[k1 * P1] = y;
                }
            }
        }
        __syncthreads();
        if constexpr (PF)
            if (ts + 1 < n_samples) prefetch(s + 1);  // the staging buffer is free until the next step 1
        // step 2: (k1, j3), j3 fastest
#pragma unroll
        for (int u = 0; u < T2; ++u) {
            const int t = tid + u * kS3Threads;
            if (t < W * L1 * L3) {
                const int j3 = t % L3, k1 = (t / L3) % L1, w = t / (L3 * L1);
                float2* row = lines + w * PLANE + k1 * P1 + j3;
                float2 v[L2];
#pragma unroll
                for (int j2 = 0; j2 < L2; ++j2) v[j2] = row[j2 * P2];
                fft_dif<L2, false>(v);
                const Pow16 pw(twv(L1 * j3));  // w_M^(j3 k2) = w_L^(L1 j3 k2)
#pragma unroll
                for (int k2 = 0; k2 < L2; ++k2) {
                    float2 y = v[brev(k2, LOG2)];
                    if (k2) y = cmul(y, pw(k2));
                    row[k2 * P2] = y;
                }
            }
        }
        __syncthreads();
        // step 3: (k1, k2), k2 fastest; X[k1 + L1 k2 + L1 L2 k3]
        float2 out[T3][L3];
#pragma unroll
        for (int u = 0; u < T3; ++u) {
            const int t = tid + u * kS3Threads;
            if (t < W * L1 * L2) {
                const int k2 = t % L2, k1 = (t / L2) % L1, w = t / (L2 * L1);
                const float2* r = lines + w * PLANE + k1 * P1 + k2 * P2;
                float2 v[L3];
#pragma unroll
                for (int j3 = 0; j3 < L3; ++j3) v[j3] = r[j3];
                fft_dif<L3, false>(v);
#pragma unroll
                for (int k3 = 0; k3 < L3; ++k3) {
                    out[u][k3] = v[brev(k3, LOG3)];
                    if constexpr (MODE == MODE_LAST) acc[u][k3] += cnorm(out[u][k3]);
                }
            }
        }
        if constexpr (MODE != MODE_LAST) {
            // the spectrum in natural order through shared memory, then contiguous stores
            __syncthreads();
#pragma unroll
            for (int u = 0; u < T3; ++u) {
                const int t = tid + u * kS3Threads;
                if (t < W * L1 * L2) {
                    const int k2 = t % L2, k1 = (t / L2) % L1, w = t / (L2 * L1);
#pragma unroll
                    for (int k3 = 0; k3 < L3; ++k3)
                        lines[w * PLANE + out_at(k1 + L1 * k2 + L1 * L2 * k3)] = out[u][k3];
                }
            }
            __syncthreads();
            if constexpr (!FWD) {
                // inverse: the kept lags, slot q = bin (q - q_shift) mod L; the last
                // pass conjugates and scales (the inverse runs as a forward FFT)
                const int Q = p.q_out;
                for (int e = tid; e < W * Q; e += kS3Threads) {
                    int w, q;
                    if constexpr (ROWS) {
                        w = e / Q;
                        q = e - w * Q;
                    } else {
                        q = e / W;
                        w = e - q * W;
                    }
                    if (!line_ok(w)) continue;
                    const float2 x = lines[w * PLANE + out_at(inv_bin(q, p.q_shift, L))];
                    const int64_t o = ROWS ? o0 + w : o0, i = ROWS ? 0 : i0 + w;
                    const int64_t at = (o * Q + q) * inner + i;
                    if constexpr (MODE == MODE_INV_MID)
                        a.dst[s * a.dst_stride + at] = x;
                    else
                        a.V[(a.c0 + s) * a.V_stride + at] = make_double2((double)x.x * a.scale, -(double)x.y * a.scale);
                }
            } else {
                float2* d = a.dst + s * a.dst_stride;
                for (int e = tid; e < W * L; e += kS3Threads) {
                    int w, k;
                    if constexpr (ROWS) {
                        w = e / L;
                        k = e - w * L;
                    } else {
                        k = e / W;
                        w = e - k * W;
                    }
                    if (!line_ok(w)) continue;
                    const float2 x = lines[w * PLANE + out_at(k)];
                    if constexpr (ROWS) d[(o0 + w) * (int64_t)L + k] = x;
                    else d[o0 * (int64_t)L * inner + (int64_t)k * inner + i0 + w] = x;
                }
            }
        }
        __syncthreads();
    }
    if constexpr (PF) cp_async_wait_all();  // nothing left in flight at exit
    if constexpr (MODE == MODE_LAST) {
        double* P = a.P + (a.c0 + cc) * a.P_stride;
#pragma unroll
        for (int u = 0; u < T3; ++u) {
            const int t = tid + u * kS3Threads;
            if (t < W * L1 * L2) {
                const int k2 = t % L2, k1 = (t / L2) % L1, w = t / (L2 * L1);
                if (!line_ok(w)) continue;
#pragma unroll
                for (int k3 = 0; k3 < L3; ++k3)
                    P[(int64_t)(k1 + L1 * k2 + L1 * L2 * k3) * inner + i0 + w] += (double)acc[u][k3];
            }
        }
    }
}

template <int L1, int L2, int L3, int W, int MODE, bool PF>
constexpr size_t s3_smem() {
    constexpr int L = L1 * L2 * L3;
    return sizeof(float2) * ((MODE == MODE_LAST ? 0 : (size_t)L) + (size_t)W * S3Geom<L1, L2, L3, W>::PLANE +
                             (PF ? (size_t)W * (L / 2) : 0));
}

// the prefetch form: LAST from the scratch buffer with 16-byte aligned input rows
inline bool s3_prefetch(const Pass& p, const PassArgs& a) {
    return p.mode == MODE_LAST && a.src_kind == SRC_BUF && p.inner % 2 == 0 && a.src_stride % 2 == 0 &&
           (reinterpret_cast<uintptr_t>(a.src) & 15) == 0;
}

template <int L1, int L2, int L3, int W, bool ROWS, int MODE, int SRC, bool PF>
cudaError_t launch_s3(const Pass& p, const PassArgs& a, cudaStream_t st) {
    int64_t blocks;
    if (ROWS) blocks = a.S * ((p.outer + W - 1) / W);
    else blocks = (MODE == MODE_LAST ? a.S : a.S * p.outer) * ((p.inner + W - 1) / W);
    if (blocks <= 0) return cudaSuccess;
    constexpr size_t smem = s3_smem<L1, L2, L3, W, MODE, PF>();
    auto k = pass_smem3<L1, L2, L3, W, ROWS, MODE, SRC, PF>;
    cudaError_t e = smem_limit_once((const void*)k, smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)blocks, s3_threads<MODE>(), smem, st>>>(p, a);
    return cudaGetLastError();
}

// one length: lines along a strided axis (W = WC; WL for LAST) or along the innermost axis (W = WR)
template <int L1, int L2, int L3, int WC, int WR, int WL>
cudaError_t launch_s3_len(const Pass& p, const PassArgs& a, cudaStream_t st) {
    const bool fwd = p.mode == MODE_MID || p.mode == MODE_LAST;
    if (p.n > (fwd ? L1 * L2 * L3 / 2 : L1 * L2 * L3)) return cudaErrorInvalidValue;
    const bool rows = p.mode != MODE_LAST && p.inner == 1;
    if (p.W != (rows ? WR : p.mode == MODE_LAST ? WL : WC)) return cudaErrorInvalidValue;
    if (p.mode == MODE_LAST) {
        if (s3_prefetch(p, a)) return launch_s3<L1, L2, L3, WL, false, MODE_LAST, SRC_BUF, true>(p, a, st);
        return dispatch_src<MODE_LAST>(a.src_kind, [&](auto S) {
            return launch_s3<L1, L2, L3, WL, false, MODE_LAST, decltype(S)::value, false>(p, a, st);
        });
    }
    return dispatch_mode(p.mode, [&](auto Mc) {
        constexpr int MO = decltype(Mc)::value;
        if constexpr (MO == MODE_LAST) {
            return cudaErrorInvalidValue;
        } else {
            return dispatch_src<MO>(a.src_kind, [&](auto S) {
                return rows ? launch_s3<L1, L2, L3, WR, true, MO, decltype(S)::value, false>(p, a, st)
                            : launch_s3<L1, L2, L3, WC, false, MO, decltype(S)::value, false>(p, a, st);
            });
        }
    });
}

// occupancy of the form a LAST pass reading src_kind launches (the prefetch form
// for the scratch buffer)
template <int L1, int L2, int L3, int WL>
cudaError_t s3_last_occupancy_len(const Pass& p, int src_kind, int* blocks_per_sm) {
    return dispatch_src<MODE_LAST>(src_kind, [&](auto S) {
        constexpr int SK = decltype(S)::value;
        constexpr bool PF = SK == SRC_BUF;
        constexpr size_t smem = s3_smem<L1, L2, L3, WL, MODE_LAST, PF>();
        auto k = pass_smem3<L1, L2, L3, WL, false, MODE_LAST, SK, PF>;
        cudaError_t e = smem_limit_once((const void*)k, smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, s3_threads<MODE_LAST>(), smem);
    });
}

}  // namespace

// this unit's copies of the twiddle tables (static per translation unit)
cudaError_t upload_twiddles_smem3() { return upload_twiddles(); }

bool smem3_supports(int L) { return L == 2048 || L == 4096; }

int smem3_lines(int L, int mode, int64_t inner) {
    const bool rows = mode != MODE_LAST && inner == 1;
    if (L == 2048) return rows ? 4 : mode == MODE_LAST ? 4 : 8;
    return rows ? 2 : mode == MODE_LAST ? 2 : 4;
}

cudaError_t launch_smem3(const Pass& p, const PassArgs& a, cudaStream_t st) {
    switch (p.L) {
        case 2048: return launch_s3_len<16, 16, 8, 8, 4, 4>(p, a, st);
        case 4096: return launch_s3_len<16, 16, 16, 4, 2, 2>(p, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t smem3_last_occupancy(const Pass& p, int src_kind, int* blocks_per_sm) {
    switch (p.L) {
        case 2048: return s3_last_occupancy_len<16, 16, 8, 4>(p, src_kind, blocks_per_sm);
        case 4096: return s3_last_occupancy_len<16, 16, 16, 2>(p, src_kind, blocks_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace omni
