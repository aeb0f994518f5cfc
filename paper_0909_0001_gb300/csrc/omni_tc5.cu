// omni_tc5.cu -- stage B of the mixed-precision path on 5th-generation tensor
// cores (tcgen05.mma: A operands and accumulators in tensor memory).
//
// Stage B takes the level-1 spectra Z[b][kA] (b = 8 m4 + m3 indexes the 8x8
// grid of blocks, kA the 32x32 level-1 frequencies, scaled by 1/16) and, for
// every kA, computes the padded 2-D DFT over the level-2 grid (8x8 -> 16x16),
// squares it and sums over the chunk's samples (Sec. II.C's |FFT|^2 summed over
// time; Appendix A step 5).  A CTA owns 16 consecutive kA of one channel and,
// per sample, runs two real GEMMs of M = 128, N = 32, K = 16 on FP16 hi/lo
// operands (three products hi*hi + lo*hi + hi*lo, FP32 accumulation):
//   GEMM 3: rows (kA, m4):  D3 = [Zr | Zi] . V16           (1 row tile)
//   GEMM 4: rows (kA, k3):  D4 = [D3r | D3i]^T . V16       (2 row tiles)
// with V16 = [[Vr, Vi], [-Vi, Vr]], V[m][k] = exp(-2 pi i m k / 16): K rows
// (re m | im m), N columns (re k | im k).
//
// The A operands live in tensor memory: each thread owns one row (one line of
// the transform), splits it into FP16 hi/lo and writes it with tcgen05.st, so
// the MMAs read only the 1 KB B tables from shared memory.  Between the GEMMs
// the D3 rows (lines (kA, m4)) are turned into GEMM 4's rows (lines (kA, k3))
// through a padded FP32 shared-memory buffer (the 2-D DFT's transpose).  The
// samples are software-pipelined: while GEMM 4 of sample t and GEMM 3 of sample
// t+1 run, the threads split and store sample t+2's GEMM-3 operand (double
// buffered) and square sample t-1's GEMM-4 output (double buffered).  |D4|^2
// is summed in registers over the chunk and folded into FP64 once.
//
// Every wait on an MMA completion is bounded; on expiry the CTA sets the
// plan's error word, waits (bounded) for its in-flight MMAs, frees its tensor
// memory and returns.
#include "omni_fft_common.cuh"

#include <cuda_fp16.h>

#include <cmath>
#include <cstring>

namespace omni {
namespace {

constexpr int kT5Tile = 16;            // level-1 frequencies per CTA
constexpr int kT5Threads = 128;        // threads per warpgroup: one per tensor-memory lane
constexpr int kLBO = 144;              // B table: bytes between K-adjacent core matrices
constexpr int kSBO = 272;              // B table: bytes between 8-row groups
constexpr int kBBytes = 4 * kSBO;      // the N = 32, K = 16 B operand
constexpr uint32_t kTmemCols = 256;    // two CTAs per SM
constexpr double kT5Fold = 256.0;      // undoes stage A's 1/16 scale, squared
constexpr float kScale16 = 1.0f / 16.0f;
// tensor-memory columns (256 per CTA, two CTAs per SM)
constexpr int kA3Slots = 4;            // GEMM-3 operands prepared ahead of the MMAs
constexpr uint32_t kColA3 = 0;         // GEMM-3 operand, kA3Slots slots of 16: hi (8) + lo (8)
constexpr uint32_t kColD3 = 64;        // GEMM-3 result, N = 32
constexpr uint32_t kColA4 = 96;        // GEMM-4 operand, two row tiles of 16
constexpr uint32_t kColD4 = 128;       // GEMM-4 result, two row tiles of N = 64
// transpose buffer [kA_l][k3][m4] float2; rows of one kA_l padded by 16 bytes
// so that both the writes (lines (kA, m4)) and the reads (lines (kA, k3)) take
// the minimum number of shared-memory wavefronts
constexpr int kXRow = 16 * 8 * 8 + 16;
constexpr int kXBytes = 16 * kXRow;
// dynamic shared memory: the B tables, the transpose buffer, and padding that
// keeps at most two CTAs on an SM (two x 256 tensor-memory columns)
constexpr size_t kT5Smem = 80 * 1024;
static_assert(2 * kBBytes + kXBytes <= (int)kT5Smem, "stage-B shared memory");

// B operand (V16 real form) hi and lo, already in the shared-memory layout.
__device__ __align__(16) unsigned char g_t5B[2][kBBytes];

__host__ __device__ inline int tile_off(int row, int k) {
    return (row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t sdesc(const void* p) {
    const uint32_t a = smem_u32(p);
    return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)(kLBO >> 4) << 16) |
           ((uint64_t)(kSBO >> 4) << 32) | ((uint64_t)1 << 46);
}

// kind::f16, FP32 accumulate, FP16 A and B, K-major, M = 128, N = 32 or 64
constexpr uint32_t kIdesc32 = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdesc64 = (1u << 4) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

// D[d] (+)= A[a] . B: A from tensor memory (row = lane, K = 16 FP16 in 8
// columns).  Executed by a whole warp in uniform control flow with one elected
// lane issuing: a single divergent thread issuing tcgen05.mma measured ~100
// cycles per MMA on this part, a warp-uniform elected issue ~30.
__device__ __forceinline__ void mma_ta(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile("{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
                 " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
                 :: "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Arrive on bar once the warp's earlier MMAs complete (one elected lane commits).
__device__ __forceinline__ void commit_t5(uint64_t* bar) {
    asm volatile("{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
                 " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n"
                 :: "r"(smem_u32(bar)));
}

constexpr long long kWaitCycles = 4000000000LL;   // ~2 s
constexpr long long kTestWaitCycles = 1000000LL;  // the forced-expiry test hook: ~0.5 ms

// Wait for phase `parity` of bar, giving up after `budget` clock cycles.
__device__ __forceinline__ bool wait_t5(uint64_t* bar, uint32_t parity, long long budget = kWaitCycles) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(bar)), "r"(parity));
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}

__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                   "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                   "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// tcgen05.ld of 16 columns without the wait (tcgen05.wait::ld before use)
__device__ __forceinline__ void ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
                 "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]),
                    "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]),
                    "r"(r[13]), "r"(r[14]), "r"(r[15]));
}

__device__ __forceinline__ uint32_t h2u(__half2 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

// (x0, x1) -> hi = fp16(x), lo = fp16(x - hi), packed with x0 in the low half
// (the even K element of a tensor-memory column).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    hi = h2u(h);
    lo = h2u(__floats2half2_rn(x0 - hf.x, x1 - hf.y));
}

// Eight complex values (one line, K = re 0..7 | im 0..7) -> the 16 columns of a
// tensor-memory A row: hi words 0..7, lo words 8..15.
__device__ __forceinline__ void split_row(const float2 (&z)[8], float s, uint32_t (&r)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        split2(z[2 * q].x * s, z[2 * q + 1].x * s, r[q], r[8 + q]);
        split2(z[2 * q].y * s, z[2 * q + 1].y * s, r[4 + q], r[12 + q]);
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" :: "r"(smem_u32(bar)));
}
// Warpgroup 0's own barrier (id 1, 128 threads), OR-reducing a flag.
__device__ __forceinline__ bool wg0_sync_or(bool v) {
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.b32 q, %1, 0;\n"
                 " barrier.cta.red.or.pred p, 1, 128, q;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(r) : "r"((int)v));
    return r != 0;
}

// Two warpgroups with one tensor-memory lane each per thread (lane = tid % 128).
// Warpgroup 1 prepares the GEMM-3 operands (level-1 spectra split into FP16
// hi/lo) up to kA3Slots samples ahead and squares the GEMM-4 results;
// warpgroup 0 turns D3 into the GEMM-4 operand (the transpose) and its warp 0
// issues every MMA (warp-uniform, one elected lane).  They hand off through
// mbarriers (full: written, empty: consumed).  GEMM 3 of sample t+1 is issued
// before the transpose of sample t, so it runs while warpgroup 0 works.
// GEMM 3 is three N = 32 products into one accumulator; GEMM 4 is per row tile
// one N = 64 product of the hi operand with [V16 hi | V16 lo] (the B tables
// are stored back to back, so the pair is one N = 64 operand) plus one N = 32
// product of the lo operand with V16 hi, and the squarer adds the two halves.
__global__ void __launch_bounds__(2 * kT5Threads, 2) tc5_stage_b(Pass p, PassArgs a) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    unsigned char* bh = dsm;               // V16 hi (N = 32); with bl after it, [hi | lo] (N = 64)
    unsigned char* bl = dsm + kBBytes;     // V16 lo
    unsigned char* xbuf = dsm + 2 * kBBytes;
    __shared__ __align__(8) uint64_t a3_full[kA3Slots], a3_empty[kA3Slots], d3_full, d4_full, d4_empty;
    __shared__ __align__(8) uint64_t drain, never_bar;  // never_bar: test hook, nothing arrives
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int wg = tid >> 7, ltid = tid & 127;
    const int64_t tiles = p.inner / kT5Tile;
    const int64_t cc = blockIdx.x / tiles;
    const int64_t kA0 = (blockIdx.x - cc * tiles) * kT5Tile;
    const int64_t s0 = cc * a.tc;
    const int tc = a.tc;
    const long long budget = a.force_expire ? kTestWaitCycles : kWaitCycles;

    for (int i = tid; i < 2 * kBBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(bh)[i] = reinterpret_cast<const uint4*>(&g_t5B[0][0])[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < kA3Slots; ++i) {
            mbar_init(&a3_full[i], kT5Threads);
            mbar_init(&a3_empty[i], 1);
        }
        mbar_init(&d3_full, 1);
        mbar_init(&d4_full, 1);
        mbar_init(&d4_empty, kT5Threads);
        mbar_init(&drain, 1);
        mbar_init(&never_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t row = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this thread's lane
    // GEMM-3 line of this thread's lane: (kA_l, m4), a half-warp holding two m4
    // x eight kA_l so that its transpose stores hit 16 distinct bank pairs;
    // GEMM-4 lines: (kA_l, k3) = (ltid % 16, 8 j + ltid / 16), j = 0, 1
    const int h16 = ltid >> 4;
    const int a_kl = (ltid & 7) + 8 * (h16 & 1), a_m4 = 2 * (h16 >> 1) + ((ltid >> 3) & 1);
    const int kl = ltid & 15, hi4 = ltid >> 4;
    bool aborted = false;

    if (wg == 1 && tc > 0) {
        // ---- warpgroup 1: GEMM-3 operands in (ahead), |GEMM-4|^2 out
        // GEMM-3 line (kA_l, m4): Z[8 m4 + m3][kA], m3 = 0..7 (a warp reads two
        // 128-byte runs per m3)
        const float in_scale = p.unscaled_in ? kScale16 : 1.0f;
        const float2* zline = reinterpret_cast<const float2*>(a.src) + kA0 + a_kl + (int64_t)(8 * a_m4) * p.inner;
        float2 pre[8];
        auto fetch = [&](int64_t s) {
            const float2* b = zline + src_base(a, s);
#pragma unroll
            for (int m3 = 0; m3 < 8; ++m3) pre[m3] = __ldg(b + (int64_t)m3 * p.inner);
        };
        // operand of sample u (its voltages in pre) into slot u % kA3Slots; the
        // next sample's spectra are loaded meanwhile
        auto produce = [&](int u) {
            const int sl = u % kA3Slots;
            // warp-uniform verdicts: the tcgen05.st below is .sync.aligned
            if (u >= kA3Slots &&
                !__all_sync(0xffffffffu, wait_t5(&a3_empty[sl], (u / kA3Slots - 1) & 1, budget)))
                return false;
            uint32_t r[16];
            split_row(pre, in_scale, r);
            if (u + 1 < tc) fetch(s0 + u + 1);
            st16(row + kColA3 + 16 * sl, r);
            asm volatile("tcgen05.wait::st.sync.aligned;");
            tc_before_sync();
            mbar_arrive(&a3_full[sl]);
            return true;
        };
        float acc[2][16];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[j][k] = 0.f;
        auto square = [&](int t) {  // |D4|^2 of sample t, then release D4
            if (!__all_sync(0xffffffffu, wait_t5(&d4_full, t & 1, budget))) return false;
            tc_after_sync();
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint32_t v[2][16], w[2][16];  // [re, im] of (A_hi + A_lo) . V hi and A_hi . V lo
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    ld16_async(row + kColD4 + 64 * j + 16 * part, v[part]);
                    ld16_async(row + kColD4 + 64 * j + 32 + 16 * part, w[part]);
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int k4 = 0; k4 < 16; ++k4) {
                    const float re = __uint_as_float(v[0][k4]) + __uint_as_float(w[0][k4]);
                    const float im = __uint_as_float(v[1][k4]) + __uint_as_float(w[1][k4]);
                    acc[j][k4] = fmaf(re, re, fmaf(im, im, acc[j][k4]));
                }
            }
            tc_before_sync();
            mbar_arrive(&d4_empty);
            return true;
        };
        fetch(s0);
        for (int u = 0; u < tc && u < kA3Slots && !aborted; ++u)
            if (!produce(u)) aborted = true;
        for (int t = 0; t < tc && !aborted; ++t) {
            if (!square(t)) aborted = true;
            else if (t + kA3Slots < tc && !produce(t + kA3Slots)) aborted = true;
        }
        if (aborted) {
            atomicExch(a.err, 1);
        } else {
            // fold: lines (kA_l, k3 = 8 j + ltid / 16); P row 16 k4 + k3, a warp
            // writes two 128-byte runs of kA per (j, k4)
            double* P = a.P + (a.c0 + cc) * a.P_stride + kA0 + kl;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int k3 = 8 * j + hi4;
#pragma unroll
                for (int k4 = 0; k4 < 16; ++k4)
                    P[(int64_t)(16 * k4 + k3) * p.inner] += kT5Fold * (double)acc[j][k4];
            }
        }
    } else if (wg == 0 && tc > 0) {
        // ---- warpgroup 0: D3 -> transpose -> GEMM-4 operand; warp 0 issues the MMAs
        const uint64_t dbh = sdesc(bh), dbl = sdesc(bl);
        const bool issuer = warp == 0;
        auto issue_gemm3 = [&](int u) {
            const int sl = u % kA3Slots;
            const uint32_t d = tmem + kColD3, ah = tmem + kColA3 + 16 * sl, al = ah + 8;
            mma_ta(d, ah, dbh, kIdesc32, 0);
            mma_ta(d, al, dbh, kIdesc32, 1);
            mma_ta(d, ah, dbl, kIdesc32, 1);
            commit_t5(&a3_empty[sl]);
            commit_t5(&d3_full);
        };
        bool bad = false;  // warp 0: a wait before an MMA issue expired
        if (issuer) {
            bad = !__all_sync(0xffffffffu, wait_t5(&a3_full[0], 0, budget));
            if (!bad) {
                tc_after_sync();
                issue_gemm3(0);
            }
        }
        aborted = wg0_sync_or(bad);
        float2* xw = reinterpret_cast<float2*>(xbuf + a_kl * kXRow) + a_m4;
        for (int t = 0; t < tc && !aborted; ++t) {
            // D3 of sample t
            const bool ok = (a.force_expire && t == 0) ? wait_t5(&never_bar, 0, kTestWaitCycles)
                                                       : wait_t5(&d3_full, t & 1, budget);
            if (wg0_sync_or(!ok || bad)) {
                aborted = true;
                break;
            }
            tc_after_sync();
            float v[32];
            ld32(row + kColD3, v);
            // transpose through shared memory: D3 rows (kA_l, m4) -> GEMM-4 rows (kA_l, k3)
#pragma unroll
            for (int k3 = 0; k3 < 16; ++k3) xw[8 * k3] = make_float2(v[k3], v[16 + k3]);
            tc_before_sync();
            // every D3 row read (GEMM 3 of sample t+1 may overwrite it) and every
            // transpose row written
            asm volatile("barrier.cta.sync 1, 128;");
            if (issuer && t + 1 < tc) {
                tc_after_sync();
                bad = !__all_sync(0xffffffffu,
                                  wait_t5(&a3_full[(t + 1) % kA3Slots], ((t + 1) / kA3Slots) & 1, budget));
                if (!bad) {
                    tc_after_sync();
                    issue_gemm3(t + 1);
                }
            }
            uint32_t r[2][16];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float4* xr = reinterpret_cast<const float4*>(xbuf + kl * kXRow + (8 * j + hi4) * 64);
                float2 z[8];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 f = xr[q];
                    z[2 * q] = make_float2(f.x, f.y);
                    z[2 * q + 1] = make_float2(f.z, f.w);
                }
                split_row(z, 1.0f, r[j]);
            }
            // GEMM 4 of sample t-1 has read A4 (its completion also means D4 is full)
            const bool ok4 = t == 0 || wait_t5(&d4_full, (t - 1) & 1, budget);
            if (wg0_sync_or(!ok4)) {
                aborted = true;
                break;
            }
            tc_after_sync();
            st16(row + kColA4, r[0]);
            st16(row + kColA4 + 16, r[1]);
            asm volatile("tcgen05.wait::st.sync.aligned;");
            tc_before_sync();
            // every A4 row written and every transpose read done: GEMM 4 of sample t
            // once the squarer has read D4 of sample t-1
            if (wg0_sync_or(bad)) {
                aborted = true;
                break;
            }
            if (issuer) {
                tc_after_sync();
                if (t >= 1) bad = !__all_sync(0xffffffffu, wait_t5(&d4_empty, (t - 1) & 1, budget));
                if (!bad) {
                    tc_after_sync();
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const uint32_t d = tmem + kColD4 + 64 * j;
                        const uint32_t ah = tmem + kColA4 + 16 * j, al = ah + 8;
                        mma_ta(d, ah, dbh, kIdesc64, 0);   // A_hi . [V hi | V lo]
                        mma_ta(d, al, dbh, kIdesc32, 1);   // + A_lo . V hi
                    }
                    commit_t5(&d4_full);
                }
            }
        }
        if (!aborted && wg0_sync_or(bad)) aborted = true;
        if (aborted && ltid == 0) atomicExch(a.err, 1);
    }
    // every MMA this CTA issued has completed before its tensor memory is freed
    __syncthreads();
    if (warp == 0 && tc > 0) {
        tc_after_sync();
        commit_t5(&drain);
        if (!__all_sync(0xffffffffu, wait_t5(&drain, 0, kWaitCycles)) && tid == 0) atomicExch(a.err, 1);
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
}

double v16_real(int row, int col) {
    // [[Vr, Vi], [-Vi, Vr]], V[m][k] = exp(-2 pi i m k / 16); rows (re m | im m), cols (re k | im k)
    const int m = row % 8, k = col % 16;
    const double ang = -6.283185307179586476925286766559 * (double)m * k / 16.0;
    const bool im_row = row >= 8, im_col = col >= 16;
    if (!im_row && !im_col) return std::cos(ang);
    if (!im_row && im_col) return std::sin(ang);
    if (im_row && !im_col) return -std::sin(ang);
    return std::cos(ang);
}

}  // namespace

cudaError_t upload_tc5_tables() {
    static unsigned char B[2][kBBytes];
    memset(B, 0, sizeof B);
    for (int n = 0; n < 32; ++n)
        for (int k = 0; k < 16; ++k) {
            const double w = v16_real(k, n);
            const __half hi = __float2half_rn((float)w);
            const __half lo = __float2half_rn((float)(w - (double)__half2float(hi)));
            memcpy(&B[0][tile_off(n, k)], &hi, 2);
            memcpy(&B[1][tile_off(n, k)], &lo, 2);
        }
    return cudaMemcpyToSymbol(g_t5B, B, sizeof B);
}

int tc5_stage_b_tile() { return kT5Tile; }

cudaError_t tc5_occupancy(int* blocks_per_sm) {
    cudaError_t e = smem_limit_once((const void*)tc5_stage_b, kT5Smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tc5_stage_b, 2 * kT5Threads, kT5Smem);
    if (e == cudaSuccess && *blocks_per_sm > 2) *blocks_per_sm = 2;  // tensor memory: 2 x 256 columns
    return e;
}

cudaError_t launch_tc5(const Pass& p, const PassArgs& a, cudaStream_t st) {
    if (a.src_kind != SRC_BUF || p.inner % kT5Tile || !a.err) return cudaErrorInvalidValue;
    const int64_t blocks = a.S * (p.inner / kT5Tile);
    if (blocks <= 0 || a.tc <= 0) return cudaSuccess;
    cudaError_t e = smem_limit_once((const void*)tc5_stage_b, kT5Smem);
    if (e != cudaSuccess) return e;
    tc5_stage_b<<<(unsigned)blocks, 2 * kT5Threads, kT5Smem, st>>>(p, a);
    return cudaGetLastError();
}

}  // namespace omni
