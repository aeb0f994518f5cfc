// omni_xspec5.cu -- tile hybrid (Sec. III) between-tile product on 5th-generation
// tensor cores: the cross-spectra of every tile pair, summed over time, as one
// GEMM per tile frequency with the samples as the contraction axis.
//
// For a tile frequency k let x_t = [Re Y_0..Y_{n-1}(k) | Im Y_0..Y_{n-1}(k)]
// (n <= 64 tiles, padded with zeros to 128 components) be sample t's synthesized
// beams.  Then G = sum_t x_t x_t^T (128 x 128, real) holds every cross-spectrum
//   S_ij(k) = sum_t Y_i(k) conj Y_j(k) = (G[i][j] + G[64+i][64+j]) + i (G[64+i][j] - G[i][64+j]),
// so the (N/M)^2 term of Sec. III is a real GEMM D[m][n] = sum_t X[m][t] X[n][t]
// with M = N = 128 and K = the chunk's samples, accumulated in tensor memory.
// X is split into FP16 hi + lo and each group of 16 samples adds three
// products, hi.hi^T + hi.lo^T + lo.hi^T (about 22 bits, FP32 accumulation), or
// (BF16) into h + m + l with six products, hh + hm + mh + hl + lh + mm (about 24
// bits; BF16 has FP32's exponent range, so no scaling).
// FP16 scaling: the spectra are multiplied by a power of two 2^-e before the
// split so that |Y| 2^-e <= 2^12 (|Y| <= antennas per block x max|x| x sqrt 2):
// e fixed from the block size for int8 voltages, or per channel from the
// chunk's measured max |x| for float voltages; the FP64 fold multiplies by
// 2^(2e) (and by 256 more when the level-1 pass already scaled by 1/16).
//
// CTA = (channel of the chunk, 4 consecutive frequencies); 512 tensor-memory
// columns hold the 4 accumulators, one CTA per SM.  Warp 9 brings each step's
// raw spectra (16 samples x every tile x the 4 frequencies, FP32) into a
// shared-memory ring with one tensor-map box.  Warps 0-7 split them into FP16
// hi/lo and write the K-major operand tiles of a stage.  Warp 8 issues the MMAs
// (warp-uniform, one elected lane) once a stage is full and releases it through
// an MMA-completion barrier.  At the end warps 0-7 combine the four 64 x 64
// blocks of each G into Re S and Im S in shared memory and fold them into the
// FP64 accumulator.  EPI_PAIRS adds every S_ij (layout [k][i][j], so that a
// CTA's update is one contiguous run; launch_xspec5_transpose turns it into
// the [i][j][k] layout of the inverse passes once per integration).  EPI_LAGS
// first sums S_ij over the block pairs of each grid offset, one grid axis at a
// time.  Every wait is bounded; on expiry the CTA sets the plan's error word,
// waits (bounded) for its MMAs and its copies, frees its tensor memory and
// returns.
#include "omni_fft_common.cuh"

#include <cuda.h>            // CUtensorMap; the encoder is fetched from the driver at run time
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

namespace omni {
namespace {

constexpr int kXF = 4;            // frequencies per CTA (32-byte load runs)
constexpr int kXT = 64;           // most tiles (2 x 64 = 128 GEMM rows)
constexpr int kXThreads = 320;    // warps 0-7 convert / epilogue, warp 8 MMA issue, warp 9 TMA
constexpr int kXProducers = 256;
constexpr int kLBO = 128;         // bytes between K-adjacent core matrices (dense, 128-byte aligned)
constexpr int kSBO = 256;         // bytes between 8-row groups
constexpr int kTileBytes = 16 * kSBO;                 // 128 rows x 16 samples, 16-bit
// operand stages: FP16 three of hi, lo per frequency; BF16 two of h, m, l
constexpr int kStageRing = 3 * kXF * 2 * kTileBytes;  // 96 KB either way
template <int PREC> struct Prec {
    static constexpr int parts = PREC ? 3 : 2;
    static constexpr int stages = PREC ? 2 : 3;
    static constexpr int stage_bytes = kXF * parts * kTileBytes;
    static_assert(stages * stage_bytes == kStageRing, "operand ring size");
};
constexpr int kXStagesMax = 3;
// raw spectra brought in by the tensor-memory-access unit, kXRaw steps in
// flight: per step one box of the spectra [sample][tile][K], 16 samples x 64
// tiles x 4 frequencies x (re, im) FP32 (32-byte rows), landing as
// [sample][tile][4 frequencies]
constexpr int kXRaw = 3;
constexpr int kRawBytes = 16 * 2 * 64 * 16;
// epilogue staging in the (then idle) stage and raw buffers: per frequency the
// real and imaginary 64 x 64 cross-spectrum matrices, and the partial lag sums
constexpr int kEp = 68;                               // floats per row (conflict-free 16-byte rows)
constexpr int kEpMat = 64 * kEp;                      // floats per matrix
constexpr int kMaxU = 960;                            // partial sums per frequency (8 x 8 grid: 8 x 8 x 15)
constexpr int kMaxQ2 = 225;                           // coarse lags of at most 64 blocks (8 x 8: 15 x 15)
static_assert(kXF * 2 * kEpMat * 4 + kXF * (kMaxU + kMaxQ2) * 8 <= kStageRing + kXRaw * kRawBytes,
              "epilogue staging fits the pipeline buffers");
// more than half of an SM's shared memory (one CTA per SM, so that two CTAs
// never ask for 512 tensor-memory columns on the same SM)
constexpr size_t kXSmem = (size_t)kStageRing + (size_t)kXRaw * kRawBytes + 1024;
static_assert(kXSmem > 114 * 1024 && kXSmem <= 227 * 1024, "one CTA per SM");
constexpr uint32_t kTmemCols = 512;
constexpr int kXScaleTarget = 12;  // FP16: |Y| 2^-e <= 2^12
// kind::f16, FP32 accumulate, K-major, M = 128, N = 128; A and B FP16 or (bits 7, 10) BF16
constexpr uint32_t kIdesc128 = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdesc128Bf16 = kIdesc128 | (1u << 7) | (1u << 10);
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s
constexpr long long kTestWaitCycles = 1000000LL;  // the forced-expiry test hook: ~0.5 ms

__host__ __device__ inline int tile_off(int row, int k) {
    return (row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t sdesc(const void* p) {
    const uint32_t a = smem_u32(p);
    return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)(kLBO >> 4) << 16) |
           ((uint64_t)(kSBO >> 4) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, int acc, uint32_t idesc) {
    asm volatile("{\n .reg .pred p, e;\n setp.ne.b32 p, %3, 0;\n elect.sync _|e, 0xffffffff;\n"
                 " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(acc), "r"(idesc));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
                 " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n"
                 :: "r"(smem_u32(bar)));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" :: "r"(smem_u32(bar)));
}
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, long long budget = kWaitCycles) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(bar)), "r"(parity));
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}
// 64 consecutive columns of the warp's 32 lanes: two loads, one wait
__device__ __forceinline__ void ld64(uint32_t taddr, float (&v)[64]) {
    uint32_t r[64];
#pragma unroll
    for (int half = 0; half < 2; ++half)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                     "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                     "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                     : "=r"(r[32 * half + 0]), "=r"(r[32 * half + 1]), "=r"(r[32 * half + 2]),
                       "=r"(r[32 * half + 3]), "=r"(r[32 * half + 4]), "=r"(r[32 * half + 5]),
                       "=r"(r[32 * half + 6]), "=r"(r[32 * half + 7]), "=r"(r[32 * half + 8]),
                       "=r"(r[32 * half + 9]), "=r"(r[32 * half + 10]), "=r"(r[32 * half + 11]),
                       "=r"(r[32 * half + 12]), "=r"(r[32 * half + 13]), "=r"(r[32 * half + 14]),
                       "=r"(r[32 * half + 15]), "=r"(r[32 * half + 16]), "=r"(r[32 * half + 17]),
                       "=r"(r[32 * half + 18]), "=r"(r[32 * half + 19]), "=r"(r[32 * half + 20]),
                       "=r"(r[32 * half + 21]), "=r"(r[32 * half + 22]), "=r"(r[32 * half + 23]),
                       "=r"(r[32 * half + 24]), "=r"(r[32 * half + 25]), "=r"(r[32 * half + 26]),
                       "=r"(r[32 * half + 27]), "=r"(r[32 * half + 28]), "=r"(r[32 * half + 29]),
                       "=r"(r[32 * half + 30]), "=r"(r[32 * half + 31])
                     : "r"(taddr + 32 * half));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ uint32_t h2u(__half2 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}
// (x0, x1) -> hi = fp16(x), lo = fp16(x - hi), x0 in the low half (the even K element)
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    hi = h2u(h);
    lo = h2u(__floats2half2_rn(x0 - hf.x, x1 - hf.y));
}
__device__ __forceinline__ uint32_t b2u(__nv_bfloat162 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}
// (x0, x1) -> h = bf16(x), m = bf16(x - h), l = bf16(x - h - m)
__device__ __forceinline__ void split3(float x0, float x1, uint32_t& h, uint32_t& m, uint32_t& l) {
    const __nv_bfloat162 bh = __floats2bfloat162_rn(x0, x1);
    const float2 fh = __bfloat1622float2(bh);
    const float r0 = x0 - fh.x, r1 = x1 - fh.y;
    const __nv_bfloat162 bm = __floats2bfloat162_rn(r0, r1);
    const float2 fm = __bfloat1622float2(bm);
    h = b2u(bh);
    m = b2u(bm);
    l = b2u(__floats2bfloat162_rn(r0 - fm.x, r1 - fm.y));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes));
}
// One box of the 3-D tensor map into shared memory, completing on bar.
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z),
                    "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool elect_one() {
    uint32_t e;
    asm volatile("{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}\n" : "=r"(e));
    return e != 0;
}
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }

// EPI_PAIRS: add every S_ij(k) to the accumulator [k][i][j] (tile hybrid).
// EPI_LAGS: the tiles are the n3 x n4 blocks of a 2-level hierarchy (index
// m3 + n3 m4) and only the sums of S_ij over block pairs with equal grid
// offset (d3, d4) = g(i) - g(j) are kept, in the accumulator [k][q2] with
// q2 = (d3 + n3 - 1) + (2 n3 - 1)(d4 + n4 - 1): the coarse level's
// correlation (Eq. ProofEq2 over the level-2 axes) done in lag space.
enum { EPI_PAIRS = 0, EPI_LAGS = 1 };

// The power of two 2^-e applied to channel cc's spectra before the FP16 split, and
// the fold factor that undoes it (and the level-1 pass's own 1/16, if any).
__device__ __forceinline__ int scale_exp(const Pass& p, const PassArgs& a, int64_t cc) {
    if (p.bf16) return 0;
    if (p.scale_n <= 0) return p.scale_e;
    const float m = a.chan_max[cc];
    if (!(m > 0.f)) return 0;
    // smallest e with scale_n m sqrt 2 2^-e <= 2^12 (clamped before the conversion: m may be inf)
    const float v = ceilf(log2f((float)p.scale_n * m * 1.41422f)) - (float)kXScaleTarget;
    return v >= 100.f ? 100 : (v <= -100.f ? -100 : (int)v);
}

template <int EPI, int PREC>
__global__ void __launch_bounds__(kXThreads, 1) xspec5(Pass p, PassArgs a, const __grid_constant__ CUtensorMap tmap) {
    using PR = Prec<PREC>;
    constexpr int kXStages = PR::stages, kStageBytes = PR::stage_bytes, kParts = PR::parts;
    extern __shared__ unsigned char dsm_raw[];
    // operand stages, 1024-byte aligned
    unsigned char* dsm = reinterpret_cast<unsigned char*>(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kXStagesMax], empty[kXStagesMax], done, raw_full[kXRaw], raw_empty[kXRaw];
    __shared__ __align__(8) uint64_t never_bar;  // test hook: nothing arrives on it
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int NT = (int)p.outer;            // tiles
    const int64_t K = p.L;                  // tile frequencies
    const int64_t groups = K / kXF;
    const int64_t cc = blockIdx.x / groups;
    const int64_t k0 = (blockIdx.x - cc * groups) * kXF;
    const int tc = a.tc;
    const int steps = (tc + 15) / 16;
    const int e_scale = scale_exp(p, a, cc);
    // pipeline waits (the test hook shortens them and makes the converters' first
    // one wait for a phase that never comes); the drains keep the full budget, so
    // that no copy or MMA is in flight when the CTA frees its memory
    const long long budget = a.force_expire ? kTestWaitCycles : kWaitCycles;
    const double fold = ldexp(1.0, 2 * e_scale) * (p.unscaled_in || p.bf16 ? 1.0 : 256.0);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < kXStages; ++i) {
            mbar_init(&full[i], kXProducers);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&done, 1);
        mbar_init(&never_bar, 1);
        for (int i = 0; i < kXRaw; ++i) {
            mbar_init(&raw_full[i], 1);
            mbar_init(&raw_empty[i], kXProducers);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp < 8) {
        // ---- converters: warp w takes tiles 16 (w % 4) .. + 15 and half g = w / 4
        // of the step's 16 samples; lane (tile j, frequency pair fp = lane / 16)
        // splits its 8 samples x 2 frequencies into FP16 hi/lo and writes, per
        // frequency and re/im part, one 16-byte core-matrix row (K = 8 samples).  A
        // warp's raw reads are 512 contiguous bytes and its operand writes 4 whole
        // 128-byte runs (no bank conflicts).  Samples past the chunk's end (the box
        // runs on into the next channel) count as zero.
        const int j = 16 * (warp & 3) + (tid & 15), g = warp >> 2, fp = (tid >> 4) & 1;
        const bool live = j < NT;
        const float in_scale = ldexpf(1.0f, -e_scale);
        const unsigned char* raw = dsm + (size_t)kStageRing;
        bool ok = true;
        for (int n = 0; n < steps && ok; ++n) {
            const int st = n % kXStages, rs = n % kXRaw;
            ok = __all_sync(0xffffffffu, (a.force_expire && n == 0) ? wait_bar(&never_bar, 0, budget)
                                                                     : wait_bar(&raw_full[rs], (n / kXRaw) & 1, budget));
            if (!ok) break;
            float4 cur[8];  // samples 8 g + q: (re, im) of frequencies 2 fp, 2 fp + 1
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int ts = 8 * g + q, t = 16 * n + ts;
                cur[q] = (live && t < tc) ? *reinterpret_cast<const float4*>(
                                                raw + (size_t)rs * kRawBytes + ((ts * NT + j) * 2 + fp) * 16)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (n >= kXStages) ok = __all_sync(0xffffffffu, wait_bar(&empty[st], (n / kXStages - 1) & 1, budget));
            if (!ok) break;
            unsigned char* stage = dsm + (size_t)st * kStageBytes;
#pragma unroll
            for (int fl = 0; fl < 2; ++fl) {
                // the frequency's operand tiles: hi, lo (FP16) or h, m, l (BF16)
                unsigned char* t0 = stage + (kParts * (2 * fp + fl)) * kTileBytes;
#pragma unroll
                for (int part = 0; part < 2; ++part) {  // rows j (re) and 64 + j (im)
                    uint32_t h[4], m[4], l[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 a0 = cur[2 * q], a1 = cur[2 * q + 1];
                        const float x0 = (fl == 0 ? (part == 0 ? a0.x : a0.y) : (part == 0 ? a0.z : a0.w)) * in_scale;
                        const float x1 = (fl == 0 ? (part == 0 ? a1.x : a1.y) : (part == 0 ? a1.z : a1.w)) * in_scale;
                        if (PREC) split3(x0, x1, h[q], m[q], l[q]);
                        else split2(x0, x1, h[q], l[q]);
                    }
                    const int off = tile_off(j + 64 * part, 8 * g);
                    *reinterpret_cast<uint4*>(t0 + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    if (PREC) {
                        *reinterpret_cast<uint4*>(t0 + kTileBytes + off) = make_uint4(m[0], m[1], m[2], m[3]);
                        *reinterpret_cast<uint4*>(t0 + 2 * kTileBytes + off) = make_uint4(l[0], l[1], l[2], l[3]);
                    } else {
                        *reinterpret_cast<uint4*>(t0 + kTileBytes + off) = make_uint4(l[0], l[1], l[2], l[3]);
                    }
                }
            }
            // the raw values have been consumed (split and stored) and the operand
            // stores are ordered before the MMAs' and the next box's asynchronous
            // accesses: release both
            asm volatile("fence.proxy.async.shared::cta;");
            mbar_arrive(&full[st]);
            mbar_arrive(&raw_empty[rs]);
        }
        if (!ok) atomicExch(&abort_flag, 1);
    } else if (warp == 9) {
        // ---- warp 9: the raw loads, kXRaw steps ahead: one tensor-map box (x = 8
        // floats from frequency k0, y = every tile, z = 16 samples) per step
        bool ok = true;
        const uint32_t box_bytes = (uint32_t)(16 * NT * 32);
        int issued = 0;
        for (int n = 0; n < steps && ok; ++n) {
            const int rs = n % kXRaw;
            if (n >= kXRaw) ok = __all_sync(0xffffffffu, wait_bar(&raw_empty[rs], (n / kXRaw - 1) & 1, budget));
            if (!ok) break;
            unsigned char* slot = dsm + (size_t)kStageRing + (size_t)rs * kRawBytes;
            if (elect_one()) {
                mbar_expect_tx(&raw_full[rs], box_bytes);
                tma_load3(slot, &tmap, (int)(2 * k0), 0, (int)(cc * tc + 16 * n), &raw_full[rs]);
            }
            __syncwarp();
            issued = n + 1;
        }
        // every box issued has landed before the CTA can leave (bounded; on the
        // normal path the converters already waited for each of them)
        for (int n = issued > kXRaw ? issued - kXRaw : 0; n < issued; ++n)
            if (!wait_bar(&raw_full[n % kXRaw], (n / kXRaw) & 1)) ok = false;
        if (!__all_sync(0xffffffffu, ok)) atomicExch(&abort_flag, 1);
    } else {
        // ---- warp 8: MMA issue, per stage 3 (FP16) or 6 (BF16) products per frequency
        bool ok = true;
        for (int n = 0; n < steps && ok; ++n) {
            const int st = n % kXStages;
            ok = __all_sync(0xffffffffu, wait_bar(&full[st], (n / kXStages) & 1, budget));
            if (!ok) break;
            tc_after_sync();
            unsigned char* stage = dsm + (size_t)st * kStageBytes;
#pragma unroll
            for (int f = 0; f < kXF; ++f) {
                const uint32_t d = tmem + 128 * f;
                if (PREC) {
                    const uint64_t h = sdesc(stage + (3 * f) * kTileBytes);
                    const uint64_t m = sdesc(stage + (3 * f + 1) * kTileBytes);
                    const uint64_t l = sdesc(stage + (3 * f + 2) * kTileBytes);
                    mma_ss(d, h, h, n > 0, kIdesc128Bf16);
                    mma_ss(d, h, m, 1, kIdesc128Bf16);
                    mma_ss(d, m, h, 1, kIdesc128Bf16);
                    mma_ss(d, h, l, 1, kIdesc128Bf16);
                    mma_ss(d, l, h, 1, kIdesc128Bf16);
                    mma_ss(d, m, m, 1, kIdesc128Bf16);
                } else {
                    const uint64_t hi = sdesc(stage + (2 * f) * kTileBytes);
                    const uint64_t lo = sdesc(stage + (2 * f + 1) * kTileBytes);
                    mma_ss(d, hi, hi, n > 0, kIdesc128);   // hi hi^T
                    mma_ss(d, hi, lo, 1, kIdesc128);       // hi lo^T
                    mma_ss(d, lo, hi, 1, kIdesc128);       // lo hi^T
                }
            }
            commit(&empty[st]);
        }
        if (!ok) atomicExch(&abort_flag, 1);
        commit(&done);  // completion of every MMA issued
    }
    __syncthreads();
    bool fine = abort_flag == 0;
    // lag sums: this CTA's 4 Q2 accumulator values (contiguous, k-major), loaded
    // while the last MMAs run
    const int n3 = p.L1, n4 = p.L2, w3 = 2 * n3 - 1, Q2 = w3 * (2 * n4 - 1);
    double2* S = reinterpret_cast<double2*>(a.P + (a.c0 + cc) * a.P_stride);
    double2 pre[4];
    if (EPI == EPI_LAGS && warp < 8 && fine && steps > 0) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int e = tid + kXProducers * m;
            if (e < kXF * Q2) pre[m] = S[k0 * Q2 + e];
        }
    }
    if (warp < 8 && fine && steps > 0) {
        // accumulators complete
        fine = __all_sync(0xffffffffu, wait_bar(&done, 0));
    }
    if (!__syncthreads_and(fine)) {
        if (tid == 256) atomicExch(a.err, 1);
        if (warp == 8) wait_bar(&done, 0);  // its MMAs finish before the memory is freed
    } else if (steps > 0) {
        tc_after_sync();
        // epilogue: S_ij(k) = (G[i][j] + G[64+i][64+j]) + i (G[64+i][j] - G[i][64+j])
        // for the 4 frequencies into shared memory as Re[f][i][j], Im[f][i][j].  Warp
        // (lane quarter q = w % 4, column half h = w / 4) reads rows 32 q + lane of
        // tensor memory; the rows i < 64 store their parts, then the rows 64 + i add
        // theirs (each thread its own row of the two matrices, no races).
        float* mats = reinterpret_cast<float*>(dsm);  // the stage and raw buffers are free now
        const int q = warp & 3, h = (warp >> 2) & 1;
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
        const int i = 32 * (q & 1) + (tid & 31);
        if (warp < 8) {
            // the upper-row warps store frequency f while the lower-row warps add
            // frequency f - 1 (named barrier 1 + f between them)
            const int phase = q >> 1;
            for (int f = 0; f < kXF; ++f) {
                if (phase) asm volatile("bar.sync %0, %1;" :: "r"(1 + f), "r"(kXProducers) : "memory");
                // phase 0: h = 0 -> Re (G[i][c]), h = 1 -> Im (-G[i][64 + c]);
                // phase 1: h = 0 -> Im (+G[64 + i][c]), h = 1 -> Re (+G[64 + i][64 + c])
                float* row = mats + (2 * f + (h ^ phase)) * kEpMat + i * kEp;
                const float sign = (phase == 0 && h == 1) ? -1.f : 1.f;
                float v[64];
                ld64(lane_addr + 128 * f + 64 * h, v);
#pragma unroll
                for (int c = 0; c < 64; c += 4) {
                    float4* d = reinterpret_cast<float4*>(row + c);
                    float4 o = phase ? *d : make_float4(0.f, 0.f, 0.f, 0.f);
                    o.x += sign * v[c];
                    o.y += sign * v[c + 1];
                    o.z += sign * v[c + 2];
                    o.w += sign * v[c + 3];
                    *d = o;
                }
                if (!phase) asm volatile("bar.arrive %0, %1;" :: "r"(1 + f), "r"(kXProducers) : "memory");
            }
        }
        __syncthreads();
        if (EPI == EPI_PAIRS && warp < 8) {
            // thread (i parity, j) adds S_ij(k) to the accumulator [k][i][j]: consecutive
            // threads, consecutive j, so a warp's accesses are 512 contiguous bytes
            const int jj = tid & 63, ih = tid >> 6;  // i = ih, ih + 4, ...
            if (jj < NT) {
                for (int f = 0; f < kXF; ++f) {
                    const float* re = mats + (2 * f) * kEpMat;
                    const float* im = re + kEpMat;
                    double2* col = S + ((k0 + f) * (int64_t)NT) * NT + jj;
                    constexpr int kIB = 16;  // accumulator loads in flight per thread
                    for (int i0 = ih; i0 < NT; i0 += 4 * kIB) {
                        double2 cur[kIB];
#pragma unroll
                        for (int u = 0; u < kIB; ++u) {
                            const int ii = i0 + 4 * u;
                            if (ii < NT) cur[u] = col[(int64_t)ii * NT];
                        }
#pragma unroll
                        for (int u = 0; u < kIB; ++u) {
                            const int ii = i0 + 4 * u;
                            if (ii < NT) {
                                cur[u].x += fold * (double)re[ii * kEp + jj];
                                cur[u].y += fold * (double)im[ii * kEp + jj];
                                col[(int64_t)ii * NT] = cur[u];
                            }
                        }
                    }
                }
            }
        }
        if (EPI == EPI_LAGS) {
            // the sum over block pairs of equal grid offset, one axis at a time: with
            // block i = a_A s_A + a_B s_B (A the longer grid axis),
            //   U[f][a_B][b_B][d_A] = sum_{a_A} S_{(a_A, a_B), (a_A - d_A, b_B)}
            //   R[f][d_A][d_B]      = sum_{a_B} U[f][a_B][a_B - d_B][d_A]
            // (at most max(n3, n4) terms per output instead of n3 n4)
            const bool a3 = n3 >= n4;
            const int na = a3 ? n3 : n4, nb = a3 ? n4 : n3, sA = a3 ? 1 : n3, sB = a3 ? n3 : 1;
            const int wA = 2 * na - 1, wB = 2 * nb - 1, nU = nb * nb * wA;
            float2* U = reinterpret_cast<float2*>(mats + kXF * 2 * kEpMat);
            float2* R = U + kXF * nU;
            const int lane = tid & 31;
            // stage 1, warp task (f, a_B, 8 offsets d_A, 4 blocks b_B): every lane of
            // the warp at the same a_A, so its reads are 32 distinct words of one row;
            // the 10 warps take consecutive runs of tasks, 8 a_A per batch of loads
            {
                const int ndg = (wA + 7) / 8, nbg = (nb + 3) / 4, ntask = kXF * nb * nbg * ndg;
                const int ld = lane & 7, lb = lane >> 3;
                const int t0 = warp * ntask / 10, t1 = (warp + 1) * ntask / 10;
                int dg = t0 % ndg, bg = (t0 / ndg) % nbg, aB = (t0 / (ndg * nbg)) % nb, f = t0 / (ndg * nbg * nb);
                for (int task = t0; task < t1; ++task) {
                    const int dAi = 8 * dg + ld, bB = 4 * bg + lb, dA = dAi - (na - 1);
                    const bool live = dAi < wA && bB < nb;
                    const float* re = mats + (2 * f) * kEpMat + (aB * sB) * kEp + bB * sB - dA * sA;
                    const float* im = re + kEpMat;
                    float sr = 0.f, si = 0.f;
                    for (int a0 = 0; a0 < na; a0 += 8) {
                        float vr[8], vi[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int aA = a0 + u;
                            const bool ok = live && aA < na && aA - dA >= 0 && aA - dA < na;
                            vr[u] = ok ? re[aA * sA * (kEp + 1)] : 0.f;
                            vi[u] = ok ? im[aA * sA * (kEp + 1)] : 0.f;
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            sr += vr[u];
                            si += vi[u];
                        }
                    }
                    if (live) U[((f * nb + aB) * nb + bB) * wA + dAi] = make_float2(sr, si);
                    if (++dg == ndg) {
                        dg = 0;
                        if (++bg == nbg) {
                            bg = 0;
                            if (++aB == nb) aB = 0, ++f;
                        }
                    }
                }
            }
            __syncthreads();
            // stage 2, warp task (f, d_B, 32 offsets d_A)
            {
                const int ndg = (wA + 31) / 32, ntask = kXF * wB * ndg;
                const int t0 = warp * ntask / 10, t1 = (warp + 1) * ntask / 10;
                int dg = t0 % ndg, dBi = (t0 / ndg) % wB, f = t0 / (ndg * wB);
                for (int task = t0; task < t1; ++task) {
                    const int dAi = 32 * dg + lane, dB = dBi - (nb - 1);
                    if (dAi < wA) {
                        const float2* Uf = U + f * nU + dAi;
                        float sr = 0.f, si = 0.f;
                        for (int a0 = 0; a0 < nb; a0 += 8) {
                            float2 v[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const int aB = a0 + u;
                                const bool ok = aB < nb && aB - dB >= 0 && aB - dB < nb;
                                v[u] = ok ? Uf[(aB * nb + aB - dB) * wA] : make_float2(0.f, 0.f);
                            }
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                sr += v[u].x;
                                si += v[u].y;
                            }
                        }
                        R[f * Q2 + (a3 ? dAi + w3 * dBi : dBi + w3 * dAi)] = make_float2(sr, si);
                    }
                    if (++dg == ndg) {
                        dg = 0;
                        if (++dBi == wB) dBi = 0, ++f;
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int e = tid + kXProducers * m;
                if (warp < 8 && e < kXF * Q2) {
                    double2 r = pre[m];
                    r.x += fold * (double)R[e].x;
                    r.y += fold * (double)R[e].y;
                    S[k0 * Q2 + e] = r;
                }
            }
        }
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
}

// [K][NP] -> [NP][K] complex FP64 per channel (32 x 32 tiles through shared
// memory), the layout the inverse passes read; NP = tile pairs or coarse lags.
__global__ void __launch_bounds__(256) xspec5_transpose(const double2* __restrict__ src, int64_t src_stride,
                                                        double2* __restrict__ dst, int64_t K, int64_t NP) {
    __shared__ double2 tile[32][33];
    const int64_t c = blockIdx.z;
    const int64_t p0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
    const double2* s = src + c * src_stride;
    double2* d = dst + c * K * NP;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < 32; r += 8) {
        const int64_t k = k0 + r, pp = p0 + tx;
        if (k < K && pp < NP) tile[r][tx] = s[k * NP + pp];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t pp = p0 + r, k = k0 + tx;
        if (k < K && pp < NP) d[pp * K + k] = tile[tx][r];
    }
}

}  // namespace

cudaError_t launch_xspec5_transpose(const double* P, int64_t P_stride, int64_t cv, int64_t K, int64_t NP,
                                    float2* dst, cudaStream_t st) {
    if (cv <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((NP + 31) / 32), (unsigned)((K + 31) / 32), (unsigned)cv);
    xspec5_transpose<<<grid, 256, 0, st>>>(reinterpret_cast<const double2*>(P), P_stride / 2,
                                          reinterpret_cast<double2*>(dst), K, NP);
    return cudaGetLastError();
}

bool xspec5_supports(int64_t n_tiles, int64_t K) { return n_tiles >= 1 && n_tiles <= kXT && K % kXF == 0; }

int64_t xspec5_ctas_per_channel(const Pass& p) { return p.L / kXF; }

cudaError_t xspec5_occupancy(int* blocks_per_sm) {
    cudaError_t e = smem_limit_once((const void*)xspec5<EPI_PAIRS, 0>, kXSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, xspec5<EPI_PAIRS, 0>, kXThreads, kXSmem);
    if (e == cudaSuccess && *blocks_per_sm > 1) *blocks_per_sm = 1;  // 512 tensor-memory columns
    return e;
}

// 3-D map of the spectra [samples][tiles][2K floats]; a box (x: the 8 floats of
// the CTA's 4 frequencies, y: every tile, z: 16 samples) lands as [z][y][x].
static cudaError_t encode_map(const PassArgs& a, const Pass& p, CUtensorMap* map) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t K = (cuuint64_t)p.L, NT = (cuuint64_t)p.outer;
    const cuuint64_t dims[3] = {2 * K, NT, (cuuint64_t)(a.S * a.tc)};
    const cuuint64_t strides[2] = {K * 8, NT * K * 8};
    const cuuint32_t box[3] = {8, (cuuint32_t)NT, 16};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(a.src), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_xspec5(const Pass& p, const PassArgs& a, cudaStream_t st) {
    if (a.src_kind != SRC_BUF || !xspec5_supports(p.outer, p.L) || !a.err) return cudaErrorInvalidValue;
    const int64_t blocks = a.S * xspec5_ctas_per_channel(p);
    if (blocks <= 0 || a.tc <= 0) return cudaSuccess;
    // the TMA unit wants a 16-byte aligned base and row pitches
    if (reinterpret_cast<uintptr_t>(a.src) % 16 || (p.L * 8) % 16) return cudaErrorInvalidValue;
    CUtensorMap map;
    const cudaError_t me = encode_map(a, p, &map);
    if (me != cudaSuccess) return me;
    if (p.scale_n > 0 && !p.bf16 && !a.chan_max) return cudaErrorInvalidValue;
    void (*kern)(Pass, PassArgs, const CUtensorMap) = nullptr;
    if (p.kind == KIND_COV5) {
        if (p.L1 < 1 || p.L2 < 1 || p.L1 * p.L2 != p.outer) return cudaErrorInvalidValue;
        const int na = std::max(p.L1, p.L2), nb = std::min(p.L1, p.L2);
        if (nb * nb * (2 * na - 1) > kMaxU || (2 * p.L1 - 1) * (2 * p.L2 - 1) > kMaxQ2) return cudaErrorInvalidValue;
        kern = p.bf16 ? xspec5<EPI_LAGS, 1> : xspec5<EPI_LAGS, 0>;
    } else {
        kern = p.bf16 ? xspec5<EPI_PAIRS, 1> : xspec5<EPI_PAIRS, 0>;
    }
    cudaError_t e = smem_limit_once((const void*)kern, kXSmem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, kXThreads, kXSmem, st>>>(p, a, map);
    return cudaGetLastError();
}

namespace {
// one CTA per (channel, slice of its samples); block max in shared memory, then
// one atomicMax per CTA on the float's bits (non-negative floats order as integers)
template <int SRC>
__global__ void __launch_bounds__(256) chan_absmax(const void* volts, int64_t vc0, int64_t T, int64_t t0, int64_t N,
                                                   int64_t tc, float* out) {
    __shared__ float red[8];
    const int64_t c = blockIdx.y;
    const int64_t per = tc * N;  // complex values of the channel in the chunk
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / N, n = i - t * N;
        const int64_t e = ((vc0 + c) * T + t0 + t) * N + n;
        float re, im;
        if (SRC == SRC_CI8) {
            const char2 v = reinterpret_cast<const char2*>(volts)[e];
            re = (float)v.x;
            im = (float)v.y;
        } else {
            const float2 v = reinterpret_cast<const float2*>(volts)[e];
            re = v.x;
            im = v.y;
        }
        m = fmaxf(m, fmaxf(fabsf(re), fabsf(im)));
    }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < 8 ? red[threadIdx.x] : 0.f;
        for (int o = 4; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        // NaN-free by construction of fmaxf; +inf orders above every finite value
        if (threadIdx.x == 0) atomicMax(reinterpret_cast<int*>(out + c), __float_as_int(m));
    }
}
}  // namespace

cudaError_t launch_chan_absmax(const void* volts, int src_kind, int64_t vc0, int64_t T, int64_t t0, int64_t N,
                               int64_t cc, int64_t tc, float* out, cudaStream_t st) {
    if (cc <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)cc * sizeof(float), st);
    if (e != cudaSuccess || tc <= 0 || N <= 0) return e;
    const int64_t per = tc * N;
    const unsigned bx = (unsigned)std::min<int64_t>(64, (per + 255) / 256);
    const dim3 grid(bx, (unsigned)cc);
    if (src_kind == SRC_CI8)
        chan_absmax<SRC_CI8><<<grid, 256, 0, st>>>(volts, vc0, T, t0, N, tc, out);
    else if (src_kind == SRC_CF32)
        chan_absmax<SRC_CF32><<<grid, 256, 0, st>>>(volts, vc0, T, t0, N, tc, out);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace omni
