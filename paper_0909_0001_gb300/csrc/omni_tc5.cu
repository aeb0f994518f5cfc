// omni_tc5.cu -- stage B of the mixed-precision path on 5th-generation tensor
// cores (tcgen05.mma, accumulators in tensor memory).
//
// Stage B takes the level-1 spectra Y[b][kA] (b = 8 m4 + m3 indexes the 8x8
// grid of blocks, kA the 32x32 level-1 frequencies, scaled by 1/16) and, for
// every kA, computes the padded 2-D DFT over the level-2 grid (8x8 -> 16x16),
// squares it and sums over the chunk's samples (Sec. II.C's |FFT|^2 summed over
// time; Appendix A step 5).  A CTA owns 16 consecutive kA and, per sample, runs
// two batched real GEMMs of M = 128, N = 32, K = 16 on FP16 hi/lo operands:
//   GEMM 3: rows (kA, m4):  D2 = [Zr | Zi] . V16        (1 tile  x 3 terms)
//   GEMM 4: rows (kA, k3):  D3 = [D2r | D2i]^T . V16    (2 tiles x 3 terms)
// with V16 = [[Vr, Vi], [-Vi, Vr]], V[m][k] = exp(-2 pi i m k / 16), K rows
// (re m | im m), N columns (re k | im k).  Between the GEMMs the threads read D2
// out of tensor memory, split it into FP16 hi/lo and write it transposed (rows
// (kA, k3), K = m4) into shared memory as GEMM 4's A operand.  |D3|^2 is summed
// in registers over the samples and folded into FP64 once per chunk.
// The samples are software-pipelined: GEMM 3 of sample t+1 is issued together
// with GEMM 4 of sample t, so each sample costs one MMA round trip and one CTA
// barrier; 128 tensor-memory columns per CTA let four CTAs share an SM.
//
// Operands sit in shared memory in the no-swizzle K-major layout: 8-row x
// 16-byte core matrices, K-adjacent core matrices 144 bytes apart (leading
// byte offset), 8-row groups 272 bytes apart (stride byte offset).  The 16-byte
// paddings put the 32 words a warp writes when it transposes D2 into 32
// distinct shared-memory banks.  Every wait
// on an MMA completion is bounded; on expiry the CTA sets the plan's error word,
// frees its tensor memory and returns.
#include "omni_fft_common.cuh"

#include <cuda_fp16.h>

#include <cmath>
#include <cstring>

namespace omni {
namespace {

constexpr int kT5Tile = 16;           // level-1 frequencies per CTA
constexpr int kT5Threads = 128;
constexpr int kLBO = 144;             // bytes between K-adjacent core matrices
constexpr int kSBO = 272;             // bytes between 8-row groups
constexpr int kTileBytes = 16 * kSBO; // one M = 128, K = 16 FP16 operand tile
constexpr int kBBytes = 4 * kSBO;     // the N = 32, K = 16 B operand
constexpr int kTmemCols = 128;        // D2: columns 0..31, D3: two tiles at 32..95
constexpr double kT5Fold = 256.0;     // undoes stage A's 1/16 scale, squared
constexpr int kFoldPitch = 257;       // floats per kA row of the fold staging

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

// kind::f16, FP32 accumulate, FP16 A and B, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_t5(uint32_t d, uint64_t a, uint64_t b, int acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void commit_t5(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
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

__device__ __forceinline__ uint32_t pack_h2(__half lo, __half hi) {
    uint16_t a, b;
    memcpy(&a, &lo, 2);
    memcpy(&b, &hi, 2);
    return (uint32_t)a | ((uint32_t)b << 16);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }

__global__ void __launch_bounds__(kT5Threads, 4) tc5_stage_b(Pass p, PassArgs a) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    unsigned char* a3h = dsm;                      // 1 tile
    unsigned char* a3l = dsm + 1 * kTileBytes;
    unsigned char* a4h = dsm + 2 * kTileBytes;     // 2 tiles
    unsigned char* a4l = dsm + 4 * kTileBytes;
    unsigned char* bh = dsm + 6 * kTileBytes;
    unsigned char* bl = bh + kBBytes;
    float* sfold = reinterpret_cast<float*>(dsm);  // after the last sample
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t never_bar;  // test hook: a barrier nothing arrives on
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tiles = p.inner / kT5Tile;
    const int64_t cc = blockIdx.x / tiles;
    const int64_t kA0 = (blockIdx.x - cc * tiles) * kT5Tile;
    const int64_t s0 = cc * a.tc;
    const int tc = a.tc;

    for (int i = tid; i < 2 * kBBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(bh)[i] = reinterpret_cast<const uint4*>(&g_t5B[0][0])[i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&never_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;  // this warp's tensor-memory lanes
    uint32_t parity = 0;
    bool aborted = false;

    // GEMM 3 input: thread = (kA_l, m4), the 8 values Z[m4][m3] of one kA
    const int kl_in = 4 * warp + (lane >> 3), m4_in = lane & 7;
    float2 pre[8];
    auto fetch = [&](int64_t s) {
        const float2* base = reinterpret_cast<const float2*>(a.src) + src_base(a, s) + kA0 + kl_in;
#pragma unroll
        for (int m3 = 0; m3 < 8; ++m3) pre[m3] = base[(int64_t)(8 * m4_in + m3) * p.inner];
    };
    // A operand of GEMM 3: row 8 kA_l + m4, K = (re m3 | im m3), hi and lo
    auto write_a3 = [&]() {
        const int off = tile_off(8 * kl_in + m4_in, 0);
        uint32_t hr[4], lr[4], hi_[4], li[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 z0 = pre[2 * q], z1 = pre[2 * q + 1];
            const __half h0 = __float2half_rn(z0.x), h1 = __float2half_rn(z1.x);
            const __half g0 = __float2half_rn(z0.y), g1 = __float2half_rn(z1.y);
            hr[q] = pack_h2(h0, h1);
            lr[q] = pack_h2(__float2half_rn(z0.x - __half2float(h0)), __float2half_rn(z1.x - __half2float(h1)));
            hi_[q] = pack_h2(g0, g1);
            li[q] = pack_h2(__float2half_rn(z0.y - __half2float(g0)), __float2half_rn(z1.y - __half2float(g1)));
        }
        *reinterpret_cast<uint4*>(a3h + off) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
        *reinterpret_cast<uint4*>(a3h + off + kLBO) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
        *reinterpret_cast<uint4*>(a3l + off) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
        *reinterpret_cast<uint4*>(a3l + off + kLBO) = make_uint4(li[0], li[1], li[2], li[3]);
    };
    // D2 row (kA_l, m4) of this thread -> GEMM 4's A operand rows (kA_l, k3), K = (re m4 | im m4)
    auto d2_to_a4 = [&]() {
        float v[32];
        ld32(tmem + lane_base, v);
        const int r = 32 * warp + lane;
        const int kl = r >> 3, m4 = r & 7;
        const bool even = (m4 & 1) == 0;
#pragma unroll
        for (int k3 = 0; k3 < 16; ++k3) {
            const float re = v[k3], im = v[16 + k3];
            const float pre_ = __shfl_xor_sync(0xffffffffu, re, 1);
            const float pim = __shfl_xor_sync(0xffffffffu, im, 1);
            // even lanes write the real pair (K = m4, m4+1), odd lanes the imaginary pair
            const float x0 = even ? re : pim, x1 = even ? pre_ : im;
            const int k0 = even ? m4 : 8 + m4 - 1;
            const int R = 16 * kl + k3;
            const int off = (R >> 7) * kTileBytes + tile_off(R & 127, k0);
            const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
            *reinterpret_cast<uint32_t*>(a4h + off) = pack_h2(h0, h1);
            *reinterpret_cast<uint32_t*>(a4l + off) =
                pack_h2(__float2half_rn(x0 - __half2float(h0)), __float2half_rn(x1 - __half2float(h1)));
        }
    };
    auto issue_gemm3 = [&]() {
        const uint64_t dbh = sdesc(bh), dbl = sdesc(bl);
        mma_t5(tmem, sdesc(a3h), dbh, 0);
        mma_t5(tmem, sdesc(a3l), dbh, 1);
        mma_t5(tmem, sdesc(a3h), dbl, 1);
    };
    auto issue_gemm4 = [&]() {
        const uint64_t dbh = sdesc(bh), dbl = sdesc(bl);
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const uint32_t d = tmem + 32 + 32 * m;
            mma_t5(d, sdesc(a4h + m * kTileBytes), dbh, 0);
            mma_t5(d, sdesc(a4l + m * kTileBytes), dbh, 1);
            mma_t5(d, sdesc(a4h + m * kTileBytes), dbl, 1);
        }
    };
    // handshake: threads' shared-memory operands -> MMA issue
    auto to_mma = [&]() {
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
    };
    float acc[2][16];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[j][k] = 0.f;

    // prologue: GEMM 3 of sample 0, A4(0) and A3(1) ready
    fetch(s0);
    write_a3();
    if (tc > 1) fetch(s0 + 1);
    to_mma();
    if (tid == 0) {
        issue_gemm3();
        commit_t5(&mbar);
    }
    {
        // test hook: wait on a barrier that nothing arrives on, with a short budget
        const bool ok = a.force_expire ? wait_t5(&never_bar, 0, kTestWaitCycles)
                                       : wait_t5(&mbar, parity);
        parity ^= 1;
        if (__syncthreads_or(!ok)) aborted = true;
    }
    if (!aborted) {
        tc_after_sync();
        d2_to_a4();
        if (tc > 1) {
            write_a3();
            if (tc > 2) fetch(s0 + 2);
        }
        to_mma();
        for (int t = 0; t < tc; ++t) {
            // GEMM 3 of sample t+1 and GEMM 4 of sample t in flight together
            if (tid == 0) {
                if (t + 1 < tc) issue_gemm3();
                issue_gemm4();
                commit_t5(&mbar);
            }
            const bool ok = wait_t5(&mbar, parity);
            parity ^= 1;
            if (__syncthreads_or(!ok)) { aborted = true; break; }
            tc_after_sync();
#pragma unroll
            for (int j = 0; j < 2; ++j) {  // |D3|^2 of sample t
                float v[32];
                ld32(tmem + lane_base + 32 + 32 * j, v);
#pragma unroll
                for (int k4 = 0; k4 < 16; ++k4)
                    acc[j][k4] = fmaf(v[k4], v[k4], fmaf(v[16 + k4], v[16 + k4], acc[j][k4]));
            }
            if (t + 1 < tc) d2_to_a4();   // A4(t+1)
            if (t + 2 < tc) {             // A3(t+2), next voltages in flight
                write_a3();
                if (t + 3 < tc) fetch(s0 + t + 3);
            }
            to_mma();
        }
    }
    if (aborted) {
        // the MMA that did not complete may still be in flight: wait once more
        // (bounded) before the tensor memory is freed
        if (tid == 0) {
            atomicExch(a.err, 1);
            wait_t5(&mbar, parity ^ 1);
        }
    } else {
        // fold through shared memory so the FP64 updates run along kA
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int R = 128 * j + 32 * warp + lane;  // (kA_l, k3) row
            const int kl = R >> 4, k3 = R & 15;
#pragma unroll
            for (int k4 = 0; k4 < 16; ++k4) sfold[kl * kFoldPitch + k4 * 16 + k3] = acc[j][k4];
        }
        __syncthreads();
        double* P = a.P + (a.c0 + cc) * a.P_stride;
        for (int e = tid; e < 256 * kT5Tile; e += blockDim.x) {
            const int kl = e % kT5Tile, row = e / kT5Tile;  // row = k4 * 16 + k3
            P[(int64_t)row * p.inner + kA0 + kl] += kT5Fold * (double)sfold[kl * kFoldPitch + row];
        }
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
}

constexpr size_t kT5Smem = 6 * kTileBytes + 2 * kBBytes;  // A3 hi/lo, A4 hi/lo (2 tiles), B hi/lo

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

cudaError_t tc5_occupancy(int* blocks_per_sm) {
    cudaError_t e = smem_limit_once((const void*)tc5_stage_b, kT5Smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tc5_stage_b, kT5Threads, kT5Smem);
}

cudaError_t launch_tc5(const Pass& p, const PassArgs& a, cudaStream_t st) {
    if (a.src_kind != SRC_BUF || p.inner % kT5Tile || !a.err) return cudaErrorInvalidValue;
    const int64_t blocks = a.S * (p.inner / kT5Tile);
    if (blocks <= 0) return cudaSuccess;
    cudaError_t e = smem_limit_once((const void*)tc5_stage_b, kT5Smem);
    if (e != cudaSuccess) return e;
    tc5_stage_b<<<(unsigned)blocks, kT5Threads, kT5Smem, st>>>(p, a);
    return cudaGetLastError();
}

}  // namespace omni
