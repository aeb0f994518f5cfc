// omni_internal.h -- types shared by the host orchestration and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace omni {

constexpr int kMaxDims = 16;
constexpr int kTwiddleN = 4096;  // longest padded axis handled by an FFT pass

// Where a pass reads its lines from.
enum SrcKind : int {
    SRC_BUF = 0,   // float2 scratch buffer written by the previous pass
    SRC_CF32 = 1,  // caller voltages, complex float32 [.][T][N]
    SRC_CI8 = 2,   // caller voltages, complex int8   [.][T][N]
    SRC_P64 = 3,   // FP64 |F|^2 accumulator [C][L] (real), inverse passes
    SRC_PC64 = 4   // FP64 complex cross-spectrum accumulator (re, im), tile-hybrid inverse
};

// What a pass does with the transformed lines.
enum PassMode : int {
    MODE_MID = 0,      // forward: write the float2 buffer
    MODE_LAST = 1,     // forward: |F|^2 summed over the chunk's samples, folded into FP64
    MODE_INV_MID = 2,  // inverse: gather the kept lags into the float2 buffer
    MODE_INV_LAST = 3  // inverse: gather, conjugate, scale by 1/L, write complex128
};

// How a pass transforms one line.
enum PassKind : int {
    KIND_REG = 0,    // whole line in one thread's registers (power of two <= 64)
    KIND_SMEM = 1,   // four-step L = L1 * L2 through shared memory (power of two <= 4096)
    KIND_DIRECT = 2, // direct DFT from a twiddle table (any length)
    KIND_LEVEL = 3,  // both axes of one square level (L_a = L_b <= 64) in shared memory
    KIND_TC_A = 4,   // mixed precision, finest level as split-FP16 tensor-core GEMMs
    KIND_TC_B = 5,   // mixed precision, coarse level + |F|^2 as tensor-core GEMMs (LAST, mma.sync)
    KIND_TC5_B = 6,  // the same on 5th-generation tensor cores (tcgen05, tensor memory)
    KIND_XSPEC = 7,  // tile hybrid: cross-spectra of every tile pair summed over samples (LAST)
    KIND_XSPEC5 = 8, // the same as a tcgen05 GEMM per tile frequency over the samples (mixed precision)
    KIND_COV5 = 9,   // 2-level mixed path: block cross-spectra per level-1 frequency (tcgen05 GEMM over
                     // the samples) summed by level-2 grid offset (LAST; L1 x L2 = the level-2 shape)
    KIND_SMEM3 = 10  // forward three-step 16 x 16 x (8 | 16) through shared memory (2048, 4096 points)
};

// One axis transform.  The data of one sample (or channel) is viewed as
// [outer][len][inner] with the transformed axis in the middle: inputs
// [outer][n][inner], outputs [outer][q_out][inner].  A KIND_LEVEL pass
// transforms two adjacent axes (axis, axis+1) of equal length L at once:
// [outer][n][n][inner] -> [outer][L][L][inner].
struct Pass {
    int axis;
    int kind;
    int mode;
    int L;          // transform length (padded axis length)
    int n;          // inputs per line (n_d forward, L_d inverse)
    int q_out;      // outputs kept per line (L_d forward, 2 n_d - 1 inverse)
    int q_shift;    // inverse: output q holds lag q - q_shift, i.e. bin (q - q_shift) mod L
    int L1, L2;     // KIND_SMEM split
    int W;          // KIND_SMEM / KIND_LEVEL: consecutive inner indices per unit
    int grid_cap;   // KIND_LEVEL finest MID: CTAs of the persistent kernel (0 = not used)
    int unscaled_in;  // KIND_TC_B/COV5/XSPEC5: level-1 spectra from the FP32 pass, not pre-scaled by 1/16
    int bf16;         // KIND_COV5/XSPEC5: BF16 operands split three ways (else FP16 split two ways)
    int scale_e;      // KIND_COV5/XSPEC5, FP16: the spectra are multiplied by 2^-scale_e before the split
    int scale_n;      // ... or, when > 0, by a power of two per channel from PassArgs::chan_max
                      //     (scale_n = antennas per block or tile, bounding |Y| by scale_n max|x| sqrt 2)
    int64_t inner, outer;
    const float2* tw;  // KIND_DIRECT: w_L^m = exp(-2 pi i m / L), m < L
};

// Launch-time arguments of one pass.
struct PassArgs {
    const void* src;
    int src_kind;
    int64_t src_stride;  // SRC_BUF/SRC_P64: elements per sample (or channel)
    int64_t vc0;         // voltages: first channel row of the chunk in src
    int64_t T, t0, N;    // voltages: samples per channel row, first sample, antennas
    int tc;              // samples per channel in this chunk
    int64_t S;           // MID/INV: samples (channels) in the launch; LAST: channels
    int64_t c0;          // channel of the first sample in P / V
    float2* dst;
    int64_t dst_stride;  // elements per sample of dst
    double* P;           // LAST / SRC_P64: accumulator
    int64_t P_stride;    // elements per channel of P (= L)
    double2* V;          // INV_LAST output
    int64_t V_stride;    // lags per channel
    double scale;        // INV_LAST: 1/L
    int* err;            // device error word (bounded waits that expired set it to 1)
    int force_expire;    // test hook: make the first bounded wait expire
    double fold_scale;   // FP32 LAST passes: factor on the FP64 fold (0 means 1)
    const float* chan_max;  // per chunk channel: max |re|, |im| of its voltages (KIND_COV5/XSPEC5 with scale_n)
};

// Upload the twiddle tables to the current device (once per device).
cudaError_t init_device_tables();

// Kernel family of an axis pass from its length (register FFT up to 64 points,
// four-step shared-memory FFT up to 4096, direct DFT otherwise).
void choose_kind(Pass& p);

// Launch one pass on stream.
cudaError_t launch_pass(const Pass& p, const PassArgs& a, cudaStream_t stream);

// Resident CTAs per SM of the LAST-mode kernel of a KIND_LEVEL pass.
cudaError_t level_last_occupancy(const Pass& p, int src_kind, int* blocks_per_sm);

// Resident CTAs per SM of the persistent finest-level MID kernel.
cudaError_t level_stream_occupancy(const Pass& p, int src_kind, int* blocks_per_sm);

// Mixed-precision (tensor-core) path: supported lattices, tables, launches.
bool tc_supports(const int32_t* n, int D, int dtype_is_ci8);
cudaError_t upload_tc_tables();
cudaError_t tc_occupancy(int kind, int* blocks_per_sm);
int tc_stage_b_tile();  // level-1 frequencies per stage-B CTA

cudaError_t launch_tc(const Pass& p, const PassArgs& a, cudaStream_t stream);
cudaError_t upload_tc5_tables();
cudaError_t tc5_occupancy(int* blocks_per_sm);
int tc5_stage_b_tile();  // level-1 frequencies per tcgen05 stage-B CTA
cudaError_t launch_tc5(const Pass& p, const PassArgs& a, cudaStream_t stream);

// Tile hybrid: cross-spectrum accumulation between the tiles' padded spectra.
cudaError_t launch_xspec(const Pass& p, const PassArgs& a, cudaStream_t stream);
cudaError_t xspec_occupancy(int* blocks_per_sm);
int64_t xspec_ctas_per_channel(const Pass& p);
// Forward three-step passes of 2048 and 4096 points: lines per CTA (W consecutive
// inner indices, or for an innermost MID axis W consecutive outer lines).
bool smem3_supports(int L);
int smem3_lines(int L, int mode, int64_t inner);
cudaError_t launch_smem3(const Pass& p, const PassArgs& a, cudaStream_t stream);
cudaError_t smem3_last_occupancy(const Pass& p, int src_kind, int* blocks_per_sm);
bool xspec5_supports(int64_t n_tiles, int64_t K);  // <= 64 tiles, K a multiple of 4
cudaError_t launch_xspec5(const Pass& p, const PassArgs& a, cudaStream_t stream);
cudaError_t xspec5_occupancy(int* blocks_per_sm);
int64_t xspec5_ctas_per_channel(const Pass& p);
// Per channel of a chunk: max over its voltages of |re| and |im| (out[cc] zeroed
// first; non-negative floats compared as integers).  src_kind SRC_CF32 or SRC_CI8.
cudaError_t launch_chan_absmax(const void* volts, int src_kind, int64_t vc0, int64_t T, int64_t t0, int64_t N,
                               int64_t cc, int64_t tc, float* out, cudaStream_t stream);
// An accumulator [cv channels from P][K][NP] complex FP64 (NP tile pairs or
// coarse lags) transposed to [NP][K] in dst (the inverse passes' source layout).
cudaError_t launch_xspec5_transpose(const double* P, int64_t P_stride, int64_t cv, int64_t K, int64_t NP,
                                    float2* dst, cudaStream_t stream);

// F-engine: frames per antenna, scratch bytes, CTAs of the largest launch, and
// the launches (fused for F <= 256; else spectra into scratch [N][T][F], then
// calibrated, quantised or not, transposed to [F][T][N]).
int64_t fengine_frames(int64_t n_samples, int32_t F, int32_t P);
int64_t fengine_scratch_bytes(int64_t N, int64_t S, int32_t F, int32_t P);
int64_t fengine_ctas(int64_t N, int64_t T, int32_t F);  // largest launch, CTAs
cudaError_t launch_fengine(const int8_t* raw, int64_t N, int64_t S, int32_t F, int32_t P,
                           const float* window, const float2* gains, float scale, int out_i8,
                           void* out, float2* scratch, cudaStream_t stream);

// Set the calling thread's omni_last_error() message.
void set_last_error(const char* msg);

}  // namespace omni
