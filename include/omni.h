/*
 * omni.h -- C ABI of the GB300 hierarchical-grid ("hypercube") FFT correlator.
 *
 * The method (Tegmark & Zaldarriaga, "Omniscopes", Sec. II): antennas sit on
 * an n-level hierarchical grid r = sum_k A_k m_k (Eq. GridEq).  Placing the
 * voltages f_r of one time sample and frequency channel in the 2n-D hypercube
 * F_{i1 i2 ...} (Eq. ProofEq2), zero-padding it, taking the 2n-D FFT, squaring
 * the modulus, summing over time and inverse-transforming gives G, the
 * visibilities summed over every antenna pair with the same 2n-D separation
 * (Sec. II.C: "zero-padded FFT, squaring the result and inverse transforming").
 *
 * Conventions (all entry points):
 *  - A hierarchy is given as n_levels omni_level records, level 1 (finest)
 *    first.  The lattice has D = 2 n_levels dimensions with sizes
 *    (n1 of level 1, n2 of level 1, n1 of level 2, ...); dimension 0 varies
 *    fastest.
 *  - Voltages are [C][T][N] complex values, interleaved (re, im), N = prod n_d,
 *    antenna index row-major with dimension 0 fastest, i.e. antenna i has
 *    m_0 = i mod n_0, m_1 = (i / n_0) mod n_1, ...
 *  - Lags: each dimension d runs D_d = -(n_d-1) .. n_d-1, dimension 0 fastest;
 *    Q = prod_d (2 n_d - 1) lags per channel.  The visibility of lag D is
 *    V(D) = sum_t sum_m x_t(m + D) conj(x_t(m)), i.e. V_ij = x_i x_j^* summed
 *    over all pairs with m_i - m_j = D (the conjugate is the complex-voltage
 *    reading of Eq. ConvolutionDefEq, which the paper writes for real f).
 *  - The forward transform uses exp(-2 pi i k.m / L), the padded length is
 *    L_d = 2 n_d (1 when n_d = 1), and the output is normalised by 1/L only
 *    once, in the inverse transform; visibilities are summed, not averaged,
 *    over time.
 *  - Every call returns an omni_status; omni_last_error() gives a message for
 *    the calling thread's last failure.  Device work is asynchronous on the
 *    stream passed in (a cudaStream_t passed as void*, NULL = legacy default
 *    stream); a device-side failure is reported by the next call that
 *    synchronises (omni_visibilities*) or by omni_sync.
 *  - Nothing here frees or retains memory owned by the caller.
 */
#ifndef OMNI_H
#define OMNI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One level of the hierarchy (Eq. GridEq): an n1 x n2 block placed by the
 * row-major 2x2 matrix A = [a_k | a_{k+n}] (the level's two lattice vectors as
 * columns), r = A (m1, m2)^T.  Sec. II.D numbers the first axes a_1..a_n and
 * the second axes a_{n+1}..a_{2n}. */
typedef struct omni_level {
    int32_t n1;
    int32_t n2;
    double A[4];
} omni_level;

typedef enum omni_status {
    OMNI_OK = 0,
    OMNI_ERR_INVALID_ARG = 1,  /* null pointer, non-positive size, bad enum */
    OMNI_ERR_COLLISION = 2,    /* two antennas coincide: the map r -> (m_k) is
                                  not unique, which Sec. II.D requires */
    OMNI_ERR_UNSUPPORTED = 3,  /* a size this build does not handle */
    OMNI_ERR_OOM = 4,          /* device or pinned-host allocation failed */
    OMNI_ERR_CUDA = 5,         /* a CUDA runtime call or kernel failed */
    OMNI_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up */
} omni_status;

typedef enum omni_dtype {
    OMNI_IN_CF32 = 0,  /* float re, float im (8 bytes per antenna-sample) */
    OMNI_IN_CI8 = 1    /* int8 re, int8 im (2 bytes), values in [-127, 127] */
} omni_dtype;

/* Mixed precision (2-level hierarchies and tile plans): the coarse level is
 * evaluated in lag space (Sec. II.D's convolution over the level-2 axes as a
 * sum over level-1 block pairs of equal grid offset): per level-1 frequency, the
 * blocks' cross-spectra summed over time as one tensor-core GEMM with the
 * samples as the contraction axis, FP32 accumulation, FP64 fold per chunk.
 * Level 1 runs as split-FP16 DFT-GEMMs (int8 voltages, 16x16 blocks, FP16
 * precision) or as the FP32 FFT.  Both mixed forms keep relative errors near
 * 1e-6 against the FP64 oracle. */
typedef enum omni_precision {
    OMNI_FP32 = 0,        /* all FFT arithmetic in FP32 */
    OMNI_MIXED_FP16 = 1,  /* GEMM operands split in two FP16 halves (3 products); the
                           * spectra scaled by a power of two first: fixed from the
                           * block size for int8 voltages, per channel and chunk from
                           * the voltages' max |re|, |im| for float voltages */
    OMNI_MIXED_BF16 = 2   /* GEMM operands split in three BF16 parts (6 products, about
                           * 24 bits, FP32's range: no scaling) */
} omni_precision;

typedef struct omni_plan omni_plan;

/* Lattice sizes of a hierarchy without creating a plan (host only, no GPU).
 * n_antennas = prod n_d, n_lags = prod (2 n_d - 1). */
omni_status omni_lattice_shape(const omni_level* levels, int n_levels,
                               int64_t* n_antennas, int64_t* n_lags);

/* Baseline table of a hierarchy (host only, no GPU; bit-exact integers).
 * dm [n_lags][2 n_levels] int32: the 2n-D lag of every output slot
 *   (Eq. ProofEq2: each G index runs over -(n-1)..(n-1));
 * redundancy [n_lags] int64: number of antenna pairs sharing that lag,
 *   prod_d (n_d - |D_d|) (the baseline distribution d = l * l^- of Sec. III
 *   for a layout map of ones);
 * dr [n_lags][2] double: the physical baseline sum_k A_k (D_{2k}, D_{2k+1}).
 * Any of the three outputs may be NULL.  Returns OMNI_ERR_COLLISION when two
 * antennas coincide within 1e-9 * max|r|. */
omni_status omni_baselines(const omni_level* levels, int n_levels, int32_t* dm,
                           int64_t* redundancy, double* dr);

/* Create a plan on the current CUDA device for C channels of voltages of the
 * given type.  The plan owns its device accumulator ([C][L] FP64, L =
 * prod L_d; mixed plans [C][L1 L2 of level 1][(2 n3 - 1)(2 n4 - 1)] complex),
 * scratch buffers and staging memory; all are allocated here.  The samples of
 * each omni_correlate call are processed in chunks the plan sizes itself (from
 * its buffer target, the kernels' occupancy and, for mixed plans, whole waves
 * of CTAs); results do not depend on the chunking.
 * Errors: INVALID_ARG, COLLISION, UNSUPPORTED (more than 8 levels, a padded
 * axis longer than 4096, or a non-power-of-two padded axis longer than 1024;
 * mixed precision outside 2-level hierarchies of at most 64 level-1 blocks
 * whose padded level-1 size 4 n1 n2 is a multiple of 4), OOM, CUDA. */
omni_status omni_plan_create(const omni_level* levels, int n_levels, int64_t n_channels,
                             omni_dtype dtype, omni_precision precision, omni_plan** out);

/* Autotuned plan: times candidate plans for this problem on the caller's
 * voltages volts_dev ([C][T][N], as omni_correlate takes them) and returns the
 * fastest.  Candidates: chunk buffer size (384, 768, 1536, 3072 MB) x overlap of
 * consecutive chunks' passes x, for the FP32 path, level passes (both axes of
 * a square level in one kernel) or one pass per axis, or, for the mixed path,
 * the share of each chunk's last pass on tensor cores (all, 0.3, 0.6) with the
 * rest on the FP32 level kernel, and level 1 on tensor cores or as the FP32
 * FFT; and for padded axes of 2048 or 4096 points the radix split of their forward
 * passes, three steps 16 x 16 x (8 | 16) or four steps 64 x (32 | 64).  Each candidate
 * runs one warm-up and two timed omni_correlate calls on a
 * private stream (their accumulators are discarded).  cache_path (or NULL): a text file of one JSON object per line,
 * keyed by level shapes, precision, dtype, C, T and device name; a hit skips
 * the search (*from_cache = 1), a search appends its winner.  Errors: as
 * omni_plan_create; INVALID_ARG for NULL volts_dev or T < 1. */
omni_status omni_plan_create_tuned(const omni_level* levels, int n_levels, int64_t n_channels,
                                   omni_dtype dtype, omni_precision precision, const void* volts_dev,
                                   int64_t T, const char* cache_path, int* from_cache, omni_plan** out);

/* The choices a plan was built with (any output may be NULL). */
omni_status omni_plan_knobs(const omni_plan* plan, int64_t* chunk_mb, int* overlap, int* level_passes,
                            double* split_tc);

/* Beam-space plan (Appendix A, steps 4-5): each level-1 block is Fourier
 * transformed unpadded, giving n1 x n2 digital pointings k = (k_a, k_b), and
 * the correlation runs over the axes of levels 2..n only:
 *   y_t(k; m') = sum_{m1} x_t(m1, m') exp(-2 pi i (k_a m1_a / n1 + k_b m1_b / n2)),
 *   B_c(k; D') = sum_t sum_{m'} y_t(k; m' + D') conj(y_t(k; m')),
 * with m' the index on levels 2..n and D' its lag.  omni_correlate* take the
 * same voltages [C][T][N]; omni_visibilities* write B as complex128
 * [C][Q'][n1 n2], the pointing index k_a + n1 k_b fastest and the lags of
 * levels 2..n in the order omni_baselines gives for levels + 1 (the lag table
 * of the coarser levels alone).  omni_plan_info reports n_lags = Q' n1 n2 and
 * the level-1 axes as unpadded.  FP32 path only.
 * Errors: as omni_plan_create; UNSUPPORTED for a single level or when every
 * coarser level is 1 x 1. */
omni_status omni_plan_create_beams(const omni_level* levels, int n_levels, int64_t n_channels,
                                   omni_dtype dtype, omni_plan** out);

/* Tile hybrid (Sec. III): n_tiles identical tiles, each the one-level grid
 * *tile (n1 x n2, matrix A), placed at arbitrary offsets o_j (offsets
 * [n_tiles][2], metres, antenna j*n1*n2 + a + n1 b at o_j + A (a, b)).  Each
 * tile is FFT-correlated within itself (zero-padded 2-D FFT per sample) and
 * the tiles' spectra are correlated pairwise by brute force:
 *   V_c(i, j; D) = sum_t sum_{m} x_{t,i}(m + D) conj(x_{t,j}(m)),
 * for every ordered tile pair (i, j) and intra-tile offset D (the physical
 * baseline is o_i - o_j + A D).  omni_correlate* take voltages [C][T][N]
 * with N = n_tiles n1 n2, tile slowest; omni_visibilities* write complex128
 * [C][n_tiles][n_tiles][(2 n1 - 1)(2 n2 - 1)], lags dimension 0 fastest.
 * omni_plan_info reports dims (n1, n2, n_tiles, 1) and n_lags = n_tiles^2 Q.
 * The plan's accumulator is [C][n_tiles][n_tiles][4 n1 n2] complex FP64
 * ([C][4 n1 n2][n_tiles][n_tiles] on the mixed path, transposed once per
 * omni_visibilities call into the plan's scratch before the inverse).
 * precision OMNI_FP32: the cross-spectra are summed on CUDA cores in FP32;
 * OMNI_MIXED_FP16 / _BF16: per tile frequency they are one tensor-core GEMM over
 * the samples (tcgen05, operands split as the precision says, FP32 accumulation
 * in tensor memory), for at most 64 tiles and 4 n1 n2 a multiple of 4.
 * Errors: as omni_plan_create; INVALID_ARG for n_tiles < 1 or a NULL or
 * non-finite offset; UNSUPPORTED beyond 4096 tiles or outside the mixed
 * path's limits; COLLISION if two antennas of different tiles coincide. */
omni_status omni_plan_create_tiles(const omni_level* tile, int64_t n_tiles, const double* offsets,
                                   int64_t n_channels, omni_dtype dtype, omni_precision precision,
                                   omni_plan** out);

/* F-engine (Appendix A, step 2): channelise every antenna's real int8 sample
 * stream into the correlator's input voltages.  Frame t of antenna a, with
 * frame length 2F and P taps (polyphase filter bank):
 *   u_t(n) = sum_{p<P} w[p 2F + n] r_a[(t + p) 2F + n],  n < 2F
 *   X_t(f) = sum_{n<2F} u_t(n) exp(-2 pi i f n / 2F),    f < F (Nyquist dropped)
 *   y_t(f) = scale g[f][a] X_t(f)
 * raw_dev [n_antennas][n_samples] int8 (device); window_dev [P][2F] float or
 * NULL (all ones); gains_dev [F][n_antennas] complex float (re, im) or NULL
 * (1); out_dev [F][T][n_antennas] complex, OMNI_IN_CI8 (round half to even,
 * clipped to +-127) or OMNI_IN_CF32, T = floor((n_samples - (P-1) 2F) / 2F)
 * (returned in *n_frames): exactly what omni_correlate reads with C = F.
 * scratch_dev: at least omni_fengine_scratch_bytes(...) bytes, 8-byte aligned,
 * owned by the caller (0 bytes, and scratch_dev may be NULL, when F <= 256: one
 * fused pass; larger F stage the spectra [N][T][F] FP32 there).  Asynchronous
 * on stream; nothing is allocated.
 * Errors: INVALID_ARG (NULL pointers, F not a power of two in [2, 4096], taps
 * outside [1, 64], misaligned out/gains/scratch, scratch too small, a launch
 * larger than 2^31 - 1 CTAs), CUDA. */
int64_t omni_fengine_scratch_bytes(int64_t n_antennas, int64_t n_samples, int32_t n_channels,
                                   int32_t taps);
omni_status omni_fengine(const int8_t* raw_dev, int64_t n_antennas, int64_t n_samples,
                         int32_t n_channels, int32_t taps, const float* window_dev,
                         const float* gains_dev, float scale, omni_dtype out_dtype, void* out_dev,
                         void* scratch_dev, int64_t scratch_bytes, int64_t* n_frames, void* stream);

/* A plan for n_arrays independent arrays of possibly different hierarchies
 * (Sec. III: several separate omniscopes, each correlated on its own), all with
 * n_channels channels of the same dtype.  levels_per_array[a] has
 * n_levels_per_array[a] levels.  Runs of consecutive arrays with the same level
 * shapes are correlated together, one launch per transform pass for the whole
 * run, so ordering the arrays by shape gives the fewest launches.
 * The same omni_correlate*, omni_visibilities*, omni_reset, omni_sync,
 * omni_profile_* and omni_plan_destroy calls apply:
 *   voltages: the arrays' [C][T][N_a] blocks concatenated in array order;
 *   visibilities: the arrays' [C][n_lags_a] complex128 blocks concatenated.
 * omni_plan_info on a batch plan reports n_dims = 0, n_antennas = sum N_a and
 * n_lags = sum n_lags_a; omni_batch_info gives the per-array sizes. */
omni_status omni_plan_create_batch(const omni_level* const* levels_per_array,
                                   const int* n_levels_per_array, int n_arrays,
                                   int64_t n_channels, omni_dtype dtype,
                                   omni_precision precision, omni_plan** out);

/* Per-array sizes of a batch plan (n_arrays = 1 for a single-array plan):
 * antennas[a] = N_a, lags[a] = n_lags_a (arrays may be NULL to query n_arrays). */
omni_status omni_batch_info(const omni_plan* plan, int* n_arrays, int64_t* antennas,
                            int64_t* lags);

/* Free everything the plan owns (synchronises its device work first). */
void omni_plan_destroy(omni_plan* plan);

/* Shape of a plan: n_dims = 2 n_levels; dims/padded receive n_d and L_d
 * ([n_dims] each, may be NULL). */
omni_status omni_plan_info(const omni_plan* plan, int* n_dims, int32_t* dims,
                           int32_t* padded, int64_t* n_antennas, int64_t* n_lags,
                           int64_t* n_channels);

/* Accumulate T samples of every channel (Sec. II.C: FFT, |.|^2, summed over
 * time; Appendix A steps 3-5).  volts_dev: DEVICE pointer to [C][T][N]
 * complex voltages of the plan's dtype, owned by the caller and only read,
 * aligned to its element size (2 bytes for int8, 8 for float32; 16 bytes for
 * mixed-precision plans whose level 1 runs on tensor cores: int8 16x16 blocks).  T >= 0 (T = 0 is a no-op).  Asynchronous on stream. */
omni_status omni_correlate(omni_plan* plan, const void* volts_dev, int64_t T, void* stream);

/* Same as omni_correlate for voltages in HOST memory (pageable or pinned):
 * the plan copies them to the device in chunks, overlapping the copies with
 * the transforms, and returns once the host buffer may be reused (the
 * transforms may still be running on stream). */
omni_status omni_correlate_host(omni_plan* plan, const void* volts_host, int64_t T,
                                void* stream);

/* Inverse-transform the accumulated |F|^2 into visibilities (Sec. II.C) and
 * write them to vis_dev, a DEVICE pointer to [C][n_lags] complex128
 * (interleaved re, im doubles) owned by the caller.  reset != 0 clears the
 * accumulator afterwards so that the next omni_correlate starts a new
 * integration.  Synchronises the stream and reports earlier device errors. */
omni_status omni_visibilities(omni_plan* plan, double* vis_dev, int reset, void* stream);

/* Same as omni_visibilities with vis_host in HOST memory. */
omni_status omni_visibilities_host(omni_plan* plan, double* vis_host, int reset,
                                   void* stream);

/* Clear the accumulator (start a new integration) without producing output. */
omni_status omni_reset(omni_plan* plan, void* stream);

/* Wait for the plan's work on stream and report any device error. */
omni_status omni_sync(omni_plan* plan, void* stream);

/* Per-kernel statistics of a plan (see omni_profile_*). */
typedef struct omni_kernel_stat {
    char name[64];     /* pass name, e.g. "fwd axis3 reg16 last" */
    int64_t launches;  /* kernel launches of this pass */
    double total_ms;   /* summed durations from CUDA events recorded around each
                          launch on the launching stream (0 unless profiling) */
    double bytes;      /* algorithmic bytes of all launches: inputs read plus
                          outputs written at their stored precision */
    double flops;      /* algorithmic floating-point operations of all launches:
                          5 L log2 L per L-point line transform plus 3 per |F|^2
                          term for the FFT passes; the executed m16n8k16 products
                          (4096 each) for the tensor-core passes */
    int32_t tensor;    /* 1 when the pass runs on tensor cores */
} omni_kernel_stat;

/* Start (enable != 0) or stop recording a CUDA event pair around every kernel
 * launch of the plan.  Launch counts are kept whether or not profiling is on. */
omni_status omni_profile_enable(omni_plan* plan, int enable);

/* Copy up to max per-pass statistics into out (n_out receives how many);
 * waits for the recorded events.  clear != 0 resets the statistics. */
omni_status omni_profile_read(omni_plan* plan, omni_kernel_stat* out, int max, int* n_out,
                              int clear);

/* ---- Physical-baseline epilogue (Sec. II.D, Sec. III) ----
 * The hypercube output has one value per 2n-D lag; lags whose physical
 * baselines dr = sum_k A_k (D_{2k}, D_{2k+1}) coincide (possible for
 * interleaved hierarchies, Sec. II.D) measure the same uv point, and binning
 * |dr| radially gives the one-dimensional baseline distribution (Figs. 2-5,
 * bottom panels, for a layout map of ones). */

/* Radial bins (host only, no GPU): bin_of_lag[q] = floor(|dr_q| / bin_width)
 * for lags inside the first n_bins bins, else -1; pairs_per_bin[b] = number of
 * antenna pairs in bin b (sum of the lags' redundancies).  Either output may
 * be NULL. */
omni_status omni_radial_bins(const omni_level* levels, int n_levels, double bin_width,
                             int64_t n_bins, int32_t* bin_of_lag, int64_t* pairs_per_bin);

/* Distinct physical baselines (host only, no GPU): lags whose dr agree within
 * 1e-9 * max|dr| share a group; groups are numbered in order of their first
 * lag.  n_unique receives the group count; group_of_lag [n_lags];
 * dr_unique [n_lags][2] and pairs_unique [n_lags] (first n_unique entries
 * used) receive each group's baseline and antenna-pair count.  Outputs other
 * than n_unique may be NULL. */
omni_status omni_unique_baselines(const omni_level* levels, int n_levels, int64_t* n_unique,
                                  int32_t* group_of_lag, double* dr_unique, int64_t* pairs_unique);

/* Sum visibilities by group on the GPU: out[c][g] = sum of vis[c][q] over
 * the lags q with group_dev[q] == g (group -1: skipped).  vis_dev: DEVICE
 * [C][Q] complex128; group_dev: DEVICE [Q] int32; out_dev: DEVICE
 * [C][n_groups] complex128, overwritten.  FP64 sums (atomic, so the order of
 * the additions is not fixed).  Asynchronous on stream. */
omni_status omni_sum_groups(const double* vis_dev, int64_t C, int64_t Q, const int32_t* group_dev,
                            int64_t n_groups, double* out_dev, void* stream);

/* Size of the device array that omni_correlate_noalloc uses as scratch. */
#define OMNI_NOALLOC_SCRATCH_BYTES (64ull * 1024ull * 1024ull)

/* One whole integration without any device allocation.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc, such as code
 * running under another framework's memory pool or allocator hooks, processes
 * that reserve all device memory up front, and real-time pipelines that forbid
 * allocation after start-up.
 *
 * Computes the visibilities of T samples of C channels of a hierarchy, exactly
 * as omni_plan_create + omni_correlate + omni_visibilities would, and returns
 * after they are written.  volts_dev: DEVICE [C][T][N] complex voltages of
 * dtype (16-byte aligned, read only); vis_dev: DEVICE [C][n_lags] complex128
 * output (16-byte aligned).  Both belong to the caller.
 *
 * Scratch (the FP64 accumulator, the pass buffers, the direct-DFT twiddles) is
 * one static device array of OMNI_NOALLOC_SCRATCH_BYTES (64 MiB) inside the
 * library; every GPU that loads this part of the library holds it until the
 * process exits.  The call allocates nothing: no cudaMalloc, no cudaFree.  A
 * problem whose scratch (C x L x 8 bytes of accumulator plus two pass buffers
 * of at least one sample or channel each) does not fit returns
 * OMNI_ERR_UNSUPPORTED with the sizes in omni_last_error().
 *
 * The first call on each device does the set-up (uploads the twiddle tables
 * and looks up the array's device address).  Every call also copies the direct-DFT twiddles
 * (when the lattice has a non-power-of-two axis) from host memory and
 * synchronises stream before returning.  Every call shares the one array and
 * the accumulator is cleared at the start of each call: calls that overlap on
 * the GPU (other streams, other host threads) race on it and must be
 * serialised by the caller. */
omni_status omni_correlate_noalloc(const omni_level* levels, int n_levels, int64_t n_channels,
                                   omni_dtype dtype, const void* volts_dev, int64_t T,
                                   double* vis_dev, void* stream);

/* Message describing the calling thread's most recent failure ("" if none). */
const char* omni_last_error(void);

/* Static name of a status code. */
const char* omni_status_string(omni_status status);

#ifdef __cplusplus
}
#endif

#endif /* OMNI_H */
