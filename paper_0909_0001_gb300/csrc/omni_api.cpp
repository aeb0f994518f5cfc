// omni_api.cpp -- host side of the C ABI declared in include/omni.h.
//
// Validates hierarchies, builds the lattice geometry (Eq. GridEq) and the
// baseline tables (Eq. ProofEq2 index ranges, Sec. III redundancy), owns the
// device accumulator and scratch, and sequences the per-axis passes of the
// correlator: forward passes over chunks of samples with |F|^2 summed into the
// FP64 accumulator, then inverse passes that produce the visibilities.
#include "omni.h"
#include "omni_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

namespace omni {
// Resident CTAs per SM of a four-step LAST pass (omni_dispatch.cpp).
cudaError_t smem_last_occupancy(const Pass& p, int src_kind, int* blocks_per_sm);
}  // namespace omni

using namespace omni;

namespace {

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

thread_local std::string g_last_error;

omni_status fail(omni_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

omni_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? OMNI_ERR_OOM : OMNI_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define OMNI_CUDA(call, what)                        \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }


struct Geometry;
omni_status tile_geometry(Geometry& g, int64_t n_tiles, const double* offsets);
omni_status check_unique_positions(const std::vector<double>& r, int64_t N);

// Lattice geometry of a validated hierarchy.
struct Geometry {
    int n_levels = 0;
    int D = 0;
    int32_t n[kMaxDims] = {};
    int32_t Lp[kMaxDims] = {};
    int64_t N = 1, L = 1, Q = 1;
    std::vector<double> A;  // [n_levels][4]
};

// beams: the level-1 axes are transformed unpadded (n_d points -> n_d digital
// pointings, Appendix A step 4); they carry the pointing index, not a lag.
omni_status make_geometry(const omni_level* levels, int n_levels, Geometry& g, bool beams = false) {
    if (!levels) return fail(OMNI_ERR_INVALID_ARG, "levels is NULL");
    if (n_levels < 1 || n_levels > kMaxDims / 2)
        return fail(OMNI_ERR_INVALID_ARG, "n_levels must be in [1, %d], got %d", kMaxDims / 2, n_levels);
    g.n_levels = n_levels;
    g.D = 2 * n_levels;
    g.A.assign(4 * n_levels, 0.0);
    for (int k = 0; k < n_levels; ++k) {
        const omni_level& lv = levels[k];
        if (lv.n1 < 1 || lv.n2 < 1)
            return fail(OMNI_ERR_INVALID_ARG, "level %d has shape %d x %d; sizes must be >= 1", k + 1,
                        lv.n1, lv.n2);
        for (int c = 0; c < 4; ++c) {
            if (!std::isfinite(lv.A[c])) return fail(OMNI_ERR_INVALID_ARG, "level %d matrix is not finite", k + 1);
            g.A[4 * k + c] = lv.A[c];
        }
        g.n[2 * k] = lv.n1;
        g.n[2 * k + 1] = lv.n2;
    }
    for (int d = 0; d < g.D; ++d) {
        const int64_t nd = g.n[d];
        const bool beam_axis = beams && d < 2;
        const int64_t Ld = (nd > 1 && !beam_axis) ? 2 * nd : nd;
        if (g.N > (int64_t(1) << 40) / nd) return fail(OMNI_ERR_UNSUPPORTED, "too many antennas");
        g.N *= nd;
        g.L *= Ld;
        g.Q *= beam_axis ? nd : 2 * nd - 1;
        if (Ld > kTwiddleN) return fail(OMNI_ERR_UNSUPPORTED, "padded axis %d has length %lld > %d", d, (long long)Ld, kTwiddleN);
        if (!is_pow2(Ld) && Ld > 1024)
            return fail(OMNI_ERR_UNSUPPORTED, "padded axis %d has non-power-of-two length %lld > 1024", d, (long long)Ld);
        g.Lp[d] = (int32_t)Ld;
    }
    return OMNI_OK;
}

// Antenna positions r_i = sum_k A_k m_k (Eq. GridEq), antenna order dimension 0 fastest.
void positions(const Geometry& g, std::vector<double>& r) {
    r.assign(2 * g.N, 0.0);
    for (int64_t i = 0; i < g.N; ++i) {
        int64_t rest = i;
        double x = 0.0, y = 0.0;
        for (int k = 0; k < g.n_levels; ++k) {
            const int64_t m1 = rest % g.n[2 * k];
            rest /= g.n[2 * k];
            const int64_t m2 = rest % g.n[2 * k + 1];
            rest /= g.n[2 * k + 1];
            const double* a = &g.A[4 * k];
            x += a[0] * m1 + a[1] * m2;
            y += a[2] * m1 + a[3] * m2;
        }
        r[2 * i] = x;
        r[2 * i + 1] = y;
    }
}

// Tile hybrid: n_tiles copies of the one-level geometry g at the given
// offsets ([n_tiles][2]); the tile index becomes an untransformed third axis
// (no padding, no lag), and every antenna position o_j + A m must be unique.
omni_status tile_geometry(Geometry& g, int64_t n_tiles, const double* offsets) {
    if (g.D != 2) return fail(OMNI_ERR_INVALID_ARG, "a tile is one level");
    std::vector<double> r;
    positions(g, r);
    const int64_t M = g.N;
    std::vector<double> all(2 * M * n_tiles);
    for (int64_t j = 0; j < n_tiles; ++j) {
        if (!std::isfinite(offsets[2 * j]) || !std::isfinite(offsets[2 * j + 1]))
            return fail(OMNI_ERR_INVALID_ARG, "tile %lld offset is not finite", (long long)j);
        for (int64_t a = 0; a < M; ++a) {
            all[2 * (j * M + a)] = offsets[2 * j] + r[2 * a];
            all[2 * (j * M + a) + 1] = offsets[2 * j + 1] + r[2 * a + 1];
        }
    }
    omni_status st = check_unique_positions(all, M * n_tiles);
    if (st != OMNI_OK) return st;
    g.D = 4;
    g.n_levels = 2;
    g.n[2] = (int32_t)n_tiles;
    g.n[3] = 1;
    g.Lp[2] = g.Lp[3] = 1;
    g.N = M * n_tiles;
    g.Q *= n_tiles * n_tiles;
    g.A.resize(8, 0.0);
    return OMNI_OK;
}

// Sec. II.D requires the map from r to the index set to be unique: reject two
// antennas closer than 1e-9 max|r| (exactly coincident when max|r| = 0).
// Spatial hash with cells of the tolerance size; each point checks the 3x3
// neighbouring cells.
omni_status check_unique(const Geometry& g) {
    if (g.N < 2) return OMNI_OK;
    std::vector<double> r;
    positions(g, r);
    return check_unique_positions(r, g.N);
}

omni_status check_unique_positions(const std::vector<double>& r, int64_t N) {
    if (N < 2) return OMNI_OK;
    double rmax = 0.0;
    for (int64_t i = 0; i < N; ++i) rmax = std::max(rmax, std::hypot(r[2 * i], r[2 * i + 1]));
    const double tol = 1e-9 * rmax;
    const double cell = tol > 0.0 ? tol : 1.0;
    struct Key {
        int64_t x, y;
        bool operator==(const Key& o) const { return x == o.x && y == o.y; }
    };
    struct KeyHash {
        size_t operator()(const Key& k) const {
            return std::hash<int64_t>()(k.x * 0x9E3779B97F4A7C15ULL ^ (uint64_t)k.y);
        }
    };
    std::unordered_map<Key, std::vector<int64_t>, KeyHash> grid;
    grid.reserve((size_t)N * 2);
    for (int64_t i = 0; i < N; ++i) {
        const Key k{(int64_t)std::floor(r[2 * i] / cell), (int64_t)std::floor(r[2 * i + 1] / cell)};
        for (int64_t dx = -1; dx <= 1; ++dx)
            for (int64_t dy = -1; dy <= 1; ++dy) {
                auto it = grid.find(Key{k.x + dx, k.y + dy});
                if (it == grid.end()) continue;
                for (int64_t j : it->second)
                    if (std::hypot(r[2 * i] - r[2 * j], r[2 * i + 1] - r[2 * j + 1]) <= tol)
                        return fail(OMNI_ERR_COLLISION,
                                    "antennas %lld and %lld coincide at (%g, %g): the hierarchy "
                                    "does not map positions to unique indices",
                                    (long long)j, (long long)i, r[2 * i], r[2 * i + 1]);
            }
        grid[k].push_back(i);
    }
    return OMNI_OK;
}

}  // namespace

void omni::set_last_error(const char* msg) { g_last_error = msg; }

// ----------------------------------------------------------------------------- plan

// Tunable choices of a plan (the autotuner searches these; environment
// variables override the defaults for experiments).
struct Knobs {
    int64_t chunk_mb = 3072;      // target size of each chunk scratch buffer (OMNI_CHUNK_MB)
    int64_t chunk_channels = 0;   // channels per chunk, 0 = one wave of the last pass (OMNI_CHUNK_CHANNELS)
    int overlap = -1;             // overlap the two passes of consecutive chunks (OMNI_OVERLAP; -1:
                                  // on, except before the one-CTA-per-SM cross-spectrum GEMMs,
                                  // where both passes are bound by HBM traffic and the overlap
                                  // measured 13.69 vs 13.72 ms per step on the 2-level workload)
    int level_passes = 1;         // both axes of a square level in one pass (OMNI_LEVEL_PASSES)
    double split_tc = 0.0;        // mixed: share of a chunk's channels on tensor cores, 0 = all (OMNI_SPLIT_TC)
    int tc_stage_a = 1;           // mixed: level 1 on tensor cores (1) or the FP32 FFT (0) (OMNI_TC_STAGE_A;
                                  // measured on the 2-level workload: 20.8 vs 23.9 ms per step)
    int lag_sum = 1;              // mixed: level 2 as block cross-spectra over time summed by grid
                                  // offset on tcgen05 (1), or per-sample level-2 DFT-GEMMs (0)
                                  // (OMNI_MIXED_LAGSUM)
    int fft3 = 1;                 // 2048/4096-point axes as three steps 16 x 16 x (8|16) (1)
                                  // or four steps 64 x (32|64) (0) (OMNI_FFT3; grid1024 FP32:
                                  // 23.6 vs 60.3 ms per step)
};

Knobs knobs_from_env() {
    Knobs k;
    if (const char* e = std::getenv("OMNI_CHUNK_MB")) k.chunk_mb = std::max<int64_t>(1, std::atoll(e));
    if (const char* e = std::getenv("OMNI_CHUNK_CHANNELS")) k.chunk_channels = std::max<int64_t>(0, std::atoll(e));
    if (const char* e = std::getenv("OMNI_OVERLAP")) k.overlap = std::atoi(e) != 0;
    if (const char* e = std::getenv("OMNI_LEVEL_PASSES")) k.level_passes = std::atoi(e) != 0;
    if (const char* e = std::getenv("OMNI_SPLIT_TC")) k.split_tc = std::atof(e);
    if (const char* e = std::getenv("OMNI_TC_STAGE_A")) k.tc_stage_a = std::atoi(e) != 0;
    if (const char* e = std::getenv("OMNI_MIXED_LAGSUM")) k.lag_sum = std::atoi(e) != 0;
    if (const char* e = std::getenv("OMNI_FFT3")) k.fft3 = std::atoi(e) != 0;
    return k;
}

struct omni_plan {
    int device = 0;
    Knobs knobs;
    Geometry g;
    int64_t C = 0;
    omni_dtype dtype = OMNI_IN_CF32;
    omni_precision precision = OMNI_FP32;
    std::vector<Pass> fwd, inv;
    int64_t Cc = 1, Tc = 1;   // forward chunk: channels x samples
    bool beams = false;       // beam-space plan: level-1 axes unpadded, no lag over them
    int64_t n_tiles = 0;      // tile-hybrid plan: identical tiles at arbitrary offsets
    int64_t lag_pairs = 0;    // mixed 2-level plan with a lag-sum level 2: coarse lags kept per
                              // level-1 frequency (the accumulator is [L1 L2 of level 1][lag_pairs])
    double inv_scale = 1.0;   // 1 / (points of the inverse transform)
    int64_t Cv = 1;           // inverse batch: channels
    int64_t fwd_elems = 0;    // float2 per sample, largest non-final forward output
    int64_t inv_elems = 0;    // float2 per channel, largest non-final inverse output
    float2* buf[2] = {nullptr, nullptr};
    float* chan_max = nullptr;  // FP16 plans of float voltages: per chunk channel max |x|, two chunk slots
    int64_t buf_elems = 0;
    double* P = nullptr;      // [C][L]
    int* dev_err = nullptr;   // device error word of bounded waits
    int force_expire = 0;     // OMNI_TEST_FORCE_TIMEOUT: tensor-core waits expire (tests)
    std::vector<float2*> tw_tables;
    // host-input staging
    void* stage[2] = {nullptr, nullptr};
    size_t stage_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ready[2] = {nullptr, nullptr};
    cudaEvent_t freed[2] = {nullptr, nullptr};
    // two-pass plans: the first pass of chunk j+1 runs on aux_stream while the
    // last pass of chunk j runs on the caller's stream (double-buffered scratch)
    bool overlap = false;
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t mid_done[2] = {nullptr, nullptr};
    cudaEvent_t last_done[2] = {nullptr, nullptr};
    cudaEvent_t start_ev = nullptr;
    // mixed plans: part of each chunk's channels go through the FP32 last pass on
    // split_stream, concurrently with the tensor-core last pass (CUDA cores and
    // tensor cores busy at once)
    bool split = false;
    double split_tc = 1.0;          // fraction of a chunk's channels on tensor cores
    Pass split_pass{};
    cudaStream_t split_stream = nullptr;
    cudaEvent_t split_done[2] = {nullptr, nullptr};
    double2* vis_tmp = nullptr;  // device staging for omni_visibilities_host
    // statistics per pass: forward passes first, then inverse passes
    std::vector<omni_kernel_stat> stats;
    bool profiling = false;
    struct Pending {
        int pass;
        cudaEvent_t start, stop;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    // batch plan: runs of same-shape arrays, each correlated by one member plan
    // whose channels are (array, channel) pairs
    std::vector<omni_plan*> members;
    std::vector<int> member_arrays;      // arrays per member
    std::vector<int64_t> array_antennas;  // per array
    std::vector<int64_t> array_lags;      // per array
};

// Kernel family and shared-memory split of one axis pass, from its length
// (also used by omni_correlate_noalloc).
void omni::choose_kind(Pass& p) {
    if (p.L == 1) {
        p.kind = KIND_DIRECT;
    } else if (is_pow2(p.L) && p.L >= 4 && p.L <= 64) {
        p.kind = KIND_REG;
    } else if (is_pow2(p.L) && p.L <= kTwiddleN) {
        p.kind = KIND_SMEM;
        switch (p.L) {
            case 128: p.L1 = 16; p.L2 = 8; break;
            case 256: p.L1 = 16; p.L2 = 16; break;
            case 512: p.L1 = 32; p.L2 = 16; break;
            case 1024: p.L1 = 32; p.L2 = 32; break;
            case 2048: p.L1 = 64; p.L2 = 32; break;
            default: p.L1 = 64; p.L2 = 64; break;
        }
        int W = 256 / p.L1;
        while (W > 1 && W / 2 >= p.inner) W /= 2;
        p.W = W;
    } else {
        p.kind = KIND_DIRECT;
    }
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int elem_bytes(omni_dtype t) { return t == OMNI_IN_CI8 ? 2 : 8; }

// Level pass tiling (fixed at compile time in the kernels): the finest level
// (inner == 1) packs whole blocks, W = 1; a coarser level takes W consecutive
// inner indices, W = 256 * LPT / L with LPT = 2 lines per thread (1 for
// 64-point axes) in a LAST pass and 1 in a MID pass.
void choose_level(Pass& p) {
    p.kind = KIND_LEVEL;
    const int lpt = p.mode == MODE_LAST ? (p.L >= 64 ? 1 : 2) : 1;
    p.W = p.inner == 1 ? 1 : 256 * lpt / p.L;
}

// Passes of 2048 and 4096 points: the three-step kernel (16-point register
// transforms; the four-step split 64 x 32 or 64 x 64 held a 64-point column in
// registers: 210-255 registers per thread, one or two CTAs per SM).
// Four-step passes along the innermost axis (inner == 1) other than LAST: W
// consecutive outer lines per CTA (256 threads) instead of one line per CTA of
// L1 threads.
void rows_lines(Pass& p) {
    if (p.kind == KIND_SMEM && p.inner == 1 && p.mode != MODE_LAST) p.W = 256 / p.L1;
}

void use_smem3(Pass& p, const Knobs& k) {
    if (!k.fft3 || p.kind != KIND_SMEM || !smem3_supports(p.L)) return;
    const bool fwd = p.mode == MODE_MID || p.mode == MODE_LAST;
    if (fwd && 2 * p.n > p.L) return;
    p.kind = KIND_SMEM3;
    p.W = smem3_lines(p.L, p.mode, p.inner);
}

// FP64 values of one channel's accumulator: |F|^2 over the padded lattice, or
// for a tile-hybrid plan the complex cross-spectra [n_tiles][n_tiles][L1 L2].
int64_t acc_doubles(const omni_plan* pl) {
    if (pl->n_tiles) return 2 * pl->n_tiles * pl->n_tiles * (int64_t)pl->g.Lp[0] * pl->g.Lp[1];
    if (pl->lag_pairs) return 2 * pl->lag_pairs * (int64_t)pl->g.Lp[0] * pl->g.Lp[1];
    return pl->g.L;
}

omni_status build_passes(omni_plan* pl) {
    const Geometry& g = pl->g;
    std::vector<int> axes;
    for (int d = 0; d < (pl->n_tiles ? 2 : g.D); ++d)
        if (g.Lp[d] > 1) axes.push_back(d);
    if (axes.empty()) axes.push_back(0);  // a single antenna: an identity "transform"
    // forward: increasing axis order; inputs [outer n_e>d][n_d][inner L_e<d].
    // A level whose two axes have the same power-of-two padded length <= 64 is
    // transformed by one level pass (both axes in shared memory); other axes
    // get one pass each (knob level_passes = 0 forces one pass per axis).
    const bool use_level = pl->knobs.level_passes != 0;
    std::vector<std::pair<int, bool>> stages;  // (first axis, is a level pass)
    for (size_t a = 0; a < axes.size(); ++a) {
        const int d = axes[a];
        const bool pair = use_level && (d % 2 == 0) && a + 1 < axes.size() && axes[a + 1] == d + 1 &&
                          g.Lp[d] == g.Lp[d + 1] && is_pow2(g.Lp[d]) && g.Lp[d] <= 64 &&
                          !(pl->beams && d < 2);
        stages.push_back({d, pair});
        if (pair) ++a;
    }
    pl->fwd.clear();
    pl->fwd_elems = 0;
    if (pl->precision != OMNI_FP32 && !pl->n_tiles) {
        const bool tc_shape = pl->precision == OMNI_MIXED_FP16 && tc_supports(g.n, g.D, pl->dtype == OMNI_IN_CI8);
        // level 1 on tensor cores (mma.sync split-FP16 DFT-GEMMs) for int8 16x16 blocks,
        // else the FP32 level-1 FFT; level 2 in lag space (tcgen05) unless the knob asks
        // for the per-sample DFT-GEMM forms, which exist for the 16x16-on-8x8 shape only
        const bool tc_a = tc_shape && pl->knobs.tc_stage_a;
        const bool lag = pl->knobs.lag_sum || !tc_shape;
        Pass pa{};
        pa.axis = 0;
        pa.kind = KIND_TC_A;
        pa.mode = MODE_MID;
        pa.L = g.Lp[0];
        pa.n = g.n[0];
        pa.q_out = g.Lp[0] * g.Lp[1];
        pa.inner = 1;
        pa.outer = (int64_t)g.n[2] * g.n[3];
        if (!tc_a && !lag) choose_level(pa);
        std::vector<Pass> level1;
        if (tc_a || !lag) {
            level1.push_back(pa);
        } else {
            // the generic level-1 passes (a level pass, or one pass per axis), MID mode,
            // leaving [block][L0 L1] per sample for the lag-sum pass
            for (const auto& stg : stages) {
                if (stg.first >= 2) continue;
                const int d = stg.first, last_axis = stg.second ? d + 1 : d;
                Pass q{};
                q.axis = d;
                q.L = g.Lp[d];
                q.n = g.n[d];
                q.q_out = stg.second ? g.Lp[d] * g.Lp[d] : g.Lp[d];
                q.inner = 1;
                q.outer = 1;
                for (int e = 0; e < d; ++e) q.inner *= g.Lp[e];
                for (int e = last_axis + 1; e < g.D; ++e) q.outer *= g.n[e];
                q.mode = MODE_MID;
                if (stg.second) {
                    choose_level(q);
                } else {
                    choose_kind(q);
                    if (q.n == q.L && q.L > 1 && q.kind == KIND_SMEM) q.kind = KIND_DIRECT;
                    rows_lines(q);
                    use_smem3(q, pl->knobs);
                }
                level1.push_back(q);
            }
        }
        stages.clear();
        Pass pb{};
        pb.axis = 2;
        pb.mode = MODE_LAST;
        if (lag) {
            // level 2 in lag space: per level-1 frequency the block cross-spectra
            // summed over the chunk's samples (one tcgen05 GEMM with the samples as
            // K), then summed over block pairs of equal grid offset
            pb.kind = KIND_COV5;
            pb.L = g.Lp[0] * g.Lp[1];
            pb.n = g.n[2] * g.n[3];
            pb.outer = (int64_t)g.n[2] * g.n[3];
            pb.inner = 1;
            pb.q_out = pb.L;
            pb.L1 = g.n[2];
            pb.L2 = g.n[3];
            pb.bf16 = pl->precision == OMNI_MIXED_BF16;
            pb.unscaled_in = tc_a ? 0 : 1;
            if (!pb.bf16 && !tc_a) {
                // FP16 operands: a power of two keeps |Y| <= 2^12 (int8: from the block size;
                // float voltages: per channel from the chunk's max |x|)
                const int64_t nb = (int64_t)g.n[0] * g.n[1];
                if (pl->dtype == OMNI_IN_CI8)
                    pb.scale_e = (int)std::ceil(std::log2((double)nb * 127.0 * 1.41422)) - 12;
                else
                    pb.scale_n = (int)nb;
            }
            pl->lag_pairs = (int64_t)(2 * g.n[2] - 1) * (2 * g.n[3] - 1);
        } else {
            // per-sample level-2 DFT-GEMMs + |F|^2: warp-level mma.sync by default,
            // OMNI_TCGEN05=1 selects the tensor-memory (tcgen05) variant
            pb.kind = KIND_TC_B;
            if (const char* env = std::getenv("OMNI_TCGEN05"))
                if (std::atoi(env) != 0) pb.kind = KIND_TC5_B;
            pb.L = g.Lp[2];
            pb.n = g.n[2];
            pb.q_out = g.Lp[2] * g.Lp[3];
            pb.inner = (int64_t)g.Lp[0] * g.Lp[1];
            pb.outer = 1;
            pb.W = pb.kind == KIND_TC_B ? tc_stage_b_tile() : tc5_stage_b_tile();
            pb.unscaled_in = tc_a ? 0 : 1;
        }
        for (const Pass& q : level1) {
            pl->fwd.push_back(q);
            pl->fwd_elems = std::max(pl->fwd_elems, q.outer * q.q_out * q.inner);
        }
        pl->fwd.push_back(pb);
    }
    for (size_t k = 0; k < stages.size(); ++k) {
        const int d = stages[k].first;
        const bool level = stages[k].second;
        const int last_axis = level ? d + 1 : d;
        Pass p{};
        p.axis = d;
        p.L = g.Lp[d];
        p.n = g.n[d];
        p.q_out = level ? g.Lp[d] * g.Lp[d] : g.Lp[d];
        p.inner = 1;
        p.outer = 1;
        for (int e = 0; e < d; ++e) p.inner *= g.Lp[e];
        for (int e = last_axis + 1; e < g.D; ++e) p.outer *= g.n[e];
        p.mode = (k + 1 == stages.size() && !pl->n_tiles) ? MODE_LAST : MODE_MID;
        if (level) {
            choose_level(p);
        } else {
            choose_kind(p);
            // unpadded (beam) axes: full-length register FFTs up to 64 points,
            // direct DFTs otherwise (the shared-memory kernels assume padding)
            if (p.n == p.L && p.L > 1 && p.kind == KIND_SMEM) p.kind = KIND_DIRECT;
            rows_lines(p);
            use_smem3(p, pl->knobs);
        }
        if (p.mode == MODE_MID) pl->fwd_elems = std::max(pl->fwd_elems, p.outer * p.q_out * p.inner);
        pl->fwd.push_back(p);
    }
    if (pl->n_tiles) {
        // tile hybrid: cross-spectra of every tile pair, per frequency of the tile
        Pass x{};
        x.axis = 0;
        x.kind = pl->precision != OMNI_FP32 ? KIND_XSPEC5 : KIND_XSPEC;
        x.unscaled_in = 1;  // the tile FFT writes unscaled spectra
        x.bf16 = pl->precision == OMNI_MIXED_BF16;
        if (pl->precision == OMNI_MIXED_FP16) {
            const int64_t nt = (int64_t)g.n[0] * g.n[1];
            if (pl->dtype == OMNI_IN_CI8)
                x.scale_e = (int)std::ceil(std::log2((double)nt * 127.0 * 1.41422)) - 12;
            else
                x.scale_n = (int)nt;
        }
        x.mode = MODE_LAST;
        x.L = g.Lp[0] * g.Lp[1];
        x.n = (int)pl->n_tiles;
        x.outer = pl->n_tiles;
        x.inner = 1;
        x.q_out = x.L;
        pl->fwd.push_back(x);
    }
    // inverse: decreasing axis order; inputs [outer Q_e>d][L_d][inner L_e<d]
    // (tile hybrid: [tile pair][L2][L1], the pair index outermost)
    pl->inv.clear();
    pl->inv_elems = 0;
    std::vector<int> inv_axes;
    for (int d : axes)
        if (!(pl->beams && d < 2) && !(pl->lag_pairs && d >= 2)) inv_axes.push_back(d);
    if (inv_axes.empty())
        return fail(OMNI_ERR_UNSUPPORTED, "a beam-space plan needs a coarser level with more than one block");
    for (size_t a = inv_axes.size(); a-- > 0;) {
        const int d = inv_axes[a];
        Pass p{};
        p.axis = d;
        p.L = g.Lp[d];
        p.n = g.Lp[d];
        p.q_out = 2 * g.n[d] - 1;
        p.q_shift = g.n[d] - 1;
        p.inner = 1;
        p.outer = 1;
        for (int e = 0; e < d; ++e) p.inner *= g.Lp[e];
        for (int e = d + 1; e < (pl->n_tiles ? 2 : g.D); ++e) p.outer *= 2 * g.n[e] - 1;
        if (pl->n_tiles) p.outer *= pl->n_tiles * pl->n_tiles;
        p.mode = (a == 0) ? MODE_INV_LAST : MODE_INV_MID;
        choose_kind(p);
        rows_lines(p);
        use_smem3(p, pl->knobs);
        if (p.mode == MODE_INV_MID) pl->inv_elems = std::max(pl->inv_elems, p.outer * p.q_out * p.inner);
        pl->inv.push_back(p);
    }
    double inv_points = 1.0;
    for (int d : inv_axes) inv_points *= (double)g.Lp[d];
    pl->inv_scale = 1.0 / inv_points;
    // direct-DFT twiddle tables w_L^m, m < L, computed in double
    for (auto* list : {&pl->fwd, &pl->inv})
        for (Pass& p : *list) {
            if (p.kind != KIND_DIRECT) continue;
            std::vector<float2> h(p.L);
            for (int m = 0; m < p.L; ++m) {
                const double ang = 6.283185307179586476925286766559 * m / p.L;
                h[m] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
            }
            float2* dptr = nullptr;
            OMNI_CUDA(cudaMalloc(&dptr, sizeof(float2) * p.L), "cudaMalloc(twiddles)");
            pl->tw_tables.push_back(dptr);
            OMNI_CUDA(cudaMemcpy(dptr, h.data(), sizeof(float2) * p.L, cudaMemcpyHostToDevice),
                      "cudaMemcpy(twiddles)");
            p.tw = dptr;
        }
    return OMNI_OK;
}

// Chunk sizes: the last pass gets one wave of resident CTAs (channels x inner
// tiles), and each scratch buffer holds about chunk_mb MB of samples (3072, the
// autotuner's pick on the 2-level workload for both paths; OMNI_CHUNK_MB overrides):
// long chunks amortise the FP64 fold and the launch ramp (measured on the
// 2-level workload, FP32 path: 96 MB 33.7 ms, 192 MB 26.6, 384 MB 22.6,
// 768 MB 21.3, 1536 MB 20.8 ms per step; correlate alone, tuner: 3072 MB 20.25 ms).
void choose_chunks(omni_plan* pl) {
    const int64_t mb = pl->knobs.chunk_mb;
    const int64_t target = mb << 20;
    // CTAs the last pass runs per channel of a chunk
    const Pass& last = pl->fwd.back();
    int64_t ctas = 1;
    switch (last.kind) {
        case KIND_LEVEL:
        case KIND_TC_B:
        case KIND_TC5_B:
        case KIND_SMEM:
        case KIND_SMEM3: ctas = (last.inner + last.W - 1) / last.W; break;
        case KIND_REG: ctas = (last.inner + 255) / 256; break;
        case KIND_XSPEC: ctas = xspec_ctas_per_channel(last); break;
        case KIND_XSPEC5:
        case KIND_COV5: ctas = xspec5_ctas_per_channel(last); break;
        default: ctas = (last.L * last.inner + 255) / 256; break;
    }
    // resident CTA slots of the GPU for that kernel
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device) != cudaSuccess) sms = 0;
    const int first_src = pl->fwd.size() == 1 ? (pl->dtype == OMNI_IN_CI8 ? SRC_CI8 : SRC_CF32) : SRC_BUF;
    if (last.kind == KIND_LEVEL && level_last_occupancy(last, first_src, &per_sm) != cudaSuccess) per_sm = 0;
    if (last.kind == KIND_SMEM && smem_last_occupancy(last, first_src, &per_sm) != cudaSuccess) per_sm = 0;
    if (last.kind == KIND_SMEM3 && smem3_last_occupancy(last, first_src, &per_sm) != cudaSuccess) per_sm = 0;
    if (last.kind == KIND_TC_B && tc_occupancy(KIND_TC_B, &per_sm) != cudaSuccess) per_sm = 0;
    if (last.kind == KIND_TC5_B && tc5_occupancy(&per_sm) != cudaSuccess) per_sm = 0;
    if (last.kind == KIND_XSPEC && xspec_occupancy(&per_sm) != cudaSuccess) per_sm = 0;
    if ((last.kind == KIND_XSPEC5 || last.kind == KIND_COV5) && xspec5_occupancy(&per_sm) != cudaSuccess)
        per_sm = 0;
    cudaGetLastError();
    int64_t slots = (int64_t)std::max(sms, 1) * std::max(per_sm, 2);
    if (sms <= 0) slots = 304;
    // fill one wave of the last pass: as many channels as the slots hold
    pl->Cc = std::min<int64_t>(pl->C, std::max<int64_t>(1, slots / ctas));
    const int64_t per_sample = std::max<int64_t>(1, pl->fwd_elems) * (int64_t)sizeof(float2);
    const bool gemm_last = last.kind == KIND_XSPEC5 || last.kind == KIND_COV5;
    if (gemm_last) {
        // one CTA per SM and a long accumulation per CTA (its epilogue costs several
        // of its 16-sample steps): 1024 samples per chunk, and channels per chunk
        // chosen so that the chunks' CTAs fill whole waves (256 CTAs per channel on
        // 152 SMs: 6-channel chunks run 10.1 waves in 11, 16-channel chunks 26.9 in
        // 27), within four times the chunk-buffer target (equal ties: fewer channels)
        const int64_t cap = 4 * target;
        pl->Tc = std::max<int64_t>(1, std::min<int64_t>(1024, cap / per_sample));
        const int64_t cmax = std::min<int64_t>(pl->C, std::max<int64_t>(1, cap / (per_sample * pl->Tc)));
        const int64_t sl = sms > 0 ? (int64_t)sms * std::max(per_sm, 1) : 152;  // one CTA per SM
        int64_t best = 1, best_waves = INT64_MAX;
        for (int64_t cc = 1; cc <= cmax; ++cc) {
            const int64_t n = (pl->C + cc - 1) / cc, cb = (pl->C + n - 1) / n, tail = pl->C - (n - 1) * cb;
            const int64_t waves = (n - 1) * ((cb * ctas + sl - 1) / sl) + (tail * ctas + sl - 1) / sl;
            if (waves < best_waves) best = cc, best_waves = waves;
        }
        pl->Cc = best;
    }
    if (pl->knobs.chunk_channels > 0) pl->Cc = std::min<int64_t>(pl->C, pl->knobs.chunk_channels);
    const int64_t samples = std::max<int64_t>(1, target / per_sample);
    if (!gemm_last) pl->Tc = std::max<int64_t>(1, std::min<int64_t>(1024, samples / pl->Cc));
    const int64_t per_chan = std::max<int64_t>(1, pl->inv_elems) * (int64_t)sizeof(float2);
    pl->Cv = std::min<int64_t>(pl->C, std::max<int64_t>(1, target / per_chan));
    pl->buf_elems = std::max(pl->Cc * pl->Tc * pl->fwd_elems, pl->Cv * pl->inv_elems);
    if (last.kind == KIND_XSPEC5 || last.kind == KIND_COV5)  // the second buffer also holds the transposed accumulator
        pl->buf_elems = std::max(pl->buf_elems, pl->Cv * acc_doubles(pl));
}

// After a stream synchronisation: report (and clear) an expired device wait.
omni_status check_device_error(omni_plan* pl) {
    if (!pl->dev_err) return OMNI_OK;
    int h = 0;
    OMNI_CUDA(cudaMemcpy(&h, pl->dev_err, sizeof(int), cudaMemcpyDeviceToHost), "reading the device error word");
    if (h) {
        cudaMemset(pl->dev_err, 0, sizeof(int));
        return fail(OMNI_ERR_TIMEOUT, "a bounded wait for a tensor-core operation expired; the "
                                      "accumulated visibilities are incomplete");
    }
    return OMNI_OK;
}

void release(omni_plan* pl) {
    for (omni_plan* sub : pl->members) release(sub);
    pl->members.clear();
    DeviceGuard dg(pl->device);
    if (pl->copy_stream) cudaStreamSynchronize(pl->copy_stream);
    cudaFree(pl->buf[0]);
    cudaFree(pl->buf[1]);
    cudaFree(pl->chan_max);
    cudaFree(pl->P);
    cudaFree(pl->dev_err);
    cudaFree(pl->vis_tmp);
    for (float2* t : pl->tw_tables) cudaFree(t);
    for (int b = 0; b < 2; ++b) {
        cudaFree(pl->stage[b]);
        if (pl->ready[b]) cudaEventDestroy(pl->ready[b]);
        if (pl->freed[b]) cudaEventDestroy(pl->freed[b]);
    }
    if (pl->copy_stream) cudaStreamDestroy(pl->copy_stream);
    if (pl->aux_stream) {
        cudaStreamSynchronize(pl->aux_stream);
        cudaStreamDestroy(pl->aux_stream);
    }
    if (pl->start_ev) cudaEventDestroy(pl->start_ev);
    if (pl->split_stream) {
        cudaStreamSynchronize(pl->split_stream);
        cudaStreamDestroy(pl->split_stream);
    }
    for (int b = 0; b < 2; ++b)
        if (pl->split_done[b]) cudaEventDestroy(pl->split_done[b]);
    for (int b = 0; b < 2; ++b) {
        if (pl->mid_done[b]) cudaEventDestroy(pl->mid_done[b]);
        if (pl->last_done[b]) cudaEventDestroy(pl->last_done[b]);
    }
    for (auto& q : pl->pending) {
        cudaEventDestroy(q.start);
        cudaEventDestroy(q.stop);
    }
    for (cudaEvent_t e : pl->event_pool) cudaEventDestroy(e);
    delete pl;
}

const char* kind_name(int k) {
    return k == KIND_REG ? "reg" : k == KIND_SMEM ? "smem" : k == KIND_SMEM3 ? "smem3x" : k == KIND_LEVEL ? "level"
         : k == KIND_TC_A || k == KIND_TC_B ? "tc" : k == KIND_TC5_B ? "tcgen05-"
         : k == KIND_XSPEC ? "xspec" : k == KIND_XSPEC5 ? "xspec-tcgen05-" : k == KIND_COV5 ? "lagsum-tcgen05-"
         : "direct";
}
const char* mode_name(int m) {
    return m == MODE_MID ? "mid" : m == MODE_LAST ? "last" : m == MODE_INV_MID ? "mid" : "last";
}

void init_stats(omni_plan* pl) {
    pl->stats.clear();
    for (int inv = 0; inv < 2; ++inv)
        for (const Pass& p : inv ? pl->inv : pl->fwd) {
            omni_kernel_stat st{};
            if (p.kind == KIND_LEVEL || p.kind == KIND_TC_A || p.kind == KIND_TC_B || p.kind == KIND_TC5_B)
                snprintf(st.name, sizeof st.name, "%s axis%d+%d %s%d %s", inv ? "inv" : "fwd", p.axis,
                         p.axis + 1, kind_name(p.kind), p.L, mode_name(p.mode));
            else
                snprintf(st.name, sizeof st.name, "%s axis%d %s%s%d %s", inv ? "inv" : "fwd", p.axis,
                         kind_name(p.kind), p.bf16 ? "bf16-" : "", p.L, mode_name(p.mode));
            st.tensor = (p.kind == KIND_TC_A || p.kind == KIND_TC_B || p.kind == KIND_TC5_B ||
                         p.kind == KIND_XSPEC5 || p.kind == KIND_COV5) ? 1 : 0;
            pl->stats.push_back(st);
        }
    if (pl->split) {  // the FP32 share of a split last pass
        omni_kernel_stat st{};
        snprintf(st.name, sizeof st.name, "fwd axis%d+%d level%d last (FP32 share)", pl->split_pass.axis,
                 pl->split_pass.axis + 1, pl->split_pass.L);
        pl->stats.push_back(st);
    }
}

cudaEvent_t pool_event(omni_plan* pl) {
    if (!pl->event_pool.empty()) {
        cudaEvent_t e = pl->event_pool.back();
        pl->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Input element size of a pass source, bytes.
double src_bytes(int src_kind) {
    return src_kind == SRC_CI8 ? 2.0 : src_kind == SRC_P64 ? 8.0 : 8.0;
}

// Algorithmic bytes of one launch: inputs read plus outputs written.
double pass_bytes(const Pass& p, const PassArgs& a) {
    if (p.kind == KIND_COV5)  // every block's level-1 spectrum once; the coarse-lag FP64 fold
        return (double)a.S * a.tc * p.outer * p.L * 8.0 +
               (double)a.S * p.L * (2.0 * p.L1 - 1) * (2.0 * p.L2 - 1) * 32.0;
    if (p.kind == KIND_XSPEC || p.kind == KIND_XSPEC5)  // every tile's spectrum once; the FP64 complex fold
        return (double)a.S * a.tc * p.outer * p.L * 8.0 + (double)a.S * p.outer * p.outer * p.L * 32.0;
    const double in = src_bytes(a.src_kind);
    const bool two_axes = p.kind == KIND_LEVEL || p.kind == KIND_TC_A || p.kind == KIND_TC_B ||
                          p.kind == KIND_TC5_B;
    const double n_in = two_axes ? (double)p.n * p.n : (double)p.n;
    switch (p.mode) {
        case MODE_MID:
            return (double)a.S * p.outer * p.inner * (n_in * in + p.q_out * 8.0);
        case MODE_LAST:
            return (double)a.S * a.tc * p.inner * n_in * in + (double)a.S * p.q_out * p.inner * 16.0;
        case MODE_INV_MID:
            return (double)a.S * p.outer * p.inner * (p.n * in + p.q_out * 8.0);
        default:
            return (double)a.S * p.outer * p.inner * (p.n * in + p.q_out * 16.0);
    }
}

// Algorithmic flops of one launch (see omni_kernel_stat).
double pass_flops(const Pass& p, const PassArgs& a) {
    const double lg = std::log2((double)std::max(p.L, 2));
    const double line = 5.0 * p.L * lg;
    switch (p.kind) {
        case KIND_XSPEC:  // one complex multiply-add per tile pair, frequency and sample
            return (double)a.S * a.tc * p.outer * p.outer * p.L * 8.0;
        case KIND_COV5:
        case KIND_XSPEC5:  // the same products in real form: 3 (FP16 split) or 6 (BF16) x (2 n_tiles)^2 MACs
            return (double)a.S * a.tc * p.L * (p.bf16 ? 6.0 : 3.0) * (2.0 * p.outer) * (2.0 * p.outer) * 2.0;
        case KIND_TC_A:  // per 16x16 block: 32 + 96 products
            return (double)a.S * p.outer * 128.0 * 4096.0;
        case KIND_TC_B:  // per level-1 frequency and sample: 6 + 12 products, |F|^2
        case KIND_TC5_B:  // the same products as 128x32x16 tiles (18 x 4096 per frequency)
            return (double)a.S * a.tc * p.inner * (18.0 * 4096.0 + 3.0 * p.q_out);
        case KIND_LEVEL: {
            const double per_unit = (double)p.n * line + (double)p.L * line;  // axis a, axis b
            if (p.mode == MODE_LAST)
                return (double)a.S * a.tc * p.inner * (per_unit + 3.0 * p.q_out);
            return (double)a.S * p.outer * p.inner * per_unit;
        }
        default: {
            const double lines = (p.mode == MODE_LAST) ? (double)a.S * a.tc * p.inner
                                                       : (double)a.S * p.outer * p.inner;
            const double extra = (p.mode == MODE_LAST) ? 3.0 * p.L : 0.0;
            const double per = p.kind == KIND_DIRECT ? 8.0 * p.n * p.q_out : line;
            return lines * (per + extra);
        }
    }
}

// Launch pass number idx (index into stats) with optional event timing.
cudaError_t launch_counted(omni_plan* pl, int idx, const Pass& p, const PassArgs& a,
                           cudaStream_t st) {
    omni_kernel_stat& s = pl->stats[idx];
    s.launches += 1;
    s.bytes += pass_bytes(p, a);
    s.flops += pass_flops(p, a);
    if (!pl->profiling) return launch_pass(p, a, st);
    cudaEvent_t e0 = pool_event(pl), e1 = pool_event(pl);
    if (!e0 || !e1) return cudaErrorMemoryAllocation;
    cudaEventRecord(e0, st);
    cudaError_t e = launch_pass(p, a, st);
    cudaEventRecord(e1, st);
    pl->pending.push_back({idx, e0, e1});
    return e;
}

// One chunk of forward passes: channels [c0, c0+cc) x samples [t0, t0+tc).
omni_status run_chunk(omni_plan* pl, const void* volts, int64_t vc0, int64_t Tsrc, int64_t t0,
                      int64_t c0, int64_t cc, int64_t tc, cudaStream_t st, int slot = -1) {
    const void* src = volts;
    int src_kind = pl->dtype == OMNI_IN_CI8 ? SRC_CI8 : SRC_CF32;
    int64_t src_stride = 0;
    // FP16 plans of float voltages: the chunk's per-channel max |x| (one slot per
    // overlapped chunk), measured before its first pass
    float* chan_max = pl->chan_max ? pl->chan_max + (slot >= 0 ? slot : 0) * pl->Cc : nullptr;
    for (size_t k = 0; k < pl->fwd.size(); ++k) {
        const Pass& p = pl->fwd[k];
        PassArgs a{};
        a.chan_max = chan_max;
        a.src = src;
        a.src_kind = src_kind;
        a.src_stride = src_stride;
        a.vc0 = vc0;
        a.T = Tsrc;
        a.t0 = t0;
        a.N = pl->g.N;
        a.tc = (int)tc;
        a.c0 = c0;
        a.P = pl->P;
        a.P_stride = acc_doubles(pl);
        a.err = pl->dev_err;
        a.force_expire = pl->force_expire;
        float2* dst = pl->buf[slot >= 0 ? slot : (int)(k & 1)];
        cudaStream_t launch_stream = st;
        if (slot >= 0 && p.mode == MODE_MID) {
            // first pass of an overlapped chunk: on the aux stream, after the last
            // pass that read this buffer two chunks ago
            launch_stream = pl->aux_stream;
            OMNI_CUDA(cudaStreamWaitEvent(launch_stream, pl->last_done[slot], 0), "cudaStreamWaitEvent");
        }
        if (k == 0 && chan_max) {
            cudaError_t e = launch_chan_absmax(volts, src_kind, vc0, Tsrc, t0, pl->g.N, cc, tc, chan_max,
                                               launch_stream);
            if (e != cudaSuccess) return cuda_fail(e, "channel scale launch");
        }
        if (p.mode == MODE_LAST) {
            a.S = cc;
        } else {
            a.S = cc * tc;
            a.dst = dst;
            a.dst_stride = p.outer * p.q_out * p.inner;
        }
        if (slot >= 0 && p.mode == MODE_LAST)
            OMNI_CUDA(cudaStreamWaitEvent(st, pl->mid_done[slot], 0), "cudaStreamWaitEvent");
        int64_t cc_split = 0;  // channels of this chunk that go through the FP32 last pass
        if (slot >= 0 && p.mode == MODE_LAST && pl->split && cc > 1) {
            cc_split = cc - std::max<int64_t>(1, std::min<int64_t>(cc - 1, (int64_t)(cc * pl->split_tc + 0.5)));
            const int64_t cc_tc = cc - cc_split;
            PassArgs b = a;
            b.S = cc_split;
            b.c0 = c0 + cc_tc;
            b.src = (const float2*)src + cc_tc * tc * src_stride;
            // the tensor-core first pass scales the spectra by 1/16, the FP32 one does not
            b.fold_scale = pl->fwd.front().kind == KIND_TC_A ? 256.0 : 1.0;
            a.S = cc_tc;
            OMNI_CUDA(cudaStreamWaitEvent(pl->split_stream, pl->mid_done[slot], 0), "cudaStreamWaitEvent");
            cudaError_t e2 = launch_counted(pl, (int)(pl->fwd.size() + pl->inv.size()), pl->split_pass, b,
                                            pl->split_stream);
            if (e2 != cudaSuccess) return cuda_fail(e2, "forward pass launch");
            OMNI_CUDA(cudaEventRecord(pl->split_done[slot], pl->split_stream), "cudaEventRecord");
        }
        cudaError_t e = launch_counted(pl, (int)k, p, a, launch_stream);
        if (e != cudaSuccess) return cuda_fail(e, "forward pass launch");
        if (cc_split > 0)
            OMNI_CUDA(cudaStreamWaitEvent(st, pl->split_done[slot], 0), "cudaStreamWaitEvent");
        if (slot >= 0)
            OMNI_CUDA(cudaEventRecord(p.mode == MODE_MID ? pl->mid_done[slot] : pl->last_done[slot],
                                      launch_stream), "cudaEventRecord");
        src = dst;
        src_kind = SRC_BUF;
        src_stride = p.outer * p.q_out * p.inner;
    }
    return OMNI_OK;
}

omni_status check_plan(omni_plan* pl) {
    if (!pl) return fail(OMNI_ERR_INVALID_ARG, "plan is NULL");
    return OMNI_OK;
}

omni_status run_inverse(omni_plan* pl, double2* V, cudaStream_t st) {
    // mixed tile plans and lag-sum plans accumulate [K][pair]; transposed to
    // [pair][K] per channel group
    const bool kmajor = pl->fwd.back().kind == KIND_XSPEC5 || pl->fwd.back().kind == KIND_COV5;
    const int64_t n_pairs = pl->lag_pairs ? pl->lag_pairs : pl->n_tiles * pl->n_tiles;
    for (int64_t c0 = 0; c0 < pl->C; c0 += pl->Cv) {
        const int64_t cv = std::min(pl->Cv, pl->C - c0);
        const void* src = pl->P;
        int src_kind = (pl->n_tiles || pl->lag_pairs) ? SRC_PC64 : SRC_P64;
        int64_t src_stride = (pl->n_tiles || pl->lag_pairs) ? acc_doubles(pl) / 2 : pl->g.L;
        if (kmajor) {
            const int64_t K = (int64_t)pl->g.Lp[0] * pl->g.Lp[1];
            cudaError_t e = launch_xspec5_transpose(pl->P + c0 * acc_doubles(pl), acc_doubles(pl), cv, K,
                                                    n_pairs, pl->buf[1], st);
            if (e != cudaSuccess) return cuda_fail(e, "accumulator transpose");
            // the passes index the source by channel c0 + s; the group starts at buf[1]
            src = reinterpret_cast<const void*>(reinterpret_cast<uintptr_t>(pl->buf[1]) -
                                                (uintptr_t)(c0 * src_stride * (int64_t)sizeof(double2)));
        }
        for (size_t k = 0; k < pl->inv.size(); ++k) {
            const Pass& p = pl->inv[k];
            PassArgs a{};
            a.src = src;
            a.src_kind = src_kind;
            a.src_stride = src_stride;
            a.S = cv;
            a.c0 = c0;
            a.tc = 1;
            float2* dst = pl->buf[k & 1];
            if (p.mode == MODE_INV_LAST) {
                a.V = V;
                a.V_stride = pl->g.Q;
                a.scale = pl->inv_scale;
            } else {
                a.dst = dst;
                a.dst_stride = p.outer * p.q_out * p.inner;
            }
            cudaError_t e = launch_counted(pl, (int)(pl->fwd.size() + k), p, a, st);
            if (e != cudaSuccess) return cuda_fail(e, "inverse pass launch");
            // later passes read the scratch buffer, indexed from 0 per channel of the
            // batch (c0 only offsets P and V)
            src = dst;
            src_kind = SRC_BUF;
            src_stride = p.outer * p.q_out * p.inner;
        }
    }
    return OMNI_OK;
}

}  // namespace

// ----------------------------------------------------------------------------- C ABI

extern "C" {

omni_status omni_lattice_shape(const omni_level* levels, int n_levels, int64_t* n_antennas,
                               int64_t* n_lags) {
    Geometry g;
    omni_status st = make_geometry(levels, n_levels, g);
    if (st != OMNI_OK) return st;
    if (n_antennas) *n_antennas = g.N;
    if (n_lags) *n_lags = g.Q;
    return OMNI_OK;
}

omni_status omni_baselines(const omni_level* levels, int n_levels, int32_t* dm, int64_t* redundancy,
                           double* dr) {
    Geometry g;
    omni_status st = make_geometry(levels, n_levels, g);
    if (st != OMNI_OK) return st;
    st = check_unique(g);
    if (st != OMNI_OK) return st;
    int32_t lag[kMaxDims];
    for (int d = 0; d < g.D; ++d) lag[d] = -(g.n[d] - 1);
    for (int64_t q = 0; q < g.Q; ++q) {
        int64_t red = 1;
        double x = 0.0, y = 0.0;
        for (int d = 0; d < g.D; ++d) {
            if (dm) dm[q * g.D + d] = lag[d];
            red *= g.n[d] - std::abs(lag[d]);
        }
        for (int k = 0; k < g.n_levels; ++k) {
            const double* a = &g.A[4 * k];
            x += a[0] * lag[2 * k] + a[1] * lag[2 * k + 1];
            y += a[2] * lag[2 * k] + a[3] * lag[2 * k + 1];
        }
        if (redundancy) redundancy[q] = red;
        if (dr) {
            dr[2 * q] = x;
            dr[2 * q + 1] = y;
        }
        for (int d = 0; d < g.D; ++d) {  // odometer, dimension 0 fastest
            if (++lag[d] <= g.n[d] - 1) break;
            lag[d] = -(g.n[d] - 1);
        }
    }
    return OMNI_OK;
}

omni_status omni_radial_bins(const omni_level* levels, int n_levels, double bin_width, int64_t n_bins,
                             int32_t* bin_of_lag, int64_t* pairs_per_bin) {
    if (!(bin_width > 0.0) || !std::isfinite(bin_width) || n_bins < 0)
        return fail(OMNI_ERR_INVALID_ARG, "bin_width must be > 0 and n_bins >= 0");
    int64_t N = 0, Q = 0;
    omni_status st = omni_lattice_shape(levels, n_levels, &N, &Q);
    if (st != OMNI_OK) return st;
    std::vector<int64_t> red(Q);
    std::vector<double> dr(2 * Q);
    if ((st = omni_baselines(levels, n_levels, nullptr, red.data(), dr.data())) != OMNI_OK) return st;
    if (pairs_per_bin) std::fill(pairs_per_bin, pairs_per_bin + n_bins, 0);
    for (int64_t q = 0; q < Q; ++q) {
        const double len = std::hypot(dr[2 * q], dr[2 * q + 1]);
        const double b = std::floor(len / bin_width);
        const int64_t bi = b < (double)n_bins ? (int64_t)b : -1;
        if (bin_of_lag) bin_of_lag[q] = (int32_t)bi;
        if (bi >= 0 && pairs_per_bin) pairs_per_bin[bi] += red[q];
    }
    return OMNI_OK;
}

omni_status omni_unique_baselines(const omni_level* levels, int n_levels, int64_t* n_unique,
                                  int32_t* group_of_lag, double* dr_unique, int64_t* pairs_unique) {
    if (!n_unique) return fail(OMNI_ERR_INVALID_ARG, "n_unique is NULL");
    int64_t N = 0, Q = 0;
    omni_status st = omni_lattice_shape(levels, n_levels, &N, &Q);
    if (st != OMNI_OK) return st;
    if (Q > INT32_MAX) return fail(OMNI_ERR_UNSUPPORTED, "too many lags for int32 group indices");
    std::vector<int64_t> red(Q);
    std::vector<double> dr(2 * Q);
    if ((st = omni_baselines(levels, n_levels, nullptr, red.data(), dr.data())) != OMNI_OK) return st;
    double rmax = 0.0;
    for (int64_t q = 0; q < Q; ++q) rmax = std::max(rmax, std::hypot(dr[2 * q], dr[2 * q + 1]));
    const double tol = 1e-9 * rmax;
    const double cell = tol > 0.0 ? tol : 1.0;
    // spatial hash of group representatives; each lag looks in the 3x3 cells around it
    struct Key {
        int64_t x, y;
        bool operator==(const Key& o) const { return x == o.x && y == o.y; }
    };
    struct KeyHash {
        size_t operator()(const Key& k) const {
            return std::hash<int64_t>()(k.x * 0x9E3779B97F4A7C15ULL ^ (uint64_t)k.y);
        }
    };
    std::unordered_map<Key, std::vector<int64_t>, KeyHash> grid;
    std::vector<double> rep;  // [group][2]
    std::vector<int64_t> pairs;
    for (int64_t q = 0; q < Q; ++q) {
        const double x = dr[2 * q], y = dr[2 * q + 1];
        const Key k{(int64_t)std::floor(x / cell), (int64_t)std::floor(y / cell)};
        int64_t found = -1;
        for (int64_t dx = -1; dx <= 1 && found < 0; ++dx)
            for (int64_t dy = -1; dy <= 1 && found < 0; ++dy) {
                auto it = grid.find(Key{k.x + dx, k.y + dy});
                if (it == grid.end()) continue;
                for (int64_t gi : it->second)
                    if (std::hypot(x - rep[2 * gi], y - rep[2 * gi + 1]) <= tol) {
                        found = gi;
                        break;
                    }
            }
        if (found < 0) {
            found = (int64_t)pairs.size();
            rep.push_back(x);
            rep.push_back(y);
            pairs.push_back(0);
            grid[k].push_back(found);
        }
        pairs[found] += red[q];
        if (group_of_lag) group_of_lag[q] = (int32_t)found;
    }
    *n_unique = (int64_t)pairs.size();
    for (size_t gi = 0; gi < pairs.size(); ++gi) {
        if (dr_unique) {
            dr_unique[2 * gi] = rep[2 * gi];
            dr_unique[2 * gi + 1] = rep[2 * gi + 1];
        }
        if (pairs_unique) pairs_unique[gi] = pairs[gi];
    }
    return OMNI_OK;
}

static omni_status create_plan(const omni_level* levels, int n_levels, int64_t n_channels,
                               omni_dtype dtype, omni_precision precision, const Knobs& knobs,
                               omni_plan** out, bool beams = false, int64_t n_tiles = 0,
                               const double* tile_offsets = nullptr);

omni_status omni_plan_create(const omni_level* levels, int n_levels, int64_t n_channels,
                             omni_dtype dtype, omni_precision precision, omni_plan** out) {
    return create_plan(levels, n_levels, n_channels, dtype, precision, knobs_from_env(), out);
}

omni_status omni_plan_create_beams(const omni_level* levels, int n_levels, int64_t n_channels,
                                   omni_dtype dtype, omni_plan** out) {
    return create_plan(levels, n_levels, n_channels, dtype, OMNI_FP32, knobs_from_env(), out, true);
}

// ---------------------------------------------------------------- autotuner

}  // extern "C"

namespace {

// Cache key: the problem (level shapes, precision, input type, channels,
// samples per call) and the device.
std::string tune_key(const Geometry& g, omni_precision precision, omni_dtype dtype, int64_t C,
                     int64_t T, int device) {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) prop.name[0] = 0;
    std::string k;
    for (int d = 0; d < g.D; ++d) k += std::to_string(g.n[d]) + (d + 1 < g.D ? "x" : "");
    k += "|p" + std::to_string((int)precision) + "|d" + std::to_string((int)dtype) + "|C" +
         std::to_string(C) + "|T" + std::to_string(T) + "|" + prop.name + "|v2";
    for (char& c : k)
        if (c == '"' || c == '\\' || c == '\n') c = '_';
    return k;
}

// One cache entry per line: {"key": "...", "chunk_mb": M, "chunk_channels": K,
// "overlap": O, "level_passes": L, "split_tc": S, "tc_stage_a": A, "ms": X}
bool tune_cache_read(const char* path, const std::string& key, Knobs& k) {
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    const std::string want = "\"key\": \"" + key + "\"";
    while (std::fgets(line, sizeof line, f)) {
        if (!std::strstr(line, want.c_str())) continue;
        Knobs t;
        long long mb = 0, ch = 0;
        int ov = 0, lp = 0;
        double sp = 0.0;
        const char* q = std::strstr(line, "\"chunk_mb\":");
        int sa = 0;
        if (!q || std::sscanf(q, "\"chunk_mb\": %lld, \"chunk_channels\": %lld, \"overlap\": %d, "
                                 "\"level_passes\": %d, \"split_tc\": %lf, \"tc_stage_a\": %d",
                              &mb, &ch, &ov, &lp, &sp, &sa) != 6)
            continue;
        t.chunk_mb = std::max<long long>(1, mb);
        t.chunk_channels = std::max<long long>(0, ch);
        t.overlap = ov != 0;
        t.level_passes = lp != 0;
        t.split_tc = sp;
        t.tc_stage_a = sa != 0;
        int f3 = 1;
        if (const char* r = std::strstr(line, "\"fft3\":")) std::sscanf(r, "\"fft3\": %d", &f3);
        t.fft3 = f3 != 0;
        k = t;
        found = true;  // the last matching line wins
    }
    std::fclose(f);
    return found;
}

void tune_cache_write(const char* path, const std::string& key, const Knobs& k, double ms) {
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"key\": \"%s\", \"chunk_mb\": %lld, \"chunk_channels\": %lld, \"overlap\": %d, "
                    "\"level_passes\": %d, \"split_tc\": %.3f, \"tc_stage_a\": %d, \"fft3\": %d, \"ms\": %.4f}\n",
                 key.c_str(), (long long)k.chunk_mb, (long long)k.chunk_channels, k.overlap, k.level_passes,
                 k.split_tc, k.tc_stage_a, k.fft3, ms);
    std::fclose(f);
}

}  // namespace

extern "C" {

omni_status omni_plan_create_tuned(const omni_level* levels, int n_levels, int64_t n_channels,
                                   omni_dtype dtype, omni_precision precision, const void* volts_dev,
                                   int64_t T, const char* cache_path, int* from_cache, omni_plan** out) {
    if (!out) return fail(OMNI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (from_cache) *from_cache = 0;
    if (!volts_dev || T < 1) return fail(OMNI_ERR_INVALID_ARG, "the tuner needs device voltages and T >= 1");
    Geometry g;
    omni_status st = make_geometry(levels, n_levels, g);
    if (st != OMNI_OK) return st;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return fail(OMNI_ERR_CUDA, "cudaGetDevice failed");
    const std::string key = tune_key(g, precision, dtype, n_channels, T, device);
    Knobs best;
    if (tune_cache_read(cache_path, key, best)) {
        if (from_cache) *from_cache = 1;
        return create_plan(levels, n_levels, n_channels, dtype, precision, best, out);
    }
    // candidates: chunk size x chunk overlap x level passes (FP32) or the
    // tensor-core / FP32 split of the last pass (mixed)
    std::vector<Knobs> cands;
    for (int64_t mb : {384, 768, 1536, 3072})
        for (int ov : {1, 0}) {
            if (precision == OMNI_MIXED_BF16) {
                Knobs k;
                k.chunk_mb = mb;
                k.overlap = ov;
                cands.push_back(k);
            } else if (precision == OMNI_MIXED_FP16) {
                for (int sa : {0, 1})
                    for (double sp : {0.0, 0.3, 0.6}) {
                        Knobs k;
                        k.chunk_mb = mb;
                        k.overlap = ov;
                        k.split_tc = sp;
                        k.tc_stage_a = sa;
                        if (sp > 0.0 && !ov) continue;  // the split needs the overlapped schedule
                        cands.push_back(k);
                    }
            } else {
                // FP32: level passes or one pass per axis, and for 2048/4096-point axes
                // the three- or four-step radix split
                bool long_axes = false;
                for (int d = 0; d < g.D; ++d) long_axes = long_axes || g.Lp[d] == 2048 || g.Lp[d] == 4096;
                for (int lp : {1, 0})
                    for (int f3 : {1, 0}) {
                        if (!long_axes && f3 == 0) continue;
                        Knobs k;
                        k.chunk_mb = mb;
                        k.overlap = ov;
                        k.level_passes = lp;
                        k.fft3 = f3;
                        cands.push_back(k);
                    }
            }
        }
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (stream) cudaStreamDestroy(stream);
        if (e0) cudaEventDestroy(e0);
        return fail(OMNI_ERR_CUDA, "tuner stream/events");
    }
    double best_ms = -1.0;
    omni_status last_err = OMNI_OK;
    for (const Knobs& k : cands) {
        omni_plan* pl = nullptr;
        st = create_plan(levels, n_levels, n_channels, dtype, precision, k, &pl);
        if (st != OMNI_OK) {  // e.g. a chunk size that does not fit: skip it
            last_err = st;
            cudaGetLastError();
            continue;
        }
        float ms = 0.f;
        st = omni_correlate(pl, volts_dev, T, stream);  // warm-up
        if (st == OMNI_OK) {
            cudaEventRecord(e0, stream);
            for (int r = 0; r < 2 && st == OMNI_OK; ++r) st = omni_correlate(pl, volts_dev, T, stream);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                st = OMNI_ERR_CUDA;
        }
        if (st == OMNI_OK) st = check_device_error(pl);
        omni_plan_destroy(pl);
        if (st != OMNI_OK) {
            last_err = st;
            continue;
        }
        if (best_ms < 0.0 || ms / 2.0 < best_ms) {
            best_ms = ms / 2.0;
            best = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(stream);
    if (best_ms < 0.0)
        return last_err != OMNI_OK ? last_err : fail(OMNI_ERR_UNSUPPORTED, "no tuner candidate ran");
    tune_cache_write(cache_path, key, best, best_ms);
    return create_plan(levels, n_levels, n_channels, dtype, precision, best, out);
}

omni_status omni_plan_knobs(const omni_plan* pl, int64_t* chunk_mb, int* overlap, int* level_passes,
                            double* split_tc) {
    if (!pl) return fail(OMNI_ERR_INVALID_ARG, "plan is NULL");
    const omni_plan* q = pl->members.empty() ? pl : pl->members.front();
    if (chunk_mb) *chunk_mb = q->knobs.chunk_mb;
    if (overlap) *overlap = q->overlap ? 1 : 0;
    if (level_passes) *level_passes = q->knobs.level_passes;
    if (split_tc) *split_tc = q->split ? q->split_tc : 0.0;
    return OMNI_OK;
}

int64_t omni_fengine_scratch_bytes(int64_t n_antennas, int64_t n_samples, int32_t n_channels,
                                   int32_t taps) {
    if (n_antennas < 1 || n_channels < 1 || taps < 1) return 0;
    return fengine_scratch_bytes(n_antennas, n_samples, n_channels, taps);
}

omni_status omni_fengine(const int8_t* raw_dev, int64_t n_antennas, int64_t n_samples,
                         int32_t n_channels, int32_t taps, const float* window_dev,
                         const float* gains_dev, float scale, omni_dtype out_dtype, void* out_dev,
                         void* scratch_dev, int64_t scratch_bytes, int64_t* n_frames, void* stream) {
    const int64_t F = n_channels;
    if (n_antennas < 1 || n_samples < 0) return fail(OMNI_ERR_INVALID_ARG, "need n_antennas >= 1, n_samples >= 0");
    if (F < 2 || F > 4096 || !is_pow2(F))
        return fail(OMNI_ERR_INVALID_ARG, "n_channels must be a power of two in [2, 4096], got %d", n_channels);
    if (taps < 1 || taps > 64) return fail(OMNI_ERR_INVALID_ARG, "taps must be in [1, 64], got %d", taps);
    if (out_dtype != OMNI_IN_CI8 && out_dtype != OMNI_IN_CF32)
        return fail(OMNI_ERR_INVALID_ARG, "unknown output dtype %d", (int)out_dtype);
    const int64_t T = fengine_frames(n_samples, n_channels, taps);
    if (n_frames) *n_frames = T;
    if (T == 0) return OMNI_OK;  // fewer samples than one frame: nothing to write
    const int64_t need = omni_fengine_scratch_bytes(n_antennas, n_samples, n_channels, taps);
    if (!raw_dev || !out_dev || (need > 0 && !scratch_dev))
        return fail(OMNI_ERR_INVALID_ARG, "NULL raw, out or scratch");
    if ((uintptr_t)out_dev % (out_dtype == OMNI_IN_CI8 ? 2 : 8) || (uintptr_t)scratch_dev % 8 ||
        (gains_dev && (uintptr_t)gains_dev % 8) || (window_dev && (uintptr_t)window_dev % 4))
        return fail(OMNI_ERR_INVALID_ARG, "misaligned out, scratch, gains or window pointer");
    if (scratch_bytes < need)
        return fail(OMNI_ERR_INVALID_ARG, "scratch holds %lld bytes, need %lld", (long long)scratch_bytes,
                    (long long)need);
    if (fengine_ctas(n_antennas, T, n_channels) > INT32_MAX)
        return fail(OMNI_ERR_INVALID_ARG, "launch too large: split the antennas or the samples");
    cudaError_t e = launch_fengine(raw_dev, n_antennas, n_samples, n_channels, taps, window_dev,
                                   reinterpret_cast<const float2*>(gains_dev), scale,
                                   out_dtype == OMNI_IN_CI8, out_dev, reinterpret_cast<float2*>(scratch_dev),
                                   (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "F-engine launch");
    return OMNI_OK;
}

omni_status omni_plan_create_tiles(const omni_level* tile, int64_t n_tiles, const double* offsets,
                                   int64_t n_channels, omni_dtype dtype, omni_precision precision,
                                   omni_plan** out) {
    if (n_tiles < 1) return fail(OMNI_ERR_INVALID_ARG, "n_tiles must be >= 1");
    if (!offsets) return fail(OMNI_ERR_INVALID_ARG, "offsets is NULL");
    if (n_tiles > 4096) return fail(OMNI_ERR_UNSUPPORTED, "at most 4096 tiles");
    return create_plan(tile, 1, n_channels, dtype, precision, knobs_from_env(), out, false, n_tiles, offsets);
}

static omni_status create_plan(const omni_level* levels, int n_levels, int64_t n_channels,
                               omni_dtype dtype, omni_precision precision, const Knobs& knobs,
                               omni_plan** out, bool beams, int64_t n_tiles,
                               const double* tile_offsets) {
    if (!out) return fail(OMNI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_channels < 1) return fail(OMNI_ERR_INVALID_ARG, "n_channels must be >= 1");
    if (dtype != OMNI_IN_CF32 && dtype != OMNI_IN_CI8) return fail(OMNI_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if (precision != OMNI_FP32 && precision != OMNI_MIXED_FP16 && precision != OMNI_MIXED_BF16)
        return fail(OMNI_ERR_INVALID_ARG, "unknown precision %d", (int)precision);
    if (beams && precision != OMNI_FP32)
        return fail(OMNI_ERR_UNSUPPORTED, "beam-space plans run the FP32 path");
    if (beams && levels && n_levels < 2)
        return fail(OMNI_ERR_UNSUPPORTED, "a beam-space plan needs at least two levels");
    omni_plan* pl = new omni_plan();
    pl->beams = beams;
    pl->n_tiles = n_tiles;
    pl->knobs = knobs;
    omni_status st = make_geometry(levels, n_levels, pl->g, beams);
    if (st == OMNI_OK) st = n_tiles ? tile_geometry(pl->g, n_tiles, tile_offsets) : check_unique(pl->g);
    if (st != OMNI_OK) {
        delete pl;
        return st;
    }
    if (n_tiles && precision != OMNI_FP32 &&
        !xspec5_supports(n_tiles, (int64_t)pl->g.Lp[0] * pl->g.Lp[1])) {
        delete pl;
        return fail(OMNI_ERR_UNSUPPORTED,
                    "mixed-precision tile-hybrid plans support at most 64 tiles whose padded "
                    "lattice size is a multiple of 4");
    }
    if (!n_tiles && precision != OMNI_FP32 &&
        !(pl->g.D == 4 && (int64_t)pl->g.n[2] * pl->g.n[3] <= 64 &&
          xspec5_supports((int64_t)pl->g.n[2] * pl->g.n[3], (int64_t)pl->g.Lp[0] * pl->g.Lp[1]))) {
        delete pl;
        return fail(OMNI_ERR_UNSUPPORTED,
                    "the mixed-precision path supports 2-level hierarchies of at most 64 level-1 "
                    "blocks whose padded level-1 lattice size is a multiple of 4");
    }
    pl->C = n_channels;
    pl->dtype = dtype;
    pl->precision = precision;
    if (const char* env = std::getenv("OMNI_TEST_FORCE_TIMEOUT")) pl->force_expire = std::atoi(env) != 0;
    cudaError_t e = cudaGetDevice(&pl->device);
    if (e != cudaSuccess) {
        delete pl;
        return cuda_fail(e, "cudaGetDevice");
    }
    e = init_device_tables();
    if (e != cudaSuccess) {
        delete pl;
        return cuda_fail(e, "twiddle table upload");
    }
    st = build_passes(pl);
    if (st != OMNI_OK) {
        release(pl);
        return st;
    }
    choose_chunks(pl);
    // overlap the two passes of consecutive chunks (OMNI_OVERLAP=0 turns it off)
    {
        const int lk = pl->fwd.back().kind;
        const bool gemm_last = lk == KIND_COV5 || lk == KIND_XSPEC5;
        pl->overlap = pl->fwd.size() == 2 && (pl->knobs.overlap > 0 || (pl->knobs.overlap < 0 && !gemm_last));
    }
    if (pl->overlap) {
        if ((e = cudaStreamCreateWithFlags(&pl->aux_stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&pl->start_ev, cudaEventDisableTiming)) != cudaSuccess) {
            release(pl);
            return cuda_fail(e, "creating the overlap stream");
        }
        for (int b = 0; b < 2; ++b)
            if ((e = cudaEventCreateWithFlags(&pl->mid_done[b], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&pl->last_done[b], cudaEventDisableTiming)) != cudaSuccess) {
                release(pl);
                return cuda_fail(e, "creating the overlap events");
            }
    }
    // mixed plans: split each chunk's last pass between tensor cores and CUDA cores
    if (pl->overlap && pl->precision == OMNI_MIXED_FP16 && pl->fwd.back().kind == KIND_TC_B) {
        // fraction of a chunk's channels on tensor cores (off by default: with
        // 768 MB chunks on the 2-level workload, no split 22.56 ms, 0.6 22.47,
        // 0.3 24.07 ms per step -- both kernels are issue-limited)
        const double frac = pl->knobs.split_tc;
        if (frac < 1.0 && frac > 0.0) {
            const Pass& last = pl->fwd.back();
            Pass sp{};
            sp.axis = last.axis;
            sp.mode = MODE_LAST;
            sp.L = last.L;
            sp.n = last.n;
            sp.q_out = last.q_out;
            sp.inner = last.inner;
            sp.outer = 1;
            choose_level(sp);
            pl->split_pass = sp;
            pl->split_tc = frac;
            if ((e = cudaStreamCreateWithFlags(&pl->split_stream, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&pl->split_done[0], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&pl->split_done[1], cudaEventDisableTiming)) != cudaSuccess) {
                release(pl);
                return cuda_fail(e, "creating the split stream");
            }
            pl->split = true;
        }
    }
    // persistent finest-level passes: one wave of resident CTAs
    for (size_t k = 0; k < pl->fwd.size(); ++k) {
        Pass& p = pl->fwd[k];
        if (p.kind == KIND_TC_A) {
            int per_sm = 0, sms = 0;
            if (tc_occupancy(KIND_TC_A, &per_sm) == cudaSuccess &&
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device) == cudaSuccess)
                p.grid_cap = per_sm * sms;
            cudaGetLastError();
            continue;
        }
        if (p.kind != KIND_LEVEL || p.mode != MODE_MID || p.inner != 1) continue;
        const int src = k == 0 ? (pl->dtype == OMNI_IN_CI8 ? SRC_CI8 : SRC_CF32) : SRC_BUF;
        int per_sm = 0, sms = 0;
        if (level_stream_occupancy(p, src, &per_sm) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device) == cudaSuccess)
            p.grid_cap = per_sm * sms;
        cudaGetLastError();
    }
    init_stats(pl);
    const size_t buf_bytes = (size_t)std::max<int64_t>(1, pl->buf_elems) * sizeof(float2);
    const size_t P_bytes = (size_t)pl->C * acc_doubles(pl) * sizeof(double);
    bool data_scale = false;
    for (const Pass& q : pl->fwd) data_scale = data_scale || (q.scale_n > 0 && !q.bf16);
    if (data_scale && (e = cudaMalloc(&pl->chan_max, (size_t)2 * pl->Cc * sizeof(float))) != cudaSuccess) {
        release(pl);
        return cuda_fail(e, "cudaMalloc");
    }
    if ((e = cudaMalloc(&pl->buf[0], buf_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&pl->buf[1], buf_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&pl->P, P_bytes)) != cudaSuccess ||
        (e = cudaMemset(pl->P, 0, P_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&pl->dev_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(pl->dev_err, 0, sizeof(int))) != cudaSuccess) {
        release(pl);
        return cuda_fail(e, "allocating plan buffers");
    }
    *out = pl;
    return OMNI_OK;
}

omni_status omni_plan_create_batch(const omni_level* const* levels_per_array,
                                   const int* n_levels_per_array, int n_arrays, int64_t n_channels,
                                   omni_dtype dtype, omni_precision precision, omni_plan** out) {
    if (!out) return fail(OMNI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!levels_per_array || !n_levels_per_array || n_arrays < 1)
        return fail(OMNI_ERR_INVALID_ARG, "need n_arrays >= 1 and non-NULL level lists");
    if (n_channels < 1) return fail(OMNI_ERR_INVALID_ARG, "n_channels must be >= 1");
    std::vector<Geometry> geos(n_arrays);
    for (int a = 0; a < n_arrays; ++a) {
        omni_status st = make_geometry(levels_per_array[a], n_levels_per_array[a], geos[a]);
        if (st == OMNI_OK) st = check_unique(geos[a]);
        if (st != OMNI_OK) {
            fail(st, "array %d: %s", a, omni_last_error());
            return st;
        }
    }
    omni_plan* pl = new omni_plan();
    pl->C = n_channels;
    pl->dtype = dtype;
    pl->precision = precision;
    cudaGetDevice(&pl->device);
    for (int a = 0; a < n_arrays; ++a) {
        pl->array_antennas.push_back(geos[a].N);
        pl->array_lags.push_back(geos[a].Q);
    }
    auto same_shape = [&](int x, int y) {
        if (geos[x].D != geos[y].D) return false;
        for (int d = 0; d < geos[x].D; ++d)
            if (geos[x].n[d] != geos[y].n[d]) return false;
        return true;
    };
    for (int a = 0; a < n_arrays;) {
        int b = a + 1;
        while (b < n_arrays && same_shape(a, b)) ++b;
        omni_plan* sub = nullptr;
        omni_status st = create_plan(levels_per_array[a], n_levels_per_array[a],
                                     (int64_t)(b - a) * n_channels, dtype, precision, knobs_from_env(), &sub);
        if (st != OMNI_OK) {
            release(pl);
            return st;
        }
        pl->members.push_back(sub);
        pl->member_arrays.push_back(b - a);
        a = b;
    }
    *out = pl;
    return OMNI_OK;
}

omni_status omni_batch_info(const omni_plan* pl, int* n_arrays, int64_t* antennas, int64_t* lags) {
    if (!pl) return fail(OMNI_ERR_INVALID_ARG, "plan is NULL");
    if (pl->members.empty()) {
        if (n_arrays) *n_arrays = 1;
        if (antennas) antennas[0] = pl->g.N;
        if (lags) lags[0] = pl->g.Q;
        return OMNI_OK;
    }
    if (n_arrays) *n_arrays = (int)pl->array_antennas.size();
    for (size_t a = 0; a < pl->array_antennas.size(); ++a) {
        if (antennas) antennas[a] = pl->array_antennas[a];
        if (lags) lags[a] = pl->array_lags[a];
    }
    return OMNI_OK;
}

void omni_plan_destroy(omni_plan* plan) {
    if (plan) release(plan);
}

omni_status omni_plan_info(const omni_plan* pl, int* n_dims, int32_t* dims, int32_t* padded,
                           int64_t* n_antennas, int64_t* n_lags, int64_t* n_channels) {
    if (!pl) return fail(OMNI_ERR_INVALID_ARG, "plan is NULL");
    if (!pl->members.empty()) {
        int64_t N = 0, Q = 0;
        for (size_t a = 0; a < pl->array_antennas.size(); ++a) {
            N += pl->array_antennas[a];
            Q += pl->array_lags[a];
        }
        if (n_dims) *n_dims = 0;
        if (n_antennas) *n_antennas = N;
        if (n_lags) *n_lags = Q;
        if (n_channels) *n_channels = pl->C;
        return OMNI_OK;
    }
    if (n_dims) *n_dims = pl->g.D;
    for (int d = 0; d < pl->g.D; ++d) {
        if (dims) dims[d] = pl->g.n[d];
        if (padded) padded[d] = pl->g.Lp[d];
    }
    if (n_antennas) *n_antennas = pl->g.N;
    if (n_lags) *n_lags = pl->g.Q;
    if (n_channels) *n_channels = pl->C;
    return OMNI_OK;
}

omni_status omni_correlate(omni_plan* pl, const void* volts_dev, int64_t T, void* stream) {
    omni_status st = check_plan(pl);
    if (st != OMNI_OK) return st;
    if (!pl->members.empty()) {
        if (T < 0) return fail(OMNI_ERR_INVALID_ARG, "T must be >= 0");
        const char* p = (const char*)volts_dev;
        for (size_t m = 0; m < pl->members.size(); ++m) {
            omni_plan* sub = pl->members[m];
            if ((st = omni_correlate(sub, p, T, stream)) != OMNI_OK) return st;
            p += (size_t)sub->C * T * sub->g.N * elem_bytes(sub->dtype);
        }
        return OMNI_OK;
    }
    if (T < 0) return fail(OMNI_ERR_INVALID_ARG, "T must be >= 0");
    if (T == 0) return OMNI_OK;
    if (!volts_dev) return fail(OMNI_ERR_INVALID_ARG, "volts_dev is NULL");
    if ((uintptr_t)volts_dev % elem_bytes(pl->dtype) != 0)
        return fail(OMNI_ERR_INVALID_ARG, "volts_dev must be aligned to its element size");
    if (pl->fwd.front().kind == KIND_TC_A && (uintptr_t)volts_dev % 16 != 0)
        return fail(OMNI_ERR_INVALID_ARG, "mixed-precision plans need 16-byte aligned volts_dev");
    DeviceGuard dg(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (pl->overlap) {
        // the aux stream starts after everything already queued on the caller's stream
        OMNI_CUDA(cudaEventRecord(pl->start_ev, s), "cudaEventRecord");
        OMNI_CUDA(cudaStreamWaitEvent(pl->aux_stream, pl->start_ev, 0), "cudaStreamWaitEvent");
        if (pl->split)
            OMNI_CUDA(cudaStreamWaitEvent(pl->split_stream, pl->start_ev, 0), "cudaStreamWaitEvent");
        for (int b = 0; b < 2; ++b) OMNI_CUDA(cudaEventRecord(pl->last_done[b], s), "cudaEventRecord");
    }
    // equal-sized chunks (no short tail chunk paying a whole fold and launch)
    const int64_t Cb = ceil_div(pl->C, ceil_div(pl->C, pl->Cc));
    const int64_t Tb = ceil_div(T, ceil_div(T, pl->Tc));
    int64_t j = 0;
    for (int64_t c0 = 0; c0 < pl->C; c0 += Cb) {
        const int64_t cc = std::min(Cb, pl->C - c0);
        for (int64_t t0 = 0; t0 < T; t0 += Tb, ++j) {
            const int64_t tc = std::min(Tb, T - t0);
            st = run_chunk(pl, volts_dev, c0, T, t0, c0, cc, tc, s, pl->overlap ? (int)(j & 1) : -1);
            if (st != OMNI_OK) return st;
        }
    }
    return OMNI_OK;
}

omni_status omni_correlate_host(omni_plan* pl, const void* volts_host, int64_t T, void* stream) {
    omni_status st = check_plan(pl);
    if (st != OMNI_OK) return st;
    if (!pl->members.empty()) {
        if (T < 0) return fail(OMNI_ERR_INVALID_ARG, "T must be >= 0");
        const char* p = (const char*)volts_host;
        for (size_t m = 0; m < pl->members.size(); ++m) {
            omni_plan* sub = pl->members[m];
            if ((st = omni_correlate_host(sub, p, T, stream)) != OMNI_OK) return st;
            p += (size_t)sub->C * T * sub->g.N * elem_bytes(sub->dtype);
        }
        return OMNI_OK;
    }
    if (T < 0) return fail(OMNI_ERR_INVALID_ARG, "T must be >= 0");
    if (T == 0) return OMNI_OK;
    if (!volts_host) return fail(OMNI_ERR_INVALID_ARG, "volts_host is NULL");
    DeviceGuard dg(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t eb = (size_t)elem_bytes(pl->dtype);
    const size_t row = (size_t)pl->g.N * eb;  // one sample of one channel
    const size_t need = (size_t)pl->Cc * pl->Tc * row;
    if (pl->stage_bytes < need) {
        OMNI_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        for (int b = 0; b < 2; ++b) {
            cudaFree(pl->stage[b]);
            pl->stage[b] = nullptr;
        }
        pl->stage_bytes = 0;
        for (int b = 0; b < 2; ++b) OMNI_CUDA(cudaMalloc(&pl->stage[b], need), "cudaMalloc(staging)");
        pl->stage_bytes = need;
    }
    if (!pl->copy_stream) {
        OMNI_CUDA(cudaStreamCreateWithFlags(&pl->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        for (int b = 0; b < 2; ++b) {
            OMNI_CUDA(cudaEventCreateWithFlags(&pl->ready[b], cudaEventDisableTiming), "cudaEventCreate");
            OMNI_CUDA(cudaEventCreateWithFlags(&pl->freed[b], cudaEventDisableTiming), "cudaEventCreate");
        }
    }
    // copies of chunk j must wait for the compute stream to have consumed the
    // staging buffer of chunk j-2 ('freed'); compute waits for 'ready'.
    OMNI_CUDA(cudaEventRecord(pl->freed[0], s), "cudaEventRecord");
    OMNI_CUDA(cudaEventRecord(pl->freed[1], s), "cudaEventRecord");
    if (pl->overlap) {
        // as in omni_correlate: the first pass of chunk j+1 (auxiliary stream)
        // overlaps the last pass of chunk j; the auxiliary streams start after
        // everything already queued on the caller's stream
        OMNI_CUDA(cudaEventRecord(pl->start_ev, s), "cudaEventRecord");
        OMNI_CUDA(cudaStreamWaitEvent(pl->aux_stream, pl->start_ev, 0), "cudaStreamWaitEvent");
        if (pl->split)
            OMNI_CUDA(cudaStreamWaitEvent(pl->split_stream, pl->start_ev, 0), "cudaStreamWaitEvent");
        for (int b = 0; b < 2; ++b) OMNI_CUDA(cudaEventRecord(pl->last_done[b], s), "cudaEventRecord");
    }
    // chunks growing from a quarter of the plan's chunk: nothing overlaps the
    // first chunk's copy, and each next copy (host copies ran at 210 GB/s, about
    // three quarters of the transforms' rate on the 2-level workload) must fit in
    // the previous chunk's transforms, so the channel count grows by 30% a chunk
    const int64_t Cb = ceil_div(pl->C, ceil_div(pl->C, pl->Cc));
    const int64_t Tb = ceil_div(T, ceil_div(T, pl->Tc));
    int64_t next = std::max<int64_t>(1, Cb / 4);
    int64_t j = 0;
    for (int64_t c0 = 0; c0 < pl->C;) {
        const int64_t cc = std::min(next, pl->C - c0);
        next = std::min<int64_t>(Cb, std::max<int64_t>(next + 1, (next * 13 + 9) / 10));
        for (int64_t t0 = 0; t0 < T; t0 += Tb, ++j) {
            const int64_t tc = std::min(Tb, T - t0);
            const int b = (int)(j & 1);
            OMNI_CUDA(cudaStreamWaitEvent(pl->copy_stream, pl->freed[b], 0), "cudaStreamWaitEvent");
            for (int64_t k = 0; k < cc; ++k) {
                const char* hsrc = (const char*)volts_host + ((size_t)(c0 + k) * T + t0) * row;
                char* ddst = (char*)pl->stage[b] + (size_t)k * tc * row;
                OMNI_CUDA(cudaMemcpyAsync(ddst, hsrc, (size_t)tc * row, cudaMemcpyHostToDevice, pl->copy_stream),
                          "cudaMemcpyAsync(H2D)");
            }
            OMNI_CUDA(cudaEventRecord(pl->ready[b], pl->copy_stream), "cudaEventRecord");
            // the first pass reads the staging buffer: on the auxiliary stream when overlapped
            OMNI_CUDA(cudaStreamWaitEvent(pl->overlap ? pl->aux_stream : s, pl->ready[b], 0),
                      "cudaStreamWaitEvent");
            st = run_chunk(pl, pl->stage[b], 0, tc, 0, c0, cc, tc, s, pl->overlap ? b : -1);
            if (st != OMNI_OK) return st;
            OMNI_CUDA(cudaEventRecord(pl->freed[b], s), "cudaEventRecord");
        }
        c0 += cc;
    }
    OMNI_CUDA(cudaStreamSynchronize(pl->copy_stream), "cudaStreamSynchronize(copy)");
    return OMNI_OK;
}

omni_status omni_visibilities(omni_plan* pl, double* vis_dev, int reset, void* stream) {
    omni_status st = check_plan(pl);
    if (st != OMNI_OK) return st;
    if (!pl->members.empty()) {
        double* v = vis_dev;
        for (omni_plan* sub : pl->members) {
            if ((st = omni_visibilities(sub, v, reset, stream)) != OMNI_OK) return st;
            v += 2 * sub->C * sub->g.Q;
        }
        return OMNI_OK;
    }
    if (!vis_dev) return fail(OMNI_ERR_INVALID_ARG, "vis_dev is NULL");
    if ((uintptr_t)vis_dev % 16 != 0) return fail(OMNI_ERR_INVALID_ARG, "vis_dev must be 16-byte aligned");
    DeviceGuard dg(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    st = run_inverse(pl, reinterpret_cast<double2*>(vis_dev), s);
    if (st != OMNI_OK) return st;
    if (reset) OMNI_CUDA(cudaMemsetAsync(pl->P, 0, (size_t)pl->C * acc_doubles(pl) * sizeof(double), s), "cudaMemsetAsync");
    OMNI_CUDA(cudaStreamSynchronize(s), "device error during correlation");
    return check_device_error(pl);
}

omni_status omni_visibilities_host(omni_plan* pl, double* vis_host, int reset, void* stream) {
    omni_status st = check_plan(pl);
    if (st != OMNI_OK) return st;
    if (!pl->members.empty()) {
        double* v = vis_host;
        for (omni_plan* sub : pl->members) {
            if ((st = omni_visibilities_host(sub, v, reset, stream)) != OMNI_OK) return st;
            v += 2 * sub->C * sub->g.Q;
        }
        return OMNI_OK;
    }
    if (!vis_host) return fail(OMNI_ERR_INVALID_ARG, "vis_host is NULL");
    DeviceGuard dg(pl->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)pl->C * pl->g.Q * sizeof(double2);
    if (!pl->vis_tmp) OMNI_CUDA(cudaMalloc(&pl->vis_tmp, bytes), "cudaMalloc(visibility staging)");
    st = run_inverse(pl, pl->vis_tmp, s);
    if (st != OMNI_OK) return st;
    if (reset) OMNI_CUDA(cudaMemsetAsync(pl->P, 0, (size_t)pl->C * acc_doubles(pl) * sizeof(double), s), "cudaMemsetAsync");
    OMNI_CUDA(cudaMemcpyAsync(vis_host, pl->vis_tmp, bytes, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(D2H)");
    OMNI_CUDA(cudaStreamSynchronize(s), "device error during correlation");
    return check_device_error(pl);
}

omni_status omni_reset(omni_plan* pl, void* stream) {
    omni_status st = check_plan(pl);
    if (st != OMNI_OK) return st;
    if (!pl->members.empty()) {
        for (omni_plan* sub : pl->members)
            if ((st = omni_reset(sub, stream)) != OMNI_OK) return st;
        return OMNI_OK;
    }
    DeviceGuard dg(pl->device);
    OMNI_CUDA(cudaMemsetAsync(pl->P, 0, (size_t)pl->C * acc_doubles(pl) * sizeof(double), (cudaStream_t)stream),
              "cudaMemsetAsync");
    return OMNI_OK;
}

omni_status omni_sync(omni_plan* pl, void* stream) {
    omni_status st = check_plan(pl);
    if (st != OMNI_OK) return st;
    DeviceGuard dg(pl->device);
    OMNI_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "device error");
    for (omni_plan* sub : pl->members)
        if ((st = check_device_error(sub)) != OMNI_OK) return st;
    return check_device_error(pl);
}

omni_status omni_profile_enable(omni_plan* pl, int enable) {
    omni_status st = check_plan(pl);
    if (st != OMNI_OK) return st;
    for (omni_plan* sub : pl->members)
        if ((st = omni_profile_enable(sub, enable)) != OMNI_OK) return st;
    pl->profiling = enable != 0;
    return OMNI_OK;
}

omni_status omni_profile_read(omni_plan* pl, omni_kernel_stat* out, int max, int* n_out, int clear) {
    omni_status st = check_plan(pl);
    if (st != OMNI_OK) return st;
    if (!pl->members.empty()) {
        // members' statistics one after another, names prefixed with the member index
        int total = 0;
        for (size_t m = 0; m < pl->members.size(); ++m) {
            int n = 0;
            const int room = std::max(0, max - total);
            if ((st = omni_profile_read(pl->members[m], out ? out + std::min(total, max) : nullptr, room,
                                        &n, clear)) != OMNI_OK)
                return st;
            if (out)
                for (int i = total; i < std::min(total + n, max); ++i) {
                    char buf[64];
                    snprintf(buf, sizeof buf, "a%zu %s", m, out[i].name);
                    memcpy(out[i].name, buf, sizeof buf);
                }
            total += n;
        }
        if (n_out) *n_out = total;
        return OMNI_OK;
    }
    DeviceGuard dg(pl->device);
    for (auto& q : pl->pending) {
        OMNI_CUDA(cudaEventSynchronize(q.stop), "cudaEventSynchronize");
        float ms = 0.f;
        OMNI_CUDA(cudaEventElapsedTime(&ms, q.start, q.stop), "cudaEventElapsedTime");
        pl->stats[q.pass].total_ms += ms;
        pl->event_pool.push_back(q.start);
        pl->event_pool.push_back(q.stop);
    }
    pl->pending.clear();
    const int n = (int)std::min<size_t>(pl->stats.size(), max > 0 ? (size_t)max : 0);
    if (out)
        for (int i = 0; i < n; ++i) out[i] = pl->stats[i];
    if (n_out) *n_out = (int)pl->stats.size();
    if (clear)
        for (auto& s : pl->stats) {
            s.launches = 0;
            s.total_ms = 0.0;
            s.bytes = 0.0;
            s.flops = 0.0;
        }
    return OMNI_OK;
}

const char* omni_last_error(void) { return g_last_error.c_str(); }

const char* omni_status_string(omni_status s) {
    switch (s) {
        case OMNI_OK: return "OMNI_OK";
        case OMNI_ERR_INVALID_ARG: return "OMNI_ERR_INVALID_ARG";
        case OMNI_ERR_COLLISION: return "OMNI_ERR_COLLISION";
        case OMNI_ERR_UNSUPPORTED: return "OMNI_ERR_UNSUPPORTED";
        case OMNI_ERR_OOM: return "OMNI_ERR_OOM";
        case OMNI_ERR_CUDA: return "OMNI_ERR_CUDA";
        case OMNI_ERR_TIMEOUT: return "OMNI_ERR_TIMEOUT";
    }
    return "OMNI_ERR_UNKNOWN";
}

}  // extern "C"
