// omni_noalloc.cu -- a correlation entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator hooks, processes whose device memory is
// fully reserved up front, and real-time pipelines that forbid allocation
// after start-up.  omni_correlate_noalloc serves them: it runs the same
// transform kernels as the plan API, but its scratch (the FP64 |F|^2
// accumulator, the two pass buffers and the direct-DFT twiddle tables) lives
// in one file-scope device array, g_scratch, of OMNI_NOALLOC_SCRATCH_BYTES.
// Every GPU that loads this part of the library holds that array until the
// process exits.
//
// In host code g_scratch is only a host-side stand-in for the device array,
// not a device address: a kernel given it would fault or, where the GPU can
// reach host memory, silently use the wrong memory.  So at set-up, once per
// device and with that device current, the address is obtained with
// cudaGetSymbolAddress and that pointer is what the kernels receive.  The
// set-up happens inside the first call on each device.
#include "omni.h"
#include "omni_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>

namespace {

using namespace omni;

constexpr size_t kScratchBytes = (size_t)OMNI_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Record a failure for omni_last_error() and return its status.
omni_status failf(omni_status st, const char* fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

// Device address of g_scratch on the current device, looked up once per device.
omni_status scratch_address(unsigned char** out) {
    static std::mutex mu;
    static std::vector<std::pair<int, unsigned char*>> known;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return failf(OMNI_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(mu);
    for (auto& k : known)
        if (k.first == dev) {
            *out = k.second;
            return OMNI_OK;
        }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
        return failf(OMNI_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    known.push_back({dev, (unsigned char*)p});
    *out = (unsigned char*)p;
    return OMNI_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" omni_status omni_correlate_noalloc(const omni_level* levels, int n_levels,
                                              int64_t n_channels, omni_dtype dtype,
                                              const void* volts_dev, int64_t T, double* vis_dev,
                                              void* stream) {
    // geometry and collision checks of the public API (sets omni_last_error)
    omni_status st = omni_baselines(levels, n_levels, nullptr, nullptr, nullptr);
    if (st != OMNI_OK) return st;
    if (n_channels < 1) return failf(OMNI_ERR_INVALID_ARG, "n_channels must be >= 1");
    if (T < 0) return failf(OMNI_ERR_INVALID_ARG, "T must be >= 0");
    if (dtype != OMNI_IN_CF32 && dtype != OMNI_IN_CI8) return failf(OMNI_ERR_INVALID_ARG, "unknown dtype");
    if (!vis_dev || (uintptr_t)vis_dev % 16) return failf(OMNI_ERR_INVALID_ARG, "vis_dev must be a 16-byte aligned device pointer");
    if (T > 0 && (!volts_dev || (uintptr_t)volts_dev % 16))
        return failf(OMNI_ERR_INVALID_ARG, "volts_dev must be a 16-byte aligned device pointer");

    const int D = 2 * n_levels;
    int n[kMaxDims], Lp[kMaxDims];
    int64_t L = 1, Q = 1, N = 1;
    for (int k = 0; k < n_levels; ++k) {
        n[2 * k] = levels[k].n1;
        n[2 * k + 1] = levels[k].n2;
    }
    for (int d = 0; d < D; ++d) {
        Lp[d] = n[d] > 1 ? 2 * n[d] : 1;
        L *= Lp[d];
        Q *= 2 * n[d] - 1;
        N *= n[d];
    }

    // the same pass lists the plan API builds: forward over increasing axes,
    // inverse over decreasing axes, kernel family by axis length
    std::vector<int> axes;
    for (int d = 0; d < D; ++d)
        if (Lp[d] > 1) axes.push_back(d);
    if (axes.empty()) axes.push_back(0);
    // kernel family by axis length: the plan API's choice (choose_kind)
    std::vector<Pass> fwd, inv;
    int64_t fwd_elems = 0, inv_elems = 0, tw_floats = 0;
    for (size_t a = 0; a < axes.size(); ++a) {
        const int d = axes[a];
        Pass p{};
        p.axis = d;
        p.L = Lp[d];
        p.n = n[d];
        p.q_out = Lp[d];
        p.inner = p.outer = 1;
        for (int e = 0; e < d; ++e) p.inner *= Lp[e];
        for (int e = d + 1; e < D; ++e) p.outer *= n[e];
        p.mode = (a + 1 == axes.size()) ? MODE_LAST : MODE_MID;
        choose_kind(p);
        if (p.mode == MODE_MID) fwd_elems = std::max(fwd_elems, p.outer * p.L * p.inner);
        if (p.kind == KIND_DIRECT) tw_floats += 2 * p.L;
        fwd.push_back(p);
    }
    for (size_t a = axes.size(); a-- > 0;) {
        const int d = axes[a];
        Pass p{};
        p.axis = d;
        p.L = Lp[d];
        p.n = Lp[d];
        p.q_out = 2 * n[d] - 1;
        p.q_shift = n[d] - 1;
        p.inner = p.outer = 1;
        for (int e = 0; e < d; ++e) p.inner *= Lp[e];
        for (int e = d + 1; e < D; ++e) p.outer *= 2 * n[e] - 1;
        p.mode = (a == 0) ? MODE_INV_LAST : MODE_INV_MID;
        choose_kind(p);
        if (p.mode == MODE_INV_MID) inv_elems = std::max(inv_elems, p.outer * p.q_out * p.inner);
        if (p.kind == KIND_DIRECT) tw_floats += 2 * p.L;
        inv.push_back(p);
    }

    // carve the static array: [P: C x L doubles][twiddles][buffer 0][buffer 1]
    const size_t P_bytes = align256((size_t)n_channels * L * sizeof(double));
    const size_t tw_bytes = align256((size_t)tw_floats * sizeof(float));
    const size_t per_sample = (size_t)std::max<int64_t>(1, fwd_elems) * sizeof(float2);
    const size_t per_chan = (size_t)std::max<int64_t>(1, inv_elems) * sizeof(float2);
    const size_t min_buf = align256(std::max(per_sample, per_chan));
    const size_t need = P_bytes + tw_bytes + 2 * min_buf;
    if (need > kScratchBytes)
        return failf(OMNI_ERR_UNSUPPORTED,
                     "omni_correlate_noalloc needs %zu bytes of scratch for %lld channels of this "
                     "lattice (L = %lld); its static array holds %zu bytes (use the plan API)",
                     need, (long long)n_channels, (long long)L, kScratchBytes);
    const size_t buf_bytes = ((kScratchBytes - P_bytes - tw_bytes) / 2) & ~size_t(255);
    const int64_t Tc = std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(T, 1), (int64_t)(buf_bytes / per_sample)));
    const int64_t Cv = std::max<int64_t>(1, std::min<int64_t>(n_channels, (int64_t)(buf_bytes / per_chan)));

    // set-up on this device: twiddle tables of the kernels, scratch address
    cudaError_t e = init_device_tables();
    if (e != cudaSuccess) return failf(OMNI_ERR_CUDA, "twiddle upload: %s", cudaGetErrorString(e));
    unsigned char* base = nullptr;
    st = scratch_address(&base);
    if (st != OMNI_OK) return st;
    double* P = (double*)base;
    float2* tw = (float2*)(base + P_bytes);
    float2* buf[2] = {(float2*)(base + P_bytes + tw_bytes),
                      (float2*)(base + P_bytes + tw_bytes + buf_bytes)};
    cudaStream_t s = (cudaStream_t)stream;

    // direct-DFT twiddles w_L^m from double precision, copied into the array
    if (tw_floats > 0) {
        std::vector<float2> h;
        for (auto* list : {&fwd, &inv})
            for (Pass& p : *list) {
                if (p.kind != KIND_DIRECT) continue;
                p.tw = tw + h.size();
                for (int m = 0; m < p.L; ++m) {
                    const double ang = 6.283185307179586476925286766559 * m / p.L;
                    h.push_back(make_float2((float)std::cos(ang), (float)-std::sin(ang)));
                }
            }
        e = cudaMemcpyAsync(tw, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return failf(OMNI_ERR_CUDA, "twiddle copy: %s", cudaGetErrorString(e));
        e = cudaStreamSynchronize(s);  // h is freed on return
        if (e != cudaSuccess) return failf(OMNI_ERR_CUDA, "twiddle copy: %s", cudaGetErrorString(e));
    }

    // the array keeps the previous call's contents: the accumulator starts at zero
    e = cudaMemsetAsync(P, 0, (size_t)n_channels * L * sizeof(double), s);
    if (e != cudaSuccess) return failf(OMNI_ERR_CUDA, "clearing scratch: %s", cudaGetErrorString(e));

    // forward passes, one channel x Tc samples per chunk
    for (int64_t c = 0; c < n_channels && T > 0; ++c)
        for (int64_t t0 = 0; t0 < T; t0 += Tc) {
            const int64_t tc = std::min(Tc, T - t0);
            const void* src = volts_dev;
            int src_kind = dtype == OMNI_IN_CI8 ? SRC_CI8 : SRC_CF32;
            int64_t src_stride = 0;
            for (size_t k = 0; k < fwd.size(); ++k) {
                const Pass& p = fwd[k];
                PassArgs a{};
                a.src = src;
                a.src_kind = src_kind;
                a.src_stride = src_stride;
                a.vc0 = c;
                a.T = T;
                a.t0 = t0;
                a.N = N;
                a.tc = (int)tc;
                a.c0 = c;
                a.P = P;
                a.P_stride = L;
                if (p.mode == MODE_LAST) {
                    a.S = 1;
                } else {
                    a.S = tc;
                    a.dst = buf[k & 1];
                    a.dst_stride = p.outer * p.L * p.inner;
                }
                e = launch_pass(p, a, s);
                if (e != cudaSuccess) return failf(OMNI_ERR_CUDA, "forward pass: %s", cudaGetErrorString(e));
                src = buf[k & 1];
                src_kind = SRC_BUF;
                src_stride = p.outer * p.L * p.inner;
            }
        }
    // inverse passes into the caller's visibilities
    for (int64_t c0 = 0; c0 < n_channels; c0 += Cv) {
        const int64_t cv = std::min(Cv, n_channels - c0);
        const void* src = P;
        int src_kind = SRC_P64;
        int64_t src_stride = L;
        for (size_t k = 0; k < inv.size(); ++k) {
            const Pass& p = inv[k];
            PassArgs a{};
            a.src = src;
            a.src_kind = src_kind;
            a.src_stride = src_stride;
            a.S = cv;
            a.c0 = c0;
            a.tc = 1;
            if (p.mode == MODE_INV_LAST) {
                a.V = reinterpret_cast<double2*>(vis_dev);
                a.V_stride = Q;
                a.scale = 1.0 / (double)L;
            } else {
                a.dst = buf[k & 1];
                a.dst_stride = p.outer * p.q_out * p.inner;
            }
            e = launch_pass(p, a, s);
            if (e != cudaSuccess) return failf(OMNI_ERR_CUDA, "inverse pass: %s", cudaGetErrorString(e));
            src = buf[k & 1];
            src_kind = SRC_BUF;
            src_stride = p.outer * p.q_out * p.inner;
        }
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return failf(OMNI_ERR_CUDA, "device error: %s", cudaGetErrorString(e));
    return OMNI_OK;
}
