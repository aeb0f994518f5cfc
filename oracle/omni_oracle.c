/*
 * omni_oracle.c -- CPU FP64 oracle for the hierarchical-grid correlator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA library: no headers, no tables, no helpers.
 *
 * What it computes is the plain definition of the visibilities, with no FFT:
 *
 *   V_c(D) = sum_t sum_{m : m, m+D in the box} x_{c,t}(m + D) * conj(x_{c,t}(m))
 *
 * for every 2n-D lag D with D_d in [-(n_d-1), n_d-1].  This is the
 * convolution of the voltage hypercube with its parity-reversed copy,
 * Eq. ConvolutionDefEq (Sec. II.C) generalised to the hypercube of
 * Eq. ProofEq2 (Sec. II.D), with the second factor conjugated so that the
 * result is V_ij = x_i x_j^* summed over antenna pairs with m_i - m_j = D.
 * Sec. IV states that the hypercube algorithm yields exactly these numbers.
 *
 * Conventions: dimension 0 varies fastest, both in the antenna order of x and
 * in the lag order of V; lags run from -(n_d-1) to n_d-1 along each
 * dimension (the listings of Eqs. ConvolutionExampleEq1/2).
 *
 * Parity pinned by tests/test_oracle_pins.py (paper values, closed forms,
 * invariants, a naive-DFT route and a numpy.fft route).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_DIMS 16

/* Element x[i] of a [N][2] interleaved complex array of the given type. */
static inline void load_x(const void *x, int dtype, int64_t i, double *re, double *im)
{
    if (dtype == 0) {                      /* complex128 */
        const double *p = (const double *)x;
        *re = p[2 * i];
        *im = p[2 * i + 1];
    } else if (dtype == 1) {               /* complex64 */
        const float *p = (const float *)x;
        *re = (double)p[2 * i];
        *im = (double)p[2 * i + 1];
    } else {                               /* complex int8 */
        const int8_t *p = (const int8_t *)x;
        *re = (double)p[2 * i];
        *im = (double)p[2 * i + 1];
    }
}

static size_t elem_bytes(int dtype) { return dtype == 0 ? 16 : dtype == 1 ? 8 : 2; }

int64_t oracle_n_antennas(int D, const int32_t *n)
{
    int64_t N = 1;
    for (int d = 0; d < D; ++d) N *= n[d];
    return N;
}

int64_t oracle_n_lags(int D, const int32_t *n)
{
    int64_t L = 1;
    for (int d = 0; d < D; ++d) L *= 2 * (int64_t)n[d] - 1;
    return L;
}

/* Lag vector of lag index q (dimension 0 fastest, each from -(n_d-1)). */
static void lag_of_index(int D, const int32_t *n, int64_t q, int32_t *lag)
{
    for (int d = 0; d < D; ++d) {
        int64_t w = 2 * (int64_t)n[d] - 1;
        lag[d] = (int32_t)(q % w) - (n[d] - 1);
        q /= w;
    }
}

/*
 * Lag table: dm[q][d] = D_d and red[q] = number of antenna pairs with that
 * 2n-D separation, prod_d (n_d - |D_d|) (the baseline distribution d = l*l^-
 * of Sec. III for a layout map of ones).
 */
void oracle_lag_table(int D, const int32_t *n, int32_t *dm, int64_t *red)
{
    int64_t Q = oracle_n_lags(D, n);
    for (int64_t q = 0; q < Q; ++q) {
        int32_t lag[OR_MAX_DIMS];
        lag_of_index(D, n, q, lag);
        int64_t r = 1;
        for (int d = 0; d < D; ++d) {
            dm[q * D + d] = lag[d];
            r *= n[d] - abs(lag[d]);
        }
        red[q] = r;
    }
}

/*
 * Antenna positions, Eq. GridEq: r = sum_k A_k (m_{2k}, m_{2k+1}), with A_k
 * row-major 2x2 per level (level 1 first).  shape[2k], shape[2k+1] are the
 * level-k sizes.  r is [N][2].
 */
void oracle_positions(int n_levels, const int32_t *shape, const double *A, double *r)
{
    int D = 2 * n_levels;
    int64_t N = oracle_n_antennas(D, shape);
    for (int64_t i = 0; i < N; ++i) {
        int64_t rest = i;
        double x = 0.0, y = 0.0;
        for (int k = 0; k < n_levels; ++k) {
            int64_t m1 = rest % shape[2 * k];
            rest /= shape[2 * k];
            int64_t m2 = rest % shape[2 * k + 1];
            rest /= shape[2 * k + 1];
            const double *a = A + 4 * k;
            x += a[0] * (double)m1 + a[1] * (double)m2;
            y += a[2] * (double)m1 + a[3] * (double)m2;
        }
        r[2 * i] = x;
        r[2 * i + 1] = y;
    }
}

/* Physical baseline of each lag: dr[q] = sum_k A_k (D_{2k}, D_{2k+1}). */
void oracle_baseline_vectors(int n_levels, const double *A, int64_t Q,
                             const int32_t *dm, double *dr)
{
    int D = 2 * n_levels;
    for (int64_t q = 0; q < Q; ++q) {
        double x = 0.0, y = 0.0;
        for (int k = 0; k < n_levels; ++k) {
            const double *a = A + 4 * k;
            double d1 = dm[q * D + 2 * k], d2 = dm[q * D + 2 * k + 1];
            x += a[0] * d1 + a[1] * d2;
            y += a[2] * d1 + a[3] * d2;
        }
        dr[2 * q] = x;
        dr[2 * q + 1] = y;
    }
}

/*
 * Uniqueness of the map r <-> integer indices (Sec. II.D requires every grid
 * point to have a unique index set).  Returns 1 when two antennas lie closer
 * than tol_rel * max|r| (or exactly coincide when max|r| is 0), else 0.
 * Plain O(N^2) pair loop.
 */
int oracle_collides(int64_t N, const double *r, double tol_rel)
{
    double rmax = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double v = hypot(r[2 * i], r[2 * i + 1]);
        if (v > rmax) rmax = v;
    }
    double tol = tol_rel * rmax;
    int hit = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : hit)
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t j = i + 1; j < N; ++j) {
            double dx = r[2 * i] - r[2 * j], dy = r[2 * i + 1] - r[2 * j + 1];
            if (hypot(dx, dy) <= tol) hit = 1;
        }
    }
    return hit;
}

/*
 * Visibility of one lag for one channel: sum over samples t and over every
 * lattice point m with both m and m+D inside the box of
 * x_t(m+D) * conj(x_t(m)).  xc points at the channel's [T][N] block.
 */
static void one_lag(int D, const int32_t *n, const int64_t *stride, int64_t N, int64_t T,
                    const void *xc, int dtype, const int32_t *lag, double *vre, double *vim)
{
    int32_t lo[OR_MAX_DIMS], hi[OR_MAX_DIMS], m[OR_MAX_DIMS];
    int64_t shift = 0;
    for (int d = 0; d < D; ++d) {
        lo[d] = lag[d] < 0 ? -lag[d] : 0;          /* m_d >= 0 and m_d + D_d >= 0 */
        hi[d] = lag[d] > 0 ? n[d] - lag[d] : n[d]; /* m_d < n_d and m_d + D_d < n_d */
        if (hi[d] <= lo[d]) { *vre = 0.0; *vim = 0.0; return; }
        shift += (int64_t)lag[d] * stride[d];
    }
    double sre = 0.0, sim = 0.0;
    size_t eb = elem_bytes(dtype);
    for (int64_t t = 0; t < T; ++t) {
        const char *xt = (const char *)xc + (size_t)(t * N) * eb;
        for (int d = 0; d < D; ++d) m[d] = lo[d];
        for (;;) {
            int64_t j = 0;
            for (int d = 0; d < D; ++d) j += (int64_t)m[d] * stride[d];
            double ar, ai, br, bi;
            load_x(xt, dtype, j + shift, &ar, &ai);   /* x(m + D) */
            load_x(xt, dtype, j, &br, &bi);           /* x(m)     */
            sre += ar * br + ai * bi;                 /* a * conj(b) */
            sim += ai * br - ar * bi;
            int d = 0;
            while (d < D) {
                if (++m[d] < hi[d]) break;
                m[d] = lo[d];
                ++d;
            }
            if (d == D) break;
        }
    }
    *vre = sre;
    *vim = sim;
}

/*
 * Full brute-force correlator.  x is [C][T][N] complex of type dtype
 * (0 = complex128, 1 = complex64, 2 = complex int8); V is [C][Q][2] with
 * Q = prod_d (2 n_d - 1).  Parallel over lags.
 */
void oracle_correlate(int D, const int32_t *n, int64_t C, int64_t T, int dtype,
                      const void *x, double *V)
{
    int64_t N = oracle_n_antennas(D, n);
    int64_t Q = oracle_n_lags(D, n);
    int64_t stride[OR_MAX_DIMS];
    int64_t s = 1;
    for (int d = 0; d < D; ++d) { stride[d] = s; s *= n[d]; }
    size_t eb = elem_bytes(dtype);
    for (int64_t c = 0; c < C; ++c) {
        const char *xc = (const char *)x + (size_t)(c * T * N) * eb;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t q = 0; q < Q; ++q) {
            int32_t lag[OR_MAX_DIMS];
            lag_of_index(D, n, q, lag);
            one_lag(D, n, stride, N, T, xc, dtype, lag, &V[2 * (c * Q + q)],
                    &V[2 * (c * Q + q) + 1]);
        }
    }
}

/*
 * The same definition evaluated only at selected (channel, lag) pairs:
 * chan[s], lag_index[s] for s < S; V is [S][2].  Used for sampled checks at
 * sizes where the full N^2 sum is out of reach.
 */
void oracle_correlate_selected(int D, const int32_t *n, int64_t C, int64_t T, int dtype,
                               const void *x, int64_t S, const int64_t *chan,
                               const int64_t *lag_index, double *V)
{
    int64_t N = oracle_n_antennas(D, n);
    int64_t stride[OR_MAX_DIMS];
    int64_t s = 1;
    for (int d = 0; d < D; ++d) { stride[d] = s; s *= n[d]; }
    size_t eb = elem_bytes(dtype);
    (void)C;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < S; ++k) {
        int32_t lag[OR_MAX_DIMS];
        lag_of_index(D, n, lag_index[k], lag);
        const char *xc = (const char *)x + (size_t)(chan[k] * T * N) * eb;
        one_lag(D, n, stride, N, T, xc, dtype, lag, &V[2 * k], &V[2 * k + 1]);
    }
}

/*
 * Beam-space variant (Appendix A, steps 4 and 5), in those two steps:
 *
 *   4. every level-1 block (dimensions 0 and 1, sizes n1 x n2) is Fourier
 *      transformed without padding, giving n1 x n2 digital pointings k:
 *        y_t(k; m') = sum_{a < n1, b < n2} x_t(a, b, m')
 *                     * exp(-2 pi i (k_a a / n1 + k_b b / n2)),
 *      evaluated term by term (a direct DFT, no FFT);
 *   5. each pointing is correlated over the remaining dimensions (levels
 *      2..n) by the same brute-force definition as oracle_correlate:
 *        B_c(k; D') = sum_t sum_{m'} y_t(k; m' + D') conj(y_t(k; m')).
 *
 * x is [C][T][N] of type dtype (antenna order dimension 0 fastest, so
 * antenna a + n1 (b + n2 m')); B is [C][Q'][n1 n2][2] with Q' = prod_{d >= 2}
 * (2 n_d - 1), lags in oracle_lag_table order over dimensions 2.., pointing
 * index k_a + n1 k_b fastest.  Needs D >= 3.
 */
void oracle_beam_correlate(int D, const int32_t *n, int64_t C, int64_t T, int dtype,
                           const void *x, double *B)
{
    const int32_t n1 = n[0], n2 = n[1];
    const int64_t nb = (int64_t)n1 * n2;
    const int Dc = D - 2;
    const int32_t *nc = n + 2;
    const int64_t Nc = oracle_n_antennas(Dc, nc);
    const int64_t Qc = oracle_n_lags(Dc, nc);
    const int64_t N = nb * Nc;
    int64_t stride[OR_MAX_DIMS];
    int64_t s = 1;
    for (int d = 0; d < Dc; ++d) { stride[d] = s; s *= nc[d]; }
    const double two_pi = 6.283185307179586476925286766559;
    size_t eb = elem_bytes(dtype);
    double *y = (double *)malloc(sizeof(double) * 2 * (size_t)(nb * T * Nc));
    if (!y) return;
    for (int64_t c = 0; c < C; ++c) {
        const char *xc = (const char *)x + (size_t)(c * T * N) * eb;
        /* step 4: y[k][t][m'] */
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t k = 0; k < nb; ++k) {
            const int64_t ka = k % n1, kb = k / n1;
            for (int64_t t = 0; t < T; ++t) {
                const char *xt = xc + (size_t)(t * N) * eb;
                for (int64_t mc = 0; mc < Nc; ++mc) {
                    double sre = 0.0, sim = 0.0;
                    for (int64_t b = 0; b < n2; ++b)
                        for (int64_t a = 0; a < n1; ++a) {
                            double xr, xi;
                            load_x(xt, dtype, a + n1 * (b + n2 * mc), &xr, &xi);
                            const double ph = -two_pi * ((double)((ka * a) % n1) / n1 +
                                                         (double)((kb * b) % n2) / n2);
                            const double wr = cos(ph), wi = sin(ph);
                            sre += xr * wr - xi * wi;
                            sim += xr * wi + xi * wr;
                        }
                    double *o = y + 2 * ((k * T + t) * Nc + mc);
                    o[0] = sre;
                    o[1] = sim;
                }
            }
        }
        /* step 5: brute-force correlation of each pointing over levels 2..n */
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t k = 0; k < nb; ++k) {
            const double *yk = y + 2 * (k * T * Nc);
            for (int64_t q = 0; q < Qc; ++q) {
                int32_t lag[OR_MAX_DIMS];
                lag_of_index(Dc, nc, q, lag);
                double *o = B + 2 * ((c * Qc + q) * nb + k);
                one_lag(Dc, nc, stride, Nc, T, yk, 0, lag, &o[0], &o[1]);
            }
        }
    }
    free(y);
}

/*
 * Tile hybrid (the variant of Sec. III that FFT-correlates within tiles and
 * correlates the tiles' beams pairwise): n_tiles identical n1 x n2 tiles at
 * arbitrary offsets.  For every ordered tile pair (i, j) and intra-tile lag
 * D (D_d in [-(n_d-1), n_d-1]):
 *
 *   V_c(i, j; D) = sum_t sum_{m, m+D in the tile} x_{c,t,i}(m + D) conj(x_{c,t,j}(m)),
 *
 * the brute-force sum over the antenna pairs (a in tile i, b in tile j)
 * with m_a - m_b = D.  x is [C][T][n_tiles * n1 * n2] (tile slowest, then
 * dimension 1, dimension 0 fastest); V is [C][n_tiles][n_tiles][Q][2] with
 * Q = (2 n1 - 1)(2 n2 - 1), lags dimension 0 fastest.
 */
void oracle_tile_correlate(int n1, int n2, int n_tiles, int64_t C, int64_t T, int dtype,
                           const void *x, double *V)
{
    const int64_t M = (int64_t)n1 * n2, N = M * n_tiles;
    const int64_t Q1 = 2 * (int64_t)n1 - 1, Q2 = 2 * (int64_t)n2 - 1, Q = Q1 * Q2;
    size_t eb = elem_bytes(dtype);
    for (int64_t c = 0; c < C; ++c) {
        const char *xc = (const char *)x + (size_t)(c * T * N) * eb;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
        for (int64_t i = 0; i < n_tiles; ++i)
            for (int64_t j = 0; j < n_tiles; ++j)
                for (int64_t q = 0; q < Q; ++q) {
                    const int64_t d1 = q % Q1 - (n1 - 1), d2 = q / Q1 - (n2 - 1);
                    double sre = 0.0, sim = 0.0;
                    for (int64_t t = 0; t < T; ++t) {
                        const char *xt = xc + (size_t)(t * N) * eb;
                        for (int64_t b = 0; b < n2; ++b) {
                            if (b + d2 < 0 || b + d2 >= n2) continue;
                            for (int64_t a = 0; a < n1; ++a) {
                                if (a + d1 < 0 || a + d1 >= n1) continue;
                                double ar, ai, br, bi;
                                load_x(xt, dtype, i * M + (a + d1) + n1 * (b + d2), &ar, &ai);
                                load_x(xt, dtype, j * M + a + n1 * b, &br, &bi);
                                sre += ar * br + ai * bi;
                                sim += ai * br - ar * bi;
                            }
                        }
                    }
                    double *o = V + 2 * (((c * n_tiles + i) * n_tiles + j) * Q + q);
                    o[0] = sre;
                    o[1] = sim;
                }
    }
}

/*
 * F-engine (Appendix A, step 2: each antenna's samples Fourier transformed in
 * time to separate the frequency channels, then calibrated), as a polyphase
 * filter bank written out term by term.  Frame t of antenna a, with frame
 * length 2F and P taps:
 *
 *   u_t(n)  = sum_{p < P} w(p 2F + n) r_a((t + p) 2F + n),        n < 2F,
 *   X_t(f)  = sum_{n < 2F} u_t(n) exp(-2 pi i f n / (2F)),          f < F,
 *   y_t(f)  = scale g(f, a) X_t(f),
 *
 * (a direct DFT; the Nyquist bin f = F is dropped).  raw is [N][S] int8, w is
 * [P][2F] (NULL: all ones), g is [F][N] complex (NULL: 1).  out is [F][T][N]
 * complex FP64 with T = floor((S - (P - 1) 2F) / 2F): the channel-major
 * voltage layout the correlator reads.
 */
void oracle_fengine(const int8_t *raw, int64_t N, int64_t S, int F, int P, const double *w,
                    const double *g, double scale, double *out)
{
    const int64_t M = 2 * (int64_t)F;
    const int64_t T = S >= (P - 1) * M ? (S - (P - 1) * M) / M : 0;
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int64_t a = 0; a < N; ++a)
        for (int64_t t = 0; t < T; ++t) {
            double *u = (double *)malloc(sizeof(double) * (size_t)M);
            if (!u) continue;
            for (int64_t n = 0; n < M; ++n) {
                double acc = 0.0;
                for (int p = 0; p < P; ++p)
                    acc += (w ? w[p * M + n] : 1.0) * (double)raw[a * S + (t + p) * M + n];
                u[n] = acc;
            }
            for (int64_t f = 0; f < F; ++f) {
                double xr = 0.0, xi = 0.0;
                for (int64_t n = 0; n < M; ++n) {
                    const double ph = -two_pi * (double)((f * n) % M) / (double)M;
                    xr += u[n] * cos(ph);
                    xi += u[n] * sin(ph);
                }
                double gr = 1.0, gi = 0.0;
                if (g) {
                    gr = g[2 * (f * N + a)];
                    gi = g[2 * (f * N + a) + 1];
                }
                double *o = out + 2 * ((f * T + t) * N + a);
                o[0] = scale * (gr * xr - gi * xi);
                o[1] = scale * (gr * xi + gi * xr);
            }
            free(u);
        }
}

/* Quantiser of the F-engine output: round half to even, clip to [-127, 127]. */
void oracle_quantize(const float *x, int64_t n, int8_t *q)
{
    for (int64_t i = 0; i < n; ++i) {
        double v = nearbyint((double)x[i]);   /* default rounding mode: half to even */
        if (v > 127.0) v = 127.0;
        if (v < -127.0) v = -127.0;
        q[i] = (int8_t)v;
    }
}

int oracle_max_dims(void) { return OR_MAX_DIMS; }

/* Threads the OpenMP loops above use. */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
