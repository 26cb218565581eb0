/*
 * acf_oracle.c -- plain, slow, obviously correct CPU oracle for the AARTFAAC
 * correlator stage (Prasad et al., "The AARTFAAC All Sky Monitor: System
 * Design and Implementation", arXiv 1609.04205).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the package smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * library.
 *
 * Arithmetic: IEEE fp64 for every floating-point step, int64 for the exact
 * integer correlation.  Steps follow the paper's order (Sec. 4.2.3 polyphase
 * filter bank = FIR then FFT; Sec. 4.2.4 bandpass weights then transpose;
 * Sec. 4.2.5 correlation of one triangle of the Hermitian matrix).  Each step
 * is its plain definition: a direct FIR, a naive DFT, a brute-force pair sum.
 *
 * Readings where the paper is silent (they are also the readings the CUDA
 * path implements):
 *   - prototype filter: Hann-windowed sinc of length L = P*C, normalised to
 *     unit sum (Sec. 4.2.3 only says "256 channel, 16-tap");
 *   - FIR indexing: spectrum m uses stream samples [m*C, m*C + L) with
 *     y_m[n] = sum_k h[k*C + n] * x[m*C + k*C + n];
 *   - DFT sign exp(-2 pi i c n / C), natural channel order, no fftshift;
 *   - correlation convention V_ij = sum_t x_i[t] * conj(x_j[t]), i >= j,
 *     stored packed lower-triangular at bl = i*(i+1)/2 + j;
 *   - gain model M = G R G^H, loss sum over channels of the squared Frobenius
 *     norm of M - V over the full Hermitian matrix, gradient in the
 *     d/dRe + i d/dIm convention.
 *
 * Parity pins (tests/test_oracle_*.py): closed forms (pure tone, impulse),
 * Parseval, numpy FFT, brute-force einsum on tiny inputs, Python-int exact
 * sums, Hermitian/Cauchy-Schwarz invariants, the rank-1 point-source phase,
 * and central finite differences for the gain gradient.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* ---------------------------------------------------------------------------
 * Sec. 4.2.3: prototype of the 16-tap polyphase filter bank.
 * h[n] = w[n] * sinc((n - (L-1)/2) / C), w = symmetric Hann, then sum(h) = 1.
 * Returns 0 on success, -1 on bad arguments.
 * ------------------------------------------------------------------------- */
int oracle_prototype(int n_taps, int n_channels, double *h)
{
    if (n_taps < 1 || n_channels < 1 || !h) return -1;
    const long L = (long)n_taps * n_channels;
    if (L == 1) { h[0] = 1.0; return 0; }
    double sum = 0.0;
    for (long n = 0; n < L; ++n) {
        const double w = 0.5 - 0.5 * cos(2.0 * ORACLE_PI * (double)n / (double)(L - 1));
        const double u = ((double)n - 0.5 * (double)(L - 1)) / (double)n_channels;
        const double s = (u == 0.0) ? 1.0 : sin(ORACLE_PI * u) / (ORACLE_PI * u);
        h[n] = w * s;
        sum += h[n];
    }
    for (long n = 0; n < L; ++n) h[n] /= sum;
    return 0;
}

/* Number of complete FIR windows in a stream of `len` samples:
 * spectrum m exists when m*C + P*C <= len. */
long oracle_n_spectra(long len, int n_taps, int n_channels)
{
    const long L = (long)n_taps * n_channels;
    if (len < L) return 0;
    return (len - L) / n_channels + 1;
}

/* ---------------------------------------------------------------------------
 * Sec. 4.2.3 + 4.2.4 for a set of inputs: direct FIR, naive DFT, bandpass.
 *
 *   x    : [S][N][2] fp64 complex samples, inputs contiguous (the transposed
 *          order the data router delivers, Sec. 3.3).
 *   h    : prototype, length P*C.
 *   w    : bandpass weights, length C (NULL = all ones).
 *   spectra m in [m_begin, m_end) are produced; chans[0..n_chans) selects the
 *   output channels (the DFT is evaluated only there).
 *   X    : [n_chans][N][m_end - m_begin][2] -- channel, input, time, i.e. the
 *          "exchange the parallelism axis" transpose of Sec. 4.2.4.
 * Returns 0, or -1 when a window would read past S.
 * ------------------------------------------------------------------------- */
int oracle_channelise(const double *x, long S, int N, const double *h, int P, int C,
                      const double *w, long m_begin, long m_end, const int *chans,
                      int n_chans, double *X)
{
    if (m_end < m_begin) return -1;
    if (m_end > m_begin && (m_end - 1) * (long)C + (long)P * C > S) return -1;
    const long T = m_end - m_begin;
    /* DFT kernel exp(-2 pi i c q / C) for the selected channels, evaluated once */
    double *wr = (double *)malloc(sizeof(double) * (size_t)n_chans * C);
    double *wi = (double *)malloc(sizeof(double) * (size_t)n_chans * C);
    for (int ci = 0; ci < n_chans; ++ci)
        for (int q = 0; q < C; ++q) {
            const double ang = -2.0 * ORACLE_PI * (double)(((long)chans[ci] * q) % C) / (double)C;
            wr[(size_t)ci * C + q] = cos(ang);
            wi[(size_t)ci * C + q] = sin(ang);
        }
#pragma omp parallel
    {
        double *y = (double *)malloc(sizeof(double) * 2 * (size_t)C);
#pragma omp for schedule(dynamic, 1)
        for (int n = 0; n < N; ++n) {
            for (long m = m_begin; m < m_end; ++m) {
                /* FIR: one polyphase branch per channel phase q */
                for (int q = 0; q < C; ++q) {
                    double re = 0.0, im = 0.0;
                    for (int k = 0; k < P; ++k) {
                        const long t = m * C + (long)k * C + q;
                        const double hk = h[(long)k * C + q];
                        re += hk * x[(t * N + n) * 2 + 0];
                        im += hk * x[(t * N + n) * 2 + 1];
                    }
                    y[2 * q + 0] = re;
                    y[2 * q + 1] = im;
                }
                /* naive DFT, then the channel's bandpass weight */
                for (int ci = 0; ci < n_chans; ++ci) {
                    const int c = chans[ci];
                    double re = 0.0, im = 0.0;
                    for (int q = 0; q < C; ++q) {
                        const double cr = wr[(size_t)ci * C + q], sr = wi[(size_t)ci * C + q];
                        re += y[2 * q] * cr - y[2 * q + 1] * sr;
                        im += y[2 * q] * sr + y[2 * q + 1] * cr;
                    }
                    const double wc = w ? w[c] : 1.0;
                    double *o = X + (((size_t)ci * N + n) * T + (m - m_begin)) * 2;
                    o[0] = wc * re;
                    o[1] = wc * im;
                }
            }
        }
        free(y);
    }
    free(wr);
    free(wi);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Sec. 4.2.5: correlation, one triangle of the Hermitian matrix per channel.
 *   X : [n_ch][N][T][2]; V : [n_ch][N(N+1)/2][2], ACCUMULATED (V += ...).
 * ------------------------------------------------------------------------- */
void oracle_correlate_f64(const double *X, int n_ch, int N, long T, double *V)
{
    const long NB = (long)N * (N + 1) / 2;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int c = 0; c < n_ch; ++c) {
        for (int i = 0; i < N; ++i) {
            const double *xi = X + ((size_t)c * N + i) * T * 2;
            for (int j = 0; j <= i; ++j) {
                const double *xj = X + ((size_t)c * N + j) * T * 2;
                double re = 0.0, im = 0.0;
                for (long t = 0; t < T; ++t) {
                    /* x_i * conj(x_j) */
                    re += xi[2 * t] * xj[2 * t] + xi[2 * t + 1] * xj[2 * t + 1];
                    im += xi[2 * t + 1] * xj[2 * t] - xi[2 * t] * xj[2 * t + 1];
                }
                double *v = V + ((size_t)c * NB + (long)i * (i + 1) / 2 + j) * 2;
                v[0] += re;
                v[1] += im;
            }
        }
    }
}

/* Exact integer correlation of raw (unchannelised) samples.
 *   x : [T][N][2] int16 (covers complex int8 and int16 inputs);
 *   V : [N(N+1)/2][2] int64, ACCUMULATED. */
void oracle_correlate_i64(const int16_t *x, int N, long T, int64_t *V)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < N; ++i) {
        for (int j = 0; j <= i; ++j) {
            int64_t re = 0, im = 0;
            for (long t = 0; t < T; ++t) {
                const int64_t ar = x[(t * N + i) * 2], ai = x[(t * N + i) * 2 + 1];
                const int64_t br = x[(t * N + j) * 2], bi = x[(t * N + j) * 2 + 1];
                re += ar * br + ai * bi;
                im += ai * br - ar * bi;
            }
            int64_t *v = V + ((long)i * (i + 1) / 2 + j) * 2;
            v[0] += re;
            v[1] += im;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Gain-corrupted correlation M = G R G^H (G = diag(g)), residual E = M - V,
 * loss L = sum_c ||E_c||_F^2 over the full Hermitian matrix, and the gradient
 *   grad_k = dL/dRe g_k + i dL/dIm g_k = 4 sum_c sum_j E_kj conj(R_kj) g_j.
 *   R, V : [C][N(N+1)/2][2] packed lower triangles; g : [N][2].
 *   grad : [N][2] or NULL.  Returns L.
 * The full matrix is walked element by element; the upper triangle is the
 * conjugate of the stored lower one.
 * ------------------------------------------------------------------------- */
double oracle_gain(const double *R, const double *V, const double *g, int N, int C,
                   double *grad)
{
    const long NB = (long)N * (N + 1) / 2;
    double loss = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * 2 * (size_t)N);
    for (int c = 0; c < C; ++c) {
        for (int i = 0; i < N; ++i) {
            for (int j = 0; j < N; ++j) {
                const int lo = i >= j ? i : j, hi = i >= j ? j : i;
                const double *r = R + ((size_t)c * NB + (long)lo * (lo + 1) / 2 + hi) * 2;
                const double *v = V + ((size_t)c * NB + (long)lo * (lo + 1) / 2 + hi) * 2;
                const double sgn = (i >= j) ? 1.0 : -1.0; /* conj for the upper triangle */
                const double rr = r[0], ri = sgn * r[1];
                const double vr = v[0], vi = sgn * v[1];
                /* g_i * R_ij * conj(g_j) */
                const double gir = g[2 * i], gii = g[2 * i + 1];
                const double gjr = g[2 * j], gji = -g[2 * j + 1];
                const double tr = gir * rr - gii * ri, ti = gir * ri + gii * rr;
                const double mr = tr * gjr - ti * gji, mi = tr * gji + ti * gjr;
                const double er = mr - vr, ei = mi - vi;
                loss += er * er + ei * ei;
                if (grad) {
                    /* E_ij * conj(R_ij) * g_j, added to row i */
                    const double pr = er * rr + ei * ri, pi = ei * rr - er * ri;
                    const double qr = pr * g[2 * j] - pi * g[2 * j + 1];
                    const double qi = pr * g[2 * j + 1] + pi * g[2 * j];
                    grad[2 * i] += 4.0 * qr;
                    grad[2 * i + 1] += 4.0 * qi;
                }
            }
        }
    }
    return loss;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
