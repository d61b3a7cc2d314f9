/*
 * graphic_oracle.c -- plain, slow, FP64 CPU oracle for the ADI hot path of
 * GRAPHIC (Hugelier et al., arXiv:1510.04331).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (each function names the passage it follows):
 *   - a hand-written radix-2 complex FFT and a brute-force DFT (Sect. 3.3.1,
 *     the Fourier transform definitions);
 *   - the Fourier sub-pixel shift of a zero-padded frame as ONE 2-D transform
 *     multiplied by the separable phasor (Sect. 3.3.1, shift theorem, 2-D
 *     phasor, frames padded to twice their size or more);
 *   - the three-shear Fourier rotation (Sect. 3.4, shear decomposition and
 *     the Fourier form of each shear, double sized frame);
 *   - the angle gate, the optional maximum time separation t_max, and the
 *     per-frame median PSF subtraction (Sect. 3.3, parallactic angle /
 *     reference-frame conditions; the median is subtracted as it is, with no
 *     fitted weights);
 *   - the final median collapse (Sect. 3.4, the derotated frames combined
 *     into one image by their median).
 *
 * Conventions where the paper is silent or garbled (also listed in the
 * design notes): shift(d) moves content by +d (out(x) = in(x - d)); signed
 * frequency bins k in [-M/2, M/2); the Nyquist bin of an even line is
 * multiplied by cos(pi d); padding is exactly M = 2N with the frame at
 * offset N/2; the rotation centre is pixel N/2; rotation by theta moves
 * content counter-clockwise, (x,y) -> (x cos - y sin, x sin + y cos);
 * theta is split into 90q + theta', |theta'| <= 45, the 90q part is an
 * exact index map; alpha_min = 2 asin(n_fwhm FWHM / (2 r)); an empty
 * reference set falls back to the frame(s) farthest in angle among those
 * within t_max of the frame (all frames without a time gate); medians use
 * the IEEE total order, even counts average the two middle values.
 *
 * Threading: frames (geometric steps) and pixels (median steps) are spread
 * over OpenMP threads when compiled with -fopenmp; the arithmetic of each
 * frame or pixel is the same with or without threads.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* 1-D transforms (Sect. 3.3.1: forward kernel exp(-i 2 pi nu x), inverse   */
/* kernel exp(+i 2 pi nu x)).  Discrete, unnormalised forward, 1/M inverse. */
/* ---------------------------------------------------------------------- */

static int is_pow2(int64_t m) { return m > 0 && (m & (m - 1)) == 0; }

/* In-place iterative radix-2 FFT: bit-reversal permutation, then log2(M)
 * butterfly layers.  sign = -1 forward, +1 inverse (no scaling here).
 * The twiddle of butterfly j in a layer of span len is evaluated directly
 * as exp(sign i 2 pi j / len) with cos/sin, per index. */
static void fft_inplace(cplx *x, int M, int sign)
{
    for (int i = 1, j = 0; i < M; i++) {
        int bit = M >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (int len = 2; len <= M; len <<= 1) {
        int half = len >> 1;
        for (int j = 0; j < half; j++) {
            double ang = sign * 2.0 * ORACLE_PI * ((double)j / (double)len);
            cplx w = cos(ang) + I * sin(ang);
            for (int s = 0; s < M; s += len) {
                cplx u = x[s + j];
                cplx v = x[s + j + half] * w;
                x[s + j] = u + v;
                x[s + j + half] = u - v;
            }
        }
    }
}

static void fft_fwd(cplx *x, int M) { fft_inplace(x, M, -1); }
static void fft_inv(cplx *x, int M)
{
    fft_inplace(x, M, +1);
    for (int i = 0; i < M; i++) x[i] /= (double)M;
}

/* Exported: FFT of interleaved (re, im) doubles, in place.  inverse != 0
 * applies the +i kernel and the 1/M factor.  Returns -1 if M is not a
 * power of two. */
int oracle_fft(double *re_im, int M, int inverse)
{
    if (!is_pow2(M)) return -1;
    cplx *x = (cplx *)malloc(sizeof(cplx) * (size_t)M);
    for (int i = 0; i < M; i++) x[i] = re_im[2 * i] + I * re_im[2 * i + 1];
    if (inverse) fft_inv(x, M); else fft_fwd(x, M);
    for (int i = 0; i < M; i++) { re_im[2 * i] = creal(x[i]); re_im[2 * i + 1] = cimag(x[i]); }
    free(x);
    return 0;
}

/* Exported: brute-force O(M^2) DFT (any M), the definition written out. */
int oracle_dft(const double *in_re_im, double *out_re_im, int M, int inverse)
{
    if (M <= 0) return -1;
    double sign = inverse ? 1.0 : -1.0;
    for (int k = 0; k < M; k++) {
        cplx acc = 0;
        for (int n = 0; n < M; n++) {
            long long nk = ((long long)n * k) % M;
            double ang = sign * 2.0 * ORACLE_PI * (double)nk / (double)M;
            acc += (in_re_im[2 * n] + I * in_re_im[2 * n + 1]) * (cos(ang) + I * sin(ang));
        }
        if (inverse) acc /= (double)M;
        out_re_im[2 * k] = creal(acc);
        out_re_im[2 * k + 1] = cimag(acc);
    }
    return 0;
}

/* Phasor of one axis (Sect. 3.3.1 shift theorem, read as: content moves by
 * +d, so bin k is multiplied by exp(-i 2 pi k d / M), k the signed bin).
 * The Nyquist bin k = M/2 of an even M gets cos(pi d), the Hermitian
 * average of the +M/2 and -M/2 phasors, which keeps a real line real. */
static cplx axis_phasor(int k, int M, double d)
{
    if (2 * k == M) return cos(ORACLE_PI * d);
    int ks = (k < M / 2) ? k : k - M;
    double ang = -2.0 * ORACLE_PI * (double)ks * d / (double)M;
    return cos(ang) + I * sin(ang);
}

/* Largest |imag| seen by the real-part extractions of the last exported
 * shift / rotate call (each pass maps a real line to a real line, so this
 * must stay at rounding level).  Per-frame maxima are merged once. */
static double g_max_imag = 0.0;
double oracle_last_max_imag(void) { return g_max_imag; }
static void merge_imag(double local)
{
#ifdef _OPENMP
#pragma omp critical(oracle_imag)
#endif
    if (local > g_max_imag) g_max_imag = local;
}
#define NOTE_IMAG(acc, v) do { double a_ = fabs(v); if (a_ > (acc)) (acc) = a_; } while (0)

/* Exported: periodic Fourier shift of one real line of length M by d
 * (FFT, multiply by the axis phasor, inverse FFT, real part). */
int oracle_shift_line(const double *in, double *out, int M, double d)
{
    if (!is_pow2(M) || M < 2) return -1;
    cplx *x = (cplx *)malloc(sizeof(cplx) * (size_t)M);
    for (int i = 0; i < M; i++) x[i] = in[i];
    fft_fwd(x, M);
    for (int k = 0; k < M; k++) x[k] *= axis_phasor(k, M, d);
    fft_inv(x, M);
    double mi = 0.0;
    for (int i = 0; i < M; i++) { out[i] = creal(x[i]); NOTE_IMAG(mi, cimag(x[i])); }
    g_max_imag = mi;
    free(x);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Shift (Sect. 3.3.1): pad the N x N frame to M = 2N (frame at offset     */
/* N/2), 2-D FFT, multiply by phasor(kx, dx) * phasor(ky, dy), inverse 2-D  */
/* FFT, real part, crop the same window.                                    */
/* ---------------------------------------------------------------------- */

static void fft2(cplx *a, int M, int inverse)
{
    cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)M);
    for (int r = 0; r < M; r++) {
        if (inverse) fft_inv(a + (size_t)r * M, M); else fft_fwd(a + (size_t)r * M, M);
    }
    for (int c = 0; c < M; c++) {
        for (int r = 0; r < M; r++) col[r] = a[(size_t)r * M + c];
        if (inverse) fft_inv(col, M); else fft_fwd(col, M);
        for (int r = 0; r < M; r++) a[(size_t)r * M + c] = col[r];
    }
    free(col);
}

static void shift_frame(const double *in, double *out, int N, double dx, double dy)
{
    int M = 2 * N, off = N / 2;
    cplx *a = (cplx *)calloc((size_t)M * M, sizeof(cplx));
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) a[(size_t)(i + off) * M + (j + off)] = in[(size_t)i * N + j];
    fft2(a, M, 0);
    for (int ky = 0; ky < M; ky++) {
        cplx py = axis_phasor(ky, M, dy);
        for (int kx = 0; kx < M; kx++) a[(size_t)ky * M + kx] *= py * axis_phasor(kx, M, dx);
    }
    fft2(a, M, 1);
    double mi = 0.0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            cplx v = a[(size_t)(i + off) * M + (j + off)];
            out[(size_t)i * N + j] = creal(v);
            NOTE_IMAG(mi, cimag(v));
        }
    merge_imag(mi);
    free(a);
}

/* Exported: shift every frame of a [T][N][N] cube by (dx[t], dy[t]). */
int oracle_shift(const double *cube, double *out, long long T, int N, const double *dx, const double *dy)
{
    if (T < 0 || N < 2 || (N & 1)) return -1;
    g_max_imag = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long long t = 0; t < T; t++)
        shift_frame(cube + (size_t)t * N * N, out + (size_t)t * N * N, N, dx[t], dy[t]);
    return 0;
}

/* Exported, for the flux / Parseval pins: shift of one frame WITHOUT the
 * crop; writes the full M x M real part. */
int oracle_shift_padded(const double *in, double *out_MM, int N, double dx, double dy)
{
    if (N < 2 || (N & 1)) return -1;
    int M = 2 * N, off = N / 2;
    cplx *a = (cplx *)calloc((size_t)M * M, sizeof(cplx));
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) a[(size_t)(i + off) * M + (j + off)] = in[(size_t)i * N + j];
    fft2(a, M, 0);
    for (int ky = 0; ky < M; ky++) {
        cplx py = axis_phasor(ky, M, dy);
        for (int kx = 0; kx < M; kx++) a[(size_t)ky * M + kx] *= py * axis_phasor(kx, M, dx);
    }
    fft2(a, M, 1);
    for (size_t p = 0; p < (size_t)M * M; p++) out_MM[p] = creal(a[p]);
    free(a);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Rotation (Sect. 3.4).                                                    */
/* ---------------------------------------------------------------------- */

/* Exact rotation by 90 q degrees about pixel (N/2, N/2), content moving
 * counter-clockwise, zero where the source pixel falls outside the frame.
 * With x = col - N/2, y = row - N/2 the output at (x, y) takes the input
 * at R(-90 q)(x, y). */
static void rot90_frame(const double *in, double *out, int N, int q)
{
    q = ((q % 4) + 4) % 4;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            int si, sj;
            switch (q) {
            case 0: si = i; sj = j; break;
            case 1: si = N - j; sj = i; break;      /* in(y, -x) */
            case 2: si = N - i; sj = N - j; break;  /* in(-x, -y) */
            default: si = j; sj = N - i; break;     /* in(-y, x) */
            }
            out[(size_t)i * N + j] = (si >= 0 && si < N && sj >= 0 && sj < N) ? in[(size_t)si * N + sj] : 0.0;
        }
}

/* One Fourier shear pass over the padded M x M frame held as real values.
 * axis 0: every row r is shifted along x by d = coef * y, y = r - M/2.
 * axis 1: every column c is shifted along y by d = coef * x, x = c - M/2.
 * Each line: FFT, multiply by the axis phasor, inverse FFT, real part. */
static double shear_pass(double *P, int M, int axis, double coef)
{
    double mi = 0.0;
    cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)M);
    for (int l = 0; l < M; l++) {
        double d = coef * (double)(l - M / 2);
        for (int m = 0; m < M; m++) line[m] = axis == 0 ? P[(size_t)l * M + m] : P[(size_t)m * M + l];
        fft_fwd(line, M);
        for (int k = 0; k < M; k++) line[k] *= axis_phasor(k, M, d);
        fft_inv(line, M);
        for (int m = 0; m < M; m++) {
            if (axis == 0) P[(size_t)l * M + m] = creal(line[m]); else P[(size_t)m * M + l] = creal(line[m]);
            NOTE_IMAG(mi, cimag(line[m]));
        }
    }
    free(line);
    return mi;
}

/* Rotate one frame by theta degrees.  reduce90 != 0: theta = 90 q + theta',
 * q = floor(theta / 90 + 1/2), the 90 q part exact, the 3-shear on theta'
 * (skipped when theta' is exactly zero).  reduce90 == 0: the raw 3-shear on
 * theta (test hook for the 90-degree pin). */
static void rotate_frame(const double *in, double *out, int N, double theta_deg, int reduce90)
{
    int M = 2 * N, off = N / 2;
    int q = 0;
    double tp = theta_deg;
    if (reduce90) {
        q = (int)floor(theta_deg / 90.0 + 0.5);
        tp = theta_deg - 90.0 * (double)q;
    }
    double *g = (double *)malloc(sizeof(double) * (size_t)N * N);
    rot90_frame(in, g, N, q);
    if (tp == 0.0) {
        memcpy(out, g, sizeof(double) * (size_t)N * N);
        free(g);
        return;
    }
    double th = tp * ORACLE_PI / 180.0;
    double a = tan(th / 2.0);   /* S_x(-tan(theta/2)) moves content by -a y */
    double s = sin(th);         /* S_y(sin theta) moves content by +s x     */
    double *P = (double *)calloc((size_t)M * M, sizeof(double));
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) P[(size_t)(i + off) * M + (j + off)] = g[(size_t)i * N + j];
    double mi = shear_pass(P, M, 0, -a);
    double m2 = shear_pass(P, M, 1, s);
    double m3 = shear_pass(P, M, 0, -a);
    merge_imag(fmax(mi, fmax(m2, m3)));
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) out[(size_t)i * N + j] = P[(size_t)(i + off) * M + (j + off)];
    free(P);
    free(g);
}

/* Exported: rotate every frame of a [T][N][N] cube by theta_deg[t]. */
int oracle_rotate(const double *cube, double *out, long long T, int N, const double *theta_deg, int reduce90)
{
    if (T < 0 || N < 2 || (N & 1)) return -1;
    g_max_imag = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long long t = 0; t < T; t++)
        rotate_frame(cube + (size_t)t * N * N, out + (size_t)t * N * N, N, theta_deg[t], reduce90);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Angle gate and medians (Sect. 3.3).                                      */
/* ---------------------------------------------------------------------- */

/* alpha_min for an annulus whose inner radius is r (pixels), in degrees:
 * 2 asin(n_fwhm FWHM / (2 r)), the argument clamped to 1. */
double oracle_alpha_min_deg(double fwhm, double n_fwhm, double r)
{
    double arg = n_fwhm * fwhm / (2.0 * r);
    if (!(arg < 1.0)) arg = 1.0;
    return 2.0 * asin(arg) * 180.0 / ORACLE_PI;
}

/* Exported: reference set of frame i for one alpha_min, as a 0/1 mask over
 * the T frames (Sect. 3.3): |t_k - t_i| < t_max and |alpha_k - alpha_i| >
 * alpha_min.  times == NULL drops the time condition.  When no frame
 * qualifies, the frame(s) with the largest |alpha_k - alpha_i| among those
 * meeting the time condition. */
int oracle_gate_mask_t(const double *parang, const double *times, double t_max, long long T, long long i,
                       double amin, unsigned char *mask)
{
    long long n = 0;
    for (long long k = 0; k < T; k++) {
        int in_time = times == NULL || fabs(times[k] - times[i]) < t_max;
        mask[k] = in_time && fabs(parang[k] - parang[i]) > amin;
        n += mask[k];
    }
    if (n == 0) {
        double best = -1.0;
        for (long long k = 0; k < T; k++) {
            if (times != NULL && !(fabs(times[k] - times[i]) < t_max)) continue;
            double dk = fabs(parang[k] - parang[i]);
            if (dk > best) best = dk;
        }
        for (long long k = 0; k < T; k++) {
            int in_time = times == NULL || fabs(times[k] - times[i]) < t_max;
            mask[k] = in_time && fabs(parang[k] - parang[i]) == best;
        }
    }
    return 0;
}

int oracle_gate_mask(const double *parang, long long T, long long i, double amin, unsigned char *mask)
{
    return oracle_gate_mask_t(parang, NULL, 0.0, T, i, amin, mask);
}

/* IEEE total-order keys: a larger key means a larger value, -0 < +0. */
static uint64_t key64(double v)
{
    uint64_t b;
    memcpy(&b, &v, 8);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
static uint32_t key32(float v)
{
    uint32_t b;
    memcpy(&b, &v, 4);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}
static int cmp64(const void *a, const void *b)
{
    uint64_t x = key64(*(const double *)a), y = key64(*(const double *)b);
    return (x > y) - (x < y);
}
static int cmp32(const void *a, const void *b)
{
    uint32_t x = key32(*(const float *)a), y = key32(*(const float *)b);
    return (x > y) - (x < y);
}

/* Median of n values (sorted copy): odd n the middle value, even n the
 * mean of the two middle values, computed in the type of the data. */
static double median64(double *v, long long n)
{
    qsort(v, (size_t)n, sizeof(double), cmp64);
    if (n & 1) return v[n / 2];
    return (v[n / 2 - 1] + v[n / 2]) * 0.5;
}
static float median32(float *v, long long n)
{
    qsort(v, (size_t)n, sizeof(float), cmp32);
    if (n & 1) return v[n / 2];
    float s = v[n / 2 - 1] + v[n / 2];
    return s * 0.5f;
}

/* Annulus of pixel (i, j): index a with edges[a]^2 <= rho^2 < edges[a+1]^2,
 * rho^2 = x^2 + y^2, x = j - N/2, y = i - N/2; -1 outside [edges[0], edges[A]). */
static int annulus_of(int i, int j, int N, const double *edges, int n_edges)
{
    long long x = j - N / 2, y = i - N / 2;
    double rho2 = (double)(x * x + y * y);
    for (int a = 0; a + 1 < n_edges; a++)
        if (edges[a] * edges[a] <= rho2 && rho2 < edges[a + 1] * edges[a + 1]) return a;
    return -1;
}

int oracle_annulus_of(int i, int j, int N, const double *edges, int n_edges)
{
    return annulus_of(i, j, N, edges, n_edges);
}

/* Exported: angle-gated median PSF subtraction for a list of pixels
 * (flat indices p = i N + j), FP64.  out[n][t] = cube[t][p_n] - median of
 * cube[k][p_n] over the reference set of frame t; 0 for pixels outside the
 * annuli. */
int oracle_adi_subtract_pixels_t(const double *cube, long long T, int N, const double *parang,
                                 const double *times, double t_max, double fwhm, double n_fwhm,
                                 const double *edges, int n_edges, const long long *pix, long long n_pix,
                                 double *out)
{
    if (T < 1 || N < 2 || n_edges < 2) return -1;
    int A = n_edges - 1;
    double *amin = (double *)malloc(sizeof(double) * (size_t)A);
    for (int a = 0; a < A; a++) amin[a] = oracle_alpha_min_deg(fwhm, n_fwhm, edges[a]);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long long n = 0; n < n_pix; n++) {
        long long p = pix[n];
        int a = annulus_of((int)(p / N), (int)(p % N), N, edges, n_edges);
        unsigned char *mask = (unsigned char *)malloc((size_t)T);
        double *sel = (double *)malloc(sizeof(double) * (size_t)T);
        for (long long t = 0; t < T; t++) {
            if (a < 0) { out[n * T + t] = 0.0; continue; }
            oracle_gate_mask_t(parang, times, t_max, T, t, amin[a], mask);
            long long m = 0;
            for (long long k = 0; k < T; k++)
                if (mask[k]) sel[m++] = cube[(size_t)k * N * N + p];
            out[n * T + t] = cube[(size_t)t * N * N + p] - median64(sel, m);
        }
        free(mask);
        free(sel);
    }
    free(amin);
    return 0;
}

int oracle_adi_subtract_pixels(const double *cube, long long T, int N, const double *parang, double fwhm,
                               double n_fwhm, const double *edges, int n_edges, const long long *pix,
                               long long n_pix, double *out)
{
    return oracle_adi_subtract_pixels_t(cube, T, N, parang, NULL, 0.0, fwhm, n_fwhm, edges, n_edges, pix, n_pix,
                                        out);
}

/* Exported: the same on FP32 data with FP32 median arithmetic and an FP32
 * subtraction (for the bit-exact comparison on identical inputs). */
int oracle_adi_subtract_pixels_f32_t(const float *cube, long long T, int N, const double *parang,
                                     const double *times, double t_max, double fwhm, double n_fwhm,
                                     const double *edges, int n_edges, const long long *pix, long long n_pix,
                                     float *out)
{
    if (T < 1 || N < 2 || n_edges < 2) return -1;
    int A = n_edges - 1;
    double *amin = (double *)malloc(sizeof(double) * (size_t)A);
    for (int a = 0; a < A; a++) amin[a] = oracle_alpha_min_deg(fwhm, n_fwhm, edges[a]);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long long n = 0; n < n_pix; n++) {
        long long p = pix[n];
        int a = annulus_of((int)(p / N), (int)(p % N), N, edges, n_edges);
        unsigned char *mask = (unsigned char *)malloc((size_t)T);
        float *sel = (float *)malloc(sizeof(float) * (size_t)T);
        for (long long t = 0; t < T; t++) {
            if (a < 0) { out[n * T + t] = 0.0f; continue; }
            oracle_gate_mask_t(parang, times, t_max, T, t, amin[a], mask);
            long long m = 0;
            for (long long k = 0; k < T; k++)
                if (mask[k]) sel[m++] = cube[(size_t)k * N * N + p];
            float med = median32(sel, m);
            out[n * T + t] = cube[(size_t)t * N * N + p] - med;
        }
        free(mask);
        free(sel);
    }
    free(amin);
    return 0;
}

int oracle_adi_subtract_pixels_f32(const float *cube, long long T, int N, const double *parang, double fwhm,
                                   double n_fwhm, const double *edges, int n_edges, const long long *pix,
                                   long long n_pix, float *out)
{
    return oracle_adi_subtract_pixels_f32_t(cube, T, N, parang, NULL, 0.0, fwhm, n_fwhm, edges, n_edges, pix,
                                            n_pix, out);
}

/* Exported: median over the T frames for a list of pixels (FP64 / FP32). */
int oracle_collapse_median_pixels(const double *cube, long long T, int N, const long long *pix, long long n_pix,
                                  double *out)
{
    if (T < 1) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (long long n = 0; n < n_pix; n++) {
        double *v = (double *)malloc(sizeof(double) * (size_t)T);
        for (long long t = 0; t < T; t++) v[t] = cube[(size_t)t * N * N + pix[n]];
        out[n] = median64(v, T);
        free(v);
    }
    return 0;
}

int oracle_collapse_median_pixels_f32(const float *cube, long long T, int N, const long long *pix, long long n_pix,
                                      float *out)
{
    if (T < 1) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (long long n = 0; n < n_pix; n++) {
        float *v = (float *)malloc(sizeof(float) * (size_t)T);
        for (long long t = 0; t < T; t++) v[t] = cube[(size_t)t * N * N + pix[n]];
        out[n] = median32(v, T);
        free(v);
    }
    return 0;
}

/* Exported: the whole reduction in FP64 -- shift by (dx, dy), median PSF
 * subtraction, derotation by theta = -parang, median collapse.  work must
 * hold T N N doubles; out holds N N. */
int oracle_reduce_t(const double *cube, double *work, long long T, int N, const double *dx, const double *dy,
                    const double *parang, const double *times, double t_max, double fwhm, double n_fwhm,
                    const double *edges, int n_edges, double *out)
{
    if (T < 1 || N < 2 || (N & 1) || n_edges < 2) return -1;
    size_t NN = (size_t)N * N;
    double *tmp = (double *)malloc(sizeof(double) * NN * (size_t)T);
    long long *pix = (long long *)malloc(sizeof(long long) * NN);
    double *res = (double *)malloc(sizeof(double) * NN * (size_t)T);
    double *theta = (double *)malloc(sizeof(double) * (size_t)T);
    oracle_shift(cube, work, T, N, dx, dy);
    for (size_t p = 0; p < NN; p++) pix[p] = (long long)p;
    oracle_adi_subtract_pixels_t(work, T, N, parang, times, t_max, fwhm, n_fwhm, edges, n_edges, pix,
                                 (long long)NN, res);
    for (long long t = 0; t < T; t++)
        for (size_t p = 0; p < NN; p++) tmp[(size_t)t * NN + p] = res[p * (size_t)T + t];
    for (long long t = 0; t < T; t++) theta[t] = -parang[t];
    oracle_rotate(tmp, work, T, N, theta, 1);
    oracle_collapse_median_pixels(work, T, N, pix, (long long)NN, out);
    free(tmp);
    free(pix);
    free(res);
    free(theta);
    return 0;
}

int oracle_reduce(const double *cube, double *work, long long T, int N, const double *dx, const double *dy,
                  const double *parang, double fwhm, double n_fwhm, const double *edges, int n_edges, double *out)
{
    return oracle_reduce_t(cube, work, T, N, dx, dy, parang, NULL, 0.0, fwhm, n_fwhm, edges, n_edges, out);
}

/* ---------------------------------------------------------------------- */
/* Image-quality pre-processing (Sect. 3.2)                               */
/* ---------------------------------------------------------------------- */

/* Exported: master sky (Sect. 3.2, master sky): per pixel the median over
 * the T frames of the values that are finite and lie outside the star mask
 * of their frame (distance to (mask_x[t], mask_y[t]) below mask_r, pixel
 * coordinates x = column, y = row; mask_x == NULL: no mask).  A pixel with
 * no such value gets NaN.  FP32 data, FP32 median rule (the two middle
 * values averaged for even counts). */
int oracle_sky_median_f32(const float *cube, long long T, int N, const double *mask_x, const double *mask_y,
                          double mask_r, float *sky)
{
    if (T < 1 || N < 1) return -1;
    size_t NN = (size_t)N * N;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (long long p = 0; p < (long long)NN; p++) {
        float *v = (float *)malloc(sizeof(float) * (size_t)T);
        long long m = 0;
        double x = (double)(p % N), y = (double)(p / N);
        for (long long t = 0; t < T; t++) {
            float f = cube[(size_t)t * NN + p];
            if (!isfinite(f)) continue;
            if (mask_x) {
                double ddx = x - mask_x[t], ddy = y - mask_y[t];
                if (ddx * ddx + ddy * ddy < mask_r * mask_r) continue;
            }
            v[m++] = f;
        }
        sky[p] = m ? median32(v, m) : NAN;
        free(v);
    }
    return 0;
}

/* Exported: sky subtraction (Sect. 3.2): out[t] = in[t] - skies[j], j the
 * master sky closest in time to frame t (the earlier one on a tie). */
int oracle_sky_subtract_f32(const float *cube, float *out, long long T, int N, const float *skies, int n_skies,
                            const double *frame_times, const double *sky_times)
{
    if (T < 0 || n_skies < 1) return -1;
    size_t NN = (size_t)N * N;
    for (long long t = 0; t < T; t++) {
        int j = 0;
        for (int s = 1; s < n_skies; s++)
            if (fabs(sky_times[s] - frame_times[t]) < fabs(sky_times[j] - frame_times[t])) j = s;
        for (size_t p = 0; p < NN; p++) out[(size_t)t * NN + p] = cube[(size_t)t * NN + p] - skies[(size_t)j * NN + p];
    }
    return 0;
}

/* Exported: bad pixel map (Sect. 3.2, bad pixel correction): map[p] = 1
 * when |ref[p] - median(ref)| > C sigma, sigma the population standard
 * deviation of ref (FP64), the median of the N x N values in FP32 (two
 * middle values averaged for an even count), the comparison in FP64. */
int oracle_bad_pixel_map_f32(const float *ref, int N, double C, unsigned char *map)
{
    size_t NN = (size_t)N * N;
    if (NN < 1) return -1;
    float *v = (float *)malloc(sizeof(float) * NN);
    double mean = 0.0;
    for (size_t p = 0; p < NN; p++) {
        v[p] = ref[p];
        mean += ref[p];
    }
    mean /= (double)NN;
    double ss = 0.0;
    for (size_t p = 0; p < NN; p++) ss += ((double)ref[p] - mean) * ((double)ref[p] - mean);
    double sigma = sqrt(ss / (double)NN);
    float med = median32(v, (long long)NN);
    for (size_t p = 0; p < NN; p++) map[p] = fabs((double)ref[p] - (double)med) > C * sigma;
    free(v);
    return 0;
}

/* Exported: bad pixel correction (Sect. 3.2): in every frame the flagged
 * pixels (map != NULL) and the non-finite ones become NaN, then each NaN
 * pixel with at least one finite 8-neighbour takes the median of those
 * neighbours (FP32 median rule), all pixels of a pass reading the previous
 * pass's values, until no NaN is left (clumps fill from their border
 * inwards).  Returns 0, or 1 when a frame has no finite pixel at all. */
int oracle_bad_pixel_fix_f32(float *cube, long long T, int N, const unsigned char *map)
{
    size_t NN = (size_t)N * N;
    int status = 0;
    for (long long t = 0; t < T; t++) {
        float *f = cube + (size_t)t * NN;
        float *g = (float *)malloc(sizeof(float) * NN);
        long long nan_left = 0;
        for (size_t p = 0; p < NN; p++) {
            if ((map && map[p]) || !isfinite(f[p])) f[p] = NAN;
            nan_left += isnan(f[p]) ? 1 : 0;
        }
        while (nan_left > 0) {
            long long fixed = 0;
            memcpy(g, f, sizeof(float) * NN);
            for (int i = 0; i < N; i++)
                for (int j = 0; j < N; j++) {
                    if (!isnan(g[(size_t)i * N + j])) continue;
                    float nb[8];
                    long long m = 0;
                    for (int di = -1; di <= 1; di++)
                        for (int dj = -1; dj <= 1; dj++) {
                            if (!di && !dj) continue;
                            int ii = i + di, jj = j + dj;
                            if (ii < 0 || ii >= N || jj < 0 || jj >= N) continue;
                            float w = g[(size_t)ii * N + jj];
                            if (!isnan(w)) nb[m++] = w;
                        }
                    if (m) {
                        f[(size_t)i * N + j] = median32(nb, m);
                        fixed++;
                    }
                }
            if (fixed == 0) {
                status = 1;
                break;
            }
            nan_left -= fixed;
        }
        free(g);
    }
    return status;
}

/* ---------------------------------------------------------------------- */
/* Registration (Sect. 3.1): centroid patch search and Moffat fit          */
/* ---------------------------------------------------------------------- */

/* Exported: centroid search of one frame (Sect. 3.1, a connected group of
 * pixels above a threshold): the seed is the
 * brightest pixel (the first in row-major order on a tie); the patch is the
 * 8-connected set of pixels with value > thresh reachable from the seed
 * inside the box of half-size R around it (clipped to the frame).  The
 * centroid is found when the seed is above thresh, the patch touches no box
 * edge that lies inside the frame (else it may continue beyond the box) and
 * min_size <= |patch| <= max_size; it is then the flux-weighted centre of
 * mass sum v (x, y) / sum v of the patch (x = column, y = row, FP64).
 * Returns found (0/1); *size receives |patch|. */
int oracle_centroid_frame_f32(const float *f, int N, double thresh, int R, int min_size, int max_size, double *cx,
                              double *cy, int *size)
{
    size_t NN = (size_t)N * N, best = 0;
    for (size_t p = 1; p < NN; p++)
        if (f[p] > f[best]) best = p;
    int r0 = (int)(best / N), c0 = (int)(best % N);
    int rlo = r0 - R < 0 ? 0 : r0 - R, rhi = r0 + R >= N ? N - 1 : r0 + R;
    int clo = c0 - R < 0 ? 0 : c0 - R, chi = c0 + R >= N ? N - 1 : c0 + R;
    int H = rhi - rlo + 1, W = chi - clo + 1;
    *size = 0;
    *cx = *cy = 0.0;
    if (!((double)f[best] > thresh)) return 0;
    unsigned char *lab = (unsigned char *)calloc((size_t)H * W, 1);
    int *stack = (int *)malloc(sizeof(int) * (size_t)H * W);
    int top = 0, n = 0, touch = 0;
    double sv = 0.0, sx = 0.0, sy = 0.0;
    lab[(size_t)(r0 - rlo) * W + (c0 - clo)] = 1;
    stack[top++] = (r0 - rlo) * W + (c0 - clo);
    while (top > 0) {
        int q = stack[--top];
        int r = q / W, c = q % W;
        double v = (double)f[(size_t)(r + rlo) * N + (c + clo)];
        n++;
        sv += v;
        sx += v * (double)(c + clo);
        sy += v * (double)(r + rlo);
        if ((r == 0 && rlo > 0) || (r == H - 1 && rhi < N - 1) || (c == 0 && clo > 0) || (c == W - 1 && chi < N - 1))
            touch = 1;
        for (int dr = -1; dr <= 1; dr++)
            for (int dc = -1; dc <= 1; dc++) {
                int rr = r + dr, cc = c + dc;
                if ((!dr && !dc) || rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
                size_t k = (size_t)rr * W + cc;
                if (lab[k]) continue;
                if ((double)f[(size_t)(rr + rlo) * N + (cc + clo)] > thresh) {
                    lab[k] = 1;
                    stack[top++] = (int)k;
                }
            }
    }
    free(lab);
    free(stack);
    *size = n;
    if (touch || n < min_size || n > max_size) return 0;
    *cx = sx / sv;
    *cy = sy / sv;
    return 1;
}

/* Moffat model (Sect. 3.1) and its partial derivatives in the parameters
 * p = (I0, x0, y0, alpha, beta, Bg) at pixel (x, y). */
static double moffat_eval(const double *p, double x, double y, double *grad)
{
    double I0 = p[0], x0 = p[1], y0 = p[2], al = p[3], be = p[4];
    double dx = x - x0, dy = y - y0, rho2 = dx * dx + dy * dy;
    double u = 1.0 + rho2 / (al * al);
    double P = exp(-be * log(u));
    double A = I0 * (be - 1.0) / (ORACLE_PI * al * al);
    if (grad) {
        double Pu = P / u;   /* u^(-beta-1) */
        grad[0] = (be - 1.0) / (ORACLE_PI * al * al) * P;
        grad[1] = A * be * Pu * 2.0 * dx / (al * al);
        grad[2] = A * be * Pu * 2.0 * dy / (al * al);
        grad[3] = -2.0 * A / al * P + A * 2.0 * be * rho2 * Pu / (al * al * al);
        grad[4] = I0 / (ORACLE_PI * al * al) * P - A * log(u) * P;
        grad[5] = 1.0;
    }
    return A * P + p[5];
}

static double moffat_cost(const double *p, const float *f, int N, int r0, int r1, int c0, int c1)
{
    double s = 0.0;
    for (int r = r0; r <= r1; r++)
        for (int c = c0; c <= c1; c++) {
            double e = moffat_eval(p, (double)c, (double)r, NULL) - (double)f[(size_t)r * N + c];
            s += e * e;
        }
    return s;
}

/* 6 x 6 symmetric positive definite solve by Cholesky; 0 on failure. */
static int chol6(const double *A, const double *b, double *x)
{
    double L[36] = {0};
    for (int i = 0; i < 6; i++)
        for (int j = 0; j <= i; j++) {
            double s = A[i * 6 + j];
            for (int k = 0; k < j; k++) s -= L[i * 6 + k] * L[j * 6 + k];
            if (i == j) {
                if (!(s > 0)) return 0;
                L[i * 6 + i] = sqrt(s);
            } else {
                L[i * 6 + j] = s / L[j * 6 + j];
            }
        }
    double y[6];
    for (int i = 0; i < 6; i++) {
        double s = b[i];
        for (int k = 0; k < i; k++) s -= L[i * 6 + k] * y[k];
        y[i] = s / L[i * 6 + i];
    }
    for (int i = 5; i >= 0; i--) {
        double s = y[i];
        for (int k = i + 1; k < 6; k++) s -= L[k * 6 + i] * x[k];
        x[i] = s / L[i * 6 + i];
    }
    return 1;
}

/* Exported: Moffat fit of one frame (Sect. 3.1) by Levenberg-Marquardt over
 * the window of half-size w around the rounded initial centre (clipped to
 * the frame).  Start: (x0, y0) = (cx, cy), Bg = window minimum, beta = 2.5,
 * alpha = alpha0, I0 = sum over the window of (v - Bg).  Iteration: normal
 * equations of the analytic Jacobian, damped by lambda * diag (lambda from
 * 1e-3, /10 on an accepted step, *10 on a rejected one or on alpha <= 0,
 * beta <= 1), stop when an accepted step lowers the cost by less than 1e-14
 * of it, when no damping up to 10 tries lowers it, or after 200 iterations.
 * p_out = (I0, x0, y0, alpha, beta, Bg); returns the iterations made. */
int oracle_moffat_fit_f32(const float *f, int N, double cx, double cy, double alpha0, int w, double *p_out)
{
    int rc_ = (int)floor(cy + 0.5), cc_ = (int)floor(cx + 0.5);
    int r0 = rc_ - w < 0 ? 0 : rc_ - w, r1 = rc_ + w >= N ? N - 1 : rc_ + w;
    int c0 = cc_ - w < 0 ? 0 : cc_ - w, c1 = cc_ + w >= N ? N - 1 : cc_ + w;
    double bg = (double)f[(size_t)r0 * N + c0];
    for (int r = r0; r <= r1; r++)
        for (int c = c0; c <= c1; c++) bg = fmin(bg, (double)f[(size_t)r * N + c]);
    double I0 = 0.0;
    for (int r = r0; r <= r1; r++)
        for (int c = c0; c <= c1; c++) I0 += (double)f[(size_t)r * N + c] - bg;
    double p[6] = {I0, cx, cy, alpha0, 2.5, bg};
    double lambda = 1e-3;
    double cost = moffat_cost(p, f, N, r0, r1, c0, c1);
    int it;
    for (it = 0; it < 200; it++) {
        double JJ[36] = {0}, g[6] = {0};
        for (int r = r0; r <= r1; r++)
            for (int c = c0; c <= c1; c++) {
                double gr[6];
                double e = moffat_eval(p, (double)c, (double)r, gr) - (double)f[(size_t)r * N + c];
                for (int i = 0; i < 6; i++) {
                    g[i] += gr[i] * e;
                    for (int j = 0; j <= i; j++) JJ[i * 6 + j] += gr[i] * gr[j];
                }
            }
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < i; j++) JJ[j * 6 + i] = JJ[i * 6 + j];
        int accepted = 0;
        double newcost = cost;
        for (int tries = 0; tries < 10; tries++) {
            double A[36], mg[6], d[6], q[6];
            for (int i = 0; i < 36; i++) A[i] = JJ[i];
            for (int i = 0; i < 6; i++) {
                double di = JJ[i * 6 + i] > 0 ? JJ[i * 6 + i] : 1e-12;
                A[i * 6 + i] += lambda * di;
                mg[i] = -g[i];
            }
            if (!chol6(A, mg, d)) {
                lambda *= 10.0;
                continue;
            }
            for (int i = 0; i < 6; i++) q[i] = p[i] + d[i];
            if (!(q[3] > 0) || !(q[4] > 1.0)) {
                lambda *= 10.0;
                continue;
            }
            newcost = moffat_cost(q, f, N, r0, r1, c0, c1);
            if (newcost < cost) {
                for (int i = 0; i < 6; i++) p[i] = q[i];
                lambda = fmax(lambda / 10.0, 1e-12);
                accepted = 1;
                break;
            }
            lambda *= 10.0;
        }
        if (!accepted) break;
        double drop = cost - newcost;
        cost = newcost;
        if (drop <= 1e-14 * cost) {
            it++;
            break;
        }
    }
    for (int i = 0; i < 6; i++) p_out[i] = p[i];
    return it;
}

/* FWHM of the Moffat profile (Sect. 3.1): 2 alpha sqrt(2^(1/beta) - 1). */
double oracle_moffat_fwhm(double alpha, double beta)
{
    return 2.0 * alpha * sqrt(pow(2.0, 1.0 / beta) - 1.0);
}

/* ---------------------------------------------------------------------- */
/* Photometric-accuracy and binning experiments (Sect. 4.2, 4.3)           */
/* ---------------------------------------------------------------------- */

/* Exported: median binning (Sect. 4.3, each run of ten frames replaced by
 * its median frame; the quick-look binning of Sect. 3.1): group g
 * holds frames [g B, min(T, (g + 1) B)) (the last group may be shorter) and
 * out[g](p) is the median of its values at pixel p, by the median rule of
 * the collapse (sort, middle value, mean of the two middle values in FP32
 * for an even count).  out has ceil(T / B) frames. */
int oracle_bin_median_f32(const float *cube, long long T, int N, int B, float *out)
{
    if (T < 0 || N < 1 || B < 1) return -1;
    long long G = (T + B - 1) / B, NN = (long long)N * N;
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < G * NN; q++) {
        long long g = q / NN, p = q % NN;
        long long f0 = g * B, f1 = f0 + B < T ? f0 + B : T;
        float v[4096];
        float *buf = (f1 - f0) <= 4096 ? v : (float *)malloc(sizeof(float) * (size_t)(f1 - f0));
        for (long long f = f0; f < f1; f++) buf[f - f0] = cube[f * NN + p];
        out[g * NN + p] = median32(buf, f1 - f0);
        if (buf != v) free(buf);
    }
    return 0;
}

/* Exported: fake companion injection (Sect. 4.2: companions injected into
 * the raw frames at an angle following the field rotation).  Companion j of
 * frame t sits at (xc[t] + r_j cos(pa0_j + parang_t), yc[t] + r_j sin(pa0_j +
 * parang_t)) (x = column, y = row, degrees, counter-clockwise from +x), its
 * profile the Moffat function of Sect. 3.1 with total flux flux_j and the
 * frame's alpha[t], beta[t]: flux_j (beta - 1) / (pi alpha^2) (1 + rho^2 /
 * alpha^2)^(-beta), evaluated in FP64 on the pixels of the square window of
 * half-size `half` around the rounded position (clipped to the frame) and
 * added to the FP32 frame as (float)((double)v + sum of the companions). */
int oracle_inject_f32(float *cube, long long T, int N, const double *parang, const double *xc, const double *yc,
                      int n_comp, const double *r, const double *pa0, const double *flux, const double *alpha,
                      const double *beta, int half)
{
    if (T < 0 || N < 1 || n_comp < 0 || half < 0) return -1;
    long long NN = (long long)N * N;
#pragma omp parallel for schedule(static)
    for (long long t = 0; t < T; t++) {
        double *add = (double *)calloc((size_t)NN, sizeof(double));
        for (int j = 0; j < n_comp; j++) {
            double ang = (pa0[j] + parang[t]) * ORACLE_PI / 180.0;
            double xp = xc[t] + r[j] * cos(ang), yp = yc[t] + r[j] * sin(ang);
            long long cr = (long long)floor(yp + 0.5), cc = (long long)floor(xp + 0.5);
            double al = alpha[t], be = beta[t];
            double A = flux[j] * (be - 1.0) / (ORACLE_PI * al * al);
            for (long long row = cr - half; row <= cr + half; row++) {
                if (row < 0 || row >= N) continue;
                for (long long col = cc - half; col <= cc + half; col++) {
                    if (col < 0 || col >= N) continue;
                    double dx = (double)col - xp, dy = (double)row - yp;
                    add[row * N + col] += A * pow(1.0 + (dx * dx + dy * dy) / (al * al), -be);
                }
            }
        }
        for (long long p = 0; p < NN; p++)
            if (add[p] != 0.0) cube[t * NN + p] = (float)((double)cube[t * NN + p] + add[p]);
        free(add);
    }
    return 0;
}

/* Exported: aperture photometry for the recovered flux (Sect. 4.2): out[k]
 * = sum of img over the pixels whose centres lie within `radius` of (x[k],
 * y[k]), (col - x)^2 + (row - y)^2 <= radius^2, in FP64. */
int oracle_aperture_f32(const float *img, int N, int n_ap, const double *x, const double *y, double radius,
                        double *out)
{
    if (N < 1 || n_ap < 0 || !(radius >= 0)) return -1;
    for (int k = 0; k < n_ap; k++) {
        double s = 0.0;
        for (int row = 0; row < N; row++)
            for (int col = 0; col < N; col++) {
                double dx = (double)col - x[k], dy = (double)row - y[k];
                if (dx * dx + dy * dy <= radius * radius) s += (double)img[(size_t)row * N + col];
            }
        out[k] = s;
    }
    return 0;
}
