/*
 * rs_oracle.c -- plain, slow FP64 CPU oracle for separable image resampling
 * with reconstruction filters.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product path (paper_1110_5450_b300/) never links, loads or calls it, and it
 * shares no code, header, table or constant with that path.
 *
 * What it computes (the plain definition, evaluated literally):
 *
 *   out[y][x][c] = sum_j sum_i  wy(y, j) * wx(x, i) * in[B_h(j)][B_w(i)][c]
 *
 * a direct two-dimensional summation (not separable in evaluation order) in
 * double precision, where for one axis with n_in input and n_out output
 * samples:
 *
 *  - Coordinates: half-pixel centres.  Output sample i sits at input
 *    coordinate c_i = (i + 1/2) * n_in / n_out; input sample j sits at j + 1/2.
 *  - Antialiasing: the kernel is widened by sc = max(1, n_in / n_out), i.e. it
 *    is evaluated at x = (j + 1/2 - c_i) / sc.  Multiplying out gives an exact
 *    integer numerator and denominator:
 *        x = ((2j+1) n_out - (2i+1) n_in) / D,  D = 2 max(n_in, n_out)
 *    (D = 2 n_out when antialiasing is switched off).
 *  - Taps: every integer j with |x| < R (R = kernel support radius), found by
 *    scanning candidate j with that exact integer test.
 *  - Kernels (standard published definitions):
 *        linear (tent), R = 1:          1 - |x|
 *        Keys cubic convolution, R = 2 (R. Keys, IEEE Trans. ASSP 29(6), 1981):
 *            (a+2)|x|^3 - (a+3)|x|^2 + 1           |x| < 1
 *            a|x|^3 - 5a|x|^2 + 8a|x| - 4a         1 <= |x| < 2
 *        Lanczos-R windowed sinc (C. Duchon, J. Appl. Meteor. 18, 1979):
 *            sinc(x) sinc(x / R),  sinc(t) = sin(pi t) / (pi t),  sinc(0) = 1
 *        cubic B-spline beta^3, R = 2 (M. Unser, IEEE SP Mag. 16(6), 1999):
 *            2/3 - |x|^2 + |x|^3 / 2               |x| < 1
 *            (2 - |x|)^3 / 6                       1 <= |x| < 2
 *        Mitchell-Netravali cubic, R = 2 (D. Mitchell, A. Netravali,
 *        SIGGRAPH 1988), with B = param and C = (1 - B) / 2:
 *            ((12 - 9B - 6C)|x|^3 + (-18 + 12B + 6C)|x|^2 + (6 - 2B)) / 6
 *                                                  |x| < 1
 *            ((-B - 6C)|x|^3 + (6B + 30C)|x|^2 + (-12B - 48C)|x|
 *             + (8B + 24C)) / 6                    1 <= |x| < 2
 *        Gaussian, sigma = param in (0, 4], truncated at R = ceil(3 sigma):
 *            exp(-x^2 / (2 sigma^2))               |x| < R
 *  - Normalisation: w <- w / sum(w) over the taps (for the truncate boundary,
 *    over the in-range taps only).
 *  - Boundary maps B for an index j on an axis of n samples:
 *        clamp       min(max(j, 0), n - 1)
 *        mirror      half-sample symmetric, period 2n:
 *                    m = j mod 2n (non-negative); m < n ? m : 2n - 1 - m
 *        reflect101  whole-sample symmetric, period 2n - 2 (n = 1: always 0)
 *        truncate    taps outside [0, n) are dropped
 *  - No clamping of the output: overshoot of cubic and Lanczos is kept.
 *
 * The paper this build follows states no resampling formula of its own;
 * every definition above is the standard one cited beside it.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

enum { ORA_LINEAR = 0, ORA_CUBIC = 1, ORA_LANCZOS = 2, ORA_BSPLINE3 = 3, ORA_MITCHELL = 4, ORA_GAUSSIAN = 5 };
enum { ORA_CLAMP = 0, ORA_MIRROR = 1, ORA_REFLECT101 = 2, ORA_TRUNCATE = 3 };

#define ORA_PI 3.14159265358979323846

/* Support radius R of each kernel (integer; Lanczos takes it as parameter). */
int ora_support(int kernel, double param, int64_t *R)
{
    switch (kernel) {
    case ORA_LINEAR: *R = 1; return 0;
    case ORA_CUBIC: *R = 2; return 0;
    case ORA_BSPLINE3: *R = 2; return 0;
    case ORA_LANCZOS:
        if (!(param >= 1.0 && param <= 16.0) || param != floor(param)) return -1;
        *R = (int64_t)param;
        return 0;
    case ORA_MITCHELL:
        if (!(param >= 0.0 && param <= 1.0)) return -1;
        *R = 2;
        return 0;
    case ORA_GAUSSIAN:
        if (!(param > 0.0 && param <= 4.0)) return -1;
        *R = (int64_t)ceil(3.0 * param);
        return 0;
    }
    return -1;
}

/* sin(pi t) with exact argument reduction: t = k + f, k the nearest integer,
 * |f| <= 1/2, so sin(pi t) = (-1)^k sin(pi f).  Exact zero at integer t. */
static double ora_sin_pi(double t)
{
    double k = nearbyint(t);
    double f = t - k; /* exact: t and k are within 1/2 of each other */
    if (f == 0.0) return 0.0;
    double s = sin(ORA_PI * f);
    return (fmod(k, 2.0) != 0.0) ? -s : s;
}

static double ora_sinc(double t)
{
    if (t == 0.0) return 1.0;
    return ora_sin_pi(t) / (ORA_PI * t);
}

/* Kernel value K(x), zero outside the support |x| < R. */
double ora_kernel_value(int kernel, double param, double x)
{
    double t = fabs(x);
    switch (kernel) {
    case ORA_LINEAR:
        return t < 1.0 ? 1.0 - t : 0.0;
    case ORA_CUBIC: {
        double a = param;
        if (t < 1.0) return (a + 2.0) * t * t * t - (a + 3.0) * t * t + 1.0;
        if (t < 2.0) return a * t * t * t - 5.0 * a * t * t + 8.0 * a * t - 4.0 * a;
        return 0.0;
    }
    case ORA_LANCZOS: {
        double R = param;
        if (t >= R) return 0.0;
        return ora_sinc(x) * ora_sinc(x / R);
    }
    case ORA_BSPLINE3:
        if (t < 1.0) return 2.0 / 3.0 - t * t + t * t * t / 2.0;
        if (t < 2.0) return (2.0 - t) * (2.0 - t) * (2.0 - t) / 6.0;
        return 0.0;
    case ORA_MITCHELL: {
        double B = param, C = (1.0 - B) / 2.0;
        if (t < 1.0)
            return ((12.0 - 9.0 * B - 6.0 * C) * t * t * t + (-18.0 + 12.0 * B + 6.0 * C) * t * t + (6.0 - 2.0 * B)) /
                   6.0;
        if (t < 2.0)
            return ((-B - 6.0 * C) * t * t * t + (6.0 * B + 30.0 * C) * t * t + (-12.0 * B - 48.0 * C) * t +
                    (8.0 * B + 24.0 * C)) /
                   6.0;
        return 0.0;
    }
    case ORA_GAUSSIAN: {
        double R = ceil(3.0 * param);
        if (t >= R) return 0.0;
        return exp(-(x * x) / (2.0 * param * param));
    }
    }
    return 0.0;
}

/* Denominator D of the kernel argument x = N / D (see header). */
static int64_t ora_denominator(int64_t n_in, int64_t n_out, int antialias)
{
    if (antialias && n_in > n_out) return 2 * n_in;
    return 2 * n_out;
}

/* Raw taps of output i: first index j_first (may be negative or >= n_in) and
 * the number of consecutive j with |x| < R.  Found by scanning candidates in a
 * generous bracket around the output centre with the exact integer test
 * |(2j+1) n_out - (2i+1) n_in| < R D. */
int ora_axis_taps(int64_t n_in, int64_t n_out, int kernel, double param,
                  int antialias, int64_t i, int64_t *j_first, int64_t *count)
{
    int64_t R;
    if (n_in < 1 || n_out < 1 || i < 0 || i >= n_out) return -1;
    if (ora_support(kernel, param, &R)) return -1;
    int64_t D = ora_denominator(n_in, n_out, antialias);
    double sc = (double)D / (2.0 * (double)n_out);
    double centre = ((double)(2 * i + 1) * (double)n_in) / (2.0 * (double)n_out);
    int64_t lo = (int64_t)floor(centre - 0.5 - (double)R * sc) - 2;
    int64_t hi = (int64_t)ceil(centre - 0.5 + (double)R * sc) + 2;
    int64_t first = 0, n = 0;
    for (int64_t j = lo; j <= hi; ++j) {
        int64_t num = (2 * j + 1) * n_out - (2 * i + 1) * n_in;
        if (num < 0) num = -num;
        if (num < R * D) {
            if (n == 0) first = j;
            else if (j != first + n) return -2; /* taps must be consecutive */
            ++n;
        }
    }
    *j_first = first;
    *count = n;
    return 0;
}

/* Boundary map; returns -1 for a dropped tap (truncate). */
int64_t ora_boundary_map(int64_t j, int64_t n, int boundary)
{
    switch (boundary) {
    case ORA_CLAMP:
        return j < 0 ? 0 : (j >= n ? n - 1 : j);
    case ORA_MIRROR: {
        int64_t p = 2 * n;
        int64_t m = j % p;
        if (m < 0) m += p;
        return m < n ? m : p - 1 - m;
    }
    case ORA_REFLECT101: {
        if (n == 1) return 0;
        int64_t p = 2 * n - 2;
        int64_t m = j % p;
        if (m < 0) m += p;
        return m < n ? m : p - m;
    }
    case ORA_TRUNCATE:
        return (j < 0 || j >= n) ? -1 : j;
    }
    return -1;
}

/* Normalised weights of output i on one axis.  idx[k] is the boundary-mapped
 * input index of raw tap k (or -1 when dropped), w[k] its normalised weight
 * (0 when dropped).  Returns the raw tap count in *count (<= cap). */
int ora_axis_weights(int64_t n_in, int64_t n_out, int kernel, double param,
                     int boundary, int antialias, int64_t i, int64_t cap,
                     int64_t *j_first, int64_t *count, int64_t *idx, double *w)
{
    int64_t first, n;
    int rc = ora_axis_taps(n_in, n_out, kernel, param, antialias, i, &first, &n);
    if (rc) return rc;
    if (n > cap) return -3;
    int64_t D = ora_denominator(n_in, n_out, antialias);
    double sum = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = first + k;
        int64_t num = (2 * j + 1) * n_out - (2 * i + 1) * n_in;
        double x = (double)num / (double)D;
        int64_t m = ora_boundary_map(j, n_in, boundary);
        idx[k] = m;
        w[k] = (m < 0) ? 0.0 : ora_kernel_value(kernel, param, x);
        sum += w[k];
    }
    if (!(sum != 0.0)) return -4;
    for (int64_t k = 0; k < n; ++k) w[k] = w[k] / sum;
    *j_first = first;
    *count = n;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Two-dimensional direct summation, threaded over output rows.            */

typedef struct {
    const double *in;
    double *out;
    int64_t in_h, in_w, ch, out_h, out_w;
    int64_t y_begin, y_end;
    int kernel, boundary, antialias;
    double param;
    int64_t cap_h, cap_w;
    /* per-column weights, computed once: */
    const int64_t *cnt_w, *idx_w;
    const double *wt_w;
    int64_t next_row; /* shared work counter */
    pthread_mutex_t lock;
    int status;
} ora_job;

static void *ora_worker(void *arg)
{
    ora_job *J = (ora_job *)arg;
    int64_t *idx_h = (int64_t *)malloc(sizeof(int64_t) * (size_t)J->cap_h);
    double *wt_h = (double *)malloc(sizeof(double) * (size_t)J->cap_h);
    if (!idx_h || !wt_h) {
        pthread_mutex_lock(&J->lock);
        J->status = -5;
        pthread_mutex_unlock(&J->lock);
        free(idx_h);
        free(wt_h);
        return NULL;
    }
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t y = J->next_row++;
        pthread_mutex_unlock(&J->lock);
        if (y >= J->y_end) break;
        int64_t first, n;
        int rc = ora_axis_weights(J->in_h, J->out_h, J->kernel, J->param, J->boundary,
                                  J->antialias, y, J->cap_h, &first, &n, idx_h, wt_h);
        if (rc) {
            pthread_mutex_lock(&J->lock);
            J->status = rc;
            pthread_mutex_unlock(&J->lock);
            break;
        }
        double *orow = J->out + (y - J->y_begin) * J->out_w * J->ch;
        for (int64_t x = 0; x < J->out_w; ++x) {
            int64_t nx = J->cnt_w[x];
            const int64_t *ix = J->idx_w + x * J->cap_w;
            const double *wx = J->wt_w + x * J->cap_w;
            for (int64_t c = 0; c < J->ch; ++c) {
                double acc = 0.0;
                for (int64_t ty = 0; ty < n; ++ty) {
                    if (idx_h[ty] < 0) continue;
                    const double *irow = J->in + idx_h[ty] * J->in_w * J->ch;
                    for (int64_t tx = 0; tx < nx; ++tx) {
                        if (ix[tx] < 0) continue;
                        acc += wt_h[ty] * wx[tx] * irow[ix[tx] * J->ch + c];
                    }
                }
                orow[x * J->ch + c] = acc;
            }
        }
    }
    free(idx_h);
    free(wt_h);
    return NULL;
}

/* Upper bound on the raw tap count of one axis: the tap centres (2j+1) n_out
 * are spaced 2 n_out apart inside an open interval of length 2 R D. */
static int64_t ora_tap_cap(int64_t n_in, int64_t n_out, int antialias, int64_t R)
{
    int64_t D = ora_denominator(n_in, n_out, antialias);
    return (2 * R * D) / (2 * n_out) + 2;
}

/* Resample output rows [y_begin, y_end) of an HWC image.  out holds
 * (y_end - y_begin) * out_w * ch doubles.  nthreads <= 0 uses every online
 * core.  Returns 0 on success. */
int ora_resample_rows(const double *in, int64_t in_h, int64_t in_w, int64_t ch,
                      int64_t out_h, int64_t out_w, int kernel, double param,
                      int boundary, int antialias, int64_t y_begin, int64_t y_end,
                      double *out, int nthreads)
{
    int64_t R;
    if (in_h < 1 || in_w < 1 || ch < 1 || out_h < 1 || out_w < 1) return -1;
    if (y_begin < 0 || y_end > out_h || y_begin > y_end) return -1;
    if (boundary < ORA_CLAMP || boundary > ORA_TRUNCATE) return -1;
    if (ora_support(kernel, param, &R)) return -1;
    if (y_begin == y_end) return 0;

    ora_job J;
    memset(&J, 0, sizeof J);
    J.in = in; J.out = out;
    J.in_h = in_h; J.in_w = in_w; J.ch = ch; J.out_h = out_h; J.out_w = out_w;
    J.y_begin = y_begin; J.y_end = y_end; J.next_row = y_begin;
    J.kernel = kernel; J.boundary = boundary; J.antialias = antialias; J.param = param;
    J.cap_h = ora_tap_cap(in_h, out_h, antialias, R);
    J.cap_w = ora_tap_cap(in_w, out_w, antialias, R);

    int64_t *cnt_w = (int64_t *)malloc(sizeof(int64_t) * (size_t)out_w);
    int64_t *idx_w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(out_w * J.cap_w));
    double *wt_w = (double *)malloc(sizeof(double) * (size_t)(out_w * J.cap_w));
    if (!cnt_w || !idx_w || !wt_w) {
        free(cnt_w); free(idx_w); free(wt_w);
        return -5;
    }
    for (int64_t x = 0; x < out_w; ++x) {
        int64_t first;
        int rc = ora_axis_weights(in_w, out_w, kernel, param, boundary, antialias, x,
                                  J.cap_w, &first, &cnt_w[x], idx_w + x * J.cap_w,
                                  wt_w + x * J.cap_w);
        if (rc) {
            free(cnt_w); free(idx_w); free(wt_w);
            return rc;
        }
    }
    J.cnt_w = cnt_w; J.idx_w = idx_w; J.wt_w = wt_w;
    pthread_mutex_init(&J.lock, NULL);

    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t tid[256];
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (pthread_create(&tid[t], NULL, ora_worker, &J) != 0) break;
        ++started;
    }
    if (started == 0) ora_worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    pthread_mutex_destroy(&J.lock);
    free(cnt_w); free(idx_w); free(wt_w);
    return J.status;
}

/* Whole image. */
int ora_resample(const double *in, int64_t in_h, int64_t in_w, int64_t ch,
                 int64_t out_h, int64_t out_w, int kernel, double param,
                 int boundary, int antialias, double *out, int nthreads)
{
    return ora_resample_rows(in, in_h, in_w, ch, out_h, out_w, kernel, param,
                             boundary, antialias, 0, out_h, out, nthreads);
}

/* Number of worker threads ora_resample uses when nthreads <= 0. */
int ora_default_threads(void)
{
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    if (n < 1) n = 1;
    if (n > 256) n = 256;
    return (int)n;
}
