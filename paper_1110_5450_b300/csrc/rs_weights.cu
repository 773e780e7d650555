// rs_weights.cu -- FP64 weight-table kernel and register-band builder.
//
// One thread per output sample of an axis.  Tap indices come from a closed
// form in 64-bit integers (exact), weights from the kernel evaluated in FP64
// at x = ((2j+1) n_out - (2i+1) n_in) / D (one correctly rounded division of
// exact integers), normalised by their FP64 sum, folded through the boundary
// map into a window of t_eff consecutive in-range inputs, then rounded to the
// working precision with the rounding residual put back on the largest tap.
//
// Kernel definitions (standard): tent; Keys cubic convolution (R. Keys, IEEE
// Trans. ASSP 29(6), 1981); Lanczos windowed sinc (C. Duchon, J. Appl.
// Meteor. 18, 1979); cubic B-spline (M. Unser, IEEE SP Mag. 16(6), 1999).
#include "rs_internal.h"

namespace rs {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

enum : int { kErrTaps = 101, kErrSum = 102, kErrBand = 103 };

__device__ __forceinline__ void flag_error(int *err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

// floor(a / b) and ceil(a / b) for b > 0.
__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
__device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    return (a % b != 0 && a > 0) ? q + 1 : q;
}

__device__ double kernel_eval(int kernel, double a, int64_t R, double x)
{
    const double t = fabs(x);
    switch (kernel) {
    case RS_K_LINEAR:
        return t < 1.0 ? 1.0 - t : 0.0;
    case RS_K_CUBIC:
        if (t < 1.0) return ((a + 2.0) * t - (a + 3.0)) * t * t + 1.0;
        if (t < 2.0) return ((a * t - 5.0 * a) * t + 8.0 * a) * t - 4.0 * a;
        return 0.0;
    case RS_K_LANCZOS: {
        if (t >= double(R)) return 0.0;
        if (x == 0.0) return 1.0;
        const double xr = x / double(R);
        return (sinpi(x) / (kPi * x)) * (sinpi(xr) / (kPi * xr));
    }
    case RS_K_BSPLINE3:
        if (t < 1.0) return (0.5 * t - 1.0) * t * t + 2.0 / 3.0;
        if (t < 2.0) {
            const double u = 2.0 - t;
            return u * u * u / 6.0;
        }
        return 0.0;
    }
    return 0.0;
}

// Boundary map; -1 drops the tap (truncate).
__device__ __forceinline__ int64_t map_index(int64_t j, int64_t n, int boundary)
{
    if (j >= 0 && j < n) return j;
    switch (boundary) {
    case RS_B_CLAMP:
        return j < 0 ? 0 : n - 1;
    case RS_B_MIRROR: {
        const int64_t p = 2 * n;
        int64_t m = j % p;
        if (m < 0) m += p;
        return m < n ? m : p - 1 - m;
    }
    case RS_B_REFLECT101: {
        if (n == 1) return 0;
        const int64_t p = 2 * n - 2;
        int64_t m = j % p;
        if (m < 0) m += p;
        return m < n ? m : p - m;
    }
    default:
        return -1;
    }
}

__device__ void axis_weights(const WeightArgs &A, int64_t i)
{
    const AxisGeom &g = A.g;
    const AxisTables &T = A.t;
    const int64_t N0 = (2 * i + 1) * g.n_in;
    const int64_t two_out = 2 * g.n_out;
    const int64_t RD = g.R * g.D;
    // first raw tap: smallest j with (2j+1) n_out > N0 - R D
    const int64_t jlo = floor_div(N0 - RD - g.n_out, two_out) + 1;
    // last raw tap: largest j with (2j+1) n_out < N0 + R D
    const int64_t jhi = ceil_div(N0 + RD - g.n_out, two_out) - 1;
    const int64_t cnt = jhi - jlo + 1;
    T.jlo[i] = int32_t(jlo);
    T.cnt[i] = int32_t(cnt);
    const int te = g.t_eff;
    double *w = T.w64 + i * te;
    if (cnt < 1 || cnt > g.t_raw) {
        flag_error(A.err, kErrTaps);
        T.start[i] = 0;
        for (int k = 0; k < te; ++k) w[k] = 0.0;
        return;
    }
    const double D = double(g.D);
    double sum = 0.0;
    int64_t mlo = g.n_in, mhi = -1;
    for (int64_t k = 0; k < cnt; ++k) {
        const int64_t j = jlo + k;
        const int64_t m = map_index(j, g.n_in, g.boundary);
        if (m < 0) continue;
        const double x = double((2 * j + 1) * g.n_out - N0) / D;
        sum += kernel_eval(g.kernel, g.param, g.R, x);
        mlo = m < mlo ? m : mlo;
        mhi = m > mhi ? m : mhi;
    }
    int64_t start = mlo < g.n_in - te ? mlo : g.n_in - te;
    if (start < 0) start = 0;
    T.start[i] = int32_t(start);
    for (int k = 0; k < te; ++k) w[k] = 0.0;
    if (!(sum != 0.0) || mhi < 0 || mhi - start >= te) {
        flag_error(A.err, kErrSum);
        return;
    }
    for (int64_t k = 0; k < cnt; ++k) {
        const int64_t j = jlo + k;
        const int64_t m = map_index(j, g.n_in, g.boundary);
        if (m < 0) continue;
        const double x = double((2 * j + 1) * g.n_out - N0) / D;
        w[m - start] += kernel_eval(g.kernel, g.param, g.R, x) / sum;
    }
    if (A.work_is_double) {
        double *ww = static_cast<double *>(T.wwork) + i * te;
        for (int k = 0; k < te; ++k) ww[k] = w[k];
        return;
    }
    // Round to FP32, then put the rounding residual back on the largest tap.
    float *ww = static_cast<float *>(T.wwork) + i * te;
    double s = 0.0, big = -1.0;
    int kbig = 0;
    for (int k = 0; k < te; ++k) {
        const float f = __double2float_rn(w[k]);
        ww[k] = f;
        s += double(f);
        if (fabs(w[k]) > big) {
            big = fabs(w[k]);
            kbig = k;
        }
    }
    ww[kbig] = __double2float_rn(double(ww[kbig]) + (1.0 - s));
}

__global__ void weights_kernel(WeightArgs a0, WeightArgs a1)
{
    const int64_t n0 = a0.g.n_out, n1 = a1.g.n_out;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n0 + n1;
         t += int64_t(gridDim.x) * blockDim.x) {
        if (t < n0)
            axis_weights(a0, t);
        else
            axis_weights(a1, t - n0);
    }
}

template <typename W>
__device__ void axis_band(const WeightArgs &A, int64_t grp)
{
    const AxisGeom &g = A.g;
    const AxisTables &T = A.t;
    const int G = T.G, J = T.J, te = g.t_eff;
    int64_t b0 = g.n_in, hi = 0;
    for (int r = 0; r < G; ++r) {
        const int64_t i = grp * G + r;
        if (i >= g.n_out) break;
        const int64_t s = T.start[i];
        b0 = s < b0 ? s : b0;
        hi = s + te > hi ? s + te : hi;
    }
    int64_t b = g.n_in >= J ? (b0 < g.n_in - J ? b0 : g.n_in - J) : 0;
    if (hi - b > J) flag_error(A.err, kErrBand);
    T.band_base[grp] = int32_t(b);
    const W *ww = static_cast<const W *>(T.wwork);
    W *out = static_cast<W *>(T.band_w) + grp * G * J;
    for (int r = 0; r < G; ++r) {
        const int64_t i = grp * G + r;
        const int64_t off = i < g.n_out ? T.start[i] - b : 0;
        for (int j = 0; j < J; ++j) {
            W v = W(0);
            if (i < g.n_out && j >= off && j < off + te && (hi - b) <= J) v = ww[i * te + (j - off)];
            out[r * J + j] = v;
        }
    }
}

__global__ void band_kernel(WeightArgs a0, WeightArgs a1)
{
    const int64_t n0 = a0.t.groups, n1 = a1.t.groups;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n0 + n1;
         t += int64_t(gridDim.x) * blockDim.x) {
        const WeightArgs &A = t < n0 ? a0 : a1;
        const int64_t grp = t < n0 ? t : t - n0;
        if (A.work_is_double)
            axis_band<double>(A, grp);
        else
            axis_band<float>(A, grp);
    }
}

} // namespace

cudaError_t launch_weights(const WeightArgs &a0, const WeightArgs &a1, cudaStream_t s)
{
    const int64_t n = a0.g.n_out + a1.g.n_out;
    const int threads = 128;
    int blocks = int((n + threads - 1) / threads);
    if (blocks > 4096) blocks = 4096;
    weights_kernel<<<blocks, threads, 0, s>>>(a0, a1);
    return cudaGetLastError();
}

cudaError_t launch_band(const WeightArgs &a0, const WeightArgs &a1, cudaStream_t s)
{
    const int64_t n = int64_t(a0.t.groups) + a1.t.groups;
    const int threads = 128;
    int blocks = int((n + threads - 1) / threads);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    band_kernel<<<blocks, threads, 0, s>>>(a0, a1);
    return cudaGetLastError();
}

} // namespace rs
