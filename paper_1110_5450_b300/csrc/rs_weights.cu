// rs_weights.cu -- FP64 weight-table kernel and register-band builder.
//
// A block per SM owns a run of outputs of an axis and their mirror outputs.
// Tap indices come from a closed form in 64-bit integers (exact), weights
// from the kernel evaluated in FP64 at x = N / D with the exact integer
// numerator N = (2j+1) n_out - (2i+1) n_in (Lanczos: both sine arguments
// reduced exactly in integers first), normalised by their FP64 sum, folded
// through the boundary map into a window of t_eff consecutive in-range
// inputs, then rounded to the working precision with the rounding residual
// put back on the largest tap.
//
// Kernel definitions (standard): tent; Keys cubic convolution (R. Keys, IEEE
// Trans. ASSP 29(6), 1981); Lanczos windowed sinc (C. Duchon, J. Appl.
// Meteor. 18, 1979); cubic B-spline (M. Unser, IEEE SP Mag. 16(6), 1999);
// Mitchell-Netravali cubic (D. Mitchell, A. Netravali, SIGGRAPH 1988);
// Gaussian.
#include "rs_internal.h"

namespace rs {
namespace {

enum : int { kErrTaps = 101, kErrSum = 102, kErrBand = 103 };

__device__ __forceinline__ void flag_error(int *err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

// Division by an invariant positive d through its reciprocal
// m = floor((2^64 - 1) / d), computed on the host (T. Granlund and
// P. Montgomery, "Division by invariant integers using multiplication", PLDI
// 1994): for n < 2^63, mulhi(n, m) is the quotient or one less, and the
// remainder tells which.  Exact, and a few integer instructions instead of
// the emulated 64-bit division.
struct Divisor {
    uint64_t d = 1, m = ~uint64_t(0);
};
__device__ __forceinline__ uint64_t udiv(uint64_t n, const Divisor &v)
{
    uint64_t q = __umul64hi(n, v.m);
    if (n - q * v.d >= v.d) ++q;
    return q;
}
// floor(a / d) and ceil(a / d), |a| < 2^62.
__device__ __forceinline__ int64_t floor_div(int64_t a, const Divisor &v)
{
    return a >= 0 ? int64_t(udiv(uint64_t(a), v)) : -int64_t(udiv(uint64_t(-a) + v.d - 1, v));
}
__device__ __forceinline__ int64_t ceil_div(int64_t a, const Divisor &v) { return -floor_div(-a, v); }

// An FP64 operation has a dependency latency of a few hundred cycles on this
// part (its FP64 pipe runs at 1/64 of the FP32 rate), so the table kernel is
// bound by the depth of its FP64 dependency chains; the helpers below keep
// them short.

// 1 / a from the FP32 reciprocal refined by two Newton-Raphson steps
// y <- y + y (1 - a y) (each squares the relative error: 2^-23 -> 2^-46 ->
// below FP64 rounding); within about one ulp.  |a| inside the FP32 range.
__device__ __forceinline__ double rcp64(double a)
{
    double y = double(__frcp_rn(__double2float_rn(a)));
    y = fma(y, fma(-a, y, 1.0), y);
    return fma(y, fma(-a, y, 1.0), y);
}

// sin(pi r) for |r| <= 1/2 as r P(r^2), P with the Taylor coefficients
// (-1)^k pi^(2k+1) / (2k+1)! of sin(pi r) / r up to k = 11 (truncation error
// below 1e-20 at |r| = 1/2): the tail k >= 2 by Estrin's scheme (short
// dependency chain), the two leading terms by Horner steps (accuracy).
// Relative error about 2.5 ulp.
__device__ __forceinline__ double sinpi_reduced(double r)
{
    constexpr double c0 = 0x1.921fb54442d18p+1, c1 = -0x1.4abbce625be53p+2, c2 = 0x1.466bc6775aae2p+1,
                     c3 = -0x1.32d2cce62bd86p-1, c4 = 0x1.50783487ee782p-4, c5 = -0x1.e3074fde8871fp-8,
                     c6 = 0x1.e8f434d018d63p-12, c7 = -0x1.6fadb9f155744p-16, c8 = 0x1.aaec32af93359p-21,
                     c9 = -0x1.8a404211f9547p-26, c10 = 0x1.2877020d52cf0p-31, c11 = -0x1.7215f879e1ac9p-37;
    const double z = r * r, z2 = z * z, z4 = z2 * z2, z8 = z4 * z4;
    const double p0 = fma(c3, z, c2), p1 = fma(c5, z, c4), p2 = fma(c7, z, c6), p3 = fma(c9, z, c8),
                 p4 = fma(c11, z, c10);
    const double t = fma(p4, z8, fma(fma(p3, z2, p2), z4, fma(p1, z2, p0)));
    return r * fma(z, fma(z, t, c1), c0);
}

// Host-computed constants of one axis: the divisors of the tap formula (2 n_out)
// and of the Lanczos argument reductions (2 D, 2 R D), and 1 / D, 1 / (R D),
// R D^2 / pi^2 (an FP64 division would lengthen the chains).
struct AxisConst {
    Divisor two_out, two_D, two_RD;
    double inv_D = 0.0, inv_RD = 0.0, lanczos_scale = 0.0;
};

// Lanczos-R at x = N / D from the exact integer numerator N, |N| < R D, N != 0:
// sin(pi x) = (-1)^m sin(pi r) with m the integer nearest N / D and
// r = (N - m D) / D (an exact integer over D: no loss near the zeros), the
// same for x / R with R D, and sinc(x) sinc(x / R) = sin(pi x) sin(pi x / R)
// R D^2 / (pi^2 N^2).
__device__ __forceinline__ double lanczos_value(int64_t N, int64_t D, int64_t RD, const AxisConst &K)
{
    const int64_t m1 = floor_div(2 * N + D, K.two_D), m2 = floor_div(2 * N + RD, K.two_RD);
    const double s1 = sinpi_reduced(double(N - m1 * D) * K.inv_D);
    const double s2 = sinpi_reduced(double(N - m2 * RD) * K.inv_RD);
    const double v = (s1 * s2) * (K.lanczos_scale * rcp64(double(N * N)));
    return ((m1 + m2) & 1) ? -v : v;
}

// Kernel value at x (Lanczos: lanczos_value).
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
    case RS_K_BSPLINE3:
        if (t < 1.0) return (0.5 * t - 1.0) * t * t + 2.0 / 3.0;
        if (t < 2.0) {
            const double u = 2.0 - t;
            return u * u * u / 6.0;
        }
        return 0.0;
    case RS_K_MITCHELL: {
        // Mitchell-Netravali cubic on the B + 2C = 1 line (B = a), Horner form
        const double B = a, Cm = 0.5 * (1.0 - B);
        if (t < 1.0) return (((12.0 - 9.0 * B - 6.0 * Cm) * t + (-18.0 + 12.0 * B + 6.0 * Cm)) * t * t + (6.0 - 2.0 * B)) / 6.0;
        if (t < 2.0)
            return (((-B - 6.0 * Cm) * t + (6.0 * B + 30.0 * Cm)) * t + (-12.0 * B - 48.0 * Cm)) * t / 6.0 +
                   (8.0 * B + 24.0 * Cm) / 6.0;
        return 0.0;
    }
    case RS_K_GAUSSIAN:
        // a = sigma, truncated at the integer support R = ceil(3 sigma)
        if (t >= double(R)) return 0.0;
        return exp(-0.5 * (x / a) * (x / a));
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
        // one reflection covers a support shorter than the axis
        if (j >= -n && j < 2 * n) return j < 0 ? -1 - j : 2 * n - 1 - j;
        const int64_t p = 2 * n;
        int64_t m = j % p;
        if (m < 0) m += p;
        return m < n ? m : p - 1 - m;
    }
    case RS_B_REFLECT101: {
        if (n == 1) return 0;
        if (j > -n && j < 2 * n - 1) return j < 0 ? -j : 2 * n - 2 - j;
        const int64_t p = 2 * n - 2;
        int64_t m = j % p;
        if (m < 0) m += p;
        return m < n ? m : p - m;
    }
    default:
        return -1;
    }
}

// Shared-memory budget of one block: per logical output its tap range,
// window start and normalisation, per primary raw tap its kernel value, per
// logical output and window slot its folded weight.
constexpr int kThreadsW = 256;
constexpr int kMaxPrim = kThreadsW / 2; // primary outputs per block
constexpr int kFlat = 2048;             // raw kernel values / folded weights staged per block

// The kernel argument of output n_out-1-i at tap n_in-1-j is minus that of
// output i at tap j (the numerator changes sign), so with a symmetric kernel
// the mirror output has the raw values of its primary in reverse order: a
// block evaluates the kernel for primaries i < ceil(n_out / 2) only.  Logical
// slot l of a block with primaries [p0, p0 + np) is primary p0 + l for
// l < np, else the mirror of primary p0 + l - np (-1 for the middle output of
// an odd axis, its own mirror).
__device__ __forceinline__ int64_t logical_output(const AxisGeom &g, int64_t p0, int np, int l)
{
    if (l < np) return p0 + l;
    const int64_t i = p0 + (l - np);
    const int64_t m = g.n_out - 1 - i;
    return m == i ? -1 : m;
}

struct BlockSmem {
    int64_t jlo[2 * kMaxPrim];
    int64_t start[2 * kMaxPrim];
    double inv[2 * kMaxPrim];
    int cnt[2 * kMaxPrim];
    double val[kFlat];  // [np][t_raw] kernel values of the primaries
    double acc[kFlat];  // [2 np][t_eff] folded normalised weights
    float acc32[kFlat]; // the same rounded to FP32, residual included
};

// One block computes the tables of its logical outputs in phases, all
// intermediate results in shared memory: (A) a thread per output finds its
// taps with the exact integer formula, (B) a thread per (primary, tap)
// evaluates the kernel in FP64 at x = numerator / D, (C1) a thread per
// output sums its in-range taps and takes the reciprocal of the sum, (C2) a
// thread per (output, window slot) normalises and folds mapped duplicates
// into the window, (C3) a thread per output rounds its window to FP32 with
// the rounding residual put back on the largest tap, (D) a thread per
// (output, window slot) stores the tables.
__device__ void axis_block(const WeightArgs &A, const AxisConst &K, int64_t p0, int np, BlockSmem &sm)
{
    const AxisGeom &g = A.g;
    const AxisTables &T = A.t;
    const int tr = g.t_raw, te = g.t_eff, nl = 2 * np;
    const int64_t RD = g.R * g.D;
    // (A) tap ranges
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
        const int64_t i = logical_output(g, p0, np, l);
        int64_t jlo = 0, cnt = 0;
        if (i >= 0) {
            const int64_t N0 = (2 * i + 1) * g.n_in;
            // first raw tap: smallest j with (2j+1) n_out > N0 - R D
            jlo = floor_div(N0 - RD - g.n_out, K.two_out) + 1;
            // last raw tap: largest j with (2j+1) n_out < N0 + R D
            const int64_t jhi = ceil_div(N0 + RD - g.n_out, K.two_out) - 1;
            cnt = jhi - jlo + 1;
            T.jlo[i] = int32_t(jlo);
            T.cnt[i] = int32_t(cnt);
            if (cnt < 1 || cnt > tr) {
                flag_error(A.err, kErrTaps);
                cnt = 0;
            }
        }
        sm.jlo[l] = jlo;
        sm.cnt[l] = int(cnt);
    }
    __syncthreads();
    // (B) kernel values of the primaries, all lanes busy
    for (int e = threadIdx.x; e < np * tr; e += blockDim.x) {
        const int q = e / tr, k = e - q * tr;
        double v = 0.0;
        if (k < sm.cnt[q]) {
            const int64_t j = sm.jlo[q] + k;
            const int64_t N = (2 * j + 1) * g.n_out - (2 * (p0 + q) + 1) * g.n_in;
            if (g.kernel == RS_K_LANCZOS)
                v = N == 0 ? 1.0 : (N >= RD || N <= -RD) ? 0.0 : lanczos_value(N, g.D, RD, K);
            else
                v = kernel_eval(g.kernel, g.param, g.R, double(N) * K.inv_D);
        }
        sm.val[e] = v;
    }
    __syncthreads();
    // (C1) a thread per output: sum of the in-range taps, mapped range,
    // window start
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
        const int64_t i = logical_output(g, p0, np, l);
        const int cnt = sm.cnt[l];
        double inv = 0.0;
        int64_t start = 0;
        if (i >= 0 && cnt > 0) {
            const bool rev = l >= np;
            const int q = rev ? l - np : l;
            if (rev && (cnt != sm.cnt[q] || sm.jlo[l] != g.n_in - sm.jlo[q] - cnt)) flag_error(A.err, kErrTaps);
            const double *vl = sm.val + q * tr;
            const int64_t jlo = sm.jlo[l];
            // eight partial sums (taps k mod 8) shorten the FP64 dependency chain
            double part[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            int64_t mlo = g.n_in, mhi = -1;
            for (int k0 = 0; k0 < cnt; k0 += 8)
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = k0 + u;
                    if (k >= cnt) break;
                    const int64_t m = map_index(jlo + k, g.n_in, g.boundary);
                    if (m < 0) continue;
                    part[u] += vl[rev ? cnt - 1 - k : k];
                    mlo = m < mlo ? m : mlo;
                    mhi = m > mhi ? m : mhi;
                }
            const double sum = ((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7]));
            start = mlo < g.n_in - te ? mlo : g.n_in - te;
            if (start < 0) start = 0;
            const bool ok = sum != 0.0 && mhi >= 0 && mhi - start < te;
            if (!ok) flag_error(A.err, kErrSum);
            inv = ok ? rcp64(sum) : 0.0;
        }
        sm.inv[l] = inv;
        sm.start[l] = start;
    }
    __syncthreads();
    // (C2) a thread per (output, window slot): normalise and fold, all lanes busy
    for (int e = threadIdx.x; e < nl * te; e += blockDim.x) {
        const int l = e / te, s = e - l * te;
        const double inv = sm.inv[l];
        double acc = 0.0;
        if (inv != 0.0) {
            const int cnt = sm.cnt[l];
            const bool rev = l >= np;
            const double *vl = sm.val + (rev ? l - np : l) * tr;
            const int64_t jlo = sm.jlo[l], start = sm.start[l];
            if (jlo >= 0 && jlo + cnt <= g.n_in) { // every tap maps to itself
                const int64_t k = start + s - jlo;
                if (k >= 0 && k < cnt) acc = vl[rev ? cnt - 1 - k : k] * inv;
            } else {
                for (int k = 0; k < cnt; ++k)
                    if (map_index(jlo + k, g.n_in, g.boundary) == start + s) acc += vl[rev ? cnt - 1 - k : k] * inv;
            }
        }
        sm.acc[e] = acc;
        sm.acc32[e] = __double2float_rn(acc);
    }
    __syncthreads();
    // (C3) a thread per output: put the FP32 rounding residual back on the
    // largest tap (first index on ties) and re-round it
    if (!A.work_is_double) {
        for (int l = threadIdx.x; l < nl; l += blockDim.x) {
            const double *w = sm.acc + l * te;
            float *ww = sm.acc32 + l * te;
            // the sum of the FP32 weights as an unevaluated pair hi + lo of
            // FP32 numbers, accumulated with Knuth's TwoSum (error-free FP32
            // additions: short latency); the largest |w| compared as the
            // integer bit patterns of non-negative doubles (same order)
            float hi = 0.f, lo = 0.f;
            int64_t big = -1;
            int kbig = 0;
            for (int q = 0; q < te; ++q) {
                const float a = ww[q], s = __fadd_rn(hi, a), bb = __fsub_rn(s, hi);
                lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(a, bb)));
                hi = s;
                const int64_t mag = __double_as_longlong(w[q]) & 0x7fffffffffffffffll;
                if (mag > big) {
                    big = mag;
                    kbig = q;
                }
            }
            // residual 1 - (hi + lo); 1 - hi is exact (hi near 1)
            ww[kbig] = __double2float_rn(double(ww[kbig]) + (double(1.f - hi) - double(lo)));
        }
        __syncthreads();
    }
    // (D) store the tables
    for (int e = threadIdx.x; e < nl * te; e += blockDim.x) {
        const int l = e / te, s = e - l * te;
        const int64_t i = logical_output(g, p0, np, l);
        if (i < 0) continue;
        if (s == 0) T.start[i] = int32_t(sm.start[l]);
        T.w64[i * te + s] = sm.acc[e];
        if (A.work_is_double)
            static_cast<double *>(T.wwork)[i * te + s] = sm.acc[e];
        else
            static_cast<float *>(T.wwork)[i * te + s] = sm.acc32[e];
    }
}

__global__ void __launch_bounds__(kThreadsW) weights_kernel(WeightArgs a0, WeightArgs a1, AxisConst k0,
                                                            AxisConst k1, int np0, int np1, int blocks0)
{
    __shared__ BlockSmem sm;
    const bool first = int(blockIdx.x) < blocks0;
    const WeightArgs &A = first ? a0 : a1;
    const int np_full = first ? np0 : np1;
    const int64_t p0 = int64_t(first ? blockIdx.x : blockIdx.x - blocks0) * np_full;
    const int64_t rem = (A.g.n_out + 1) / 2 - p0;
    const int np = int(rem < np_full ? rem : np_full);
    if (np > 0) axis_block(A, first ? k0 : k1, p0, np, sm);
}

// Band tables.  A block takes kBandSlots consecutive slots of one axis: its
// threads stage the window starts of the slots' group members in shared
// memory, one thread per group derives the group's base (the smallest start,
// kept inside the axis or rounded down to a multiple of align) and checks
// that the members' windows fit J inputs from it, then a thread per band
// entry gathers its weight.  Layouts (rs_internal.h): band_w[slot * JS +
// (j * G + r) * dup + d] with d a duplicate, or with pairing
// band_w[slot * JS + (j * G + r) * 2 + d] with d the group of the pair;
// entries past J * G * width are zero padding.
constexpr int kBandSlots = 4;
constexpr int kMaxG = 8; // largest band group the builders use
constexpr int kThreadsB = 256;

struct BandSmem {
    int32_t st[kBandSlots * 2 * kMaxG]; // member starts, [slot][d][r]
    int64_t grp[kBandSlots * 2];        // group of (slot, d); -1: none
    int32_t base[kBandSlots * 2];
    int32_t fits[kBandSlots * 2];
};

template <typename W> __device__ void band_block(const WeightArgs &A, int64_t s0, int ns, BandSmem &sm)
{
    const AxisGeom &g = A.g;
    const AxisTables &T = A.t;
    const int G = T.G, J = T.J, te = g.t_eff, JS = band_slot_stride(T);
    const bool pair = T.pair_ngx > 0;
    const int width = pair ? 2 : T.dup; // entries per (j, r)
    if (G > kMaxG) {
        if (threadIdx.x == 0) flag_error(A.err, kErrBand);
        return;
    }
    // groups of the block's slots
    for (int u = threadIdx.x; u < 2 * ns; u += blockDim.x) {
        const int64_t slot = s0 + (u >> 1);
        const int d = u & 1;
        int64_t grp = -1;
        if (pair) {
            const int ppt = (T.pair_ngx + 1) / 2;
            const int64_t tile = slot / ppt;
            const int local = 2 * int(slot - tile * ppt) + d;
            if (local < T.pair_ngx && tile * T.pair_ngx + local < T.groups) grp = tile * T.pair_ngx + local;
        } else if (d == 0) {
            grp = slot;
        }
        sm.grp[u] = grp;
    }
    __syncthreads();
    // member starts (n_in marks a member past the axis)
    for (int u = threadIdx.x; u < 2 * ns * G; u += blockDim.x) {
        const int gi = u / G, r = u - gi * G;
        const int64_t grp = sm.grp[gi], i = grp * G + r;
        sm.st[gi * kMaxG + r] = (grp >= 0 && i < g.n_out) ? T.start[i] : int32_t(g.n_in);
    }
    __syncthreads();
    for (int u = threadIdx.x; u < 2 * ns; u += blockDim.x) {
        const int64_t grp = sm.grp[u];
        if (grp < 0) continue;
        int64_t b0 = g.n_in, hi = 0;
        for (int r = 0; r < G; ++r) {
            const int64_t st = sm.st[u * kMaxG + r];
            if (st >= g.n_in) break;
            b0 = st < b0 ? st : b0;
            hi = st + te > hi ? st + te : hi;
        }
        const int64_t b = T.align > 1 ? b0 - b0 % T.align : (g.n_in >= J ? (b0 < g.n_in - J ? b0 : g.n_in - J) : 0);
        const bool fits = (hi - b) <= J;
        sm.base[u] = int32_t(b);
        sm.fits[u] = fits;
        T.band_base[grp] = int32_t(b);
        if (!fits) flag_error(A.err, kErrBand);
    }
    __syncthreads();
    // band entries
    const W *wwork = static_cast<const W *>(T.wwork);
    W *band = static_cast<W *>(T.band_w);
    const int real = J * G * width;
#pragma unroll 4
    for (int e = threadIdx.x; e < ns * JS; e += blockDim.x) {
        const int sl = e / JS, f = e - sl * JS;
        W v = W(0);
        if (f < real) {
            const int d = pair ? (f & 1) : 0;
            const int idx = f / width, j = idx / G, r = idx - j * G;
            const int u = 2 * sl + d;
            const int64_t grp = sm.grp[u];
            if (grp >= 0 && sm.fits[u]) {
                const int32_t st = sm.st[u * kMaxG + r];
                const int off = st - sm.base[u];
                if (st < g.n_in && j >= off && j < off + te) v = wwork[(grp * G + r) * te + (j - off)];
            }
        }
        band[(s0 + sl) * JS + f] = v;
    }
}

__global__ void __launch_bounds__(kThreadsB) band_kernel(WeightArgs a0, WeightArgs a1, int blocks0)
{
    __shared__ BandSmem sm;
    const bool first = int(blockIdx.x) < blocks0;
    const WeightArgs &A = first ? a0 : a1;
    const int64_t s0 = int64_t(first ? blockIdx.x : blockIdx.x - blocks0) * kBandSlots;
    const int64_t rem = band_slots(A.t) - s0;
    const int ns = int(rem < kBandSlots ? rem : kBandSlots);
    if (ns <= 0 || A.t.J <= 0) return;
    if (A.work_is_double)
        band_block<double>(A, s0, ns, sm);
    else
        band_block<float>(A, s0, ns, sm);
}

} // namespace

// Primary outputs per block: the primaries of both axes spread over one
// block per SM, at most kMaxPrim of them, kFlat staged kernel values and
// kFlat folded weights (2 np t_eff).
static int primaries_per_block(const AxisGeom &g, int64_t total_primaries)
{
    int64_t np = (total_primaries + 147) / 148;
    np = np < 1 ? 1 : np;
    np = np > kMaxPrim ? kMaxPrim : np;
    const int64_t cap_raw = kFlat / (g.t_raw > 0 ? g.t_raw : 1);
    const int64_t cap_eff = kFlat / (2 * (g.t_eff > 0 ? g.t_eff : 1));
    np = np > cap_raw ? cap_raw : np;
    np = np > cap_eff ? cap_eff : np;
    return int(np < 1 ? 1 : np);
}

static Divisor divisor(int64_t d)
{
    Divisor v;
    v.d = uint64_t(d > 0 ? d : 1);
    v.m = ~uint64_t(0) / v.d;
    return v;
}

static AxisConst axis_const(const AxisGeom &g)
{
    constexpr double kPi2 = 9.869604401089358618834490999876151135; // pi^2
    AxisConst k;
    k.two_out = divisor(2 * g.n_out);
    k.two_D = divisor(2 * g.D);
    k.two_RD = divisor(2 * g.R * g.D);
    k.inv_D = g.D > 0 ? 1.0 / double(g.D) : 0.0;
    k.inv_RD = g.R * g.D > 0 ? 1.0 / double(g.R * g.D) : 0.0;
    k.lanczos_scale = double(g.R) * double(g.D) * double(g.D) / kPi2;
    return k;
}

void preload_weights()
{
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, weights_kernel) != cudaSuccess) cudaGetLastError();
    if (cudaFuncGetAttributes(&a, band_kernel) != cudaSuccess) cudaGetLastError();
}

cudaError_t launch_weights(const WeightArgs &a0, const WeightArgs &a1, cudaStream_t s)
{
    const int64_t h0 = (a0.g.n_out + 1) / 2, h1 = (a1.g.n_out + 1) / 2;
    const int np0 = primaries_per_block(a0.g, h0 + h1), np1 = primaries_per_block(a1.g, h0 + h1);
    const int64_t b0 = (h0 + np0 - 1) / np0, b1 = (h1 + np1 - 1) / np1;
    weights_kernel<<<int(b0 + b1), kThreadsW, 0, s>>>(a0, a1, axis_const(a0.g), axis_const(a1.g), np0, np1,
                                                       int(b0));
    return cudaGetLastError();
}

cudaError_t launch_band(const WeightArgs &a0, const WeightArgs &a1, cudaStream_t s)
{
    const int64_t b0 = a0.t.J > 0 ? (band_slots(a0.t) + kBandSlots - 1) / kBandSlots : 0;
    const int64_t b1 = a1.t.J > 0 ? (band_slots(a1.t) + kBandSlots - 1) / kBandSlots : 0;
    if (b0 + b1 == 0) return cudaSuccess;
    band_kernel<<<int(b0 + b1), kThreadsB, 0, s>>>(a0, a1, int(b0));
    return cudaGetLastError();
}

} // namespace rs
