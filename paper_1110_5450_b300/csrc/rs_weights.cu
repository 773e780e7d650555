// rs_weights.cu -- FP64 weight-table kernel and register-band builder.
//
// Blocks of consecutive output samples of an axis.  Tap indices come from a closed
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
        return (sinpi(x) * sinpi(xr)) / ((kPi * x) * (kPi * xr));
    }
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

// Shared-memory budget of one block: per output its tap range, per raw tap
// its mapped index and kernel value.
constexpr int kThreadsW = 256;
constexpr int kFlat = 2048; // raw taps staged per block

// One block computes the tables of outputs [o0, o0 + nb) of one axis in
// phases: (A) a thread per output finds its taps with the exact integer
// formula, (B) a thread per (output, tap) evaluates the kernel in FP64 and the
// boundary map, (C1) a thread per output sums its taps in index order,
// (C2) a thread per (output, window slot) normalises and folds mapped
// duplicates into the stored window and rounds to the working precision,
// (C3) a thread per output puts the rounding residual back.
__device__ void axis_block(const WeightArgs &A, int64_t o0, int nb, int64_t *jlo_s, int *cnt_s, int64_t *slot_s,
                           double *val_s, double *sum_s, int64_t *start_s)
{
    const AxisGeom &g = A.g;
    const AxisTables &T = A.t;
    const int tr = g.t_raw, te = g.t_eff;
    const int64_t two_out = 2 * g.n_out;
    const int64_t RD = g.R * g.D;
    // (A) tap ranges
    for (int o = threadIdx.x; o < nb; o += blockDim.x) {
        const int64_t i = o0 + o;
        const int64_t N0 = (2 * i + 1) * g.n_in;
        // first raw tap: smallest j with (2j+1) n_out > N0 - R D
        const int64_t jlo = floor_div(N0 - RD - g.n_out, two_out) + 1;
        // last raw tap: largest j with (2j+1) n_out < N0 + R D
        const int64_t jhi = ceil_div(N0 + RD - g.n_out, two_out) - 1;
        int64_t cnt = jhi - jlo + 1;
        T.jlo[i] = int32_t(jlo);
        T.cnt[i] = int32_t(cnt);
        if (cnt < 1 || cnt > tr) {
            flag_error(A.err, kErrTaps);
            cnt = 0;
        }
        jlo_s[o] = jlo;
        cnt_s[o] = int(cnt);
    }
    __syncthreads();
    // (B) kernel values and mapped indices, all lanes busy
    const double D = double(g.D);
    for (int e = threadIdx.x; e < nb * tr; e += blockDim.x) {
        const int o = e / tr, k = e - o * tr;
        int64_t m = -1;
        double v = 0.0;
        if (k < cnt_s[o]) {
            const int64_t i = o0 + o;
            const int64_t j = jlo_s[o] + k;
            m = map_index(j, g.n_in, g.boundary);
            if (m >= 0) {
                const double x = double((2 * j + 1) * g.n_out - (2 * i + 1) * g.n_in) / D;
                v = kernel_eval(g.kernel, g.param, g.R, x);
            }
        }
        slot_s[e] = m;
        val_s[e] = v;
    }
    __syncthreads();
    // (C1) a thread per output: tap sum in index order, mapped range, window start
    for (int o = threadIdx.x; o < nb; o += blockDim.x) {
        const int64_t i = o0 + o;
        const int cnt = cnt_s[o];
        const int64_t *sl = slot_s + o * tr;
        const double *vl = val_s + o * tr;
        double sum = 0.0;
        int64_t mlo = g.n_in, mhi = -1;
        for (int k = 0; k < cnt; ++k) {
            sum += vl[k];
            if (sl[k] >= 0) {
                mlo = sl[k] < mlo ? sl[k] : mlo;
                mhi = sl[k] > mhi ? sl[k] : mhi;
            }
        }
        int64_t start = mlo < g.n_in - te ? mlo : g.n_in - te;
        if (start < 0) start = 0;
        T.start[i] = int32_t(start);
        const bool ok = cnt != 0 && sum != 0.0 && mhi >= 0 && mhi - start < te;
        if (cnt != 0 && !ok) flag_error(A.err, kErrSum);
        sum_s[o] = ok ? sum : 0.0;
        start_s[o] = start;
    }
    __syncthreads();
    // (C2) a thread per (output, window slot): normalise and fold, all lanes busy
    for (int e = threadIdx.x; e < nb * te; e += blockDim.x) {
        const int o = e / te, q = e - o * te;
        const int64_t i = o0 + o;
        const double sum = sum_s[o];
        double acc = 0.0;
        if (sum != 0.0) {
            const int cnt = cnt_s[o];
            const int64_t *sl = slot_s + o * tr;
            const double *vl = val_s + o * tr;
            const int64_t jlo = jlo_s[o], start = start_s[o];
            if (jlo >= 0 && jlo + cnt <= g.n_in) { // every tap maps to itself
                const int64_t k = start + q - jlo;
                if (k >= 0 && k < cnt) acc = vl[k] / sum;
            } else {
                for (int k = 0; k < cnt; ++k)
                    if (sl[k] == start + q) acc += vl[k] / sum;
            }
        }
        T.w64[i * te + q] = acc;
        if (A.work_is_double)
            static_cast<double *>(T.wwork)[i * te + q] = acc;
        else
            static_cast<float *>(T.wwork)[i * te + q] = __double2float_rn(acc);
    }
    if (A.work_is_double) return;
    __syncthreads();
    // (C3) a thread per output: put the FP32 rounding residual back on the
    // largest tap (first index on ties) and re-round it
    for (int o = threadIdx.x; o < nb; o += blockDim.x) {
        const int64_t i = o0 + o;
        const double *w = T.w64 + i * te;
        float *ww = static_cast<float *>(T.wwork) + i * te;
        double s32 = 0.0, big = -1.0;
        int kbig = 0;
        for (int q = 0; q < te; ++q) {
            s32 += double(ww[q]);
            if (fabs(w[q]) > big) {
                big = fabs(w[q]);
                kbig = q;
            }
        }
        ww[kbig] = __double2float_rn(double(ww[kbig]) + (1.0 - s32));
    }
}

__global__ void __launch_bounds__(kThreadsW) weights_kernel(WeightArgs a0, WeightArgs a1, int nb0, int nb1,
                                                            int blocks0)
{
    __shared__ int64_t jlo_s[kThreadsW];
    __shared__ int cnt_s[kThreadsW];
    __shared__ int64_t slot_s[kFlat];
    __shared__ double val_s[kFlat];
    __shared__ double sum_s[kThreadsW];
    __shared__ int64_t start_s[kThreadsW];
    const bool first = int(blockIdx.x) < blocks0;
    const WeightArgs &A = first ? a0 : a1;
    const int nb_full = first ? nb0 : nb1;
    const int64_t o0 = int64_t(first ? blockIdx.x : blockIdx.x - blocks0) * nb_full;
    const int64_t rem = A.g.n_out - o0;
    const int nb = int(rem < nb_full ? rem : nb_full);
    if (nb > 0) axis_block(A, o0, nb, jlo_s, cnt_s, slot_s, val_s, sum_s, start_s);
}

// Base of band group grp (the smallest window start of its members, kept
// inside the axis) and whether the members' windows fit J inputs from it.
__device__ int64_t band_group_base(const WeightArgs &A, int64_t grp, bool *fits)
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
    const int64_t b = T.align > 1 ? b0 - b0 % T.align : (g.n_in >= J ? (b0 < g.n_in - J ? b0 : g.n_in - J) : 0);
    *fits = (hi - b) <= J;
    return b;
}

// Weight of member r of group grp at band input j (0 outside its window).
template <typename W>
__device__ W band_weight(const WeightArgs &A, int64_t grp, int64_t b, bool fits, int j, int r)
{
    const AxisGeom &g = A.g;
    const AxisTables &T = A.t;
    const int64_t i = grp * T.G + r;
    if (j >= T.J || i >= g.n_out || !fits) return W(0);
    const int64_t off = T.start[i] - b;
    if (j >= off && j < off + g.t_eff) return static_cast<const W *>(T.wwork)[i * g.t_eff + (j - off)];
    return W(0);
}

// Band element e of slot `slot` of one axis (layouts in rs_internal.h):
// band_w[slot * JS + (j * G + r) * dup + d] with d a duplicate, or with
// pairing band_w[slot * JS + (j * G + r) * 2 + d] with d the group of the pair.
template <typename W>
__device__ void band_element(const WeightArgs &A, int64_t slot, int e)
{
    const AxisTables &T = A.t;
    const int G = T.G, JS = band_slot_stride(T);
    int64_t grp;
    int idx;
    bool real = true;
    if (T.pair_ngx > 0) {
        const int ppt = (T.pair_ngx + 1) / 2;
        const int64_t tile = slot / ppt;
        const int pq = int(slot % ppt), d = e & 1;
        const int local = 2 * pq + d;
        grp = tile * T.pair_ngx + local;
        real = local < T.pair_ngx && grp < T.groups;
        idx = e >> 1;
        if (real && e == d) {
            bool fits;
            const int64_t b = band_group_base(A, grp, &fits);
            T.band_base[grp] = int32_t(b);
            if (!fits) flag_error(A.err, kErrBand);
        }
    } else {
        grp = slot;
        idx = e / T.dup;
        if (e == 0) {
            bool fits;
            const int64_t b = band_group_base(A, grp, &fits);
            T.band_base[grp] = int32_t(b);
            if (!fits) flag_error(A.err, kErrBand);
        }
    }
    W v = W(0);
    if (real) {
        bool fits;
        const int64_t b = band_group_base(A, grp, &fits);
        v = band_weight<W>(A, grp, b, fits, idx / G, idx % G);
    }
    static_cast<W *>(T.band_w)[slot * JS + e] = v;
}

__global__ void band_kernel(WeightArgs a0, WeightArgs a1)
{
    const int64_t js0 = band_slot_stride(a0.t), js1 = band_slot_stride(a1.t);
    const int64_t n0 = band_slots(a0.t) * js0, n1 = band_slots(a1.t) * js1;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n0 + n1;
         t += int64_t(gridDim.x) * blockDim.x) {
        const bool first = t < n0;
        const WeightArgs &A = first ? a0 : a1;
        const int64_t u = first ? t : t - n0;
        const int64_t js = first ? js0 : js1;
        if (A.work_is_double)
            band_element<double>(A, u / js, int(u % js));
        else
            band_element<float>(A, u / js, int(u % js));
    }
}

} // namespace

// Outputs per block: enough blocks to cover the GPU twice, at most kThreadsW
// outputs and kFlat staged taps.
static int outputs_per_block(const AxisGeom &g, int64_t total_outputs)
{
    int64_t nb = (total_outputs + 295) / 296;
    nb = nb < 1 ? 1 : nb;
    nb = nb > kThreadsW ? kThreadsW : nb;
    const int64_t cap = kFlat / (g.t_raw > 0 ? g.t_raw : 1);
    nb = nb > cap ? cap : nb;
    return int(nb < 1 ? 1 : nb);
}

cudaError_t launch_weights(const WeightArgs &a0, const WeightArgs &a1, cudaStream_t s)
{
    const int64_t total = a0.g.n_out + a1.g.n_out;
    const int nb0 = outputs_per_block(a0.g, total), nb1 = outputs_per_block(a1.g, total);
    const int64_t b0 = (a0.g.n_out + nb0 - 1) / nb0, b1 = (a1.g.n_out + nb1 - 1) / nb1;
    weights_kernel<<<int(b0 + b1), kThreadsW, 0, s>>>(a0, a1, nb0, nb1, int(b0));
    return cudaGetLastError();
}

cudaError_t launch_band(const WeightArgs &a0, const WeightArgs &a1, cudaStream_t s)
{
    const int64_t n = band_slots(a0.t) * band_slot_stride(a0.t) + band_slots(a1.t) * band_slot_stride(a1.t);
    const int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    if (blocks > 148 * 16) blocks = 148 * 16;
    if (blocks < 1) blocks = 1;
    band_kernel<<<int(blocks), threads, 0, s>>>(a0, a1);
    return cudaGetLastError();
}

} // namespace rs
