// rs_prefilter.cu -- the interpolating cubic B-spline: before resampling with
// the cubic B-spline kernel, the image is replaced by its B-spline
// coefficients c, the solution of
//
//     (c[k-1] + 4 c[k] + c[k+1]) / 6 = s[k],   k = 0 .. n-1,
//
// along each axis, where c beyond the ends follows the plan's boundary rule
// (clamp and mirror: c[-1] = c[0], c[n] = c[n-1]; reflect101: c[-1] = c[1],
// c[n] = c[n-2]), so that the resampled B-spline passes through the samples
// (M. Unser, IEEE Signal Processing Magazine 16(6), 1999).  Each axis is one
// tridiagonal system per line, solved by forward elimination and back
// substitution (Thomas' algorithm; the matrix is diagonally dominant, so it
// is stable without pivoting).  The elimination factors depend only on the
// axis length and boundary, so they are computed once per plan in FP64 on the
// host and kept in the working precision.
//
//   rows:    one thread per (row, channel, segment of the row);
//   columns: one thread per (column, channel, segment of the column)
//            (neighbouring threads touch neighbouring samples: coalesced).
// The coefficients go to a plan-owned buffer with the input's row pitch, and
// the resampling kernels then read that buffer instead of the input.
#include <vector>

#include "rs_plan.h"

namespace rs {
namespace prefilter {
namespace {

constexpr int kThreads = 128;

template <typename A> struct Line {
    const A *inv_w; // [n] 1 / pivot
    const A *g;     // [n] super-diagonal factor after elimination
    const A *l;     // [n] sub-diagonal coefficient
};

// Both recurrences decay: away from the ends the pivots tend to 2 + sqrt(3)
// and the factors g to 2 - sqrt(3) = 0.268, so a step forgets its start
// value by that factor.  A line is therefore cut into segments of kSeg
// samples solved in parallel: each starts its recurrence kWarm samples early
// from zero (forward) or from d' (backward), and 0.268^32 < 1e-18 leaves the
// result unchanged at double precision; the first and last segments start at
// the line's ends exactly.  Forward elimination writes d' to a scratch
// buffer, back substitution reads it (including the next segment's warm-up
// samples) and writes the coefficients.  Loads are issued kChunk steps ahead
// of the arithmetic, so the latency is paid once per chunk.
constexpr int kSeg = 256, kWarm = 32, kChunk = 16;

template <typename T, typename A>
__device__ __forceinline__ void forward_seg(const T *src, A *dp, int64_t k0, int64_t k1, int64_t step,
                                            const Line<A> &L)
{
    A prev = A(0);
    for (int64_t c0 = k0 >= kWarm ? k0 - kWarm : 0; c0 < k1; c0 += kChunk) {
        A s[kChunk], lk[kChunk], iw[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
            const int64_t k = c0 + u;
            s[u] = k < k1 ? A(src[k * step]) : A(0);
            lk[u] = k < k1 ? __ldg(L.l + k) : A(0);
            iw[u] = k < k1 ? __ldg(L.inv_w + k) : A(0);
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
            const int64_t k = c0 + u;
            if (k < k1) {
                prev = (A(6) * s[u] - lk[u] * prev) * iw[u];
                if (k >= k0) dp[k * step] = prev;
            }
        }
    }
}

template <typename A>
__device__ __forceinline__ void backward_seg(const A *dp, A *out, int64_t k0, int64_t k1, int64_t n, int64_t step,
                                             const Line<A> &L)
{
    const int64_t e = k1 + kWarm <= n ? k1 - 1 + kWarm : n - 1; // c[n-1] = d'[n-1] exactly
    A next = dp[e * step];
    if (e < k1) out[e * step] = next;
    for (int64_t c0 = e - 1; c0 >= k0; c0 -= kChunk) {
        A d[kChunk], gk[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
            const int64_t k = c0 - u;
            d[u] = k >= k0 ? dp[k * step] : A(0);
            gk[u] = k >= k0 ? __ldg(L.g + k) : A(0);
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
            const int64_t k = c0 - u;
            if (k >= k0) {
                next = d[u] - gk[u] * next;
                if (k < k1) out[k * step] = next;
            }
        }
    }
}

// rows: x = (row, channel) lines, y = segments along the row
template <typename T, typename A>
__global__ void __launch_bounds__(kThreads) rows_fwd(const T *in, A *dp, int64_t rows, int64_t cols, int C,
                                                     int64_t stride, Line<A> L)
{
    const int64_t t = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (t >= rows * C) return;
    const int64_t r = t / C, c = t - r * C, k0 = int64_t(blockIdx.y) * kSeg;
    forward_seg<T, A>(in + r * stride + c, dp + r * stride + c, k0, min(k0 + kSeg, cols), C, L);
}

template <typename A>
__global__ void __launch_bounds__(kThreads) rows_bwd(const A *dp, A *out, int64_t rows, int64_t cols, int C,
                                                     int64_t stride, Line<A> L)
{
    const int64_t t = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (t >= rows * C) return;
    const int64_t r = t / C, c = t - r * C, k0 = int64_t(blockIdx.y) * kSeg;
    backward_seg<A>(dp + r * stride + c, out + r * stride + c, k0, min(k0 + kSeg, cols), cols, C, L);
}

// columns: x = (column, channel) samples of a row (coalesced), y = segments down
template <typename A>
__global__ void __launch_bounds__(kThreads) cols_fwd(const A *in, A *dp, int64_t rows, int64_t cols, int C,
                                                     int64_t stride, Line<A> L)
{
    const int64_t t = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (t >= cols * C) return;
    const int64_t k0 = int64_t(blockIdx.y) * kSeg;
    forward_seg<A, A>(in + t, dp + t, k0, min(k0 + kSeg, rows), stride, L);
}

template <typename A>
__global__ void __launch_bounds__(kThreads) cols_bwd(const A *dp, A *out, int64_t rows, int64_t cols, int C,
                                                     int64_t stride, Line<A> L)
{
    const int64_t t = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (t >= cols * C) return;
    const int64_t k0 = int64_t(blockIdx.y) * kSeg;
    backward_seg<A>(dp + t, out + t, k0, min(k0 + kSeg, rows), rows, stride, L);
}

// Elimination factors of one axis (FP64 on the host).
void factors(int64_t n, int boundary, std::vector<double> &inv_w, std::vector<double> &g, std::vector<double> &l)
{
    inv_w.assign(n, 0.0);
    g.assign(n, 0.0);
    l.assign(n, 0.0);
    std::vector<double> lo(n, 1.0), di(n, 4.0), up(n, 1.0);
    lo[0] = 0.0;
    up[n - 1] = 0.0;
    if (n == 1) {
        di[0] = 6.0; // both neighbours are the sample itself
    } else if (boundary == RS_B_REFLECT101) {
        up[0] = 2.0;      // c[-1] = c[1]
        lo[n - 1] = 2.0;  // c[n] = c[n-2]
    } else {
        di[0] = 5.0;      // c[-1] = c[0]
        di[n - 1] = 5.0;  // c[n] = c[n-1]
    }
    double gp = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const double w = di[k] - lo[k] * gp;
        inv_w[k] = 1.0 / w;
        g[k] = up[k] / w;
        l[k] = lo[k];
        gp = g[k];
    }
}

} // namespace

rs_status setup(rs_plan *p)
{
    const rs_plan_desc &d = p->desc;
    const size_t asz = d.in_dtype == RS_F64 ? 8 : 4;
    const int64_t H = d.in_h, W = d.in_w;
    std::vector<double> iw_h, g_h, l_h, iw_w, g_w, l_w;
    factors(H, d.boundary, iw_h, g_h, l_h);
    factors(W, d.boundary, iw_w, g_w, l_w);
    Carver cv;
    const size_t o_coef = cv.take(size_t(H) * size_t(d.in_row_stride) * asz);
    const size_t o_dp = cv.take(size_t(H) * size_t(d.in_row_stride) * asz); // forward-elimination scratch
    const size_t o_h = cv.take(size_t(3 * H) * asz);
    const size_t o_w = cv.take(size_t(3 * W) * asz);
    cudaError_t e = cudaMalloc(&p->pbufs.p, cv.off);
    if (e != cudaSuccess) return cuda_fail(e, "allocating the B-spline coefficients");
    p->pbufs.n = cv.off;
    char *base = static_cast<char *>(p->pbufs.p);
    // per axis: [inv_w | g | l] in the working precision
    std::vector<unsigned char> host(size_t(3 * std::max(H, W)) * asz);
    auto upload = [&](size_t off, int64_t n, const std::vector<double> &a, const std::vector<double> &b,
                      const std::vector<double> &c) -> cudaError_t {
        for (int64_t k = 0; k < n; ++k) {
            const double v[3] = {a[k], b[k], c[k]};
            for (int q = 0; q < 3; ++q) {
                if (asz == 8) {
                    reinterpret_cast<double *>(host.data())[q * n + k] = v[q];
                } else {
                    reinterpret_cast<float *>(host.data())[q * n + k] = float(v[q]);
                }
            }
        }
        return cudaMemcpy(base + off, host.data(), size_t(3 * n) * asz, cudaMemcpyHostToDevice);
    };
    e = upload(o_h, H, iw_h, g_h, l_h);
    if (e == cudaSuccess) e = upload(o_w, W, iw_w, g_w, l_w);
    if (e != cudaSuccess) return cuda_fail(e, "uploading the prefilter factors");
    p->coef = base + o_coef;
    p->pf_dp = base + o_dp;
    p->pf_h = base + o_h;
    p->pf_w = base + o_w;
    return RS_OK;
}

template <typename T, typename A> cudaError_t run(rs_plan *p, const T *in, cudaStream_t s)
{
    const rs_plan_desc &d = p->desc;
    const int C = d.channels;
    const int64_t H = d.in_h, W = d.in_w, stride = d.in_row_stride;
    const A *fh = static_cast<const A *>(p->pf_h), *fw = static_cast<const A *>(p->pf_w);
    const Line<A> lw{fw, fw + W, fw + 2 * W}, lh{fh, fh + H, fh + 2 * H};
    A *coef = static_cast<A *>(p->coef), *dp = static_cast<A *>(p->pf_dp);
    const dim3 gr(unsigned((H * C + kThreads - 1) / kThreads), unsigned((W + kSeg - 1) / kSeg));
    const dim3 gc(unsigned((W * C + kThreads - 1) / kThreads), unsigned((H + kSeg - 1) / kSeg));
    rows_fwd<T, A><<<gr, kThreads, 0, s>>>(in, dp, H, W, C, stride, lw);
    rows_bwd<A><<<gr, kThreads, 0, s>>>(dp, coef, H, W, C, stride, lw);
    cols_fwd<A><<<gc, kThreads, 0, s>>>(coef, dp, H, W, C, stride, lh);
    cols_bwd<A><<<gc, kThreads, 0, s>>>(dp, coef, H, W, C, stride, lh);
    return cudaGetLastError();
}

rs_status launch(rs_plan *p, const void *d_in, cudaStream_t s)
{
    const cudaError_t e = p->desc.in_dtype == RS_F64 ? run<double, double>(p, static_cast<const double *>(d_in), s)
                                                     : run<float, float>(p, static_cast<const float *>(d_in), s);
    if (e != cudaSuccess) return cuda_fail(e, "prefilter launch");
    return RS_OK;
}

} // namespace prefilter
} // namespace rs
