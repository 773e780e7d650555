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
// host and kept in the working precision; a thread then runs one line.
//
//   rows:    one thread per (row, channel), sequential along the row;
//   columns: one thread per (column, channel), sequential down the columns
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

// One line of n samples at stride `step` (samples) from src into dst (may be
// the same buffer): forward elimination into dst, then back substitution.
template <typename T, typename A>
__device__ __forceinline__ void solve_line(const T *src, A *dst, int64_t n, int64_t step, const Line<A> &L)
{
    A prev = A(0);
    for (int64_t k = 0; k < n; ++k) {
        const A s = A(6) * A(src[k * step]);
        prev = (s - L.l[k] * prev) * L.inv_w[k];
        dst[k * step] = prev;
    }
    A next = dst[(n - 1) * step];
    for (int64_t k = n - 2; k >= 0; --k) {
        next = dst[k * step] - L.g[k] * next;
        dst[k * step] = next;
    }
}

template <typename T, typename A>
__global__ void __launch_bounds__(kThreads) rows_kernel(const T *in, A *out, int64_t rows, int64_t cols, int C,
                                                        int64_t stride, Line<A> L)
{
    const int64_t t = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (t >= rows * C) return;
    const int64_t r = t / C, c = t - r * C;
    solve_line<T, A>(in + r * stride + c, out + r * stride + c, cols, C, L);
}

template <typename A>
__global__ void __launch_bounds__(kThreads) cols_kernel(A *buf, int64_t rows, int64_t cols, int C, int64_t stride,
                                                        Line<A> L)
{
    const int64_t t = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (t >= cols * C) return;
    solve_line<A, A>(buf + t, buf + t, rows, stride, L);
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
    p->pf_h = base + o_h;
    p->pf_w = base + o_w;
    return RS_OK;
}

rs_status launch(rs_plan *p, const void *d_in, cudaStream_t s)
{
    const rs_plan_desc &d = p->desc;
    const int C = d.channels;
    const int64_t H = d.in_h, W = d.in_w, stride = d.in_row_stride;
    const unsigned gr = unsigned((H * C + kThreads - 1) / kThreads), gc = unsigned((W * C + kThreads - 1) / kThreads);
    if (d.in_dtype == RS_F64) {
        const double *fh = static_cast<const double *>(p->pf_h), *fw = static_cast<const double *>(p->pf_w);
        const Line<double> lw{fw, fw + W, fw + 2 * W}, lh{fh, fh + H, fh + 2 * H};
        double *coef = static_cast<double *>(p->coef);
        rows_kernel<double, double><<<gr, kThreads, 0, s>>>(static_cast<const double *>(d_in), coef, H, W, C, stride, lw);
        cols_kernel<double><<<gc, kThreads, 0, s>>>(coef, H, W, C, stride, lh);
    } else {
        const float *fh = static_cast<const float *>(p->pf_h), *fw = static_cast<const float *>(p->pf_w);
        const Line<float> lw{fw, fw + W, fw + 2 * W}, lh{fh, fh + H, fh + 2 * H};
        float *coef = static_cast<float *>(p->coef);
        rows_kernel<float, float><<<gr, kThreads, 0, s>>>(static_cast<const float *>(d_in), coef, H, W, C, stride, lw);
        cols_kernel<float><<<gc, kThreads, 0, s>>>(coef, H, W, C, stride, lh);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "prefilter launch");
    return RS_OK;
}

} // namespace prefilter
} // namespace rs
