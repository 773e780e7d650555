// rs_warp.cu -- affine warps with elliptical weighted average (EWA)
// filtering (P. Heckbert, "Fundamentals of Texture Mapping and Image
// Warping", 1989; N. Greene and P. Heckbert, IEEE CG&A 6(6), 1986): the
// non-separable counterpart of the separable resampler.
//
// Output pixel (x, y) maps to the input point c = A (x + 1/2, y + 1/2) + t.
// The filter is a Gaussian of covariance V = sigma^2 (J J^T + I) in input
// pixels (reconstruction filter of width sigma convolved with the prefilter
// of width sigma in output pixels carried back by the Jacobian J = A), so a
// minifying warp widens it along the directions it shrinks -- the elliptical
// footprint.  Sample s gets exp(-Q/2) - exp(-r^2/2) for
// Q = (s - c)^T V^-1 (s - c) < r^2: the Gaussian truncated at the ellipse and
// lowered to reach zero there (continuous weights); the result is normalised
// by the weight sum.  Boundary maps as for resampling.
//
// One thread per output pixel.  The input point is computed in FP64 and
// split into an integer base and a fraction, so the per-tap offsets (small
// numbers) are exact to FP32 rounding; weights and sums are FP32.  Along a
// row of taps the quadratic form is advanced by forward differences (two
// additions per tap), the exponential is the fast intrinsic, and the
// boundary map is skipped when the whole footprint lies inside the image.
// The weights are continuous (zero at the ellipse), so rounding that moves a
// tap across the ellipse changes nothing measurable.
#include <cmath>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rs_plan.h"

namespace rs {
namespace warp {
namespace {

constexpr int kThreads = 128;

struct Args {
    const void *in;
    void *out;
    int64_t in_stride, out_stride; // samples
    int32_t in_h, in_w, out_h, out_w, boundary;
    double a0, a1, a2, a3, a4, a5;
    float vi00, vi01, vi11; // V^-1
    float r2, wcut;         // cutoff^2, exp(-cutoff^2 / 2)
    double eu, ev;          // half-extents of the ellipse's bounding box
};

template <typename T> __device__ __forceinline__ float ld(const T *p);
template <> __device__ __forceinline__ float ld<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<__half>(const __half *p) { return __half2float(*p); }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
template <typename T> __device__ __forceinline__ T st(float v);
template <> __device__ __forceinline__ float st<float>(float v) { return v; }
template <> __device__ __forceinline__ __half st<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 st<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Boundary map of index j on an axis of n samples (-1: dropped).
__device__ __forceinline__ int64_t map_idx(int64_t j, int64_t n, int boundary)
{
    if (j >= 0 && j < n) return j;
    switch (boundary) {
    case RS_B_CLAMP: return j < 0 ? 0 : n - 1;
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
    }
    return -1; // truncate
}

template <typename T, int C> __global__ void __launch_bounds__(kThreads, 4) warp_kernel(const Args a)
{
    const int64_t t = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (t >= int64_t(a.out_h) * a.out_w) return;
    const int64_t y = t / a.out_w, x = t - y * a.out_w;
    const double px = double(x) + 0.5, py = double(y) + 0.5;
    const double cu = a.a0 * px + a.a1 * py + a.a2, cv = a.a3 * px + a.a4 * py + a.a5;
    const int64_t i0 = int64_t(ceil(cu - a.eu - 0.5)), i1 = int64_t(floor(cu + a.eu - 0.5));
    const int64_t j0 = int64_t(ceil(cv - a.ev - 0.5)), j1 = int64_t(floor(cv + a.ev - 0.5));
    // offsets of the first tap, exact in FP64, small enough for FP32
    const float fu = float(double(i0) + 0.5 - cu), fv = float(double(j0) + 0.5 - cv);
    const T *src = static_cast<const T *>(a.in);
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.f;
    float wsum = 0.f;
    const bool inside = i0 >= 0 && i1 < a.in_w && j0 >= 0 && j1 < a.in_h;
    const int ni = int(i1 - i0) + 1;
    const float dd = 2.f * a.vi00; // second difference of q along a row
    for (int64_t j = j0; j <= j1; ++j) {
        const int64_t mj = inside ? j : map_idx(j, a.in_h, a.boundary);
        if (mj < 0) continue;
        const float dv = fv + float(j - j0);
        const float qv = a.vi11 * dv * dv;
        const float quv = 2.f * a.vi01 * dv;
        const T *row = src + mj * a.in_stride;
        // q(du) = vi00 du^2 + quv du + qv at du = fu, fu + 1, ...
        float q = fmaf(fmaf(a.vi00, fu, quv), fu, qv);
        float d = fmaf(a.vi00, fmaf(2.f, fu, 1.f), quv);
        if (inside) {
            const T *s = row + i0 * C;
            for (int k = 0; k < ni; ++k, s += C) {
                if (q < a.r2) {
                    const float w = __expf(-0.5f * q) - a.wcut;
#pragma unroll
                    for (int c = 0; c < C; ++c) acc[c] = fmaf(w, ld<T>(s + c), acc[c]);
                    wsum += w;
                }
                q += d;
                d += dd;
            }
        } else {
            for (int k = 0; k < ni; ++k) {
                if (q < a.r2) {
                    const int64_t mi = map_idx(i0 + k, a.in_w, a.boundary);
                    if (mi >= 0) {
                        const float w = __expf(-0.5f * q) - a.wcut;
                        const T *s = row + mi * C;
#pragma unroll
                        for (int c = 0; c < C; ++c) acc[c] = fmaf(w, ld<T>(s + c), acc[c]);
                        wsum += w;
                    }
                }
                q += d;
                d += dd;
            }
        }
    }
    T *o = static_cast<T *>(a.out) + y * a.out_stride + x * C;
    const float inv = wsum > 0.f ? 1.f / wsum : 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) o[c] = st<T>(acc[c] * inv);
}

template <typename T> const void *fn_for(int C)
{
    switch (C) {
    case 1: return reinterpret_cast<const void *>(&warp_kernel<T, 1>);
    case 2: return reinterpret_cast<const void *>(&warp_kernel<T, 2>);
    case 3: return reinterpret_cast<const void *>(&warp_kernel<T, 3>);
    case 4: return reinterpret_cast<const void *>(&warp_kernel<T, 4>);
    }
    return nullptr;
}

} // namespace
} // namespace warp
} // namespace rs

using namespace rs;

extern "C" rs_status rs_warp(const rs_warp_desc *desc, const void *d_in, void *d_out, void *stream)
{
    const Range range("rs_warp");
    if (!desc || !d_in || !d_out) return fail(RS_ERR_INVALID_ARG, "warp: NULL descriptor or buffer");
    const rs_warp_desc &d = *desc;
    if (d.in_h < 1 || d.in_w < 1 || d.out_h < 1 || d.out_w < 1 || d.channels < 1 || d.channels > 4)
        return fail(RS_ERR_INVALID_ARG, "warp: sizes >= 1 and 1..4 channels");
    if (d.boundary < RS_B_CLAMP || d.boundary > RS_B_TRUNCATE) return fail(RS_ERR_INVALID_ARG, "warp: boundary");
    if (d.dtype != RS_F32 && d.dtype != RS_F16 && d.dtype != RS_BF16)
        return fail(RS_ERR_UNSUPPORTED, "warp: FP32, FP16 or BF16 storage");
    for (double v : d.a)
        if (!std::isfinite(v)) return fail(RS_ERR_INVALID_ARG, "warp: non-finite transform");
    if (!(d.sigma > 0.0 && d.sigma <= 64.0) || !(d.cutoff > 0.0 && d.cutoff <= 8.0))
        return fail(RS_ERR_INVALID_ARG, "warp: sigma in (0, 64], cutoff in (0, 8]");
    const int64_t in_stride = d.in_row_stride ? d.in_row_stride : int64_t(d.in_w) * d.channels;
    const int64_t out_stride = d.out_row_stride ? d.out_row_stride : int64_t(d.out_w) * d.channels;
    if (in_stride < int64_t(d.in_w) * d.channels || out_stride < int64_t(d.out_w) * d.channels)
        return fail(RS_ERR_INVALID_ARG, "warp: row stride shorter than a row");
    // covariance V = sigma^2 (J J^T + I) and its inverse, in FP64
    const double s2 = d.sigma * d.sigma;
    const double v00 = s2 * (d.a[0] * d.a[0] + d.a[1] * d.a[1] + 1.0);
    const double v01 = s2 * (d.a[0] * d.a[3] + d.a[1] * d.a[4]);
    const double v11 = s2 * (d.a[3] * d.a[3] + d.a[4] * d.a[4] + 1.0);
    const double det = v00 * v11 - v01 * v01;
    const double eu = d.cutoff * std::sqrt(v00), ev = d.cutoff * std::sqrt(v11);
    if (!(det > 0.0) || eu > 4096.0 || ev > 4096.0) return fail(RS_ERR_UNSUPPORTED, "warp: footprint too large");
    warp::Args a;
    a.in = d_in;
    a.out = d_out;
    a.in_stride = in_stride;
    a.out_stride = out_stride;
    a.in_h = d.in_h;
    a.in_w = d.in_w;
    a.out_h = d.out_h;
    a.out_w = d.out_w;
    a.boundary = d.boundary;
    a.a0 = d.a[0];
    a.a1 = d.a[1];
    a.a2 = d.a[2];
    a.a3 = d.a[3];
    a.a4 = d.a[4];
    a.a5 = d.a[5];
    a.vi00 = float(v11 / det);
    a.vi01 = float(-v01 / det);
    a.vi11 = float(v00 / det);
    a.r2 = float(d.cutoff * d.cutoff);
    a.wcut = float(std::exp(-0.5 * d.cutoff * d.cutoff));
    a.eu = eu;
    a.ev = ev;
    const void *fn = d.dtype == RS_F16    ? warp::fn_for<__half>(d.channels)
                     : d.dtype == RS_BF16 ? warp::fn_for<__nv_bfloat16>(d.channels)
                                          : warp::fn_for<float>(d.channels);
    void *args[1] = {&a};
    const int64_t n = int64_t(d.out_h) * d.out_w;
    if ((n + warp::kThreads - 1) / warp::kThreads > int64_t(0x7fffffff))
        return fail(RS_ERR_UNSUPPORTED, "warp: output too large for one launch");
    const cudaError_t e = cudaLaunchKernel(fn, dim3(unsigned((n + warp::kThreads - 1) / warp::kThreads)),
                                           dim3(warp::kThreads), args, 0, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "warp kernel launch");
    return RS_OK;
}
