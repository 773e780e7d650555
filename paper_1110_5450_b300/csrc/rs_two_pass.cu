// rs_two_pass.cu -- separate horizontal and vertical pass kernels.
//
// The horizontal pass filters every input row into an intermediate buffer in
// HBM (accumulation precision, in_h x out_w x C), the vertical pass filters
// that buffer's columns into the output.  This is the plain order "H then V":
//
//   tmp[y][x][c] = sum_k wx[x][k] in[y][start_x[x] + k][c]
//   out[y][x][c] = sum_k wy[y][k] tmp[start_y[y] + k][x][c]
//
// with the boundary-folded tables from rs_weights.cu (every index in range).
// It handles any channel count and tap count and serves as the reference
// order for the fused kernel; it moves the intermediate through HBM, so it is
// not the fast path.
#include "rs_internal.h"

namespace rs {
namespace {

template <typename A, typename T> __device__ __forceinline__ A to_acc(T v);
template <> __device__ __forceinline__ float to_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float to_acc<float, __half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_acc<float, __nv_bfloat16>(__nv_bfloat16 v)
{
    return __bfloat162float(v);
}
template <> __device__ __forceinline__ double to_acc<double, double>(double v) { return v; }

template <typename T, typename A> __device__ __forceinline__ T from_acc(A v);
template <> __device__ __forceinline__ float from_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_acc<__half, float>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16, float>(float v)
{
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ double from_acc<double, double>(double v) { return v; }

template <typename T, typename A>
__global__ void hpass_kernel(const T *__restrict__ in, A *__restrict__ tmp, int64_t in_h, int64_t out_w,
                             int64_t C, int64_t in_stride, const int32_t *__restrict__ start_x,
                             const A *__restrict__ w_x, int t)
{
    const int64_t n = in_h * out_w * C;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < n;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = idx % C;
        const int64_t xo = (idx / C) % out_w;
        const int64_t y = idx / (C * out_w);
        const T *row = in + y * in_stride + int64_t(start_x[xo]) * C + c;
        const A *w = w_x + xo * t;
        A acc = A(0);
        for (int k = 0; k < t; ++k) acc += w[k] * to_acc<A, T>(row[int64_t(k) * C]);
        tmp[idx] = acc;
    }
}

template <typename T, typename A>
__global__ void vpass_kernel(const A *__restrict__ tmp, T *__restrict__ out, int64_t out_h, int64_t out_w,
                             int64_t C, int64_t out_stride, const int32_t *__restrict__ start_y,
                             const A *__restrict__ w_y, int t)
{
    const int64_t row = out_w * C;
    const int64_t n = out_h * row;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < n;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t s = idx % row;
        const int64_t yo = idx / row;
        const A *col = tmp + int64_t(start_y[yo]) * row + s;
        const A *w = w_y + yo * t;
        A acc = A(0);
        for (int k = 0; k < t; ++k) acc += w[k] * col[int64_t(k) * row];
        out[yo * out_stride + s] = from_acc<T, A>(acc);
    }
}

template <typename T, typename A> cudaError_t run(const TwoPassArgs &a, cudaStream_t s)
{
    const int threads = 256;
    auto blocks_for = [&](int64_t n) {
        int64_t b = (n + threads - 1) / threads;
        return int(b > 148 * 64 ? 148 * 64 : (b < 1 ? 1 : b));
    };
    hpass_kernel<T, A><<<blocks_for(a.in_h * a.out_w * a.C), threads, 0, s>>>(
        static_cast<const T *>(a.in), static_cast<A *>(a.tmp), a.in_h, a.out_w, a.C, a.in_stride,
        a.start_x, static_cast<const A *>(a.w_x), a.t_x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    vpass_kernel<T, A><<<blocks_for(a.out_h * a.out_w * a.C), threads, 0, s>>>(
        static_cast<const A *>(a.tmp), static_cast<T *>(a.out), a.out_h, a.out_w, a.C, a.out_stride,
        a.start_y, static_cast<const A *>(a.w_y), a.t_y);
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_two_pass(const TwoPassArgs &a, cudaStream_t s)
{
    switch (a.dtype) {
    case RS_F64: return run<double, double>(a, s);
    case RS_F32: return run<float, float>(a, s);
    case RS_F16: return run<__half, float>(a, s);
    case RS_BF16: return run<__nv_bfloat16, float>(a, s);
    }
    return cudaErrorInvalidValue;
}

} // namespace rs
