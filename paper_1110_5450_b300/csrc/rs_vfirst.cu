// rs_vfirst.cu -- the two-pass path for strong vertical downscales: the
// vertical pass first, input -> FP32 intermediate of out_h x in_w samples, then
// the horizontal pass, intermediate -> output.  Each pass reads its source
// once from HBM (the vertical pass's overlapping row windows re-read from L2)
// with no tile halo: at x0.3 the intermediate is 0.3 of the input, at x0.125
// an eighth, which is what makes this cheaper than a fused tile whose staged
// halo grows with the band (48 taps at x0.125).
//
//   vertical:   one thread = 4 consecutive samples of a row x G_v = 8 output
//               rows; the block's row group is shared, so its J_v x 8 weights
//               are staged in shared memory once and read as broadcasts; each
//               tap is one 16-byte (FP32) or 8-byte (16-bit) coalesced load.
//   horizontal: one thread = one output row x a group of 4 output pixels with
//               its 4-pixel aligned band of J_h inputs; the intermediate row
//               carries J_h zero pixels after its end, so bands that run past
//               the image read zeros (their weights there are zero too).
//
// Both bands come from the weight tables through the band kernel, so the
// boundary rule and the FP64 normalisation are the plan's own.
#include <algorithm>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rs_plan.h"

namespace rs {
namespace vfirst {
namespace {

constexpr int kThreads = 128;
constexpr int kGV = 8;       // output rows per vertical thread
constexpr int kG = 4;        // output pixels per horizontal thread
constexpr int kMaxTaps = 256; // J_v and J_h limits (shared weights: J_v x 8 floats)

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// 4 consecutive samples (vector load when `vec`, else one by one, fewer at a
// row's end: n valid samples, the rest 0).
template <typename T> __device__ __forceinline__ float4 load4(const T *p, bool vec, int n)
{
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            return __ldg(reinterpret_cast<const float4 *>(p));
        } else {
            const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
            const T *h = reinterpret_cast<const T *>(&u);
            return make_float4(to_f<T>(h[0]), to_f<T>(h[1]), to_f<T>(h[2]), to_f<T>(h[3]));
        }
    }
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = 0; i < 4 && i < n; ++i) v[i] = to_f<T>(p[i]);
    return make_float4(v[0], v[1], v[2], v[3]);
}

template <typename T> __device__ __forceinline__ void store4(T *p, float4 a, bool vec, int n)
{
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(p) = a;
        } else {
            T h[4] = {from_f<T>(a.x), from_f<T>(a.y), from_f<T>(a.z), from_f<T>(a.w)};
            *reinterpret_cast<uint2 *>(p) = *reinterpret_cast<const uint2 *>(h);
        }
        return;
    }
    const float v[4] = {a.x, a.y, a.z, a.w};
    for (int i = 0; i < 4 && i < n; ++i) p[i] = from_f<T>(v[i]);
}

struct VArgs {
    const void *in;
    float *tmp;
    int64_t in_stride, tmp_stride; // samples
    int32_t row_samples;           // in_w * C
    int32_t out_h, JV;
    const int32_t *base; // [groups] first input row of each group of 8 output rows
    const float *band;   // [groups][stride]: per tap the 8 rows' weights
    int32_t band_stride;
    int32_t vec; // 1: 4-sample vector loads are aligned
};

// grid: x = 4-sample chunks / kThreads, y = groups of 8 output rows
template <typename T> __global__ void __launch_bounds__(kThreads) v_kernel(const VArgs a)
{
    __shared__ __align__(16) float w_s[kMaxTaps * kGV];
    const int g = blockIdx.y;
    const float *wg = a.band + int64_t(g) * a.band_stride;
    for (int e = threadIdx.x; e < a.JV * kGV; e += kThreads) w_s[e] = __ldg(wg + e);
    __syncthreads();
    const int ch = blockIdx.x * kThreads + threadIdx.x;
    const int s0 = ch * 4;
    if (s0 >= a.row_samples) return;
    const int n = min(4, a.row_samples - s0);
    const bool vec = a.vec && n == 4;
    const T *src = static_cast<const T *>(a.in) + int64_t(__ldg(a.base + g)) * a.in_stride + s0;
    float acc[kGV][4];
#pragma unroll
    for (int r = 0; r < kGV; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
#pragma unroll 4
    for (int j = 0; j < a.JV; ++j) {
        const float4 x = load4<T>(src + int64_t(j) * a.in_stride, vec, n);
        const float4 *w4 = reinterpret_cast<const float4 *>(w_s + j * kGV);
        const float4 wa = w4[0], wb = w4[1];
        const float w[kGV] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
        for (int r = 0; r < kGV; ++r) {
            acc[r][0] = fmaf(w[r], x.x, acc[r][0]);
            acc[r][1] = fmaf(w[r], x.y, acc[r][1]);
            acc[r][2] = fmaf(w[r], x.z, acc[r][2]);
            acc[r][3] = fmaf(w[r], x.w, acc[r][3]);
        }
    }
#pragma unroll
    for (int r = 0; r < kGV; ++r) {
        const int y = g * kGV + r;
        if (y >= a.out_h) break;
        store4<float>(a.tmp + int64_t(y) * a.tmp_stride + s0, make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]),
                      n == 4, n);
    }
}

struct HArgs {
    const float *tmp;
    void *out;
    int64_t tmp_stride, out_stride; // samples
    int32_t out_h, out_w, groups, JH;
    const int32_t *base; // [groups] first input pixel of each group (multiple of 4)
    const float *band;   // [groups][stride]: per input pixel the 4 outputs' weights
    int32_t band_stride;
    int32_t vec; // 1: the output base and pitch allow 4-sample vector stores
};

// grid: x = groups of 4 output pixels / kThreads, y = output rows
template <typename T, int C> __global__ void __launch_bounds__(kThreads) h_kernel(const HArgs a)
{
    const int q = blockIdx.x * kThreads + threadIdx.x;
    const int y = blockIdx.y;
    if (q >= a.groups) return;
    const float4 *src = reinterpret_cast<const float4 *>(a.tmp + int64_t(y) * a.tmp_stride +
                                                          int64_t(__ldg(a.base + q)) * C);
    const float4 *wq = reinterpret_cast<const float4 *>(a.band + int64_t(q) * a.band_stride);
    float acc[kG][C];
#pragma unroll
    for (int g = 0; g < kG; ++g)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[g][c] = 0.f;
    for (int t0 = 0; t0 < a.JH; t0 += 4) {
        float d[4 * C];
#pragma unroll
        for (int v = 0; v < C; ++v) {
            const float4 x = __ldg(src + v);
            d[4 * v] = x.x;
            d[4 * v + 1] = x.y;
            d[4 * v + 2] = x.z;
            d[4 * v + 3] = x.w;
        }
        src += C;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float4 w = __ldg(wq + t);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float x = d[t * C + c];
                acc[0][c] = fmaf(w.x, x, acc[0][c]);
                acc[1][c] = fmaf(w.y, x, acc[1][c]);
                acc[2][c] = fmaf(w.z, x, acc[2][c]);
                acc[3][c] = fmaf(w.w, x, acc[3][c]);
            }
        }
        wq += 4;
    }
    // the group's 4 x C samples are consecutive in the output row
    float o[kG * C];
#pragma unroll
    for (int g = 0; g < kG; ++g)
#pragma unroll
        for (int c = 0; c < C; ++c) o[g * C + c] = acc[g][c];
    T *dst = static_cast<T *>(a.out) + int64_t(y) * a.out_stride + int64_t(q) * kG * C;
    const int n = (min(a.out_w - q * kG, kG)) * C; // valid samples of the group
#pragma unroll
    for (int v = 0; v < C; ++v) {
        const int nv = n - 4 * v;
        if (nv <= 0) break;
        store4<T>(dst + 4 * v, make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]), a.vec && nv >= 4, nv);
    }
}

template <typename T> const void *h_fn(int C)
{
    return C == 1 ? reinterpret_cast<const void *>(&h_kernel<T, 1>) : reinterpret_cast<const void *>(&h_kernel<T, 3>);
}

} // namespace

rs_status setup(rs_plan *p, cudaStream_t s)
{
    p->vfirst_ok = 0;
    const rs_plan_desc &d = p->desc;
    const int C = d.channels;
    if ((d.in_dtype != RS_F32 && d.in_dtype != RS_F16 && d.in_dtype != RS_BF16) || (C != 1 && C != 3))
        return RS_ERR_UNSUPPORTED;
    const AxisGeom &gx = p->gx, &gy = p->gy;
    if (gy.n_out > gy.n_in) return RS_ERR_UNSUPPORTED; // the intermediate would outgrow the input
    if (gy.n_out > 65535) return RS_ERR_UNSUPPORTED; // grid rows of the horizontal pass
    const std::vector<int32_t> &sx = p->host_start_x, &sy = p->host_start_y;
    // vertical: groups of 8 rows, the widest group span
    int JV = 0;
    for (size_t i = 0; i < sy.size(); i += kGV) {
        int lo = sy[i], hi = sy[i] + gy.t_eff;
        for (size_t r = 1; r < size_t(kGV) && i + r < sy.size(); ++r) {
            lo = std::min(lo, int(sy[i + r]));
            hi = std::max(hi, int(sy[i + r]) + gy.t_eff);
        }
        JV = std::max(JV, hi - lo);
    }
    // horizontal: groups of 4 outputs on 4-pixel aligned bases
    const int groups_x = int((gx.n_out + kG - 1) / kG);
    int JH = 0;
    for (int q = 0; q < groups_x; ++q) {
        int lo = int(gx.n_in), hi = 0;
        for (int m = 0; m < kG && q * kG + m < gx.n_out; ++m) {
            lo = std::min(lo, int(sx[q * kG + m]));
            hi = std::max(hi, int(sx[q * kG + m]) + gx.t_eff);
        }
        JH = std::max(JH, hi - (lo & ~3));
    }
    JH = (JH + 3) / 4 * 4;
    if (JV > kMaxTaps || JV > gy.n_in || JH > kMaxTaps) return RS_ERR_UNSUPPORTED;

    const int groups_y = int((gy.n_out + kGV - 1) / kGV);
    // intermediate rows of in_w samples followed by JH zero pixels, a whole
    // number of 16-byte words
    const int64_t tmp_stride = (int64_t(gx.n_in + JH) * C + 3) / 4 * 4;
    Carver cv;
    const size_t o_vb = cv.take(size_t(groups_y) * 4);
    const size_t o_vw = cv.take(size_t(groups_y) * band_stride(kGV, JV) * 4);
    const size_t o_hb = cv.take(size_t(groups_x) * 4);
    const size_t o_hw = cv.take(size_t(groups_x) * band_stride(kG, JH) * 4);
    const size_t o_tmp = cv.take(size_t(gy.n_out) * size_t(tmp_stride) * 4);
    if (p->vbufs.p) {
        cudaFree(p->vbufs.p);
        p->vbufs.p = nullptr;
    }
    cudaError_t e = cudaMalloc(&p->vbufs.p, cv.off);
    if (e != cudaSuccess) return cuda_fail(e, "allocating the vertical-first intermediate");
    p->vbufs.n = cv.off;
    char *base = static_cast<char *>(p->vbufs.p);
    // the zero tail of every intermediate row is never written again
    e = cudaMemsetAsync(base + o_tmp, 0, size_t(gy.n_out) * size_t(tmp_stride) * 4, s);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the vertical-first intermediate");
    VfParams &v = p->vf;
    v = VfParams{};
    v.JV = JV;
    v.JH = JH;
    v.groups_y = groups_y;
    v.groups_x = groups_x;
    v.tmp_stride = tmp_stride;
    v.vbase = reinterpret_cast<int32_t *>(base + o_vb);
    v.vband = reinterpret_cast<float *>(base + o_vw);
    v.hbase = reinterpret_cast<int32_t *>(base + o_hb);
    v.hband = reinterpret_cast<float *>(base + o_hw);
    v.tmp = reinterpret_cast<float *>(base + o_tmp);
    const rs_status st = rebuild(p, s);
    if (st != RS_OK) return st;
    p->vfirst_ok = 1;
    p->scratch_bytes = int64_t(p->tables.n + p->bands.n + p->tmp.n + p->sbufs.n + p->vbufs.n);
    return RS_OK;
}

rs_status rebuild(rs_plan *p, cudaStream_t s)
{
    const VfParams &v = p->vf;
    AxisTables vt = p->ty;
    vt.G = kGV;
    vt.J = v.JV;
    vt.groups = v.groups_y;
    vt.dup = 1;
    vt.pair_ngx = 0;
    vt.align = 0;
    vt.band_base = v.vbase;
    vt.band_w = v.vband;
    AxisTables ht = p->tx;
    ht.G = kG;
    ht.J = v.JH;
    ht.groups = v.groups_x;
    ht.dup = 1;
    ht.pair_ngx = 0;
    ht.align = 4;
    ht.band_base = v.hbase;
    ht.band_w = v.hband;
    WeightArgs a0, a1;
    a0.g = p->gy;
    a0.t = vt;
    a1.g = p->gx;
    a1.t = ht;
    a0.work_is_double = a1.work_is_double = 0;
    a0.err = a1.err = p->d_err;
    const cudaError_t e = launch_band(a0, a1, s);
    if (e != cudaSuccess) return cuda_fail(e, "vertical-first band launch");
    return RS_OK;
}

rs_status launch(rs_plan *p, const void *d_in, void *d_out, cudaStream_t s)
{
    const rs_plan_desc &d = p->desc;
    const VfParams &v = p->vf;
    const int C = d.channels, es = int(dt_size(d.in_dtype));
    VArgs va;
    va.in = d_in;
    va.tmp = v.tmp;
    va.in_stride = d.in_row_stride;
    va.tmp_stride = v.tmp_stride;
    va.row_samples = int32_t(p->gx.n_in * C);
    va.out_h = int32_t(p->gy.n_out);
    va.JV = v.JV;
    va.base = v.vbase;
    va.band = v.vband;
    va.band_stride = band_stride(kGV, v.JV);
    va.vec = ((reinterpret_cast<uintptr_t>(d_in) | uintptr_t(d.in_row_stride * es)) & uintptr_t(4 * es - 1)) == 0;
    const int nchunks = (va.row_samples + 3) / 4;
    const dim3 gv((nchunks + kThreads - 1) / kThreads, v.groups_y);
    void *vargs[1] = {&va};
    const void *vfn = d.in_dtype == RS_F16    ? reinterpret_cast<const void *>(&v_kernel<__half>)
                      : d.in_dtype == RS_BF16 ? reinterpret_cast<const void *>(&v_kernel<__nv_bfloat16>)
                                              : reinterpret_cast<const void *>(&v_kernel<float>);
    cudaError_t e = cudaLaunchKernel(vfn, gv, dim3(kThreads), vargs, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "vertical-first vertical pass launch");
    HArgs ha;
    ha.tmp = v.tmp;
    ha.out = d_out;
    ha.tmp_stride = v.tmp_stride;
    ha.out_stride = d.out_row_stride;
    ha.out_h = int32_t(p->gy.n_out);
    ha.out_w = int32_t(p->gx.n_out);
    ha.groups = v.groups_x;
    ha.JH = v.JH;
    ha.base = v.hbase;
    ha.band = v.hband;
    ha.band_stride = band_stride(kG, v.JH);
    ha.vec = ((reinterpret_cast<uintptr_t>(d_out) | uintptr_t(d.out_row_stride * es)) & uintptr_t(4 * es - 1)) == 0;
    void *hargs[1] = {&ha};
    const void *hfn = d.in_dtype == RS_F16 ? h_fn<__half>(C) : d.in_dtype == RS_BF16 ? h_fn<__nv_bfloat16>(C) : h_fn<float>(C);
    const dim3 gh((v.groups_x + kThreads - 1) / kThreads, unsigned(p->gy.n_out));
    e = cudaLaunchKernel(hfn, gh, dim3(kThreads), hargs, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "vertical-first horizontal pass launch");
    return RS_OK;
}

} // namespace vfirst
} // namespace rs
