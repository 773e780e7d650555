// rs_tcstream.cu -- host side of the tensor-core streaming downscale
// (rs_tcstream.cuh): eligibility, the strips' staged windows, the per-strip
// weight matrices (built on the device from the plan's window tables), the
// work split and the launch.  FP16 and BF16 plans of 1 or 3 channels that
// downscale both axes, with in_w * channels a multiple of 8, a 16-byte row
// pitch and at most 128 vertical taps.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rs_plan.h"
#include "rs_tcstream.cuh"

namespace rs {
namespace tcstream {
namespace {

template <typename T, int C> const void *fn_of() { return reinterpret_cast<const void *>(&tcstream_kernel<T, C>); }

const void *kernel_for(int dtype, int C)
{
    if (dtype == RS_BF16) return C == 1 ? fn_of<__nv_bfloat16, 1>() : C == 3 ? fn_of<__nv_bfloat16, 3>() : nullptr;
    if (dtype == RS_F16) return C == 1 ? fn_of<__half, 1>() : C == 3 ? fn_of<__half, 3>() : nullptr;
    return nullptr;
}

// B of every strip: hi and lo 16-bit parts of the window weights, in the
// canonical K-major layout (core matrices of 8 outputs x 8 samples).  Block
// (strip, n) fills column n.
template <typename T>
__global__ void build_b_kernel(const int32_t *start_x, const float *wx, int t_x, int out_w, int C, int NP, int Kc,
                               const int32_t *g0, unsigned char *bmat)
{
    const int s = blockIdx.x, n = blockIdx.y;
    const int j = s * NP + n / C, c = n % C;
    const size_t bpart = b_bytes(Kc);
    unsigned char *bh = bmat + size_t(s) * 2 * bpart, *bl = bh + bpart;
    const int gz = g0[s];
    const bool valid = j < out_w;
    const int st = valid ? start_x[j] : 0;
    for (int k = threadIdx.x; k < Kc; k += blockDim.x) {
        const int sample = gz * 8 + k, x = sample / C, cs = sample - x * C;
        float w = 0.f;
        if (valid && cs == c && x >= st && x < st + t_x) w = wx[size_t(j) * t_x + (x - st)];
        const T hi = fused::from_acc<T, float>(w);
        const T lo = fused::from_acc<T, float>(w - fused::to_acc<float, T>(hi));
        const size_t off = size_t(n / 8) * size_t(Kc) * 16 + size_t(k / 8) * 128 + size_t(n % 8) * 16 + size_t(k % 8) * 2;
        *reinterpret_cast<T *>(bh + off) = hi;
        *reinterpret_cast<T *>(bl + off) = lo;
    }
}

// The vertical band of every row group q (output rows 4 q .. 4 q + 3): at
// union row u (input row sy[4 q] + u) the 4 rows' window weights, zero outside
// a row's own window and past the image's last row; and per group its first
// union row and union rows.  Block q fills group q.
__global__ void build_vband_kernel(const int32_t *sy, const float *wy, int t_y, int out_h, int gpr, int Uv,
                                   float4 *vband, int2 *vinfo)
{
    const int q = blockIdx.x;
    if (q >= gpr) return;
    const int i0 = q * kVG, n = min(kVG, out_h - i0);
    const int s0 = sy[i0];
    int st[kVG];
#pragma unroll
    for (int r = 0; r < kVG; ++r) st[r] = r < n ? sy[i0 + r] - s0 : -1;
    for (int u = threadIdx.x; u < Uv; u += blockDim.x) {
        float w[kVG];
#pragma unroll
        for (int r = 0; r < kVG; ++r) {
            const int t = u - st[r];
            w[r] = (st[r] >= 0 && t >= 0 && t < t_y) ? wy[size_t(i0 + r) * t_y + t] : 0.f;
        }
        vband[size_t(q) * Uv + u] = make_float4(w[0], w[1], w[2], w[3]);
    }
    if (threadIdx.x == 0) vinfo[q] = make_int2(s0, st[n - 1] + t_y);
}

struct Geometry {
    int C = 0, NP = 0, n_strips = 0, Kc = 0, Ty = 0, Uv = 0, gpr = 0;
    std::vector<int32_t> g0;
};

rs_status geometry(const rs_plan *p, Geometry &g)
{
    const rs_plan_desc &d = p->desc;
    g.C = d.channels;
    if ((d.in_dtype != RS_F16 && d.in_dtype != RS_BF16) || d.out_dtype != d.in_dtype || (g.C != 1 && g.C != 3) ||
        (d.flags & (RS_NO_STREAM | RS_FORCE_SIMT)) || p->prefilter || p->work_double)
        return RS_ERR_UNSUPPORTED;
    if (!tma_layout_ok(p) || (p->gx.n_in * g.C) % 8 != 0) return RS_ERR_UNSUPPORTED;
    if (p->gx.n_out >= p->gx.n_in || p->gy.n_out >= p->gy.n_in) return RS_ERR_UNSUPPORTED; // downscales
    g.Ty = p->gy.t_eff;
    if (g.Ty > kMaxTy || p->gy.n_in >= (int64_t(1) << 30)) return RS_ERR_UNSUPPORTED;
    const std::vector<int32_t> &sx = p->host_start_x;
    if (int64_t(sx.size()) != p->gx.n_out || int64_t(p->host_start_y.size()) != p->gy.n_out) return RS_ERR_UNSUPPORTED;
    g.NP = kN / g.C;
    const int out_w = int(p->gx.n_out), tx = p->gx.t_eff;
    g.n_strips = (out_w + g.NP - 1) / g.NP;
    g.g0.resize(size_t(g.n_strips));
    int need = 0;
    for (int s = 0; s < g.n_strips; ++s) {
        const int j0 = s * g.NP, j1 = std::min(out_w, j0 + g.NP);
        int lo = sx[size_t(j0)], hi = sx[size_t(j0)] + tx;
        for (int j = j0; j < j1; ++j) {
            lo = std::min(lo, int(sx[size_t(j)]));
            hi = std::max(hi, int(sx[size_t(j)]) + tx);
        }
        const int gz = lo * g.C / 8;
        g.g0[size_t(s)] = gz;
        need = std::max(need, hi * g.C - 8 * gz);
    }
    g.Kc = (need + kKC - 1) / kKC * kKC;
    // rows spanned by a row group's windows (kVG output rows from a multiple of kVG)
    const std::vector<int32_t> &sy = p->host_start_y;
    g.gpr = int((sy.size() + kVG - 1) / kVG);
    g.Uv = 0;
    for (size_t i = 0; i < sy.size(); i += kVG) {
        const size_t j = std::min(sy.size() - 1, i + kVG - 1);
        g.Uv = std::max(g.Uv, int(sy[j] - sy[i]) + g.Ty);
    }
    if (g.Uv > kMaxTy) return RS_ERR_UNSUPPORTED; // a band must span at most two blocks
    return RS_OK;
}

} // namespace

bool eligible(const rs_plan *p)
{
    Geometry g;
    return geometry(p, g) == RS_OK;
}

size_t space_bound(const AxisGeom &gx, const AxisGeom &gy, int C)
{
    const int64_t np = kN / C;
    const int64_t n_strips = (gx.n_out + np - 1) / np;
    // a strip's windows span at most (np - 1) n_in / n_out + 1 starts plus t_eff inputs
    const int64_t span = ((np - 1) * gx.n_in + gx.n_out - 1) / gx.n_out + 1 + gx.t_eff;
    const int64_t kc = (span * C + 8 + kKC - 1) / kKC * kKC;
    // a row group's windows span at most 3 n_in / n_out + 1 starts plus t_eff rows
    const int64_t gpr = (gy.n_out + kVG - 1) / kVG;
    const int64_t uv = std::min<int64_t>(kMaxTy, (3 * gy.n_in + gy.n_out - 1) / gy.n_out + 1 + gy.t_eff);
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    return size_t(n_strips) * 2 * b_bytes(int(kc)) + up(size_t(n_strips) * 4) + up(size_t(gpr * uv) * 16) +
           up(size_t(gpr) * 8) + 512;
}

void preload(int dtype)
{
    for (const int C : {1, 3})
        if (const void *fn = kernel_for(dtype, C)) occupancy(fn, 32 * (kFixedWarps + 4), 0);
}

rs_status setup(rs_plan *p, cudaStream_t s, const stream::Opts &o)
{
    p->tcs_on = 0;
    Geometry g;
    const rs_status gs = geometry(p, g);
    if (gs != RS_OK) return gs;
    const rs_plan_desc &d = p->desc;
    const bool vw_set = o.ex == 2 && o.vw > 0;
    int VW = vw_set ? std::min(kMaxVW, o.vw) : 8;
    int NA = o.ex == 2 && o.ni_min >= 2 ? std::min(kMaxNA, o.ni_min) : 4;
    const void *fn = kernel_for(d.in_dtype, g.C);
    int nthreads = 32 * (kFixedWarps + VW);
    // three blocks in the filtered-row ring where they fit (the read-back then
    // runs a block ahead of the vertical pass), else two; then the staged chunks
    int NS = kMaxNS;
    auto fits = [&](int na, int ns) {
        const size_t t = layout(g.Kc, na, g.Uv, VW, ns).total;
        return t <= 227 * 1024 && occupancy(fn, nthreads, t) >= 1;
    };
    if (!fits(NA, NS)) NS = 2;
    if (!vw_set && !fits(NA, NS)) {
        // wide strips (strong downscales) are bound by the latency of the
        // staged input, not by the vertical pass: keep the staged chunks and
        // take 4 vertical warps (x0.125: 4 chunks and 4 warps 45 us, 3 chunks
        // and 8 warps 49 us)
        VW = 4;
        nthreads = 32 * (kFixedWarps + VW);
    }
    while (NA > 2 && !fits(NA, NS)) --NA;
    if (!fits(NA, NS)) return RS_ERR_UNSUPPORTED;
    const size_t smem = layout(g.Kc, NA, g.Uv, VW, NS).total;
    if (o.ex == 2 && o.ni_min >= 2 && NA != std::min(kMaxNA, o.ni_min)) return RS_ERR_UNSUPPORTED;

    // device tables: per-strip weight matrices, first staged groups
    Carver cv;
    const size_t o_b = cv.take(size_t(g.n_strips) * 2 * b_bytes(g.Kc));
    const size_t o_g = cv.take(size_t(g.n_strips) * 4);
    const size_t o_vb = cv.take(size_t(g.gpr) * g.Uv * 16);
    const size_t o_vi = cv.take(size_t(g.gpr) * 8);
    char *base = nullptr;
    cudaError_t e = cudaSuccess;
    if (p->ext_base) {
        // the caller's space, the starts uploaded through its pinned staging on `s`
        if (cv.off > p->ext_bytes || size_t(g.n_strips) * 4 > p->ext_staging_bytes) return RS_ERR_UNSUPPORTED;
        std::memcpy(p->ext_staging, g.g0.data(), size_t(g.n_strips) * 4);
        e = cudaMemcpyAsync(p->ext_base + o_g, p->ext_staging, size_t(g.n_strips) * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "uploading tensor-core strip starts");
        base = p->ext_base;
    } else {
        if (p->tcbufs.p) {
            cudaFree(p->tcbufs.p);
            p->tcbufs.p = nullptr;
        }
        e = cudaMalloc(&p->tcbufs.p, cv.off);
        if (e != cudaSuccess) return cuda_fail(e, "allocating tensor-core strip tables");
        p->tcbufs.n = cv.off;
        base = static_cast<char *>(p->tcbufs.p);
        e = cudaMemcpy(base + o_g, g.g0.data(), size_t(g.n_strips) * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "uploading tensor-core strip starts");
    }
    Params &tp = p->tcp;
    std::memset(&tp, 0, sizeof tp);
    tp.in_h = int32_t(p->gy.n_in);
    tp.out_h = int32_t(p->gy.n_out);
    tp.out_w = int32_t(p->gx.n_out);
    tp.C = g.C;
    tp.out_stride = d.out_row_stride;
    tp.bmat = reinterpret_cast<const unsigned char *>(base + o_b);
    tp.g0 = reinterpret_cast<const int32_t *>(base + o_g);
    tp.sy = p->ty.start;
    tp.vband = reinterpret_cast<const float4 *>(base + o_vb);
    tp.vinfo = reinterpret_cast<const int2 *>(base + o_vi);
    tp.gpr = g.gpr;
    tp.Kc = g.Kc;
    tp.NP = g.NP;
    tp.n_strips = g.n_strips;
    tp.Ty = g.Ty;
    tp.Uv = g.Uv;
    tp.NS = NS;
    tp.NA = NA;
    tp.VW = VW;
    tp.pf = o.ex == 2 && o.pf ? 2 * NA : 0;
    const int64_t total = int64_t(g.n_strips) * g.gpr;
    // a CTA per SM; runs of at least 4 row groups (each run re-reads its
    // windows' first rows)
    tp.per_cta = std::max<int64_t>((total + p->num_sms - 1) / p->num_sms, std::min<int64_t>(4, g.gpr));
    tp.err = p->d_err;
    p->tcs_on = 1;
    p->x_on = 0;
    const rs_status st = rebuild(p, s);
    if (st != RS_OK) {
        p->tcs_on = 0;
        return st;
    }
    p->s_fn = fn;
    p->s_block = nthreads;
    p->s_smem = smem;
    p->s_grid = int((total + tp.per_cta - 1) / tp.per_cta);
    p->s_ctas = 1;
    p->stmap_ptr = nullptr;
    stream::Opts used;
    used.ex = 2;
    used.ni_min = NA;
    used.vw = VW;
    used.sw = g.NP;
    used.pf = tp.pf ? 1 : 0;
    p->stream_code = used.code();
    p->stream_ok = 1;
    return RS_OK;
}

rs_status rebuild(rs_plan *p, cudaStream_t s)
{
    const Params &tp = p->tcp;
    const dim3 grid(unsigned(tp.n_strips), unsigned(kN));
    const int32_t *sx = p->tx.start;
    const float *wx = static_cast<const float *>(p->tx.wwork);
    unsigned char *bm = const_cast<unsigned char *>(tp.bmat);
    if (p->desc.in_dtype == RS_BF16)
        build_b_kernel<__nv_bfloat16><<<grid, 128, 0, s>>>(sx, wx, p->gx.t_eff, tp.out_w, tp.C, tp.NP, tp.Kc, tp.g0, bm);
    else
        build_b_kernel<__half><<<grid, 128, 0, s>>>(sx, wx, p->gx.t_eff, tp.out_w, tp.C, tp.NP, tp.Kc, tp.g0, bm);
    build_vband_kernel<<<unsigned(tp.gpr), 64, 0, s>>>(p->ty.start, static_cast<const float *>(p->ty.wwork),
                                                       p->gy.t_eff, tp.out_h, tp.gpr, tp.Uv,
                                                       const_cast<float4 *>(tp.vband), const_cast<int2 *>(tp.vinfo));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core weight matrix launch");
    return RS_OK;
}

rs_status launch(rs_plan *p, const void *d_in, void *d_out, cudaStream_t s)
{
    const rs_plan_desc &d = p->desc;
    if (p->stmap_ptr != d_in) {
        // boxes of 64 samples (128 bytes) x 128 rows, landed with the 128-byte
        // swizzle: the kernel's K-major operand layout
        cuuint64_t dims[2] = {cuuint64_t(p->gx.n_in * d.channels), cuuint64_t(p->gy.n_in)};
        cuuint64_t strides[1] = {cuuint64_t(d.in_row_stride * 2)};
        cuuint32_t box[2] = {cuuint32_t(kKC), cuuint32_t(kM)};
        cuuint32_t estr[2] = {1, 1};
        const CUtensorMapDataType ty =
            d.in_dtype == RS_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        CUresult r = encode_fn()(&p->stmap, ty, 2, const_cast<void *>(d_in), dims, strides, box, estr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(RS_ERR_CUDA, "tensor-core stream tensor map encoding failed");
        p->stmap_ptr = d_in;
    }
    Params tp = p->tcp;
    tp.out = d_out;
    void *args[2] = {&p->stmap, &tp};
    const cudaError_t e = cudaLaunchKernel(p->s_fn, dim3(p->s_grid), dim3(p->s_block), args, p->s_smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core stream kernel launch");
    return RS_OK;
}

} // namespace tcstream
} // namespace rs
