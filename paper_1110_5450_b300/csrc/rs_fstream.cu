// rs_fstream.cu -- host side of the FP32 streaming downscale (rs_fstream.cuh):
// eligibility, the strips' staged windows and horizontal bands, the vertical
// band table, the work split and the launch.  FP32 plans of 1 or 3 channels
// that downscale both axes, with a 16-byte row pitch, bands of at most 64
// pixels per group of 4 outputs and at most 128 rows per group of 4 output
// rows.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rs_fstream.cuh"
#include "rs_plan.h"

namespace rs {
namespace fstream {
namespace {

template <int C> const void *fn_of() { return reinterpret_cast<const void *>(&fstream_kernel<C>); }

const void *kernel_for(int C) { return C == 1 ? fn_of<1>() : C == 3 ? fn_of<3>() : nullptr; }

// The horizontal band of every (strip, group): at band pixel j (input pixel
// hb + j, hb the group's 4-pixel aligned base) the weights of its 4 outputs,
// zero outside an output's own window and past the image's last output.
// Block (strip, group) fills one band.
__global__ void build_hband_kernel(const int32_t *sx, const float *wx, int t_x, int out_w, int NP, int ngx, int JH,
                                   float4 *hband)
{
    const int s = blockIdx.x, q = blockIdx.y;
    const int j0 = s * NP + 4 * q;
    int st[4], hb = 1 << 30;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        st[g] = j0 + g < out_w ? sx[j0 + g] : -1;
        if (st[g] >= 0) hb = min(hb, st[g]);
    }
    hb = hb == (1 << 30) ? 0 : hb & ~3;
    for (int j = threadIdx.x; j < JH; j += blockDim.x) {
        float w[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int t = hb + j - st[g];
            w[g] = (st[g] >= 0 && t >= 0 && t < t_x) ? wx[size_t(j0 + g) * t_x + t] : 0.f;
        }
        hband[(size_t(s) * ngx + q) * JH + j] = make_float4(w[0], w[1], w[2], w[3]);
    }
}

struct Geometry {
    int C = 0, NP = 0, ngx = 0, n_strips = 0, P = 0, JH = 0, Ty = 0, Uv = 0, gpr = 0;
    std::vector<int32_t> xs, hoff;
};

rs_status geometry(const rs_plan *p, Geometry &g)
{
    const rs_plan_desc &d = p->desc;
    g.C = d.channels;
    if (d.in_dtype != RS_F32 || d.out_dtype != RS_F32 || (g.C != 1 && g.C != 3) || (d.flags & RS_NO_STREAM) ||
        p->prefilter || p->work_double)
        return RS_ERR_UNSUPPORTED;
    if (!tma_layout_ok(p)) return RS_ERR_UNSUPPORTED;
    if (p->gx.n_out >= p->gx.n_in || p->gy.n_out >= p->gy.n_in) return RS_ERR_UNSUPPORTED; // downscales
    g.Ty = p->gy.t_eff;
    if (g.Ty > tcstream::kMaxTy || p->gy.n_in >= (int64_t(1) << 30)) return RS_ERR_UNSUPPORTED;
    const std::vector<int32_t> &sx = p->host_start_x, &sy = p->host_start_y;
    if (int64_t(sx.size()) != p->gx.n_out || int64_t(sy.size()) != p->gy.n_out) return RS_ERR_UNSUPPORTED;
    const int tx = p->gx.t_eff, out_w = int(p->gx.n_out), C = g.C;
    g.NP = kN / C;
    g.ngx = g.NP / 4;
    g.n_strips = (out_w + g.NP - 1) / g.NP;
    // group bases (4-pixel aligned) and the widest band
    std::vector<int32_t> hb(size_t(g.n_strips) * g.ngx, -1);
    int jh = 0;
    for (int s = 0; s < g.n_strips; ++s)
        for (int q = 0; q < g.ngx; ++q) {
            const int j0 = s * g.NP + 4 * q;
            if (j0 >= out_w) continue;
            int lo = sx[size_t(j0)], hi = 0;
            for (int j = j0; j < std::min(out_w, j0 + 4); ++j) {
                lo = std::min(lo, int(sx[size_t(j)]));
                hi = std::max(hi, int(sx[size_t(j)]) + tx);
            }
            lo &= ~3;
            hb[size_t(s) * g.ngx + q] = lo;
            jh = std::max(jh, hi - lo);
        }
    g.JH = (jh + 3) / 4 * 4;
    if (g.JH > kMaxJH) return RS_ERR_UNSUPPORTED;
    // per strip: the first staged sample and the groups' offsets from it
    g.xs.assign(size_t(g.n_strips), 0);
    g.hoff.assign(size_t(g.n_strips) * g.ngx, 0);
    int need = 0;
    for (int s = 0; s < g.n_strips; ++s) {
        int x0 = 1 << 30, x1 = 0;
        for (int q = 0; q < g.ngx; ++q) {
            const int b = hb[size_t(s) * g.ngx + q];
            if (b < 0) continue;
            x0 = std::min(x0, b * C);
            x1 = std::max(x1, (b + g.JH) * C);
        }
        g.xs[size_t(s)] = x0;
        for (int q = 0; q < g.ngx; ++q) {
            const int b = hb[size_t(s) * g.ngx + q];
            g.hoff[size_t(s) * g.ngx + q] = b < 0 ? 0 : b * C - x0; // groups past the image: zero weights
        }
        need = std::max(need, x1 - x0);
    }
    // the row pitch: whole 16-byte words, an odd number of them (lanes on
    // consecutive rows reading 16 bytes hit distinct banks)
    g.P = (need + 3) / 4 * 4;
    if ((g.P / 4) % 2 == 0) g.P += 4;
    if (g.P > kMaxP) return RS_ERR_UNSUPPORTED;
    g.gpr = int((sy.size() + tcstream::kVG - 1) / tcstream::kVG);
    g.Uv = tcstream::vband_rows(sy, g.Ty);
    if (g.Uv > tcstream::kMaxTy) return RS_ERR_UNSUPPORTED;
    return RS_OK;
}

} // namespace

bool eligible(const rs_plan *p)
{
    Geometry g;
    return geometry(p, g) == RS_OK;
}

void preload()
{
    for (const int C : {1, 3})
        if (const void *fn = kernel_for(C)) occupancy(fn, 32 * 13, 0);
}

rs_status rebuild(rs_plan *p, cudaStream_t s)
{
    const Params &fp = p->fsp;
    const dim3 grid(unsigned(fp.n_strips), unsigned(fp.ngx));
    build_hband_kernel<<<grid, 64, 0, s>>>(p->tx.start, static_cast<const float *>(p->tx.wwork), p->gx.t_eff,
                                          fp.out_w, fp.NP, fp.ngx, fp.JH, const_cast<float4 *>(fp.hband));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = tcstream::launch_vband(p, fp.gpr, fp.Uv, const_cast<float4 *>(fp.vband), const_cast<int2 *>(fp.vinfo), s);
    if (e != cudaSuccess) return cuda_fail(e, "FP32 stream band launch");
    return RS_OK;
}

rs_status setup(rs_plan *p, cudaStream_t s, const stream::Opts &o)
{
    p->fs_on = 0;
    Geometry g;
    const rs_status gs = geometry(p, g);
    if (gs != RS_OK) return gs;
    if (p->ext_base) return RS_ERR_UNSUPPORTED; // no external placement of its tables
    const bool forced = o.ex == 3;
    const bool hw_set = forced && o.hw > 0;
    int HW = hw_set ? std::min(kMaxHW, o.hw) : 10;
    const int VW = forced && o.vw > 0 ? std::min(kMaxVW, o.vw) : 6;
    int NA = forced && o.ni_min >= 2 ? std::min(kMaxNA, o.ni_min) : 4;
    if (!hw_set) HW = std::min(HW, kMaxWarps - 1 - VW);
    if (1 + HW + VW > kMaxWarps) return RS_ERR_UNSUPPORTED;
    const void *fn = kernel_for(g.C);
    int nthreads = 32 * (1 + HW + VW);
    int NS = kMaxNS;
    auto fits = [&](int na, int ns) {
        const size_t t = layout(g.P, na, g.Uv, VW, ns).total;
        return t <= 227 * 1024 && occupancy(fn, nthreads, t) >= 1;
    };
    if (!fits(NA, NS)) NS = 2;
    while (NA > 2 && !fits(NA, NS)) --NA;
    if (!fits(NA, NS)) return RS_ERR_UNSUPPORTED;
    if (forced && o.ni_min >= 2 && NA != std::min(kMaxNA, o.ni_min)) return RS_ERR_UNSUPPORTED;
    // a horizontal warp's next task must be at most NA staged blocks ahead
    if (!hw_set) HW = std::min(HW, NA * g.ngx);
    if ((HW + g.ngx - 1) / g.ngx > NA) return RS_ERR_UNSUPPORTED;
    nthreads = 32 * (1 + HW + VW);
    const size_t smem = layout(g.P, NA, g.Uv, VW, NS).total;

    // device tables: strip starts, group offsets, horizontal bands, vertical bands
    Carver cv;
    const size_t o_xs = cv.take(size_t(g.n_strips) * 4);
    const size_t o_ho = cv.take(size_t(g.n_strips) * g.ngx * 4);
    const size_t o_hb = cv.take(size_t(g.n_strips) * g.ngx * g.JH * 16);
    const size_t o_vb = cv.take(size_t(g.gpr) * g.Uv * 16);
    const size_t o_vi = cv.take(size_t(g.gpr) * 8);
    if (p->fsbufs.p) {
        cudaFree(p->fsbufs.p);
        p->fsbufs.p = nullptr;
    }
    cudaError_t e = cudaMalloc(&p->fsbufs.p, cv.off);
    if (e != cudaSuccess) return cuda_fail(e, "allocating FP32 stream tables");
    p->fsbufs.n = cv.off;
    char *base = static_cast<char *>(p->fsbufs.p);
    e = cudaMemcpy(base + o_xs, g.xs.data(), g.xs.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_ho, g.hoff.data(), g.hoff.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "uploading FP32 stream strip tables");

    const rs_plan_desc &d = p->desc;
    Params &fp = p->fsp;
    std::memset(&fp, 0, sizeof fp);
    fp.in_h = int32_t(p->gy.n_in);
    fp.out_h = int32_t(p->gy.n_out);
    fp.out_w = int32_t(p->gx.n_out);
    fp.C = g.C;
    fp.out_stride = d.out_row_stride;
    fp.sy = p->ty.start;
    fp.vband = reinterpret_cast<const float4 *>(base + o_vb);
    fp.vinfo = reinterpret_cast<const int2 *>(base + o_vi);
    fp.NP = g.NP;
    fp.n_strips = g.n_strips;
    fp.Ty = g.Ty;
    fp.Uv = g.Uv;
    fp.gpr = g.gpr;
    fp.NS = NS;
    fp.NA = NA;
    fp.VW = VW;
    fp.HW = HW;
    const int64_t total = int64_t(g.n_strips) * g.gpr;
    fp.per_cta = std::max<int64_t>((total + p->num_sms - 1) / p->num_sms, std::min<int64_t>(4, g.gpr));
    fp.err = p->d_err;
    fp.xs = reinterpret_cast<const int32_t *>(base + o_xs);
    fp.hoff = reinterpret_cast<const int32_t *>(base + o_ho);
    fp.hband = reinterpret_cast<const float4 *>(base + o_hb);
    fp.P = g.P;
    fp.JH = g.JH;
    fp.ngx = g.ngx;
    p->fs_on = 1;
    p->x_on = 0;
    p->tcs_on = 0;
    const rs_status st = rebuild(p, s);
    if (st != RS_OK) {
        p->fs_on = 0;
        return st;
    }
    p->s_fn = fn;
    p->s_block = nthreads;
    p->s_smem = smem;
    p->s_grid = int((total + fp.per_cta - 1) / fp.per_cta);
    p->s_ctas = 1;
    p->stmap_ptr = nullptr;
    stream::Opts used;
    used.ex = 3;
    used.hw = HW;
    used.ni_min = NA;
    used.vw = VW;
    used.sw = g.NP;
    p->stream_code = used.code();
    p->stream_ok = 1;
    return RS_OK;
}

rs_status launch(rs_plan *p, const void *d_in, void *d_out, cudaStream_t s)
{
    const rs_plan_desc &d = p->desc;
    if (p->stmap_ptr != d_in) {
        // boxes of P samples x 32 rows, rows P samples apart in shared memory
        cuuint64_t dims[2] = {cuuint64_t(p->gx.n_in * d.channels), cuuint64_t(p->gy.n_in)};
        cuuint64_t strides[1] = {cuuint64_t(d.in_row_stride * 4)};
        cuuint32_t box[2] = {cuuint32_t(p->fsp.P), cuuint32_t(kSB)};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = encode_fn()(&p->stmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(d_in), dims,
                                 strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(RS_ERR_CUDA, "FP32 stream tensor map encoding failed");
        p->stmap_ptr = d_in;
    }
    Params fp = p->fsp;
    fp.out = d_out;
    void *args[2] = {&p->stmap, &fp};
    const cudaError_t e = cudaLaunchKernel(p->s_fn, dim3(p->s_grid), dim3(p->s_block), args, p->s_smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "FP32 stream kernel launch");
    return RS_OK;
}

} // namespace fstream
} // namespace rs
