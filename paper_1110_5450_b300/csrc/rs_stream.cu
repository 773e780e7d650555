// rs_stream.cu -- host side of the row-streaming kernel (rs_stream.cuh): its
// band tables, configuration, tensor map and launch.  Used by FP32 plans of 1
// or 3 channels whose horizontal band is narrow (upscales and mild
// downscales); every other plan runs the tile kernel.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rs_plan.h"
#include "rs_stream.cuh"

namespace rs {
namespace stream {
namespace {

// Instantiated kernels: channels x vertical taps x rows per vertical group (a
// plan's band is padded with zero weights to the next instantiated width):
// groups of 8 rows up to 16 taps, groups of 4 rows up to 32.
constexpr int kJV8[] = {8, 10, 12, 14, 16};
constexpr int kJV4[] = {4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32};

template <int C, int JV, int GV> const void *kernel_of(bool ws)
{
    return ws ? reinterpret_cast<const void *>(&stream_ws_kernel<C, JV, GV>)
              : reinterpret_cast<const void *>(&stream_kernel<C, JV, GV>);
}

template <int C, int GV> const void *kernel_jv(int jv, bool ws)
{
    switch (jv) {
    case 4: return GV == 4 ? kernel_of<C, 4, 4>(ws) : nullptr;
    case 6: return GV == 4 ? kernel_of<C, 6, 4>(ws) : nullptr;
    case 8: return kernel_of<C, 8, GV>(ws);
    case 10: return kernel_of<C, 10, GV>(ws);
    case 12: return kernel_of<C, 12, GV>(ws);
    case 14: return kernel_of<C, 14, GV>(ws);
    case 16: return kernel_of<C, 16, GV>(ws);
    case 20: return GV == 4 ? kernel_of<C, 20, 4>(ws) : nullptr;
    case 24: return GV == 4 ? kernel_of<C, 24, 4>(ws) : nullptr;
    case 28: return GV == 4 ? kernel_of<C, 28, 4>(ws) : nullptr;
    case 32: return GV == 4 ? kernel_of<C, 32, 4>(ws) : nullptr;
    }
    return nullptr;
}

const void *kernel_for(int C, int jv, int gv, bool ws)
{
    if (C == 1) return gv == 8 ? kernel_jv<1, 8>(jv, ws) : kernel_jv<1, 4>(jv, ws);
    if (C == 3) return gv == 8 ? kernel_jv<3, 8>(jv, ws) : kernel_jv<3, 4>(jv, ws);
    return nullptr;
}

// Vertical taps of groups of GV output rows, rounded up to an instantiated
// width (0 if none is wide enough).
int vertical_taps(const std::vector<int32_t> &sy, int t_eff, int GV)
{
    int J = 0;
    for (size_t i = 0; i < sy.size(); i += GV) {
        int lo = sy[i], hi = sy[i] + t_eff;
        for (size_t r = 1; r < size_t(GV) && i + r < sy.size(); ++r) {
            lo = std::min(lo, int(sy[i + r]));
            hi = std::max(hi, int(sy[i + r]) + t_eff);
        }
        J = std::max(J, hi - lo);
    }
    if (GV == 8) {
        for (int c : kJV8)
            if (c >= J) return c;
    } else {
        for (int c : kJV4)
            if (c >= J) return c;
    }
    return 0;
}

int pad_pitch(int n) // multiple of 4 with n / 4 odd, >= n
{
    int p = (n + 3) / 4 * 4;
    if ((p / 4) % 2 == 0) p += 4;
    return p;
}

} // namespace

rs_status setup(rs_plan *p, cudaStream_t s, const Opts &opts)
{
    p->stream_ok = 0;
    const rs_plan_desc &d = p->desc;
    const int C = d.channels;
    if (d.in_dtype != RS_F32 || (C != 1 && C != 3) || (d.flags & RS_NO_STREAM)) return RS_ERR_UNSUPPORTED;
    if (!tma_layout_ok(p)) return RS_ERR_UNSUPPORTED;
    const std::vector<int32_t> &sx = p->host_start_x, &sy = p->host_start_y;
    const AxisGeom &gx = p->gx, &gy = p->gy;
    // horizontal band: 4-pixel aligned group bases
    const int groups_x = int((gx.n_out + kG - 1) / kG);
    std::vector<int32_t> hb(groups_x);
    int JH = 0;
    for (int q = 0; q < groups_x; ++q) {
        int lo = int(gx.n_in), hi = 0;
        for (int m = 0; m < kG && q * kG + m < gx.n_out; ++m) {
            lo = std::min(lo, int(sx[q * kG + m]));
            hi = std::max(hi, int(sx[q * kG + m]) + gx.t_eff);
        }
        hb[q] = lo & ~3;
        JH = std::max(JH, hi - hb[q]);
    }
    JH = (JH + 3) / 4 * 4;
    // vertical band (the tile kernel's band code): groups of 8 rows while the
    // band stays within 16 taps, else groups of 4
    int GV = 8, JV = vertical_taps(sy, gy.t_eff, 8);
    if (JV == 0) {
        GV = 4;
        JV = vertical_taps(sy, gy.t_eff, 4);
    }
    if (JH > 40 || JV == 0 || JV > gy.n_in) return RS_ERR_UNSUPPORTED;
    // row bases of the groups (as the band kernel computes them) and the most
    // groups whose last row falls in one 32-row block
    const int pairs = int((gy.n_out + GV - 1) / GV);
    std::vector<int32_t> vb(pairs);
    for (int q = 0; q < pairs; ++q) {
        int lo = sy[GV * q];
        for (int r = 1; r < GV && GV * q + r < int(sy.size()); ++r) lo = std::min(lo, int(sy[GV * q + r]));
        vb[q] = gy.n_in >= JV ? std::min<int64_t>(lo, gy.n_in - JV) : 0;
    }
    int WP = 0;
    for (int a = 0, b = 0; a < pairs; ++a) {
        while (b < pairs && vb[b] + JV <= vb[a] + JV + kRB - 1) ++b;
        WP = std::max(WP, b - a);
    }
    WP = std::max(WP, 1);
    // the widest strip (multiple of 4 outputs, at most 128) whose staged width
    // fits the TMA boxes and whose CTA keeps two CTAs per SM; the warp-
    // specialised kernel first (its filtered-row ring holds two blocks)
    int SW = 0, P = 0, offB = 0, Q = 0, NI = 0, NW = 0, HR = 0, M = JV - 1;
    size_t smem = 0;
    for (int ws = 1; ws >= 0 && SW == 0; --ws) {
    if (opts.ws >= 0 && ws != opts.ws) continue;
    const int hr = (ws ? 2 : 1) * kRB + JV;
    // narrow strips (one box per block, three staged blocks) where one fits;
    // else wide strips (two boxes per block: the second starts early enough
    // that every group's band fits one of them)
    // (passes: narrow with >= 3 staged blocks, wide, narrow with 2 blocks)
    for (int pass = 0; pass < 3 && SW == 0; ++pass)
    for (int sw = 128; sw >= 16 && SW == 0; sw -= 4) {
        const int ngx = sw / kG;
        int need = 0;
        for (int g0 = 0; g0 < groups_x; g0 += ngx) {
            const int gl = std::min(groups_x, g0 + ngx) - 1;
            need = std::max(need, (hb[gl] + JH - hb[g0]) * C);
        }
        int pp = 0, ob = 0;
        if (pass != 1) {
            pp = pad_pitch(need);
            if (pp > 256) pp = 0;
        } else {
            // boxes A = [0, P) and B = [ob, ob + P) of the strip's samples:
            // ob <= P - JH C (overlap of a band) and ob + P >= need
            for (int cand = pad_pitch((need + JH * C + 1) / 2); cand <= 256 && !pp; cand += 8) {
                const int o = (cand - JH * C) / 4 * 4;
                if (o > 0 && o + cand >= need) {
                    pp = cand;
                    ob = o;
                }
            }
        }
        if (pp == 0) continue;
        const int qq = (hr + M) | 1; // odd: the vertical pass's 16-byte loads are conflict-free
        for (int ni = kMaxNI; ni >= 2; --ni) {
            const size_t t = ws ? layout_ws(ni, 2, pp, qq, sw * C / 4, ngx, JH, WP, JV, ob != 0, GV).total
                                : layout(ni, pp, qq, sw * C / 4, ngx, JH, WP, JV, ob != 0, GV).total;
            if (t <= 113 * 1024 && (ni >= opts.ni_min || pass > 0)) {
                SW = sw;
                P = pp;
                offB = ob;
                Q = qq;
                NI = ni;
                NW = ws ? 2 : 0;
                HR = hr;
                smem = t;
                break;
            }
        }
    }
    }
    if (SW == 0) return RS_ERR_UNSUPPORTED;
    const int ngx = SW / kG;
    const void *fn = kernel_for(C, JV, GV, NW != 0);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return cuda_fail(e, "setting shared memory size");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (occ < 1) return RS_ERR_UNSUPPORTED;
    // row ranges: enough CTAs for whole waves (>= 90% of the last wave busy),
    // each range within the kernel's per-CTA block budget
    const int n_strips = (groups_x + ngx - 1) / ngx;
    const int slots = occ * p->num_sms;
    auto blocks_ok = [&](int ppr) {
        for (int q0 = 0; q0 < pairs; q0 += ppr) {
            const int q1 = std::min(pairs, q0 + ppr) - 1;
            if ((vb[q1] + JV - vb[q0] + kRB - 1) / kRB > kMaxBlk) return false;
        }
        return true;
    };
    int ppr = 0;
    for (int nr = 1; nr <= 1024; ++nr) {
        const int cand = (pairs + nr - 1) / nr;
        if (cand < 8 && nr > 1 && ppr) break;
        if (!blocks_ok(cand)) continue;
        const int64_t grid = int64_t(n_strips) * ((pairs + cand - 1) / cand);
        const int64_t waves = (grid + slots - 1) / slots;
        ppr = cand;
        if (grid >= slots && double(grid) / double(waves * slots) >= 0.9) break;
    }
    if (ppr == 0) return RS_ERR_UNSUPPORTED;

    // device tables: horizontal base + band, vertical base + band
    Carver cv;
    const size_t o_hb = cv.take(size_t(groups_x) * 4);
    const size_t o_hw = cv.take(size_t(groups_x) * JH * kG * 4);
    const size_t o_vb = cv.take(size_t((pairs + 3) & ~3) * 4); // the kernel copies whole 16-byte words
    const size_t o_vw = cv.take(size_t(pairs) * JV * vtap_floats(GV) * 4);
    if (p->sbufs.p) {
        cudaFree(p->sbufs.p);
        p->sbufs.p = nullptr;
    }
    e = cudaMalloc(&p->sbufs.p, cv.off);
    if (e != cudaSuccess) return cuda_fail(e, "allocating stream tables");
    p->sbufs.n = cv.off;
    char *base = static_cast<char *>(p->sbufs.p);
    Params &sp = p->sp;
    std::memset(&sp, 0, sizeof sp);
    sp.in_h = gy.n_in;
    sp.in_w = gx.n_in;
    sp.out_h = gy.n_out;
    sp.out_w = gx.n_out;
    sp.in_stride = d.in_row_stride;
    sp.out_stride = d.out_row_stride;
    sp.hbase = reinterpret_cast<const int32_t *>(base + o_hb);
    sp.hband = reinterpret_cast<const float *>(base + o_hw);
    sp.vbase = reinterpret_cast<const int32_t *>(base + o_vb);
    sp.vband = reinterpret_cast<const float *>(base + o_vw);
    sp.JH = JH;
    sp.JV = JV;
    sp.SW = SW;
    sp.n_strips = n_strips;
    sp.pairs = pairs;
    sp.pairs_per_range = ppr;
    sp.groups_x = groups_x;
    sp.P = P;
    sp.offB = offB;
    sp.Q = Q;
    sp.NI = NI;
    sp.NW = NW;
    sp.HW = opts.hw > 0 ? std::min(6, std::max(2, opts.hw)) : 4;
    {
        Opts used = opts;
        used.ws = NW ? 1 : 0;
        used.hw = NW ? sp.HW : 0;
        p->stream_code = used.code();
    }
    sp.HR = HR;
    sp.M = M;
    sp.WP = WP;
    sp.GV = GV;
    sp.err = p->d_err;
    rs_status st = rebuild(p, s);
    if (st != RS_OK) return st;
    p->s_fn = fn;
    p->s_smem = smem;
    p->s_grid = n_strips * ((pairs + ppr - 1) / ppr);
    p->s_ctas = occ;
    p->stmap_ptr = nullptr;
    p->stream_ok = 1;
    p->scratch_bytes = int64_t(p->tables.n + p->bands.n + p->tmp.n + p->sbufs.n);
    return RS_OK;
}

rs_status rebuild(rs_plan *p, cudaStream_t s)
{
    // both bands in one launch of the band kernel:
    //  * vertical: groups of 4 rows, every weight twice -> per tap (w0, w0, .., w3, w3);
    //  * horizontal: groups of 4 outputs, 4-pixel aligned bases, per pixel (w0, .., w3)
    const Params &sp = p->sp;
    AxisTables vt = p->ty;
    vt.G = sp.GV;
    vt.J = sp.JV;
    vt.groups = sp.pairs;
    vt.dup = sp.GV == 4 ? 2 : 1; // groups of 4 rows: every weight twice (packed FMAs)
    vt.pair_ngx = 0;
    vt.align = 0;
    vt.band_base = const_cast<int32_t *>(sp.vbase);
    vt.band_w = const_cast<float *>(sp.vband);
    AxisTables ht = p->tx;
    ht.G = kG;
    ht.J = sp.JH;
    ht.groups = sp.groups_x;
    ht.dup = 1;
    ht.pair_ngx = 0;
    ht.align = 4;
    ht.band_base = const_cast<int32_t *>(sp.hbase);
    ht.band_w = const_cast<float *>(sp.hband);
    WeightArgs a0, a1;
    a0.g = p->gy;
    a0.t = vt;
    a1.g = p->gx;
    a1.t = ht;
    a0.work_is_double = a1.work_is_double = 0;
    a0.err = a1.err = p->d_err;
    const cudaError_t e = launch_band(a0, a1, s);
    if (e != cudaSuccess) return cuda_fail(e, "stream band launch");
    return RS_OK;
}

rs_status launch(rs_plan *p, const void *d_in, void *d_out, cudaStream_t s)
{
    const rs_plan_desc &d = p->desc;
    if (p->stmap_ptr != d_in) {
        cuuint64_t dims[2] = {cuuint64_t(p->gx.n_in * d.channels), cuuint64_t(p->gy.n_in)};
        cuuint64_t strides[1] = {cuuint64_t(d.in_row_stride * 4)};
        cuuint32_t box[2] = {cuuint32_t(p->sp.P), cuuint32_t(kRB)};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = encode_fn()(&p->stmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(d_in), dims,
                                 strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(RS_ERR_CUDA, "stream tensor map encoding failed");
        p->stmap_ptr = d_in;
    }
    Params sp = p->sp;
    sp.in = static_cast<const float *>(d_in);
    sp.out = static_cast<float *>(d_out);
    void *args[2] = {&p->stmap, &sp};
    cudaError_t e = cudaLaunchKernel(p->s_fn, dim3(p->s_grid), dim3(kThreads), args, p->s_smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "stream kernel launch");
    return RS_OK;
}

} // namespace stream
} // namespace rs
