// rs_stream.cu -- host side of the row-streaming kernel (rs_stream.cuh): its
// band tables, configuration, tensor map and launch.  Used by FP32, FP16 and
// BF16 plans of 1 or 3 channels whose horizontal band is narrow (upscales and
// downscales to about x0.3); every other plan runs the tile kernel.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rs_plan.h"
#include "rs_stream.cuh"

namespace rs {
namespace stream {
namespace {

// Vertical band widths the kernels are instantiated for (rs_stream.cuh).
constexpr int kJV8[] = {8, 10, 12, 14, 16};
constexpr int kJV4[] = {4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32};

const void *kernel_for(int dtype, int C, int jv, int gv, bool ws, bool multi = false)
{
    switch (dtype) {
    case RS_F32: return kernel_f32(C, jv, gv, ws, multi);
    case RS_F16: return kernel_f16(C, jv, gv, ws, multi);
    case RS_BF16: return kernel_bf16(C, jv, gv, ws, multi);
    }
    return nullptr;
}

} // namespace

const void *multi_kernel(const rs_plan *p)
{
    if (!p->stream_ok || p->x_on || p->tcs_on) return nullptr;
    return kernel_for(p->desc.in_dtype, p->desc.channels, p->sp.JV, p->sp.GV, p->sp.NW != 0, true);
}

void preload(int dtype)
{
    for (const int C : {1, 3})
        for (const bool ws : {false, true}) {
            for (const int jv : kJV8)
                if (const void *fn = kernel_for(dtype, C, jv, 8, ws)) occupancy(fn, kThreads, 0);
            for (const int jv : kJV4)
                if (const void *fn = kernel_for(dtype, C, jv, 4, ws)) occupancy(fn, kThreads, 0);
        }
}

namespace {

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

// Staged pitch >= n samples: a whole number of 16-byte words per row (TMA),
// odd in 16-byte words so that lanes on consecutive rows reading 16 bytes
// (FP32) hit distinct banks; 16-bit rows are read 8 bytes at a time and meet
// 2-way conflicts at best.
int pad_pitch(int n, int es)
{
    const int u = 16 / es; // samples per 16-byte word
    int p = (n + u - 1) / u * u;
    if ((p / u) % 2 == 0) p += u;
    return p;
}

struct Strip {
    int sw, P, offB, Q, NI, NW, HR, occ, ppr;
    size_t smem;
    double cost;
};

// Every strip width (multiple of 4 outputs, at most 128; 252 for one channel) whose staged width
// fits the TMA boxes and whose CTA keeps two CTAs per SM, for the first
// staging form that admits any: the warp-specialised kernel first (its
// filtered-row ring holds two blocks), then narrow strips with >= ni_min
// staged blocks, wide strips (two boxes per block: the second starts early
// enough that every group's band fits one of them), narrow with 2 blocks.
// Each gets its row ranges and a modelled time: whole waves of CTAs, each
// CTA's work (strip width plus a fixed share worth 64 outputs -- the
// per-block barriers, waits and task rounding, fitted to measured widths --
// times the rows of its range plus the band and the pipeline fill); cheapest
// first.
} // namespace

// Row-range counts worth modelling: the cost of a configuration depends on
// its waves of CTAs (or CTAs per SM) and on its rows per range, which fall as
// ranges are added, so for each count of waves only the largest range count
// that still fits it can be best; plus the first few counts.  Beyond a few
// waves more ranges only trade rows for waves one for one while adding each
// range's pipeline fill, so waves stop at 8 (which also keeps the search
// cheap enough for a server to run per request).  Ascending.
std::vector<int> range_counts(int n_strips, int64_t slots, int max_nr)
{
    std::vector<int> c;
    for (int nr = 1; nr <= 8 && nr <= max_nr; ++nr) c.push_back(nr);
    for (int64_t w = 1; w <= 8; ++w) {
        const int64_t v = w * slots / std::max(1, n_strips);
        for (int64_t x = v - 1; x <= v + 1; ++x)
            if (x >= 1 && x <= max_nr) c.push_back(int(x));
    }
    std::sort(c.begin(), c.end());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    return c;
}

namespace {

std::vector<Strip> strips(rs_plan *p, const Opts &opts_in, int C, int groups_x, const std::vector<int32_t> &hb,
                          int JH, int JV, int GV, int WP, const std::vector<int32_t> &vb, int pairs)
{
    const int dtype = p->desc.in_dtype, es = dt_size(dtype);
    // unless the caller fixes the form: groups of 8 rows (narrow vertical
    // bands) run the phase-alternating kernel with 2 staged blocks, groups of
    // 4 (wide bands) the warp-specialised one -- the faster form of each as
    // measured on 4096x4096x3 at x1.37 and x0.3
    Opts opts = opts_in;
    const int first = opts.ws >= 0 ? opts.ws : (GV == 8 ? 0 : 1);
    if (opts.ws < 0 && GV == 8) opts.ni_min = std::min(opts.ni_min, 2);
    std::vector<Strip> out;
    const int M = JV - 1;
    for (int i = 0; i < 2 && out.empty(); ++i) {
        const int ws = i == 0 ? first : 1 - first;
        if (i == 1 && opts.ws >= 0) break; // a fixed form has no fallback
        const int hr = (ws ? 2 : 1) * kRB + JV;
        for (int pass = 0; pass < 3 && out.empty(); ++pass)
            for (int sw = C == 1 ? 252 : 128; sw >= 16; sw -= 4) {
                const int ngx = sw / kG;
                int need = 0;
                for (int g0 = 0; g0 < groups_x; g0 += ngx) {
                    const int gl = std::min(groups_x, g0 + ngx) - 1;
                    // (16-bit boxes start up to 4 samples before the first band)
                    need = std::max(need, (hb[gl] + JH - hb[g0]) * C + (es == 2 ? 4 : 0));
                }
                int pp = 0, ob = 0;
                if (pass != 1) {
                    pp = pad_pitch(need, es);
                    if (pp > 256) pp = 0;
                } else {
                    // boxes A = [0, P) and B = [ob, ob + P) of the strip's samples:
                    // ob <= P - JH C (overlap of a band) and ob + P >= need
                    const int u = 16 / es;
                    for (int cand = pad_pitch((need + JH * C + 1) / 2, es); cand <= 256 && !pp; cand += 2 * u) {
                        const int o = (cand - JH * C) / u * u;
                        if (o > 0 && o + cand >= need) {
                            pp = cand;
                            ob = o;
                        }
                    }
                }
                if (pp == 0) continue;
                const int qq = (hr + M) | 1; // odd: the vertical pass's 16-byte loads are conflict-free
                for (int ni = kMaxNI; ni >= 2; --ni) {
                    const size_t t = ws ? layout_ws(ni, 2, pp, qq, sw * C / 4, ngx, JH, WP, JV, ob != 0, GV, es).total
                                        : layout(ni, pp, qq, sw * C / 4, ngx, JH, WP, JV, ob != 0, GV, es).total;
                    if (t <= 113 * 1024 && (ni >= opts.ni_min || pass > 0)) {
                        out.push_back({sw, pp, ob, qq, ni, ws ? 2 : 0, hr, 0, 0, t, 0.0});
                        break;
                    }
                }
            }
    }
    auto blocks_ok = [&](int ppr) {
        for (int q0 = 0; q0 < pairs; q0 += ppr) {
            const int q1 = std::min(pairs, q0 + ppr) - 1;
            if ((vb[q1] + JV - vb[q0] + kRB - 1) / kRB > kMaxBlk) return false;
        }
        return true;
    };
    std::vector<Strip> ok;
    for (Strip c : out) {
        const void *fn = kernel_for(dtype, C, JV, GV, c.NW != 0);
        c.occ = rs::occupancy(fn, kThreads, c.smem);
        if (c.occ < 1) continue;
        const int n_strips = (groups_x + c.sw / kG - 1) / (c.sw / kG);
        const int64_t slots = int64_t(c.occ) * p->num_sms;
        c.cost = 1e300;
        for (const int nr : range_counts(n_strips, slots, 1024)) {
            const int cand = (pairs + nr - 1) / nr;
            if (cand < 8 && nr > 1) break;
            if (!blocks_ok(cand)) continue;
            const int ranges = (pairs + cand - 1) / cand;
            int rows = 0;
            for (int q0 = 0; q0 < pairs; q0 += cand) {
                const int q1 = std::min(pairs, q0 + cand) - 1;
                rows = std::max(rows, vb[q1] + JV - vb[q0]);
            }
            const int64_t grid = int64_t(n_strips) * ranges;
            const int64_t waves = (grid + slots - 1) / slots;
            const double cost = double(waves) * (c.sw + 64) * (rows + 2 * kRB);
            if (cost < c.cost * 0.999) {
                c.cost = cost;
                c.ppr = cand;
            }
            if (ranges >= pairs) break;
        }
        if (c.ppr) ok.push_back(c);
    }
    std::stable_sort(ok.begin(), ok.end(), [](const Strip &a, const Strip &b) { return a.cost < b.cost; });
    return ok;
}

// The plan's bands for the streaming kernel: 4-pixel aligned horizontal
// group bases and taps, the vertical group size, taps and row bases, and the
// most groups whose last row falls in one 32-row block.
struct Bands {
    int C = 0, groups_x = 0, JH = 0, GV = 8, JV = 0, pairs = 0, WP = 0;
    std::vector<int32_t> hb, vb;
};

rs_status bands_of(const rs_plan *p, Bands &b)
{
    const rs_plan_desc &d = p->desc;
    b.C = d.channels;
    if ((d.in_dtype != RS_F32 && d.in_dtype != RS_F16 && d.in_dtype != RS_BF16) || d.out_dtype != d.in_dtype ||
        (b.C != 1 && b.C != 3) || (d.flags & RS_NO_STREAM))
        return RS_ERR_UNSUPPORTED;
    if (!tma_layout_ok(p)) return RS_ERR_UNSUPPORTED;
    const std::vector<int32_t> &sx = p->host_start_x, &sy = p->host_start_y;
    const AxisGeom &gx = p->gx, &gy = p->gy;
    b.groups_x = int((gx.n_out + kG - 1) / kG);
    b.hb.assign(b.groups_x, 0);
    int JH = 0;
    for (int q = 0; q < b.groups_x; ++q) {
        int lo = int(gx.n_in), hi = 0;
        for (int m = 0; m < kG && q * kG + m < gx.n_out; ++m) {
            lo = std::min(lo, int(sx[q * kG + m]));
            hi = std::max(hi, int(sx[q * kG + m]) + gx.t_eff);
        }
        b.hb[q] = lo & ~3;
        JH = std::max(JH, hi - b.hb[q]);
    }
    b.JH = (JH + 3) / 4 * 4;
    // vertical band (the tile kernel's band code): groups of 8 rows while the
    // band stays within 16 taps, else groups of 4
    b.GV = 8;
    b.JV = vertical_taps(sy, gy.t_eff, 8);
    if (b.JV == 0) {
        b.GV = 4;
        b.JV = vertical_taps(sy, gy.t_eff, 4);
    }
    if (b.JH > 40 || b.JV == 0 || b.JV > gy.n_in) return RS_ERR_UNSUPPORTED;
    const int GV = b.GV, JV = b.JV;
    b.pairs = int((gy.n_out + GV - 1) / GV);
    b.vb.assign(b.pairs, 0);
    for (int q = 0; q < b.pairs; ++q) {
        int lo = sy[GV * q];
        for (int r = 1; r < GV && GV * q + r < int(sy.size()); ++r) lo = std::min(lo, int(sy[GV * q + r]));
        b.vb[q] = gy.n_in >= JV ? std::min<int64_t>(lo, gy.n_in - JV) : 0;
    }
    int WP = 0;
    for (int a = 0, e = 0; a < b.pairs; ++a) {
        while (e < b.pairs && b.vb[e] + JV <= b.vb[a] + JV + kRB - 1) ++e;
        WP = std::max(WP, e - a);
    }
    b.WP = std::max(WP, 1);
    return RS_OK;
}

} // namespace

int widths(rs_plan *p, const Opts &opts, int *out, int n)
{
    if (opts.ex == 2) {
        if (!tcstream::eligible(p) || n < 1) return 0;
        out[0] = tcstream::kN / p->desc.channels; // one strip width
        return 1;
    }
    if (opts.ex > 0) return xstream::widths(p, opts, out, n);
    Bands b;
    if (bands_of(p, b) != RS_OK) return 0;
    const std::vector<Strip> c = strips(p, opts, b.C, b.groups_x, b.hb, b.JH, b.JV, b.GV, b.WP, b.vb, b.pairs);
    int k = 0;
    for (; k < n && k < int(c.size()); ++k) out[k] = c[k].sw;
    return k;
}

rs_status setup(rs_plan *p, cudaStream_t s, const Opts &opts)
{
    p->stream_ok = 0;
    if (opts.ex == 2) return tcstream::setup(p, s, opts);
    // the exact-window form where it applies (or when asked for)
    if (opts.ex != 0) {
        const rs_status xs = xstream::setup(p, s, opts);
        if (xs == RS_OK || opts.ex > 0) return xs;
        // then the tensor-core downscale where it applies and the horizontal
        // windows are wide (12 or more taps: it was measured slower than the
        // band kernels at x0.6 Lanczos-3, 10 taps, and 1.6-2.8x faster at
        // x0.3 and x0.125)
        if (p->gx.t_eff >= 12) {
            const rs_status ts = tcstream::setup(p, s, opts);
            if (ts != RS_ERR_UNSUPPORTED) return ts;
        }
    }
    p->x_on = 0;
    p->tcs_on = 0;
    Bands bd;
    const rs_status bst = bands_of(p, bd);
    if (bst != RS_OK) return bst;
    const rs_plan_desc &d = p->desc;
    const AxisGeom &gx = p->gx, &gy = p->gy;
    const int C = bd.C, groups_x = bd.groups_x, JH = bd.JH, GV = bd.GV, JV = bd.JV, pairs = bd.pairs, WP = bd.WP;
    const std::vector<int32_t> &hb = bd.hb, &vb = bd.vb;
    std::vector<Strip> cands = strips(p, opts, C, groups_x, hb, JH, JV, GV, WP, vb, pairs);
    if (cands.empty()) return RS_ERR_UNSUPPORTED;
    const Strip *pick = &cands[0];
    if (opts.sw > 0) {
        pick = nullptr;
        for (const Strip &c : cands)
            if (c.sw == opts.sw) pick = &c;
        if (!pick) return RS_ERR_UNSUPPORTED;
    }
    const int SW = pick->sw, P = pick->P, offB = pick->offB, Q = pick->Q, NI = pick->NI, NW = pick->NW,
              HR = pick->HR, M = JV - 1, occ = pick->occ, ppr = pick->ppr;
    const size_t smem = pick->smem;
    const int ngx = SW / kG;
    const int n_strips = (groups_x + ngx - 1) / ngx;
    const void *fn = kernel_for(d.in_dtype, C, JV, GV, NW != 0);
    cudaError_t e = cudaSuccess;

    // device tables: horizontal base + band, vertical base + band
    Carver cv;
    const size_t o_hb = cv.take(size_t(groups_x) * 4);
    const size_t o_hw = cv.take(size_t(groups_x) * JH * kG * 4);
    const size_t o_vb = cv.take(size_t((pairs + 3) & ~3) * 4); // the kernel copies whole 16-byte words
    const size_t o_vw = cv.take(size_t(pairs) * JV * vtap_floats(GV) * 4);
    char *base = nullptr;
    if (p->ext_base) {
        if (cv.off > p->ext_bytes) return fail(RS_ERR_BUDGET, "streaming tables exceed their reserved space");
        base = p->ext_base;
    } else {
        if (p->sbufs.p) {
            cudaFree(p->sbufs.p);
            p->sbufs.p = nullptr;
        }
        e = cudaMalloc(&p->sbufs.p, cv.off);
        if (e != cudaSuccess) return cuda_fail(e, "allocating stream tables");
        p->sbufs.n = cv.off;
        base = static_cast<char *>(p->sbufs.p);
    }
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
        used.sw = SW;
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
    p->s_block = kThreads;
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
    if (p->tcs_on) return tcstream::rebuild(p, s);
    if (p->x_on) return RS_OK; // the exact-window kernel reads the weight tables directly
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

rs_status encode_input_map(const rs_plan *p, const void *d_in, CUtensorMap *map)
{
    const rs_plan_desc &d = p->desc;
    cuuint64_t dims[2] = {cuuint64_t(p->gx.n_in * d.channels), cuuint64_t(p->gy.n_in)};
    const int es = dt_size(d.in_dtype);
    cuuint64_t strides[1] = {cuuint64_t(d.in_row_stride * es)};
    cuuint32_t box[2] = {cuuint32_t(p->x_on ? p->xp.P : p->sp.P), cuuint32_t(kRB)};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType ty = d.in_dtype == RS_F16    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : d.in_dtype == RS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = encode_fn()(map, ty, 2, const_cast<void *>(d_in), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(RS_ERR_CUDA, "stream tensor map encoding failed");
    return RS_OK;
}

rs_status launch(rs_plan *p, const void *d_in, void *d_out, cudaStream_t s)
{
    if (p->tcs_on) return tcstream::launch(p, d_in, d_out, s);
    if (p->stmap_ptr != d_in) {
        const rs_status st = encode_input_map(p, d_in, &p->stmap);
        if (st != RS_OK) return st;
        p->stmap_ptr = d_in;
    }
    Params sp = p->sp;
    sp.in = d_in;
    sp.out = d_out;
    xstream::Params xp = p->xp;
    xp.in = d_in;
    xp.out = d_out;
    void *args[2] = {&p->stmap, p->x_on ? static_cast<void *>(&xp) : static_cast<void *>(&sp)};
    cudaError_t e = cudaLaunchKernel(p->s_fn, dim3(p->s_grid), dim3(p->x_on ? p->s_block : kThreads), args, p->s_smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "stream kernel launch");
    return RS_OK;
}

} // namespace stream
} // namespace rs
