// rs_xstream.cu -- host side of the pipelined streaming kernel
// (rs_xstream.cuh): eligibility, the group descriptors, strip and row-range
// choice, launch parameters.  Used by FP32, FP16 and BF16 plans of 1 or 3
// channels that upscale (or keep) both axes with 4 or 6 taps per output
// (cubic, Mitchell-Netravali, Lanczos-2, Lanczos-3, B-spline); the launch
// itself goes through the row-streaming path's tensor map (rs_stream.cu).
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "rs_plan.h"
#include "rs_xstream.cuh"

namespace rs {
namespace xstream {
namespace {

const void *kernel_for(int dtype, int C, int taps, int big)
{
    switch (dtype) {
    case RS_F32: return kernel_f32(C, taps, big);
    case RS_F16: return kernel_f16(C, taps, big);
    case RS_BF16: return kernel_bf16(C, taps, big);
    }
    return nullptr;
}

} // namespace

void preload(int dtype)
{
    for (const int C : {1, 3})
        for (const int taps : {4, 6})
            for (const int big : {0, 1})
                if (const void *fn = kernel_for(dtype, C, taps, big))
                    occupancy(fn, 32 * (big ? kMaxWarps : kSmallWarps), 0);
}

const void *multi_kernel(const rs_plan *p)
{
    if (!p->x_on) return nullptr;
    const int big = p->s_block > 32 * kSmallWarps ? 1 : 0;
    // blocks of at most kMidWarps warps: the variant with the higher register cap
    if (!big && p->s_block <= 32 * kMidWarps)
        return kernel_for(p->desc.in_dtype, p->desc.channels, int(p->gx.t_eff), 4);
    return kernel_for(p->desc.in_dtype, p->desc.channels, int(p->gx.t_eff), 2 + big);
}

namespace {

// Staged pitch >= n samples: whole 16-byte words, odd in 16-byte words (lanes
// on consecutive rows reading 16 bytes hit distinct banks).
int pad_pitch(int n, int es)
{
    const int u = 16 / es;
    int p = (n + u - 1) / u * u;
    if ((p / u) % 2 == 0) p += u;
    return p;
}

// Group descriptors of one axis: per group of 4 outputs the first window's
// start (rounded down to a multiple of `align`), the pattern, and the run of
// inputs the group reads.  False if a step between neighbouring windows is not
// 0 or 1 (not an upscale) or a side is too large for the 24-bit field.
bool groups_of(const std::vector<int32_t> &st, int n_in, int T, int align, std::vector<int32_t> &info,
               std::vector<int32_t> &run_end)
{
    const int n = int(st.size());
    const int groups = (n + kG - 1) / kG;
    if (n_in >= (1 << 24)) return false;
    info.assign(groups, 0);
    run_end.assign(groups, 0);
    for (int q = 0; q < groups; ++q) {
        int s[kG];
        for (int g = 0; g < kG; ++g) s[g] = st[std::min(n - 1, kG * q + g)];
        const int base = align > 1 ? s[0] / align * align : s[0];
        const int o0 = s[0] - base;
        int pat = align > 1 ? o0 : 0;
        for (int g = 1; g < kG; ++g) {
            const int d = s[g] - s[g - 1];
            if (d != 0 && d != 1) return false;
            pat |= d << (align > 1 ? g + 1 : g - 1);
        }
        info[q] = base | (pat << 24);
        run_end[q] = s[kG - 1] + T; // one past the last input of the group's windows
    }
    return true;
}

struct Choice {
    int sw = 0, P = 0, offB = 0, gpr = 0, nblk = 0, occ = 0, grid = 0;
    size_t smem = 0;
    double cost = 1e300;
};

struct Geometry {
    int C = 0, T = 0, es = 0, groups_x = 0, groups_y = 0, JH = 0, JV = 0, WP = 0;
    std::vector<int32_t> hinfo, vinfo, hend, vend;
};

rs_status geometry(const rs_plan *p, Geometry &g)
{
    const rs_plan_desc &d = p->desc;
    g.C = d.channels;
    if ((d.in_dtype != RS_F32 && d.in_dtype != RS_F16 && d.in_dtype != RS_BF16) || d.out_dtype != d.in_dtype ||
        (g.C != 1 && g.C != 3) || (d.flags & RS_NO_STREAM) || p->prefilter)
        return RS_ERR_UNSUPPORTED;
    if (!tma_layout_ok(p)) return RS_ERR_UNSUPPORTED;
    g.T = p->gx.t_eff;
    if (p->gy.t_eff != g.T || (g.T != 4 && g.T != 6) || !kernel_for(d.in_dtype, g.C, g.T, 0))
        return RS_ERR_UNSUPPORTED;
    g.es = int(dt_size(d.in_dtype));
    if (!groups_of(p->host_start_x, int(p->gx.n_in), g.T, 4, g.hinfo, g.hend)) return RS_ERR_UNSUPPORTED;
    if (!groups_of(p->host_start_y, int(p->gy.n_in), g.T, 1, g.vinfo, g.vend)) return RS_ERR_UNSUPPORTED;
    g.groups_x = int(g.hinfo.size());
    g.groups_y = int(g.vinfo.size());
    // a group's band covers T + 3 inputs from its first window, which starts
    // 0..3 pixels into the group's run of 3 chunks (12 pixels) across
    g.JH = 12;
    g.JV = g.T + 3;
    // most row groups whose last window row falls in one block of kRB rows
    g.WP = 1;
    for (int a = 0, e = 0; a < g.groups_y; ++a) {
        e = std::max(e, a);
        while (e < g.groups_y && g.vend[e] <= g.vend[a] + kRB - 1) ++e;
        g.WP = std::max(g.WP, e - a);
    }
    return RS_OK;
}

// Every strip width (a multiple of 4 outputs) whose staged rows fit one or two
// TMA boxes, with its best row ranges by a cost model (the busiest SM's CTAs
// times each CTA's work), cheapest first.
std::vector<Choice> choices(const rs_plan *p, const Geometry &g, int NI, int nthreads, int nr_force)
{
    std::vector<Choice> out;
    const int C = g.C, es = g.es;
    const int HR = 2 * kRB + g.JV, M = g.JV - 1, Q = (HR + M) | 1;
    const void *fn = kernel_for(p->desc.in_dtype, C, g.T, nthreads > 32 * kSmallWarps ? 1 : 0);
    if (rs::occupancy(fn, nthreads, 0) < 1) return out;
    const int sw_max = C == 1 ? 252 : 128;
    for (int sw = 8; sw <= sw_max; sw += 4) {
        const int ngx = sw / kG, nch = sw * C / 4;
        const int n_strips = (g.groups_x + ngx - 1) / ngx;
        int need = 0;
        for (int g0 = 0; g0 < g.groups_x; g0 += ngx) {
            const int gl = std::min(g.groups_x, g0 + ngx) - 1;
            need = std::max(need, ((g.hinfo[gl] & 0xffffff) + g.JH - (g.hinfo[g0] & 0xffffff)) * C + (es == 2 ? 4 : 0));
        }
        int P = pad_pitch(need, es), offB = 0;
        if (P > 256) {
            // boxes A = [0, P) and B = [offB, offB + P): offB <= P - JH C (a run that
            // leaves box A lies inside box B) and offB + P >= need
            const int u = 16 / es;
            P = 0;
            for (int cand = pad_pitch((need + g.JH * C + 1) / 2, es); cand <= 256 && !P; cand += 2 * u) {
                const int o = (cand - g.JH * C) / u * u;
                if (o > 0 && o + cand >= need) {
                    P = cand;
                    offB = o;
                }
            }
            if (!P) continue;
        }
        Choice best;
        const std::vector<int> nrs =
            nr_force > 0 ? std::vector<int>{nr_force} : stream::range_counts(n_strips, p->num_sms, 4096);
        for (const int nr : nrs) {
            const int gpr = (g.groups_y + nr - 1) / nr;
            if (gpr < 8 && nr > 1 && nr_force <= 0) break;
            const int ranges = (g.groups_y + gpr - 1) / gpr;
            int rows = 0;
            for (int q0 = 0; q0 < g.groups_y; q0 += gpr) {
                const int q1 = std::min(g.groups_y, q0 + gpr) - 1;
                rows = std::max(rows, g.vend[q1] - (g.vinfo[q0] & 0xffffff));
            }
            const int nblk = (rows + kRB - 1) / kRB;
            if (nblk <= 512) {
                const size_t smem = layout(NI, P, Q, nch, ngx, g.T, g.WP, nblk, offB != 0, es).total;
                const int occ = rs::occupancy(fn, nthreads, smem);
                if (occ >= 1) {
                    const int64_t grid = int64_t(n_strips) * ranges;
                    const int64_t per_sm = (grid + p->num_sms - 1) / p->num_sms;
                    // the busiest SM's CTAs share its throughput: their rows
                    // (plus the pipeline fill) times the strip width plus a
                    // fixed share worth 40 outputs per block (hand-offs, the
                    // vertical bands, the staged halo), fitted to measured
                    // widths; a lone CTA per SM hides latency worse
                    const double cost =
                        double(per_sm) * (rows + 2 * kRB) * (sw + 40.0) * (occ >= 2 ? 1.0 : 1.35);
                    if (cost < best.cost * 0.999) {
                        best.sw = sw;
                        best.P = P;
                        best.offB = offB;
                        best.gpr = gpr;
                        best.nblk = nblk;
                        best.occ = occ;
                        best.grid = int(grid);
                        best.smem = smem;
                        best.cost = cost;
                    }
                }
            }
            if (ranges >= g.groups_y) break;
        }
        if (best.sw) out.push_back(best);
    }
    std::stable_sort(out.begin(), out.end(), [](const Choice &a, const Choice &b) { return a.cost < b.cost; });
    return out;
}

// Warps of the two passes: the caller's choice (ex = 1; zeros: the
// defaults), else 4 horizontal and 4 vertical warps (the fastest split of the
// 4096x4096x3 x1.37 plan).
void warps_of(const stream::Opts &o, int &HW, int &VW)
{
    HW = 4;
    VW = 4;
    if (o.ex > 0) {
        if (o.hw >= 1) HW = o.hw;
        if (o.vw >= 1) VW = o.vw;
    }
    if (1 + HW + VW > kMaxWarps) VW = std::max(1, kMaxWarps - 1 - HW);
}

} // namespace

bool eligible(const rs_plan *p)
{
    Geometry g;
    return geometry(p, g) == RS_OK;
}

int widths(rs_plan *p, const stream::Opts &o, int *out, int n)
{
    Geometry g;
    if (geometry(p, g) != RS_OK) return 0;
    const int NI = o.ex > 0 && o.ni_min >= 2 && o.ni_min <= kMaxNI ? o.ni_min : 2;
    int HW, VW;
    warps_of(o, HW, VW);
    const std::vector<Choice> c = choices(p, g, NI, 32 * (1 + HW + VW), o.ex > 0 ? o.nr : 0);
    int k = 0;
    for (; k < n && k < int(c.size()); ++k) out[k] = c[k].sw;
    return k;
}

rs_status setup(rs_plan *p, cudaStream_t s, const stream::Opts &o)
{
    p->x_on = 0;
    Geometry g;
    const rs_status gs = geometry(p, g);
    if (gs != RS_OK) return gs;
    // the caller's choices apply to this form only when it asked for it (ex = 1)
    const int NI = o.ex > 0 && o.ni_min >= 2 && o.ni_min <= kMaxNI ? o.ni_min : 2;
    int HW, VW;
    warps_of(o, HW, VW);
    const std::vector<Choice> cands = choices(p, g, NI, 32 * (1 + HW + VW), o.ex > 0 ? o.nr : 0);
    if (cands.empty()) return RS_ERR_UNSUPPORTED;
    const Choice *pick = &cands[0];
    if (o.sw > 0) {
        pick = nullptr;
        for (const Choice &c : cands)
            if (c.sw == o.sw) pick = &c;
        if (!pick) return RS_ERR_UNSUPPORTED;
    }
    const rs_plan_desc &d = p->desc;
    // device descriptors: column groups, row groups (padded for 16-byte copies)
    Carver cv;
    const size_t o_h = cv.take(size_t(g.groups_x) * 4);
    const size_t nvi = size_t((g.groups_y + 3) & ~3) + 4;
    const size_t o_v = cv.take(nvi * 4);
    std::vector<int32_t> host(cv.off / 4, 0);
    std::memcpy(host.data() + o_h / 4, g.hinfo.data(), g.hinfo.size() * 4);
    std::memcpy(host.data() + o_v / 4, g.vinfo.data(), g.vinfo.size() * 4);
    char *base = nullptr;
    cudaError_t e = cudaSuccess;
    if (p->ext_base) {
        // the caller's space, uploaded through its pinned staging on `s`
        if (cv.off > p->ext_bytes || cv.off > p->ext_staging_bytes)
            return fail(RS_ERR_BUDGET, "pipelined-kernel descriptors exceed their reserved space");
        std::memcpy(p->ext_staging, host.data(), cv.off);
        e = cudaMemcpyAsync(p->ext_base, p->ext_staging, cv.off, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "uploading pipelined-kernel descriptors");
        base = p->ext_base;
    } else {
        if (p->xbufs.p) {
            cudaFree(p->xbufs.p);
            p->xbufs.p = nullptr;
        }
        e = cudaMalloc(&p->xbufs.p, cv.off);
        if (e != cudaSuccess) return cuda_fail(e, "allocating pipelined-kernel descriptors");
        p->xbufs.n = cv.off;
        e = cudaMemcpy(p->xbufs.p, host.data(), cv.off, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "uploading pipelined-kernel descriptors");
        base = static_cast<char *>(p->xbufs.p);
    }
    Params &xp = p->xp;
    std::memset(&xp, 0, sizeof xp);
    xp.in_h = p->gy.n_in;
    xp.in_w = p->gx.n_in;
    xp.out_h = p->gy.n_out;
    xp.out_w = p->gx.n_out;
    xp.in_stride = d.in_row_stride;
    xp.out_stride = d.out_row_stride;
    xp.hinfo = reinterpret_cast<const int32_t *>(base + o_h);
    xp.wx = static_cast<const float *>(p->tx.wwork);
    xp.vinfo = reinterpret_cast<const int32_t *>(base + o_v);
    xp.wy = static_cast<const float *>(p->ty.wwork);
    xp.SW = pick->sw;
    xp.n_strips = (g.groups_x + pick->sw / kG - 1) / (pick->sw / kG);
    xp.groups_x = g.groups_x;
    xp.groups_y = g.groups_y;
    xp.gpr = pick->gpr;
    xp.P = pick->P;
    xp.offB = pick->offB;
    xp.JH = g.JH;
    xp.JV = g.JV;
    xp.HR = 2 * kRB + g.JV;
    xp.M = g.JV - 1;
    xp.Q = (xp.HR + xp.M) | 1;
    xp.NI = NI;
    xp.WP = g.WP;
    xp.nblk = pick->nblk;
    xp.HW = HW;
    xp.VW = VW;
    xp.pf = o.ex > 0 && o.pf ? 1 : 0;

    xp.err = p->d_err;
    {
        stream::Opts used;
        used.ex = 1;
        used.ws = 0;
        used.hw = HW;
        used.vw = VW;
        used.nr = o.ex > 0 ? o.nr : 0;
        used.ni_min = NI;
        used.sw = pick->sw;
        used.pf = xp.pf;

        p->stream_code = used.code();
    }
    p->s_fn = kernel_for(d.in_dtype, g.C, g.T, 1 + HW + VW > kSmallWarps ? 1 : 0);
    p->s_block = 32 * (1 + HW + VW);
    p->s_smem = pick->smem;
    p->s_grid = pick->grid;
    p->s_ctas = pick->occ;
    p->stmap_ptr = nullptr;
    p->x_on = 1;
    p->tcs_on = 0;
    p->stream_ok = 1;
    p->scratch_bytes = int64_t(p->tables.n + p->bands.n + p->tmp.n + p->sbufs.n + p->xbufs.n);
    return RS_OK;
}

} // namespace xstream
} // namespace rs
