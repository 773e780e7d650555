// rs_capi.cu -- the C ABI (include/rs.h): plans, geometry, path choice and
// launches.  Host code only; the arithmetic runs in the kernels of
// rs_weights.cu, rs_two_pass.cu and rs_fused*.cu.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include "rs_plan.h"

namespace rs {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

namespace fused {
const Variant *variants_f64(int *n);
const Variant *variants_f32(int *n);
const Variant *variants_f16(int *n);
const Variant *variants_bf16(int *n);
} // namespace fused

const fused::Variant *find_variant(int dtype, int C, int G)
{
    int n = 0;
    const fused::Variant *v = nullptr;
    switch (dtype) {
    case RS_F64: v = fused::variants_f64(&n); break;
    case RS_F32: v = fused::variants_f32(&n); break;
    case RS_F16: v = fused::variants_f16(&n); break;
    case RS_BF16: v = fused::variants_bf16(&n); break;
    default: return nullptr;
    }
    for (int i = 0; i < n; ++i)
        if (v[i].C == C && v[i].G == G) return &v[i];
    return nullptr;
}

EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

int64_t env_plan_flags()
{
    static const int64_t flags = [] {
        const char *v = std::getenv("RS_PLAN_FLAGS");
        if (!v || !*v) return int64_t(0);
        static const struct {
            const char *name;
            uint32_t bit;
        } known[] = {{"FORCE_SIMT", RS_FORCE_SIMT},     {"FORCE_TC", RS_FORCE_TC},       {"TWO_PASS", RS_TWO_PASS},
                     {"CHECK", RS_CHECK},               {"NO_STREAM", RS_NO_STREAM},     {"FORCE_STREAM", RS_FORCE_STREAM},
                     {"FORCE_VFIRST", RS_FORCE_VFIRST}};
        int64_t f = 0;
        std::string s(v);
        size_t a = 0;
        while (a <= s.size()) {
            size_t b = s.find(',', a);
            if (b == std::string::npos) b = s.size();
            std::string name = s.substr(a, b - a);
            while (!name.empty() && name.front() == ' ') name.erase(name.begin());
            while (!name.empty() && name.back() == ' ') name.pop_back();
            if (!name.empty()) {
                bool hit = false;
                for (const auto &k : known)
                    if (name == k.name) {
                        f |= k.bit;
                        hit = true;
                    }
                if (!hit) return int64_t(-1);
            }
            a = b + 1;
        }
        return f;
    }();
    return flags;
}

int support_radius(int kernel, double param)
{
    switch (kernel) {
    case RS_K_LINEAR: return 1;
    case RS_K_CUBIC: return 2;
    case RS_K_BSPLINE3: return 2;
    case RS_K_LANCZOS:
        if (!(param >= 1.0 && param <= 16.0) || param != std::floor(param)) return 0;
        return int(param);
    case RS_K_MITCHELL:
        if (!(param >= 0.0 && param <= 1.0)) return 0;
        return 2;
    case RS_K_GAUSSIAN:
        if (!(param > 0.0 && param <= 4.0)) return 0;
        return int(std::ceil(3.0 * param));
    }
    return 0;
}



} // namespace rs

using namespace rs;

namespace rs {

rs_status fail(rs_status s, const std::string &msg)
{
    set_error(msg);
    return s;
}

rs_status cuda_fail(cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? RS_ERR_OOM : RS_ERR_CUDA, m);
}

bool axis_setup(AxisGeom &g, int64_t n_in, int64_t n_out, const rs_plan_desc &d, std::string &why)
{
    g.n_in = n_in;
    g.n_out = n_out;
    g.R = support_radius(d.kernel, d.param);
    if (g.R == 0) {
        why = "kernel/param invalid (Lanczos needs an integer R in 1..16)";
        return false;
    }
    const bool aa = !(d.flags & RS_NO_ANTIALIAS);
    g.D = (aa && n_in > n_out) ? 2 * n_in : 2 * n_out;
    const int64_t traw = (g.R * g.D + n_out - 1) / n_out;
    if (traw > kMaxTaps) {
        why = "more than 256 taps per output on one axis";
        return false;
    }
    g.t_raw = int32_t(traw);
    g.t_eff = int32_t(std::min<int64_t>(traw, n_in));
    g.kernel = d.kernel;
    g.boundary = d.boundary;
    g.param = d.param;
    return true;
}

int64_t derive_out(int32_t given, int64_t n, double scale)
{
    if (given > 0) return given;
    if (!(scale > 0.0) || !std::isfinite(scale)) return -1;
    const double v = std::floor(double(n) * scale + 0.5);
    if (!(v < double(kMaxSide) + 1.0)) return -1;
    return std::max<int64_t>(1, int64_t(v));
}

// Checks a descriptor the way every entry point that takes one does, derives
// the output size from the scale where it is 0 and the packed row strides
// where they are 0; on failure sets the error message.
rs_status validate_desc(const rs_plan_desc &in, rs_plan_desc *out)
{
    rs_plan_desc d = in;
    if (d.in_h < 1 || d.in_w < 1 || d.in_h > kMaxSide || d.in_w > kMaxSide)
        return fail(RS_ERR_INVALID_ARG, "input size out of range");
    if (d.channels < 1 || d.channels > 64) return fail(RS_ERR_INVALID_ARG, "channels must be 1..64");
    if (d.out_h < 0 || d.out_w < 0) return fail(RS_ERR_INVALID_ARG, "negative output size");
    if (d.kernel < RS_K_LINEAR || d.kernel > RS_K_GAUSSIAN) return fail(RS_ERR_INVALID_ARG, "unknown kernel");
    if (d.boundary < RS_B_CLAMP || d.boundary > RS_B_TRUNCATE) return fail(RS_ERR_INVALID_ARG, "unknown boundary");
    if (d.in_dtype < RS_F64 || d.in_dtype > RS_BF16 || d.out_dtype < RS_F64 || d.out_dtype > RS_BF16)
        return fail(RS_ERR_INVALID_ARG, "unknown dtype");
    if (d.in_dtype != d.out_dtype) return fail(RS_ERR_UNSUPPORTED, "in_dtype and out_dtype must be equal");
    if (d.flags & ~uint32_t(0x1ff)) return fail(RS_ERR_INVALID_ARG, "unknown flag bits");
    if ((d.flags & RS_PREFILTER) &&
        (d.kernel != RS_K_BSPLINE3 || d.boundary == RS_B_TRUNCATE || (d.in_dtype != RS_F32 && d.in_dtype != RS_F64)))
        return fail(RS_ERR_UNSUPPORTED, "RS_PREFILTER needs RS_K_BSPLINE3, FP32 or FP64 storage and the clamp, "
                                        "mirror or reflect101 boundary");
    if (support_radius(d.kernel, d.param) == 0)
        return fail(RS_ERR_INVALID_ARG, "kernel parameter out of range (Lanczos: an integer R in 1..16; "
                                        "Mitchell-Netravali: B in [0, 1]; Gaussian: sigma in (0, 4])");
    if (d.kernel == RS_K_CUBIC && !std::isfinite(d.param)) return fail(RS_ERR_INVALID_ARG, "cubic a not finite");
    const int64_t oh = derive_out(d.out_h, d.in_h, d.scale_h);
    const int64_t ow = derive_out(d.out_w, d.in_w, d.scale_w);
    if (oh < 1 || ow < 1 || oh > kMaxSide || ow > kMaxSide)
        return fail(RS_ERR_INVALID_ARG, "output size out of range (scale must be finite and > 0)");
    d.out_h = int32_t(oh);
    d.out_w = int32_t(ow);
    if (d.in_row_stride == 0) d.in_row_stride = int64_t(d.in_w) * d.channels;
    if (d.out_row_stride == 0) d.out_row_stride = int64_t(d.out_w) * d.channels;
    if (d.in_row_stride < int64_t(d.in_w) * d.channels || d.out_row_stride < int64_t(d.out_w) * d.channels)
        return fail(RS_ERR_INVALID_ARG, "row stride smaller than a row");

    *out = d;
    return RS_OK;
}

// Weight-table launch for both axes; when the axes are identical the column
// tables alias the row tables and only the rows are computed.
cudaError_t launch_plan_weights(rs_plan *p, cudaStream_t s);

WeightArgs weight_args(rs_plan *p, int axis)
{
    WeightArgs a;
    a.g = axis == 0 ? p->gy : p->gx;
    a.t = axis == 0 ? p->ty : p->tx;
    a.work_is_double = p->work_double;
    a.err = p->d_err;
    return a;
}

cudaError_t launch_plan_weights(rs_plan *p, cudaStream_t s)
{
    WeightArgs a1 = weight_args(p, 1);
    if (p->axes_alias) a1.g.n_out = 0; // the column tables are the row tables
    return launch_weights(weight_args(p, 0), a1, s);
}

// Largest band span (max start - min start within a group) + t_eff.
int band_needed(const std::vector<int32_t> &start, int G, int t_eff)
{
    int need = 0;
    const int n = int(start.size());
    for (int g0 = 0; g0 < n; g0 += G) {
        int lo = start[g0], hi = start[g0];
        for (int r = 1; r < G && g0 + r < n; ++r) {
            lo = std::min(lo, int(start[g0 + r]));
            hi = std::max(hi, int(start[g0 + r]));
        }
        need = std::max(need, hi - lo + t_eff);
    }
    return need;
}

// Staged extent of every tile along one axis: max over tiles of
// (max base + J) - min base, in samples (times C, after aligning the start
// down to `vec` when `vec` > 1).
int tile_extent(const std::vector<int32_t> &base, int groups_per_tile, int J, int C, int vec)
{
    int need = 0;
    const int n = int(base.size());
    for (int g0 = 0; g0 < n; g0 += groups_per_tile) {
        int lo = base[g0], hi = base[g0];
        for (int r = 1; r < groups_per_tile && g0 + r < n; ++r) {
            lo = std::min(lo, int(base[g0 + r]));
            hi = std::max(hi, int(base[g0 + r]));
        }
        const int s0 = lo * C;
        const int xs = vec > 1 ? s0 - (s0 % vec) : s0;
        need = std::max(need, (hi + J) * C - xs);
    }
    return need;
}

// Group bases as the band kernel computes them (used here only to size
// candidate tiles; the kernel's own bases are read back and re-checked).
std::vector<int32_t> group_bases(const std::vector<int32_t> &start, int G, int J, int64_t n_in, int t_eff)
{
    const int n = int(start.size());
    std::vector<int32_t> b((n + G - 1) / G);
    for (int g = 0; g < int(b.size()); ++g) {
        int64_t b0 = n_in;
        for (int r = 0; r < G && g * G + r < n; ++r) b0 = std::min<int64_t>(b0, start[g * G + r]);
        b[g] = int32_t(n_in >= J ? std::min<int64_t>(b0, n_in - J) : 0);
    }
    (void)t_eff;
    return b;
}

// Rows per TMA box when a tile's staged rows need n_sub boxes (<= 256 rows
// each).  With several boxes the height is a multiple of 8 rows so that each
// box's shared-memory destination stays 128-byte aligned (a row is a multiple
// of 16 bytes).
int sub_height(int rows, int n_sub)
{
    if (n_sub <= 1) return rows;
    const int h = (rows + n_sub - 1) / n_sub;
    return (h + 7) / 8 * 8;
}


// Cost model of one candidate (SM cycles per output pixel, lower is better).
// Per tile: instruction estimates of the two passes (FMA + shared loads per
// tap, plus a fixed tail per warp task).  The pipelined CTA runs pass 1 on n1
// warps and pass 2 on the rest, so its tile time is the slower group's
// critical path; k resident CTAs overlap their tiles, but the SM cannot issue
// more than 4 instructions per cycle nor fill shared memory from L2 faster
// than ~64 B per cycle.  Also picks the warp split n1.
double model_cost(Candidate &c, int C, size_t esz, size_t asz, int V)
{
    const int ngy = c.tile_h / c.G, ngx = c.tile_w / c.G;
    const int w1 = (c.box_w + 32 * V - 1) / (32 * V) * (32 * V);
    const int nchunk = w1 / (32 * V);
    const int rb = std::min(32, c.tile_h);
    const int t1 = ngy * nchunk;
    const int npairs = fused::pair_slots(ngx);
    const int t2 = ((c.tile_h + rb - 1) / rb) * ((npairs + 32 / rb - 1) / (32 / rb));
    const int W = fused::kWarps;
    // per tap: packed FMAs + sample loads + weight loads, plus a fixed tail
    const double task1 = c.J * (double(c.G * V) / 2.0 + V / 2.0 + c.G / 2.0 + 1.0) + 24.0 + c.G * V;
    const double task2 = c.J * (double(c.G * C) + 2.0 * C + c.G / 2.0 + 1.0) + 30.0 + 2.0 * C * c.G;
    const double issue = (t1 * task1 + t2 * task2 + 200.0) / 4.0 * 1.25;
    const double fill = (double(c.box_h) * c.box_w * esz + double(ngy + ngx) * band_stride(c.G, c.J) * asz) / 64.0;
    const int ctas = int(std::min<size_t>(8, (227 * 1024) / std::max<size_t>(c.smem, 1)));
    double best = 1e300;
    for (int n1 = 1; n1 < W; ++n1) {
        const double crit = std::max(std::ceil(double(t1) / n1) * task1, std::ceil(double(t2) / (W - n1)) * task2);
        const double per_tile = std::max(std::max(issue, fill), crit * 2.0 / std::max(1, ctas));
        if (per_tile < best) {
            best = per_tile;
            c.n1 = n1;
        }
    }
    return best / (double(c.tile_h) * c.tile_w);
}

// Builds the band tables for a chosen candidate and fills the kernel
// parameters (shared by the model-based choice and the autotuner).
rs_status apply_fused(rs_plan *p, cudaStream_t stream, const Candidate &c, bool tma_layout)
{
    const rs_plan_desc &d = p->desc;
    const int C = d.channels;
    const int dt = d.in_dtype;
    const size_t esz = dt_size(dt);
    const size_t asz = p->work_double ? 8 : 4;
    const int vec = int(16 / esz);
    p->variant = find_variant(dt, C, c.G);
    if (!p->variant) return RS_ERR_UNSUPPORTED;
    // the tensor map encodes the box size: a new configuration needs a new map
    p->tmap_ptr = nullptr;
    p->G = c.G;
    p->J = c.J;
    // the vertical band of the FP32 SIMT path stores every weight twice (packed
    // pairs); the tensor-core path reads it once per weight-matrix element
    p->ty.dup = (p->work_double || c.tc) ? 1 : 2;
    p->tx.dup = 1;
    p->tx.pair_ngx = c.tile_w / c.G; // the horizontal band interleaves group pairs
    p->ty.G = p->tx.G = c.G;
    p->ty.J = p->tx.J = c.J;
    const int js_y = band_stride(c.G * p->ty.dup, c.J), js_x = band_slot_stride(p->tx);
    p->ty.groups = int32_t((p->gy.n_out + c.G - 1) / c.G);
    p->tx.groups = int32_t((p->gx.n_out + c.G - 1) / c.G);
    Carver cv;
    const size_t o_by = cv.take(size_t(p->ty.groups) * 4);
    const size_t o_bx = cv.take(size_t(p->tx.groups) * 4);
    const size_t o_wy = cv.take(size_t(p->ty.groups) * js_y * asz);
    const size_t o_wx = cv.take(size_t(band_slots(p->tx)) * js_x * asz);
    if (p->bands.p) {
        cudaFree(p->bands.p);
        p->bands.p = nullptr;
    }
    cudaError_t e = cudaMalloc(&p->bands.p, cv.off);
    if (e != cudaSuccess) return cuda_fail(e, "allocating band tables");
    p->bands.n = cv.off;
    char *base = static_cast<char *>(p->bands.p);
    p->ty.band_base = reinterpret_cast<int32_t *>(base + o_by);
    p->tx.band_base = reinterpret_cast<int32_t *>(base + o_bx);
    p->ty.band_w = base + o_wy;
    p->tx.band_w = base + o_wx;
    e = launch_band(weight_args(p, 0), weight_args(p, 1), stream);
    if (e != cudaSuccess) return cuda_fail(e, "band kernel launch");
    p->tile_bands_stale = 0;
    std::vector<int32_t> by(p->ty.groups), bx(p->tx.groups);
    e = cudaMemcpyAsync(by.data(), p->ty.band_base, by.size() * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bx.data(), p->tx.band_base, bx.size() * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading band tables");

    // exact staged extents from the kernel's own bases
    const int ngy = c.tile_h / c.G, ngx = c.tile_w / c.G;
    const int rows = tile_extent(by, ngy, c.J, 1, 1);
    const int bw = (tile_extent(bx, ngx, c.J, C, vec) + vec - 1) / vec * vec;
    fused::Params &fp = p->fp;
    std::memset(&fp, 0, sizeof fp);
    fp.in_h = p->gy.n_in;
    fp.in_w = p->gx.n_in;
    fp.out_h = p->gy.n_out;
    fp.out_w = p->gx.n_out;
    fp.in_stride = d.in_row_stride;
    fp.out_stride = d.out_row_stride;
    fp.base_y = p->ty.band_base;
    fp.base_x = p->tx.band_base;
    fp.band_y = p->ty.band_w;
    fp.band_x = p->tx.band_w;
    fp.J = c.J;
    fp.js_y = js_y;
    fp.js_x = js_x;
    fp.tile_h = c.tile_h;
    fp.tile_w = c.tile_w;
    if (c.tc) {
        // whole 128-sample M blocks, K rows padded to the MMA's 16
        const int kpad = (rows + 15) / 16 * 16;
        const int nmb = (tile_extent(bx, ngx, c.J, C, 8) + 127) / 128;
        int cols = 32;
        while (cols < nmb * c.tile_h) cols <<= 1;
        if (!tma_layout || kpad > 256 || nmb * 16 > 256 || cols > 512 || c.tile_h % 16 || c.tile_h > 256)
            return RS_ERR_UNSUPPORTED;
        fp.n_sub = 1;
        fp.sub_h = kpad;
        fp.box_h = kpad;
        fp.box_w = nmb * 128;
        fp.w1 = fp.box_w;
        fp.pitch_t = fp.box_w + 1;
        fp.tc_nmb = nmb;
        fp.tc_kpad = kpad;
    } else {
        fp.n_sub = (rows + 255) / 256;
        fp.sub_h = sub_height(rows, fp.n_sub);
        fp.box_h = fp.n_sub * fp.sub_h;
        fp.box_w = bw;
        const int V = p->variant->V;
        fp.w1 = (bw + 32 * V - 1) / (32 * V) * (32 * V);
        fp.pitch_t = fp.w1 | 1;
    }
    fp.groups_y = p->ty.groups;
    fp.groups_x = p->tx.groups;
    fp.tiles_y = int32_t((p->gy.n_out + c.tile_h - 1) / c.tile_h);
    fp.tiles_x = int32_t((p->gx.n_out + c.tile_w - 1) / c.tile_w);
    fp.stages = c.stages;
    fp.n1 = c.tc ? 4 : c.n1; // the tensor-memory epilogue needs four warps (128 lanes)
    fp.err = p->d_err;
    p->tma_ok = (tma_layout && (c.tc || bw <= 256)) ? 1 : 0;
    p->smem = fused::layout(esz, asz, fp.box_h, fp.box_w, ngy, ngx, js_y, js_x, fp.tile_h, fp.pitch_t,
                            p->tma_ok ? fp.stages : 1)
                  .total +
              (c.tc ? fused::align_up(size_t(4) * fp.tile_h * fp.tc_kpad, 128) : 0);
    if (p->smem > 227 * 1024) return RS_ERR_UNSUPPORTED;
    p->kernel_fn = c.tc ? p->variant->fn_tc : p->variant->fn;
    // The limit is a property of the kernel function, shared by every plan that
    // uses this variant, so opt in to the whole per-block maximum once rather
    // than to this plan's size (occupancy follows the size passed at launch).
    e = cudaFuncSetAttribute(p->kernel_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return cuda_fail(e, "setting shared memory size");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, p->kernel_fn, fused::kThreads, p->smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (c.tc) {
        // Resident CTAs hold their tensor memory for the whole launch: pad the
        // shared-memory request until they fit the SM's 512 columns together,
        // so that no allocation has to wait for another CTA to finish.
        int cols = 32;
        while (cols < fp.tc_nmb * fp.tile_h) cols <<= 1;
        const int max_ctas = 512 / cols;
        while (occ > max_ctas && p->smem < 227 * 1024) {
            p->smem = std::min<size_t>(227 * 1024, p->smem + 8 * 1024);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, p->kernel_fn, fused::kThreads, p->smem);
            if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
        }
        if (occ > max_ctas || occ < 1) return RS_ERR_UNSUPPORTED;
    }
    if (occ < 1) return RS_ERR_UNSUPPORTED;
    const int64_t tiles = int64_t(fp.tiles_y) * fp.tiles_x;
    p->grid = int(std::min<int64_t>(tiles, int64_t(occ) * p->num_sms));
    p->ctas_per_sm = occ;
    p->chosen = c;
    p->chosen.n1 = fp.n1;
    return RS_OK;
}

// Cost of a tensor-core candidate in modelled SM cycles per output pixel.
// Pass 1 (four warps): building the hi/lo weight matrices, the MMAs (two per
// 128 x N x 16 step at ~8K FLOP per SM cycle) and the tensor-memory epilogue;
// pass 2 as in the SIMT model on the other four warps; the tile fill at
// ~64 B per cycle.
double model_cost_tc(const Candidate &c, int C, int kpad, int nmb, size_t esz, size_t asz)
{
    const int ngx = c.tile_w / c.G;
    const int N = c.tile_h;
    const double build = double(N) * kpad * 12.0 / 128.0;
    const double mma = 4.0 * 128.0 * N * kpad * nmb / 8192.0;
    const double epi = double(nmb) * N * 2.0;
    const double pass1 = build + mma + epi + 300.0;
    const int rb = std::min(32, c.tile_h);
    const int npairs = fused::pair_slots(ngx);
    const int t2 = ((c.tile_h + rb - 1) / rb) * ((npairs + 32 / rb - 1) / (32 / rb));
    const double task2 = c.J * (double(c.G * C) + 2.0 * C + c.G / 2.0 + 1.0) + 30.0 + 2.0 * C * c.G;
    const double pass2 = std::ceil(double(t2) / (fused::kWarps - 4)) * task2;
    const double fill = (double(kpad) * nmb * 128 * esz + double(c.tile_h / c.G + ngx) * band_stride(c.G, c.J) * asz) / 64.0;
    return std::max(std::max(pass1, pass2), fill) / (double(c.tile_h) * c.tile_w);
}

// Whether a plan can run its vertical pass on the tensor cores: 16-bit
// storage, TMA tile copies, and rows of whole 8-sample (16-byte) chunks so
// that the 3-D tensor map never reads past a row.
bool tc_eligible(const rs_plan *p, bool tma_layout)
{
    const rs_plan_desc &d = p->desc;
    return tma_layout && (d.in_dtype == RS_F16 || d.in_dtype == RS_BF16) && (int64_t(d.in_w) * d.channels) % 8 == 0 &&
           !(d.flags & RS_FORCE_SIMT);
}

// Every feasible fused configuration of a plan (host start tables needed):
// SIMT configurations, or with tc the tensor-core ones.
std::vector<Candidate> enumerate_candidates(rs_plan *p, bool tma_layout, bool tc)
{
    const rs_plan_desc &d = p->desc;
    const int C = d.channels;
    const int dt = d.in_dtype;
    const size_t esz = dt_size(dt);
    const size_t asz = p->work_double ? 8 : 4;
    const int vec = int(16 / esz);
    const size_t smem_cap = 227 * 1024;
    const std::vector<int32_t> &sy = p->host_start_y, &sx = p->host_start_x;
    std::vector<Candidate> out;
    if (tc) {
        if (!tc_eligible(p, tma_layout)) return out;
        for (int G : {4, 2, 1}) {
            if (!find_variant(dt, C, G)) continue;
            const int J = std::max(band_needed(sy, G, p->gy.t_eff), band_needed(sx, G, p->gx.t_eff));
            if (J > 256) continue;
            const std::vector<int32_t> by = group_bases(sy, G, J, p->gy.n_in, p->gy.t_eff);
            const std::vector<int32_t> bx = group_bases(sx, G, J, p->gx.n_in, p->gx.t_eff);
            for (int tile_h : {16, 32, 64, 128}) {
                if (tile_h / G > 32) continue;
                if (tile_h > 16 && tile_h / 2 >= p->gy.n_out) continue;
                const int rows = tile_extent(by, tile_h / G, J, 1, 1);
                const int kpad = (rows + 15) / 16 * 16;
                if (kpad > 256) continue;
                for (int ngx = 1; ngx <= 32; ++ngx) {
                    const int tile_w = ngx * G;
                    if (tile_w > ((p->gx.n_out + G - 1) / G) * G && ngx > 1) break;
                    const int nmb = (tile_extent(bx, ngx, J, C, 8) + 127) / 128;
                    if (nmb > 16 || nmb * tile_h > 512) break;
                    const int box_w = nmb * 128;
                    for (int stages : {2, 1}) {
                        Candidate c;
                        c.tc = 1;
                        c.G = G;
                        c.J = J;
                        c.tile_h = tile_h;
                        c.tile_w = tile_w;
                        c.stages = stages;
                        c.box_h = kpad;
                        c.sub_h = kpad;
                        c.n_sub = 1;
                        c.box_w = box_w;
                        c.n1 = 4;
                        c.smem = fused::layout(esz, asz, kpad, box_w, tile_h / G, ngx, band_stride(G, J),
                                               band_stride(2 * G, J), tile_h, box_w + 1, stages)
                                     .total +
                                 fused::align_up(size_t(4) * tile_h * kpad, 128);
                        if (c.smem > smem_cap) continue;
                        c.cost = model_cost_tc(c, C, kpad, nmb, esz, asz);
                        out.push_back(c);
                    }
                }
            }
        }
        return out;
    }
    for (int G : {4, 2, 1}) {
        const fused::Variant *var = find_variant(dt, C, G);
        if (!var) continue;
        const int V = var->V;
        const int J = std::max(band_needed(sy, G, p->gy.t_eff), band_needed(sx, G, p->gx.t_eff));
        if (J > 256) continue;
        const std::vector<int32_t> by = group_bases(sy, G, J, p->gy.n_in, p->gy.t_eff);
        const std::vector<int32_t> bx = group_bases(sx, G, J, p->gx.n_in, p->gx.t_eff);
        const int max_h = int(std::min<int64_t>(64, (p->gy.n_out + G - 1) / G * G));
        for (int tile_h : {8, 16, 32, 64}) {
            if (tile_h % G || tile_h / G > 32) continue;
            if (tile_h > std::max(8, max_h) * 2 && tile_h > 8) continue;
            const int rows = tile_extent(by, tile_h / G, J, 1, 1);
            const int n_sub = (rows + 255) / 256;
            const int sub_h = sub_height(rows, n_sub);
            for (int ngx = 1; ngx <= 32; ++ngx) {
                const int tile_w = ngx * G;
                if (tile_w > ((p->gx.n_out + G - 1) / G) * G && ngx > 1) break;
                const int bw = (tile_extent(bx, ngx, J, C, vec) + vec - 1) / vec * vec;
                if (tma_layout && bw > 256) break;
                if (bw > 4096) break;
                for (int stages : {2, 1}) {
                    if (stages == 2 && !tma_layout) continue;
                    Candidate c;
                    c.G = G;
                    c.J = J;
                    c.tile_h = tile_h;
                    c.tile_w = tile_w;
                    c.stages = stages;
                    c.box_h = n_sub * sub_h;
                    c.box_w = bw;
                    c.n_sub = n_sub;
                    c.sub_h = sub_h;
                    const int w1 = (bw + 32 * V - 1) / (32 * V) * (32 * V);
                    const int dup = p->work_double ? 1 : 2;
                    c.smem = fused::layout(esz, asz, c.box_h, bw, tile_h / G, ngx, band_stride(G * dup, J),
                                           band_stride(2 * G, J), tile_h, w1 | 1, stages)
                                 .total;
                    if (c.smem > smem_cap) continue;
                    c.cost = model_cost(c, C, esz, asz, V);
                    out.push_back(c);
                }
            }
        }
    }
    return out;
}

bool tma_layout_ok(const rs_plan *p)
{
    return ((p->desc.in_row_stride * int64_t(dt_size(p->desc.in_dtype))) % 16) == 0 && encode_fn() != nullptr;
}

// Tensor-core vertical pass for wide antialiasing (16 or more vertical taps)
// on 16-bit storage, or whenever the plan asks for it.
bool use_tc(const rs_plan *p, bool tma_layout)
{
    if (!tc_eligible(p, tma_layout)) return false;
    return (p->desc.flags & RS_FORCE_TC) || p->gy.t_raw >= 16;
}

rs_status choose_fused(rs_plan *p, cudaStream_t stream)
{
    // start tables back to the host (plan creation synchronises once)
    p->host_start_y.resize(p->gy.n_out);
    p->host_start_x.resize(p->gx.n_out);
    cudaError_t e = cudaMemcpyAsync(p->host_start_y.data(), p->ty.start, p->host_start_y.size() * 4,
                                    cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->host_start_x.data(), p->tx.start, p->host_start_x.size() * 4,
                            cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading weight tables");
    const bool tma = tma_layout_ok(p);
    const bool tc = use_tc(p, tma);
    if ((p->desc.flags & RS_FORCE_TC) && !tc)
        return fail(RS_ERR_UNSUPPORTED, "tensor-core path needs F16/BF16 storage, a 16-byte row pitch and rows of "
                                        "whole 8-sample chunks");
    // cheapest modelled configuration first; a tensor-core plan with no
    // feasible tile falls back to the SIMT kernel unless it was forced
    for (int mode = tc ? 1 : 0; mode >= 0; --mode) {
        std::vector<Candidate> cands = enumerate_candidates(p, tma, mode == 1);
        std::stable_sort(cands.begin(), cands.end(),
                         [](const Candidate &a, const Candidate &b) { return a.cost < b.cost; });
        for (const Candidate &c : cands) {
            const rs_status s = apply_fused(p, stream, c, tma);
            if (s != RS_ERR_UNSUPPORTED) return s;
        }
        if (p->desc.flags & RS_FORCE_TC) return fail(RS_ERR_UNSUPPORTED, "no tensor-core tile fits this plan");
    }
    return RS_ERR_UNSUPPORTED;
}

rs_status encode_tensor_map(const rs_plan *p, const void *d_in, CUtensorMap *map)
{
    const rs_plan_desc &d = p->desc;
    CUtensorMapDataType t = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    switch (d.in_dtype) {
    case RS_F64: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
    case RS_F32: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    case RS_F16: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
    case RS_BF16: t = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
    }
    const size_t esz = dt_size(d.in_dtype);
    CUresult r;
    if (p->chosen.tc) {
        // {8 samples, rows, 8-sample chunks}: the box lands in the tensor cores'
        // canonical MN-major layout (rows 16 bytes apart, chunks rows*16 apart)
        const int64_t row = p->gx.n_in * d.channels;
        cuuint64_t dims[3] = {8, cuuint64_t(p->gy.n_in), cuuint64_t((row + 7) / 8)};
        cuuint64_t strides[2] = {cuuint64_t(d.in_row_stride * int64_t(esz)), 16};
        cuuint32_t box[3] = {8, cuuint32_t(p->fp.tc_kpad), cuuint32_t(p->fp.box_w / 8)};
        cuuint32_t estr[3] = {1, 1, 1};
        r = encode_fn()(map, t, 3, const_cast<void *>(d_in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        cuuint64_t dims[2] = {cuuint64_t(p->gx.n_in * d.channels), cuuint64_t(p->gy.n_in)};
        cuuint64_t strides[1] = {cuuint64_t(d.in_row_stride * int64_t(esz))};
        cuuint32_t box[2] = {cuuint32_t(p->fp.box_w), cuuint32_t(p->fp.sub_h)};
        cuuint32_t estr[2] = {1, 1};
        r = encode_fn()(map, t, 2, const_cast<void *>(d_in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d)", int(r));
        return fail(RS_ERR_CUDA, buf);
    }
    return RS_OK;
}

rs_status encode_map(rs_plan *p, const void *d_in)
{
    if (p->tmap_ptr == d_in) return RS_OK;
    rs_status s = encode_tensor_map(p, d_in, &p->tmap);
    if (s != RS_OK) return s;
    p->tmap_ptr = d_in;
    return RS_OK;
}

void work_regions(const rs_plan *p, fused::Work *w)
{
    const fused::Params &fp = p->fp;
    const size_t esz = dt_size(p->desc.in_dtype), asz = p->work_double ? 8 : 4;
    const fused::Layout L = fused::layout(esz, asz, fp.box_h, fp.box_w, fp.tile_h / p->G, fp.tile_w / p->G,
                                          fp.js_y, fp.js_x, fp.tile_h, fp.pitch_t, 1);
    w->tin_bytes = int32_t(L.tin);
    w->wy_bytes = int32_t(L.wy);
    w->wx_bytes = int32_t(L.wx);
    w->tt_bytes = int32_t(L.tt);
    w->rec2_bytes = int32_t(L.rec2);
}

fused::Work single_work(const rs_plan *p, int use_tma)
{
    fused::Work w;
    std::memset(&w, 0, sizeof w);
    const fused::Params &fp = p->fp;
    w.n_images = 1;
    w.total_tiles = fp.tiles_y * fp.tiles_x;
    work_regions(p, &w);
    w.stages = use_tma ? fp.stages : 1;
    w.n1 = fp.n1;
    w.use_tma = use_tma;
    if (p->chosen.tc) {
        w.tc_b_bytes = int32_t(4 * fp.tile_h * fp.tc_kpad);
        int cols = 32;
        while (cols < fp.tc_nmb * fp.tile_h) cols <<= 1;
        w.tc_cols = cols;
    }
    return w;
}

// ---------------------------------------------------------------- autotuner

std::string tune_key(const rs_plan *p)
{
    cudaDeviceProp prop;
    std::string dev = "unknown";
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) dev = prop.name;
    for (char &ch : dev)
        if (ch == '"' || ch == '|') ch = '_';
    const rs_plan_desc &d = p->desc;
    char buf[320];
    std::snprintf(buf, sizeof buf, "%s|v1|dt%d|c%d|k%d|p%.17g|b%d|f%u|%dx%d->%dx%d|is%lld|tc%d", dev.c_str(),
                  d.in_dtype, d.channels, d.kernel, d.param, d.boundary, d.flags & RS_NO_ANTIALIAS, d.in_h, d.in_w,
                  d.out_h, d.out_w, (long long)d.in_row_stride, p->chosen.tc);
    return buf;
}

bool cache_lookup(const char *path, const std::string &key, int *G, int *th, int *tw, int *st, int *n1,
                  int *use_stream, int *tc, int *vf, int *tp)
{
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    const std::string needle = "\"key\": \"" + key + "\"";
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        if (!std::strstr(line, needle.c_str())) continue;
        const char *q = std::strstr(line, "\"G\":");
        if (q && std::sscanf(q, "\"G\": %d, \"tile_h\": %d, \"tile_w\": %d, \"stages\": %d, \"n1\": %d", G, th, tw,
                             st, n1) == 5) {
            found = true; // the last matching line wins
            const char *r = std::strstr(line, "\"stream\":");
            *use_stream = (r && std::sscanf(r, "\"stream\": %d", use_stream) == 1) ? *use_stream : 0;
            const char *t = std::strstr(line, "\"tc\":");
            *tc = (t && std::sscanf(t, "\"tc\": %d", tc) == 1) ? *tc : -1; // -1: the plan's own choice
            const char *v = std::strstr(line, "\"vfirst\":");
            *vf = (v && std::sscanf(v, "\"vfirst\": %d", vf) == 1) ? *vf : 0;
            const char *w = std::strstr(line, "\"two_pass\":");
            *tp = (w && std::sscanf(w, "\"two_pass\": %d", tp) == 1) ? *tp : 0;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const Candidate &c, double us, int use_stream, int vf,
                 int tp)
{
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"key\": \"%s\", \"G\": %d, \"tile_h\": %d, \"tile_w\": %d, \"stages\": %d, \"n1\": %d, "
                 "\"band\": %d, \"us\": %.3f, \"stream\": %d, \"tc\": %d, \"vfirst\": %d, \"two_pass\": %d}\n",
                 key.c_str(), c.G, c.tile_h, c.tile_w, c.stages, c.n1, c.J, us, use_stream, c.tc, vf, tp);
    std::fclose(f);
}

// The two-pass path's intermediate (in_h x out_w x C samples of the
// accumulation type), allocated on first use.
rs_status ensure_two_pass_tmp(rs_plan *p)
{
    if (p->tmp.p) return RS_OK;
    const size_t bytes =
        size_t(p->desc.in_h) * size_t(p->desc.out_w) * size_t(p->desc.channels) * (p->work_double ? 8 : 4);
    const cudaError_t e = cudaMalloc(&p->tmp.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        p->tmp.p = nullptr;
        return RS_ERR_OOM;
    }
    p->tmp.n = bytes;
    p->scratch_bytes += int64_t(bytes);
    return RS_OK;
}

void release_two_pass_tmp(rs_plan *p)
{
    if (!p->tmp.p) return;
    p->scratch_bytes -= int64_t(p->tmp.n);
    p->tmp.~DeviceBuf();
    new (&p->tmp) DeviceBuf();
}

// Mean launch time (µs) of the plan's current configuration.
rs_status time_plan(rs_plan *p, const void *d_in, void *d_out, cudaStream_t s, double *us);

} // namespace rs

extern "C" {

const char *rs_status_string(rs_status s)
{
    switch (s) {
    case RS_OK: return "ok";
    case RS_ERR_INVALID_ARG: return "invalid argument";
    case RS_ERR_UNSUPPORTED: return "unsupported";
    case RS_ERR_OOM: return "out of device memory";
    case RS_ERR_BUDGET: return "memory budget exceeded";
    case RS_ERR_CUDA: return "CUDA error";
    case RS_ERR_TIMEOUT: return "timeout";
    case RS_ERR_BUSY: return "busy";
    case RS_ERR_DEVICE: return "device-side check failed";
    }
    return "unknown status";
}

const char *rs_last_error(void) { return g_last_error.c_str(); }

int32_t rs_version(void) { return 1; }

rs_status rs_desc_out_size(const rs_plan_desc *desc, int32_t *out_h, int32_t *out_w)
{
    if (!desc || !out_h || !out_w) return fail(RS_ERR_INVALID_ARG, "NULL argument");
    rs_plan_desc d;
    const rs_status s = validate_desc(*desc, &d);
    if (s != RS_OK) return s;
    *out_h = d.out_h;
    *out_w = d.out_w;
    return RS_OK;
}

rs_status rs_plan_create(const rs_plan_desc *desc, void *stream_v, rs_plan **out)
{
    const Range range("rs_plan_create");
    if (!out) return fail(RS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(RS_ERR_INVALID_ARG, "desc is NULL");
    rs_plan_desc d = *desc;
    const int64_t ef = env_plan_flags();
    if (ef < 0) return fail(RS_ERR_INVALID_ARG, "RS_PLAN_FLAGS names an unknown flag");
    d.flags |= uint32_t(ef);
    const rs_status vs = validate_desc(d, &d);
    if (vs != RS_OK) return vs;

    rs_plan *p = new (std::nothrow) rs_plan();
    if (!p) return fail(RS_ERR_OOM, "host allocation failed");
    p->desc = d;
    std::string why;
    if (!axis_setup(p->gy, d.in_h, d.out_h, d, why) || !axis_setup(p->gx, d.in_w, d.out_w, d, why)) {
        delete p;
        return fail(RS_ERR_UNSUPPORTED, why);
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "querying the device");
    }
    p->work_double = d.in_dtype == RS_F64 ? 1 : 0;
    const size_t wsz = p->work_double ? 8 : 4;

    // weight tables of both axes and the error word, one allocation; identical
    // axes (same sizes, kernel, boundary) share one set of tables
    const AxisGeom &ga = p->gy, &gb = p->gx;
    p->axes_alias = (ga.n_in == gb.n_in && ga.n_out == gb.n_out && ga.D == gb.D && ga.R == gb.R &&
                     ga.t_raw == gb.t_raw && ga.t_eff == gb.t_eff && ga.kernel == gb.kernel &&
                     ga.boundary == gb.boundary && ga.param == gb.param)
                        ? 1
                        : 0;
    Carver cv;
    const size_t o_err = cv.take(16);
    size_t o[2][5];
    for (int a = 0; a < 2 - p->axes_alias; ++a) {
        const AxisGeom &g = a == 0 ? p->gy : p->gx;
        o[a][0] = cv.take(size_t(g.n_out) * 4);
        o[a][1] = cv.take(size_t(g.n_out) * 4);
        o[a][2] = cv.take(size_t(g.n_out) * 4);
        // (the weight tables get 4 spare rows: kernels that read outputs in
        // groups of 4 may read a last group's missing members)
        o[a][3] = cv.take(size_t(g.n_out + 4) * g.t_eff * 8);
        o[a][4] = cv.take(size_t(g.n_out + 4) * g.t_eff * wsz);
    }
    e = cudaMalloc(&p->tables.p, cv.off);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "allocating weight tables");
    }
    p->tables.n = cv.off;
    char *base = static_cast<char *>(p->tables.p);
    p->d_err = reinterpret_cast<int *>(base + o_err);
    for (int a = 0; a < 2; ++a) {
        AxisTables &t = a == 0 ? p->ty : p->tx;
        const int b = p->axes_alias ? 0 : a;
        t.jlo = reinterpret_cast<int32_t *>(base + o[b][0]);
        t.cnt = reinterpret_cast<int32_t *>(base + o[b][1]);
        t.start = reinterpret_cast<int32_t *>(base + o[b][2]);
        t.w64 = reinterpret_cast<double *>(base + o[b][3]);
        t.wwork = base + o[b][4];
    }
    e = cudaMemsetAsync(p->tables.p, 0, p->tables.n, stream); // error word and spare rows start at zero
    if (e == cudaSuccess) e = launch_plan_weights(p, stream);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "weight kernel launch");
    }

    rs_status st = RS_ERR_UNSUPPORTED;
    const bool fusable = !(d.flags & RS_TWO_PASS) && (d.channels == 1 || d.channels == 3);
    if ((d.flags & RS_FORCE_TC) && !fusable) {
        delete p;
        return fail(RS_ERR_UNSUPPORTED, "tensor-core path needs the fused kernel (1 or 3 channels, no RS_TWO_PASS)");
    }
    if (fusable) {
        st = choose_fused(p, stream);
        if (st != RS_OK && (st != RS_ERR_UNSUPPORTED || (d.flags & RS_FORCE_TC))) {
            delete p;
            return st;
        }
    }
    if (st == RS_OK) {
        p->path = 0;
        // the row-streaming kernel, where it applies, replaces the tile kernel
        // (which stays configured for inputs it cannot take)
        // (a 16-bit wide downscale keeps its tensor-core tiles unless the
        // streaming kernel is forced; the autotuner times both)
        const rs_status ss = stream::setup(p, stream);
        if (ss == RS_OK) {
            // (the tensor-core downscale form is itself a tensor-core kernel)
            p->use_stream =
                (!p->chosen.tc || (d.flags & RS_FORCE_STREAM) || (p->tcs_on && !(d.flags & RS_FORCE_TC))) ? 1 : 0;
        } else if (ss != RS_ERR_UNSUPPORTED) {
            delete p;
            return ss;
        }
    }
    if ((d.flags & RS_FORCE_STREAM) && !p->stream_ok) {
        delete p;
        return fail(RS_ERR_UNSUPPORTED, "row-streaming kernel needs FP32, FP16 or BF16, 1 or 3 channels, a 16-byte row pitch, "
                                        "a horizontal band of at most 40 and a vertical band of at most 32 inputs");
    }
    if (d.flags & RS_FORCE_VFIRST) {
        const rs_status vs = vfirst::setup(p, stream);
        if (vs != RS_OK) {
            delete p;
            return vs == RS_ERR_UNSUPPORTED
                       ? fail(RS_ERR_UNSUPPORTED, "vertical-first path needs FP32, FP16 or BF16, 1 or 3 channels, "
                                                  "out_h <= in_h and bands of at most 256 inputs")
                       : vs;
        }
        p->use_vfirst = 1;
        p->use_stream = 0;
    }
    if (st != RS_OK) {
        p->path = 1;
    }
    if (st != RS_OK && !p->use_vfirst) {
        const size_t bytes = size_t(d.in_h) * size_t(d.out_w) * size_t(d.channels) * wsz;
        e = cudaMalloc(&p->tmp.p, bytes);
        if (e != cudaSuccess) {
            delete p;
            return cuda_fail(e, "allocating the two-pass intermediate");
        }
        p->tmp.n = bytes;
    }
    if (d.flags & RS_PREFILTER) {
        const rs_status ps = prefilter::setup(p);
        if (ps != RS_OK) {
            delete p;
            return ps;
        }
        p->prefilter = 1;
    }
    // read the error word once: a failing table means a bad plan
    int herr = 0;
    e = cudaMemcpyAsync(&herr, p->d_err, 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "plan synchronisation");
    }
    if (herr != 0) {
        delete p;
        char buf[64];
        std::snprintf(buf, sizeof buf, "weight-table kernel reported %d", herr);
        return fail(RS_ERR_DEVICE, buf);
    }
    p->scratch_bytes = int64_t(p->tables.n + p->bands.n + p->tmp.n);
    *out = p;
    return RS_OK;
}

rs_status rs_resample(rs_plan *p, const void *d_in, void *d_out, void *stream_v)
{
    const Range range("rs_resample");
    if (!p || !d_in || !d_out) return fail(RS_ERR_INVALID_ARG, "NULL plan or buffer");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    const rs_plan_desc &d = p->desc;
    cudaError_t e;
    if (p->prefilter) {
        // the resampling kernels read the B-spline coefficients instead
        const rs_status ps = prefilter::launch(p, d_in, stream);
        if (ps != RS_OK) return ps;
        d_in = p->coef;
    }
    if (d.flags & RS_CHECK) {
        e = launch_table_check(p, stream);
        if (e != cudaSuccess) return cuda_fail(e, "table check launch");
    }
    if (p->use_vfirst) return vfirst::launch(p, d_in, d_out, stream);
    if (p->path == 0) {
        fused::Params fp = p->fp;
        fp.in = d_in;
        fp.out = d_out;
        fp.use_tma = (p->tma_ok && (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0) ? 1 : 0;
        if (p->chosen.tc && !fp.use_tma)
            return fail(RS_ERR_INVALID_ARG, "tensor-core plan: the input must be 16-byte aligned");
        if (p->use_stream && fp.use_tma) return stream::launch(p, d_in, d_out, stream);
        if (p->tile_bands_stale) {
            e = launch_band(weight_args(p, 0), weight_args(p, 1), stream);
            if (e != cudaSuccess) return cuda_fail(e, "band kernel launch");
            p->tile_bands_stale = 0;
        }
        size_t smem = p->smem;
        if (fp.use_tma) {
            rs_status s = encode_map(p, d_in);
            if (s != RS_OK) return s;
        } else {
            fp.stages = 1;
        }
        fused::Work w = single_work(p, fp.use_tma);
        void *args[3] = {&p->tmap, &fp, &w};
        e = cudaLaunchKernel(p->kernel_fn, dim3(p->grid), dim3(fused::kThreads), args, smem, stream);
        if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
        return RS_OK;
    }
    TwoPassArgs a;
    a.in = d_in;
    a.out = d_out;
    a.tmp = p->tmp.p;
    a.in_h = d.in_h;
    a.in_w = d.in_w;
    a.out_h = d.out_h;
    a.out_w = d.out_w;
    a.C = d.channels;
    a.in_stride = d.in_row_stride;
    a.out_stride = d.out_row_stride;
    a.start_x = p->tx.start;
    a.start_y = p->ty.start;
    a.w_x = p->tx.wwork;
    a.w_y = p->ty.wwork;
    a.t_x = p->gx.t_eff;
    a.t_y = p->gy.t_eff;
    a.dtype = d.in_dtype;
    e = launch_two_pass(a, stream);
    if (e != cudaSuccess) return cuda_fail(e, "two-pass launch");
    return RS_OK;
}

rs_status rs_plan_autotune(rs_plan *p, const void *d_in, void *d_out, void *stream_v, const char *cache_path)
{
    const Range range("rs_plan_autotune");
    if (!p || !d_in || !d_out) return fail(RS_ERR_INVALID_ARG, "NULL plan or buffer");
    if (p->path != 0) return RS_OK; // only the fused path has choices to tune
    if (p->desc.flags & RS_FORCE_VFIRST) return RS_OK; // a forced kernel has nothing to choose
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    const bool tma = tma_layout_ok(p);
    const bool tc = p->chosen.tc != 0, force_tc = (p->desc.flags & RS_FORCE_TC) != 0;
    // a tensor-core plan also times the SIMT tiles (and the streaming kernel)
    // unless the tensor cores were forced
    std::vector<Candidate> cands = enumerate_candidates(p, tma, tc);
    if (tc && !force_tc) {
        const std::vector<Candidate> simt = enumerate_candidates(p, tma, false);
        cands.insert(cands.end(), simt.begin(), simt.end());
    }
    if (cands.empty()) return RS_OK;
    const std::string key = tune_key(p);
    // the tile configurations are timed on the tile kernel; the streaming
    // kernel (if any) is compared with the winner at the end
    const int stream_ok = p->stream_ok && !force_tc;
    p->use_stream = 0;
    p->use_vfirst = 0;
    // the vertical-first kernels are a candidate unless another kernel is forced
    const bool vf_try = !(p->desc.flags & (RS_FORCE_TC | RS_FORCE_STREAM));
    // the two-pass path (H then V through HBM) likewise
    const bool tp_try = !(p->desc.flags & (RS_FORCE_TC | RS_FORCE_STREAM));
    int G, th, tw, st, n1, us_cached = 0, tc_cached = -1, vf_cached = 0, tp_cached = 0;
    if (cache_lookup(cache_path, key, &G, &th, &tw, &st, &n1, &us_cached, &tc_cached, &vf_cached, &tp_cached)) {
        for (const Candidate &c : cands)
            if (c.G == G && c.tile_h == th && c.tile_w == tw && c.stages == st &&
                (tc_cached < 0 ? c.tc == int(tc) : c.tc == tc_cached)) {
                Candidate k = c;
                k.n1 = n1;
                const rs_status s2 = apply_fused(p, stream, k, tma);
                if (s2 != RS_OK) return s2;
                if (stream_ok && us_cached) {
                    // the cached streaming configuration
                    const rs_status s3 = stream::setup(p, stream, stream::Opts::decode(us_cached));
                    if (s3 != RS_OK && s3 != RS_ERR_UNSUPPORTED) return s3;
                    p->use_stream = s3 == RS_OK ? 1 : 0;
                }
                if (vf_cached && vf_try) {
                    const rs_status s4 = p->vfirst_ok ? RS_OK : vfirst::setup(p, stream);
                    if (s4 != RS_OK && s4 != RS_ERR_UNSUPPORTED) return s4;
                    p->use_vfirst = s4 == RS_OK ? 1 : 0;
                }
                if (tp_cached && tp_try && ensure_two_pass_tmp(p) == RS_OK) {
                    p->path = 1;
                    p->use_stream = 0;
                    p->use_vfirst = 0;
                    p->tile_bands_stale = 1;
                }
                return RS_OK;
            }
    }
    const Candidate before = p->chosen;
    // Stage 1: per (G, tile_h, stages) the widest feasible tile and two
    // narrower ones, warp split from the model.
    std::vector<Candidate> trial;
    for (size_t i = 0; i < cands.size(); ++i) {
        const Candidate &c = cands[i];
        int widest = 0;
        for (const Candidate &o : cands)
            if (o.G == c.G && o.tile_h == c.tile_h && o.stages == c.stages && o.tc == c.tc)
                widest = std::max(widest, o.tile_w);
        const int ng = widest / c.G;
        const int a = std::max(1, (2 * ng + 2) / 3), b = std::max(1, (ng + 2) / 3);
        const int g = c.tile_w / c.G;
        if (g == ng || g == a || g == b) trial.push_back(c);
    }
    Candidate best = before;
    double best_us = 1e300;
    std::vector<std::pair<double, Candidate>> scored;
    for (const Candidate &c : trial) {
        rs_status s = apply_fused(p, stream, c, tma);
        if (s != RS_OK) continue;
        double us = 0;
        s = time_plan(p, d_in, d_out, stream, &us);
        if (s != RS_OK) return s;
        scored.push_back({us, c});
        if (us < best_us) {
            best_us = us;
            best = c;
        }
    }
    // Stage 2: every warp split for the four fastest.
    std::sort(scored.begin(), scored.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
    for (size_t r = 0; r < scored.size() && r < 4; ++r) {
        if (scored[r].second.tc) continue; // the tensor-core warp split is fixed
        for (int k1 = 1; k1 < fused::kWarps; ++k1) {
            Candidate c = scored[r].second;
            if (c.n1 == k1) continue;
            c.n1 = k1;
            if (apply_fused(p, stream, c, tma) != RS_OK) continue;
            double us = 0;
            rs_status s = time_plan(p, d_in, d_out, stream, &us);
            if (s != RS_OK) return s;
            if (us < best_us) {
                best_us = us;
                best = c;
            }
        }
    }
    rs_status s = apply_fused(p, stream, best, tma);
    if (s != RS_OK) return s;
    int stream_choice = 0;
    if (stream_ok) {
        // tile winner against the streaming configurations
        double us_tile = 0;
        s = time_plan(p, d_in, d_out, stream, &us_tile);
        if (s != RS_OK) return s;
        // {form (0 band kernels, 1 pipelined, 2 tensor-core downscale), warp-specialised,
        //  horizontal warps, staged blocks (chunks), L2 prefetch, unused, vertical warps}
        const int cands_s[][7] = {{0, 0, 0, 3, 0, 0, 0}, {0, 0, 0, 2, 0, 0, 0}, {0, 1, 4, 3, 0, 0, 0},
                                  {0, 1, 4, 2, 0, 0, 0}, {0, 1, 3, 3, 0, 0, 0}, {0, 1, 5, 3, 0, 0, 0},
                                  {0, 1, 5, 2, 0, 0, 0}, {1, 0, 4, 2, 0, 0, 4}, {1, 0, 4, 2, 0, 0, 3},
                                  {1, 0, 5, 2, 0, 0, 4}, {1, 0, 4, 2, 0, 0, 5}, {1, 0, 3, 2, 0, 0, 4},
                                  {1, 0, 4, 3, 0, 0, 4}, {1, 0, 7, 2, 0, 0, 8}, {1, 0, 8, 2, 0, 0, 7},
                                  {2, 0, 0, 4, 0, 0, 4}, {2, 0, 0, 4, 0, 0, 6}, {2, 0, 0, 4, 0, 0, 8},
                                  {2, 0, 0, 4, 0, 0, 10}, {2, 0, 0, 3, 0, 0, 6}, {2, 0, 0, 6, 0, 0, 6},
                                  {2, 0, 0, 4, 1, 0, 8}, {2, 0, 0, 4, 1, 0, 10}};
        const bool x_ok = xstream::eligible(p), t_ok = tcstream::eligible(p);
        double best_s = 1e300;
        int best_code = 0;
        for (const auto &c : cands_s) {
            if ((c[0] == 1 && !x_ok) || (c[0] == 2 && !t_ok)) continue;
            stream::Opts o;
            o.ex = c[0];
            o.ws = c[1];
            o.hw = c[2];
            o.ni_min = c[3];
            o.pf = c[4];
            o.vw = c[6];
            // the cost model's three best strip widths for this configuration
            int w[3];
            const int nw = stream::widths(p, o, w, 3);
            for (int i = 0; i < nw; ++i) {
                o.sw = w[i];
                const rs_status ss = stream::setup(p, stream, o);
                if (ss == RS_ERR_UNSUPPORTED) continue;
                if (ss != RS_OK) return ss;
                p->use_stream = 1;
                double us = 0;
                s = time_plan(p, d_in, d_out, stream, &us);
                if (s != RS_OK) return s;
                if (us < best_s) {
                    best_s = us;
                    best_code = p->stream_code;
                }
            }
        }
        p->use_stream = 0;
        if (best_code && (best_s < us_tile || (p->desc.flags & RS_FORCE_STREAM))) {
            s = stream::setup(p, stream, stream::Opts::decode(best_code));
            if (s != RS_OK) return s;
            p->use_stream = 1;
            stream_choice = best_code;
        } else if (best_code) {
            // keep a streaming configuration for an explicit switch back
            stream::setup(p, stream, stream::Opts::decode(best_code));
        }
        best_us = std::min(us_tile, best_s);
    }
    // the vertical-first kernels against the winner so far
    int vf_choice = 0;
    if (vf_try) {
        if (best_us >= 1e299) {
            s = time_plan(p, d_in, d_out, stream, &best_us);
            if (s != RS_OK) return s;
        }
        const rs_status s4 = p->vfirst_ok ? RS_OK : vfirst::setup(p, stream);
        if (s4 != RS_OK && s4 != RS_ERR_UNSUPPORTED) return s4;
        if (s4 == RS_OK) {
            p->use_vfirst = 1;
            double us_vf = 0;
            s = time_plan(p, d_in, d_out, stream, &us_vf);
            if (s != RS_OK) return s;
            if (us_vf < best_us) {
                best_us = us_vf;
                vf_choice = 1;
            } else {
                // not kept: release its intermediate
                p->use_vfirst = 0;
                p->vfirst_ok = 0;
                p->vbufs.~DeviceBuf();
                new (&p->vbufs) DeviceBuf();
            }
        }
    }
    // the two-pass path against the winner so far (it wins on small problems
    // whose work is too little to fill the GPU in tiles, e.g. FP64 256x256)
    int tp_choice = 0;
    if (tp_try) {
        if (best_us >= 1e299) {
            s = time_plan(p, d_in, d_out, stream, &best_us);
            if (s != RS_OK) return s;
        }
        if (ensure_two_pass_tmp(p) == RS_OK) {
            const int keep_stream = p->use_stream, keep_vfirst = p->use_vfirst;
            p->path = 1;
            p->use_stream = 0;
            p->use_vfirst = 0;
            double us_tp = 0;
            s = time_plan(p, d_in, d_out, stream, &us_tp);
            if (s != RS_OK) return s;
            if (us_tp < best_us) {
                best_us = us_tp;
                tp_choice = 1;
                stream_choice = 0;
                p->tile_bands_stale = 1;
                if (vf_choice) {
                    vf_choice = 0;
                    p->vfirst_ok = 0;
                    p->vbufs.~DeviceBuf();
                    new (&p->vbufs) DeviceBuf();
                }
            } else {
                p->path = 0;
                p->use_stream = keep_stream;
                p->use_vfirst = keep_vfirst;
                release_two_pass_tmp(p);
            }
        }
    }
    if (best_us < 1e299) cache_store(cache_path, key, best, best_us, stream_choice, vf_choice, tp_choice);
    return RS_OK;
}

rs_status rs_plan_set_stream_form(rs_plan *p, const rs_stream_form *f, void *stream_v)
{
    if (!p || !f) return fail(RS_ERR_INVALID_ARG, "NULL plan or form");
    if (f->kind == 3) {
        // the tensor-core downscale: staged chunks (2..6) and vertical warps (1..8); no other choice
        if (f->h_warps || (f->prefetch != 0 && f->prefetch != 1) || f->row_ranges || f->strip_width ||
            f->staged_blocks < 0 ||
            f->staged_blocks == 1 || f->staged_blocks > tcstream::kMaxNA || f->v_warps < 0 ||
            f->v_warps > tcstream::kMaxVW)
            return fail(RS_ERR_INVALID_ARG, "malformed streaming form");
    } else if (f->kind < 0 || f->kind > 2 || f->h_warps < 0 || f->h_warps > 8 || (f->kind != 2 && f->h_warps > 6) ||
        f->v_warps < 0 || f->v_warps > 12 || (f->v_warps && f->kind != 2) || f->h_warps + f->v_warps > 15 ||
        f->row_ranges < 0 || f->row_ranges > 255 ||
        (f->row_ranges && f->kind != 2) || f->staged_blocks < 0 ||
        f->staged_blocks > 4 || (f->staged_blocks > 0 && f->staged_blocks < 2) || f->strip_width < 0 ||
        f->strip_width > 252 || f->strip_width % 4 || (f->prefetch != 0 && f->prefetch != 1) ||
        (f->prefetch && f->kind != 2))
        return fail(RS_ERR_INVALID_ARG, "malformed streaming form");
    if (p->path != 0 || p->prefilter)
        return fail(RS_ERR_UNSUPPORTED, "the plan has no fused path for the streaming kernel");
    stream::Opts o;
    o.ex = f->kind == 3 ? 2 : f->kind == 2 ? 1 : 0;
    o.ws = f->kind == 1 ? 1 : 0;
    o.hw = f->h_warps;
    if (f->kind == 1 && f->h_warps == 1) return fail(RS_ERR_INVALID_ARG, "kind 1 takes 2..6 horizontal warps");
    o.ni_min = f->staged_blocks ? f->staged_blocks : (f->kind == 2 ? 2 : f->kind == 3 ? 0 : 3);
    o.sw = f->strip_width;
    o.pf = f->prefetch;
    o.vw = f->v_warps;
    o.nr = f->row_ranges;
    // keep the previous configuration if the form cannot apply
    const int keep_code = p->stream_ok ? p->stream_code : 0, keep_use = p->use_stream;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    const rs_status s = stream::setup(p, stream, o);
    if (s != RS_OK) {
        if (keep_code) stream::setup(p, stream, stream::Opts::decode(keep_code));
        p->use_stream = keep_use;
        return s == RS_ERR_UNSUPPORTED ? fail(s, "the plan cannot take this streaming form") : s;
    }
    p->use_stream = 1;
    p->use_vfirst = 0;
    return RS_OK;
}

rs_status rs_plan_get_stream_form(const rs_plan *p, rs_stream_form *f)
{
    if (!p || !f) return fail(RS_ERR_INVALID_ARG, "NULL plan or form");
    if (!p->stream_ok) return fail(RS_ERR_UNSUPPORTED, "the plan has no streaming configuration");
    const stream::Opts o = stream::Opts::decode(p->stream_code);
    if (p->tcs_on) {
        f->kind = 3;
        f->h_warps = 0;
        f->staged_blocks = p->tcp.NA;
        f->strip_width = p->tcp.NP;
        f->prefetch = p->tcp.pf ? 1 : 0;
        f->v_warps = p->tcp.VW;
        f->row_ranges = 0;
        return RS_OK;
    }
    f->kind = o.ex > 0 ? 2 : (o.ws > 0 ? 1 : 0);
    f->h_warps = p->x_on ? p->xp.HW : (o.ws > 0 ? p->sp.HW : 0);
    f->staged_blocks = p->x_on ? p->xp.NI : p->sp.NI;
    f->strip_width = p->x_on ? p->xp.SW : p->sp.SW;
    f->prefetch = p->x_on ? p->xp.pf : 0;
    f->v_warps = p->x_on ? p->xp.VW : 0;
    f->row_ranges = p->x_on ? (p->xp.groups_y + p->xp.gpr - 1) / p->xp.gpr : 0;
    return RS_OK;
}

rs_status rs_plan_recompute(rs_plan *p, void *stream_v)
{
    const Range range("rs_plan_recompute");
    if (!p) return fail(RS_ERR_INVALID_ARG, "NULL plan");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    cudaError_t e = launch_plan_weights(p, stream);
    if (e != cudaSuccess) return cuda_fail(e, "weight kernel launch");
    if (p->path == 1) {
        // the two-pass kernels read the weight tables directly; the other
        // kernels' bands are rebuilt only if one of them is chosen again
        p->tile_bands_stale = 1;
        return RS_OK;
    }
    if (p->use_vfirst) {
        // the other kernels' bands are rebuilt only if one of them is chosen again
        p->tile_bands_stale = 1;
        if (p->stream_ok) {
            const rs_status s = stream::rebuild(p, stream);
            if (s != RS_OK) return s;
        }
        return vfirst::rebuild(p, stream);
    }
    if (p->vfirst_ok) {
        const rs_status s = vfirst::rebuild(p, stream);
        if (s != RS_OK) return s;
    }
    if (p->path == 0 && p->use_stream) {
        // the tile kernel's bands are rebuilt only if a tile launch needs them
        p->tile_bands_stale = 1;
        return stream::rebuild(p, stream);
    }
    if (p->path == 0) e = launch_band(weight_args(p, 0), weight_args(p, 1), stream);
    if (e != cudaSuccess) return cuda_fail(e, "band kernel launch");
    if (p->stream_ok) return stream::rebuild(p, stream);
    return RS_OK;
}

rs_status rs_destroy(rs_plan *p)
{
    if (!p) return RS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    delete p;
    if (e != cudaSuccess) return cuda_fail(e, "synchronising before destroy");
    return RS_OK;
}

rs_status rs_plan_get_info(const rs_plan *p, rs_plan_info *info)
{
    if (!p || !info) return fail(RS_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof *info);
    info->out_h = p->desc.out_h;
    info->out_w = p->desc.out_w;
    info->taps_h = p->gy.t_raw;
    info->taps_w = p->gx.t_raw;
    info->table_h = p->gy.t_eff;
    info->table_w = p->gx.t_eff;
    info->path = (p->path == 0 && p->chosen.tc) ? 2 : p->path;
    if (p->use_vfirst) {
        info->path = 4;
        info->tile_h = info->tile_w = 0;
        info->group_h = 8; // vertical-first kernels: 8 rows x 4 samples, 4 pixels per thread
        info->group_w = 4;
        info->span_h = p->vf.JV;
        info->span_w = p->vf.JH;
        info->warps_pass1 = 0;
        info->stages = 0;
        info->smem_bytes = 0;
        info->ctas_per_sm = 0;
    } else if (p->path == 0 && p->use_stream && p->tcs_on) {
        info->path = 5;
        info->tile_h = tcstream::kM;   // input rows per tensor-core block
        info->tile_w = p->tcp.NP;      // output pixels per strip
        info->group_h = 1;
        info->group_w = p->tcp.NP;
        info->span_h = p->tcp.Ty;
        info->span_w = p->tcp.Kc / p->desc.channels; // staged input pixels per strip
        info->warps_pass1 = 0;
        info->stages = p->tcp.NA;
        info->smem_bytes = int32_t(p->s_smem);
        info->ctas_per_sm = p->s_ctas;
    } else if (p->path == 0 && p->use_stream && p->x_on) {
        info->path = 3;
        info->tile_h = xstream::kRB;
        info->tile_w = p->xp.SW;
        info->group_h = info->group_w = xstream::kG;
        info->span_h = p->xp.JV;
        info->span_w = p->xp.JH;
        info->warps_pass1 = p->xp.HW; // horizontal warps (vertical: 7 - this)
        info->stages = p->xp.NI;
        info->smem_bytes = int32_t(p->s_smem);
        info->ctas_per_sm = p->s_ctas;
    } else if (p->path == 0 && p->use_stream) {
        info->path = 3;
        info->tile_h = stream::kRB;
        info->tile_w = p->sp.SW;
        info->group_h = p->sp.GV;
        info->group_w = stream::kG;
        info->span_h = p->sp.JV;
        info->span_w = p->sp.JH;
        info->warps_pass1 = 0;
        info->stages = p->sp.NI;
        info->smem_bytes = int32_t(p->s_smem);
        info->ctas_per_sm = p->s_ctas;
    } else if (p->path == 0) {
        info->tile_h = p->fp.tile_h;
        info->tile_w = p->fp.tile_w;
        info->group_h = info->group_w = p->G;
        info->span_h = info->span_w = p->J;
        info->warps_pass1 = p->fp.n1;
        info->stages = p->tma_ok ? p->fp.stages : 1;
        info->smem_bytes = int32_t(p->smem);
        info->ctas_per_sm = p->ctas_per_sm;
    }
    info->scratch_bytes = p->scratch_bytes;
    return RS_OK;
}

rs_status rs_plan_get_tables(const rs_plan *p, int axis, int32_t *h_jlo, int32_t *h_count, int32_t *h_start,
                             double *h_w64, double *h_wwork)
{
    if (!p || (axis != 0 && axis != 1)) return fail(RS_ERR_INVALID_ARG, "bad plan or axis");
    const AxisGeom &g = axis == 0 ? p->gy : p->gx;
    const AxisTables &t = axis == 0 ? p->ty : p->tx;
    cudaError_t e = cudaDeviceSynchronize();
    const size_t n = size_t(g.n_out), te = size_t(g.t_eff);
    if (e == cudaSuccess && h_jlo) e = cudaMemcpy(h_jlo, t.jlo, n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_count) e = cudaMemcpy(h_count, t.cnt, n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_start) e = cudaMemcpy(h_start, t.start, n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_w64) e = cudaMemcpy(h_w64, t.w64, n * te * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_wwork) {
        if (p->work_double) {
            e = cudaMemcpy(h_wwork, t.wwork, n * te * 8, cudaMemcpyDeviceToHost);
        } else {
            std::vector<float> tmp(n * te);
            e = cudaMemcpy(tmp.data(), t.wwork, n * te * 4, cudaMemcpyDeviceToHost);
            for (size_t i = 0; i < tmp.size(); ++i) h_wwork[i] = double(tmp[i]);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "copying tables");
    return RS_OK;
}

rs_status rs_plan_check(rs_plan *p)
{
    if (!p) return fail(RS_ERR_INVALID_ARG, "NULL plan");
    cudaError_t e = cudaDeviceSynchronize();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, p->d_err, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && herr) e = cudaMemset(p->d_err, 0, 4);
    if (e != cudaSuccess) return cuda_fail(e, "checking the device error word");
    if (herr) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "device error word %d%s", herr,
                      herr == fused::kErrTimeout ? " (a bounded device wait ran out)"
                      : herr == fused::kErrCheck ? " (RS_CHECK: a table window or its weights)"
                                                 : "");
        return fail(herr == fused::kErrTimeout ? RS_ERR_TIMEOUT : RS_ERR_DEVICE, buf);
    }
    return RS_OK;
}

rs_status rs_plan_set_weights(rs_plan *p, int32_t axis, const double *h_wwork, void *stream_v)
{
    if (!p || !h_wwork || (axis != 0 && axis != 1)) return fail(RS_ERR_INVALID_ARG, "bad plan, axis or weights");
    if (p->axes_alias) return fail(RS_ERR_UNSUPPORTED, "the plan's two axes share one table (identical geometry)");
    const AxisGeom &g = axis == 0 ? p->gy : p->gx;
    const AxisTables &t = axis == 0 ? p->ty : p->tx;
    const size_t n = size_t(g.n_out) * size_t(g.t_eff);
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    cudaError_t e = cudaSuccess;
    if (p->work_double) {
        e = cudaMemcpyAsync(t.wwork, h_wwork, n * 8, cudaMemcpyHostToDevice, stream);
    } else {
        std::vector<float> w(n);
        for (size_t i = 0; i < n; ++i) w[i] = float(h_wwork[i]);
        e = cudaMemcpyAsync(t.wwork, w.data(), n * 4, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream); // w is released on return
    }
    if (e != cudaSuccess) return cuda_fail(e, "copying weights");
    // the kernels that read bands of these weights get them rebuilt
    if (p->vfirst_ok) {
        const rs_status s = vfirst::rebuild(p, stream);
        if (s != RS_OK) return s;
    }
    if (p->stream_ok) {
        const rs_status s = stream::rebuild(p, stream);
        if (s != RS_OK) return s;
    }
    p->tile_bands_stale = 1;
    return RS_OK;
}

rs_status rs_plan_wait_selftest(rs_plan *p, int32_t limit_us, void *stream_v)
{
    if (!p || limit_us < 1 || limit_us > 2000000) return fail(RS_ERR_INVALID_ARG, "bad plan or limit (1 us .. 2 s)");
    const cudaError_t e = launch_wait_selftest(p->d_err, uint64_t(limit_us) * 1000ull, static_cast<cudaStream_t>(stream_v));
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test launch");
    return RS_OK;
}

} // extern "C"

namespace rs {
rs_status time_plan(rs_plan *p, const void *d_in, void *d_out, cudaStream_t s, double *us)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return cuda_fail(cudaGetLastError(), "event");
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return cuda_fail(cudaGetLastError(), "event");
    }
    rs_status st = rs_resample(p, d_in, d_out, s); // warm-up
    int reps = 3;
    float ms = 0.f;
    cudaError_t e = cudaSuccess;
    for (int round = 0; st == RS_OK && round < 4; ++round) {
        e = cudaEventRecord(a, s);
        for (int r = 0; r < reps && st == RS_OK; ++r) st = rs_resample(p, d_in, d_out, s);
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) break;
        if (ms > 0.3f) break; // long enough to trust
        reps *= 4;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != RS_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "timing");
    // a device-side error during tuning (bounds or a timed-out wait) disqualifies the run
    int herr = 0;
    e = cudaMemcpy(&herr, p->d_err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the error word");
    if (herr) {
        char buf[64];
        std::snprintf(buf, sizeof buf, "device error word %d while tuning", herr);
        return fail(RS_ERR_DEVICE, buf);
    }
    *us = 1000.0 * ms / reps;
    return RS_OK;
}
} // namespace rs
