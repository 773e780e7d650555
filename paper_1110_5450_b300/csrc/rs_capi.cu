// rs_capi.cu -- the C ABI (include/rs.h): plans, geometry, path choice and
// launches.  Host code only; the arithmetic runs in the kernels of
// rs_weights.cu, rs_two_pass.cu and rs_fused*.cu.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "rs_fused.cuh"
#include "rs_internal.h"

namespace rs {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

namespace fused {
const Variant *variants_f64(int *n);
const Variant *variants_f32(int *n);
const Variant *variants_f16(int *n);
const Variant *variants_bf16(int *n);
} // namespace fused

namespace {

const fused::Variant *find_variant(int dtype, int C, int G, int J)
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
        if (v[i].C == C && v[i].G == G && v[i].J == J) return &v[i];
    return nullptr;
}

// Smallest instantiated band width >= j for (dtype, C, G); 0 if none.
int round_band(int dtype, int C, int G, int j)
{
    int n = 0;
    const fused::Variant *v = nullptr;
    switch (dtype) {
    case RS_F64: v = fused::variants_f64(&n); break;
    case RS_F32: v = fused::variants_f32(&n); break;
    case RS_F16: v = fused::variants_f16(&n); break;
    case RS_BF16: v = fused::variants_bf16(&n); break;
    default: return 0;
    }
    int best = 0;
    for (int i = 0; i < n; ++i)
        if (v[i].C == C && v[i].G == G && v[i].J >= j && (best == 0 || v[i].J < best)) best = v[i].J;
    return best;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

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

int support_radius(int kernel, double param)
{
    switch (kernel) {
    case RS_K_LINEAR: return 1;
    case RS_K_CUBIC: return 2;
    case RS_K_BSPLINE3: return 2;
    case RS_K_LANCZOS:
        if (!(param >= 1.0 && param <= 16.0) || param != std::floor(param)) return 0;
        return int(param);
    }
    return 0;
}

struct DeviceBuf {
    void *p = nullptr;
    size_t n = 0;
    ~DeviceBuf()
    {
        if (p) cudaFree(p);
    }
};

// Carve 256-byte aligned pieces out of one allocation.
struct Carver {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    }
};

} // namespace
} // namespace rs

using namespace rs;

struct rs_plan {
    rs_plan_desc desc{};
    int device = 0;
    int num_sms = 0;
    AxisGeom gy, gx;
    AxisTables ty, tx;
    int work_double = 0;
    int path = 1; // 0 fused, 1 two-pass
    DeviceBuf tables, bands, tmp, errbuf;
    int *d_err = nullptr;
    // fused
    fused::Params fp{};
    const fused::Variant *variant = nullptr;
    int G = 0, J = 0;
    size_t smem = 0;
    int grid = 0;
    int tma_ok = 0;
    CUtensorMap tmap;
    const void *tmap_ptr = nullptr;
    int64_t scratch_bytes = 0;
};

namespace {

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

WeightArgs weight_args(rs_plan *p, int axis)
{
    WeightArgs a;
    a.g = axis == 0 ? p->gy : p->gx;
    a.t = axis == 0 ? p->ty : p->tx;
    a.work_is_double = p->work_double;
    a.err = p->d_err;
    return a;
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

rs_status choose_fused(rs_plan *p, cudaStream_t stream)
{
    const rs_plan_desc &d = p->desc;
    const int C = d.channels;
    const int dt = d.in_dtype;
    // start tables back to the host (plan creation synchronises once)
    std::vector<int32_t> sy(p->gy.n_out), sx(p->gx.n_out);
    cudaError_t e = cudaMemcpyAsync(sy.data(), p->ty.start, sy.size() * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sx.data(), p->tx.start, sx.size() * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading weight tables");

    int G = 0, J = 0;
    const int limit[3][2] = {{4, 32}, {2, 48}, {1, 64}};
    for (auto &gl : limit) {
        const int g = gl[0];
        const int need = std::max(band_needed(sy, g, p->gy.t_eff), band_needed(sx, g, p->gx.t_eff));
        if (need > gl[1]) continue;
        const int j = round_band(dt, C, g, need);
        if (j == 0) continue;
        G = g;
        J = j;
        break;
    }
    if (G == 0) return RS_ERR_UNSUPPORTED;
    p->variant = find_variant(dt, C, G, J);
    if (!p->variant) return RS_ERR_UNSUPPORTED;
    p->G = G;
    p->J = J;

    // band tables
    const size_t wsz = p->work_double ? 8 : 4;
    p->ty.G = p->tx.G = G;
    p->ty.J = p->tx.J = J;
    p->ty.groups = int32_t((p->gy.n_out + G - 1) / G);
    p->tx.groups = int32_t((p->gx.n_out + G - 1) / G);
    Carver cv;
    const size_t o_by = cv.take(size_t(p->ty.groups) * 4);
    const size_t o_bx = cv.take(size_t(p->tx.groups) * 4);
    const size_t o_wy = cv.take(size_t(p->ty.groups) * G * J * wsz);
    const size_t o_wx = cv.take(size_t(p->tx.groups) * G * J * wsz);
    e = cudaMalloc(&p->bands.p, cv.off);
    if (e != cudaSuccess) return cuda_fail(e, "allocating band tables");
    p->bands.n = cv.off;
    char *base = static_cast<char *>(p->bands.p);
    p->ty.band_base = reinterpret_cast<int32_t *>(base + o_by);
    p->tx.band_base = reinterpret_cast<int32_t *>(base + o_bx);
    p->ty.band_w = base + o_wy;
    p->tx.band_w = base + o_wx;
    e = launch_band(weight_args(p, 0), weight_args(p, 1), stream);
    if (e != cudaSuccess) return cuda_fail(e, "band kernel launch");
    std::vector<int32_t> by(p->ty.groups), bx(p->tx.groups);
    e = cudaMemcpyAsync(by.data(), p->ty.band_base, by.size() * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bx.data(), p->tx.band_base, bx.size() * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading band tables");

    // tiles
    const size_t esz = dt_size(dt);
    const size_t asz = p->work_double ? 8 : 4;
    const int vec = int(16 / esz);
    const int tile_h = int(std::min<int64_t>(32, ((p->gy.n_out + G - 1) / G) * G));
    const int tile_h_g = std::max(G, tile_h - tile_h % G);
    const int rows = tile_extent(by, tile_h_g / G, J, 1, 1);
    const bool tma_layout = ((d.in_row_stride * int64_t(esz)) % 16) == 0 && encode_fn() != nullptr;
    const size_t smem_cap = 227 * 1024;
    int best_tw = 0, best_stages = 1, best_bw = 0;
    // widest tile whose staged row fits a 256-element TMA box; prefer two stages
    for (int stages = 2; stages >= 1 && best_tw == 0; --stages) {
        for (int ngx = 32; ngx >= 1; --ngx) {
            const int tw = ngx * G;
            if (tw > std::max<int64_t>(G, ((p->gx.n_out + G - 1) / G) * G) && ngx > 1) continue;
            const int bw_need = tile_extent(bx, ngx, J, C, vec);
            const int bw = (bw_need + vec - 1) / vec * vec;
            if (bw > 256) continue;
            const int pt = bw | 1;
            const int n_sub = (rows + 255) / 256;
            const int sub_h = sub_height(rows, n_sub);
            const size_t sm = fused::smem_bytes(esz, asz, n_sub * sub_h, bw, tile_h_g, pt, stages);
            const size_t per_sm_target = stages == 2 ? smem_cap / 2 : smem_cap;
            if (sm > per_sm_target) continue;
            if (tw > 64 * (C == 1 ? 2 : 1)) continue;
            best_tw = tw;
            best_stages = stages;
            best_bw = bw;
            break;
        }
    }
    if (best_tw == 0) return RS_ERR_UNSUPPORTED;

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
    fp.tile_h = tile_h_g;
    fp.tile_w = best_tw;
    fp.n_sub = (rows + 255) / 256;
    fp.sub_h = sub_height(rows, fp.n_sub);
    fp.box_h = fp.n_sub * fp.sub_h;
    fp.box_w = best_bw;
    fp.pitch_t = best_bw | 1;
    fp.groups_y = p->ty.groups;
    fp.groups_x = p->tx.groups;
    fp.tiles_y = int32_t((p->gy.n_out + tile_h_g - 1) / tile_h_g);
    fp.tiles_x = int32_t((p->gx.n_out + best_tw - 1) / best_tw);
    fp.stages = best_stages;
    fp.err = p->d_err;
    p->tma_ok = tma_layout ? 1 : 0;
    p->smem = fused::smem_bytes(esz, asz, fp.box_h, fp.box_w, fp.tile_h, fp.pitch_t, p->tma_ok ? best_stages : 1);
    e = cudaFuncSetAttribute(p->variant->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(p->smem));
    if (e != cudaSuccess) return cuda_fail(e, "setting shared memory size");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, p->variant->fn, fused::kThreads, p->smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (occ < 1) return RS_ERR_UNSUPPORTED;
    const int64_t tiles = int64_t(fp.tiles_y) * fp.tiles_x;
    p->grid = int(std::min<int64_t>(tiles, int64_t(occ) * p->num_sms));
    return RS_OK;
}

rs_status encode_map(rs_plan *p, const void *d_in)
{
    if (p->tmap_ptr == d_in) return RS_OK;
    const rs_plan_desc &d = p->desc;
    CUtensorMapDataType t = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    switch (d.in_dtype) {
    case RS_F64: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
    case RS_F32: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    case RS_F16: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
    case RS_BF16: t = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
    }
    const size_t esz = dt_size(d.in_dtype);
    cuuint64_t dims[2] = {cuuint64_t(p->gx.n_in * d.channels), cuuint64_t(p->gy.n_in)};
    cuuint64_t strides[1] = {cuuint64_t(d.in_row_stride * int64_t(esz))};
    cuuint32_t box[2] = {cuuint32_t(p->fp.box_w), cuuint32_t(p->fp.sub_h)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&p->tmap, t, 2, const_cast<void *>(d_in), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d)", int(r));
        return fail(RS_ERR_CUDA, buf);
    }
    p->tmap_ptr = d_in;
    return RS_OK;
}

} // namespace

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

rs_status rs_plan_create(const rs_plan_desc *desc, void *stream_v, rs_plan **out)
{
    if (!out) return fail(RS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(RS_ERR_INVALID_ARG, "desc is NULL");
    rs_plan_desc d = *desc;
    if (d.in_h < 1 || d.in_w < 1 || d.in_h > kMaxSide || d.in_w > kMaxSide)
        return fail(RS_ERR_INVALID_ARG, "input size out of range");
    if (d.channels < 1 || d.channels > 64) return fail(RS_ERR_INVALID_ARG, "channels must be 1..64");
    if (d.out_h < 0 || d.out_w < 0) return fail(RS_ERR_INVALID_ARG, "negative output size");
    if (d.kernel < RS_K_LINEAR || d.kernel > RS_K_BSPLINE3) return fail(RS_ERR_INVALID_ARG, "unknown kernel");
    if (d.boundary < RS_B_CLAMP || d.boundary > RS_B_TRUNCATE) return fail(RS_ERR_INVALID_ARG, "unknown boundary");
    if (d.in_dtype < RS_F64 || d.in_dtype > RS_BF16 || d.out_dtype < RS_F64 || d.out_dtype > RS_BF16)
        return fail(RS_ERR_INVALID_ARG, "unknown dtype");
    if (d.in_dtype != d.out_dtype) return fail(RS_ERR_UNSUPPORTED, "in_dtype and out_dtype must be equal");
    if (d.flags & ~uint32_t(0x1f)) return fail(RS_ERR_INVALID_ARG, "unknown flag bits");
    if (support_radius(d.kernel, d.param) == 0)
        return fail(RS_ERR_INVALID_ARG, "Lanczos needs an integer R in 1..16");
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
    if (d.flags & RS_FORCE_TC)
        return fail(RS_ERR_UNSUPPORTED, "tensor-core path not available for this plan");

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

    // weight tables of both axes and the error word, one allocation
    Carver cv;
    const size_t o_err = cv.take(16);
    size_t o[2][5];
    for (int a = 0; a < 2; ++a) {
        const AxisGeom &g = a == 0 ? p->gy : p->gx;
        o[a][0] = cv.take(size_t(g.n_out) * 4);
        o[a][1] = cv.take(size_t(g.n_out) * 4);
        o[a][2] = cv.take(size_t(g.n_out) * 4);
        o[a][3] = cv.take(size_t(g.n_out) * g.t_eff * 8);
        o[a][4] = cv.take(size_t(g.n_out) * g.t_eff * wsz);
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
        t.jlo = reinterpret_cast<int32_t *>(base + o[a][0]);
        t.cnt = reinterpret_cast<int32_t *>(base + o[a][1]);
        t.start = reinterpret_cast<int32_t *>(base + o[a][2]);
        t.w64 = reinterpret_cast<double *>(base + o[a][3]);
        t.wwork = base + o[a][4];
    }
    e = cudaMemsetAsync(p->d_err, 0, 16, stream);
    if (e == cudaSuccess) e = launch_weights(weight_args(p, 0), weight_args(p, 1), stream);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "weight kernel launch");
    }

    rs_status st = RS_ERR_UNSUPPORTED;
    const bool fusable = !(d.flags & RS_TWO_PASS) && (d.channels == 1 || d.channels == 3);
    if (fusable) {
        st = choose_fused(p, stream);
        if (st != RS_OK && st != RS_ERR_UNSUPPORTED) {
            delete p;
            return st;
        }
    }
    if (st == RS_OK) {
        p->path = 0;
    } else {
        p->path = 1;
        const size_t bytes = size_t(d.in_h) * size_t(d.out_w) * size_t(d.channels) * wsz;
        e = cudaMalloc(&p->tmp.p, bytes);
        if (e != cudaSuccess) {
            delete p;
            return cuda_fail(e, "allocating the two-pass intermediate");
        }
        p->tmp.n = bytes;
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
    if (!p || !d_in || !d_out) return fail(RS_ERR_INVALID_ARG, "NULL plan or buffer");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    const rs_plan_desc &d = p->desc;
    cudaError_t e;
    if (p->path == 0) {
        fused::Params fp = p->fp;
        fp.in = d_in;
        fp.out = d_out;
        fp.use_tma = (p->tma_ok && (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0) ? 1 : 0;
        size_t smem = p->smem;
        if (fp.use_tma) {
            rs_status s = encode_map(p, d_in);
            if (s != RS_OK) return s;
        } else {
            fp.stages = 1;
        }
        void *args[2] = {&p->tmap, &fp};
        e = cudaLaunchKernel(p->variant->fn, dim3(p->grid), dim3(fused::kThreads), args, smem, stream);
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

rs_status rs_plan_recompute(rs_plan *p, void *stream_v)
{
    if (!p) return fail(RS_ERR_INVALID_ARG, "NULL plan");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    cudaError_t e = launch_weights(weight_args(p, 0), weight_args(p, 1), stream);
    if (e == cudaSuccess && p->path == 0) e = launch_band(weight_args(p, 0), weight_args(p, 1), stream);
    if (e != cudaSuccess) return cuda_fail(e, "weight kernel launch");
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
    info->path = p->path;
    if (p->path == 0) {
        info->tile_h = p->fp.tile_h;
        info->tile_w = p->fp.tile_w;
        info->group_h = info->group_w = p->G;
        info->span_h = info->span_w = p->J;
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
        char buf[64];
        std::snprintf(buf, sizeof buf, "device error word %d", herr);
        return fail(RS_ERR_DEVICE, buf);
    }
    return RS_OK;
}

} // extern "C"
