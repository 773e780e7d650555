// rs_noalloc.cu -- rs_resample_noalloc: resampling without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs this: code that does not own the device's memory -- a plug-in
// running inside a host application whose own allocator manages every byte of
// device memory, or a real-time loop that may not pay for cudaMalloc/cudaFree
// (cudaFree synchronises the whole device).  Such a caller passes its input
// and output buffers and nothing else is allocated on its behalf.
//
// How: the weight tables and the intermediate of the separate H-then-V pass
// kernels live in one file-scope static device array of
// RS_STATIC_SCRATCH_BYTES.  Every GPU that loads this library holds that
// array until the process exits.  Host code cannot use the array's name as an
// address (on the host it is only a stand-in symbol), so the first call on
// each device looks the device address up with cudaGetSymbolAddress while
// that device is current and caches it; that first call should therefore
// happen before any stream capture.
//
// All calls share the one array and it keeps whatever the last call left in
// it: the error word is cleared on every call, and the weight-table kernel
// rewrites every table entry it uses.  Calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array; issue
// them on one stream, one after another.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "rs_internal.h"

namespace rs {
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[RS_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the static array on the current device (set-up on first use).
rs_status static_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("rs_resample_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return RS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("rs_resample_noalloc: device ordinal beyond 63");
        return RS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error(std::string("rs_resample_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return RS_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RS_OK;
}

int radius(int kernel, double param)
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

int64_t out_len(int32_t given, int64_t n, double scale)
{
    if (given > 0) return given;
    if (!(scale > 0.0) || !std::isfinite(scale)) return -1;
    const double v = std::floor(double(n) * scale + 0.5);
    if (!(v < double(kMaxSide) + 1.0)) return -1;
    return v < 1.0 ? 1 : int64_t(v);
}

rs_status bad(rs_status s, const char *msg)
{
    set_error(std::string("rs_resample_noalloc: ") + msg);
    return s;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

} // namespace
} // namespace rs

using namespace rs;

extern "C" rs_status rs_resample_noalloc(const rs_plan_desc *desc, const void *d_in, void *d_out, void *stream_v)
{
    if (!desc || !d_in || !d_out) return bad(RS_ERR_INVALID_ARG, "NULL descriptor or buffer");
    rs_plan_desc d = *desc;
    if (d.in_h < 1 || d.in_w < 1 || d.in_h > kMaxSide || d.in_w > kMaxSide)
        return bad(RS_ERR_INVALID_ARG, "input size out of range");
    if (d.channels < 1 || d.channels > 64) return bad(RS_ERR_INVALID_ARG, "channels must be 1..64");
    if (d.out_h < 0 || d.out_w < 0) return bad(RS_ERR_INVALID_ARG, "negative output size");
    if (d.kernel < RS_K_LINEAR || d.kernel > RS_K_GAUSSIAN) return bad(RS_ERR_INVALID_ARG, "unknown kernel");
    if (d.boundary < RS_B_CLAMP || d.boundary > RS_B_TRUNCATE) return bad(RS_ERR_INVALID_ARG, "unknown boundary");
    if (d.in_dtype < RS_F64 || d.in_dtype > RS_BF16 || d.in_dtype != d.out_dtype)
        return bad(RS_ERR_INVALID_ARG, "dtype unknown or in_dtype != out_dtype");
    if (d.flags & ~uint32_t(0xff)) return bad(RS_ERR_INVALID_ARG, "unknown flag bits");
    const int R = radius(d.kernel, d.param);
    if (R == 0) return bad(RS_ERR_INVALID_ARG, "Lanczos needs an integer R in 1..16");
    const int64_t oh = out_len(d.out_h, d.in_h, d.scale_h), ow = out_len(d.out_w, d.in_w, d.scale_w);
    if (oh < 1 || ow < 1 || oh > kMaxSide || ow > kMaxSide) return bad(RS_ERR_INVALID_ARG, "output size out of range");
    const int64_t in_stride = d.in_row_stride ? d.in_row_stride : int64_t(d.in_w) * d.channels;
    const int64_t out_stride = d.out_row_stride ? d.out_row_stride : ow * d.channels;
    if (in_stride < int64_t(d.in_w) * d.channels || out_stride < ow * d.channels)
        return bad(RS_ERR_INVALID_ARG, "row stride smaller than a row");

    const bool dbl = d.in_dtype == RS_F64;
    const size_t wsz = dbl ? 8 : 4;
    WeightArgs a[2];
    const int64_t n_in[2] = {d.in_h, d.in_w}, n_out[2] = {oh, ow};
    size_t need = up256(16);
    for (int ax = 0; ax < 2; ++ax) {
        AxisGeom &g = a[ax].g;
        g.n_in = n_in[ax];
        g.n_out = n_out[ax];
        g.R = R;
        g.D = (!(d.flags & RS_NO_ANTIALIAS) && g.n_in > g.n_out) ? 2 * g.n_in : 2 * g.n_out;
        const int64_t traw = (g.R * g.D + g.n_out - 1) / g.n_out;
        if (traw > kMaxTaps) return bad(RS_ERR_UNSUPPORTED, "more than 256 taps per output on one axis");
        g.t_raw = int32_t(traw);
        g.t_eff = int32_t(traw < g.n_in ? traw : g.n_in);
        g.kernel = d.kernel;
        g.boundary = d.boundary;
        g.param = d.param;
        need += 3 * up256(size_t(g.n_out) * 4) + up256(size_t(g.n_out) * g.t_eff * 8) +
                up256(size_t(g.n_out) * g.t_eff * wsz);
    }
    const size_t tmp_bytes = size_t(d.in_h) * size_t(ow) * size_t(d.channels) * wsz;
    need += up256(tmp_bytes);
    if (need > size_t(RS_STATIC_SCRATCH_BYTES)) {
        char buf[160];
        std::snprintf(buf, sizeof buf,
                      "rs_resample_noalloc: needs %zu bytes of scratch, the static scratch holds %zu "
                      "(in_h * out_w * channels * %zu bytes plus tables)",
                      need, size_t(RS_STATIC_SCRATCH_BYTES), wsz);
        set_error(buf);
        return RS_ERR_BUDGET;
    }

    void *base_v = nullptr;
    rs_status st = static_scratch(&base_v);
    if (st != RS_OK) return st;
    char *base = static_cast<char *>(base_v);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base + off;
        off += up256(bytes);
        return p;
    };
    int *err = reinterpret_cast<int *>(take(16));
    for (int ax = 0; ax < 2; ++ax) {
        AxisTables &t = a[ax].t;
        const AxisGeom &g = a[ax].g;
        t.jlo = reinterpret_cast<int32_t *>(take(size_t(g.n_out) * 4));
        t.cnt = reinterpret_cast<int32_t *>(take(size_t(g.n_out) * 4));
        t.start = reinterpret_cast<int32_t *>(take(size_t(g.n_out) * 4));
        t.w64 = reinterpret_cast<double *>(take(size_t(g.n_out) * g.t_eff * 8));
        t.wwork = take(size_t(g.n_out) * g.t_eff * wsz);
        a[ax].work_is_double = dbl ? 1 : 0;
        a[ax].err = err;
    }
    void *tmp = take(tmp_bytes);

    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    cudaError_t e = cudaMemsetAsync(err, 0, 16, stream);
    if (e == cudaSuccess) e = launch_weights(a[0], a[1], stream);
    if (e == cudaSuccess) {
        TwoPassArgs tp;
        tp.in = d_in;
        tp.out = d_out;
        tp.tmp = tmp;
        tp.in_h = d.in_h;
        tp.in_w = d.in_w;
        tp.out_h = oh;
        tp.out_w = ow;
        tp.C = d.channels;
        tp.in_stride = in_stride;
        tp.out_stride = out_stride;
        tp.start_x = a[1].t.start;
        tp.start_y = a[0].t.start;
        tp.w_x = a[1].t.wwork;
        tp.w_y = a[0].t.wwork;
        tp.t_x = a[1].g.t_eff;
        tp.t_y = a[0].g.t_eff;
        tp.dtype = d.in_dtype;
        e = launch_two_pass(tp, stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("rs_resample_noalloc: launch: ") + cudaGetErrorString(e));
        return RS_ERR_CUDA;
    }
    return RS_OK;
}
