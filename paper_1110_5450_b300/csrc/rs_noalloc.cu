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
// RS_STATIC_SCRATCH_BYTES.  The array is created when the CUDA runtime loads
// this file's device code on a device: with lazy module loading (the CUDA
// default) that is the first call of this entry point on the device, with
// eager loading (CUDA_MODULE_LOADING=EAGER) the creation of the device's
// context.  From then on the device holds it until the process exits.  Host
// code cannot use the array's name as an address (on the host it is only a
// stand-in symbol), so every call looks the device address up with
// cudaGetSymbolAddress while the device is current (no allocation once the
// array exists; the address stays right if the context was reset and the
// array re-created).  The first call on a device therefore belongs at
// start-up -- before the host application's allocator takes the device
// memory, and outside any stream capture.
//
// All calls share the one array and it keeps whatever the last call left in
// it: the error word is cleared on every call, and the weight-table kernel
// rewrites every table entry it uses.  Calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array; issue
// them on one stream, one after another.
#include <cmath>
#include <cstdio>

#include "rs_internal.h"

namespace rs {
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[RS_STATIC_SCRATCH_BYTES];

// Device address of the static array on the current device.  The lookup
// loads this file's device code on first use (which creates the array:
// cudaErrorMemoryAllocation then means the device had no room left for it).
rs_status static_scratch(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        set_error(std::string("rs_resample_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RS_ERR_OOM : RS_ERR_CUDA;
    }
    *out = p;
    return RS_OK;
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
    // the same checks, output size and strides as rs_plan_create
    rs_plan_desc d;
    const rs_status vs = validate_desc(*desc, &d);
    if (vs != RS_OK) return bad(vs, rs_last_error());
    // this path always runs the two-pass kernels: no kernel choice to make
    if (d.flags & ~uint32_t(RS_NO_ANTIALIAS))
        return bad(RS_ERR_UNSUPPORTED, "only RS_NO_ANTIALIAS applies (this path always runs the two-pass kernels)");
    const int64_t oh = d.out_h, ow = d.out_w;
    const int64_t in_stride = d.in_row_stride, out_stride = d.out_row_stride;

    const bool dbl = d.in_dtype == RS_F64;
    const size_t wsz = dbl ? 8 : 4;
    WeightArgs a[2];
    const int64_t n_in[2] = {d.in_h, d.in_w}, n_out[2] = {oh, ow};
    size_t need = up256(16);
    for (int ax = 0; ax < 2; ++ax) {
        AxisGeom &g = a[ax].g;
        std::string why;
        if (!axis_setup(g, n_in[ax], n_out[ax], d, why)) return bad(RS_ERR_UNSUPPORTED, why.c_str());
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
