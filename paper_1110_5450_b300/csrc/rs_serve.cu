// rs_serve.cu -- continuous-batching resampling server on one device.
//
// Requests (one image each, any size / scale / kernel) are submitted from any
// host thread.  A scheduler thread
//   * admits them in arrival order while their device state (weight tables,
//     band tables and, when the client passes no output buffer, the output)
//     fits the server's memory budget -- a device arena allocated once;
//   * plans each admitted request without any host synchronisation: the tap
//     span of a group of G outputs is bounded by ceil((G-1) n_in / n_out) +
//     the table width, which sizes the band and the staged tile (the kernel
//     checks every band against the staged rows and flags a violation);
//   * groups the requests admitted since the previous launch into one
//     persistent fused launch per (channels, dtype, group size, TMA) class,
//     on one of several streams, so that requests arriving while others run
//     are admitted as memory frees and their work overlaps on the device;
//   * runs every large request (2^20 output pixels or more, a 16-byte row
//     pitch) alone on the row-streaming kernels -- the same kernels a plan
//     picks untuned -- through a plan object whose tables, band tables and
//     group descriptors all live in the request's arena block (window starts
//     from their closed form on the host, uploads through the slot's pinned
//     staging), so large requests no longer queue behind the tile kernel;
//   * timestamps completion in a host callback queued behind each launch,
//     which also returns the request's tables to the arena.
// All device waits inside the kernels are bounded; the server never runs an
// unbounded device-side loop.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rs_plan.h"

using namespace rs;

namespace {

uint64_t now_ns()
{
    return uint64_t(std::chrono::duration_cast<std::chrono::nanoseconds>(
                         std::chrono::steady_clock::now().time_since_epoch())
                         .count());
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// First-fit allocator over the device arena (host bookkeeping only).
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_; // offset -> length
    size_t in_use = 0;
    void reset(size_t n)
    {
        size = n;
        free_.clear();
        free_[0] = n;
        in_use = 0;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = up256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t next = it->first + bytes;
            free_.erase(it);
            if (rest) free_[next] = rest;
            in_use += bytes;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = up256(bytes);
        in_use -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Req {
    rs_request r{};
    uint64_t ticket = 0;
    uint64_t t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
    uint64_t t_gpu_start = 0, t_gpu_end = 0;
    int32_t status = RS_ERR_BUSY;
    int32_t launch_id = -1, batch_size = 0;
    // device placement (arena offsets)
    size_t tab_off = 0, tab_bytes = 0;
    size_t out_off = 0, out_bytes = 0;
    bool own_out = false;
    void *d_out = nullptr;
    // plan
    AxisGeom gy, gx;
    AxisTables ty, tx;
    fused::Params P{};
    int G = 0, use_tma = 0, cls = 0;
    fused::Work regions{};
    // large requests: run alone on the row-streaming kernels through a plan
    // object over the request's arena block (sx: the streaming tables' part)
    bool big = false;
    rs_plan *sp = nullptr;
    size_t sx_off = 0, sx_bytes = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    std::vector<Req *> reqs;
    bool busy = false;                // owned by the scheduler (under the server mutex)
    std::atomic<bool> done{false};    // set by the completion callback
    std::atomic<uint64_t> t_done{0};  // completion time, written by the callback
    int launch_id = 0;
    // device launch arrays and their pinned staging
    DeviceBuf dparams, dmaps, doff;
    void *host = nullptr;
    size_t cap = 0;
    unsigned char *xstage = nullptr; // pinned staging of a large request's streaming descriptors
    // GPU clock (%globaltimer, ns) when the launch's work started and ended on
    // the device: written by one-thread kernels around it, copied to the
    // pinned hstamp before the completion callback
    DeviceBuf dstamp;
    uint64_t *hstamp = nullptr;
    struct rs_server *owner = nullptr;
};

constexpr size_t kXStage = 256 * 1024;       // bytes of that staging per slot
constexpr int64_t kBigPixels = int64_t(1) << 20; // output pixels from which a request streams

} // namespace

struct rs_server {
    rs_server_desc d{};
    int device = 0, num_sms = 0;
    void *arena_base = nullptr;
    Arena arena;
    DeviceBuf derr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> pending;  // submitted, not admitted
    std::vector<Req *> ready;   // admitted and planned, not launched
    std::unordered_map<uint64_t, Req *> all;
    static constexpr int kMaxSlots = 8;
    Slot slots[kMaxSlots];
    int nslots = 0;
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 1;
    int launches = 0;
    // statistics
    uint64_t completed = 0, rejected = 0, out_pixels = 0, max_batch_seen = 0, max_in_use = 0;
    std::atomic<uint64_t> streamed{0}; // launches that ran on the row-streaming kernels
    uint64_t launch_host_ns = 0, stream_host_ns = 0; // host time issuing launches (all; streamed ones)
    std::string error;
    ~rs_server()
    {
        for (auto &kv : all) delete kv.second;
        for (int k = 0; k < nslots; ++k) {
            if (slots[k].stream) cudaStreamDestroy(slots[k].stream);
            if (slots[k].host) cudaFreeHost(slots[k].host);
            if (slots[k].xstage) cudaFreeHost(slots[k].xstage);
            if (slots[k].hstamp) cudaFreeHost(slots[k].hstamp);
        }
        if (arena_base) cudaFree(arena_base);
    }
};

namespace {

// Per-request shared-memory caps (bytes) that keep two CTAs of any launch on
// an SM: region maxima over a launch stay below these.
constexpr size_t kCapTin = 36 * 1024, kCapW = 4 * 1024, kCapTt = 16 * 1024;

struct FastPlan {
    bool ok = false;
    rs_status why = RS_OK;
    const char *msg = "";
};

int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }

int64_t floor_div64(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Window starts of an axis in closed form (what the weight-table kernel
// stores): the first raw tap j_lo = floor(((2i+1) n_in - R D - n_out) /
// (2 n_out)) + 1, moved into [0, n_in - t_eff] -- for every boundary rule the
// smallest input a window's taps map to is j_lo if j_lo >= 0, else 0, and
// the stored window starts there or at the last full window.
void host_starts(const AxisGeom &g, std::vector<int32_t> &st)
{
    st.resize(size_t(g.n_out));
    const int64_t RD = g.R * g.D;
    for (int64_t i = 0; i < g.n_out; ++i) {
        const int64_t jlo = floor_div64((2 * i + 1) * g.n_in - RD - g.n_out, 2 * g.n_out) + 1;
        st[size_t(i)] = int32_t(std::min<int64_t>(std::max<int64_t>(jlo, 0), g.n_in - g.t_eff));
    }
}

// Bytes the row-streaming kernels' tables of a request may take at most:
// the band kernels' bases and bands (at most 40 taps x 4 outputs across, 32
// taps x 8 floats down per group of 4 rows), the pipelined kernel's group
// descriptors or the tensor-core downscale's per-strip weight matrices,
// whichever is largest.
size_t stream_space(const AxisGeom &gy, const AxisGeom &gx, int C)
{
    const size_t gxn = size_t((gx.n_out + 3) / 4), gyn = size_t((gy.n_out + 3) / 4);
    const size_t band = up256(gxn * 4) + up256(gxn * 40 * 4 * 4) + up256((gyn + 4) * 4) + up256(gyn * 32 * 8 * 4);
    const size_t desc = up256(gxn * 4) + up256((gyn + 8) * 4);
    const size_t tcs = gx.n_out < gx.n_in && gy.n_out < gy.n_in ? tcstream::space_bound(gx, gy, C) : 0;
    return std::max(std::max(band, desc), tcs) + 256;
}

// Geometry and kernel configuration of a request from closed-form bounds
// (no device readback).  Fills r->gy/gx/G/P (except pointers) and the byte
// size of its tables.
FastPlan fast_plan(rs_server *S, Req *q)
{
    FastPlan f;
    rs_plan_desc &d = q->r.desc;
    const int C = d.channels;
    if (C != 1 && C != 3) return {false, RS_ERR_UNSUPPORTED, "server: 1 or 3 channels"};
    if (d.in_dtype != d.out_dtype || d.in_dtype < RS_F64 || d.in_dtype > RS_BF16)
        return {false, RS_ERR_INVALID_ARG, "server: dtype"};
    if (d.kernel < RS_K_LINEAR || d.kernel > RS_K_GAUSSIAN || d.boundary < RS_B_CLAMP || d.boundary > RS_B_TRUNCATE)
        return {false, RS_ERR_INVALID_ARG, "server: kernel or boundary"};
    const int R = support_radius(d.kernel, d.param);
    if (!R) return {false, RS_ERR_INVALID_ARG, "server: kernel parameter"};
    if (d.flags & RS_PREFILTER) return {false, RS_ERR_UNSUPPORTED, "server: RS_PREFILTER is per plan only"};
    if (d.in_h < 1 || d.in_w < 1 || d.in_h > kMaxSide || d.in_w > kMaxSide)
        return {false, RS_ERR_INVALID_ARG, "server: input size"};
    auto derive = [](int32_t given, int64_t n, double s) -> int64_t {
        if (given > 0) return given;
        if (!(s > 0.0) || !std::isfinite(s)) return -1;
        const double v = std::floor(double(n) * s + 0.5);
        if (!(v < double(kMaxSide) + 1.0)) return -1;
        return v < 1.0 ? 1 : int64_t(v);
    };
    const int64_t oh = derive(d.out_h, d.in_h, d.scale_h), ow = derive(d.out_w, d.in_w, d.scale_w);
    if (oh < 1 || ow < 1) return {false, RS_ERR_INVALID_ARG, "server: output size"};
    d.out_h = int32_t(oh);
    d.out_w = int32_t(ow);
    if (d.in_row_stride == 0) d.in_row_stride = int64_t(d.in_w) * C;
    if (d.out_row_stride == 0) d.out_row_stride = int64_t(d.out_w) * C;
    if (d.in_row_stride < int64_t(d.in_w) * C || d.out_row_stride < int64_t(d.out_w) * C)
        return {false, RS_ERR_INVALID_ARG, "server: row stride"};
    const bool aa = !(d.flags & RS_NO_ANTIALIAS);
    AxisGeom *gs[2] = {&q->gy, &q->gx};
    const int64_t nin[2] = {d.in_h, d.in_w}, nout[2] = {oh, ow};
    for (int a = 0; a < 2; ++a) {
        AxisGeom &g = *gs[a];
        g.n_in = nin[a];
        g.n_out = nout[a];
        g.R = R;
        g.D = (aa && g.n_in > g.n_out) ? 2 * g.n_in : 2 * g.n_out;
        const int64_t traw = ceil_div64(g.R * g.D, g.n_out);
        if (traw > kMaxTaps) return {false, RS_ERR_UNSUPPORTED, "server: more than 256 taps"};
        g.t_raw = int32_t(traw);
        g.t_eff = int32_t(std::min<int64_t>(traw, g.n_in));
        g.kernel = d.kernel;
        g.boundary = d.boundary;
        g.param = d.param;
    }
    const size_t esz = dt_size(d.in_dtype), asz = d.in_dtype == RS_F64 ? 8 : 4;
    const int vec = int(16 / esz);
    const int dup = d.in_dtype == RS_F64 ? 1 : 2;
    // group span bound: ceil((G-1) n_in / n_out) + t_eff, per axis
    auto span = [](const AxisGeom &g, int64_t k) { return ceil_div64(k * g.n_in, g.n_out); };
    q->use_tma = ((d.in_row_stride * int64_t(esz)) % 16 == 0 &&
                  (reinterpret_cast<uintptr_t>(q->r.d_in) & 15u) == 0 && encode_fn() != nullptr)
                     ? 1
                     : 0;
    for (int G : {4, 2, 1}) {
        const fused::Variant *var = find_variant(d.in_dtype, C, G);
        if (!var) continue;
        const int V = var->V;
        const int64_t J = std::max(span(q->gy, G - 1) + q->gy.t_eff, span(q->gx, G - 1) + q->gx.t_eff);
        if (J > 256) continue;
        // the horizontal band interleaves group pairs
        const int js_y = band_stride(G * dup, int(J)), js_x = band_stride(2 * G, int(J));
        for (int tile_h : {32, 16, 8}) {
            if (tile_h % G) continue;
            const int ngy = tile_h / G;
            const int64_t rows = span(q->gy, int64_t(ngy - 1) * G) + J;
            for (int ngx = 32; ngx >= 1; --ngx) {
                const int64_t cols = (span(q->gx, int64_t(ngx - 1) * G) + J) * C + (vec - 1);
                const int64_t bw = (cols + vec - 1) / vec * vec;
                if (q->use_tma && bw > 256) continue;
                if (rows > 256) continue;
                const int w1 = int((bw + 32 * V - 1) / (32 * V) * (32 * V));
                const fused::Layout L = fused::layout(esz, asz, int(rows), int(bw), ngy, ngx, js_y, js_x, tile_h,
                                                      w1 | 1, 1);
                if (L.tin > kCapTin || L.wy > kCapW || L.wx > kCapW || L.tt > kCapTt || L.rec2 > kCapW + 512)
                    continue;
                // accept the first (largest) tile that fits
                q->G = G;
                fused::Params &P = q->P;
                std::memset(&P, 0, sizeof P);
                P.in_h = d.in_h;
                P.in_w = d.in_w;
                P.out_h = oh;
                P.out_w = ow;
                P.in_stride = d.in_row_stride;
                P.out_stride = d.out_row_stride;
                P.J = int32_t(J);
                P.js_y = js_y;
                P.js_x = js_x;
                P.tile_h = tile_h;
                P.tile_w = ngx * G;
                P.box_h = int32_t(rows);
                P.box_w = int32_t(bw);
                P.sub_h = int32_t(rows);
                P.n_sub = 1;
                P.w1 = w1;
                P.pitch_t = w1 | 1;
                P.tiles_y = int32_t((oh + tile_h - 1) / tile_h);
                P.tiles_x = int32_t((ow + P.tile_w - 1) / P.tile_w);
                P.groups_y = int32_t((oh + G - 1) / G);
                P.groups_x = int32_t((ow + G - 1) / G);
                P.use_tma = q->use_tma;
                P.stages = 1;
                P.n1 = S->d.warps_pass1 > 0 ? S->d.warps_pass1 : 4;
                P.err = static_cast<int *>(S->derr.p);
                q->regions.tin_bytes = int32_t(L.tin);
                q->regions.wy_bytes = int32_t(L.wy);
                q->regions.wx_bytes = int32_t(L.wx);
                q->regions.tt_bytes = int32_t(L.tt);
                q->regions.rec2_bytes = int32_t(L.rec2);
                // tables (per axis: jlo, cnt, start, w64, wwork, band base, band weights)
                size_t tb = 0;
                for (int a = 0; a < 2; ++a) {
                    const AxisGeom &g = *gs[a];
                    const int64_t groups = (g.n_out + G - 1) / G;
                    const int js = a == 0 ? js_y : js_x;
                    const int64_t slots =
                        a == 0 ? groups : (groups + ngx - 1) / ngx * fused::pair_slots(ngx);
                    tb += 3 * up256(size_t(g.n_out) * 4) + up256(size_t(g.n_out) * g.t_eff * 8) +
                          up256(size_t(g.n_out + 4) * g.t_eff * asz) + up256(size_t(groups) * 4) +
                          up256(size_t(slots) * js * asz);
                }
                // a large request streams (the tile plan above stays its fallback)
                q->big = oh * ow >= kBigPixels && q->use_tma && d.in_dtype != RS_F64 && !(d.flags & RS_NO_STREAM);
                if (q->big) {
                    q->sx_off = tb;
                    q->sx_bytes = stream_space(q->gy, q->gx, C);
                    tb += up256(q->sx_bytes);
                }
                q->tab_bytes = tb;
                q->own_out = q->r.d_out == nullptr;
                q->out_bytes = q->own_out ? size_t(oh) * size_t(d.out_row_stride) * esz : 0;
                q->cls = (C << 8) | (d.in_dtype << 4) | (G << 1) | q->use_tma;
                f.ok = true;
                return f;
            }
        }
    }
    return {false, RS_ERR_UNSUPPORTED, "server: no tile configuration fits"};
}

// Carves a request's tables out of its arena block and fills the pointers.
void place_tables(rs_server *S, Req *q)
{
    char *base = static_cast<char *>(S->arena_base) + q->tab_off;
    size_t off = 0;
    auto take = [&](size_t b) {
        char *p = base + off;
        off += up256(b);
        return p;
    };
    const size_t asz = q->r.desc.in_dtype == RS_F64 ? 8 : 4;
    AxisGeom *gs[2] = {&q->gy, &q->gx};
    AxisTables *ts[2] = {&q->ty, &q->tx};
    for (int a = 0; a < 2; ++a) {
        const AxisGeom &g = *gs[a];
        AxisTables &t = *ts[a];
        const int64_t groups = (g.n_out + q->G - 1) / q->G;
        t.G = q->G;
        t.J = q->P.J;
        t.groups = int32_t(groups);
        t.dup = (a == 0 && asz == 4) ? 2 : 1;
        t.pair_ngx = a == 1 ? q->P.tile_w / q->G : 0;
        const int js = a == 0 ? q->P.js_y : q->P.js_x;
        t.jlo = reinterpret_cast<int32_t *>(take(size_t(g.n_out) * 4));
        t.cnt = reinterpret_cast<int32_t *>(take(size_t(g.n_out) * 4));
        t.start = reinterpret_cast<int32_t *>(take(size_t(g.n_out) * 4));
        t.w64 = reinterpret_cast<double *>(take(size_t(g.n_out) * g.t_eff * 8));
        t.wwork = take(size_t(g.n_out + 4) * g.t_eff * asz); // 4 spare rows (zeroed before a streamed launch)
        t.band_base = reinterpret_cast<int32_t *>(take(size_t(groups) * 4));
        t.band_w = take(size_t(band_slots(t)) * js * asz);
    }
    q->P.base_y = q->ty.band_base;
    q->P.base_x = q->tx.band_base;
    q->P.band_y = q->ty.band_w;
    q->P.band_x = q->tx.band_w;
    q->d_out = q->own_out ? static_cast<char *>(S->arena_base) + q->out_off : q->r.d_out;
    q->P.in = q->r.d_in;
    q->P.out = q->d_out;
}

void on_launch_done(void *arg);

// One thread: the GPU clock into *t (the start or end of a launch's work).
__global__ void stamp_kernel(uint64_t *t)
{
    uint64_t v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    *t = v;
}

// After a launch's work on the slot's stream: the end stamp, the copy of both
// stamps to the host, then the completion callback.  Returns an error message
// or an empty string.
std::string finish_launch(Slot &slot)
{
    cudaStream_t st = slot.stream;
    std::string err;
    stamp_kernel<<<1, 1, 0, st>>>(static_cast<uint64_t *>(slot.dstamp.p) + 1);
    cudaMemcpyAsync(slot.hstamp, slot.dstamp.p, 16, cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaLaunchHostFunc(st, on_launch_done, &slot);
    if (e != cudaSuccess) {
        // no callback will come: complete the slot from here
        err = std::string("server callback: ") + cudaGetErrorString(e);
        cudaGetLastError();
        cudaStreamSynchronize(st);
        slot.t_done.store(now_ns());
        slot.done.store(true, std::memory_order_release);
    }
    return err;
}

// A large request alone on the row-streaming kernels (its weight tables are
// computed on the slot's stream first).  False if no streaming configuration
// takes it (the caller then runs its tile plan).
bool launch_streamed(rs_server *S, Slot &slot, Req *q)
{
    cudaStream_t st = slot.stream;
    const int dt = q->r.desc.in_dtype;
    const size_t asz = dt == RS_F64 ? 8 : 4;
    WeightArgs a0, a1;
    a0.g = q->gy;
    a0.t = q->ty;
    a1.g = q->gx;
    a1.t = q->tx;
    a0.work_is_double = a1.work_is_double = 0;
    a0.err = a1.err = static_cast<int *>(S->derr.p);
    launch_weights(a0, a1, st);
    for (const auto &at : {a0, a1}) // the spare rows that groups of 4 read past the last output
        cudaMemsetAsync(static_cast<char *>(at.t.wwork) + size_t(at.g.n_out) * at.g.t_eff * asz, 0,
                        size_t(4) * at.g.t_eff * asz, st);
    rs_plan *p = new (std::nothrow) rs_plan();
    if (!p) return false;
    p->desc = q->r.desc;
    p->device = S->device;
    p->num_sms = S->num_sms;
    p->gy = q->gy;
    p->gx = q->gx;
    p->ty = q->ty;
    p->tx = q->tx;
    p->d_err = static_cast<int *>(S->derr.p);
    p->path = 0;
    host_starts(q->gy, p->host_start_y);
    host_starts(q->gx, p->host_start_x);
    p->ext_base = static_cast<char *>(S->arena_base) + q->tab_off + q->sx_off;
    p->ext_bytes = q->sx_bytes;
    p->ext_staging = slot.xstage;
    p->ext_staging_bytes = kXStage;
    if (stream::setup(p, st, stream::Opts()) != RS_OK) {
        cudaGetLastError();
        delete p;
        return false;
    }
    p->use_stream = 1;
    if (stream::launch(p, q->r.d_in, q->d_out, st) != RS_OK) {
        cudaGetLastError();
        delete p;
        return false;
    }
    q->sp = p; // released when the launch has completed
    S->streamed.fetch_add(1, std::memory_order_relaxed);
    return true;
}

// Launches one class's group (or one large request) on a reserved slot.
// Called WITHOUT the server mutex: the group and the slot belong to the
// scheduler until the launch's completion callback fires.  Returns an error
// message or an empty string.
std::string launch(rs_server *S, Slot &slot, std::vector<Req *> &group)
{
    const int n = int(group.size());
    const Req *q0 = group[0];
    const int C = q0->r.desc.channels, dt = q0->r.desc.in_dtype;
    cudaStream_t st = slot.stream;
    stamp_kernel<<<1, 1, 0, st>>>(static_cast<uint64_t *>(slot.dstamp.p));
    bool tables_done = false;
    if (n == 1 && group[0]->big) {
        if (launch_streamed(S, slot, group[0])) return finish_launch(slot);
        tables_done = true; // the weight tables are on the stream already
    }
    // weight and band tables of every request (asynchronous, in stream order)
    for (Req *q : group) {
        WeightArgs a0, a1;
        a0.g = q->gy;
        a0.t = q->ty;
        a1.g = q->gx;
        a1.t = q->tx;
        a0.work_is_double = a1.work_is_double = dt == RS_F64 ? 1 : 0;
        a0.err = a1.err = static_cast<int *>(S->derr.p);
        if (!tables_done) launch_weights(a0, a1, st);
        launch_band(a0, a1, st);
    }
    // launch arrays: parameters, tensor maps, tile prefix sums
    const size_t pbytes = ((sizeof(fused::Params) * size_t(n) + 63) / 64) * 64;
    const size_t mbytes = sizeof(CUtensorMap) * size_t(n);
    unsigned char *hs = static_cast<unsigned char *>(slot.host);
    fused::Params *hp = reinterpret_cast<fused::Params *>(hs);
    CUtensorMap *hm = reinterpret_cast<CUtensorMap *>(hs + pbytes);
    int32_t *ho = reinterpret_cast<int32_t *>(hs + pbytes + mbytes);
    fused::Work w;
    std::memset(&w, 0, sizeof w);
    ho[0] = 0;
    for (int i = 0; i < n; ++i) {
        Req *q = group[i];
        hp[i] = q->P;
        ho[i + 1] = ho[i] + q->P.tiles_y * q->P.tiles_x;
        w.tin_bytes = std::max(w.tin_bytes, q->regions.tin_bytes);
        w.wy_bytes = std::max(w.wy_bytes, q->regions.wy_bytes);
        w.wx_bytes = std::max(w.wx_bytes, q->regions.wx_bytes);
        w.tt_bytes = std::max(w.tt_bytes, q->regions.tt_bytes);
        w.rec2_bytes = std::max(w.rec2_bytes, q->regions.rec2_bytes);
        if (q->use_tma) {
            const rs_plan_desc &d = q->r.desc;
            CUtensorMapDataType tt = dt == RS_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                     : dt == RS_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                     : dt == RS_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
            const size_t esz = dt_size(dt);
            cuuint64_t dims[2] = {cuuint64_t(int64_t(d.in_w) * C), cuuint64_t(d.in_h)};
            cuuint64_t strides[1] = {cuuint64_t(d.in_row_stride * int64_t(esz))};
            cuuint32_t box[2] = {cuuint32_t(q->P.box_w), cuuint32_t(q->P.sub_h)};
            cuuint32_t estr[2] = {1, 1};
            encode_fn()(&hm[i], tt, 2, const_cast<void *>(q->r.d_in), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        } else {
            std::memset(&hm[i], 0, sizeof(CUtensorMap));
        }
    }
    cudaMemcpyAsync(slot.dparams.p, hp, sizeof(fused::Params) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(slot.dmaps.p, hm, mbytes, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(slot.doff.p, ho, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st);
    w.imgs = static_cast<const fused::Params *>(slot.dparams.p);
    w.maps = static_cast<const CUtensorMap *>(slot.dmaps.p);
    w.tile_off = static_cast<const int32_t *>(slot.doff.p);
    w.n_images = n;
    w.total_tiles = ho[n];
    w.stages = 1;
    w.n1 = q0->P.n1;
    w.use_tma = q0->use_tma;
    const size_t smem = fused::layout_of(w.tin_bytes, w.wy_bytes, w.wx_bytes, w.tt_bytes, w.rec2_bytes, 1).total +
                        fused::batch_extra(n);
    const fused::Variant *var = find_variant(dt, C, q0->G);
    const int occ = occupancy(var->fn, fused::kThreads, smem);
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(w.total_tiles, int64_t(std::max(occ, 1)) * S->num_sms)));
    fused::Params p0;
    std::memset(&p0, 0, sizeof p0);
    p0.err = static_cast<int *>(S->derr.p);
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof dummy);
    void *args[3] = {&dummy, &p0, &w};
    std::string err;
    cudaError_t e = cudaLaunchKernel(var->fn, dim3(grid), dim3(fused::kThreads), args, smem, st);
    if (e != cudaSuccess) {
        err = std::string("server launch: ") + cudaGetErrorString(e);
        cudaGetLastError();
    }
    const std::string fin = finish_launch(slot);
    return err.empty() ? fin : err;
}

// Completion callback (driver thread): never blocks and calls no CUDA API --
// it only stamps the time and raises the slot's flag; the scheduler does the
// bookkeeping.
void on_launch_done(void *arg)
{
    Slot *slot = static_cast<Slot *>(arg);
    slot->t_done.store(now_ns(), std::memory_order_relaxed);
    slot->done.store(true, std::memory_order_release);
    slot->owner->cv.notify_all();
}

// Bookkeeping of finished launches (server mutex held).
void collect(rs_server *S)
{
    for (int k = 0; k < S->nslots; ++k) {
        Slot &slot = S->slots[k];
        if (!slot.busy || !slot.done.load(std::memory_order_acquire)) continue;
        const uint64_t t = slot.t_done.load(std::memory_order_relaxed);
        for (Req *q : slot.reqs) {
            q->t_done = t;
            q->t_gpu_start = slot.hstamp[0];
            q->t_gpu_end = slot.hstamp[1];
            q->status = S->error.empty() ? RS_OK : RS_ERR_CUDA;
            delete q->sp; // a streamed request's plan object (no device memory of its own)
            q->sp = nullptr;
            S->arena.release(q->tab_off, q->tab_bytes);
            ++S->completed;
            S->out_pixels += uint64_t(q->P.out_h) * uint64_t(q->P.out_w);
        }
        slot.reqs.clear();
        slot.done.store(false, std::memory_order_relaxed);
        slot.busy = false;
    }
}

void scheduler(rs_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    while (!S->stop) {
        collect(S);
        // admit in arrival order while the budget holds
        while (!S->pending.empty()) {
            Req *q = S->pending.front();
            size_t off = 0;
            const size_t need = up256(q->tab_bytes) + up256(q->out_bytes);
            if (need > S->arena.size) {
                q->status = RS_ERR_BUDGET;
                q->t_done = now_ns();
                ++S->rejected;
                S->pending.pop_front();
                continue;
            }
            if (!S->arena.alloc(need, &off)) break; // wait for memory to free up
            q->tab_off = off;
            q->out_off = off + up256(q->tab_bytes);
            q->tab_bytes = up256(q->tab_bytes);
            // the output part stays allocated until rs_server_release
            q->t_admit = now_ns();
            place_tables(S, q);
            S->ready.push_back(q);
            S->pending.pop_front();
            S->max_in_use = std::max<uint64_t>(S->max_in_use, S->arena.in_use);
        }
        // reserve free slots for what is ready, one class per slot, oldest class first
        std::vector<std::pair<Slot *, std::vector<Req *>>> work;
        for (int k = 0; k < S->nslots && !S->ready.empty(); ++k) {
            Slot &slot = S->slots[k];
            if (slot.busy) continue;
            const Req *first = S->ready.front();
            const int cls = first->cls;
            std::vector<Req *> group, rest;
            for (Req *q : S->ready) {
                // a large request runs alone (on the streaming kernels); the
                // others group by class
                const bool take = first->big ? group.empty() && q == first
                                             : !q->big && q->cls == cls && int(group.size()) < S->d.max_batch;
                if (take)
                    group.push_back(q);
                else
                    rest.push_back(q);
            }
            S->ready.swap(rest);
            const uint64_t t = now_ns();
            ++S->launches;
            slot.launch_id = S->launches;
            for (Req *q : group) {
                q->t_launch = t;
                q->launch_id = slot.launch_id;
                q->batch_size = int32_t(group.size());
            }
            slot.busy = true;
            slot.done.store(false);
            slot.reqs = group;
            S->max_batch_seen = std::max<uint64_t>(S->max_batch_seen, uint64_t(group.size()));
            work.emplace_back(&slot, std::move(group));
        }
        if (work.empty()) {
            S->cv.wait_for(lock, std::chrono::microseconds(200));
            continue;
        }
        // CUDA calls happen without the mutex
        lock.unlock();
        std::string err;
        uint64_t t_all = 0, t_big = 0;
        for (auto &w : work) {
            const uint64_t t0 = now_ns();
            const bool big = w.second.size() == 1 && w.second[0]->big;
            std::string e = launch(S, *w.first, w.second);
            if (!e.empty()) err = e;
            const uint64_t dt = now_ns() - t0;
            t_all += dt;
            t_big += big ? dt : 0;
        }
        lock.lock();
        S->launch_host_ns += t_all;
        S->stream_host_ns += t_big;
        if (!err.empty()) S->error = err;
        S->cv.notify_all();
    }
}

} // namespace

extern "C" {

rs_status rs_server_create(const rs_server_desc *desc, rs_server **out)
{
    if (!out) return fail(RS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc || desc->budget_bytes < (1u << 20) || desc->max_inflight < 1 || desc->max_inflight > 8 ||
        desc->max_batch < 1 || desc->max_batch > 4096 || desc->warps_pass1 < 0 || desc->warps_pass1 > 7)
        return fail(RS_ERR_INVALID_ARG, "server: budget >= 1 MiB, 1..8 launches in flight, 1..4096 per launch");
    rs_server *S = new (std::nothrow) rs_server();
    if (!S) return fail(RS_ERR_OOM, "host allocation failed");
    S->d = *desc;
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, S->device);
    if (e == cudaSuccess) e = cudaMalloc(&S->arena_base, size_t(desc->budget_bytes));
    if (e == cudaSuccess) e = cudaMalloc(&S->derr.p, 16);
    if (e == cudaSuccess) e = cudaMemset(S->derr.p, 0, 16);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "server: allocating the arena");
    }
    S->arena.reset(size_t(desc->budget_bytes));
    S->nslots = desc->max_inflight;
    const int nb = desc->max_batch;
    for (int k = 0; k < S->nslots; ++k) {
        Slot &s = S->slots[k];
        s.owner = S;
        s.cap = size_t(nb);
        const size_t host = ((sizeof(fused::Params) * nb + 63) / 64) * 64 + sizeof(CUtensorMap) * nb + 4 * (nb + 1);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&s.dparams.p, sizeof(fused::Params) * nb);
        if (e == cudaSuccess) e = cudaMalloc(&s.dmaps.p, sizeof(CUtensorMap) * nb);
        if (e == cudaSuccess) e = cudaMalloc(&s.doff.p, 4 * (nb + 1));
        if (e == cudaSuccess) e = cudaHostAlloc(&s.host, host, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&s.xstage), kXStage, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&s.dstamp.p, 16);
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&s.hstamp), 16, cudaHostAllocDefault);
    }
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "server: slots");
    }
    // load every kernel a launch may use now: under lazy module loading the
    // first launch of each would otherwise stall a request by milliseconds
    preload_weights();
    {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, stamp_kernel) != cudaSuccess) cudaGetLastError();
    }
    for (const int dt : {int(RS_F64), int(RS_F32), int(RS_F16), int(RS_BF16)}) {
        for (const int C : {1, 3})
            for (const int G : {1, 2, 4, 8})
                if (const fused::Variant *v = find_variant(dt, C, G)) occupancy(v->fn, fused::kThreads, 0);
        if (dt != RS_F64) {
            stream::preload(dt);
            xstream::preload(dt);
        }
        if (dt == RS_F16 || dt == RS_BF16) tcstream::preload(dt);
    }
    S->th = std::thread(scheduler, S);
    *out = S;
    return RS_OK;
}

rs_status rs_batch_submit(rs_server *S, const rs_request *reqs, int32_t n, uint64_t *first_ticket)
{
    if (!S || !reqs || n < 1 || !first_ticket) return fail(RS_ERR_INVALID_ARG, "server: submit arguments");
    for (int i = 0; i < n; ++i)
        if (!reqs[i].d_in) return fail(RS_ERR_INVALID_ARG, "server: request without an input");
    const uint64_t t = now_ns();
    std::vector<Req *> made;
    made.reserve(n);
    for (int i = 0; i < n; ++i) {
        Req *q = new (std::nothrow) Req();
        if (!q) {
            for (Req *m : made) delete m;
            return fail(RS_ERR_OOM, "host allocation failed");
        }
        q->r = reqs[i];
        q->t_submit = t;
        const FastPlan f = fast_plan(S, q);
        if (!f.ok) {
            q->status = f.why;
            q->t_done = t;
        }
        made.push_back(q);
    }
    {
        std::lock_guard<std::mutex> lock(S->mu);
        *first_ticket = S->next_ticket;
        for (Req *q : made) {
            q->ticket = S->next_ticket++;
            S->all[q->ticket] = q;
            if (q->status == RS_ERR_BUSY)
                S->pending.push_back(q);
            else
                ++S->rejected;
        }
    }
    S->cv.notify_all();
    return RS_OK;
}

rs_status rs_batch_poll(rs_server *S, uint64_t ticket, rs_request_state *st)
{
    if (!S || !st) return fail(RS_ERR_INVALID_ARG, "server: poll arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(RS_ERR_INVALID_ARG, "server: unknown or released ticket");
    const Req *q = it->second;
    std::memset(st, 0, sizeof *st);
    st->status = q->status;
    st->d_out = q->status == RS_OK ? q->d_out : nullptr;
    st->out_h = q->P.out_h;
    st->out_w = q->P.out_w;
    st->out_row_stride = q->P.out_stride;
    st->t_submit_ns = q->t_submit;
    st->t_admit_ns = q->t_admit;
    st->t_launch_ns = q->t_launch;
    st->t_done_ns = q->t_done;
    st->t_gpu_start_ns = q->t_gpu_start;
    st->t_gpu_end_ns = q->t_gpu_end;
    st->launch_id = q->launch_id;
    st->batch_size = q->batch_size;
    return RS_OK;
}

rs_status rs_server_release(rs_server *S, uint64_t ticket)
{
    if (!S) return fail(RS_ERR_INVALID_ARG, "server: NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(RS_ERR_INVALID_ARG, "server: unknown or released ticket");
    Req *q = it->second;
    if (q->status == RS_ERR_BUSY) return fail(RS_ERR_BUSY, "server: request still in flight");
    if (q->t_admit && q->out_bytes) S->arena.release(q->out_off, q->out_bytes);
    S->all.erase(it);
    delete q;
    S->cv.notify_all();
    return RS_OK;
}

rs_status rs_server_drain(rs_server *S, int64_t timeout_ms)
{
    if (!S) return fail(RS_ERR_INVALID_ARG, "server: NULL");
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        bool busy = !S->pending.empty() || !S->ready.empty();
        for (int k = 0; k < S->nslots; ++k) busy = busy || S->slots[k].busy;
        if (!busy) break;
        if (std::chrono::steady_clock::now() > deadline) return fail(RS_ERR_TIMEOUT, "server: drain");
        S->cv.wait_for(lock, std::chrono::milliseconds(1));
    }
    lock.unlock();
    int herr = 0;
    cudaError_t e = cudaMemcpy(&herr, S->derr.p, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "server: error word");
    if (herr) {
        char buf[64];
        std::snprintf(buf, sizeof buf, "server: device error word %d", herr);
        return fail(RS_ERR_DEVICE, buf);
    }
    if (!S->error.empty()) return fail(RS_ERR_CUDA, S->error);
    return RS_OK;
}

rs_status rs_server_get_stats(rs_server *S, rs_server_stats *st)
{
    if (!S || !st) return fail(RS_ERR_INVALID_ARG, "server: stats arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    std::memset(st, 0, sizeof *st);
    st->completed = S->completed;
    st->rejected = S->rejected;
    st->launches = uint64_t(S->launches);
    st->out_pixels = S->out_pixels;
    st->pending = uint64_t(S->pending.size() + S->ready.size());
    st->bytes_in_use = uint64_t(S->arena.in_use);
    st->max_bytes_in_use = S->max_in_use;
    st->max_batch = S->max_batch_seen;
    st->streamed = S->streamed.load(std::memory_order_relaxed);
    st->launch_host_ns = S->launch_host_ns;
    st->stream_host_ns = S->stream_host_ns;
    return RS_OK;
}

rs_status rs_server_destroy(rs_server *S)
{
    if (!S) return RS_OK;
    rs_server_drain(S, 60000);
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaError_t e = cudaDeviceSynchronize();
    delete S;
    if (e != cudaSuccess) return cuda_fail(e, "server: destroy");
    return RS_OK;
}

} // extern "C"
