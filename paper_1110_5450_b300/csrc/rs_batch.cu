// rs_batch.cu -- batches of uneven images in one persistent fused launch.
//
// Images of at least kStreamMinOut output pixels that the row-streaming
// kernels take (TMA-planned batches) leave the tile list and run on them,
// beside the persistent kernel: on large upscales they are 2-4x faster than
// the tile kernel.  The pipelined kernel's images go into one multi-image
// launch per kernel kind (their CTAs in one grid, each image's parameters and
// tensor map read from device arrays), and so do the band kernels' images.
// Where a launch takes several images, each is re-planned first for its share
// of the SMs within it (by output pixels): its strip width and row ranges are
// chosen anew for that share, so that its CTAs take wider strips and longer
// row ranges than a launch of its own would give them (narrow 16-bit strips
// stage small blocks and are bound by the latency of their copies).
//
// Each image gets an ordinary plan (exact taps, FP64 weight tables); the batch
// then re-plans every image's fused configuration under one launch-wide
// choice (kernel variant = group size G, warp split n1, staged-buffer count,
// shared-memory budget per CTA) and lays out device arrays of per-image kernel
// parameters, per-image TMA tensor maps and the tile prefix sums.  A launch is
// an explicitly built CUDA graph: upload of the parameters and tensor maps from
// pinned host memory, then the kernel.  Two such graphs
// alternate over two pinned staging buffers, so the host can prepare run k+1
// while run k is still on the GPU.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "rs_plan.h"

using namespace rs;

// (2^18: with the streamed images in multi-image launches, the C4 batch
// measured 3.93 ms at 2^18, 3.98 at 2^19, 4.09 at 2^20, 4.01 at 2^17)
constexpr int64_t kStreamMinOut = int64_t(1) << 18;
constexpr int kAux = 4; // side streams the streamed images are spread over

// Streamed images on one multi-image kernel (the pipelined kernel's
// xstream_multi_kernel, kind 0, or a band kernel's stream_multi_kernel /
// stream_ws_multi_kernel, kind 1): one launch over all their CTAs.  dev holds
// [Params][tensor maps][CTA offsets]; each run stages them in host[k]
// (pinned) and copies them up on the group's side stream before the launch.
struct MultiGroup {
    int kind = 0;
    const void *fn = nullptr;
    int block = 0;
    size_t smem = 0;
    int total = 0; // CTAs
    int aux = 0;   // side stream
    std::vector<int> imgs;
    std::vector<int32_t> off;
    size_t o_maps = 0, o_off = 0, bytes = 0;
    DeviceBuf dev;
    unsigned char *host[2] = {nullptr, nullptr};
    std::vector<const void *> st_in[2];
    std::vector<void *> st_out[2];
};

struct rs_batch {
    std::vector<rs_plan *> plans;
    std::vector<MultiGroup> groups; // streamed images, one launch per kernel
    std::vector<char> streamed; // image i runs on the row-streaming kernel
    int n_streamed = 0;
    std::vector<int> stream_order; // streamed images, largest output first
    cudaStream_t aux[kAux] = {};
    cudaEvent_t fork = nullptr, join[kAux] = {};
    int dtype = 0, C = 0;
    // launch-wide choice
    int G = 0, n1 = 4, stages = 1, use_tma = 0, budget_ctas = 2;
    const fused::Variant *variant = nullptr;
    size_t smem = 0;
    int grid = 0, ctas = 0;
    int total_tiles = 0;
    int64_t out_pixels = 0, in_bytes = 0, out_bytes = 0;
    fused::Work work{};
    fused::Params p0{}; // carries the error word
    DeviceBuf dparams, dmaps, dtileoff, derr;
    // two pinned staging buffers (parameters + tensor maps) and their graphs
    void *host_stage[2] = {nullptr, nullptr};
    std::vector<const void *> staged_in[2];
    std::vector<void *> staged_out[2];
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    int next = 0;
    CUtensorMap dummy_map;

    ~rs_batch()
    {
        for (int k = 0; k < 2; ++k) {
            if (exec[k]) cudaGraphExecDestroy(exec[k]);
            if (graph[k]) cudaGraphDestroy(graph[k]);
            if (done[k]) cudaEventDestroy(done[k]);
            if (host_stage[k]) cudaFreeHost(host_stage[k]);
        }
        for (int k = 0; k < kAux; ++k) {
            if (join[k]) cudaEventDestroy(join[k]);
            if (aux[k]) cudaStreamDestroy(aux[k]);
        }
        if (fork) cudaEventDestroy(fork);
        for (MultiGroup &g : groups)
            for (int k = 0; k < 2; ++k)
                if (g.host[k]) cudaFreeHost(g.host[k]);
        for (rs_plan *p : plans) rs_destroy(p);
    }
};

namespace {

size_t stage_bytes(int n)
{
    // parameters, then the tensor maps at a 64-byte boundary
    return ((sizeof(fused::Params) * size_t(n) + 63) / 64) * 64 + sizeof(CUtensorMap) * size_t(n);
}

// Combined shared memory of per-image configurations: each region sized for
// the largest image.
size_t combined_smem(const std::vector<Candidate> &pick, const std::vector<rs_plan *> &plans, int dtype,
                     int stages)
{
    const size_t esz = dt_size(dtype), asz = dtype == RS_F64 ? 8 : 4;
    size_t tin = 0, wy = 0, wx = 0, tt = 0, r2 = 0;
    for (size_t i = 0; i < pick.size(); ++i) {
        const Candidate &c = pick[i];
        const int dup = plans[i]->work_double ? 1 : 2;
        const int V = plans[i]->work_double ? 2 : 4;
        const int w1 = (c.box_w + 32 * V - 1) / (32 * V) * (32 * V);
        const fused::Layout L = fused::layout(esz, asz, c.box_h, c.box_w, c.tile_h / c.G, c.tile_w / c.G,
                                              band_stride(c.G * dup, c.J), band_stride(2 * c.G, c.J), c.tile_h,
                                              w1 | 1, 1);
        tin = std::max(tin, L.tin);
        wy = std::max(wy, L.wy);
        wx = std::max(wx, L.wx);
        tt = std::max(tt, L.tt);
        r2 = std::max(r2, L.rec2);
    }
    return fused::layout_of(tin, wy, wx, tt, r2, stages).total;
}

// Picks every image's configuration for a launch-wide (G, stages, budget):
// the cheapest candidate per image under a per-image cap, the cap tightened
// until the regions' maxima fit budget_ctas CTAs per SM.  Applies the picks
// when `apply`; returns the modelled total cost in SM cycles (inf if some
// image has no feasible configuration).
double plan_images(rs_batch *b, cudaStream_t stream, int G, int stages, int budget_ctas, bool apply, rs_status *st)
{
    *st = RS_OK;
    const size_t target = (227 * 1024) / size_t(budget_ctas);
    std::vector<Candidate> pick(b->plans.size());
    std::vector<std::vector<Candidate>> all(b->plans.size());
    std::vector<rs_plan *> tiled;
    std::vector<size_t> idx;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        if (b->streamed[i]) continue;
        all[i] = enumerate_candidates(b->plans[i], b->use_tma != 0);
        idx.push_back(i);
    }
    double total = INFINITY;
    for (size_t cap = target; cap >= 8 * 1024; cap = cap * 85 / 100) {
        total = 0.0;
        bool ok = true;
        std::vector<Candidate> pk;
        tiled.clear();
        for (size_t i : idx) {
            const Candidate *best = nullptr;
            for (const Candidate &c : all[i]) {
                if (c.G != G || c.stages != stages || c.smem > cap) continue;
                if (!best || c.cost < best->cost) best = &c;
            }
            if (!best) {
                ok = false;
                break;
            }
            pick[i] = *best;
            pk.push_back(*best);
            tiled.push_back(b->plans[i]);
            total += best->cost * double(b->plans[i]->gy.n_out) * double(b->plans[i]->gx.n_out);
        }
        if (!ok) return INFINITY;
        if (pk.empty() || combined_smem(pk, tiled, b->dtype, b->use_tma ? stages : 1) <= target) break;
        total = INFINITY;
    }
    if (!std::isfinite(total) || !apply) return total;
    for (size_t i : idx) {
        Candidate c = pick[i];
        c.n1 = b->n1;
        *st = apply_fused(b->plans[i], stream, c, b->use_tma != 0);
        if (*st != RS_OK) return INFINITY;
    }
    return total;
}

rs_status build_launch(rs_batch *b, cudaStream_t stream)
{
    const int n = int(b->plans.size());
    // maxima over the images carve the shared memory identically in every CTA
    fused::Work &w = b->work;
    std::memset(&w, 0, sizeof w);
    std::vector<int32_t> off(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const rs_plan *p = b->plans[i];
        const fused::Params &fp = p->fp;
        off[i + 1] = off[i] + (b->streamed[i] ? 0 : fp.tiles_y * fp.tiles_x);
        if (b->streamed[i]) continue;
        fused::Work r;
        work_regions(p, &r);
        w.tin_bytes = std::max(w.tin_bytes, r.tin_bytes);
        w.wy_bytes = std::max(w.wy_bytes, r.wy_bytes);
        w.wx_bytes = std::max(w.wx_bytes, r.wx_bytes);
        w.tt_bytes = std::max(w.tt_bytes, r.tt_bytes);
        w.rec2_bytes = std::max(w.rec2_bytes, r.rec2_bytes);
    }
    b->total_tiles = off[n];
    w.n_images = n;
    w.total_tiles = off[n];
    w.stages = b->stages;
    w.n1 = b->n1;
    w.use_tma = b->use_tma;
    b->smem = fused::layout_of(w.tin_bytes, w.wy_bytes, w.wx_bytes, w.tt_bytes, w.rec2_bytes,
                               b->use_tma ? b->stages : 1)
                  .total +
              fused::batch_extra(n);
    if (b->smem > 227 * 1024) return fail(RS_ERR_UNSUPPORTED, "batch: shared memory of the largest tiles too big");
    b->variant = b->plans[0]->variant;
    const int occ = occupancy(b->variant->fn, fused::kThreads, b->smem);
    if (occ < 1) return fail(RS_ERR_UNSUPPORTED, "batch: kernel does not fit on an SM");
    cudaError_t e = cudaSuccess;
    b->ctas = occ;
    b->grid = int(std::max<int64_t>(1, std::min<int64_t>(b->total_tiles, int64_t(occ) * b->plans[0]->num_sms)));

    // device arrays (re)allocated for this configuration
    b->dparams.~DeviceBuf();
    new (&b->dparams) DeviceBuf();
    b->dmaps.~DeviceBuf();
    new (&b->dmaps) DeviceBuf();
    b->dtileoff.~DeviceBuf();
    new (&b->dtileoff) DeviceBuf();
    e = cudaMalloc(&b->dparams.p, sizeof(fused::Params) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->dmaps.p, sizeof(CUtensorMap) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->dtileoff.p, sizeof(int32_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->dtileoff.p, off.data(), sizeof(int32_t) * (n + 1),
                                              cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch: allocating launch arrays");
    w.imgs = static_cast<const fused::Params *>(b->dparams.p);
    w.maps = static_cast<const CUtensorMap *>(b->dmaps.p);
    w.tile_off = static_cast<const int32_t *>(b->dtileoff.p);
    b->p0.err = static_cast<int *>(b->derr.p);

    // the two launch graphs
    for (int k = 0; k < 2; ++k) {
        if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
        if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
        b->exec[k] = nullptr;
        b->graph[k] = nullptr;
        b->staged_in[k].assign(n, nullptr);
        b->staged_out[k].assign(n, nullptr);
        e = cudaGraphCreate(&b->graph[k], 0);
        if (e != cudaSuccess) return cuda_fail(e, "batch: graph");
        unsigned char *hs = static_cast<unsigned char *>(b->host_stage[k]);
        const size_t pmap = ((sizeof(fused::Params) * size_t(n) + 63) / 64) * 64;
        cudaGraphNode_t n_par, n_map, n_ker;
        e = cudaGraphAddMemcpyNode1D(&n_par, b->graph[k], nullptr, 0, b->dparams.p, hs, sizeof(fused::Params) * n,
                                     cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaGraphAddMemcpyNode1D(&n_map, b->graph[k], nullptr, 0, b->dmaps.p, hs + pmap,
                                         sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice);
        void *args[3] = {&b->dummy_map, &b->p0, &b->work};
        cudaKernelNodeParams kp;
        std::memset(&kp, 0, sizeof kp);
        kp.func = const_cast<void *>(b->variant->fn);
        kp.gridDim = dim3(b->grid);
        kp.blockDim = dim3(fused::kThreads);
        kp.sharedMemBytes = unsigned(b->smem);
        kp.kernelParams = args;
        cudaGraphNode_t deps[2] = {n_par, n_map};
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n_ker, b->graph[k], deps, 2, &kp);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[k], b->graph[k], 0);
        if (e != cudaSuccess) return cuda_fail(e, "batch: building the launch graph");
    }
    return RS_OK;
}

rs_status configure(rs_batch *b, cudaStream_t stream, int G, int stages, int budget, int n1)
{
    b->G = G;
    b->stages = stages;
    b->budget_ctas = budget;
    b->n1 = n1;
    rs_status st;
    const double cost = plan_images(b, stream, G, stages, budget, true, &st);
    if (st != RS_OK) return st;
    if (!std::isfinite(cost)) return fail(RS_ERR_UNSUPPORTED, "batch: no configuration fits every image");
    return build_launch(b, stream);
}

bool valid_ptrs(const rs_batch *b, const void *const *d_in, void *const *d_out)
{
    if (!d_in || !d_out) return false;
    for (size_t i = 0; i < b->plans.size(); ++i)
        if (!d_in[i] || !d_out[i]) return false;
    return true;
}

} // namespace

extern "C" {

rs_status rs_batch_create(const rs_plan_desc *descs, int32_t n, void *stream_v, rs_batch **out)
{
    if (!out) return fail(RS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || n < 1 || n > (1 << 20)) return fail(RS_ERR_INVALID_ARG, "batch: need 1 .. 2^20 descriptors");
    for (int i = 1; i < n; ++i)
        if (descs[i].channels != descs[0].channels || descs[i].in_dtype != descs[0].in_dtype)
            return fail(RS_ERR_UNSUPPORTED, "batch: channels and dtype must be equal across the batch");
    if (descs[0].channels != 1 && descs[0].channels != 3)
        return fail(RS_ERR_UNSUPPORTED, "batch: 1 or 3 channels");
    for (int i = 0; i < n; ++i)
        if (descs[i].flags & RS_PREFILTER) return fail(RS_ERR_UNSUPPORTED, "batch: RS_PREFILTER is per plan only");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    rs_batch *b = new (std::nothrow) rs_batch();
    if (!b) return fail(RS_ERR_OOM, "host allocation failed");
    b->dtype = descs[0].in_dtype;
    b->C = descs[0].channels;
    bool all_tma = true;
    for (int i = 0; i < n; ++i) {
        rs_plan_desc d = descs[i];
        // the persistent launch runs the images on the SIMT tile kernel; large
        // ones may take the row-streaming kernel instead (decided below)
        d.flags &= ~uint32_t(RS_TWO_PASS | RS_FORCE_TC | RS_FORCE_STREAM);
        d.flags |= RS_FORCE_SIMT;
        rs_plan *p = nullptr;
        rs_status st = rs_plan_create(&d, stream, &p);
        if (st != RS_OK) {
            delete b;
            return st;
        }
        b->plans.push_back(p);
        if (p->path != 0) {
            delete b;
            return fail(RS_ERR_UNSUPPORTED, "batch: an image cannot use the fused kernel");
        }
        all_tma = all_tma && tma_layout_ok(p);
        b->out_pixels += int64_t(p->gy.n_out) * p->gx.n_out;
        b->in_bytes += int64_t(p->gy.n_in) * p->gx.n_in * b->C * int64_t(dt_size(b->dtype));
        b->out_bytes += int64_t(p->gy.n_out) * p->gx.n_out * b->C * int64_t(dt_size(b->dtype));
    }
    b->use_tma = all_tma ? 1 : 0;
    cudaError_t e = cudaMalloc(&b->derr.p, 16);
    if (e == cudaSuccess) e = cudaMemset(b->derr.p, 0, 16);
    b->streamed.assign(n, 0);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        rs_plan *p = b->plans[i];
        if (b->use_tma && p->stream_ok && int64_t(p->gy.n_out) * p->gx.n_out >= kStreamMinOut) {
            b->streamed[i] = 1;
            ++b->n_streamed;
            // one error word for the whole batch
            p->sp.err = p->xp.err = p->tcp.err = static_cast<int *>(b->derr.p);
            b->stream_order.push_back(i);
        }
    }
    std::stable_sort(b->stream_order.begin(), b->stream_order.end(), [b](int x, int y) {
        return int64_t(b->plans[x]->gy.n_out) * b->plans[x]->gx.n_out >
               int64_t(b->plans[y]->gy.n_out) * b->plans[y]->gx.n_out;
    });
    // the streamed upscales on the pipelined kernel: one multi-image launch per
    // (kernel, block size), their CTAs in order of the images (largest first);
    // where a launch takes several images, each is first re-planned for its
    // share of the SMs within it (by output pixels; its strip width and row
    // ranges chosen anew, its other choices kept), as for the band kernels
    // below
    {
        std::vector<int> rest;
        std::vector<std::tuple<const void *, int, int64_t, int>> xsum; // (kernel, block): pixels, images
        auto xsum_of = [&](const void *fn, int block) -> std::tuple<const void *, int, int64_t, int> & {
            for (auto &w : xsum)
                if (std::get<0>(w) == fn && std::get<1>(w) == block) return w;
            xsum.emplace_back(fn, block, 0, 0);
            return xsum.back();
        };
        for (const int i : b->stream_order)
            if (const void *fn = xstream::multi_kernel(b->plans[i])) {
                auto &w = xsum_of(fn, b->plans[i]->s_block);
                std::get<2>(w) += int64_t(b->plans[i]->gy.n_out) * b->plans[i]->gx.n_out;
                std::get<3>(w) += 1;
            }
        for (const int i : b->stream_order) {
            rs_plan *p = b->plans[i];
            const void *fn = xstream::multi_kernel(p);
            if (!fn) {
                rest.push_back(i);
                continue;
            }
            const auto &w = xsum_of(fn, p->s_block);
            if (std::get<3>(w) >= 2) {
                const int keep_sms = p->num_sms, keep_code = p->stream_code;
                stream::Opts o = stream::Opts::decode(keep_code);
                o.nr = 0;
                o.sw = 0;
                const double share = double(int64_t(p->gy.n_out) * p->gx.n_out) / double(std::max<int64_t>(1, std::get<2>(w)));
                p->num_sms = std::max(1, int(double(keep_sms) * share + 0.5));
                rs_status st = stream::setup(p, stream, o);
                p->num_sms = keep_sms;
                if (st != RS_OK || xstream::multi_kernel(p) != fn) st = stream::setup(p, stream, stream::Opts::decode(keep_code));
                if (st != RS_OK) {
                    delete b;
                    return st;
                }
                p->xp.err = static_cast<int *>(b->derr.p);
            }
            MultiGroup *g = nullptr;
            for (MultiGroup &h : b->groups)
                if (h.fn == fn && h.block == p->s_block) g = &h;
            if (!g) {
                b->groups.emplace_back();
                g = &b->groups.back();
                g->fn = fn;
                g->block = p->s_block;
                g->off.push_back(0);
            }
            g->imgs.push_back(i);
            g->smem = std::max(g->smem, p->s_smem);
            g->total += p->s_grid;
            g->off.push_back(g->total);
        }
        b->stream_order.swap(rest);
        // the band kernels' images (the streamed downscales): one multi-image
        // launch per band kernel, each image first re-planned for its share of
        // the SMs within its launch (by output pixels; its strip width chosen
        // anew for that share, its other choices kept); a kernel with one
        // image keeps its own launch
        std::vector<std::pair<const void *, int64_t>> wsum; // output pixels per band kernel
        auto wsum_of = [&](const void *fn) -> int64_t & {
            for (auto &w : wsum)
                if (w.first == fn) return w.second;
            wsum.emplace_back(fn, 0);
            return wsum.back().second;
        };
        for (const int i : b->stream_order)
            if (const void *fn = stream::multi_kernel(b->plans[i]))
                wsum_of(fn) += int64_t(b->plans[i]->gy.n_out) * b->plans[i]->gx.n_out;
        auto images_of = [&](const void *fn) {
            int n = 0;
            for (const int j : b->stream_order) n += stream::multi_kernel(b->plans[j]) == fn ? 1 : 0;
            return n;
        };
        rest.clear();
        for (const int i : b->stream_order) {
            rs_plan *p = b->plans[i];
            const void *fn0 = stream::multi_kernel(p);
            if (!fn0 || images_of(fn0) < 2) {
                rest.push_back(i);
                continue;
            }
            const int keep_sms = p->num_sms, keep_code = p->stream_code;
            const double w = double(int64_t(p->gy.n_out) * p->gx.n_out) / double(std::max<int64_t>(1, wsum_of(fn0)));
            p->num_sms = std::max(1, int(double(keep_sms) * w + 0.5));
            stream::Opts ob = stream::Opts::decode(keep_code);
            ob.sw = 0;
            rs_status st = stream::setup(p, stream, ob);
            p->num_sms = keep_sms;
            if (st != RS_OK || stream::multi_kernel(p) != fn0) st = stream::setup(p, stream, stream::Opts::decode(keep_code));
            if (st != RS_OK) {
                delete b;
                return st;
            }
            p->sp.err = static_cast<int *>(b->derr.p);
            const void *fn = stream::multi_kernel(p);
            MultiGroup *g = nullptr;
            for (MultiGroup &h : b->groups)
                if (h.kind == 1 && h.fn == fn) g = &h;
            if (!g) {
                b->groups.emplace_back();
                g = &b->groups.back();
                g->kind = 1;
                g->fn = fn;
                g->block = p->s_block;
                g->off.push_back(0);
            }
            g->imgs.push_back(i);
            g->smem = std::max(g->smem, p->s_smem);
            g->total += p->s_grid;
            g->off.push_back(g->total);
        }
        b->stream_order.swap(rest);
        for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
            MultiGroup &g = b->groups[gi];
            const size_t m = g.imgs.size();
            g.aux = int(gi % kAux);
            g.o_maps = ((g.kind ? sizeof(stream::Params) : sizeof(xstream::Params)) * m + 127) / 128 * 128;
            g.o_off = g.o_maps + sizeof(CUtensorMap) * m;
            g.bytes = g.o_off + sizeof(int32_t) * (m + 1);
            if (occupancy(g.fn, g.block, g.smem) < 1) {
                delete b;
                return fail(RS_ERR_UNSUPPORTED, "batch: multi-image streaming kernel does not fit an SM");
            }
            e = cudaMalloc(&g.dev.p, g.bytes);
            for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
                e = cudaHostAlloc(reinterpret_cast<void **>(&g.host[k]), g.bytes, cudaHostAllocDefault);
                if (e == cudaSuccess) {
                    std::memcpy(g.host[k] + g.o_off, g.off.data(), sizeof(int32_t) * (m + 1));
                    g.st_in[k].assign(m, nullptr);
                    g.st_out[k].assign(m, nullptr);
                }
            }
        }
    }
    if (e == cudaSuccess && b->n_streamed) {
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int k = 0; k < kAux && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
        }
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaHostAlloc(&b->host_stage[k], stage_bytes(n), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(b->done[k], stream);
    }
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "batch: allocations");
    }
    std::memset(&b->dummy_map, 0, sizeof b->dummy_map);
    // model-chosen launch-wide configuration: the cheapest (G, stages, budget)
    double best = INFINITY;
    int bg = 0, bs = 1, bb = 2;
    for (int G : {4, 2, 1}) {
        if (!b->plans[0]->variant) break;
        for (int stages : {2, 1}) {
            if (stages == 2 && !b->use_tma) continue;
            for (int budget : {2, 3}) {
                rs_status st;
                const double c = plan_images(b, stream, G, stages, budget, false, &st);
                if (c < best) {
                    best = c;
                    bg = G;
                    bs = stages;
                    bb = budget;
                }
            }
        }
    }
    if (!std::isfinite(best)) {
        delete b;
        return fail(RS_ERR_UNSUPPORTED, "batch: no configuration fits every image");
    }
    rs_status st = configure(b, stream, bg, bs, bb, 4);
    if (st != RS_OK) {
        delete b;
        return st;
    }
    *out = b;
    return RS_OK;
}

rs_status rs_batch_run(rs_batch *b, const void *const *d_in, void *const *d_out, void *stream_v)
{
    const Range range("rs_batch_run");
    if (!b || !valid_ptrs(b, d_in, d_out)) return fail(RS_ERR_INVALID_ARG, "batch: NULL batch or buffer");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    const int n = int(b->plans.size());
    if (b->use_tma)
        for (int i = 0; i < n; ++i)
            if (reinterpret_cast<uintptr_t>(d_in[i]) & 15u)
                return fail(RS_ERR_INVALID_ARG, "batch: inputs must be 16-byte aligned (planned for TMA)");
    const int k = b->next;
    b->next ^= 1;
    // the staging buffer k was last read by the run recorded on done[k]
    cudaError_t e = cudaEventSynchronize(b->done[k]);
    if (e != cudaSuccess) return cuda_fail(e, "batch: waiting for the staging buffer");
    unsigned char *hs = static_cast<unsigned char *>(b->host_stage[k]);
    fused::Params *hp = reinterpret_cast<fused::Params *>(hs);
    CUtensorMap *hm = reinterpret_cast<CUtensorMap *>(hs + ((sizeof(fused::Params) * size_t(n) + 63) / 64) * 64);
    for (int i = 0; i < n; ++i) {
        if (b->staged_in[k][i] == d_in[i] && b->staged_out[k][i] == d_out[i]) continue;
        fused::Params fp = b->plans[i]->fp;
        fp.in = d_in[i];
        fp.out = d_out[i];
        fp.use_tma = b->use_tma;
        fp.err = b->p0.err;
        hp[i] = fp;
        if (b->use_tma) {
            rs_status st = encode_tensor_map(b->plans[i], d_in[i], &hm[i]);
            if (st != RS_OK) return st;
        } else {
            std::memset(&hm[i], 0, sizeof(CUtensorMap));
        }
        b->staged_in[k][i] = d_in[i];
        b->staged_out[k][i] = d_out[i];
    }
    if (b->n_streamed) {
        // the streamed images, largest first, dealt over side streams forked
        // from `stream` (after the work already queued there) and joined back
        // after the graph, so they overlap one another and the persistent
        // kernel (whose CTAs never wait on one another)
        e = cudaEventRecord(b->fork, stream);
        for (int a = 0; a < kAux && e == cudaSuccess; ++a) e = cudaStreamWaitEvent(b->aux[a], b->fork, 0);
        if (e != cudaSuccess) return cuda_fail(e, "batch: forking the side streams");
    }
    e = cudaGraphLaunch(b->exec[k], stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch: graph launch");
    if (b->n_streamed) {
        for (MultiGroup &g : b->groups) {
            const size_t m = g.imgs.size();
            CUtensorMap *hm = reinterpret_cast<CUtensorMap *>(g.host[k] + g.o_maps);
            for (size_t j = 0; j < m; ++j) {
                const int i = g.imgs[j];
                if (g.st_in[k][j] == d_in[i] && g.st_out[k][j] == d_out[i]) continue;
                if (g.kind == 0) {
                    xstream::Params xp = b->plans[i]->xp;
                    xp.in = d_in[i];
                    xp.out = d_out[i];
                    xp.err = static_cast<int *>(b->derr.p);
                    reinterpret_cast<xstream::Params *>(g.host[k])[j] = xp;
                } else {
                    stream::Params sp = b->plans[i]->sp;
                    sp.in = d_in[i];
                    sp.out = d_out[i];
                    sp.err = static_cast<int *>(b->derr.p);
                    reinterpret_cast<stream::Params *>(g.host[k])[j] = sp;
                }
                const rs_status st = stream::encode_input_map(b->plans[i], d_in[i], &hm[j]);
                if (st != RS_OK) return st;
                g.st_in[k][j] = d_in[i];
                g.st_out[k][j] = d_out[i];
            }
            cudaStream_t as = b->aux[g.aux];
            e = cudaMemcpyAsync(g.dev.p, g.host[k], g.bytes, cudaMemcpyHostToDevice, as);
            xstream::Multi mu;
            stream::Multi ms;
            mu.ps = static_cast<const xstream::Params *>(g.dev.p);
            ms.ps = static_cast<const stream::Params *>(g.dev.p);
            mu.maps = ms.maps = reinterpret_cast<const CUtensorMap *>(static_cast<char *>(g.dev.p) + g.o_maps);
            mu.cta_off = ms.cta_off = reinterpret_cast<const int32_t *>(static_cast<char *>(g.dev.p) + g.o_off);
            mu.n = ms.n = int32_t(m);
            void *args[1] = {g.kind ? static_cast<void *>(&ms) : static_cast<void *>(&mu)};
            if (e == cudaSuccess) e = cudaLaunchKernel(g.fn, dim3(g.total), dim3(g.block), args, g.smem, as);
            if (e != cudaSuccess) return cuda_fail(e, "batch: multi-image streaming launch");
        }
        for (size_t j = 0; j < b->stream_order.size(); ++j) {
            const int i = b->stream_order[j];
            const rs_status st =
                stream::launch(b->plans[i], d_in[i], d_out[i], b->aux[(j + b->groups.size()) % kAux]);
            if (st != RS_OK) return st;
        }
        for (int a = 0; a < kAux && e == cudaSuccess; ++a) {
            e = cudaEventRecord(b->join[a], b->aux[a]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, b->join[a], 0);
        }
        if (e != cudaSuccess) return cuda_fail(e, "batch: joining the side streams");
    }
    e = cudaEventRecord(b->done[k], stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch: graph launch");
    return RS_OK;
}

rs_status rs_batch_autotune(rs_batch *b, const void *const *d_in, void *const *d_out, void *stream_v,
                            const char *cache_path)
{
    if (!b || !valid_ptrs(b, d_in, d_out)) return fail(RS_ERR_INVALID_ARG, "batch: NULL batch or buffer");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    // cache key: the count and a hash of the descriptors
    uint64_t h = 1469598103934665603ull;
    for (rs_plan *p : b->plans) {
        const unsigned char *q = reinterpret_cast<const unsigned char *>(&p->desc);
        for (size_t i = 0; i < sizeof(rs_plan_desc); ++i) h = (h ^ q[i]) * 1099511628211ull;
    }
    char key[128];
    std::snprintf(key, sizeof key, "batch|n%zu|h%016llx", b->plans.size(), (unsigned long long)h);
    if (cache_path) {
        FILE *f = std::fopen(cache_path, "r");
        if (f) {
            char line[512];
            int G = 0, st = 0, bud = 0, n1 = 0;
            bool hit = false;
            while (std::fgets(line, sizeof line, f)) {
                if (!std::strstr(line, key)) continue;
                const char *q = std::strstr(line, "\"G\":");
                if (q && std::sscanf(q, "\"G\": %d, \"stages\": %d, \"budget\": %d, \"n1\": %d", &G, &st, &bud,
                                     &n1) == 4)
                    hit = true;
            }
            std::fclose(f);
            if (hit) return configure(b, stream, G, st, bud, n1);
        }
    }
    auto time_run = [&](double *ms_out) -> rs_status {
        cudaEvent_t a, c;
        cudaEventCreate(&a);
        cudaEventCreate(&c);
        rs_status s = rs_batch_run(b, d_in, d_out, stream);
        cudaEventRecord(a, stream);
        for (int r = 0; r < 3 && s == RS_OK; ++r) s = rs_batch_run(b, d_in, d_out, stream);
        cudaEventRecord(c, stream);
        cudaError_t e = cudaEventSynchronize(c);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, c);
        cudaEventDestroy(a);
        cudaEventDestroy(c);
        if (s != RS_OK) return s;
        if (e != cudaSuccess) return cuda_fail(e, "batch: timing");
        int herr = 0;
        e = cudaMemcpy(&herr, b->derr.p, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "batch: error word");
        if (herr) return fail(RS_ERR_DEVICE, "batch: device error word set while tuning");
        *ms_out = ms / 3.0;
        return RS_OK;
    };
    struct Cfg {
        int G, stages, budget, n1;
    };
    Cfg best{b->G, b->stages, b->budget_ctas, b->n1};
    double best_ms = INFINITY;
    std::vector<Cfg> trial;
    for (int G : {4, 2, 1})
        for (int stages : {2, 1})
            for (int budget : {2, 3}) {
                if (stages == 2 && !b->use_tma) continue;
                trial.push_back({G, stages, budget, 4});
            }
    for (const Cfg &c : trial) {
        if (configure(b, stream, c.G, c.stages, c.budget, c.n1) != RS_OK) continue;
        double ms;
        rs_status s = time_run(&ms);
        if (s != RS_OK) return s;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    const Cfg coarse = best;
    for (int n1 = 2; n1 <= 6; ++n1) {
        if (n1 == coarse.n1) continue;
        Cfg c = coarse;
        c.n1 = n1;
        if (configure(b, stream, c.G, c.stages, c.budget, c.n1) != RS_OK) continue;
        double ms;
        rs_status s = time_run(&ms);
        if (s != RS_OK) return s;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    rs_status s = configure(b, stream, best.G, best.stages, best.budget, best.n1);
    if (s != RS_OK) return s;
    if (cache_path && std::isfinite(best_ms)) {
        FILE *f = std::fopen(cache_path, "a");
        if (f) {
            std::fprintf(f, "{\"key\": \"%s\", \"G\": %d, \"stages\": %d, \"budget\": %d, \"n1\": %d, \"ms\": %.4f}\n",
                         key, best.G, best.stages, best.budget, best.n1, best_ms);
            std::fclose(f);
        }
    }
    return RS_OK;
}

rs_status rs_batch_image_path(const rs_batch *b, int32_t index, int32_t *path)
{
    if (!b || !path || index < 0 || index >= int32_t(b->plans.size()))
        return fail(RS_ERR_INVALID_ARG, "batch: bad image index");
    const rs_plan *p = b->plans[size_t(index)];
    *path = b->streamed[size_t(index)] ? (p->tcs_on ? 5 : 3) : 0;
    return RS_OK;
}

rs_status rs_batch_get_info(const rs_batch *b, rs_batch_info *info)
{
    if (!b || !info) return fail(RS_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof *info);
    info->n_images = int32_t(b->plans.size());
    info->total_tiles = b->total_tiles;
    info->group = b->G;
    info->warps_pass1 = b->n1;
    info->stages = b->use_tma ? b->stages : 1;
    info->use_tma = b->use_tma;
    info->smem_bytes = int32_t(b->smem);
    info->ctas_per_sm = b->ctas;
    info->grid = b->grid;
    info->out_pixels = b->out_pixels;
    info->in_bytes = b->in_bytes;
    info->out_bytes = b->out_bytes;
    info->n_streamed = b->n_streamed;
    return RS_OK;
}

rs_status rs_batch_destroy(rs_batch *b)
{
    if (!b) return RS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    // report a device-side error raised by the batch kernel before freeing
    int herr = 0;
    if (e == cudaSuccess && b->derr.p) e = cudaMemcpy(&herr, b->derr.p, 4, cudaMemcpyDeviceToHost);
    delete b;
    if (e != cudaSuccess) return cuda_fail(e, "batch: synchronising before destroy");
    if (herr) return fail(RS_ERR_DEVICE, "batch: device error word set");
    return RS_OK;
}

} // extern "C"
