// rs_cluster.cu -- the paper's parallel merging clustering of ToF frames
// (Sec. "Parallel Merging Algorithm", "Merging Criterion"; Eq. 1, Eq. 2, the
// phi equation; Table 1), one thread block per frame, no host round trip
// between rounds.
//
// Every pixel starts as a region whose ID is its linear index, with the
// descriptor w = (z, phi), phi = arctan(d sqrt(I)).  A round has four phases
// separated by block barriers:
//   1. clear each live region's best candidate;
//   2. for every 4-neighbourhood pixel pair lying in two regions R != S whose
//      descriptors pass |dz| <= t_z and |dphi| <= t_phi, offer S to R and R
//      to S with f = alpha_z |dz| + alpha_phi |dphi|: a 64-bit atomicMin on
//      (f, ~ID) keeps the minimal f, ties going to the larger ID;
//   3. a region whose choice is mutual and whose ID is the smaller one merges
//      into its partner: the partner adds its running sums and pixel count
//      and recomputes its means (each region merges at most once a round, so
//      no two threads write one region);
//   4. boundary pairs and live regions follow the merges (pairs now inside
//      one region, and merged-away regions, leave their lists).
// Rounds stop when phase 2 finds no qualifying pair (then no region has a
// partner) or after max_rounds.  Every decision is taken in FP32 with each
// operation rounded on its own (no contraction into FMAs), so an FP32
// reference taking the same steps reaches the same partition; phi is the FP64
// arctan of the FP32 inputs rounded to FP32.
#include <cmath>
#include <cstring>
#include <new>

#include "rs_plan.h"

struct rs_cluster {
    rs_cluster_desc desc{};
    rs::DeviceBuf scratch;
    size_t per_frame = 0; // bytes of scratch per frame
};

namespace rs {
namespace cluster {
namespace {

constexpr int kThreads = 512;
constexpr unsigned long long kNone = ~0ull;

struct Args {
    const float *z, *d, *inten; // [frames][h * w]
    int32_t *labels;            // [frames][h * w]
    int32_t *rounds;            // [frames]
    float *out_z, *out_phi;     // [frames][h * w] by region ID (optional)
    int32_t *out_size;          // [frames][h * w] by region ID (optional; 0: merged away)
    unsigned char *scratch;
    size_t per_frame;
    int32_t h, w, max_rounds;
    float t_z, t_phi, a_z, a_phi;
};

__device__ __forceinline__ unsigned long long key(float f, int32_t id)
{
    return (static_cast<unsigned long long>(__float_as_uint(f)) << 32) | (0xffffffffu - static_cast<uint32_t>(id));
}

__device__ __forceinline__ int32_t partner_of(unsigned long long k)
{
    return static_cast<int32_t>(0xffffffffu - static_cast<uint32_t>(k & 0xffffffffu));
}

// Scratch of one frame of n pixels (byte offsets; every piece 16-byte aligned).
struct Layout {
    size_t sum_z, sum_p, mean_z, mean_p, size, parent, best, edges0, edges1, live0, live1, total;
};

__host__ __device__ inline Layout layout_of(size_t n)
{
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t r = o;
        o += (bytes + 15) / 16 * 16;
        return r;
    };
    L.sum_z = take(n * 4);
    L.sum_p = take(n * 4);
    L.mean_z = take(n * 4);
    L.mean_p = take(n * 4);
    L.size = take(n * 4);
    L.parent = take(n * 4);
    L.best = take(n * 8);
    L.edges0 = take(n * 16); // up to 2n edges of (label, label)
    L.edges1 = take(n * 16);
    L.live0 = take(n * 4);
    L.live1 = take(n * 4);
    L.total = (o + 255) / 256 * 256;
    return L;
}

// The rounds run over two shrinking lists instead of every pixel: the
// region-boundary edges (4-neighbourhood pixel pairs, kept as the pair of
// their current region IDs; a pair inside one region stays inside it, so it
// is dropped for good) and the live regions.  Pixel labels are resolved once
// at the end by pointer jumping along the merge links (each link points to a
// larger ID, so they form trees whose roots are the final regions).
__global__ void __launch_bounds__(kThreads) cluster_kernel(const Args a)
{
    const int64_t n = int64_t(a.h) * a.w;
    const int64_t off = int64_t(blockIdx.x) * n;
    unsigned char *sc = a.scratch + size_t(blockIdx.x) * a.per_frame;
    const Layout L = layout_of(size_t(n));
    float *sum_z = reinterpret_cast<float *>(sc + L.sum_z);
    float *sum_p = reinterpret_cast<float *>(sc + L.sum_p);
    float *mean_z = reinterpret_cast<float *>(sc + L.mean_z);
    float *mean_p = reinterpret_cast<float *>(sc + L.mean_p);
    int32_t *size = reinterpret_cast<int32_t *>(sc + L.size);
    int32_t *parent = reinterpret_cast<int32_t *>(sc + L.parent);
    unsigned long long *best = reinterpret_cast<unsigned long long *>(sc + L.best);
    int2 *edges[2] = {reinterpret_cast<int2 *>(sc + L.edges0), reinterpret_cast<int2 *>(sc + L.edges1)};
    int32_t *live[2] = {reinterpret_cast<int32_t *>(sc + L.live0), reinterpret_cast<int32_t *>(sc + L.live1)};
    int32_t *lab = a.labels + off;
    __shared__ int any, n_edges_next, n_live_next, changed;

    // every pixel a region; edge 2p = (p, right neighbour), 2p + 1 = (p, lower
    // neighbour); a missing neighbour gives an inner pair, dropped in the first merge round
    for (int64_t p = threadIdx.x; p < n; p += kThreads) {
        const float zf = a.z[off + p];
        const float ph = float(atan(double(a.d[off + p]) * sqrt(double(a.inten[off + p]))));
        parent[p] = int32_t(p);
        size[p] = 1;
        sum_z[p] = mean_z[p] = zf;
        sum_p[p] = mean_p[p] = ph;
        live[0][p] = int32_t(p);
        const int64_t y = p / a.w, x = p - y * a.w;
        edges[0][2 * p] = make_int2(int32_t(p), int32_t(x + 1 < a.w ? p + 1 : p));
        edges[0][2 * p + 1] = make_int2(int32_t(p), int32_t(y + 1 < a.h ? p + a.w : p));
    }
    int n_edges = int(2 * n), n_live = int(n), cur = 0;
    __syncthreads();

    int r = 0;
    for (; r < a.max_rounds; ++r) {
        const int2 *E = edges[cur];
        const int32_t *V = live[cur];
        // 1. clear the live regions' candidates
        for (int i = threadIdx.x; i < n_live; i += kThreads) best[V[i]] = kNone;
        if (threadIdx.x == 0) {
            any = 0;
            n_edges_next = 0;
            n_live_next = 0;
        }
        __syncthreads();
        // 2. offers over the boundary edges that pass Eq. 1
        for (int i = threadIdx.x; i < n_edges; i += kThreads) {
            const int2 e = E[i];
            const int32_t R = e.x, S = e.y;
            if (R == S) continue;
            const float dz = fabsf(__fsub_rn(mean_z[R], mean_z[S]));
            const float dp = fabsf(__fsub_rn(mean_p[R], mean_p[S]));
            if (!(dz <= a.t_z && dp <= a.t_phi)) continue;
            const float f = __fadd_rn(__fmul_rn(a.a_z, dz), __fmul_rn(a.a_phi, dp));
            atomicMin(&best[R], key(f, S));
            atomicMin(&best[S], key(f, R));
            any = 1;
        }
        __syncthreads();
        if (!any) break;
        // 3. mutual choices: the smaller ID merges into the larger
        for (int i = threadIdx.x; i < n_live; i += kThreads) {
            const int32_t R = V[i];
            const unsigned long long b = best[R];
            if (b == kNone) continue;
            const int32_t S = partner_of(b);
            const unsigned long long bs = best[S]; // never empty: offers go both ways
            if (R < S && bs != kNone && partner_of(bs) == R) {
                const float sz = __fadd_rn(sum_z[S], sum_z[R]);
                const float sp = __fadd_rn(sum_p[S], sum_p[R]);
                const int32_t cnt = size[S] + size[R];
                sum_z[S] = sz;
                sum_p[S] = sp;
                size[S] = cnt;
                size[R] = 0;
                mean_z[S] = __fdiv_rn(sz, float(cnt));
                mean_p[S] = __fdiv_rn(sp, float(cnt));
                parent[R] = S;
            }
        }
        __syncthreads();
        // 4. follow this round's merges: relabel and keep the boundary edges,
        // keep the regions that did not merge away
        int2 *En = edges[cur ^ 1];
        int32_t *Vn = live[cur ^ 1];
        for (int i = threadIdx.x; i < n_edges; i += kThreads) {
            const int2 e = E[i];
            const int32_t R = parent[e.x], S = parent[e.y];
            if (R != S) En[atomicAdd(&n_edges_next, 1)] = make_int2(R, S);
        }
        for (int i = threadIdx.x; i < n_live; i += kThreads) {
            const int32_t R = V[i];
            if (parent[R] == R) Vn[atomicAdd(&n_live_next, 1)] = R;
        }
        __syncthreads();
        n_edges = n_edges_next;
        n_live = n_live_next;
        cur ^= 1;
        __syncthreads(); // the counters are reset only after every thread has read them
    }
    // pixel labels: the root of each pixel's merge tree, by pointer jumping
    for (int it = 0; it < 64; ++it) {
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        for (int64_t p = threadIdx.x; p < n; p += kThreads) {
            const int32_t q = parent[p], g = parent[q];
            if (g != q) {
                parent[p] = g;
                changed = 1;
            }
        }
        __syncthreads();
        if (!changed) break;
        __syncthreads();
    }
    for (int64_t p = threadIdx.x; p < n; p += kThreads) lab[p] = parent[p];
    if (threadIdx.x == 0) a.rounds[blockIdx.x] = r;
    if (a.out_z || a.out_phi || a.out_size)
        for (int64_t p = threadIdx.x; p < n; p += kThreads) {
            if (a.out_z) a.out_z[off + p] = mean_z[p];
            if (a.out_phi) a.out_phi[off + p] = mean_p[p];
            if (a.out_size) a.out_size[off + p] = size[p];
        }
}

} // namespace
} // namespace cluster
} // namespace rs

using namespace rs;

extern "C" {

rs_status rs_cluster_create(const rs_cluster_desc *desc, rs_cluster **out)
{
    if (!out) return fail(RS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(RS_ERR_INVALID_ARG, "NULL descriptor");
    const rs_cluster_desc &d = *desc;
    if (d.n_frames < 1 || d.height < 1 || d.width < 1 || int64_t(d.height) * d.width > (int64_t(1) << 24))
        return fail(RS_ERR_INVALID_ARG, "cluster: need frames >= 1 and 1 <= height * width <= 2^24");
    if (!(d.t_z >= 0.0f) || !(d.t_phi >= 0.0f) || !(d.alpha_z >= 0.0f) || !(d.alpha_phi >= 0.0f) ||
        !std::isfinite(d.alpha_z) || !std::isfinite(d.alpha_phi))
        return fail(RS_ERR_INVALID_ARG, "cluster: thresholds and weights must be >= 0 (weights finite)");
    if (d.max_rounds < 0) return fail(RS_ERR_INVALID_ARG, "cluster: max_rounds < 0");
    rs_cluster *c = new (std::nothrow) rs_cluster();
    if (!c) return fail(RS_ERR_OOM, "host allocation failed");
    c->desc = d;
    const size_t n = size_t(d.height) * d.width;
    c->per_frame = cluster::layout_of(n).total;
    const cudaError_t e = cudaMalloc(&c->scratch.p, c->per_frame * size_t(d.n_frames));
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cluster: allocating the region state");
    }
    c->scratch.n = c->per_frame * size_t(d.n_frames);
    *out = c;
    return RS_OK;
}

rs_status rs_cluster_run(rs_cluster *c, const float *z, const float *d, const float *intensity, int32_t *labels,
                         int32_t *rounds, float *region_z, float *region_phi, int32_t *region_size, void *stream)
{
    const Range range("rs_cluster_run");
    if (!c || !z || !d || !intensity || !labels || !rounds)
        return fail(RS_ERR_INVALID_ARG, "cluster: NULL handle or buffer");
    const rs_cluster_desc &dd = c->desc;
    cluster::Args a;
    a.z = z;
    a.d = d;
    a.inten = intensity;
    a.labels = labels;
    a.rounds = rounds;
    a.out_z = region_z;
    a.out_phi = region_phi;
    a.out_size = region_size;
    a.scratch = static_cast<unsigned char *>(c->scratch.p);
    a.per_frame = c->per_frame;
    a.h = dd.height;
    a.w = dd.width;
    a.max_rounds = dd.max_rounds > 0 ? dd.max_rounds : int32_t(std::min<int64_t>(int64_t(dd.height) * dd.width, 1 << 30));
    a.t_z = dd.t_z;
    a.t_phi = dd.t_phi;
    a.a_z = dd.alpha_z;
    a.a_phi = dd.alpha_phi;
    void *args[1] = {&a};
    const cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void *>(&cluster::cluster_kernel),
                                           dim3(unsigned(dd.n_frames)), dim3(cluster::kThreads), args, 0,
                                           static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cluster kernel launch");
    return RS_OK;
}

rs_status rs_cluster_destroy(rs_cluster *c)
{
    if (!c) return RS_OK;
    const cudaError_t e = cudaDeviceSynchronize();
    delete c;
    if (e != cudaSuccess) return cuda_fail(e, "cluster: synchronising before destroy");
    return RS_OK;
}

} // extern "C"
