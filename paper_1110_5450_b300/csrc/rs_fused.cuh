// rs_fused.cuh -- fused separable resampling kernel (one launch per image).
//
// A persistent CTA walks output tiles of tile_h x tile_w pixels.  For each
// tile it stages in shared memory
//   * the input rectangle the tile's taps touch (TMA 2-D tile copy), and
//   * the tile's weight bands of both axes (TMA 1-D bulk copies),
// double-buffered behind one mbarrier per stage (or plain coalesced loads
// when the image's row pitch rules TMA out), then computes
//
//   pass 1 (vertical):   tt[yo][s]     = sum_j Wy[yo][j] tin[by(yo) + j][s]
//   pass 2 (horizontal): out[yo][x][c] = sum_j Wx[x][j] tt[yo][(bx(x) + j) C + c]
//
// The warps are specialised and pipelined: warps [0, n1) stage tiles and run
// pass 1 of tile i into intermediate buffer i % 2, while warps [n1, 8) run
// pass 2 of tile i - 1 from the other buffer.  The hand-off goes through
// mbarriers (tt full / tt empty per buffer, bounded waits), so no CTA-wide
// barrier separates the two passes.
//
// Weight bands: outputs are grouped G at a time along an axis; group g reads
// the J consecutive inputs [base[g], base[g] + J) and stores its weights
// j-major ([j][member]), zero outside each member's own taps, so one
// shared-memory vector load gives the G weights of input j and one data load
// feeds G fused multiply-adds (times V columns per thread in pass 1).
//
// Bank conflicts:
//   pass 1: lanes take consecutive samples of a staged row -> conflict-free
//           for any pitch, so the TMA's dense box layout is read as it lands;
//   pass 2: lanes take consecutive output ROWS (weights warp-uniform); the
//           intermediate's pitch is odd in accumulation words, so rows hit
//           distinct banks.
#pragma once

#include <cuda.h>

#include <climits>
#include <type_traits>

#include "rs_internal.h"
#include "rs_tc.cuh"

namespace rs {
namespace fused {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kErrBounds = 201;  // a band would read outside the staged tile
constexpr int kErrTimeout = 202; // an mbarrier wait ran out
constexpr int kErrCheck = 203;   // an RS_CHECK table check failed
constexpr int kOffCache = 2048;  // batch tile prefix sums kept in shared memory
constexpr int kPrefetch = 2;     // tiles ahead whose input is prefetched into L2

template <typename A, typename T> __device__ __forceinline__ A to_acc(T v);
template <> __device__ __forceinline__ float to_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float to_acc<float, __half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_acc<float, __nv_bfloat16>(__nv_bfloat16 v)
{
    return __bfloat162float(v);
}
template <> __device__ __forceinline__ double to_acc<double, double>(double v) { return v; }

template <typename T, typename A> __device__ __forceinline__ T from_acc(A v);
template <> __device__ __forceinline__ float from_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_acc<__half, float>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16, float>(float v)
{
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ double from_acc<double, double>(double v) { return v; }

template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// One wait attempt; the warp may be parked by the hardware for up to ~20 µs
// while the phase is incomplete (it wakes as soon as the phase completes), so
// waiting warps do not spin on the issue slots of working warps.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: gives up after ~2 s of wall time (a correct copy lands in
// microseconds) and reports false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 3u) == 3u && global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// 3-D tile copy; used with the box {8 samples, rows, sample chunks}, which
// lands an input tile in the canonical MN-major operand layout of the tensor
// cores (8 x 8 core matrices, rows 16 bytes apart, chunks rows*16 bytes apart).
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// L2 prefetch of a 2-D / 3-D tile (no shared memory, no completion): warms
// L2 for a later tile copy so that its latency is an L2 hit, not DRAM.
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int x, int y, int z)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void flag(int *err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

struct Params {
    const void *in;
    void *out;
    int64_t in_h, in_w, out_h, out_w;
    int64_t in_stride, out_stride;
    const int32_t *base_y, *base_x;
    const void *band_y, *band_x; // [groups][js] accumulation type
    int32_t J;                   // band width (inputs per group)
    int32_t js_y, js_x;          // slot strides (elements) of the two bands: the
                                 // vertical band of the FP32 path stores every
                                 // weight twice, the horizontal band interleaves
                                 // group pairs (both for packed-pair FMAs)
    int32_t tile_h, tile_w;      // output tile (multiples of G)
    int32_t box_h, box_w;        // staged rows, staged samples (pitch of tin)
    int32_t sub_h, n_sub;        // TMA box height and copies per tile
    int32_t pitch_t;             // pitch of the intermediate (odd, >= the pass-1 width)
    int32_t w1;                  // pass-1 width: box_w rounded up to 32*V columns
    int32_t tiles_y, tiles_x;
    int32_t groups_y, groups_x;
    int use_tma;                 // 1: TMA copies; 0: plain coalesced loads
    int stages;                  // staged buffers (2 = prefetch the next tile; TMA only)
    int n1;                      // warps running staging + pass 1 (the rest run pass 2)
    int *err;
    // tensor-core vertical pass: M blocks of 128 staged samples, staged rows
    // (= box_h, the GEMM's K, a multiple of 16); zero on the SIMT path
    int32_t tc_nmb, tc_kpad, tc_pad0, tc_pad1;
};
static_assert(sizeof(Params) % 16 == 0, "Params must keep 16-byte multiples (records copy it word by word)");

// Work of one launch: a single image, or a batch of images whose tiles are
// concatenated image after image.  CTA b takes tiles b, b + grid, b + 2 grid,
// ... of that list, so every image's tiles spread over all CTAs.
struct Work {
    const Params *imgs;      // batch: device array of per-image parameters; nullptr: single image
    const CUtensorMap *maps; // batch: per-image tensor maps in global memory (64-byte aligned)
    const int32_t *tile_off; // batch: tiles of images [0, k) = tile_off[k], n_images + 1 entries
    int32_t n_images;
    int32_t total_tiles;
    // shared-memory carving: byte sizes of the regions (maxima over the
    // images), and launch-wide choices
    int32_t tin_bytes, wy_bytes, wx_bytes, tt_bytes, rec2_bytes;
    int32_t stages, n1, use_tma;
    int32_t tc_b_bytes; // tensor-core path: weight matrices (hi + lo) region
    int32_t tc_cols;    // tensor-core path: tensor-memory columns to allocate
};

struct TileInfo {
    Params P;       // parameters of the tile's image
    int32_t img;    // image index, -1 marks the end of the work
    int32_t t;      // tile index within the image
    int32_t ry0;    // first staged input row
    int32_t xs;     // first staged input sample (aligned down to 16 bytes)
    int32_t nvy;    // valid y-groups in the tile
    int32_t nvx;    // valid x-groups in the tile
    int32_t rb[32]; // per y-group: first staged row of its band (base - ry0)
    int32_t cb[32]; // per x-group: first staged sample of its band (base * C - xs)
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Loads G consecutive weights (16-byte aligned for G = 4 floats).
template <typename A, int G> __device__ __forceinline__ void load_w(A (&w)[G], const A *p)
{
    if constexpr (G == 4 && sizeof(A) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
    } else if constexpr (G == 2 && sizeof(A) == 4) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        w[0] = v.x;
        w[1] = v.y;
    } else {
#pragma unroll
        for (int g = 0; g < G; ++g) w[g] = p[g];
    }
}

// Pass-2 record of one intermediate buffer (written by the pass-1 warps).
struct Rec2 {
    Params P;   // parameters of the tile's image
    int32_t img, ty, tx, nvx;
    int32_t cb[32];
};

// Horizontal band slots of a tile of ngx groups (groups run in pairs).
__host__ __device__ inline int pair_slots(int ngx) { return (ngx + 1) / 2; }

__host__ __device__ inline size_t rec2_bytes(int ngx, int js, size_t acc)
{
    return align_up(sizeof(Rec2) + size_t(pair_slots(ngx)) * js * acc, 128);
}

// Shared-memory layout: stages x (tin, wy, wx) | 2 x tt | 2 x (Rec2 + wx copy)
// | tensor-core weight matrices (TC path) | 2 x TileInfo | 7 mbarriers, abort
// flag, tensor-memory address | batch tile prefix sums | read slack.
struct Layout {
    size_t tin, wy, wx, stage, tt, rec2, bmat, total;
};

__host__ __device__ inline Layout layout_of(size_t tin, size_t wy, size_t wx, size_t tt, size_t rec2, int nstage,
                                            size_t bmat = 0)
{
    Layout L;
    L.tin = tin;
    L.wy = wy;
    L.wx = wx;
    L.stage = L.tin + L.wy + L.wx;
    L.tt = tt;
    L.rec2 = rec2;
    L.bmat = align_up(bmat, 128);
    L.total = 128 + size_t(nstage) * L.stage + 2 * L.tt + 2 * L.rec2 + L.bmat + align_up(2 * sizeof(TileInfo), 128) +
              64 + 1024;
    return L;
}

// Extra dynamic shared memory of a batch launch: its tile prefix sums.
__host__ __device__ inline size_t batch_extra(int n_images)
{
    return n_images + 1 <= kOffCache ? align_up(size_t(n_images + 1) * 4, 128) : 0;
}

__host__ __device__ inline Layout layout(size_t elem, size_t acc, int box_h, int box_w, int ngy, int ngx, int js_y,
                                         int js_x, int tile_h, int pitch_t, int nstage)
{
    Layout L;
    L.tin = align_up(size_t(box_h) * box_w * elem, 128);
    L.wy = align_up(size_t(ngy) * js_y * acc, 128);
    L.wx = align_up(size_t(pair_slots(ngx)) * js_x * acc, 128);
    L.stage = L.tin + L.wy + L.wx;
    L.tt = align_up(size_t(tile_h) * pitch_t * acc, 128);
    L.rec2 = rec2_bytes(ngx, js_x, acc);
    L.bmat = 0;
    // + slack because the vertical pass reads whole 32*V-column chunks past
    // the last staged row
    L.total = 128 + size_t(nstage) * L.stage + 2 * L.tt + 2 * L.rec2 + align_up(2 * sizeof(TileInfo), 128) + 64 +
              1024;
    return L;
}

// Bounded wait that also honours the CTA abort flag; false on timeout/abort.
// limit_ns: wall time before giving up (2 s in every kernel; the wait
// self-test passes a shorter one).
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err,
                                              uint64_t limit_ns = 2000000000ull)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 3u) == 3u) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > limit_ns) {
                flag(err, kErrTimeout);
                *abort_flag = 1;
                return false;
            }
        }
    }
    flag(err, kErrTimeout);
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void named_sync(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Packed FP32 pairs (Blackwell fma.rn.f32x2: two independent round-to-nearest
// FMAs in one instruction, bitwise equal to two scalar FMAs).
__device__ __forceinline__ uint64_t pack2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// Two consecutive staged samples as a packed FP32 pair (one 8-byte load for
// FP32, one 4-byte load converted for the 16-bit types).
template <typename T> __device__ __forceinline__ uint64_t load_pair(const T *p);
template <> __device__ __forceinline__ uint64_t load_pair<float>(const float *p)
{
    return *reinterpret_cast<const uint64_t *>(p);
}
template <> __device__ __forceinline__ uint64_t load_pair<__half>(const __half *p)
{
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(p));
    return pack2(f.x, f.y);
}
template <> __device__ __forceinline__ uint64_t load_pair<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    return pack2(f.x, f.y);
}
template <> __device__ __forceinline__ uint64_t load_pair<double>(const double *p)
{
    return 0ull; // unused: the FP64 path is not packed
}

// N consecutive 8-byte pairs from shared memory (16-byte loads when N is even).
template <int N> __device__ __forceinline__ void load_pairs(uint64_t (&w)[N], const uint64_t *p)
{
    if constexpr (N % 2 == 0) {
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const ulonglong2 v = reinterpret_cast<const ulonglong2 *>(p)[k];
            w[2 * k] = v.x;
            w[2 * k + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) w[k] = p[k];
    }
}

template <typename T, int C, int G, int V, bool TC = false>
__global__ void __launch_bounds__(kThreads, 3)
    fused_kernel(const __grid_constant__ CUtensorMap tmap, const Params p0, const Work w)
{
    using A = typename AccOf<T>::type;
    static_assert(!TC || sizeof(T) == 2, "the tensor-core path takes 16-bit storage");
    // FP32 accumulation uses packed-pair FMAs (the FP64 path stays scalar)
    constexpr bool kPacked = sizeof(A) == 4 && V % 2 == 0;
    constexpr int kVec = 16 / int(sizeof(T)); // elements per 16 bytes

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const bool batch = w.imgs != nullptr;
    const int nstage = (w.use_tma && w.stages == 2) ? 2 : 1;
    const Layout L =
        layout_of(w.tin_bytes, w.wy_bytes, w.wx_bytes, w.tt_bytes, w.rec2_bytes, nstage, TC ? w.tc_b_bytes : 0);
    unsigned char *after_stages = smem + nstage * L.stage;
    A *tt0 = reinterpret_cast<A *>(after_stages);
    unsigned char *rec_base = after_stages + 2 * L.tt;
    unsigned char *bmat = rec_base + 2 * L.rec2; // TC: weight matrices, hi then lo
    TileInfo *info = reinterpret_cast<TileInfo *>(bmat + L.bmat);
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(info) +
                                                  align_up(2 * sizeof(TileInfo), 128));
    uint64_t *full = bars, *ttfull = bars + 2, *ttempty = bars + 4, *mma_bar = bars + 6;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 7);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 7) + 1;
    // batch tile prefix sums cached in shared memory (up to kOffCache entries)
    int32_t *off_s = (batch && w.n_images + 1 <= kOffCache) ? reinterpret_cast<int32_t *>(bars + 8) : nullptr;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n1 = w.n1;        // staging + pass-1 warps
    const int n2 = kWarps - n1; // pass-2 warps
    int *err = p0.err;

    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&ttfull[0], 32 * n1);
        mbar_init(&ttfull[1], 32 * n1);
        mbar_init(&ttempty[0], 32 * n2);
        mbar_init(&ttempty[1], 32 * n2);
        mbar_init(mma_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (off_s)
        for (int e = threadIdx.x; e <= w.n_images; e += kThreads) off_s[e] = __ldg(w.tile_off + e);
    if constexpr (TC) {
        if (warp == 0) tc::tmem_alloc(tmem_slot, uint32_t(w.tc_cols));
        tc::fence_before_sync();
    }
    __syncthreads();
    if constexpr (TC) tc::fence_after_sync();

    auto stage_tin = [&](int s) { return reinterpret_cast<T *>(smem + s * L.stage); };
    auto stage_wy = [&](int s) { return reinterpret_cast<A *>(smem + s * L.stage + L.tin); };
    auto stage_wx = [&](int s) { return reinterpret_cast<A *>(smem + s * L.stage + L.tin + L.wy); };
    auto tt_buf = [&](int b) { return reinterpret_cast<A *>(reinterpret_cast<unsigned char *>(tt0) + b * L.tt); };
    auto rec2 = [&](int b) { return reinterpret_cast<Rec2 *>(rec_base + b * L.rec2); };
    auto rec2_w = [&](int b) { return reinterpret_cast<A *>(rec_base + b * L.rec2 + sizeof(Rec2)); };

    // The producer (warp 0) takes the k-th tile of this CTA: its image, the
    // image's parameters, the staged rectangle and the per-group offsets.
    // Returns false (and records img = -1) when the work is exhausted.
    auto take_tile = [&](int k, TileInfo *rec) -> bool {
        int item = -1, img = 0, t = 0;
        if (lane == 0) {
            const int total = batch ? w.total_tiles : p0.tiles_y * p0.tiles_x;
            const int it = int(blockIdx.x) + k * int(gridDim.x);
            if (it < total) {
                item = it;
                t = it;
                if (batch) {
                    // last image with tile_off[img] <= it (prefix sums in shared memory
                    // when they fit, else in global memory)
                    const int32_t *off = off_s ? off_s : w.tile_off;
                    int lo = 0, hi = w.n_images - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (off[mid] <= it) lo = mid; else hi = mid - 1;
                    }
                    img = lo;
                    t = it - off[lo];
                }
            }
        }
        item = __shfl_sync(0xffffffffu, item, 0);
        img = __shfl_sync(0xffffffffu, img, 0);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (item < 0) {
            if (lane == 0) rec->img = -1;
            __syncwarp();
            return false;
        }
        {   // copy the image's parameters into the record (word by word)
            const int32_t *src = reinterpret_cast<const int32_t *>(batch ? w.imgs + img : &p0);
            int32_t *dst = reinterpret_cast<int32_t *>(&rec->P);
            for (int e = lane; e < int(sizeof(Params) / 4); e += 32) dst[e] = src[e];
        }
        __syncwarp();
        const Params &P = rec->P;
        const int ngy = P.tile_h / G, ngx = P.tile_w / G;
        const int ty = t / P.tiles_x, tx = t % P.tiles_x;
        const int gy0 = ty * ngy, gx0 = tx * ngx;
        const bool vy = lane < ngy && gy0 + lane < P.groups_y;
        const bool vx = lane < ngx && gx0 + lane < P.groups_x;
        const int by = vy ? __ldg(P.base_y + gy0 + lane) : INT_MAX;
        const int bx = vx ? __ldg(P.base_x + gx0 + lane) : INT_MAX;
        int ylo = by, xlo = bx;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ylo = min(ylo, __shfl_xor_sync(0xffffffffu, ylo, o));
            xlo = min(xlo, __shfl_xor_sync(0xffffffffu, xlo, o));
        }
        const int s0 = xlo * C;
        const int xs = s0 - (s0 % kVec);
        if (vy) rec->rb[lane] = by - ylo;
        if (vx) rec->cb[lane] = bx * C - xs;
        if (lane == 0) {
            rec->img = img;
            rec->t = t;
            rec->ry0 = ylo;
            rec->xs = xs;
            rec->nvy = min(ngy, P.groups_y - gy0);
            rec->nvx = min(ngx, P.groups_x - gx0);
        }
        __syncwarp();
        return true;
    };

    // TMA producer (warp 0): take the k-th tile, lane 0 issues its copies into
    // stage s (or arrives without bytes at the end of the work).
    auto produce = [&](int k, int s) {
        const bool ok = take_tile(k, &info[s]);
        if (lane == 0) {
            if (!ok) {
                mbar_arrive(&full[s]);
                return;
            }
            const TileInfo &ti = info[s];
            const Params &P = ti.P;
            const int ngy = P.tile_h / G, ngx = P.tile_w / G;
            const int ty = ti.t / P.tiles_x, tx = ti.t % P.tiles_x;
            const uint32_t by = uint32_t(ti.nvy) * P.js_y * sizeof(A);
            const uint32_t bx = uint32_t(pair_slots(ti.nvx)) * P.js_x * sizeof(A);
            const uint32_t bt = uint32_t(P.n_sub) * P.sub_h * P.box_w * sizeof(T);
            mbar_arrive_expect_tx(&full[s], bt + by + bx);
            const CUtensorMap *map = batch ? w.maps + ti.img : &tmap;
            T *dst = stage_tin(s);
            if constexpr (TC) {
                tma_load_3d(dst, map, &full[s], 0, ti.ry0, ti.xs / 8);
            } else {
                for (int q = 0; q < P.n_sub; ++q)
                    tma_load_2d(dst + size_t(q) * P.sub_h * P.box_w, map, &full[s], ti.xs, ti.ry0 + q * P.sub_h);
            }
            bulk_load(stage_wy(s), static_cast<const A *>(P.band_y) + size_t(ty) * ngy * P.js_y, by, &full[s]);
            // warm L2 with the input of this CTA's tile kPrefetch further on
            // (single image: the tile's first groups carry its smallest bases)
            for (int a = (k == 0 ? 1 : kPrefetch); a <= kPrefetch && !batch; ++a) {
                const int tn = int(blockIdx.x) + (k + a) * int(gridDim.x);
                if (tn < P.tiles_y * P.tiles_x) {
                    const int nty = tn / P.tiles_x, ntx = tn % P.tiles_x;
                    const int ry = __ldg(P.base_y + nty * ngy);
                    const int s0 = __ldg(P.base_x + ntx * ngx) * C;
                    const int nxs = s0 - (s0 % kVec);
                    if constexpr (TC) {
                        tma_prefetch_3d(map, 0, ry, nxs / 8);
                    } else {
                        for (int q = 0; q < P.n_sub; ++q) tma_prefetch_2d(map, nxs, ry + q * P.sub_h);
                    }
                }
            }
            bulk_load(stage_wx(s), static_cast<const A *>(P.band_x) + size_t(tx) * pair_slots(ngx) * P.js_x, bx,
                      &full[s]);
        }
    };

    if (warp < n1) {
        // ======================= staging + pass 1 =======================
        const int t1n = 32 * n1;
        if (w.use_tma && warp == 0) {
            for (int k = 0; k < nstage; ++k) produce(k, k);
        }
        for (int i = 0;; ++i) {
            const int s = nstage == 2 ? (i & 1) : 0;
            const int b = i & 1;
            if (w.use_tma) {
                const uint32_t par = nstage == 2 ? uint32_t((i >> 1) & 1) : uint32_t(i & 1);
                if (!wait_or_abort(&full[s], par, abort_flag, err)) break;
            } else {
                if (warp == 0) take_tile(i, &info[0]);
                named_sync(1, t1n);
                const TileInfo &ti = info[0];
                if (ti.img >= 0) {
                    const Params &P = ti.P;
                    const T *in = static_cast<const T *>(P.in);
                    const int ngy = P.tile_h / G, ngx = P.tile_w / G;
                    const int ty = ti.t / P.tiles_x, tx = ti.t % P.tiles_x;
                    const int64_t row_len = P.in_w * C;
                    T *tin = stage_tin(0);
                    for (int r = warp; r < P.box_h; r += n1) {
                        const int64_t gy = int64_t(ti.ry0) + r;
                        T *dst = tin + size_t(r) * P.box_w;
                        for (int c = lane; c < P.box_w; c += 32) {
                            const int64_t gx = int64_t(ti.xs) + c;
                            T v = from_acc<T, A>(A(0));
                            if (gy < P.in_h && gx < row_len) v = in[gy * P.in_stride + gx];
                            dst[c] = v;
                        }
                    }
                    A *wy = stage_wy(0), *wx = stage_wx(0);
                    const A *sy = static_cast<const A *>(P.band_y) + size_t(ty) * ngy * P.js_y;
                    const A *sx = static_cast<const A *>(P.band_x) + size_t(tx) * pair_slots(ngx) * P.js_x;
                    for (int e = threadIdx.x; e < ti.nvy * P.js_y; e += t1n) wy[e] = __ldg(sy + e);
                    for (int e = threadIdx.x; e < pair_slots(ti.nvx) * P.js_x; e += t1n) wx[e] = __ldg(sx + e);
                }
                named_sync(1, t1n);
            }
            // the pass-2 warps must be done with buffer b (tile i - 2)
            if (i >= 2 && !wait_or_abort(&ttempty[b], uint32_t(((i >> 1) - 1) & 1), abort_flag, err)) break;
            const TileInfo &ti = info[s];
            Rec2 *r2 = rec2(b);
            if (ti.img < 0) {
                // end of the work: pass it on to the pass-2 warps and stop
                if (threadIdx.x == 0) r2->img = -1;
                mbar_arrive(&ttfull[b]);
                break;
            }
            const Params &P = ti.P;
            const int J = P.J;
            const int box_w = P.box_w, pitch_t = P.pitch_t;
            const T *tin = stage_tin(s);
            const A *wys = stage_wy(s);
            A *tt = tt_buf(b);

            if constexpr (TC) {
                // pass 1 on the tensor cores: D[sample][row] = sum_j In[j][sample] W[row][j]
                // A = staged input (MN-major canonical layout from the 3-D TMA box),
                // B = the tile's weight matrix (K-major), split into hi + lo 16-bit
                // parts so that weight rounding costs no accuracy; FP32 in tensor memory.
                const int N = P.tile_h, K = P.tc_kpad, nmb = P.tc_nmb;
                const uint32_t sbo = uint32_t(K) * 16u; // 8-sample (A) or 8-row (B) group stride
                const size_t bbytes = size_t(N) * K * 2;
                unsigned char *bhi = bmat, *blo = bmat + bbytes;
                if (threadIdx.x < ti.nvy && (ti.rb[threadIdx.x] < 0 || ti.rb[threadIdx.x] + J > K))
                    flag(err, kErrBounds); // a band past the staged rows would lose weights
                for (int e = threadIdx.x; e < N * K; e += t1n) {
                    const int y = e / K, j = e - y * K;
                    const int q = y / G, r = y - q * G;
                    float wv = 0.f;
                    if (q < ti.nvy) {
                        const int jj = j - ti.rb[q];
                        if (jj >= 0 && jj < J) wv = float(wys[q * P.js_y + jj * G + r]);
                    }
                    const T hi = from_acc<T, A>(wv);
                    const T lo = from_acc<T, A>(wv - to_acc<A, T>(hi));
                    const uint32_t off = uint32_t(y / 8) * sbo + uint32_t(j / 8) * 128u + uint32_t(y % 8) * 16u +
                                         uint32_t(j % 8) * 2u;
                    *reinterpret_cast<T *>(bhi + off) = hi;
                    *reinterpret_cast<T *>(blo + off) = lo;
                }
                tc::fence_proxy_async();
                named_sync(1, t1n);
                const uint32_t tmem = *tmem_slot;
                if (threadIdx.x == 0) {
                    tc::fence_after_sync();
                    const uint32_t idesc = tc::idesc_f16(sizeof(T) == 2 && !std::is_same<T, __half>::value,
                                                         true, false, 128, N);
                    const uint32_t abase = smem_addr(tin), bh = smem_addr(bhi), bl = smem_addr(blo);
                    for (int mb = 0; mb < nmb; ++mb) {
                        for (int kb = 0; kb < K / 16; ++kb) {
                            const uint64_t ad =
                                tc::smem_desc(abase + uint32_t(mb) * 16u * sbo + uint32_t(kb) * 256u, 128u, sbo);
                            const uint32_t d = tmem + uint32_t(mb * N);
                            tc::mma_f16(d, ad, tc::smem_desc(bh + uint32_t(kb) * 256u, 128u, sbo), idesc,
                                        kb > 0 ? 1u : 0u);
                            tc::mma_f16(d, ad, tc::smem_desc(bl + uint32_t(kb) * 256u, 128u, sbo), idesc, 1u);
                        }
                    }
                    tc::mma_commit(mma_bar);
                }
                if (!wait_or_abort(mma_bar, uint32_t(i & 1), abort_flag, err)) break;
                tc::fence_after_sync();
                // accumulators -> intermediate rows: warp wq reads lanes 32 wq .. 32 wq + 31
                for (int mb = 0; mb < nmb; ++mb) {
                    for (int c0 = 0; c0 < N; c0 += 16) {
                        uint32_t r16[16];
                        tc::tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(mb * N + c0), r16);
                        tc::tmem_ld_wait();
                        A *dst = tt + mb * 128 + warp * 32 + lane;
#pragma unroll
                        for (int k = 0; k < 16; ++k) dst[(c0 + k) * pitch_t] = A(__uint_as_float(r16[k]));
                    }
                }
                tc::fence_before_sync();
            } else {
            // pass 1: lanes along samples; V columns 32 apart per lane.  Chunks
                // past box_w read harmless staged data and land in the padding of
                // the intermediate (pitch_t >= w1): no predicate in the inner loop.
                const int nchunk = P.w1 / (32 * V);
                const int ntask = ti.nvy * nchunk;
                const int per = (ntask + n1 - 1) / n1;
                const int k0 = warp * per, k1 = min(ntask, k0 + per);
                for (int task = k0; task < k1; ++task) {
                    const int q = task / nchunk, k = task - q * nchunk;
                    const int rb = ti.rb[q];
                    if (rb < 0 || rb + J > P.box_h) {
                        if (lane == 0) flag(err, kErrBounds);
                        continue;
                    }
                    if constexpr (kPacked) {
                        // lane owns the column pairs (2 lane, 2 lane + 1) + 64 u: one
                        // 8-byte (FP32) or 4-byte (16-bit) load gives a pair ready
                        // for the packed FMA; the vertical band holds every
                        // weight twice, so weight pairs load as they are
                        const int c0 = k * 32 * V + 2 * lane;
                        const T *col = tin + rb * box_w + c0;
                        A *dst = tt + q * G * pitch_t + c0;
                        uint64_t acc2[G][V / 2];
    #pragma unroll
                        for (int g = 0; g < G; ++g)
    #pragma unroll
                            for (int u = 0; u < V / 2; ++u) acc2[g][u] = 0ull;
                        const uint64_t *wq = reinterpret_cast<const uint64_t *>(wys + q * P.js_y);
    #pragma unroll 4
                        for (int j = 0; j < J; ++j) {
                            uint64_t w2[G];
                            load_pairs<G>(w2, wq);
                            wq += G;
                            uint64_t dd[V / 2];
    #pragma unroll
                            for (int u = 0; u < V / 2; ++u) dd[u] = load_pair<T>(col + 64 * u);
    #pragma unroll
                            for (int u = 0; u < V / 2; ++u)
    #pragma unroll
                                for (int g = 0; g < G; ++g) acc2[g][u] = fma2(w2[g], dd[u], acc2[g][u]);
                            col += box_w;
                        }
    #pragma unroll
                        for (int g = 0; g < G; ++g)
    #pragma unroll
                            for (int u = 0; u < V / 2; ++u) {
                                float lo, hi;
                                unpack2(acc2[g][u], lo, hi);
                                dst[g * pitch_t + 64 * u] = lo;
                                dst[g * pitch_t + 64 * u + 1] = hi;
                            }
                    } else {
                        const int c0 = k * 32 * V + lane;
                        const T *col = tin + rb * box_w + c0;
                        A *dst = tt + q * G * pitch_t + c0;
                        A acc[G][V];
    #pragma unroll
                        for (int g = 0; g < G; ++g)
    #pragma unroll
                            for (int v = 0; v < V; ++v) acc[g][v] = A(0);
                        const A *wq = wys + q * P.js_y;
    #pragma unroll 4
                        for (int j = 0; j < J; ++j) {
                            A wv[G];
                            load_w<A, G>(wv, wq);
                            wq += G;
    #pragma unroll
                            for (int v = 0; v < V; ++v) {
                                const A dv = to_acc<A, T>(col[32 * v]);
    #pragma unroll
                                for (int g = 0; g < G; ++g) acc[g][v] = fma(wv[g], dv, acc[g][v]);
                            }
                            col += box_w;
                        }
    #pragma unroll
                        for (int g = 0; g < G; ++g)
    #pragma unroll
                            for (int v = 0; v < V; ++v) dst[g * pitch_t + 32 * v] = acc[g][v];
                    }
                }
            }
            // hand the pass-2 record (parameters, offsets and x weights) over with buffer b
            {
                const int32_t *src = reinterpret_cast<const int32_t *>(&ti.P);
                int32_t *dstp = reinterpret_cast<int32_t *>(&r2->P);
                for (int e = threadIdx.x; e < int(sizeof(Params) / 4); e += t1n) dstp[e] = src[e];
            }
            if (threadIdx.x < 32) {
                if (lane < P.tile_w / G) r2->cb[lane] = ti.cb[lane];
                if (lane == 0) {
                    r2->img = ti.img;
                    r2->ty = ti.t / P.tiles_x;
                    r2->tx = ti.t % P.tiles_x;
                    r2->nvx = ti.nvx;
                }
            }
            {
                const A *src = stage_wx(s);
                A *dstw = rec2_w(b);
                for (int e = threadIdx.x; e < pair_slots(ti.nvx) * P.js_x; e += t1n) dstw[e] = src[e];
            }
            mbar_arrive(&ttfull[b]);
            // every pass-1 warp is done with stage s before it is refilled
            named_sync(1, t1n);
            if (w.use_tma && warp == 0) produce(i + nstage, s);
        }
        if constexpr (TC) {
            // every pass-1 warp is done with the tensor memory before it is freed
            tc::fence_before_sync();
            named_sync(1, t1n);
            if (warp == 0) {
                tc::fence_after_sync();
                tc::tmem_dealloc(*tmem_slot, uint32_t(w.tc_cols));
            }
        }
    } else {
        // =========================== pass 2 ============================
        const int w2 = warp - n1;
        for (int i = 0;; ++i) {
            const int b = i & 1;
            if (!wait_or_abort(&ttfull[b], uint32_t((i >> 1) & 1), abort_flag, err)) break;
            const Rec2 *r2 = rec2(b);
            if (r2->img < 0) break;
            const Params &P = r2->P;
            const A *tt = tt_buf(b);
            const A *wxs = rec2_w(b);
            const int J = P.J;
            const int pitch_t = P.pitch_t, js_x = P.js_x, box_w = P.box_w, tile_h = P.tile_h;
            const int ngx = P.tile_w / G;
            const int ty = r2->ty, tx = r2->tx, nvx = r2->nvx;
            const int64_t out_h = P.out_h, out_w = P.out_w, out_stride = P.out_stride;
            T *out = static_cast<T *>(P.out);
            // Lanes run along output rows; each lane takes the pair of groups
            // (2 pq, 2 pq + 1) of its row, whose weights the band interleaves,
            // so one packed FMA advances both groups.
            const int RB = tile_h < 32 ? tile_h : 32; // rows per warp task
            const int GPW = 32 / RB;                  // group pairs per warp task
            const int rsub = lane % RB, gsub = lane / RB;
            const int nrb = (tile_h + RB - 1) / RB;
            const int npairs = pair_slots(nvx);
            const int npg = (npairs + GPW - 1) / GPW;
            const int ntask = nrb * npg;
            const int per = (ntask + n2 - 1) / n2;
            const int k0 = w2 * per, k1 = min(ntask, k0 + per);
            for (int task = k0; task < k1; ++task) {
                const int rbk = task / npg, pg = task - rbk * npg;
                const int pq = pg * GPW + gsub;
                const int row = rbk * RB + rsub;
                const int64_t yo = int64_t(ty) * tile_h + row;
                if (pq >= npairs || row >= tile_h || yo >= out_h) continue;
                const int q0 = 2 * pq;
                const bool has1 = q0 + 1 < nvx;
                const int cb0 = r2->cb[q0];
                const int cb1 = has1 ? r2->cb[q0 + 1] : cb0;
                if (cb0 < 0 || cb0 + J * C > box_w || cb1 < 0 || cb1 + J * C > box_w) {
                    flag(err, kErrBounds);
                    continue;
                }
                A acc[2][G][C];
                const A *rp0 = tt + row * pitch_t + cb0;
                const A *rp1 = tt + row * pitch_t + cb1;
                if constexpr (sizeof(A) == 4) {
                    uint64_t acc2[G][C];
#pragma unroll
                    for (int g = 0; g < G; ++g)
#pragma unroll
                        for (int c = 0; c < C; ++c) acc2[g][c] = 0ull;
                    const uint64_t *wq2 = reinterpret_cast<const uint64_t *>(wxs + pq * js_x);
#pragma unroll 4
                    for (int j = 0; j < J; ++j) {
                        uint64_t wp[G];
                        load_pairs<G>(wp, wq2);
                        wq2 += G;
#pragma unroll
                        for (int c = 0; c < C; ++c) {
                            const uint64_t dd = pack2(rp0[c], rp1[c]);
#pragma unroll
                            for (int g = 0; g < G; ++g) acc2[g][c] = fma2(wp[g], dd, acc2[g][c]);
                        }
                        rp0 += C;
                        rp1 += C;
                    }
#pragma unroll
                    for (int g = 0; g < G; ++g)
#pragma unroll
                        for (int c = 0; c < C; ++c) {
                            float lo, hi;
                            unpack2(acc2[g][c], lo, hi);
                            acc[0][g][c] = lo;
                            acc[1][g][c] = hi;
                        }
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h)
#pragma unroll
                        for (int g = 0; g < G; ++g)
#pragma unroll
                            for (int c = 0; c < C; ++c) acc[h][g][c] = A(0);
                    const A *wq = wxs + pq * js_x;
#pragma unroll 2
                    for (int j = 0; j < J; ++j) {
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            const A w0 = wq[2 * g], w1 = wq[2 * g + 1];
#pragma unroll
                            for (int c = 0; c < C; ++c) {
                                acc[0][g][c] = fma(w0, rp0[c], acc[0][g][c]);
                                acc[1][g][c] = fma(w1, rp1[c], acc[1][g][c]);
                            }
                        }
                        wq += 2 * G;
                        rp0 += C;
                        rp1 += C;
                    }
                }
                // Store G*C contiguous samples of each group's row (clipped at the right edge).
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h == 1 && !has1) break;
                    const int64_t x0 = (int64_t(tx) * ngx + q0 + h) * G;
                    T *o = out + yo * out_stride + x0 * C;
                    const int nvalid = out_w - x0 < G ? int(out_w - x0) : G;
                    constexpr int kRun = G * C;
                    constexpr int kRunBytes = kRun * int(sizeof(T));
                    if (nvalid == G && (kRunBytes % 16) == 0 && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
                        union {
                            T e[kRun];
                            uint4 v[kRunBytes / 16 > 0 ? kRunBytes / 16 : 1];
                        } u;
#pragma unroll
                        for (int g = 0; g < G; ++g)
#pragma unroll
                            for (int c = 0; c < C; ++c) u.e[g * C + c] = from_acc<T, A>(acc[h][g][c]);
                        uint4 *ov = reinterpret_cast<uint4 *>(o);
#pragma unroll
                        for (int v = 0; v < kRunBytes / 16; ++v) ov[v] = u.v[v];
                    } else {
#pragma unroll
                        for (int g = 0; g < G; ++g)
                            if (g < nvalid)
#pragma unroll
                                for (int c = 0; c < C; ++c) o[g * C + c] = from_acc<T, A>(acc[h][g][c]);
                    }
                }
            }
            mbar_arrive(&ttempty[b]);
        }
    }
    // On an abort some TMA copies may still be in flight; let them land
    // (bounded) before the CTA's shared memory is released.
    if (*abort_flag && w.use_tma && warp == 0) {
        mbar_wait_bounded(&full[0], 0u);
        mbar_wait_bounded(&full[1], 0u);
    }
}

// One instantiated kernel variant: the SIMT kernel and, for 16-bit storage,
// the kernel whose vertical pass runs on the tensor cores (else the SIMT one again).
struct Variant {
    int dtype, C, G, V;
    const void *fn;
    const void *fn_tc;
};

#define RS_FUSED_VARIANT(T, DT, C, G, V) \
    { DT, C, G, V, reinterpret_cast<const void *>(&fused_kernel<T, C, G, V>), \
      reinterpret_cast<const void *>(&fused_kernel<T, C, G, V, false>) }
#define RS_FUSED_VARIANT_TC(T, DT, C, G, V) \
    { DT, C, G, V, reinterpret_cast<const void *>(&fused_kernel<T, C, G, V>), \
      reinterpret_cast<const void *>(&fused_kernel<T, C, G, V, true>) }

} // namespace fused
} // namespace rs
