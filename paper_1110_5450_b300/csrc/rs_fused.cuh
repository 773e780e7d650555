// rs_fused.cuh -- fused separable resampling kernel (one launch per image).
//
// A persistent CTA walks output tiles of tile_h x tile_w pixels.  For each
// tile it stages the input rectangle the tile's taps touch in shared memory
// (TMA 2-D tile copy, double-buffered behind an mbarrier, or plain coalesced
// loads when the image's row pitch is not 16-byte aligned), then
//
//   pass 1 (vertical):   tt[yo][s]  = sum_j Wy[yo][j] tin[by(yo) + j][s]
//   pass 2 (horizontal): out[yo][x][c] = sum_j Wx[x][j] tt[yo][(bx(x) + j) C + c]
//
// Weights come from "register bands": outputs are grouped G at a time along an
// axis; a group reads the J consecutive inputs [base, base + J) and holds its
// G x J weights (zeros outside each output's own taps) in registers, so one
// shared-memory load feeds G fused multiply-adds.
//
// Shared-memory layout choices (bank conflicts):
//   pass 1: lanes take consecutive samples of a row -> conflict-free for any
//           pitch, so the TMA's dense box layout is read as it lands;
//   pass 2: lanes take consecutive output ROWS of one group, so that every
//           lane uses the same weights; the intermediate's pitch is odd (in
//           words of the accumulation type) so the 32 rows hit 32 banks.
#pragma once

#include <cuda.h>
#include <climits>

#include "rs_internal.h"

namespace rs {
namespace fused {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kErrBounds = 201;   // a band would read outside the staged tile
constexpr int kErrTimeout = 202;  // an mbarrier wait ran out

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

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
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
        if ((it & 255u) == 255u && global_ns() - t0 > 2000000000ull) return false;
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
    const void *band_y, *band_x;
    int32_t tile_h, tile_w;   // output tile
    int32_t box_h, box_w;     // staged rows, staged samples (pitch of tin)
    int32_t sub_h, n_sub;     // TMA box height and copies per tile
    int32_t pitch_t;          // pitch of the intermediate (odd, accumulation words)
    int32_t tiles_y, tiles_x;
    int32_t groups_y, groups_x;
    int use_tma;              // 1: TMA tile copies; 0: plain coalesced loads
    int stages;               // staged input buffers (2 = prefetch next tile; TMA only)
    int *err;
};

struct TileInfo {
    int32_t ry0;  // first staged input row
    int32_t xs;   // first staged input sample (aligned)
    int32_t rows; // rows actually needed
    int32_t cols; // samples actually needed (from xs)
};

// Compute the staged rectangle of tile t (called by one full warp).
template <int C, int GY, int JY, int GX, int JX>
__device__ __forceinline__ TileInfo tile_rect(const Params &p, int t, int vec)
{
    const int ty = t / p.tiles_x, tx = t % p.tiles_x;
    const int lane = threadIdx.x & 31;
    const int gy0 = ty * (p.tile_h / GY), ngy = p.tile_h / GY;
    const int gx0 = tx * (p.tile_w / GX), ngx = p.tile_w / GX;
    int ylo = INT_MAX, yhi = INT_MIN, xlo = INT_MAX, xhi = INT_MIN;
    if (lane < ngy && gy0 + lane < p.groups_y) {
        const int b = __ldg(p.base_y + gy0 + lane);
        ylo = b;
        yhi = b;
    }
    if (lane < ngx && gx0 + lane < p.groups_x) {
        const int b = __ldg(p.base_x + gx0 + lane);
        xlo = b;
        xhi = b;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ylo = min(ylo, __shfl_xor_sync(0xffffffffu, ylo, o));
        yhi = max(yhi, __shfl_xor_sync(0xffffffffu, yhi, o));
        xlo = min(xlo, __shfl_xor_sync(0xffffffffu, xlo, o));
        xhi = max(xhi, __shfl_xor_sync(0xffffffffu, xhi, o));
    }
    TileInfo ti;
    ti.ry0 = ylo;
    ti.rows = yhi + JY - ylo;
    const int s0 = xlo * C;
    ti.xs = s0 - (s0 % vec);
    ti.cols = (xhi + JX) * C - ti.xs;
    return ti;
}

template <typename T, int C, int GY, int JY, int GX, int JX>
__global__ void __launch_bounds__(kThreads) fused_kernel(const __grid_constant__ CUtensorMap tmap, const Params p)
{
    using A = typename AccOf<T>::type;
    constexpr int kVec = 16 / int(sizeof(T)); // elements per 16 bytes

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const size_t tin_bytes = (size_t(p.box_h) * p.box_w * sizeof(T) + 127) & ~size_t(127);
    const int nstage = (p.use_tma && p.stages == 2) ? 2 : 1;
    T *tin0 = reinterpret_cast<T *>(smem);
    T *tin1 = reinterpret_cast<T *>(smem + (nstage - 1) * tin_bytes);
    A *tt = reinterpret_cast<A *>(smem + nstage * tin_bytes);
    const size_t tt_bytes = (size_t(p.tile_h) * p.pitch_t * sizeof(A) + 127) & ~size_t(127);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + nstage * tin_bytes + tt_bytes);
    TileInfo *info = reinterpret_cast<TileInfo *>(bars + 2);
    int *abort_flag = reinterpret_cast<int *>(info + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = p.tiles_y * p.tiles_x;
    const T *in = static_cast<const T *>(p.in);
    T *out = static_cast<T *>(p.out);
    const A *band_y = static_cast<const A *>(p.band_y);
    const A *band_x = static_cast<const A *>(p.band_x);

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const uint32_t copy_bytes = uint32_t(p.n_sub) * p.sub_h * p.box_w * sizeof(T);

    // Producer step: warp 0 computes the rectangle and (TMA) lane 0 issues the copies.
    auto produce = [&](int t, int stage) {
        TileInfo ti = tile_rect<C, GY, JY, GX, JX>(p, t, kVec);
        if (lane == 0) {
            info[stage] = ti;
            if (p.use_tma) {
                T *dst = stage ? tin1 : tin0;
                mbar_arrive_expect_tx(&bars[stage], copy_bytes);
                for (int k = 0; k < p.n_sub; ++k)
                    tma_load_2d(dst + size_t(k) * p.sub_h * p.box_w, &tmap, &bars[stage], ti.xs,
                                ti.ry0 + k * p.sub_h);
            }
        }
    };

    int it = 0;
    if (p.use_tma && nstage == 2 && warp == 0 && int(blockIdx.x) < total) produce(blockIdx.x, 0);

    for (int t = blockIdx.x; t < total; t += gridDim.x, ++it) {
        const int stage = nstage == 2 ? (it & 1) : 0;
        // use count of this stage's barrier so far -> phase parity to wait for
        const uint32_t parity = nstage == 2 ? uint32_t((it >> 1) & 1) : uint32_t(it & 1);
        T *tin = stage ? tin1 : tin0;
        if (p.use_tma) {
            const int tn = t + gridDim.x;
            if (warp == 0) {
                if (nstage == 2) {
                    if (tn < total) produce(tn, stage ^ 1);
                } else {
                    produce(t, 0);
                }
            }
            if (!mbar_wait_bounded(&bars[stage], parity)) {
                flag(p.err, kErrTimeout);
                atomicExch(abort_flag, 1);
            }
            __syncthreads();
            if (*abort_flag) {
                // Let any copy still in flight land before the CTA exits.
                mbar_wait_bounded(&bars[0], 0u);
                mbar_wait_bounded(&bars[1], 0u);
                return;
            }
        } else {
            if (warp == 0) produce(t, 0);
            __syncthreads();
            const TileInfo ti = info[0];
            // Plain staging: coalesced loads, zero outside the image.
            const int64_t row_len = p.in_w * C;
            for (int r = warp; r < p.box_h; r += kWarps) {
                const int64_t gy = int64_t(ti.ry0) + r;
                T *dst = tin + size_t(r) * p.box_w;
                for (int s = lane; s < p.box_w; s += 32) {
                    const int64_t gx = int64_t(ti.xs) + s;
                    T v = from_acc<T, A>(A(0));
                    if (gy < p.in_h && gx < row_len) v = in[gy * p.in_stride + gx];
                    dst[s] = v;
                }
            }
            __syncthreads();
        }
        const TileInfo ti = info[stage];
        const int ty = t / p.tiles_x, tx = t % p.tiles_x;

        // ---------------- pass 1: vertical, lanes along samples ----------------
        {
            const int ngy = p.tile_h / GY;
            const int nchunk = (ti.cols + 31) >> 5;
            const int ntask = ngy * nchunk;
            const int per = (ntask + kWarps - 1) / kWarps;
            const int t0 = warp * per, t1 = min(ntask, t0 + per);
            int cur_q = -1;
            A w[GY][JY];
            int rb = 0;
            bool ok = true;
            for (int task = t0; task < t1; ++task) {
                const int q = task / nchunk, k = task % nchunk;
                const int gy = ty * ngy + q;
                if (gy >= p.groups_y) continue;
                if (q != cur_q) {
                    cur_q = q;
                    const A *src = band_y + size_t(gy) * GY * JY;
#pragma unroll
                    for (int r = 0; r < GY; ++r)
#pragma unroll
                        for (int j = 0; j < JY; ++j) w[r][j] = __ldg(src + r * JY + j);
                    rb = __ldg(p.base_y + gy) - ti.ry0;
                    ok = rb >= 0 && rb + JY <= p.box_h;
                    if (!ok && lane == 0) flag(p.err, kErrBounds);
                }
                if (!ok) continue;
                const int s = k * 32 + lane;
                if (s >= p.box_w) continue;
                A acc[GY];
#pragma unroll
                for (int r = 0; r < GY; ++r) acc[r] = A(0);
                const T *col = tin + size_t(rb) * p.box_w + s;
#pragma unroll
                for (int j = 0; j < JY; ++j) {
                    const A v = to_acc<A, T>(col[size_t(j) * p.box_w]);
#pragma unroll
                    for (int r = 0; r < GY; ++r) acc[r] = fma(w[r][j], v, acc[r]);
                }
                A *dst = tt + size_t(q * GY) * p.pitch_t + s;
#pragma unroll
                for (int r = 0; r < GY; ++r) dst[size_t(r) * p.pitch_t] = acc[r];
            }
        }
        __syncthreads();

        // ---------------- pass 2: horizontal, lanes along output rows ----------------
        {
            const int ngx = p.tile_w / GX;
            const int yo = ty * p.tile_h + lane;
            const bool row_ok = lane < p.tile_h && yo < p.out_h;
            for (int q = warp; q < ngx; q += kWarps) {
                const int gx = tx * ngx + q;
                if (gx >= p.groups_x) break;
                A w[GX][JX];
                const A *src = band_x + size_t(gx) * GX * JX;
#pragma unroll
                for (int g = 0; g < GX; ++g)
#pragma unroll
                    for (int j = 0; j < JX; ++j) w[g][j] = __ldg(src + g * JX + j);
                const int cb = __ldg(p.base_x + gx) * C - ti.xs;
                if (cb < 0 || cb + JX * C > p.box_w) {
                    if (lane == 0) flag(p.err, kErrBounds);
                    continue;
                }
                if (!row_ok) continue;
                A acc[GX][C];
#pragma unroll
                for (int g = 0; g < GX; ++g)
#pragma unroll
                    for (int c = 0; c < C; ++c) acc[g][c] = A(0);
                const A *row = tt + size_t(lane) * p.pitch_t + cb;
#pragma unroll
                for (int j = 0; j < JX; ++j) {
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const A v = row[j * C + c];
#pragma unroll
                        for (int g = 0; g < GX; ++g) acc[g][c] = fma(w[g][j], v, acc[g][c]);
                    }
                }
                // Store GX*C contiguous samples of this row (clipped at the right edge).
                const int64_t x0 = int64_t(gx) * GX;
                T *o = out + int64_t(yo) * p.out_stride + x0 * C;
                const int nvalid = p.out_w - x0 < GX ? int(p.out_w - x0) : GX;
                constexpr int kRun = GX * C;
                constexpr int kRunBytes = kRun * int(sizeof(T));
                if (nvalid == GX && (kRunBytes % 16) == 0 && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
                    union {
                        T e[kRun];
                        uint4 v[kRunBytes / 16 > 0 ? kRunBytes / 16 : 1];
                    } u;
#pragma unroll
                    for (int g = 0; g < GX; ++g)
#pragma unroll
                        for (int c = 0; c < C; ++c) u.e[g * C + c] = from_acc<T, A>(acc[g][c]);
                    uint4 *ov = reinterpret_cast<uint4 *>(o);
#pragma unroll
                    for (int v = 0; v < kRunBytes / 16; ++v) ov[v] = u.v[v];
                } else {
#pragma unroll
                    for (int g = 0; g < GX; ++g)
                        if (g < nvalid)
#pragma unroll
                            for (int c = 0; c < C; ++c) o[g * C + c] = from_acc<T, A>(acc[g][c]);
                }
            }
        }
        __syncthreads();
    }
}

// Dynamic shared memory the kernel needs for a parameter set.
inline size_t smem_bytes(size_t elem, size_t acc, int box_h, int box_w, int tile_h, int pitch_t, int nstage)
{
    const size_t tin = (size_t(box_h) * box_w * elem + 127) & ~size_t(127);
    const size_t tt = (size_t(tile_h) * pitch_t * acc + 127) & ~size_t(127);
    return 128 + size_t(nstage) * tin + tt + 2 * sizeof(uint64_t) + 2 * sizeof(TileInfo) + 16;
}

// One instantiated kernel variant.
struct Variant {
    int dtype, C, G, J;
    const void *fn;
};

#define RS_FUSED_VARIANT(T, DT, C, G, J) \
    { DT, C, G, J, reinterpret_cast<const void *>(&fused_kernel<T, C, G, J, G, J>) }

} // namespace fused
} // namespace rs
