// rs_xstream.cuh -- pipelined row-streaming kernel for upscales (streaming
// form 2).
//
// Same data flow as the band streaming kernels (rs_stream.cuh): a CTA owns a
// strip of SW output columns and a range of output rows, walks down the input
// in blocks of 32 rows staged by TMA, runs the horizontal pass on every staged
// row into a ring of filtered rows (FP32) and the vertical pass on that ring.
// What differs:
//
//  * Tight bands from the exact windows.  Outputs go in groups of 4 (4 output
//    columns across, 4 output rows down).  On an upscaled axis the folded
//    window start of output i + 1 is that of output i or one more, so the 4
//    windows of a group lie in the T + 3 inputs from the first window's start
//    (a pattern of three 0/1 steps says where each one sits).  Each pass
//    applies a band of T + 3 weights per output, zero outside the output's own
//    window: 9 instead of the 12 of a 4-pixel aligned band for Lanczos-3 across,
//    and 9 taps per row instead of 12 for groups of 8 rows down.  The bands are
//    built on chip from the plan's window-weight tables: the horizontal band of
//    the strip once per CTA, the vertical bands of each staged block by the
//    producer warp while the other warps filter (no band tables in HBM, no band
//    kernel launch per step).  One code path per pass: a path per step pattern
//    (exact windows, no zero weights) was measured 1.5-2.5x slower, because the
//    live variants overflow the instruction cache.
//  * Warp roles and mbarriers only.  Warp 0 (the producer) issues the TMA
//    copies (input blocks; the window weights and group descriptors of the
//    groups each block completes) and builds the vertical bands; HW warps run
//    the horizontal pass and VW warps the vertical pass.  Blocks are handed
//    over through mbarriers (no CTA-wide barrier after set-up), and each role
//    takes its tasks round-robin over a task stream that runs on across blocks,
//    so uneven task counts per block even out instead of idling warps at a
//    barrier.
//
// Summation order per output: its taps in increasing input order, FP32 FMAs
// (the band's zero weights add exact zeros).  The filtered-row ring holds two
// blocks plus a band, so the horizontal warps fill block k + 1 while the
// vertical warps read the groups block k completes.  Every wait is bounded
// (2 s); a timeout sets the plan's error word and stops the CTA, whose
// producer lets the copies still in flight land before the CTA exits.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_stream.cuh"

namespace rs {
namespace xstream {

constexpr int kMaxWarps = 16;   // producer + horizontal + vertical warps of a CTA, at most
constexpr int kSmallWarps = 12; // at most this many: the kernel variant for 2 CTAs per SM
constexpr int kMidWarps = 10;   // multi-image variant for 2 CTAs per SM of at most this many warps
constexpr int kRB = 32;   // input rows per staged block (one per lane of a horizontal task)
constexpr int kG = 4;     // outputs per group (columns across, rows down)
constexpr int kMaxNI = 4; // staged input blocks at most
constexpr int kNW = 2;    // vertical weight slots

struct Params {
    const void *in; // the image in its storage type (FP32, FP16 or BF16)
    void *out;
    int64_t in_h, in_w, out_h, out_w;
    int64_t in_stride, out_stride;
    // per column group: first pixel of its 4-pixel aligned chunk run | pattern << 24
    // (pattern: offset of the first window in the run, bits 0-1; steps of the
    // next three windows, bits 2-4)
    const int32_t *hinfo;
    const float *wx; // [>= 4 groups_x][T] the columns' window weights (the plan's table)
    // per row group: first input row of its first window | pattern << 24 (steps, bits 0-2);
    // allocated for groups_y rounded up to 4, plus 4
    const int32_t *vinfo;
    const float *wy; // [>= 4 groups_y][T] the rows' window weights
    int32_t SW;      // output pixels per strip (multiple of 4)
    int32_t n_strips, groups_x, groups_y;
    int32_t gpr;     // row groups per CTA row range
    int32_t P;       // staged input pitch in samples
    int32_t offB;    // second staged box offset (0: one box per block)
    int32_t JH;      // widest chunk run a column group reads, in pixels (multiple of 4)
    int32_t Q;       // ring rows per 4-sample column (>= HR + M, odd)
    int32_t HR, M;   // ring rows, mirrored rows
    int32_t JV;      // rows a vertical band spans (T + 3)
    int32_t NI;      // staged input blocks
    int32_t WP;      // most row groups that one block completes
    int32_t nblk;    // most blocks of a row range (shared-memory table size)
    int32_t HW, VW;  // horizontal / vertical warps (the CTA has 1 + HW + VW warps)
    int32_t pf;      // 1: prefetch the block after the ring into L2
    int *err;
};

// Shared memory: NI input blocks | weight staging (the window weights and
// group descriptors of one block, as copied) | kNW band slots (the vertical
// bands built from them and each group's first window row) | ring of filtered
// rows | the strip's horizontal band | column group offsets | per-block group
// ends | barriers.
struct Layout {
    size_t in_blk, in_ring, wv, vi, stg, vb, bslot, b_ring, hring, hw, hc, pe, bar, total;
};

__host__ __device__ inline Layout layout(int NI, int P, int Q, int nch, int ngx, int T, int WP, int nblk,
                                         bool two_boxes, int es)
{
    const int HB = T + 3;
    Layout L;
    L.in_blk = fused::align_up(size_t(kRB) * P * es * (two_boxes ? 2 : 1), 128);
    L.in_ring = size_t(NI) * L.in_blk;
    L.wv = size_t(WP) * kG * T * 4;
    L.vi = fused::align_up(size_t(WP + 8) * 4, 16);
    L.stg = fused::align_up(L.wv + L.vi, 128);
    L.vb = size_t(WP) * kG * HB * 4;
    L.bslot = fused::align_up(L.vb + size_t(WP) * 4, 128);
    L.b_ring = size_t(kNW) * L.bslot;
    L.hring = fused::align_up(size_t(nch) * Q * 16, 128);
    L.hw = fused::align_up(size_t(ngx) * kG * HB * 4, 128);
    L.hc = fused::align_up(size_t(ngx) * 4, 128);
    L.pe = fused::align_up(size_t(nblk) * 4, 128);
    L.bar = 256; // 2 kMaxNI + 3 + 2 kNW + 4 mbarriers and the abort flag
    L.total = 128 + L.in_ring + L.stg + L.b_ring + L.hring + L.hw + L.hc + L.pe + L.bar;
    return L;
}

// Window offsets of a group's members (from the first window) by pattern.
__host__ __device__ constexpr int h_off(int pat, int g)
{
    return (g > 0 ? (pat >> 2) & 1 : 0) + (g > 1 ? (pat >> 3) & 1 : 0) + (g > 2 ? (pat >> 4) & 1 : 0);
}
__host__ __device__ constexpr int v_off(int pat, int r)
{
    return (r > 0 ? pat & 1 : 0) + (r > 1 ? (pat >> 1) & 1 : 0) + (r > 2 ? (pat >> 2) & 1 : 0);
}

// One 4-pixel chunk (4 C samples) of the lane's staged row as floats.
template <typename T, int C> __device__ __forceinline__ void load_chunk(const T *p, float (&d)[4 * C])
{
#pragma unroll
    for (int v = 0; v < C; ++v) {
        const float4 x = stream::load4<T>(p + 4 * v);
        d[4 * v] = x.x;
        d[4 * v + 1] = x.y;
        d[4 * v + 2] = x.z;
        d[4 * v + 3] = x.w;
    }
}

// Horizontal pass of one column group for the lane's staged row: win = the 3
// chunks of the group's run (its first window starts O0 pixels in), w4 = the
// group's band, member-major (4 x (T + 3) weights); dst = the ring at the
// group's first column and the lane's ring row.
template <int C, int TAPS, int O0>
__device__ __forceinline__ void h_band(const float (&win)[3][4 * C], const float4 *w4, float4 *dst, int Q, int HR,
                                       int M, int hs)
{
    constexpr int HB = TAPS + 3;
    constexpr int c0 = O0 / 4, c1 = (O0 + HB + 3) / 4;
    static_assert(c1 <= 3, "a group's band lies in 3 chunks");
    float w[kG * HB];
#pragma unroll
    for (int i = 0; i < HB; ++i) {
        const float4 v = w4[i];
        w[4 * i] = v.x;
        w[4 * i + 1] = v.y;
        w[4 * i + 2] = v.z;
        w[4 * i + 3] = v.w;
    }
    float acc[kG][C];
#pragma unroll
    for (int g = 0; g < kG; ++g)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[g][c] = 0.f;
#pragma unroll
    for (int ch = c0; ch < c1; ++ch) {
#pragma unroll
        for (int px = 0; px < 4; ++px) {
            const int j = ch * 4 + px - O0;
            if (j >= 0 && j < HB) {
#pragma unroll
                for (int g = 0; g < kG; ++g)
#pragma unroll
                    for (int c = 0; c < C; ++c) acc[g][c] = fmaf(w[g * HB + j], win[ch][px * C + c], acc[g][c]);
            }
        }
    }
    float o[kG * C];
#pragma unroll
    for (int g = 0; g < kG; ++g)
#pragma unroll
        for (int c = 0; c < C; ++c) o[g * C + c] = acc[g][c];
#pragma unroll
    for (int v = 0; v < C; ++v) dst[v * Q] = make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
    if (hs < M) {
#pragma unroll
        for (int v = 0; v < C; ++v)
            dst[v * Q + HR] = make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
    }
}

template <int C, int TAPS>
__device__ __forceinline__ void h_dispatch(int o0, const float (&win)[3][4 * C], const float4 *w4, float4 *dst, int Q,
                                           int HR, int M, int hs)
{
    switch (o0) {
    case 0: h_band<C, TAPS, 0>(win, w4, dst, Q, HR, M, hs); break;
    case 1: h_band<C, TAPS, 1>(win, w4, dst, Q, HR, M, hs); break;
    case 2: h_band<C, TAPS, 2>(win, w4, dst, Q, HR, M, hs); break;
    default: h_band<C, TAPS, 3>(win, w4, dst, Q, HR, M, hs); break;
    }
}

// Vertical pass of one row group for one 4-sample ring column: src = the
// column at the group's first window row, wb = the group's band, j-major (the
// 4 rows' weights at ring row j); writes the group's 4 output rows of the
// column.
template <typename T, int TAPS>
__device__ __forceinline__ void v_band(const float4 *src, const float4 *wb, T *o, int64_t out_stride, int rows,
                                       int nsamp, bool vec_ok)
{
    constexpr int HB = TAPS + 3;
    float a[kG][4];
#pragma unroll
    for (int r = 0; r < kG; ++r) a[r][0] = a[r][1] = a[r][2] = a[r][3] = 0.f;
#pragma unroll
    for (int j = 0; j < HB; ++j) {
        const float4 d = src[j];
        const float4 wq = wb[j];
        const float wr[kG] = {wq.x, wq.y, wq.z, wq.w};
#pragma unroll
        for (int r = 0; r < kG; ++r) {
            a[r][0] = fmaf(wr[r], d.x, a[r][0]);
            a[r][1] = fmaf(wr[r], d.y, a[r][1]);
            a[r][2] = fmaf(wr[r], d.z, a[r][2]);
            a[r][3] = fmaf(wr[r], d.w, a[r][3]);
        }
    }
    if (rows == kG && nsamp == 4 && vec_ok) {
#pragma unroll
        for (int r = 0; r < kG; ++r) stream::store4<T>(o + r * out_stride, a[r][0], a[r][1], a[r][2], a[r][3]);
    } else {
#pragma unroll
        for (int r = 0; r < kG; ++r) {
            if (r >= rows) break;
            for (int i = 0; i < 4 && i < nsamp; ++i) o[r * out_stride + i] = stream::round_to<T>(a[r][i]);
        }
    }
}

// Bounded wait of every lane of a warp; true only if all lanes saw the phase.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err)
{
    const bool ok = fused::wait_or_abort(bar, parity, abort_flag, err);
    return __all_sync(0xffffffffu, ok);
}

// Several images in one launch (a batch): CTA b belongs to image i with
// cta_off[i] <= b < cta_off[i + 1] and takes that image's CTA b - cta_off[i];
// ps and maps hold each image's parameters and 64-byte aligned tensor map.
struct Multi {
    const Params *ps;
    const CUtensorMap *maps;
    const int32_t *cta_off; // [n + 1]
    int32_t n;
};

// The work of one CTA: CTA `bid` of the image that `tmap` and `p` describe.
template <typename T, int C, int TAPS, int BIG>
__device__ __forceinline__ void xstream_cta(const CUtensorMap *tmap_ptr, const Params &p, int bid)
{
    const CUtensorMap &tmap = *tmap_ptr;
    constexpr int HB = TAPS + 3; // band width
    constexpr int GB = kG * HB;  // band weights per group
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (fused::smem_addr(smem_raw) & 127u)) & 127u);
    const int ngx = p.SW / kG;
    const int P = p.P, Q = p.Q, HR = p.HR, M = p.M, NI = p.NI, WP = p.WP;
    const int nch = (p.SW * C) / 4; // 4-sample ring columns
    const Layout L = layout(NI, P, Q, nch, ngx, TAPS, WP, p.nblk, p.offB != 0, int(sizeof(T)));
    unsigned char *in_ring = smem;
    unsigned char *stg = in_ring + L.in_ring;
    unsigned char *b_ring = stg + L.stg;
    float4 *hring = reinterpret_cast<float4 *>(b_ring + L.b_ring);
    float *hw_s = reinterpret_cast<float *>(b_ring + L.b_ring + L.hring);
    int32_t *hc_s = reinterpret_cast<int32_t *>(b_ring + L.b_ring + L.hring + L.hw);
    int32_t *pe_s = reinterpret_cast<int32_t *>(b_ring + L.b_ring + L.hring + L.hw + L.hc);
    uint64_t *bars = reinterpret_cast<uint64_t *>(b_ring + L.b_ring + L.hring + L.hw + L.hc + L.pe);
    uint64_t *full_in = bars, *empty_in = bars + kMaxNI;
    uint64_t *full_w = bars + 2 * kMaxNI, *band_w = full_w + 1, *empty_w = band_w + kNW;
    uint64_t *hfull = empty_w + kNW, *vfree = hfull + 2;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(vfree + 2);
    float *stg_w = reinterpret_cast<float *>(stg);                  // [WP][4][T] as copied
    int32_t *stg_vi = reinterpret_cast<int32_t *>(stg + L.wv);       // group descriptors from a multiple of 4
    auto slot_in = [&](int s) { return reinterpret_cast<T *>(in_ring + size_t(s) * L.in_blk); };
    auto slot_vb = [&](int s) { return reinterpret_cast<float *>(b_ring + size_t(s) * L.bslot); };
    auto slot_vr = [&](int s) { return reinterpret_cast<int32_t *>(b_ring + size_t(s) * L.bslot + L.vb); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int HW = p.HW, VW = p.VW;
    const int strip = bid % p.n_strips, range = bid / p.n_strips;
    const int p0 = range * p.gpr;
    const int p1 = min(p.groups_y, p0 + p.gpr);
    if (p0 >= p1) return;
    const int g0 = strip * ngx;
    const int ngv = min(ngx, p.groups_x - g0); // column groups of the strip inside the image
    const int xs = stream::first_staged<T>((__ldg(p.hinfo + g0) & 0xffffff) * C); // first staged sample
    auto last_row = [&](int q) { // last input row of row group q's windows
        const int vi = __ldg(p.vinfo + q);
        return (vi & 0xffffff) + v_off(vi >> 24, 3) + TAPS - 1;
    };
    const int r_lo = __ldg(p.vinfo + p0) & 0xffffff;
    const int nblk = min((last_row(p1 - 1) + 1 - r_lo + kRB - 1) / kRB, p.nblk);
    const uint32_t blk_bytes = uint32_t(kRB) * P * sizeof(T) * (p.offB ? 2u : 1u);
    // one thread: the input copy of block k into slot k % NI
    auto issue_in = [&](int k) {
        const int s = k % NI;
        fused::mbar_arrive_expect_tx(&full_in[s], blk_bytes);
        fused::tma_load_2d(slot_in(s), &tmap, &full_in[s], xs, r_lo + k * kRB);
        if (p.offB) fused::tma_load_2d(slot_in(s) + kRB * P, &tmap, &full_in[s], xs + p.offB, r_lo + k * kRB);
        if (p.pf && k + NI < nblk) {
            fused::tma_prefetch_2d(&tmap, xs, r_lo + (k + NI) * kRB);
            if (p.offB) fused::tma_prefetch_2d(&tmap, xs + p.offB, r_lo + (k + NI) * kRB);
        }
    };

    if (tid == 0) {
        for (int s = 0; s < NI; ++s) {
            fused::mbar_init(&full_in[s], 1);
            fused::mbar_init(&empty_in[s], 32 * HW);
        }
        fused::mbar_init(full_w, 1);
        for (int s = 0; s < kNW; ++s) {
            fused::mbar_init(&band_w[s], 32);
            fused::mbar_init(&empty_w[s], 32 * VW);
        }
        for (int b = 0; b < 2; ++b) {
            fused::mbar_init(&hfull[b], 32 * HW);
            fused::mbar_init(&vfree[b], 32 * VW);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // the first staged blocks' copies, so their latency overlaps the set-up
        // below (which does not touch the input slots)
        for (int k = 0; k < NI && k < nblk; ++k) issue_in(k);
    }
    // the strip's horizontal band: member g's weight at input j of the run
    // from the group's first window (groups past the image: zeros)
    const int nthr = int(blockDim.x);
    for (int e = tid; e < ngx * GB; e += nthr) {
        const int q = e / GB;
        float v = 0.f;
        if (q < ngv) {
            const int r = e - q * GB, g = r / HB, j = r - g * HB;
            const int t = j - h_off(__ldg(p.hinfo + g0 + q) >> 24, g);
            if (t >= 0 && t < TAPS) v = __ldg(p.wx + (size_t(g0 + q) * kG + g) * TAPS + t);
        }
        hw_s[e] = v;
    }
    // per column group: its staged offset (the second box's sub-buffer when
    // the run does not fit the first box) | the first window's offset << 24
    for (int q = tid; q < ngx; q += nthr) {
        int o = 0, o0 = 0;
        if (q < ngv) {
            const int hi = __ldg(p.hinfo + g0 + q);
            o0 = (hi >> 24) & 3;
            o = (hi & 0xffffff) * C - xs;
            if (p.offB && o + p.JH * C > P) o += kRB * P - p.offB;
        }
        hc_s[q] = o | (o0 << 24);
    }
    // the bands read ring rows (and staged samples) outside a group's windows
    // with zero weights: start the ring finite
    for (int e = tid; e < nch * Q; e += nthr) hring[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    // row group q is complete after block kb(q) (its last window row is
    // filtered then); pe_s[k] = first row group not complete after block k
    auto kb = [&](int q) {
        const int k = (last_row(q) - r_lo) / kRB;
        return k < 0 ? 0 : (k > nblk - 1 ? nblk - 1 : k);
    };
    for (int q = p0 + tid; q < p1; q += nthr) {
        const int kp = kb(q);
        const int kn = q + 1 < p1 ? kb(q + 1) : nblk;
        for (int k = kp; k < kn; ++k) pe_s[k] = q + 1;
        if (q == p0)
            for (int k = 0; k < kp; ++k) pe_s[k] = p0;
    }
    __syncthreads();

    if (warp == 0) {
        // ====== producer: input blocks, window weights, vertical bands ======
        // Per block k: the input copy, then block k - 1's bands (from the
        // weights staged last time), then block k's weights into the staging
        // area, so the copies of block k fly while the bands are built.
        int ki = min(NI, nblk), kw = 0; // blocks whose input copies / weight copies were issued
        bool ok = true;
        // builds block j's vertical bands from the staged window weights (all lanes)
        auto build = [&](int j) {
            const int sv = j % kNW;
            if (!warp_wait(full_w, uint32_t(j & 1), abort_flag, p.err)) return false;
            // the slot held block j - 2's bands
            if (j >= kNW && !warp_wait(&empty_w[sv], uint32_t((j / kNW - 1) & 1), abort_flag, p.err)) return false;
            const int ps = j ? pe_s[j - 1] : p0, pe = pe_s[j];
            const int n = pe - ps <= WP ? pe - ps : 0;
            const int32_t *vis = stg_vi + (ps & 3);
            float *vb = slot_vb(sv);
            int32_t *vr = slot_vr(sv);
            // lane: one (group, row) pair at a time; row r of a group reads
            // its T weights and writes its column of the group's band (j-major:
            // [j][r]) -- the T weights from position o_r on, zeros elsewhere
            for (int e = lane; e < n * kG; e += 32) {
                const int gi = e >> 2, r = e & 3;
                const int o = v_off(vis[gi] >> 24, r);
                const float *src = stg_w + (gi * kG + r) * TAPS;
                float w[TAPS];
#pragma unroll
                for (int t = 0; t < TAPS; ++t) w[t] = src[t];
                float *dst = vb + gi * GB + r;
#pragma unroll
                for (int t = 0; t < TAPS; ++t) dst[(o + t) * kG] = w[t];
#pragma unroll
                for (int z = 0; z < 3; ++z) dst[(z < o ? z : z + TAPS) * kG] = 0.f;
            }
            for (int gi = lane; gi < n; gi += 32) vr[gi] = vis[gi] & 0xffffff;
            // the staging area was read: the next copy into it (async proxy) comes after
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            fused::mbar_arrive(&band_w[sv]);
            return true;
        };
        for (int k = 0; k < nblk && ok; ++k) {
            const int s = k % NI;
            if (k >= NI) { // (the first NI blocks were issued before the set-up)
                if (!warp_wait(&empty_in[s], uint32_t((k / NI - 1) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                if (lane == 0) issue_in(k);
                ki = k + 1;
            }
            if (k >= 1 && !build(k - 1)) {
                ok = false;
                break;
            }
            if (lane == 0) {
                const int ps = k ? pe_s[k - 1] : p0, pe = pe_s[k];
                int n = pe - ps;
                if (n > WP) {
                    fused::flag(p.err, fused::kErrBounds);
                    n = 0;
                }
                const int pa = ps & ~3, pb = (pe + 3) & ~3;
                const uint32_t wbytes = uint32_t(n) * kG * TAPS * 4, vbytes = n ? uint32_t(pb - pa) * 4 : 0u;
                fused::mbar_arrive_expect_tx(full_w, wbytes + vbytes);
                if (n) {
                    fused::bulk_load(stg_w, p.wy + size_t(ps) * kG * TAPS, wbytes, full_w);
                    fused::bulk_load(stg_vi, p.vinfo + pa, vbytes, full_w);
                }
            }
            kw = k + 1;
        }
        if (ok && nblk >= 1) ok = build(nblk - 1);
        if (!ok && lane == 0) {
            // let the copies still in flight land (bounded) before the CTA
            // exits: the last block issued into each input slot, the last
            // weight copy
            for (int b = max(0, ki - NI); b < ki; ++b)
                fused::mbar_wait_bounded(&full_in[b % NI], uint32_t((b / NI) & 1));
            if (kw) fused::mbar_wait_bounded(full_w, uint32_t((kw - 1) & 1));
        }
        return;
    }
    if (warp <= HW) {
        // ================ horizontal pass: block k into the ring ================
        // Warp hw takes the column groups [qa, qb) of every block, in order,
        // with the 3 chunks of the current group's run in registers: the next
        // group's run starts 0 or 4 pixels further (an upscale), so it costs
        // at most one new chunk (a jump into the second staged box reloads).
        const int hw = warp - 1;
        const int qa = hw * ngv / HW, qb = (hw + 1) * ngv / HW;
        int base_k = 0; // ring row of block k's first row
        for (int k = 0; k < nblk; ++k, base_k = base_k + kRB >= HR ? base_k + kRB - HR : base_k + kRB) {
            const int s = k % NI;
            bool good = warp_wait(&full_in[s], uint32_t((k / NI) & 1), abort_flag, p.err);
            // the ring rows of block k held block k - 2's rows
            if (good && k >= 2) good = warp_wait(&vfree[k & 1], uint32_t(((k - 2) >> 1) & 1), abort_flag, p.err);
            if (!good) break;
            int hs = base_k + lane;
            if (hs >= HR) hs -= HR;
            const T *rowp = slot_in(s) + size_t(lane) * P;
            if (qa < qb) {
                float win[3][4 * C];
                int cur = hc_s[qa] & 0xffffff;
#pragma unroll
                for (int c = 0; c < 3; ++c) load_chunk<T, C>(rowp + cur + 4 * C * c, win[c]);
                for (int q = qa; q < qb; ++q) {
                    const int hc = hc_s[q], off = hc & 0xffffff;
                    if (off == cur + 4 * C) {
#pragma unroll
                        for (int e = 0; e < 4 * C; ++e) {
                            win[0][e] = win[1][e];
                            win[1][e] = win[2][e];
                        }
                        load_chunk<T, C>(rowp + off + 8 * C, win[2]);
                    } else if (off != cur) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) load_chunk<T, C>(rowp + off + 4 * C * c, win[c]);
                    }
                    cur = off;
                    h_dispatch<C, TAPS>(hc >> 24, win, reinterpret_cast<const float4 *>(hw_s + q * GB),
                                        hring + (q * C) * Q + hs, Q, HR, M, hs);
                }
            }
            fused::mbar_arrive(&empty_in[s]);
            fused::mbar_arrive(&hfull[k & 1]);
        }
        return;
    }
    {
        // ================ vertical pass: the row groups block k completes ================
        // Items (row group, 4-sample column) of block k in a flat order (group
        // major); one task is 32 consecutive items, one per lane (lanes of a
        // task may take different groups: the code path is the same).  Warp
        // vw takes tasks vw, vw + VW, ... of the stream over all blocks.
        const int vw = warp - 1 - HW;
        const uint32_t rcp = (1u << 24) / uint32_t(nch) + 1u; // floor(f / nch) = (f rcp) >> 24 for f < 2^16
        int next = vw, tbase = 0;
        const int64_t row_samples = p.out_w * C;
        const int64_t x0s = int64_t(strip) * p.SW * C;
        const bool vec_ok =
            ((reinterpret_cast<uintptr_t>(p.out) | uintptr_t(p.out_stride * sizeof(T))) & (4 * sizeof(T) - 1)) == 0;
        int base_k = 0; // ring row of block k's first row
        for (int k = 0; k < nblk; ++k, base_k = base_k + kRB >= HR ? base_k + kRB - HR : base_k + kRB) {
            const int sv = k % kNW;
            bool good = warp_wait(&band_w[sv], uint32_t((k / kNW) & 1), abort_flag, p.err);
            if (good) good = warp_wait(&hfull[k & 1], uint32_t((k >> 1) & 1), abort_flag, p.err);
            if (!good) break;
            const int ps = k ? pe_s[k - 1] : p0, pe = pe_s[k];
            const int n = pe - ps <= WP ? pe - ps : 0;
            const int items = n * nch, ntask = (items + 31) >> 5;
            const float4 *vbs = reinterpret_cast<const float4 *>(slot_vb(sv));
            const int32_t *vrs = slot_vr(sv);
            const int r_k = r_lo + k * kRB; // block k's first input row
            for (; next < tbase + ntask; next += VW) {
                const int f = ((next - tbase) << 5) + lane;
                if (f < items) {
                    const int gi = int((uint32_t(f) * rcp) >> 24), ch = f - gi * nch;
                    // the group's first window row: within (32k - JV, 32k + 32) of r_lo
                    int hs0 = base_k + (vrs[gi] - r_k);
                    if (hs0 < 0) hs0 += HR;
                    if (hs0 >= HR) hs0 -= HR;
                    const int64_t y0 = int64_t(kG) * (ps + gi), sx = x0s + int64_t(ch) * 4;
                    const int64_t rem_rows = p.out_h - y0, rem_samp = row_samples - sx;
                    const int rows = rem_rows < kG ? int(rem_rows) : kG;
                    const int nsamp = rem_samp < 4 ? int(rem_samp) : 4;
                    if (nsamp > 0)
                        v_band<T, TAPS>(hring + ch * Q + hs0, vbs + gi * (GB / 4),
                                            static_cast<T *>(p.out) + y0 * p.out_stride + sx, p.out_stride, rows,
                                            nsamp, vec_ok);
                }
            }
            tbase += ntask;
            fused::mbar_arrive(&empty_w[sv]);
            fused::mbar_arrive(&vfree[k & 1]);
        }
    }
}

// BIG = 0: up to kSmallWarps warps, two CTAs per SM (at most 85 registers a
// thread); BIG = 1: up to kMaxWarps warps, one CTA per SM.
template <typename T, int C, int TAPS, int BIG>
__global__ void __launch_bounds__(BIG ? 32 * kMaxWarps : 32 * kSmallWarps, BIG ? 1 : 2)
    xstream_kernel(const __grid_constant__ CUtensorMap tmap, const Params p)
{
    xstream_cta<T, C, TAPS, BIG>(&tmap, p, int(blockIdx.x));
}

// The same kernel over the CTAs of several images (one launch for a batch's
// streamed upscales of one kind).  BIG = 2: two CTAs per SM of at most
// kMidWarps warps, whose higher register cap keeps the multi-image lookup
// from spilling (the single-channel 4-tap variant spilled 16 bytes under the
// 12-warp cap).
template <typename T, int C, int TAPS, int BIG>
__global__ void __launch_bounds__(BIG == 1 ? 32 * kMaxWarps : BIG == 2 ? 32 * kMidWarps : 32 * kSmallWarps,
                                  BIG == 1 ? 1 : 2)
    xstream_multi_kernel(const __grid_constant__ Multi m)
{
    const int b = int(blockIdx.x);
    int lo = 0, hi = m.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(m.cta_off + mid) <= b)
            lo = mid;
        else
            hi = mid;
    }
    const Params p = m.ps[lo];
    xstream_cta<T, C, TAPS, BIG>(m.maps + lo, p, b - __ldg(m.cta_off + lo));
}

// Instantiated kernels: storage type x channels x taps per output x the
// variant (big = 0 / 1: one image, up to kSmallWarps / kMaxWarps warps; 2 / 3:
// the multi-image kernel with the same launch bounds; 4: the multi-image
// kernel for up to kMidWarps warps).
template <typename T, int C, int TAPS> const void *kernel_big(int big)
{
    return big == 1   ? reinterpret_cast<const void *>(&xstream_kernel<T, C, TAPS, 1>)
           : big == 0 ? reinterpret_cast<const void *>(&xstream_kernel<T, C, TAPS, 0>)
           : big == 3 ? reinterpret_cast<const void *>(&xstream_multi_kernel<T, C, TAPS, 1>)
           : big == 4 ? reinterpret_cast<const void *>(&xstream_multi_kernel<T, C, TAPS, 2>)
                      : reinterpret_cast<const void *>(&xstream_multi_kernel<T, C, TAPS, 0>);
}
template <typename T> const void *kernel_table(int C, int taps, int big)
{
    if (C == 1 && taps == 4) return kernel_big<T, 1, 4>(big);
    if (C == 1 && taps == 6) return kernel_big<T, 1, 6>(big);
    if (C == 3 && taps == 4) return kernel_big<T, 3, 4>(big);
    if (C == 3 && taps == 6) return kernel_big<T, 3, 6>(big);
    return nullptr;
}

// defined in rs_xstream_f32.cu, rs_xstream_f16.cu, rs_xstream_bf16.cu
const void *kernel_f32(int C, int taps, int big);
const void *kernel_f16(int C, int taps, int big);
const void *kernel_bf16(int C, int taps, int big);

} // namespace xstream
} // namespace rs
