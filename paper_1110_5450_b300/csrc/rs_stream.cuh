// rs_stream.cuh -- the row-streaming resample kernel (horizontal pass first).
//
// A CTA owns a strip of SW output columns and a range of output-row pairs.  It
// walks down the input rows the range needs in blocks of 32 rows:
//   * a ring of NI staged input blocks is kept filled by TMA copies (thread 0
//     re-issues a slot as soon as its block has been consumed, so NI - 1
//     copies are in flight while one block is processed);
//   * the horizontal pass turns each staged input row into the strip's SW
//     output columns (lanes run along the 32 rows of a block, every lane holds
//     the 4-pixel chunks of its row in registers and applies the band of G = 4
//     outputs; the band's start is 4-pixel aligned, so chunks load as 16-byte
//     words) and appends the results to a ring of horizontally filtered rows;
//   * the vertical pass turns every group of 4 output rows whose taps are all
//     in that ring into its rows (lanes along 4-sample columns of the strip,
//     packed FP32 FMAs, each loaded sample used by the 4 rows) and writes them
//     with 16-byte stores.
// The ring of filtered rows repeats its first M slots after its end, so the
// J_v rows of a row group are always linear in shared memory.  Every wait is
// bounded (2 s); a timeout sets the plan's error word and stops the CTA.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rs_fused.cuh"

namespace rs {
namespace stream {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRB = 32; // input rows per staged block (one per lane of a horizontal task)
constexpr int kG = 4;   // outputs per horizontal band group
// Output rows per vertical band group: 8 (scalar FMAs, each loaded sample
// feeds 8 rows) where the band stays narrow, else 4 (packed FMAs on pairs of
// samples with every weight stored twice).
constexpr int kGV8 = 8, kGV4 = 4;
// floats per vertical tap of a group in the band
__host__ __device__ constexpr int vtap_floats(int GV) { return GV == 4 ? 8 : GV; }
constexpr int kMaxNI = 4;

struct Params {
    const void *in; // the image in its storage type (FP32, FP16 or BF16)
    void *out;
    int64_t in_h, in_w, out_h, out_w;
    int64_t in_stride, out_stride;
    const int32_t *hbase; // [groups_x] first input pixel of each horizontal group (multiple of 4)
    const float *hband;   // [groups_x][JH][4] weights of the group's 4 outputs per input pixel
    const int32_t *vbase; // [pairs] first input row of each group of 8 output rows ("pair" below)
    const float *vband;   // [pairs][JV][8] per tap: the weights of the group's 8 rows
    int32_t JH, JV;       // horizontal taps (multiple of 4), vertical taps (multiple of 2)
    int32_t SW;           // output pixels per strip (multiple of 4)
    int32_t n_strips, pairs, pairs_per_range, groups_x;
    int32_t P;            // staged input pitch in samples (FP32: P / 4 odd; 16-bit: P / 8 odd)
    int32_t offB;         // 0: one staged box of P x 32 samples per block; else a second box
                          //    P x 32 starting offB samples further (rows wider than one
                          //    256-element box), in its own 128-byte aligned sub-buffer
    int32_t Q;            // rows per 4-sample column of the filtered-row ring (>= HR + M, odd)
    int32_t NI;           // staged input blocks (ring slots)
    int32_t NW;           // warp-specialised kernel: vertical weight slots (0: phase-alternating kernel)
    int32_t HW;           // warp-specialised kernel: warps on the horizontal pass
    int32_t HR, M;        // filtered-row ring rows, mirrored rows
    int32_t WP;           // most row groups that become ready after one block
    int32_t GV;           // rows per vertical group (the kernel's template argument)
    int *err;
};

constexpr int kMaxBlk = 512; // staged blocks per CTA (row range) at most

// Shared memory: NI slots of (staged input block | the vertical weights and
// row bases of the pairs that block completes) | filtered-row ring |
// horizontal band | group offsets | per-block pair ends | barriers.
struct Layout {
    size_t in_blk, wv, vb, slot, hring, hb, cb, pe, total;
};

__host__ __device__ inline Layout layout(int NI, int P, int Q, int nch, int ngx, int JH, int WP, int JV,
                                         bool two_boxes, int GV, int es)
{
    Layout L;
    L.in_blk = size_t(kRB) * P * es * (two_boxes ? 2 : 1);
    L.wv = size_t(WP) * JV * vtap_floats(GV) * 4;
    L.vb = fused::align_up(size_t(WP + 8) * 4, 16);
    L.slot = fused::align_up(L.in_blk + L.wv + L.vb, 128);
    L.hring = fused::align_up(size_t(nch) * Q * 16, 128);
    L.hb = fused::align_up(size_t(ngx) * JH * kG * 4, 128);
    L.cb = fused::align_up(size_t(ngx) * 4, 128);
    L.pe = fused::align_up(size_t(kMaxBlk) * 4, 128);
    L.total = 128 + size_t(NI) * L.slot + L.hring + L.hb + L.cb + L.pe + 128;
    return L;
}

// 4 consecutive staged samples as floats: one 16-byte load (FP32) or one
// 8-byte load converted (FP16 / BF16).
template <typename T> __device__ __forceinline__ float4 load4(const T *p);
template <> __device__ __forceinline__ float4 load4<float>(const float *p)
{
    return *reinterpret_cast<const float4 *>(p);
}
template <> __device__ __forceinline__ float4 load4<__half>(const __half *p)
{
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
template <> __device__ __forceinline__ float4 load4<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// 4 consecutive output samples, rounded to nearest in the storage type: one
// 16-byte store (FP32) or one 8-byte store (FP16 / BF16).
template <typename T> __device__ __forceinline__ void store4(T *p, float a, float b, float c, float d);
template <> __device__ __forceinline__ void store4<float>(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
template <> __device__ __forceinline__ void store4<__half>(__half *p, float a, float b, float c, float d)
{
    const __half2 x = __floats2half2_rn(a, b), y = __floats2half2_rn(c, d);
    *reinterpret_cast<uint2 *>(p) = make_uint2(*reinterpret_cast<const uint32_t *>(&x),
                                               *reinterpret_cast<const uint32_t *>(&y));
}
template <> __device__ __forceinline__ void store4<__nv_bfloat16>(__nv_bfloat16 *p, float a, float b, float c, float d)
{
    const __nv_bfloat162 x = __floats2bfloat162_rn(a, b), y = __floats2bfloat162_rn(c, d);
    *reinterpret_cast<uint2 *>(p) = make_uint2(*reinterpret_cast<const uint32_t *>(&x),
                                               *reinterpret_cast<const uint32_t *>(&y));
}
template <typename T> __device__ __forceinline__ T round_to(float v);
template <> __device__ __forceinline__ float round_to<float>(float v) { return v; }
template <> __device__ __forceinline__ __half round_to<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 round_to<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// First staged sample of a strip whose first band starts at sample x0 (a
// multiple of 4): a TMA box must start on a 16-byte boundary, so 16-bit
// strips start up to 4 samples early.
template <typename T> __host__ __device__ __forceinline__ int first_staged(int x0)
{
    return sizeof(T) == 2 ? (x0 & ~7) : x0;
}

// Horizontal pass of one 4-output group for the 32 rows of a staged block:
// lane = row; rowp = the lane's staged row, hs = its ring slot.
template <typename T, int C>
__device__ __forceinline__ void h_group(const T *rowp, int cbq, const float *hbq, int JH, float4 *hring, int q,
                                        int Q, int HR, int M, int hs)
{
    const T *src = rowp + cbq;
    const float4 *wq = reinterpret_cast<const float4 *>(hbq);
    float acc[kG][C];
#pragma unroll
    for (int g = 0; g < kG; ++g)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[g][c] = 0.f;
    for (int t0 = 0; t0 < JH; t0 += 4) {
        // 4 input pixels of this lane's row (C 16-byte words) ...
        float d[4 * C];
#pragma unroll
        for (int v = 0; v < C; ++v) {
            const float4 x = load4<T>(src + 4 * v);
            d[4 * v] = x.x;
            d[4 * v + 1] = x.y;
            d[4 * v + 2] = x.z;
            d[4 * v + 3] = x.w;
        }
        src += 4 * C;
        // ... times the 4 outputs' weights at those pixels (warp-uniform)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float4 w = wq[t];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float x = d[t * C + c];
                acc[0][c] = fmaf(w.x, x, acc[0][c]);
                acc[1][c] = fmaf(w.y, x, acc[1][c]);
                acc[2][c] = fmaf(w.z, x, acc[2][c]);
                acc[3][c] = fmaf(w.w, x, acc[3][c]);
            }
        }
        wq += 4;
    }
    // the group's 4 x C filtered samples, contiguous in the ring row
    float4 o[C];
    float *of = reinterpret_cast<float *>(o);
#pragma unroll
    for (int g = 0; g < kG; ++g)
#pragma unroll
        for (int c = 0; c < C; ++c) of[g * C + c] = acc[g][c];
    float4 *dst = hring + (q * C) * Q + hs;
#pragma unroll
    for (int v = 0; v < C; ++v) dst[v * Q] = o[v];
    if (hs < M) {
#pragma unroll
        for (int v = 0; v < C; ++v) dst[v * Q + HR] = o[v];
    }
}

// Vertical pass of one row group (GV output rows) for one 4-sample column:
// src4 = the column's first tap row in the ring, wv = the group's weights.
template <typename T, int JV, int GV>
__device__ __forceinline__ void v_task(const float4 *src4, const float4 *wv, T *out, int64_t out_stride,
                                       int64_t y0, int64_t out_h, int64_t sx, int64_t row_samples, bool vec_ok)
{
    float a[GV][4];
    if constexpr (GV == 4) {
        // 4 rows x 2 sample pairs of packed accumulators; the band stores
        // every weight twice, so pairs load as they are
        const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(src4);
        const ulonglong2 *w2 = reinterpret_cast<const ulonglong2 *>(wv);
        uint64_t acc[GV][2];
#pragma unroll
        for (int r = 0; r < GV; ++r) acc[r][0] = acc[r][1] = 0ull;
#pragma unroll
        for (int j = 0; j < JV; ++j) {
            const ulonglong2 dd = src[j];
#pragma unroll
            for (int r2 = 0; r2 < GV / 2; ++r2) {
                const ulonglong2 w = w2[(GV / 2) * j + r2]; // rows 2 r2, 2 r2 + 1
                acc[2 * r2][0] = fused::fma2(w.x, dd.x, acc[2 * r2][0]);
                acc[2 * r2][1] = fused::fma2(w.x, dd.y, acc[2 * r2][1]);
                acc[2 * r2 + 1][0] = fused::fma2(w.y, dd.x, acc[2 * r2 + 1][0]);
                acc[2 * r2 + 1][1] = fused::fma2(w.y, dd.y, acc[2 * r2 + 1][1]);
            }
        }
#pragma unroll
        for (int r = 0; r < GV; ++r) {
            fused::unpack2(acc[r][0], a[r][0], a[r][1]);
            fused::unpack2(acc[r][1], a[r][2], a[r][3]);
        }
    } else {
        // 8 rows x 4 samples; each loaded sample feeds the 8 rows
#pragma unroll
        for (int r = 0; r < GV; ++r) a[r][0] = a[r][1] = a[r][2] = a[r][3] = 0.f;
#pragma unroll
        for (int j = 0; j < JV; ++j) {
            const float4 d = src4[j];
            float w[GV];
#pragma unroll
            for (int v = 0; v < GV / 4; ++v) {
                const float4 q = wv[(GV / 4) * j + v];
                w[4 * v] = q.x;
                w[4 * v + 1] = q.y;
                w[4 * v + 2] = q.z;
                w[4 * v + 3] = q.w;
            }
#pragma unroll
            for (int r = 0; r < GV; ++r) {
                a[r][0] = fmaf(w[r], d.x, a[r][0]);
                a[r][1] = fmaf(w[r], d.y, a[r][1]);
                a[r][2] = fmaf(w[r], d.z, a[r][2]);
                a[r][3] = fmaf(w[r], d.w, a[r][3]);
            }
        }
    }
    T *o = out + y0 * out_stride + sx;
    if (y0 + GV <= out_h && sx + 4 <= row_samples && vec_ok) {
        // whole rows of 4 samples: 16-byte (FP32) or 8-byte (16-bit) stores
#pragma unroll
        for (int h = 0; h < GV; ++h) store4<T>(o + h * out_stride, a[h][0], a[h][1], a[h][2], a[h][3]);
    } else {
#pragma unroll
        for (int h = 0; h < GV; ++h) {
            if (y0 + h >= out_h) break;
            for (int i = 0; i < 4 && sx + i < row_samples; ++i) o[h * out_stride + i] = round_to<T>(a[h][i]);
        }
    }
}

// The work of one CTA of the phase-alternating band kernel: CTA `bid` of the
// image that `tmap_ptr` and `p` describe.
template <typename T, int C, int JV, int GV>
__device__ __forceinline__ void stream_cta(const CUtensorMap *tmap_ptr, const Params &p, int bid)
{
    const CUtensorMap &tmap = *tmap_ptr;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (fused::smem_addr(smem_raw) & 127u)) & 127u);
    const int ngx = p.SW / kG;
    const int JH = p.JH, P = p.P, Q = p.Q, HR = p.HR, M = p.M, NI = p.NI, WP = p.WP;
    const int nch = (p.SW * C) / 4; // 4-sample columns of a filtered row
    const Layout L = layout(NI, P, Q, nch, ngx, JH, WP, JV, p.offB != 0, GV, int(sizeof(T)));
    unsigned char *slots = smem;
    // filtered rows, column-major in 4-sample columns: [nch][Q] float4, so the
    // vertical taps of a column are consecutive 16-byte words
    float4 *hring = reinterpret_cast<float4 *>(smem + NI * L.slot);
    float *hb = reinterpret_cast<float *>(smem + NI * L.slot + L.hring);
    int32_t *cb = reinterpret_cast<int32_t *>(smem + NI * L.slot + L.hring + L.hb);
    int32_t *pe_s = reinterpret_cast<int32_t *>(smem + NI * L.slot + L.hring + L.hb + L.cb);
    unsigned char *ctl = smem + NI * L.slot + L.hring + L.hb + L.cb + L.pe;
    uint64_t *full = reinterpret_cast<uint64_t *>(ctl); // [kMaxNI]
    volatile int *abort_flag = reinterpret_cast<volatile int *>(ctl + 8 * kMaxNI);
    auto slot_in = [&](int s) { return reinterpret_cast<T *>(slots + s * L.slot); };
    auto slot_wv = [&](int s) { return reinterpret_cast<const ulonglong2 *>(slots + s * L.slot + L.in_blk); };
    auto slot_vb = [&](int s) { return reinterpret_cast<const int32_t *>(slots + s * L.slot + L.in_blk + L.wv); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int strip = bid % p.n_strips, range = bid / p.n_strips;
    const int p0 = range * p.pairs_per_range;
    const int p1 = min(p.pairs, p0 + p.pairs_per_range);
    if (p0 >= p1) return;
    const int g0 = strip * ngx;
    const int ngv = min(ngx, p.groups_x - g0); // groups of the strip inside the image
    const int xs = first_staged<T>(__ldg(p.hbase + g0) * C); // first staged sample (16-byte aligned)
    const int r_lo = __ldg(p.vbase + p0);
    const int r_hi = __ldg(p.vbase + p1 - 1) + JV;
    const int nblk = min((r_hi - r_lo + kRB - 1) / kRB, kMaxBlk);
    const uint32_t blk_bytes = uint32_t(L.in_blk);

    if (tid == 0) {
        for (int s = 0; s < NI; ++s) fused::mbar_init(&full[s], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the strip's horizontal band and group offsets (groups past the image: zeros)
    for (int e = tid; e < ngx * JH * kG; e += kThreads) {
        const int q = e / (JH * kG);
        hb[e] = q < ngv ? __ldg(p.hband + size_t(g0) * JH * kG + e) : 0.f;
    }
    // per group: offset of its band window in the staged block (the second
    // box's sub-buffer when the window does not fit the first box)
    for (int q = tid; q < ngx; q += kThreads) {
        int o = q < ngv ? __ldg(p.hbase + g0 + q) * C - xs : 0;
        if (p.offB && o + JH * C > P) o += kRB * P - p.offB;
        cb[q] = o;
    }
    // pair p is complete after block kb(p) (its last row is filtered then);
    // pe_s[k] = first pair not complete after block k
    auto kb = [&](int vb) {
        const int k = (vb + JV - r_lo + kRB - 1) / kRB - 1;
        return k < 0 ? 0 : (k > nblk - 1 ? nblk - 1 : k);
    };
    for (int q = p0 + tid; q < p1; q += kThreads) {
        const int kp = kb(__ldg(p.vbase + q));
        const int kn = q + 1 < p1 ? kb(__ldg(p.vbase + q + 1)) : nblk;
        for (int k = kp; k < kn; ++k) pe_s[k] = q + 1;
        if (q == p0)
            for (int k = 0; k < kp; ++k) pe_s[k] = p0;
    }
    __syncthreads();

    // thread 0: block k's input rows plus the weights and bases of its pairs
    auto issue = [&](int k) {
        const int s = k % NI;
        const int ps = k ? pe_s[k - 1] : p0, pe = pe_s[k];
        int n = pe - ps;
        if (n > WP) {
            fused::flag(p.err, fused::kErrBounds);
            n = 0;
        }
        const int pa = ps & ~3, pb = (pe + 3) & ~3;
        const uint32_t wbytes = uint32_t(n) * JV * vtap_floats(GV) * 4, vbytes = n ? uint32_t(pb - pa) * 4 : 0u;
        fused::mbar_arrive_expect_tx(&full[s], blk_bytes + wbytes + vbytes);
        fused::tma_load_2d(slot_in(s), &tmap, &full[s], xs, r_lo + k * kRB);
        if (p.offB) // second box: its own sub-buffer right after the first (128-byte aligned)
            fused::tma_load_2d(slot_in(s) + kRB * P, &tmap, &full[s], xs + p.offB, r_lo + k * kRB);
        if (n) {
            fused::bulk_load(const_cast<ulonglong2 *>(slot_wv(s)), p.vband + size_t(ps) * JV * vtap_floats(GV), wbytes,
                             &full[s]);
            fused::bulk_load(const_cast<int32_t *>(slot_vb(s)), p.vbase + pa, vbytes, &full[s]);
        }
    };
    if (tid == 0)
        for (int k = 0; k < NI && k < nblk; ++k) issue(k);

    const int64_t row_samples = p.out_w * C;
    const int64_t x0s = int64_t(strip) * p.SW * C; // first output sample of the strip
    // vector stores of 4 samples need an aligned output and row pitch
    const bool vec_ok =
        ((reinterpret_cast<uintptr_t>(p.out) | uintptr_t(p.out_stride * sizeof(T))) & (4 * sizeof(T) - 1)) == 0;
    int k = 0;
    for (; k < nblk; ++k) {
        const int slot = k % NI;
        const bool landed = fused::wait_or_abort(&full[slot], uint32_t((k / NI) & 1), abort_flag, p.err);
        const int base_k = (k * kRB) % HR; // ring slot of the block's first row
        // ---------------- horizontal pass: 32 rows x the strip's groups ----------------
        if (landed) {
            int hs = base_k + lane;
            if (hs >= HR) hs -= HR;
            const T *rowp = slot_in(slot) + size_t(lane) * P;
            for (int q = warp; q < ngv; q += kWarps)
                h_group<T, C>(rowp, cb[q], hb + q * JH * kG, JH, hring, q, Q, HR, M, hs);
        }
        // every thread agrees on whether the block landed (a timeout stops all)
        if (!__syncthreads_and(landed ? 1 : 0)) break;
        // ---------------- vertical pass: completed pairs x 4-sample chunks ----------------
        {
            const int ps = k ? pe_s[k - 1] : p0, pe = pe_s[k];
            const int n = pe - ps <= WP ? pe - ps : 0;
            const ulonglong2 *wvs = slot_wv(slot);
            const int32_t *vbs = slot_vb(slot) - (ps & ~3); // indexed by pair
            const int ntask = n * nch;
            int po = tid / nch, ch = tid - (tid / nch) * nch;
            const int dpo = kThreads / nch, dch = kThreads - dpo * nch;
            for (int t = tid; t < ntask; t += kThreads) {
                const int pr = ps + po;
                // first row of the group: within (32k - JV, 32k + 32 - JV] of r_lo
                int hs0 = base_k + (vbs[pr] - r_lo - k * kRB);
                if (hs0 < 0) hs0 += HR;
                if (hs0 >= HR) hs0 -= HR;
                v_task<T, JV, GV>(hring + ch * Q + hs0,
                                  reinterpret_cast<const float4 *>(wvs) + po * JV * (vtap_floats(GV) / 4),
                                  static_cast<T *>(p.out),
                               p.out_stride, int64_t(GV) * pr, p.out_h, x0s + int64_t(ch) * 4, row_samples, vec_ok);
                po += dpo;
                ch += dch;
                if (ch >= nch) {
                    ch -= nch;
                    ++po;
                }
            }
        }
        __syncthreads();
        // the slot is consumed (input by the horizontal pass, weights by the
        // vertical pass): refill it with block k + NI
        if (tid == 0 && k + NI < nblk) issue(k + NI);
    }
    // On a timeout, let the copies still in flight (blocks k .. k + NI - 1)
    // land (bounded) before the CTA's shared memory is released.
    if (k < nblk && tid == 0) {
        for (int b = k; b < nblk && b < k + NI; ++b) fused::mbar_wait_bounded(&full[b % NI], uint32_t((b / NI) & 1));
    }
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

__device__ __forceinline__ int multi_image(const Multi &m, int b)
{
    int lo = 0, hi = m.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(m.cta_off + mid) <= b)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

template <typename T, int C, int JV, int GV>
__global__ void __launch_bounds__(kThreads, 2) stream_kernel(const __grid_constant__ CUtensorMap tmap, const Params p)
{
    stream_cta<T, C, JV, GV>(&tmap, p, int(blockIdx.x));
}

template <typename T, int C, int JV, int GV>
__global__ void __launch_bounds__(kThreads, 2) stream_multi_kernel(const __grid_constant__ Multi m)
{
    const int b = int(blockIdx.x), i = multi_image(m, b);
    const Params p = m.ps[i];
    stream_cta<T, C, JV, GV>(m.maps + i, p, b - __ldg(m.cta_off + i));
}

// ---------------------------------------------------------------------------
// Warp-specialised variant: the first HW warps run the horizontal pass on
// block k while the others run the vertical pass on block k - 1 (or earlier),
// so the two phases overlap instead of alternating between block barriers
// (HW follows the two passes' work per block).  The input
// blocks and the vertical weights live in separate rings, each refilled by
// its own consumer; the filtered-row ring holds two blocks plus a band.
//   hdone[k & 1]: the horizontal warps finished block k (its rows are in the ring)
//   vdone[k & 1]: the vertical warps finished block k (the ring slots of its
//                 rows may be overwritten by block k + 2)

struct LayoutWS {
    size_t in_blk, in_ring, wv, vb, wslot, w_ring, hring, hb, cb, pe, total;
};

__host__ __device__ inline LayoutWS layout_ws(int NI, int NW, int P, int Q, int nch, int ngx, int JH, int WP, int JV,
                                              bool two_boxes, int GV, int es)
{
    LayoutWS L;
    L.in_blk = size_t(kRB) * P * es * (two_boxes ? 2 : 1);
    L.in_ring = size_t(NI) * L.in_blk; // in_blk is a multiple of 128 bytes
    L.wv = size_t(WP) * JV * vtap_floats(GV) * 4;
    L.vb = fused::align_up(size_t(WP + 8) * 4, 16);
    L.wslot = fused::align_up(L.wv + L.vb, 128);
    L.w_ring = size_t(NW) * L.wslot;
    L.hring = fused::align_up(size_t(nch) * Q * 16, 128);
    L.hb = fused::align_up(size_t(ngx) * JH * kG * 4, 128);
    L.cb = fused::align_up(size_t(ngx) * 4, 128);
    L.pe = fused::align_up(size_t(kMaxBlk) * 4, 128);
    L.total = 128 + L.in_ring + L.w_ring + L.hring + L.hb + L.cb + L.pe + 128;
    return L;
}

// bar.red.and over a named barrier: every participating thread gets the AND.
__device__ __forceinline__ bool group_and(int id, int threads, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.and.pred po, %2, %3, pi;\n\tselp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"(v ? 1u : 0u), "r"(id), "r"(threads)
        : "memory");
    return r != 0;
}

// The work of one CTA of the warp-specialised band kernel.
template <typename T, int C, int JV, int GV>
__device__ __forceinline__ void stream_ws_cta(const CUtensorMap *tmap_ptr, const Params &p, int bid)
{
    const CUtensorMap &tmap = *tmap_ptr;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (fused::smem_addr(smem_raw) & 127u)) & 127u);
    const int ngx = p.SW / kG;
    const int JH = p.JH, P = p.P, Q = p.Q, HR = p.HR, M = p.M, NI = p.NI, NW = p.NW, WP = p.WP;
    const int nch = (p.SW * C) / 4;
    const LayoutWS L = layout_ws(NI, NW, P, Q, nch, ngx, JH, WP, JV, p.offB != 0, GV, int(sizeof(T)));
    unsigned char *in_ring = smem;
    unsigned char *w_ring = smem + L.in_ring;
    float4 *hring = reinterpret_cast<float4 *>(w_ring + L.w_ring);
    float *hb = reinterpret_cast<float *>(w_ring + L.w_ring + L.hring);
    int32_t *cb = reinterpret_cast<int32_t *>(w_ring + L.w_ring + L.hring + L.hb);
    int32_t *pe_s = reinterpret_cast<int32_t *>(w_ring + L.w_ring + L.hring + L.hb + L.cb);
    uint64_t *bars = reinterpret_cast<uint64_t *>(w_ring + L.w_ring + L.hring + L.hb + L.cb + L.pe);
    uint64_t *full_in = bars, *full_w = bars + kMaxNI, *hdone = bars + 2 * kMaxNI, *vdone = hdone + 2;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(vdone + 2);
    auto slot_in = [&](int s) { return reinterpret_cast<T *>(in_ring + s * L.in_blk); };
    auto slot_wv = [&](int s) { return reinterpret_cast<const float4 *>(w_ring + s * L.wslot); };
    auto slot_vb = [&](int s) { return reinterpret_cast<const int32_t *>(w_ring + s * L.wslot + L.wv); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kHWarps = p.HW, kHThreads = 32 * p.HW, kVThreads = kThreads - kHThreads;
    const int strip = bid % p.n_strips, range = bid / p.n_strips;
    const int p0 = range * p.pairs_per_range;
    const int p1 = min(p.pairs, p0 + p.pairs_per_range);
    if (p0 >= p1) return;
    const int g0 = strip * ngx;
    const int ngv = min(ngx, p.groups_x - g0);
    const int xs = first_staged<T>(__ldg(p.hbase + g0) * C);
    const int r_lo = __ldg(p.vbase + p0);
    const int r_hi = __ldg(p.vbase + p1 - 1) + JV;
    const int nblk = min((r_hi - r_lo + kRB - 1) / kRB, kMaxBlk);

    if (tid == 0) {
        for (int s = 0; s < NI; ++s) fused::mbar_init(&full_in[s], 1);
        for (int s = 0; s < NW; ++s) fused::mbar_init(&full_w[s], 1);
        for (int b = 0; b < 2; ++b) {
            fused::mbar_init(&hdone[b], kHThreads);
            fused::mbar_init(&vdone[b], kVThreads);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < ngx * JH * kG; e += kThreads) {
        const int q = e / (JH * kG);
        hb[e] = q < ngv ? __ldg(p.hband + size_t(g0) * JH * kG + e) : 0.f;
    }
    for (int q = tid; q < ngx; q += kThreads) {
        int o = q < ngv ? __ldg(p.hbase + g0 + q) * C - xs : 0;
        if (p.offB && o + JH * C > P) o += kRB * P - p.offB;
        cb[q] = o;
    }
    auto kb = [&](int vb) {
        const int k = (vb + JV - r_lo + kRB - 1) / kRB - 1;
        return k < 0 ? 0 : (k > nblk - 1 ? nblk - 1 : k);
    };
    for (int q = p0 + tid; q < p1; q += kThreads) {
        const int kp = kb(__ldg(p.vbase + q));
        const int kn = q + 1 < p1 ? kb(__ldg(p.vbase + q + 1)) : nblk;
        for (int k = kp; k < kn; ++k) pe_s[k] = q + 1;
        if (q == p0)
            for (int k = 0; k < kp; ++k) pe_s[k] = p0;
    }
    __syncthreads();

    const uint32_t blk_bytes = uint32_t(L.in_blk);
    auto issue_in = [&](int k) { // input block k (first horizontal thread)
        const int s = k % NI;
        fused::mbar_arrive_expect_tx(&full_in[s], blk_bytes);
        fused::tma_load_2d(slot_in(s), &tmap, &full_in[s], xs, r_lo + k * kRB);
        if (p.offB) fused::tma_load_2d(slot_in(s) + kRB * P, &tmap, &full_in[s], xs + p.offB, r_lo + k * kRB);
    };
    auto issue_w = [&](int k) { // weights and bases of block k's groups (first vertical thread)
        const int s = k % NW;
        const int ps = k ? pe_s[k - 1] : p0, pe = pe_s[k];
        int n = pe - ps;
        if (n > WP) {
            fused::flag(p.err, fused::kErrBounds);
            n = 0;
        }
        const int pa = ps & ~3, pb = (pe + 3) & ~3;
        const uint32_t wbytes = uint32_t(n) * JV * vtap_floats(GV) * 4, vbytes = n ? uint32_t(pb - pa) * 4 : 0u;
        fused::mbar_arrive_expect_tx(&full_w[s], wbytes + vbytes);
        if (n) {
            fused::bulk_load(const_cast<float4 *>(slot_wv(s)), p.vband + size_t(ps) * JV * vtap_floats(GV), wbytes,
                             &full_w[s]);
            fused::bulk_load(const_cast<int32_t *>(slot_vb(s)), p.vbase + pa, vbytes, &full_w[s]);
        }
    };

    int k = 0;
    bool ok = true;
    if (warp < kHWarps) {
        // ================ horizontal pass: block k into the ring ================
        if (tid == 0)
            for (int b = 0; b < NI && b < nblk; ++b) issue_in(b);
        for (; k < nblk; ++k) {
            const int slot = k % NI;
            bool good = fused::wait_or_abort(&full_in[slot], uint32_t((k / NI) & 1), abort_flag, p.err);
            // the ring slots of block k's rows held block k - 2's rows
            if (good && k >= 2) good = fused::wait_or_abort(&vdone[k & 1], uint32_t(((k - 2) >> 1) & 1), abort_flag, p.err);
            if (!group_and(1, kHThreads, good)) {
                ok = false;
                break;
            }
            const int base_k = (k * kRB) % HR;
            int hs = base_k + lane;
            if (hs >= HR) hs -= HR;
            const T *rowp = slot_in(slot) + size_t(lane) * P;
            for (int q = warp; q < ngv; q += kHWarps)
                h_group<T, C>(rowp, cb[q], hb + q * JH * kG, JH, hring, q, Q, HR, M, hs);
            fused::named_sync(1, kHThreads); // the staged block is consumed
            if (tid == 0 && k + NI < nblk) issue_in(k + NI);
            fused::mbar_arrive(&hdone[k & 1]);
        }
    } else {
        // ================ vertical pass: the groups block k completes ================
        const int vt = tid - kHThreads;
        if (vt == 0)
            for (int b = 0; b < NW && b < nblk; ++b) issue_w(b);
        const int64_t row_samples = p.out_w * C;
        const int64_t x0s = int64_t(strip) * p.SW * C;
        const bool vec_ok =
            ((reinterpret_cast<uintptr_t>(p.out) | uintptr_t(p.out_stride * sizeof(T))) & (4 * sizeof(T) - 1)) == 0;
        for (; k < nblk; ++k) {
            const int wslot = k % NW;
            bool good = fused::wait_or_abort(&full_w[wslot], uint32_t((k / NW) & 1), abort_flag, p.err);
            if (good) good = fused::wait_or_abort(&hdone[k & 1], uint32_t((k >> 1) & 1), abort_flag, p.err);
            if (!group_and(2, kVThreads, good)) {
                ok = false;
                break;
            }
            const int base_k = (k * kRB) % HR;
            const int ps = k ? pe_s[k - 1] : p0, pe = pe_s[k];
            const int n = pe - ps <= WP ? pe - ps : 0;
            const float4 *wvs = slot_wv(wslot);
            const int32_t *vbs = slot_vb(wslot) - (ps & ~3);
            const int ntask = n * nch;
            int po = vt / nch, ch = vt - (vt / nch) * nch;
            const int dpo = kVThreads / nch, dch = kVThreads - dpo * nch;
            for (int t = vt; t < ntask; t += kVThreads) {
                const int pr = ps + po;
                int hs0 = base_k + (vbs[pr] - r_lo - k * kRB);
                if (hs0 < 0) hs0 += HR;
                if (hs0 >= HR) hs0 -= HR;
                v_task<T, JV, GV>(hring + ch * Q + hs0, wvs + po * JV * (vtap_floats(GV) / 4), static_cast<T *>(p.out),
                                  p.out_stride,
                               int64_t(GV) * pr, p.out_h, x0s + int64_t(ch) * 4, row_samples, vec_ok);
                po += dpo;
                ch += dch;
                if (ch >= nch) {
                    ch -= nch;
                    ++po;
                }
            }
            fused::named_sync(2, kVThreads); // the weights slot is consumed
            if (vt == 0 && k + NW < nblk) issue_w(k + NW);
            fused::mbar_arrive(&vdone[k & 1]);
        }
    }
    // On a timeout, let the copies still in flight land (bounded) before the
    // CTA's shared memory is released.
    if (!ok) {
        if (tid == 0)
            for (int b = k; b < nblk && b < k + NI; ++b) fused::mbar_wait_bounded(&full_in[b % NI], uint32_t((b / NI) & 1));
        if (tid == kHThreads)
            for (int b = k; b < nblk && b < k + NW; ++b) fused::mbar_wait_bounded(&full_w[b % NW], uint32_t((b / NW) & 1));
    }
}

template <typename T, int C, int JV, int GV>
__global__ void __launch_bounds__(kThreads, 2) stream_ws_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                  const Params p)
{
    stream_ws_cta<T, C, JV, GV>(&tmap, p, int(blockIdx.x));
}

template <typename T, int C, int JV, int GV>
__global__ void __launch_bounds__(kThreads, 2) stream_ws_multi_kernel(const __grid_constant__ Multi m)
{
    const int b = int(blockIdx.x), i = multi_image(m, b);
    const Params p = m.ps[i];
    stream_ws_cta<T, C, JV, GV>(m.maps + i, p, b - __ldg(m.cta_off + i));
}

// ---------------------------------------------------------------------------
// Instantiated kernels: storage type x channels x vertical taps x rows per
// vertical group (a plan's band is padded with zero weights to the next
// instantiated width): groups of 8 rows up to 16 taps, groups of 4 up to 32.
// One translation unit per storage type instantiates its table.

template <typename T, int C, int JV, int GV> const void *kernel_of(bool ws, bool multi)
{
    if (multi)
        return ws ? reinterpret_cast<const void *>(&stream_ws_multi_kernel<T, C, JV, GV>)
                  : reinterpret_cast<const void *>(&stream_multi_kernel<T, C, JV, GV>);
    return ws ? reinterpret_cast<const void *>(&stream_ws_kernel<T, C, JV, GV>)
              : reinterpret_cast<const void *>(&stream_kernel<T, C, JV, GV>);
}

template <typename T, int C, int GV> const void *kernel_jv(int jv, bool ws, bool multi)
{
    switch (jv) {
    case 4: return GV == 4 ? kernel_of<T, C, 4, 4>(ws, multi) : nullptr;
    case 6: return GV == 4 ? kernel_of<T, C, 6, 4>(ws, multi) : nullptr;
    case 8: return kernel_of<T, C, 8, GV>(ws, multi);
    case 10: return kernel_of<T, C, 10, GV>(ws, multi);
    case 12: return kernel_of<T, C, 12, GV>(ws, multi);
    case 14: return kernel_of<T, C, 14, GV>(ws, multi);
    case 16: return kernel_of<T, C, 16, GV>(ws, multi);
    case 20: return GV == 4 ? kernel_of<T, C, 20, 4>(ws, multi) : nullptr;
    case 24: return GV == 4 ? kernel_of<T, C, 24, 4>(ws, multi) : nullptr;
    case 28: return GV == 4 ? kernel_of<T, C, 28, 4>(ws, multi) : nullptr;
    case 32: return GV == 4 ? kernel_of<T, C, 32, 4>(ws, multi) : nullptr;
    }
    return nullptr;
}

template <typename T> const void *kernel_table(int C, int jv, int gv, bool ws, bool multi)
{
    if (C == 1) return gv == 8 ? kernel_jv<T, 1, 8>(jv, ws, multi) : kernel_jv<T, 1, 4>(jv, ws, multi);
    if (C == 3) return gv == 8 ? kernel_jv<T, 3, 8>(jv, ws, multi) : kernel_jv<T, 3, 4>(jv, ws, multi);
    return nullptr;
}

// defined in rs_stream_f32.cu, rs_stream_f16.cu, rs_stream_bf16.cu
const void *kernel_f32(int C, int jv, int gv, bool ws, bool multi = false);
const void *kernel_f16(int C, int jv, int gv, bool ws, bool multi = false);
const void *kernel_bf16(int C, int jv, int gv, bool ws, bool multi = false);

} // namespace stream
} // namespace rs
