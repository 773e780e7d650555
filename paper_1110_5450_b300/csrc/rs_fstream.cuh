// rs_fstream.cuh -- streaming downscale for FP32 storage (streaming form 4).
//
// The pipeline of the tensor-core streaming downscale (rs_tcstream.cuh) with
// the horizontal pass on SIMT warps, since FP16 / BF16 tensor-core operands
// would not hold FP32 data:
//
//  * strips of 48 output samples (48 / C pixels), one CTA per SM on a
//    contiguous run of (strip, row group) positions;
//  * warp 0, the producer: TMA copies of 32-row blocks of the strip's staged
//    input (P samples from a multiple of 4, one box per block) into a ring of
//    NA stages;
//  * HW horizontal warps: the strip's groups of 4 output pixels, one task per
//    (staged block, group): lane = input row, the lane's row read in 16-byte
//    words along the group's band of JH pixels from a 4-pixel aligned base
//    (4 weights per pixel, one per output, warp-uniform, from the plan's band
//    table), 4 C sums per lane (packed FP32 FMAs, two outputs per
//    instruction), written as C 16-byte words into a ring of NS blocks of 128
//    filtered rows;
//  * VW vertical warps: tcstream::v_role, row groups of 4 output rows over the
//    union of their windows, straight into the output.
//
// Summation order per output sample: the horizontal band taps in increasing
// input order, then the vertical band taps in increasing input row order
// (FP32 FMAs; a band's zero weights add exact zeros).  Every wait is bounded
// (2 s); a timeout sets the plan's error word and every role stops, the
// producer letting its copies in flight land.
#pragma once

#include "rs_tcstream.cuh"

namespace rs {
namespace fstream {

using tcstream::kM;
using tcstream::kMaxNS;
using tcstream::kMaxVW;
using tcstream::kN;

constexpr int kHP = kN + 4;      // filtered-row pitch in floats (16-byte words; 13 words, odd)
constexpr int kSB = 32;          // input rows per staged block (one per lane)
constexpr int kSubs = kM / kSB;  // staged blocks per ring block
constexpr int kMaxNA = 6;        // staged blocks at most
constexpr int kMaxHW = 12;       // horizontal warps at most
constexpr int kMaxWarps = 19;    // producer + horizontal + vertical warps at most
constexpr int kMaxP = 256;       // staged samples per row at most (one TMA box)
constexpr int kMaxJH = 64;       // band pixels per group at most

struct Params {
    void *out;
    int32_t in_h, out_h, out_w, C;
    int64_t out_stride;         // elements
    const int32_t *sy;          // [out_h] vertical window starts (the plan's table)
    const float4 *vband;        // [gpr][Uv] per row group: its 4 rows' weights at each union row
    const int2 *vinfo;          // [gpr] per row group: first union row, union rows
    int32_t NP;                 // output pixels per strip (kN / C)
    int32_t n_strips;
    int32_t Ty;
    int32_t Uv;                 // union rows of a row group at most (<= tcstream::kMaxTy)
    int32_t gpr;                // row groups per strip: ceil(out_h / 4)
    int32_t NS;                 // blocks in the filtered-row ring (2 or 3)
    int32_t NA, VW, HW;
    int64_t per_cta;            // (strip, row group) positions per CTA
    int *err;
    const int32_t *xs;          // [n_strips] first staged sample (a multiple of 4)
    const int32_t *hoff;        // [n_strips][ngx] group band's first sample in the staged row (a multiple of 4)
    const float4 *hband;        // [n_strips][ngx][JH] the group's 4 weights at each band pixel
    int32_t P;                  // staged samples per row (the row pitch, a multiple of 4)
    int32_t JH;                 // band pixels per group (a multiple of 4)
    int32_t ngx;                // groups of 4 output pixels per strip (NP / 4)
};

struct Layout {
    size_t stage, a, h, w, bar, total;
};

__host__ __device__ inline Layout layout(int P, int NA, int Uv, int VW, int NS)
{
    Layout L;
    L.stage = size_t(kSB) * P * 4; // a multiple of 128 bytes (P a multiple of 4)
    L.a = size_t(NA) * L.stage;
    L.h = size_t(NS) * kM * kHP * 4;
    L.w = size_t(VW) * 2 * Uv * 16;
    L.bar = 512;
    L.total = L.a + L.h + L.w + L.bar + 128;
    return L;
}

// Horizontal pass of one group of 4 output pixels for the lane's staged row:
// row = the row in the stage, off = the group band's first sample in it,
// wq = the band (4 weights per pixel, warp-uniform), dst = the lane's ring row
// at the group's first column.
template <int C>
__device__ __forceinline__ void h_task(const float *row, int off, const float4 *wq, int JH, float *dst)
{
    const float *src = row + off;
    uint64_t acc2[2][C]; // outputs (0, 1) and (2, 3) of each channel as packed pairs
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int c = 0; c < C; ++c) acc2[h][c] = 0ull;
    for (int t0 = 0; t0 < JH; t0 += 4) {
        // 4 input pixels of this lane's row (C 16-byte words) ...
        float d[4 * C];
#pragma unroll
        for (int v = 0; v < C; ++v) {
            const float4 x = *reinterpret_cast<const float4 *>(src + 4 * v);
            d[4 * v] = x.x;
            d[4 * v + 1] = x.y;
            d[4 * v + 2] = x.z;
            d[4 * v + 3] = x.w;
        }
        src += 4 * C;
        // ... times the 4 outputs' weights at those pixels
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const ulonglong2 w = __ldg(reinterpret_cast<const ulonglong2 *>(wq + t));
#pragma unroll
            for (int c = 0; c < C; ++c) {
                uint64_t xx;
                asm("mov.b64 %0, {%1, %1};" : "=l"(xx) : "f"(d[t * C + c]));
                acc2[0][c] = fused::fma2(w.x, xx, acc2[0][c]);
                acc2[1][c] = fused::fma2(w.y, xx, acc2[1][c]);
            }
        }
        wq += 4;
    }
    // the group's 4 x C filtered samples, pixel-major as in the output
    float o[4 * C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        fused::unpack2(acc2[0][c], o[0 * C + c], o[1 * C + c]);
        fused::unpack2(acc2[1][c], o[2 * C + c], o[3 * C + c]);
    }
#pragma unroll
    for (int v = 0; v < C; ++v)
        *reinterpret_cast<float4 *>(dst + 4 * v) = make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
}

template <int C>
__global__ void __launch_bounds__(32 * kMaxWarps, 1)
    fstream_kernel(const __grid_constant__ CUtensorMap tmap, const Params p)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (fused::smem_addr(smem_raw) & 127u)) & 127u);
    const int P = p.P, NA = p.NA, VW = p.VW, HW = p.HW, NS = p.NS, Ty = p.Ty, ngx = p.ngx, JH = p.JH;
    const Layout L = layout(P, NA, p.Uv, VW, NS);
    float *stages = reinterpret_cast<float *>(smem);
    float *hring = reinterpret_cast<float *>(smem + L.a);
    float *wsm = reinterpret_cast<float *>(smem + L.a + L.h);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.a + L.h + L.w);
    uint64_t *full_s = bars, *empty_s = bars + kMaxNA;
    uint64_t *hfull = bars + 2 * kMaxNA;   // [kMaxNS]
    uint64_t *hfree = hfull + kMaxNS;      // [kMaxNS][kMaxVW]
    volatile int *abort_flag = reinterpret_cast<volatile int *>(hfree + kMaxNS * kMaxVW);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t total = int64_t(p.n_strips) * p.gpr;
    const int64_t pos0 = min(total, int64_t(blockIdx.x) * p.per_cta);
    const int64_t pos1 = min(total, pos0 + p.per_cta);
    const size_t stage_f = L.stage / 4; // floats per stage

    if (tid == 0) {
        for (int s = 0; s < kMaxNA; ++s) {
            fused::mbar_init(&full_s[s], 1);
            fused::mbar_init(&empty_s[s], uint32_t(ngx)); // one arrival per group task of the block
        }
        for (int s = 0; s < kMaxNS; ++s) {
            fused::mbar_init(&hfull[s], uint32_t(kSubs * ngx));
            for (int v = 0; v < kMaxVW; ++v) fused::mbar_init(&hfree[s * kMaxVW + v], 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto item_rows = [&](const tcstream::Item &it, int &r0, int &nblk) {
        r0 = __ldg(p.sy + it.i0);
        const int r_end = __ldg(p.sy + it.i1 - 1) + Ty;
        nblk = (r_end - r0 + kM - 1) / kM;
    };

    if (warp == 0) {
        // ================= producer: staged blocks of the strip's input =================
        if (lane == 0) {
            int64_t pos = pos0;
            int q = 0, s = 0; // staged blocks issued; q % NA kept by increments
            uint32_t rnd = 0; // q / NA
            const uint32_t stage_bytes = uint32_t(L.stage);
            bool ok = true;
            tcstream::Item it;
            while (ok && tcstream::next_item(pos, pos1, p.gpr, p.out_h, it)) {
                int r0, nblk;
                item_rows(it, r0, nblk);
                const int xs = __ldg(p.xs + it.strip);
                for (int b = 0; b < nblk && ok; ++b)
                    for (int sb = 0; sb < kSubs; ++sb) {
                        if (rnd > 0 && !fused::wait_or_abort(&empty_s[s], (rnd - 1) & 1u, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        fused::mbar_arrive_expect_tx(&full_s[s], stage_bytes);
                        fused::tma_load_2d(stages + size_t(s) * stage_f, &tmap, &full_s[s], xs, r0 + b * kM + sb * kSB);
                        ++q;
                        if (++s == NA) {
                            s = 0;
                            ++rnd;
                        }
                    }
            }
            if (!ok)
                for (int k = q - NA > 0 ? q - NA : 0; k < q; ++k)
                    fused::mbar_wait_bounded(&full_s[k % NA], uint32_t((k / NA) & 1));
        }
    } else if (warp <= HW) {
        // ================= horizontal pass: (staged block, group) tasks =================
        // One task stream for the CTA's whole run: staged block Q (counted over
        // all items; ring block Q / 4), group q; task Q ngx + q.  Warp hw takes
        // tasks hw, hw + HW, ..., so its next task is at most ceil(HW / ngx) <=
        // NA staged blocks ahead of its last one (the set-up checks it): the
        // stage it waits for is then at most one round ahead, which the
        // mbarrier parity tells apart.  Each task's warp arrives once on its
        // block's stage (ngx arrivals free it) and once on its ring block
        // (kSubs ngx arrivals fill it).
        const int hw = warp - 1;
        int64_t pos = pos0;
        int qs0 = 0;             // first staged block of the current item
        int Qg = 0, q = hw;      // this warp's task
        int s = 0, sl = 0;       // Qg % NA, (Qg / 4) % NS, kept by increments
        uint32_t rnd = 0, grnd = 0; // Qg / NA, (Qg / 4) / NS
        auto next_block = [&]() {
            ++Qg;
            if (++s == NA) {
                s = 0;
                ++rnd;
            }
            if ((Qg & 3) == 0 && ++sl == NS) {
                sl = 0;
                ++grnd;
            }
        };
        while (q >= ngx) {
            q -= ngx;
            next_block();
        }
        int freed = -1; // the last ring block this warp saw released
        bool ok = true;
        tcstream::Item it;
        while (ok && tcstream::next_item(pos, pos1, p.gpr, p.out_h, it)) {
            int r0, nblk;
            item_rows(it, r0, nblk);
            const int32_t *ho = p.hoff + size_t(it.strip) * ngx;
            const float4 *hb = p.hband + size_t(it.strip) * ngx * JH;
            const int qs1 = qs0 + nblk * kSubs;
            while (Qg < qs1 && ok) {
                const int G = Qg >> 2, sb = Qg & 3;
                // the ring block's previous rows are read by every vertical warp
                if (G != freed) {
                    if (grnd > 0)
                        for (int v = 0; v < VW && ok; ++v)
                            ok = tcstream::warp_wait(&hfree[sl * kMaxVW + v], (grnd - 1) & 1u, abort_flag, p.err);
                    freed = G;
                }
                if (ok) ok = tcstream::warp_wait(&full_s[s], rnd & 1u, abort_flag, p.err);
                if (!ok) break;
                h_task<C>(stages + size_t(s) * stage_f + size_t(lane) * P, __ldg(ho + q), hb + size_t(q) * JH, JH,
                          hring + size_t(sl * kM + sb * kSB + lane) * kHP + q * 4 * C);
                __syncwarp();
                if (lane == 0) {
                    fused::mbar_arrive(&empty_s[s]);
                    fused::mbar_arrive(&hfull[sl]);
                }
                for (q += HW; q >= ngx;) {
                    q -= ngx;
                    next_block();
                }
            }
            qs0 = qs1;
        }
    } else if (warp <= HW + VW) {
        tcstream::v_role<float, C, kHP>(p, hring, wsm, hfull, hfree, abort_flag, warp - 1 - HW, lane, pos0, pos1);
    }
    __syncthreads();
}

} // namespace fstream
} // namespace rs
