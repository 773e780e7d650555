// rs_tcstream.cuh -- streaming downscale with the horizontal pass on the
// fifth-generation tensor cores (streaming form 3; FP16 / BF16 storage).
//
// A downscale's first (horizontal) pass is the bulk of the arithmetic: every
// input row is filtered for every output column, T taps each (T = 2 R / s for
// an antialiased kernel of radius R at scale s, 20 for Lanczos-3 at x0.3).
// Here it is a dense GEMM per strip of output columns:
//
//     D[row][n] = sum_k In[row][k] B[k][n]
//
// for 128 input rows at a time (the tensor-memory lanes), where n runs over
// the strip's kN = 48 output samples (48 / C pixels, channels interleaved as
// in the output) and k over the Kc input samples the strip's windows cover
// (from a multiple of 8).  B is the strip's block of the horizontal filter
// matrix, B[k][n] = the window weight of output pixel n / C at input pixel
// (8 g0 + k) / C when that sample has channel n % C, else 0.  It is the same
// for every row, so a CTA loads it once per strip and keeps it in shared
// memory; it is stored as a high and a low 16-bit part (w = hi + lo to about
// 2^-16 relative), each multiplied in, so weight rounding costs no accuracy.
// The zeros cost tensor-core work only (Kc x 48 products for 48 T useful
// ones), which the tensor cores have to spare at these densities; the SIMT
// alternative spends its FMA issue on the same pass.
//
// Roles (one CTA per SM):
//  * warp 0, the producer: TMA copies of the input in chunks of 128 rows x 64
//    samples (128-byte rows, which the copy lands in the 128-byte swizzled
//    K-major operand layout) into a ring of NA stages, and the strip's B (one
//    bulk copy);
//  * warps 1 and 2: tensor-memory allocation (warp 1); one thread of each
//    issues the MMAs of the even or the odd K steps (M = 128, N = 96 -- the
//    hi and the lo weight parts side by side --, K = 16 per instruction) into
//    its accumulator, two sets alternating between blocks of rows, and commits
//    them to the mbarriers that free the staged chunk and hand the
//    accumulators on;
//  * warps 3-6: read the accumulators back (each warp its quarter of the 128
//    lanes), add a block's partial sums, into a ring of two blocks of
//    filtered rows (FP32);
//  * VW warps: the vertical pass, in groups of 4 output rows over the union
//    of their windows, FP32 FMAs with the group's band of weights (from a
//    per-plan table, copied into shared memory two groups ahead), straight
//    into the output.
// A CTA takes a contiguous run of (strip, row group) positions, so it changes
// strip at most a few times and its input rows run on without a halo except
// at the ends of the run.  Every wait is bounded (2 s): a timeout sets the
// plan's error word and every role stops; the producer lets its copies in
// flight land, and the MMA thread's outstanding MMAs complete before the
// tensor memory is released.
//
// Summation order per output sample: the horizontal sum as four partial sums
// in the tensor cores (the hi and lo weight parts of the even and of the odd
// K steps, each in FP32 accumulator columns), added as (hi + lo) + (hi + lo);
// then the vertical taps in increasing input row
// order (FP32 FMAs; the zero weights of a band add exact zeros).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_fused.cuh"
#include "rs_tc.cuh"

namespace rs {
namespace tcstream {

constexpr int kN = 48;               // output samples of a strip (accumulator columns)
constexpr int kM = 128;              // input rows per block (tensor-memory lanes)
constexpr int kKC = 64;              // input samples per staged chunk
constexpr int kMaxNA = 6;            // staged chunks at most
constexpr int kMaxNS = 3;            // blocks in the filtered-row ring at most (2 or 3)
constexpr int kHP = kN + 2;          // filtered-row pitch in floats (8-byte pairs; 18 banks apart)
constexpr int kMaxVW = 10;           // vertical warps at most
constexpr int kFixedWarps = 7;       // producer, 2 MMA issuers, 4 read-back warps
constexpr int kChains = 2;           // accumulators per block: the even and the odd K steps
constexpr uint32_t kTmemCols = 512;  // two blocks x kChains accumulators of 2 kN columns, to a power of two
constexpr int kMaxTy = 128;          // vertical taps at most (a window spans at most two blocks)

struct Params {
    void *out;
    int32_t in_h, out_h, out_w, C;
    int64_t out_stride;         // elements
    const unsigned char *bmat;  // per strip: B hi then B lo, [kN][Kc] in the canonical K-major layout
    const int32_t *g0;          // per strip: its first staged 8-sample group
    const int32_t *sy;          // [out_h] vertical window starts (the plan's table)
    const float4 *vband;        // [gpr][Uv] per row group: its 4 rows' weights at each union row
    const int2 *vinfo;          // [gpr] per row group: first union row, union rows
    int32_t Kc;                 // staged samples per row, a multiple of kKC
    int32_t NP;                 // output pixels per strip (kN / C)
    int32_t n_strips;
    int32_t Ty;
    int32_t Uv;                 // union rows of a row group at most (<= kMaxTy)
    int32_t gpr;                // row groups per strip: ceil(out_h / kVG)
    int32_t NS;                 // blocks in the filtered-row ring (2 or 3)
    int32_t NA, VW;
    int32_t pf;                 // chunks ahead of the copy in flight to prefetch into L2 (0: none)
    int64_t per_cta;            // (strip, row group) positions per CTA
    int *err;
};

struct Layout {
    size_t b, a, h, w, bar, total;
};

__host__ __device__ inline size_t b_bytes(int Kc) { return size_t(kN) * size_t(Kc) * 2; } // one part

constexpr int kVG = 4; // output rows a vertical warp takes at once (one band)

// Uv: the rows a band spans at most (kVG consecutive windows), VW: the vertical warps
__host__ __device__ inline Layout layout(int Kc, int NA, int Uv, int VW, int NS)
{
    Layout L;
    L.b = 2 * b_bytes(Kc);
    L.a = size_t(NA) * kM * kKC * 2;
    L.h = size_t(NS) * kM * kHP * 4;
    L.w = size_t(VW) * 2 * Uv * 16; // per vertical warp two bands of Uv rows x kVG weights
    L.bar = 512;
    L.total = L.b + L.a + L.h + L.w + L.bar + 1024; // + alignment of the dynamic shared memory
    return L;
}

// Every lane of a warp waits; true only if all saw the phase.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err)
{
    const bool ok = fused::wait_or_abort(bar, parity, abort_flag, err);
    return __all_sync(0xffffffffu, ok);
}

// The positions [pos0, pos1) of a CTA, (strip, row group of kVG output rows)
// pairs, as items (strip, first output row, end): a run of whole row groups.
struct Item {
    int strip, i0, i1;
};
__device__ __forceinline__ bool next_item(int64_t &pos, int64_t pos1, int gpr, int out_h, Item &it)
{
    if (pos >= pos1) return false;
    it.strip = int(pos / gpr);
    const int q0 = int(pos - int64_t(it.strip) * gpr);
    const int64_t rest = pos1 - pos;
    const int q1 = rest < int64_t(gpr - q0) ? q0 + int(rest) : gpr;
    it.i0 = q0 * kVG;
    it.i1 = min(out_h, q1 * kVG);
    pos += q1 - q0;
    return true;
}

template <typename T, int C>
__global__ void __launch_bounds__(32 * (kFixedWarps + kMaxVW), 1)
    tcstream_kernel(const __grid_constant__ CUtensorMap tmap, const Params p)
{
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned: the staged chunks carry the 128-byte swizzle, whose
    // pattern repeats every 8 rows of 128 bytes
    unsigned char *smem = smem_raw + ((1024u - (fused::smem_addr(smem_raw) & 1023u)) & 1023u);
    const int Kc = p.Kc, NA = p.NA, VW = p.VW, Ty = p.Ty;
    const int NS = p.NS;
    const Layout L = layout(Kc, NA, p.Uv, VW, NS);
    unsigned char *bsm = smem;                 // B hi, then B lo
    unsigned char *asm_ = smem + L.b;          // NA staged chunks
    float *hring = reinterpret_cast<float *>(asm_ + L.a);
    float *wsm = reinterpret_cast<float *>(asm_ + L.a + L.h);
    uint64_t *bars = reinterpret_cast<uint64_t *>(asm_ + L.a + L.h + L.w);
    uint64_t *full_a = bars, *empty_a = bars + kMaxNA;
    uint64_t *bfull = bars + 2 * kMaxNA, *bfree = bfull + 1;
    uint64_t *acc_full = bfree + 1, *acc_empty = acc_full + 2;
    uint64_t *hfull = acc_empty + 2;              // [kMaxNS]
    uint64_t *hfree = hfull + kMaxNS;             // [kMaxNS][kMaxVW], one per vertical warp
    uint64_t *drain = hfree + kMaxNS * kMaxVW;    // [2], one per MMA issuer
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t total = int64_t(p.n_strips) * p.gpr;
    const int64_t pos0 = min(total, int64_t(blockIdx.x) * p.per_cta);
    const int64_t pos1 = min(total, pos0 + p.per_cta);
    const uint32_t chunk_bytes = uint32_t(kM) * kKC * 2;
    const int nchunk = Kc / kKC;
    const size_t bpart = b_bytes(Kc);

    if (tid == 0) {
        // (the two MMA issuers each commit to the stage, accumulator and B barriers)
        for (int s = 0; s < kMaxNA; ++s) {
            fused::mbar_init(&full_a[s], 1);
            fused::mbar_init(&empty_a[s], 2);
        }
        fused::mbar_init(bfull, 1);
        fused::mbar_init(bfree, 2);
        for (int d = 0; d < 2; ++d) {
            fused::mbar_init(&acc_full[d], 2);
            fused::mbar_init(&acc_empty[d], 4);
        }
        for (int s = 0; s < kMaxNS; ++s) {
            fused::mbar_init(&hfull[s], 4);
            for (int v = 0; v < kMaxVW; ++v) fused::mbar_init(&hfree[s * kMaxVW + v], 1);
        }
        fused::mbar_init(&drain[0], 1);
        fused::mbar_init(&drain[1], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, kTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    // rows [r0, r_end) of an item's windows, and its blocks of kM rows
    auto item_rows = [&](const Item &it, int &r0, int &nblk) {
        r0 = __ldg(p.sy + it.i0);
        const int r_end = __ldg(p.sy + it.i1 - 1) + Ty;
        nblk = (r_end - r0 + kM - 1) / kM;
    };

    if (warp == 0) {
        // ================= producer: B per strip, input chunks =================
        if (lane == 0) {
            int64_t pos = pos0, q = 0;
            int cur = -1, nload = 0;
            int s = 0;        // q % NA, kept by increments (no division per chunk)
            uint32_t rnd = 0; // q / NA
            bool ok = true;
            Item it;
            while (ok && next_item(pos, pos1, p.gpr, p.out_h, it)) {
                if (it.strip != cur) {
                    if (nload > 0 && !fused::wait_or_abort(bfree, uint32_t((nload - 1) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    fused::mbar_arrive_expect_tx(bfull, uint32_t(2 * bpart));
                    fused::bulk_load(bsm, p.bmat + size_t(it.strip) * 2 * bpart, uint32_t(2 * bpart), bfull);
                    ++nload;
                    cur = it.strip;
                }
                int r0, nblk;
                item_rows(it, r0, nblk);
                const int gz = __ldg(p.g0 + it.strip);
                for (int b = 0; b < nblk && ok; ++b)
                    for (int c = 0; c < nchunk; ++c, ++q) {
                        if (rnd > 0 && !fused::wait_or_abort(&empty_a[s], (rnd - 1) & 1u, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        fused::mbar_arrive_expect_tx(&full_a[s], chunk_bytes);
                        fused::tma_load_2d(asm_ + size_t(s) * chunk_bytes, &tmap, &full_a[s], 8 * gz + c * kKC,
                                           r0 + b * kM);
                        if (p.pf > 0) {
                            // warm L2 for the chunk p.pf copies ahead in this item
                            const int ahead = b * nchunk + c + p.pf;
                            const int pb = ahead / nchunk, pc = ahead - pb * nchunk;
                            if (pb < nblk) fused::tma_prefetch_2d(&tmap, 8 * gz + pc * kKC, r0 + pb * kM);
                        }
                        if (++s == NA) {
                            s = 0;
                            ++rnd;
                        }
                    }
            }
            if (!ok) {
                // let the copies still in flight land (bounded) before the CTA exits
                for (int64_t k = q - NA > 0 ? q - NA : 0; k < q; ++k)
                    fused::mbar_wait_bounded(&full_a[k % NA], uint32_t((k / NA) & 1));
                if (nload) fused::mbar_wait_bounded(bfull, uint32_t((nload - 1) & 1));
            }
        }
    } else if (warp <= 2) {
        // ================= MMA issue: warp 1 the even K steps, warp 2 the odd ones =================
        // Each MMA takes B as one 96-row matrix, the hi part's 48 rows then
        // the lo part's (their layout in shared memory is exactly that), so
        // the staged input is read once for both parts; one thread per warp
        // issues, two warps keep the tensor pipe fed.
        if (lane == 0) {
            const int part = warp - 1;
            const uint32_t idesc = tc::idesc_f16(!std::is_same<T, __half>::value, false, false, kM, 2 * kN);
            const uint32_t a0 = fused::smem_addr(asm_), bw = fused::smem_addr(bsm);
            const uint32_t sbo_b = uint32_t(Kc) * 16u;
            int64_t pos = pos0, gb = 0;
            int cur = -1, nload = 0;
            int s = 0;        // stage of the next chunk, kept by increments
            uint32_t rnd = 0; // times the stage ring went round
            bool ok = true;
            Item it;
            while (ok && next_item(pos, pos1, p.gpr, p.out_h, it)) {
                if (it.strip != cur) {
                    if (!fused::wait_or_abort(bfull, uint32_t(nload & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    ++nload;
                    cur = it.strip;
                }
                int r0, nblk;
                item_rows(it, r0, nblk);
                for (int b = 0; b < nblk && ok; ++b, ++gb) {
                    const int d = int(gb & 1);
                    if (gb >= 2 && !fused::wait_or_abort(&acc_empty[d], uint32_t(((gb >> 1) - 1) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    // this warp's accumulator: columns [0, 48) hi, [48, 96) lo
                    const uint32_t dt = tmem + uint32_t((d * kChains + part) * 2 * kN);
                    for (int c = 0; c < nchunk; ++c) {
                        if (!fused::wait_or_abort(&full_a[s], rnd & 1u, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint32_t as = a0 + uint32_t(s) * chunk_bytes;
#pragma unroll
                        for (int kk = part; kk < kKC / 16; kk += 2) {
                            // A: rows of 128 bytes (64 samples) with the 128-byte swizzle, 8-row
                            // groups 1024 B apart, K advancing 32 B per 16 samples within the row;
                            // B: [8-output group][8-sample group][8][8] without swizzle
                            const uint64_t ad = tc::smem_desc_sw128(as + uint32_t(kk) * 32u, 1024u);
                            const uint32_t koff = uint32_t(c * kKC + kk * 16) * 16u;
                            const uint32_t acc = (c | (kk >> 1)) ? 1u : 0u; // the block's first MMA overwrites
                            tc::mma_f16(dt, ad, tc::smem_desc(bw + koff, 128u, sbo_b), idesc, acc);
                        }
                        tc::mma_commit(&empty_a[s]); // the chunk's stage is free once these are done
                        if (++s == NA) {
                            s = 0;
                            ++rnd;
                        }
                    }
                    if (!ok) break;
                    tc::mma_commit(&acc_full[d]);
                }
                // B stays until the run moves to another strip
                int64_t look = pos;
                Item nx;
                if (ok && next_item(look, pos1, p.gpr, p.out_h, nx) && nx.strip != cur) tc::mma_commit(bfree);
            }
            // every MMA issued has completed before the tensor memory is released
            tc::mma_commit(&drain[part]);
            fused::mbar_wait_bounded(&drain[part], 0);
        }
    } else if (warp < kFixedWarps) {
        // ================= accumulators -> filtered rows =================
        const int quad = warp & 3; // the tensor-memory lanes this warp may read
        int64_t pos = pos0, gb = 0;
        int sl = 0;        // gb % NS, kept by increments
        uint32_t rnd = 0;  // gb / NS
        bool ok = true;
        Item it;
        while (ok && next_item(pos, pos1, p.gpr, p.out_h, it)) {
            int r0, nblk;
            item_rows(it, r0, nblk);
            for (int b = 0; b < nblk; ++b, ++gb) {
                const int d = int(gb & 1);
                if (!warp_wait(&acc_full[d], uint32_t((gb >> 1) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                if (rnd > 0)
                    for (int v = 0; v < VW && ok; ++v)
                        ok = warp_wait(&hfree[sl * kMaxVW + v], (rnd - 1) & 1u, abort_flag, p.err);
                if (!ok) break;
                tc::fence_after_sync();
                float *dst = hring + size_t(sl * kM + quad * 32 + lane) * kHP;
                const uint32_t tq = tmem + (uint32_t(quad * 32) << 16) + uint32_t(d * kChains * 2 * kN);
#pragma unroll
                for (int j = 0; j < kN / 16; ++j) {
                    // even steps hi, lo; odd steps hi, lo
                    uint32_t r[4][16];
#pragma unroll
                    for (int a = 0; a < 4; ++a) tc::tmem_ld16(tq + uint32_t(a * kN + j * 16), r[a]);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int e = 0; e < 16; e += 2) {
                        // (hi + lo of the even K steps) + (hi + lo of the odd ones)
                        const float x0 = (__uint_as_float(r[0][e]) + __uint_as_float(r[1][e])) +
                                         (__uint_as_float(r[2][e]) + __uint_as_float(r[3][e]));
                        const float x1 = (__uint_as_float(r[0][e + 1]) + __uint_as_float(r[1][e + 1])) +
                                         (__uint_as_float(r[2][e + 1]) + __uint_as_float(r[3][e + 1]));
                        *reinterpret_cast<float2 *>(dst + j * 16 + e) = make_float2(x0, x1);
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) {
                    fused::mbar_arrive(&acc_empty[d]);
                    fused::mbar_arrive(&hfull[sl]);
                }
                if (++sl == NS) {
                    sl = 0;
                    ++rnd;
                }
            }
        }
    } else if (warp < kFixedWarps + VW) {
        // ================= vertical pass =================
        const int v = warp - kFixedWarps;
        int64_t pos = pos0;
        bool ok = true;
        Item it;
        const int ring_rows = NS * kM;
        // ring slots of the next block to wait for (and its round) and of the
        // next one to release, kept by increments: every block of every item is
        // waited for and released once, in order
        int w_sl = 0, r_sl = 0, gmod = 0;
        uint32_t w_rnd = 0;
        while (ok && next_item(pos, pos1, p.gpr, p.out_h, it)) {
            int r0, nblk;
            item_rows(it, r0, nblk);
            int waited = 0, released = 0;
            auto wait_block = [&](int) {
                const bool r = warp_wait(&hfull[w_sl], w_rnd & 1u, abort_flag, p.err);
                if (++w_sl == NS) {
                    w_sl = 0;
                    ++w_rnd;
                }
                return r;
            };
            auto release_block = [&](int) {
                __syncwarp();
                if (lane == 0) fused::mbar_arrive(&hfree[r_sl * kMaxVW + v]);
                if (++r_sl == NS) r_sl = 0;
            };
            const int x0 = it.strip * p.NP;
            const int ncols = min(kN, (p.out_w - x0) * C);
            T *orow = static_cast<T *>(p.out) + int64_t(x0) * C;
            // The warp takes the item's row groups v, v + VW, ...: group g is the
            // output rows i0 + 4 g + r, r < 4 (row group q = i0 / 4 + g of the
            // plan's band table).  Their windows overlap, so a group runs over the
            // union of its windows once, with the band of its 4 rows' weights at
            // each union row (zero outside a row's own window): per union row one
            // broadcast 16-byte weight load, one 8-byte load of the filtered row
            // and 8 FMAs (4 rows x the lane's 2 samples: lanes 0..23 own the
            // sample pairs (2 lane, 2 lane + 1)).  The band of the group two ahead
            // is copied from the table while this one is summed (one 16-byte
            // asynchronous copy per union row), and its (first union row, union
            // rows) pair loaded a group earlier still.
            const int col = 2 * lane;
            const bool act = col < kN;
            const int Uv = p.Uv;
            float4 *bands = reinterpret_cast<float4 *>(wsm) + size_t(v) * 2 * Uv;
            const int qb = it.i0 / kVG;
            const int ng = (it.i1 - it.i0 + kVG - 1) / kVG;
            auto fill = [&](int g, int slot) {
                if (g < ng) {
                    const float4 *src = p.vband + size_t(qb + g) * Uv;
                    float4 *bd = bands + slot * Uv;
                    for (int u = lane; u < Uv; u += 32)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(fused::smem_addr(bd + u)),
                                     "l"(src + u)
                                     : "memory");
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
            auto info = [&](int g) { return g < ng ? __ldg(p.vinfo + qb + g) : make_int2(0, 0); };
            int2 i_c = info(v), i_n = info(v + VW);
            fill(v, 0);
            fill(v + VW, 1);
            for (int k = 0, g = v; g < ng && ok; ++k, g += VW) {
                // this group's band (the older of the two in flight) has landed
                asm volatile("cp.async.wait_group 1;" ::: "memory");
                __syncwarp();
                const float4 *bd = bands + (k & 1) * Uv;
                const int rs = i_c.x - r0, U = i_c.y;
                const int lo = rs >> 7, hi = (rs + U - 1) >> 7;
                // blocks below this window are done with (fill-ordered: wait, then release)
                while (released < lo && ok) {
                    if (waited <= released) {
                        ok = wait_block(released);
                        waited = released + 1;
                    }
                    if (ok) release_block(released++);
                }
                while (waited <= hi && ok) ok = wait_block(waited++);
                if (!ok) break;
                // the union's rows in the ring: up to the ring's end, then from its start
                const int first = (gmod * kM + rs) % ring_rows; // gmod = the item's first block's slot
                const int run1 = min(U, ring_rows - first);
                float2 acc[kVG];
#pragma unroll
                for (int r = 0; r < kVG; ++r) acc[r] = make_float2(0.f, 0.f);
                if (act) {
                    auto rows = [&](int u0, int u1, const float *hr) {
                        for (int u = u0; u < u1; ++u, hr += kHP) {
                            const float4 w = bd[u];
                            const float2 h = *reinterpret_cast<const float2 *>(hr);
                            acc[0].x = fmaf(w.x, h.x, acc[0].x);
                            acc[0].y = fmaf(w.x, h.y, acc[0].y);
                            acc[1].x = fmaf(w.y, h.x, acc[1].x);
                            acc[1].y = fmaf(w.y, h.y, acc[1].y);
                            acc[2].x = fmaf(w.z, h.x, acc[2].x);
                            acc[2].y = fmaf(w.z, h.y, acc[2].y);
                            acc[3].x = fmaf(w.w, h.x, acc[3].x);
                            acc[3].y = fmaf(w.w, h.y, acc[3].y);
                        }
                    };
                    rows(0, run1, hring + first * kHP + col);
                    if (run1 < U) rows(run1, U, hring + col);
                }
                const int nrow = min(kVG, it.i1 - (it.i0 + kVG * g));
#pragma unroll
                for (int r = 0; r < kVG; ++r) {
                    if (r >= nrow) break;
                    T *o = orow + int64_t(it.i0 + kVG * g + r) * p.out_stride + col;
                    const T a = fused::from_acc<T, float>(acc[r].x), b = fused::from_acc<T, float>(acc[r].y);
                    if (col + 1 < ncols && (reinterpret_cast<uintptr_t>(o) & 3u) == 0) {
                        // both samples in one 4-byte store
                        uint16_t ua, ub;
                        memcpy(&ua, &a, 2);
                        memcpy(&ub, &b, 2);
                        *reinterpret_cast<uint32_t *>(o) = uint32_t(ua) | (uint32_t(ub) << 16);
                    } else {
                        if (col < ncols) o[0] = a;
                        if (col + 1 < ncols) o[1] = b;
                    }
                }
                // this band is free: the group two ahead goes into it
                __syncwarp();
                fill(g + 2 * VW, k & 1);
                i_c = i_n;
                i_n = info(g + 2 * VW);
            }
            // no copy may still be landing when the warp moves on
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            // the rest of the item's blocks, each released as soon as it is seen
            // full (holding one while waiting for a later one would deadlock:
            // the read-back of block m + 2 waits for block m's release)
            while (ok && released < nblk) {
                if (waited <= released) {
                    ok = wait_block(released);
                    waited = released + 1;
                }
                if (ok) release_block(released++);
            }
            gmod = (gmod + nblk) % NS;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

} // namespace tcstream
} // namespace rs
