// rs_plan.h -- internal: the plan object and the host helpers shared by the
// single-image entry points (rs_capi.cu) and the batch / serving code.
#pragma once

#include <cuda.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rs_fused.cuh"
#include "rs_internal.h"
#include "rs_stream.cuh"
#include "rs_tcstream.cuh"
#include "rs_xstream.cuh"

namespace rs {

// One fused-kernel configuration of a plan.
struct Candidate {
    int G = 0, J = 0, tile_h = 0, tile_w = 0, stages = 1, box_h = 0, box_w = 0, n_sub = 1, sub_h = 0, n1 = 4;
    int tc = 0; // 1: vertical pass on the tensor cores
    size_t smem = 0;
    double cost = 0.0; // modelled SM cycles per output pixel
};

struct DeviceBuf {
    void *p = nullptr;
    size_t n = 0;
    ~DeviceBuf()
    {
        if (p) cudaFree(p);
    }
};

// Vertical-first two-pass path (rs_vfirst.cu): bands and intermediate.
struct VfParams {
    int32_t JV = 0, JH = 0, groups_y = 0, groups_x = 0;
    int64_t tmp_stride = 0; // samples per intermediate row (in_w + JH pixels)
    int32_t *vbase = nullptr, *hbase = nullptr;
    float *vband = nullptr, *hband = nullptr, *tmp = nullptr;
};

// An NVTX range around an API call (free when no profiler is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// Kernel-choice flags from the RS_PLAN_FLAGS environment variable (comma-
// separated names without the RS_ prefix); -1 if a name is not one of them.
int64_t env_plan_flags();

// Carve 256-byte aligned pieces out of one allocation.
struct Carver {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    }
};

} // namespace rs

// The plan object behind the opaque rs_plan handle.
struct rs_plan {
    rs_plan_desc desc{};
    int device = 0;
    int num_sms = 0;
    rs::AxisGeom gy, gx;
    rs::AxisTables ty, tx;
    int work_double = 0;
    int axes_alias = 0; // identical axes: the column tables are the row tables
    int path = 1; // 0 fused, 1 two-pass
    rs::DeviceBuf tables, bands, tmp, errbuf;
    int *d_err = nullptr;
    // fused path
    rs::fused::Params fp{};
    const rs::fused::Variant *variant = nullptr;
    const void *kernel_fn = nullptr; // the variant's SIMT or tensor-core kernel
    int G = 0, J = 0;
    size_t smem = 0;
    int grid = 0;
    int ctas_per_sm = 0;
    int tma_ok = 0;
    CUtensorMap tmap;
    const void *tmap_ptr = nullptr;
    int64_t scratch_bytes = 0;
    std::vector<int32_t> host_start_y, host_start_x; // for re-planning and tuning
    rs::Candidate chosen;                            // fused configuration in use
    // row-streaming kernel (FP32 upscales and mild downscales)
    int tile_bands_stale = 0; // recomputed weights not yet in the tile kernel's bands
    int stream_ok = 0;  // a streaming configuration exists
    int stream_code = 0; // its choices (stream::Opts::code)
    int use_stream = 0; // rs_resample runs it (else the tile kernel above)
    rs::stream::Params sp{};
    rs::DeviceBuf sbufs;
    CUtensorMap stmap;
    const void *stmap_ptr = nullptr;
    const void *s_fn = nullptr;
    int s_block = 0; // threads per CTA of the streaming kernel in use
    size_t s_smem = 0;
    int s_grid = 0, s_ctas = 0;
    // the pipelined form of the streaming kernel (upscales, 4 or 6 taps):
    // when x_on, s_fn / s_smem / s_grid / s_ctas describe it and xp holds its
    // parameters (its group descriptors live in xbufs)
    int x_on = 0;
    rs::xstream::Params xp{};
    rs::DeviceBuf xbufs;
    // the tensor-core downscale form (16-bit downscales): when tcs_on, s_fn /
    // s_block / s_smem / s_grid describe it, tcp holds its parameters and
    // tcbufs its per-strip weight matrices; stmap is its 3-D input map
    int tcs_on = 0;
    rs::tcstream::Params tcp{};
    rs::DeviceBuf tcbufs;
    // external placement of the streaming kernels' tables (a serving
    // arena): when ext_base is set, the streaming set-up carves its band or
    // descriptor tables out of [ext_base, ext_base + ext_bytes) instead of
    // allocating, and uploads host data through ext_staging (pinned) with
    // copies on its stream, never synchronising
    char *ext_base = nullptr;
    size_t ext_bytes = 0;
    unsigned char *ext_staging = nullptr;
    size_t ext_staging_bytes = 0;
    // interpolating cubic B-spline: coefficients of the input (RS_PREFILTER)
    int prefilter = 0;
    rs::DeviceBuf pbufs;
    void *coef = nullptr;                       // [in_h][in_row_stride] FP32 (FP64 for RS_F64)
    const void *pf_h = nullptr, *pf_w = nullptr; // per axis: 1/pivot, factor, sub-diagonal
    void *pf_dp = nullptr;                       // forward-elimination scratch, as coef
    // vertical-first two-pass path (strong vertical downscales)
    int vfirst_ok = 0;  // configured (bands and intermediate allocated)
    int use_vfirst = 0; // rs_resample runs it
    rs::VfParams vf{};
    rs::DeviceBuf vbufs;
};

namespace rs {

rs_status fail(rs_status s, const std::string &msg);
// RS_CHECK: the plan's tables checked on the device (rs_check.cu).
cudaError_t launch_table_check(const rs_plan *p, cudaStream_t s);
// The bounded-wait self-test kernel (rs_check.cu).
cudaError_t launch_wait_selftest(int *err, uint64_t limit_ns, cudaStream_t s);
// Instantiated fused kernel for (dtype, channels, group size), or nullptr.
const fused::Variant *find_variant(int dtype, int C, int G);
// Support radius of a kernel (0 for an invalid Lanczos parameter).
int support_radius(int kernel, double param);
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
// cuTensorMapEncodeTiled through the runtime's driver entry point (nullptr if unavailable).
EncodeTiledFn encode_fn();
rs_status cuda_fail(cudaError_t e, const char *what);
// Every feasible fused configuration (needs the host start tables); with tc
// the tensor-core configurations instead of the SIMT ones.
std::vector<Candidate> enumerate_candidates(rs_plan *p, bool tma_layout, bool tc = false);
// Builds the band tables of a configuration and the kernel parameters.
rs_status apply_fused(rs_plan *p, cudaStream_t stream, const Candidate &c, bool tma_layout);
// Whether the plan's row pitch allows TMA tile copies.
bool tma_layout_ok(const rs_plan *p);
// Encodes the plan's input tensor map for d_in into *map.
rs_status encode_tensor_map(const rs_plan *p, const void *d_in, CUtensorMap *map);
// Shared-memory region sizes of a fused plan's configuration.
void work_regions(const rs_plan *p, fused::Work *w);
// Single-image work description of a fused plan.
fused::Work single_work(const rs_plan *p, int use_tma);
// Cost of a candidate in modelled SM cycles per output pixel (also sets n1).
double model_cost(Candidate &c, int C, size_t esz, size_t asz, int V);

namespace prefilter {
// Allocates the coefficient buffer and uploads the elimination factors.
rs_status setup(rs_plan *p);
// Replaces the input by its cubic B-spline coefficients in p->coef (rows,
// then columns), on `s`.
rs_status launch(rs_plan *p, const void *d_in, cudaStream_t s);
} // namespace prefilter

namespace vfirst {
// Configures the vertical-first path (allocates its bands and intermediate);
// RS_ERR_UNSUPPORTED when the plan is not eligible (FP64, channels other than
// 1 or 3, an upscale in rows, bands wider than 256).
rs_status setup(rs_plan *p, cudaStream_t s);
// Rebuilds its bands from the plan's weight tables (after a recompute).
rs_status rebuild(rs_plan *p, cudaStream_t s);
// Both passes on `s`.
rs_status launch(rs_plan *p, const void *d_in, void *d_out, cudaStream_t s);
} // namespace vfirst

namespace stream {
// Choices of a streaming configuration: ex = 1 the pipelined kernel
// (rs_xstream.cuh), 2 the tensor-core downscale (rs_tcstream.cuh), 0 the band
// kernels of rs_stream.cuh, -1 the pipelined kernel where it applies with its
// default choices, else the tensor-core downscale where it applies, else the
// band kernels (ni_min and vw give the tensor-core kernel's staged chunks and
// vertical warps when ex = 2); ws = 1
// warp-specialised band kernel, 0 phase-alternating, -1 either
// (warp-specialised first); hw = warps on the horizontal pass (0: the form's
// default); ni_min = fewest staged input blocks of a narrow strip (the
// pipelined kernel: its staged blocks); pf = 1: the pipelined kernel
// prefetches the block after its ring into L2.
struct Opts {
    int ws = -1, hw = 0, ni_min = 3;
    int sw = 0; // strip width (0: the cost model's choice)
    int ex = -1, pf = 0;
    int vw = 0; // pipelined kernel: warps on the vertical pass (0: the default)
    int nr = 0; // pipelined kernel: row ranges (0: the cost model's choice), < 256
    int code() const
    {
        return 1 + (ws > 0 ? 2 : 0) + 4 * hw + 64 * ni_min + 512 * (sw / 4) + (ex == 1 ? 32768 : 0) +
               (pf ? 65536 : 0) + (ex == 2 ? 131072 : 0) + (vw << 18) + (nr << 22);
    }
    static Opts decode(int c)
    {
        Opts o;
        o.ws = (c & 2) ? 1 : 0;
        o.hw = (c >> 2) & 15;
        o.ni_min = (c >> 6) & 7;
        o.sw = ((c >> 9) & 63) * 4;
        o.ex = ((c >> 17) & 1) ? 2 : (c >> 15) & 1;
        o.pf = (c >> 16) & 1;
        o.vw = (c >> 18) & 15;
        o.nr = (c >> 22) & 255;
        return o;
    }
};
// Configures the row-streaming kernel for a plan (needs the host start tables);
// RS_ERR_UNSUPPORTED when the plan is not eligible.
rs_status setup(rs_plan *p, cudaStream_t s, const Opts &o = Opts());
// Strip widths the configuration admits, best first by the cost model (at
// most n); 0 if the plan is not eligible.
int widths(rs_plan *p, const Opts &o, int *out, int n);
// Rebuilds its band tables from the plan's weight tables (after a recompute).
rs_status rebuild(rs_plan *p, cudaStream_t s);
rs_status launch(rs_plan *p, const void *d_in, void *d_out, cudaStream_t s);
// The input tensor map of a band or pipelined streaming configuration for d_in.
rs_status encode_input_map(const rs_plan *p, const void *d_in, CUtensorMap *map);
// Row-range counts the configuration searches model (ascending).
std::vector<int> range_counts(int n_strips, int64_t slots, int max_nr);
// The multi-image variant (stream_multi_kernel / stream_ws_multi_kernel) of
// the plan's configured band kernel, or nullptr (no band configuration).
const void *multi_kernel(const rs_plan *p);
// Loads every band-kernel instantiation of `dtype` (lazy module loading
// would otherwise load each on its first launch, in the middle of a stream's
// work) and tabulates its occupancy.
void preload(int dtype);
} // namespace stream

namespace tcstream {
// Whether the plan can run the tensor-core downscale (FP16/BF16, 1 or 3
// channels, both axes downscaled, in_w * channels a multiple of 8, a 16-byte
// row pitch, at most 128 vertical taps).
bool eligible(const rs_plan *p);
// Configures it on `s` (o.ni_min staged chunks and o.vw vertical warps when
// o.ex = 2; else the defaults): the strips' weight matrices are built on the
// device from the plan's tables.  RS_ERR_UNSUPPORTED when not eligible.
rs_status setup(rs_plan *p, cudaStream_t s, const stream::Opts &o);
// Rebuilds the weight matrices from the plan's weight tables (after a recompute).
rs_status rebuild(rs_plan *p, cudaStream_t s);
rs_status launch(rs_plan *p, const void *d_in, void *d_out, cudaStream_t s);
// Bytes of its device tables at most, for external placement (a serving arena).
size_t space_bound(const AxisGeom &gx, const AxisGeom &gy, int C);
// As stream::preload.
void preload(int dtype);
} // namespace tcstream

namespace xstream {
// As stream::preload, for the pipelined kernel.
void preload(int dtype);
// The multi-image variant (xstream_multi_kernel) of the plan's configured
// pipelined kernel, or nullptr.
const void *multi_kernel(const rs_plan *p);
// Whether the plan can run the pipelined kernel (FP32/FP16/BF16, 1 or 3
// channels, a 16-byte row pitch, 4 or 6 taps per output on both axes, window
// starts that advance by 0 or 1 per output: an upscale or scale 1).
bool eligible(const rs_plan *p);
// Configures it on `s` (o.hw horizontal warps, o.ni_min staged blocks, o.sw strip
// width, o.pf, o.vw, o.nr; zeros choose the defaults); RS_ERR_UNSUPPORTED when the plan
// is not eligible.  The kernel reads the plan's weight tables directly.
rs_status setup(rs_plan *p, cudaStream_t s, const stream::Opts &o);
// Strip widths it admits, best first by the cost model (at most n).
int widths(rs_plan *p, const stream::Opts &o, int *out, int n);
} // namespace xstream

} // namespace rs
