// rs_internal.h -- internal declarations of the B300 resampler library.
// Not installed; the public interface is include/rs.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "rs.h"

namespace rs {

// Largest raw tap count per output the plan accepts (before boundary folding).
constexpr int kMaxTaps = 256;
// Largest side length: keeps every integer of the tap formula far below 2^63.
constexpr int64_t kMaxSide = int64_t(1) << 22;

// Geometry of one axis.  The kernel argument of raw tap j for output i is
// x = ((2j+1) n_out - (2i+1) n_in) / D, and tap j belongs to output i iff the
// numerator's magnitude is below R*D.
struct AxisGeom {
    int64_t n_in = 0, n_out = 0;
    int64_t D = 0;     // 2 max(n_in, n_out), or 2 n_out without antialiasing
    int64_t R = 0;     // kernel support radius
    int32_t t_raw = 0; // bound on raw taps per output: ceil(R D / n_out)
    int32_t t_eff = 0; // stored window width after boundary folding: min(t_raw, n_in)
    int32_t kernel = 0;
    int32_t boundary = 0;
    double param = 0.0;
};

// Device tables of one axis.
struct AxisTables {
    int32_t *jlo = nullptr;   // [n_out] first raw tap
    int32_t *cnt = nullptr;   // [n_out] raw tap count
    int32_t *start = nullptr; // [n_out] first index of the folded window
    double *w64 = nullptr;    // [n_out][t_eff] folded normalised FP64 weights
    void *wwork = nullptr;    // [n_out][t_eff] working precision (float or double)
    // Weight band for the fused kernel: outputs are grouped G at a time;
    // group g reads inputs [base[g], base[g] + J) with the weight of member r
    // and input j stored `dup` times (1, or 2 for packed-pair FMAs) at
    // band_w[g * band_stride(G * dup, J) + (j * G + r) * dup + d].
    // With pair_ngx > 0 (the horizontal band of the fused kernel) the groups
    // of every tile of pair_ngx groups are taken two at a time: slot s holds
    // tile s / P, pair p = s % P (P = ceil(pair_ngx / 2)), and the weights of
    // its groups q0 = tile * pair_ngx + 2p and q0 + 1 interleaved at
    // band_w[s * band_stride(2 G, J) + (j * G + r) * 2 + d] (d selects the
    // group; zeros for a group past the tile or the axis), so that one lane
    // runs both groups with packed-pair FMAs.
    int32_t *band_base = nullptr; // [groups]
    void *band_w = nullptr;       // [band_slots][band_slot_stride] working precision
    int32_t G = 0, J = 0, groups = 0, dup = 1;
    int32_t pair_ngx = 0;
    // align > 1: group bases are the members' smallest start rounded down to a
    // multiple of align, not kept inside the axis (the row-streaming kernel's
    // horizontal band; its staged copy reads zeros past the input's end)
    int32_t align = 0;
};

// Floats per band group: J * G rounded up to a multiple of 4, so that every
// group starts on a 16-byte boundary (TMA bulk copies need that).
__host__ __device__ inline int band_stride(int G, int J) { return (J * G + 3) / 4 * 4; }

// Slots of a band (groups, or tile-local group pairs) and floats per slot.
__host__ __device__ inline int64_t band_slots(const AxisTables &t)
{
    if (t.pair_ngx <= 0) return t.groups;
    const int64_t tiles = (int64_t(t.groups) + t.pair_ngx - 1) / t.pair_ngx;
    return tiles * ((t.pair_ngx + 1) / 2);
}
__host__ __device__ inline int band_slot_stride(const AxisTables &t)
{
    return band_stride(t.G * (t.pair_ngx > 0 ? 2 : t.dup), t.J);
}

// Parameters of the weight-table kernel for one axis (passed by value).
struct WeightArgs {
    AxisGeom g;
    AxisTables t;
    int work_is_double; // working precision: 1 = FP64, 0 = FP32
    int *err;           // device error word
};

// Weight-table kernel for both axes in one launch.
cudaError_t launch_weights(const WeightArgs &a0, const WeightArgs &a1, cudaStream_t s);
// Band tables for the fused kernel (both axes, one launch).
cudaError_t launch_band(const WeightArgs &a0, const WeightArgs &a1, cudaStream_t s);
// Loads the weight-table and band kernels now rather than at their first
// launch (lazy module loading).
void preload_weights();

// Element type code shared by the pass launchers.
enum class Dt : int { F64 = RS_F64, F32 = RS_F32, F16 = RS_F16, BF16 = RS_BF16 };

inline size_t dt_size(int d)
{
    return d == RS_F64 ? 8 : d == RS_F32 ? 4 : 2;
}

// Two-pass (H then V) path through an HBM intermediate of the accumulation type.
struct TwoPassArgs {
    const void *in;
    void *out;
    void *tmp; // [in_h][out_w * C] accumulation type
    int64_t in_h, in_w, out_h, out_w, C;
    int64_t in_stride, out_stride; // elements
    int32_t *start_x, *start_y;
    const void *w_x, *w_y; // working precision [n_out][t]
    int32_t t_x, t_y;
    int dtype; // rs_dtype (in == out)
};
cudaError_t launch_two_pass(const TwoPassArgs &a, cudaStream_t s);

// Thread-local last-error string.
void set_error(const std::string &msg);

// Checks a descriptor as rs_plan_create does (sizes, channels, kernel and
// parameter, boundary, dtypes, flag bits, strides), derives the output size
// where out_h / out_w are 0 and the packed strides where they are 0; on
// failure sets the error message and returns its status.
rs_status validate_desc(const rs_plan_desc &in, rs_plan_desc *out);
// The geometry of one axis of a validated descriptor (false with a reason when
// it needs more than kMaxTaps taps per output).
bool axis_setup(AxisGeom &g, int64_t n_in, int64_t n_out, const rs_plan_desc &d, std::string &why);

// Resident CTAs per SM of kernel `fn` launched with `nthreads` threads and
// `smem` bytes of dynamic shared memory on the current device, the kernel's
// dynamic shared-memory limit raised to 227 KB.  The first call for a
// (device, kernel, block size) tabulates where the count drops (the runtime's
// occupancy query, bisected); later calls make no CUDA call.  0 when the
// kernel cannot run so (or the queries failed).  Thread-safe.
int occupancy(const void *fn, int nthreads, size_t smem);

} // namespace rs
