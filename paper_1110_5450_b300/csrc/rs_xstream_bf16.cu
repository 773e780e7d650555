// rs_xstream_bf16.cu -- the pipelined streaming kernel instantiated for
// __nv_bfloat16 storage (one translation unit per storage type keeps the builds parallel).
#include "rs_xstream.cuh"

namespace rs {
namespace xstream {

const void *kernel_bf16(int C, int taps, int big) { return kernel_table<__nv_bfloat16>(C, taps, big); }

} // namespace xstream
} // namespace rs
