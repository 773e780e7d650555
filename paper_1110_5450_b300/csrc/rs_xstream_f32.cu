// rs_xstream_f32.cu -- the pipelined streaming kernel instantiated for
// float storage (one translation unit per storage type keeps the builds parallel).
#include "rs_xstream.cuh"

namespace rs {
namespace xstream {

const void *kernel_f32(int C, int taps, int big) { return kernel_table<float>(C, taps, big); }

} // namespace xstream
} // namespace rs
