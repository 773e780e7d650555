// rs_xstream_f16.cu -- the pipelined streaming kernel instantiated for
// __half storage (one translation unit per storage type keeps the builds parallel).
#include "rs_xstream.cuh"

namespace rs {
namespace xstream {

const void *kernel_f16(int C, int taps, int big) { return kernel_table<__half>(C, taps, big); }

} // namespace xstream
} // namespace rs
