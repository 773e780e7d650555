// rs_stream_f32.cu -- the streaming kernels instantiated for float storage
// (one translation unit per storage type keeps the builds parallel).
#include "rs_stream.cuh"

namespace rs {
namespace stream {

const void *kernel_f32(int C, int jv, int gv, bool ws, bool multi) { return kernel_table<float>(C, jv, gv, ws, multi); }

} // namespace stream
} // namespace rs
