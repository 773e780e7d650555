// rs_stream_f16.cu -- the streaming kernels instantiated for __half storage
// (one translation unit per storage type keeps the builds parallel).
#include "rs_stream.cuh"

namespace rs {
namespace stream {

const void *kernel_f16(int C, int jv, int gv, bool ws, bool multi) { return kernel_table<__half>(C, jv, gv, ws, multi); }

} // namespace stream
} // namespace rs
