// rs_stream_bf16.cu -- the streaming kernels instantiated for __nv_bfloat16 storage
// (one translation unit per storage type keeps the builds parallel).
#include "rs_stream.cuh"

namespace rs {
namespace stream {

const void *kernel_bf16(int C, int jv, int gv, bool ws, bool multi) { return kernel_table<__nv_bfloat16>(C, jv, gv, ws, multi); }

} // namespace stream
} // namespace rs
