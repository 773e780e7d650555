// rs_fused_bf16.cu -- instantiations of the fused kernel for __nv_bfloat16 storage.
// The kernel template itself is in rs_fused.cuh; this file only lists the
// (channels, group size, columns per thread) combinations compiled for this
// storage type.  The band width J is a run-time parameter.
#include "rs_fused.cuh"

namespace rs {
namespace fused {

static const Variant kVariants[] = {
    RS_FUSED_VARIANT_TC(__nv_bfloat16, RS_BF16, 1, 4, 4),
    RS_FUSED_VARIANT_TC(__nv_bfloat16, RS_BF16, 1, 2, 4),
    RS_FUSED_VARIANT_TC(__nv_bfloat16, RS_BF16, 1, 1, 4),
    RS_FUSED_VARIANT_TC(__nv_bfloat16, RS_BF16, 3, 4, 4),
    RS_FUSED_VARIANT_TC(__nv_bfloat16, RS_BF16, 3, 2, 4),
    RS_FUSED_VARIANT_TC(__nv_bfloat16, RS_BF16, 3, 1, 4),
};

const Variant *variants_bf16(int *n)
{
    *n = int(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

} // namespace fused
} // namespace rs
