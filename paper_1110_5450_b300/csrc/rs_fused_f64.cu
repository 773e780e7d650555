// rs_fused_f64.cu -- instantiations of the fused kernel for double storage.
// The kernel template itself is in rs_fused.cuh; this file only lists the
// (channels, group size, columns per thread) combinations compiled for this
// storage type.  The band width J is a run-time parameter.
#include "rs_fused.cuh"

namespace rs {
namespace fused {

static const Variant kVariants[] = {
    RS_FUSED_VARIANT(double, RS_F64, 1, 4, 2),
    RS_FUSED_VARIANT(double, RS_F64, 1, 2, 2),
    RS_FUSED_VARIANT(double, RS_F64, 1, 1, 2),
    RS_FUSED_VARIANT(double, RS_F64, 3, 4, 2),
    RS_FUSED_VARIANT(double, RS_F64, 3, 2, 2),
    RS_FUSED_VARIANT(double, RS_F64, 3, 1, 2),
};

const Variant *variants_f64(int *n)
{
    *n = int(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

} // namespace fused
} // namespace rs
