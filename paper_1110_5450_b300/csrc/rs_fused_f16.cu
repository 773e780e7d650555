// rs_fused_f16.cu -- instantiations of the fused kernel for __half storage.
// The kernel template itself is in rs_fused.cuh; this file only lists the
// (channels, group, band width) combinations compiled for this storage type.
#include "rs_fused.cuh"

namespace rs {
namespace fused {

static const Variant kVariants[] = {
    RS_FUSED_VARIANT(__half, RS_F16, 1, 4, 8),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 4, 9),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 4, 12),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 4, 16),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 4, 24),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 4, 32),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 2, 16),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 2, 24),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 2, 32),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 2, 48),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 1, 32),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 1, 48),
    RS_FUSED_VARIANT(__half, RS_F16, 1, 1, 64),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 4, 8),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 4, 9),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 4, 12),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 4, 16),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 4, 24),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 4, 32),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 2, 16),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 2, 24),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 2, 32),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 2, 48),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 1, 32),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 1, 48),
    RS_FUSED_VARIANT(__half, RS_F16, 3, 1, 64),
};

const Variant *variants_f16(int *n)
{
    *n = int(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

} // namespace fused
} // namespace rs
