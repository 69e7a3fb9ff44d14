// variants_v8.cu -- persistent-kernel variants with 8 lanes per thread (own
// translation unit: the variants compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const Variant kV8[] = {
    RT_VARIANT(8, 1, 256, 2), RT_VARIANT(8, 1, 512, 1), RT_VARIANT(8, 1, 384, 2), RT_VARIANT(8, 1, 256, 4),
    RT_VARIANT(8, 1, 384, 3), RT_VARIANT(8, 1, 512, 2), RT_VARIANT(8, 1, 128, 8), RT_VARIANT(8, 1, 448, 2),
    RT_VARIANT(8, 1, 224, 4),
};

VariantTable variants_v8() { return {kV8, sizeof(kV8) / sizeof(kV8[0])}; }

}  // namespace rteaal
