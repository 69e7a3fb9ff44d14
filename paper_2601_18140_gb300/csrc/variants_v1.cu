// variants_v1.cu -- persistent-kernel variants with 1 lane per thread (own translation
// unit: the variant units compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const Variant kTable[] = {
    RT_VARIANT(1, 1, 512, 4),
    RT_VARIANT(1, 2, 512, 2),
    RT_VARIANT(1, 4, 512, 1),
};

VariantTable variants_v1() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
