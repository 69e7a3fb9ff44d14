// variants_v2.cu -- persistent-kernel variants with 2 lanes per thread (own translation
// unit: the variant units compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const Variant kTable[] = {
    RT_VARIANT(2, 1, 256, 8),
    RT_VARIANT(2, 1, 512, 4),
    RT_VARIANT(2, 1, 1024, 2),
    RT_VARIANT(2, 2, 512, 2),
    RT_VARIANT(2, 4, 512, 1),
};

VariantTable variants_v2() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
