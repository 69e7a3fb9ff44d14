// variants_v4a.cu -- persistent-kernel variants with 4 lanes per thread (own translation
// unit: the variant units compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const Variant kTable[] = {
    RT_VARIANT(4, 1, 256, 4),
    RT_VARIANT(4, 1, 512, 2),
    RT_VARIANT(4, 1, 1024, 1),
};

VariantTable variants_v4a() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
