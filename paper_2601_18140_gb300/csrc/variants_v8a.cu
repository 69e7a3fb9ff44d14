// variants_v8a.cu -- persistent-kernel variants with 8 lanes per thread (own translation
// unit: the variant units compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const Variant kTable[] = {
    RT_VARIANT(8, 1, 224, 4),
    RT_VARIANT(8, 1, 256, 2),
    RT_VARIANT(8, 1, 512, 1),
};

VariantTable variants_v8a() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
