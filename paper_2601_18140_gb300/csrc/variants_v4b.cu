// variants_v4b.cu -- persistent-kernel variants with 4 lanes per thread (own translation
// unit: the variant units compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const Variant kTable[] = {
    RT_VARIANT(4, 1, 384, 4),
    RT_VARIANT(4, 1, 256, 6),
    RT_VARIANT(4, 1, 256, 8),
};

VariantTable variants_v4b() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
