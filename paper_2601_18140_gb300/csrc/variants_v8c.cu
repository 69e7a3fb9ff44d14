// variants_v8c.cu -- persistent-kernel variants with 8 lanes per thread (own translation
// unit: the variant units compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const Variant kTable[] = {
    RT_VARIANT(8, 1, 512, 2),
    RT_VARIANT(8, 1, 128, 8),
    RT_VARIANT(8, 1, 448, 2),
};

VariantTable variants_v8c() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
