// variants_v4c.cu -- persistent-kernel variants with 4 lanes per thread (own translation
// unit: the variant units compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const Variant kTable[] = {
    RT_VARIANT(4, 1, 640, 3),
    RT_VARIANT(4, 1, 448, 4),
    RT_VARIANT(4, 2, 512, 1),
};

VariantTable variants_v4c() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
