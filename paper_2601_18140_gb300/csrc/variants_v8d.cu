// variants_v8d.cu -- persistent-kernel variants with 8 lanes per thread and two
// narrow rows in flight per thread (own translation unit: the variant units
// compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const Variant kTable[] = {
    RT_VARIANT(8, 2, 224, 4), RT_VARIANT(8, 2, 256, 3), RT_VARIANT(8, 2, 192, 4), RT_VARIANT(8, 2, 512, 2),
};

VariantTable variants_v8d() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
