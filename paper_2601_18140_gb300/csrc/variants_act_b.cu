// variants_act_b.cu -- variants of the GRID form with activity-aware evaluation
// (own translation unit: the variant units compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const ActVariant kTable[] = {
    RT_ACT_VARIANT(8, 256, 2),
    RT_ACT_VARIANT(1, 512, 4),
    RT_ACT_VARIANT(8, 512, 2),
};

ActVariantTable variants_act_b() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
