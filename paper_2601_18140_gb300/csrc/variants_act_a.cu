// variants_act_a.cu -- variants of the GRID form with activity-aware evaluation
// (own translation unit: the variant units compile in parallel).
#include "persistent.cuh"

namespace rteaal {

static const ActVariant kTable[] = {
    RT_ACT_VARIANT(4, 384, 4),
    RT_ACT_VARIANT(4, 256, 8),
    RT_ACT_VARIANT(4, 512, 2),
    RT_ACT_VARIANT(2, 512, 4),
};

ActVariantTable variants_act_a() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
