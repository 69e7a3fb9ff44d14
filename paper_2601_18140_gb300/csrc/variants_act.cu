// variants_act.cu -- variants of the GRID form with activity-aware evaluation.
#include "persistent.cuh"

namespace rteaal {

static const ActVariant kAct[] = {
    RT_ACT_VARIANT(4, 384, 4), RT_ACT_VARIANT(4, 256, 8), RT_ACT_VARIANT(4, 512, 2),
    RT_ACT_VARIANT(2, 512, 4), RT_ACT_VARIANT(8, 256, 2), RT_ACT_VARIANT(1, 512, 4), RT_ACT_VARIANT(8, 512, 2),
};

ActVariantTable act_variants() { return {kAct, sizeof(kAct) / sizeof(kAct[0])}; }

}  // namespace rteaal
