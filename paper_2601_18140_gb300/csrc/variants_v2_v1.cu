// variants_v2_v1.cu -- persistent-kernel variants with 2 and 1 lanes per thread
// (small lane counts; U = 2, 4 keep several items in flight per thread).
#include "persistent.cuh"

namespace rteaal {

static const Variant kV21[] = {
    RT_VARIANT(2, 1, 256, 8), RT_VARIANT(2, 1, 512, 4), RT_VARIANT(2, 1, 1024, 2),
    RT_VARIANT(2, 2, 512, 2), RT_VARIANT(2, 4, 512, 1),
    RT_VARIANT(1, 1, 512, 4), RT_VARIANT(1, 2, 512, 2), RT_VARIANT(1, 4, 512, 1),
};

VariantTable variants_v2_v1() { return {kV21, sizeof(kV21) / sizeof(kV21[0])}; }

}  // namespace rteaal
