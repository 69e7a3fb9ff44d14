// variants_flow.cu -- FLOW-form variants (own translation unit: the variant
// units compile in parallel).
#include "flow.cuh"

namespace rteaal {

static const FlowVariant kFlow[] = {RT_FLOW_VARIANT(64), RT_FLOW_VARIANT(128), RT_FLOW_VARIANT(256)};

FlowVariantTable variants_flow() { return {kFlow, sizeof(kFlow) / sizeof(kFlow[0])}; }

}  // namespace rteaal
