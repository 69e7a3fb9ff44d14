// variants_cluster.cu -- cluster-form variants (own translation unit: the
// variant units compile in parallel).
#include "cluster.cuh"

namespace rteaal {

static const ClusterVariant kTable[] = {
    RT_CLUSTER_VARIANT(1, 256),      RT_CLUSTER_VARIANT(1, 512),      RT_CLUSTER_VARIANT(1, 1024),
    RT_CLUSTER_VARIANT(2, 512),      RT_CLUSTER_VARIANT(4, 512),      RT_CLUSTER_VARIANT(8, 256),
    RT_CLUSTER_RES_VARIANT(256),     RT_CLUSTER_RES_VARIANT(512),     RT_CLUSTER_RES_VARIANT(1024),
};

ClusterVariantTable variants_cluster() { return {kTable, sizeof(kTable) / sizeof(kTable[0])}; }

}  // namespace rteaal
