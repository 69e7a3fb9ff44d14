// variants_v4.cu -- persistent-kernel variants with 4 lanes per thread (MAXT *
// MINB = 1,536 .. 2,048 threads per SM; U = 2 trades occupancy for in-flight items).
#include "persistent.cuh"

namespace rteaal {

static const Variant kV4[] = {
    RT_VARIANT(4, 1, 256, 4), RT_VARIANT(4, 1, 512, 2), RT_VARIANT(4, 1, 1024, 1),
    RT_VARIANT(4, 1, 384, 4), RT_VARIANT(4, 1, 256, 6), RT_VARIANT(4, 1, 256, 8),
    RT_VARIANT(4, 1, 640, 3), RT_VARIANT(4, 1, 448, 4),
    RT_VARIANT(4, 2, 512, 1),
};

VariantTable variants_v4() { return {kV4, sizeof(kV4) / sizeof(kV4[0])}; }

}  // namespace rteaal
