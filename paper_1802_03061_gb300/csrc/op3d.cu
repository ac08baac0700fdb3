// placeholder, replaced by the 3D passes
#include "internal.h"
rte_status op3d_apply64(rte_plan, MixKind, const double*, double*, double, double, double, const double*,
                        cudaStream_t) { return RTE_EUNSUPPORTED; }
rte_status op3d_apply32(rte_plan, const float*, float*, float, float, float, const float*, cudaStream_t) {
    return RTE_EUNSUPPORTED;
}
