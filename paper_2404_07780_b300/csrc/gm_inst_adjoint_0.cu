// Instances of k_adjoint, list 0 of gm_instances.h.
#include "gm_adjoint.cuh"
#include "gm_instances.h"

namespace gm {
#define GM_X(M, P) template __global__ void k_adjoint<M, P>(const __grid_constant__ AdjArgs);
GM_ADJ_LIST_0(GM_X)
#undef GM_X
}  // namespace gm
