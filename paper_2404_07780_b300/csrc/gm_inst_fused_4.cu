// Instances of k_fused, list 4 of gm_instances.h.
#include "gm_fused.cuh"
#include "gm_instances.h"

namespace gm {
#define GM_X(M, P, C, W) template __global__ void k_fused<M, P, C, W>(const __grid_constant__ FusedArgs);
GM_FUSED_LIST_4(GM_X)
#undef GM_X
}  // namespace gm
