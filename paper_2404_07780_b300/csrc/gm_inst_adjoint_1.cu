// Instances of the adjoint gradient's kernels, list 1 of gm_instances.h.
#include "gm_adjoint.cuh"
#include "gm_instances.h"

namespace gm {
#define GM_X(P) template __global__ void k_adj_resid<P>(const __grid_constant__ PixArgs);
GM_RESID_LIST_1(GM_X)
#undef GM_X
#define GM_X(P) template __global__ void k_adj_deriv<P>(const __grid_constant__ PixArgs);
GM_DERIV_LIST_1(GM_X)
#undef GM_X
}  // namespace gm
