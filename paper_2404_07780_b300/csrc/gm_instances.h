// gm_instances.h -- every template instance of the two tile kernels the library
// launches, as X-macro lists.  Each list is instantiated in its own translation
// unit (gm_inst_*.cu, compiled in parallel) and declared extern in gm_lib.cu,
// which launches the instances through function pointers.
#pragma once

// k_fused<MODE, P, CPT, WIDE>: MODE_MODEL = 0, MODE_NORMAL = 1; P free
// parameters; CPT channel pairs per thread (1: up to 512 threads; 2: up to 256
// threads with the register budget of many free parameters); WIDE = 1 with
// CPT = 2: 512 threads in four groups, 2 or 4 groups per two pairs of a pass.
#define GM_FUSED_LIST_0(X) X(0, 0, 1, 0) X(1, 0, 1, 0) X(1, 1, 1, 0) X(1, 2, 1, 0) X(1, 3, 1, 0) X(1, 4, 1, 0) X(1, 5, 1, 0) X(1, 6, 1, 0)
#define GM_FUSED_LIST_1(X) X(1, 7, 1, 0) X(1, 8, 1, 0) X(1, 9, 1, 0) X(1, 10, 1, 0) X(1, 0, 2, 0) X(1, 1, 2, 0) X(1, 2, 2, 0) X(1, 3, 2, 0)
#define GM_FUSED_LIST_2(X) X(1, 4, 2, 0) X(1, 5, 2, 0) X(1, 6, 2, 0) X(1, 7, 2, 0) X(1, 8, 2, 0) X(1, 9, 2, 0) X(1, 10, 2, 0) X(1, 11, 2, 0)
#define GM_FUSED_LIST_3(X) X(1, 12, 2, 0) X(1, 13, 2, 0) X(1, 14, 2, 0) X(1, 15, 2, 0) X(1, 16, 2, 0)

// k_adjoint<MODE> (ADJ_RESID = 0, ADJ_GRAD = 1) in list 0; k_adj_resid<P> and
// k_adj_deriv<P>, the pixel kernels of the adjoint gradient, for P free parameters
#define GM_RESID_LIST_0(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)
#define GM_RESID_LIST_1(X) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)
#define GM_DERIV_LIST_0(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)
#define GM_DERIV_LIST_1(X) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

#define GM_FUSED_LIST_4(X) \
  X(1, 1, 2, 1) X(1, 2, 2, 1) X(1, 3, 2, 1) X(1, 4, 2, 1) X(1, 5, 2, 1) X(1, 6, 2, 1) X(1, 7, 2, 1) X(1, 8, 2, 1) \
  X(1, 9, 2, 1) X(1, 10, 2, 1) X(1, 11, 2, 1) X(1, 12, 2, 1) X(1, 13, 2, 1) X(1, 14, 2, 1) X(1, 15, 2, 1) X(1, 16, 2, 1)

#define GM_FUSED_ALL(X) GM_FUSED_LIST_0(X) GM_FUSED_LIST_1(X) GM_FUSED_LIST_2(X) GM_FUSED_LIST_3(X) GM_FUSED_LIST_4(X)
#define GM_RESID_ALL(X) GM_RESID_LIST_0(X) GM_RESID_LIST_1(X)
#define GM_DERIV_ALL(X) GM_DERIV_LIST_0(X) GM_DERIV_LIST_1(X)
