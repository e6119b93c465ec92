// Kernels of the fp64 storage mode (see lb_prec_impl.cuh).
#define LBGB_PREC LB_PREC_FP64
#define LBGB_NAME fp64
#include "lb_prec_impl.cuh"
