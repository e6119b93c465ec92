// Kernels of the fp32 storage mode (see lb_prec_impl.cuh).
#define LBGB_PREC LB_PREC_FP32
#define LBGB_NAME fp32
#include "lb_prec_impl.cuh"
