// Kernels of the fp16 storage mode (see lb_prec_impl.cuh).
#define LBGB_PREC LB_PREC_FP16_DEV
#define LBGB_NAME fp16
#include "lb_prec_impl.cuh"
