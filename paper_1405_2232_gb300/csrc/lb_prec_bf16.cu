// Kernels of the bf16 storage mode (see lb_prec_impl.cuh).
#define LBGB_PREC LB_PREC_BF16_DEV
#define LBGB_NAME bf16
#include "lb_prec_impl.cuh"
