// lb_init_balanced.cu -- launcher of the start at rest under the force
// (k_init_balanced) for every storage precision.  Compiled without FMA
// contraction so that the FP64 arithmetic follows the printed formulas
// operation by operation; the FP32 and 16-bit starts are that FP64 value
// rounded once to the storage type.
#include "lb_init_balanced.cuh"
#include "lb_launch.h"

namespace lbgb {

namespace {

template <int PREC>
cudaError_t launch_typed(void* dst, const KParams& kp, const double* rho0, const double* T0,
                         cudaStream_t st) {
    using E = typename Store<PREC>::elem;
    const long long n = (long long)kp.nx * kp.ny;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    E* d = static_cast<E*>(dst);
    if (kp.beta == 0.0)
        k_init_balanced<PREC, BETA_ZERO><<<blocks, 256, 0, st>>>(d, kp, rho0, T0);
    else if (kp.beta == 1.0)
        k_init_balanced<PREC, BETA_ONE><<<blocks, 256, 0, st>>>(d, kp, rho0, T0);
    else
        k_init_balanced<PREC, BETA_MIXED><<<blocks, 256, 0, st>>>(d, kp, rho0, T0);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init_balanced(int prec, void* dst, const KParams& kp, const double* rho0,
                                 const double* T0, cudaStream_t st) {
    if (kp.walls) return cudaErrorInvalidValue;
    switch (prec) {
        case LB_PREC_FP64: return launch_typed<LB_PREC_FP64>(dst, kp, rho0, T0, st);
        case LB_PREC_FP32: return launch_typed<LB_PREC_FP32>(dst, kp, rho0, T0, st);
        case LB_PREC_FP16_DEV: return launch_typed<LB_PREC_FP16_DEV>(dst, kp, rho0, T0, st);
        case LB_PREC_BF16_DEV: return launch_typed<LB_PREC_BF16_DEV>(dst, kp, rho0, T0, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbgb
