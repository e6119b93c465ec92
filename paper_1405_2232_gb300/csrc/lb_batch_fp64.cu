// FP64 kernels of the batched solver.  Compiled without FMA contraction, like
// the FP64 single-lattice kernels, so a batch evolves each domain bit for bit
// as the printed formulas evaluated in order do.
#include <cuda_runtime.h>

#include "lb.h"
#include "lb_batch_device.cuh"

namespace lbgb {

cudaError_t launch_batch_step_fp64(const void* src, void* dst, const BatchDomain* doms,
                                   const BatchItem* items, const int* n_items, int* next_item, int eq24,
                                   int bmode, int grid, cudaStream_t stream) {
    using E = double;
    constexpr int BX = 128, ST = batch_stages<LB_PREC_FP64, BX>();
    constexpr size_t smem = batch_smem_bytes<LB_PREC_FP64, BX, ST>();
    void (*k)(const E*, E*, const BatchDomain*, const BatchItem*, const int*, int*);
    if (eq24)
        k = bmode == BETA_ZERO  ? k_batch_step<LB_PREC_FP64, BX, ST, true, BETA_ZERO>
            : bmode == BETA_ONE ? k_batch_step<LB_PREC_FP64, BX, ST, true, BETA_ONE>
                                : k_batch_step<LB_PREC_FP64, BX, ST, true, BETA_MIXED>;
    else
        k = bmode == BETA_ZERO  ? k_batch_step<LB_PREC_FP64, BX, ST, false, BETA_ZERO>
            : bmode == BETA_ONE ? k_batch_step<LB_PREC_FP64, BX, ST, false, BETA_ONE>
                                : k_batch_step<LB_PREC_FP64, BX, ST, false, BETA_MIXED>;
    // src == nullptr: set the shared-memory attribute only (once, outside capture)
    if (!src) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, strip_threads<BX>(), smem, stream>>>(static_cast<const E*>(src), static_cast<E*>(dst), doms,
                                                   items, n_items, next_item);
    return cudaGetLastError();
}

}  // namespace lbgb
