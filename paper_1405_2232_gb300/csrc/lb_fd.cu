// lb_fd.cu -- precision-independent part of the finite-difference temperature
// treatment: FP64 totals of dense moment fields (see lb_fd.cuh).
#include <cuda_runtime.h>

#include "lb_launch.h"

namespace lbgb {

__global__ void __launch_bounds__(256) k_fd_partials(const double* __restrict__ rho, const double* __restrict__ ux,
                                                      const double* __restrict__ uy, const double* __restrict__ T,
                                                      const double* __restrict__ ref_rho,
                                                      const double* __restrict__ ref_T, long long n, double cv,
                                                      double* __restrict__ part) {
    __shared__ double red[8][256];
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long s0 = (long long)blockIdx.x * per;
    const long long s1 = s0 + per < n ? s0 + per : n;
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long s = s0 + threadIdx.x; s < s1; s += 256) {
        const double r = rho[s], t = T[s];
        a[0] += r;
        a[1] += r * cv * t;
        a[2] += r * ux[s];
        a[3] += r * uy[s];
        if (ref_rho) {
            const double dr = r - ref_rho[s], dt = t - ref_T[s];
            a[4] += dr * dr;
            a[6] += dt * dt;
        }
        a[5] += r * r;
        a[7] += t * t;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 8; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 8) part[(long long)blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x][0];
}

cudaError_t launch_fd_partials(const double* rho, const double* ux, const double* uy, const double* T,
                               const double* ref_rho, const double* ref_T, long long n, double cv,
                               double* part, int blocks, cudaStream_t st) {
    k_fd_partials<<<blocks, 256, 0, st>>>(rho, ux, uy, T, ref_rho, ref_T, n, cv, part);
    return cudaGetLastError();
}

}  // namespace lbgb
