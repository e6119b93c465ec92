// lb_noalloc.cu -- an allocation-free variant of the deterministic FP64 totals
// reduction (lb_field_totals_noalloc in include/lb.h).
//
// The context-based lb_totals keeps its per-CTA partial sums in a buffer the
// library allocates with cudaMalloc when the context is created.  Some callers
// cannot allow any device allocation behind their back: code that runs while a
// stream is being captured in a mode that forbids allocation, applications that
// hand every byte of device memory to their own pool, or embedders whose memory
// budget must be fixed before the run starts.  For them this variant keeps the
// partials in one file-scope device array of fixed size instead, and reduces
// fields the caller already holds in device memory.
//
// The array (NA_MAX_BLOCKS x 8 doubles = 256 KB) is part of the library image:
// every GPU that loads the library holds it until the process exits.  All calls
// share it; a call overwrites every entry it later reads, so nothing has to be
// cleared between calls, but calls that overlap on the GPU (different streams,
// or a second call before the first finished) race on it.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "lb.h"

namespace lbgb {
lb_status record_error(lb_status st, const char* msg);
}

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_SITES_PER_THREAD = 16;
constexpr int NA_SITES_PER_BLOCK = NA_THREADS * NA_SITES_PER_THREAD;  // 4096
constexpr int NA_MAX_BLOCKS = 4096;
constexpr long long NA_MAX_SITES = (long long)NA_MAX_BLOCKS * NA_SITES_PER_BLOCK;  // 4096^2

// the scratch: per-CTA partial sums, 8 doubles each
__device__ __align__(256) double g_na_partials[NA_MAX_BLOCKS * 8];

// Per-CTA partials: mass, energy, rho ux, rho uy, |d rho|^2, rho^2, |dT|^2, T^2,
// each thread summing its 16 sites in a fixed order, then a fixed tree.
__global__ void __launch_bounds__(NA_THREADS)
    k_na_partials(long long n, double cv, const double* __restrict__ rho, const double* __restrict__ ux,
                  const double* __restrict__ uy, const double* __restrict__ T,
                  const double* __restrict__ ref_rho, const double* __restrict__ ref_T,
                  double* __restrict__ part) {
    __shared__ double s_red[NA_THREADS / 32][8];
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long base = (long long)blockIdx.x * NA_SITES_PER_BLOCK + threadIdx.x;
#pragma unroll 4
    for (int k = 0; k < NA_SITES_PER_THREAD; ++k) {
        const long long s = base + (long long)k * NA_THREADS;
        if (s >= n) break;
        const double r = rho[s], t = T[s];
        v[0] += r;
        v[1] += r * cv * t;
        v[2] += r * ux[s];
        v[3] += r * uy[s];
        if (ref_rho) {
            const double a = r - ref_rho[s], b = t - ref_T[s];
            v[4] += a * a;
            v[6] += b * b;
        }
        v[5] += r * r;
        v[7] += t * t;
    }
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((tid & 31) == 0) s_red[tid >> 5][q] = x;
    }
    __syncthreads();
    if (tid < 8) {
        double x = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) x += s_red[w][tid];
        part[(long long)blockIdx.x * 8 + tid] = x;
    }
}

// One CTA folds the partials in a fixed order and writes the five totals.
__global__ void __launch_bounds__(NA_THREADS)
    k_na_final(const double* __restrict__ part, int nblocks, long long K, int have_ref,
               double* __restrict__ out) {
    __shared__ double s[NA_THREADS][8];
    const int t = threadIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = t; p < nblocks; p += NA_THREADS)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] += part[(long long)p * 8 + q];
#pragma unroll
    for (int q = 0; q < 8; ++q) s[t][q] = acc[q];
    __syncthreads();
    for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
        if (t < w)
#pragma unroll
            for (int q = 0; q < 8; ++q) s[t][q] += s[t + w][q];
        __syncthreads();
    }
    if (t == 0) {
        out[0] = s[0][0];
        out[1] = s[0][1];
        out[2] = s[0][2];
        out[3] = s[0][3];
        double r = 0.0;
        if (have_ref) {
            const double r_rho = sqrt(s[0][4]) / ((double)K * sqrt(s[0][5]));
            const double r_T = sqrt(s[0][6]) / ((double)K * sqrt(s[0][7]));
            r = r_rho > r_T ? r_rho : r_T;
        }
        out[4] = r;
    }
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached.  The cache assumes the device is not reset
// (cudaDeviceReset) while the library is loaded.
std::mutex g_na_mu;
double* g_na_addr[64] = {};

lb_status na_scratch(int dev, double** out) {
    if (dev < 0 || dev >= 64) return lbgb::record_error(LB_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_partials);
        if (e != cudaSuccess || !p) {
            char msg[160];
            std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the reduction scratch: %s",
                          cudaGetErrorString(e));
            return lbgb::record_error(LB_ERR_CUDA, msg);
        }
        g_na_addr[dev] = static_cast<double*>(p);
    }
    *out = g_na_addr[dev];
    return LB_OK;
}

}  // namespace

extern "C" lb_status lb_field_totals_noalloc(int32_t nx, int32_t ny, double cv, const double* d_rho,
                                            const double* d_ux, const double* d_uy,
                                            const double* d_T, const double* d_ref_rho,
                                            const double* d_ref_T, int64_t K, double* d_out,
                                            void* stream) {
    if (nx < 1 || ny < 1) return lbgb::record_error(LB_ERR_ARG, "nx and ny must be >= 1");
    const long long n = (long long)nx * ny;
    if (n > NA_MAX_SITES) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "lattice of %lld sites exceeds the %lld-site limit of the allocation-free "
                      "reduction (use lb_totals)",
                      n, NA_MAX_SITES);
        return lbgb::record_error(LB_ERR_ARG, msg);
    }
    if (!d_rho || !d_ux || !d_uy || !d_T || !d_out)
        return lbgb::record_error(LB_ERR_ARG, "field or output pointer is NULL");
    const bool have_ref = d_ref_rho && d_ref_T;
    if ((d_ref_rho != nullptr) != (d_ref_T != nullptr))
        return lbgb::record_error(LB_ERR_ARG, "give both reference fields or neither");
    if (have_ref && K <= 0) return lbgb::record_error(LB_ERR_ARG, "K must be > 0 with reference fields");
    if (!(cv > 0.0)) return lbgb::record_error(LB_ERR_ARG, "c_v must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the work runs on the stream's device; the caller's current device is
    // restored before returning
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return lbgb::record_error(LB_ERR_CUDA, cudaGetErrorString(e));
    int dev = prev;
    if (st) e = cudaStreamGetDevice(st, &dev);
    if (e == cudaSuccess && dev != prev) e = cudaSetDevice(dev);
    if (e != cudaSuccess) return lbgb::record_error(LB_ERR_CUDA, cudaGetErrorString(e));
    double* part = nullptr;
    lb_status ls = na_scratch(dev, &part);
    if (ls == LB_OK) {
        const int nblocks = (int)((n + NA_SITES_PER_BLOCK - 1) / NA_SITES_PER_BLOCK);
        k_na_partials<<<nblocks, NA_THREADS, 0, st>>>(n, cv, d_rho, d_ux, d_uy, d_T,
                                                      have_ref ? d_ref_rho : nullptr,
                                                      have_ref ? d_ref_T : nullptr, part);
        k_na_final<<<1, NA_THREADS, 0, st>>>(part, nblocks, (long long)K, have_ref ? 1 : 0, d_out);
        e = cudaGetLastError();
        if (e != cudaSuccess) ls = lbgb::record_error(LB_ERR_CUDA, cudaGetErrorString(e));
    }
    if (dev != prev) {
        e = cudaSetDevice(prev);
        if (e != cudaSuccess && ls == LB_OK) ls = lbgb::record_error(LB_ERR_CUDA, cudaGetErrorString(e));
    }
    return ls;
}
