// lb_capi.cu -- host implementation of the C ABI declared in include/lb.h.
//
// A context owns two population buffers (ping-pong; 18 planes, 20 in the
// 16-bit modes), an error word,
// the FP64 reference fields of the steady-state residual and the partial-sum
// buffer of the deterministic totals reduction.  Every kernel runs on the
// context's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "lb.h"
#include "lb_launch.h"
#include "tensor_map.h"

using namespace lbgb;

namespace {

thread_local char g_err[512] = "";

lb_status fail(lb_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
lb_status fail(lb_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

lb_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CU(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

size_t elem_size(int prec) {
    switch (prec) {
        case LB_PREC_FP64: return 8;
        case LB_PREC_FP32: return 4;
        default: return 2;
    }
}

lb_status validate(const lb_params* p) {
    if (!p) return fail(LB_ERR_ARG, "params is NULL");
    if (p->nx < 3 || p->ny < 3) return fail(LB_ERR_ARG, "nx, ny must be >= 3 (got %d, %d)", p->nx, p->ny);
    if ((long long)p->nx * p->ny > (1LL << 31))
        return fail(LB_ERR_ARG, "lattice larger than 2^31 sites");
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5))
        return fail(LB_ERR_ARG, "tau_f and tau_g must be > 1/2 (got %g, %g)", p->tau_f, p->tau_g);
    if (!(p->G != 0.0) || !std::isfinite(p->G)) return fail(LB_ERR_ARG, "G must be finite and != 0");
    if (!std::isfinite(p->beta)) return fail(LB_ERR_ARG, "beta must be finite");
    if (!(p->cv > 0.0)) return fail(LB_ERR_ARG, "c_v must be > 0");
    if (p->eos < LB_EOS_CS || p->eos > LB_EOS_IDEAL) return fail(LB_ERR_ARG, "unknown eos %d", p->eos);
    if (p->thermal < LB_THERMAL_EQ7 || p->thermal > LB_THERMAL_FD26_PRINTED)
        return fail(LB_ERR_ARG, "unknown thermal treatment %d", p->thermal);
    if (p->precision < LB_PREC_FP64 || p->precision > LB_PREC_BF16_DEV)
        return fail(LB_ERR_ARG, "unknown precision %d", p->precision);
    if (p->walls != LB_WALLS_PERIODIC && p->walls != LB_WALLS_CAVITY && p->walls != LB_WALLS_CHANNEL)
        return fail(LB_ERR_ARG, "unknown boundary kind %d", p->walls);
    if (p->init_balanced != 0 && p->init_balanced != 1)
        return fail(LB_ERR_ARG, "init_balanced must be 0 or 1 (got %d)", p->init_balanced);
    if (p->init_balanced && (p->walls != LB_WALLS_PERIODIC || p->thermal >= LB_THERMAL_FD26))
        return fail(LB_ERR_UNSUPPORTED, "the start at rest under the force is for periodic lattice Boltzmann contexts");
    if (p->halo_rows != 0 && p->halo_rows != LB_HALO_ROWS)
        return fail(LB_ERR_ARG, "halo_rows must be 0 or %d (got %d)", LB_HALO_ROWS, p->halo_rows);
    if (p->halo_rows) {
        if (p->walls != LB_WALLS_PERIODIC || p->thermal >= LB_THERMAL_FD26)
            return fail(LB_ERR_UNSUPPORTED, "ghost-row sub-lattices are periodic lattice Boltzmann contexts");
        if (p->ny < 2 * p->halo_rows + 1)
            return fail(LB_ERR_ARG, "a sub-lattice with %d ghost rows each side needs ny >= %d", p->halo_rows,
                        2 * p->halo_rows + 1);
    }
    if (p->walls == LB_WALLS_CHANNEL) {
        if (p->precision != LB_PREC_FP64 && p->precision != LB_PREC_FP32)
            return fail(LB_ERR_UNSUPPORTED, "the channel stores FP64 or FP32");
        if ((p->tile_x || p->tile_y) && !(p->tile_x == 32 && p->tile_y == 8))
            return fail(LB_ERR_ARG, "the channel runs the 32x8 tile kernel");
        if (!std::isfinite(p->T_in) || !std::isfinite(p->T_w) || !std::isfinite(p->U_in) || p->g_grav != 0.0)
            return fail(LB_ERR_ARG, "channel inlet and plate values must be finite, g_grav 0");
    }
    if (p->walls == LB_WALLS_CAVITY) {
        if (p->precision != LB_PREC_FP64 && p->precision != LB_PREC_FP32)
            return fail(LB_ERR_UNSUPPORTED, "the cavity stores FP64 or FP32");
        if ((p->tile_x || p->tile_y) && !(p->tile_x == 32 && p->tile_y == 8))
            return fail(LB_ERR_ARG, "the cavity runs the 32x8 tile kernel");
        if (!std::isfinite(p->T_hot) || !std::isfinite(p->T_cold) || !std::isfinite(p->g_grav))
            return fail(LB_ERR_ARG, "cavity wall temperatures and gravity must be finite");
    }
    if (p->thermal >= LB_THERMAL_FD26) {
        if (p->precision != LB_PREC_FP64 && p->precision != LB_PREC_FP32)
            return fail(LB_ERR_UNSUPPORTED, "the finite-difference treatment stores FP64 or FP32 only");
        if ((p->tile_x || p->tile_y) && p->tile_y == 0 && p->tile_x != (p->precision == LB_PREC_FP64 ? 128 : 256))
            return fail(LB_ERR_ARG, "the finite-difference strip kernel is 256 (FP32) or 128 (FP64) columns wide");
        if ((p->tile_x || p->tile_y) && p->tile_y == 0 && p->nx < FD_STRIP_MIN_NX)
            return fail(LB_ERR_ARG, "the finite-difference strip kernel needs nx >= %d", FD_STRIP_MIN_NX);
    }
    if (p->tile_x || p->tile_y) {
        if (!step_tile_supported(p->tile_x, p->tile_y))
            return fail(LB_ERR_ARG, "unsupported tile %dx%d", p->tile_x, p->tile_y);
        if (p->tile_y == 0 && p->precision == LB_PREC_FP64 && p->tile_x != 128)
            return fail(LB_ERR_ARG, "the FP64 strip kernel is 128 columns wide");
        if (p->tile_y == 0) {
            const PopLayout L = pop_layout(p->precision, p->nx, p->ny, true);
            if (!strip_eligible(p->precision, p->nx, L.plane, p->tile_x))
                return fail(LB_ERR_ARG, "lattice too large for the strip kernel's 32-bit offsets");
        }
    }
    return LB_OK;
}

}  // namespace

namespace lbgb {
// Lets other translation units of the library report through lb_last_error().
lb_status record_error(lb_status st, const char* msg) { return fail(st, "%s", msg); }

bool step_tile_supported(int bx, int by) {
    return (bx == 32 && by == 8) || (bx == 32 && by == 16) || (bx == 64 && by == 4) ||
           (by == 0 && (bx == 128 || bx == 256));
}

// Final reduction of the per-CTA partials in a fixed order (one CTA).
__global__ void k_reduce_partials(const double* __restrict__ part, int nparts,
                                  double* __restrict__ out8) {
    __shared__ double s[256][8];
    const int t = threadIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = t; p < nparts; p += 256)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += part[(long long)p * 8 + k];
#pragma unroll
    for (int k = 0; k < 8; ++k) s[t][k] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w)
#pragma unroll
            for (int k = 0; k < 8; ++k) s[t][k] += s[t + w][k];
        __syncthreads();
    }
    if (t < 8) out8[t] = s[0][t];
}

}  // namespace lbgb

struct lb_ctx {
    lb_params p;
    KParams kp;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;             // every call makes this device current first
    void* alloc[2] = {nullptr, nullptr};  // population buffers as allocated
    void* buf[2] = {nullptr, nullptr};    // column 0 of row 0 of plane 0 in each
    int cur = 0;
    size_t buf_bytes = 0;                 // bytes per allocation
    int* d_err = nullptr;
    double* d_ref = nullptr;    // [2][n]: reference rho, T of the residual
    double* d_snap = nullptr;   // [2][n]: current rho, T written by lb_totals
    double* d_part = nullptr;   // [moments_grid_blocks][8]
    double* d_out8 = nullptr;   // [8]
    bool have_ref = false;
    int64_t ref_time = 0;
    int64_t t = 0;
    int nchunks = 1;            // strip kernel: row chunks per strip
    bool have_out_map = false;  // 16-bit strip contexts: out_map[b] describes buf[b]
    CUtensorMap out_map[2];
    long long pitch = 0, plane = 0;  // population layout (elements)
    // finite-difference temperature treatment (Eqs. 26-27)
    bool fd = false;
    void* Tf_alloc[2] = {nullptr, nullptr};  // T^n, T^{n+1}: one population plane each
    void* Tf[2] = {nullptr, nullptr};        // (storage real), column 0 of row 0 in each
    int tcur = 0;
    void *fd_rho = nullptr, *fd_ux = nullptr, *fd_uy = nullptr;  // rho^n, u^n, dense
    double* fd_u2 = nullptr;           // [2][n] velocity scratch of lb_totals
};

namespace {

int bmode_of(double beta) { return beta == 0.0 ? BETA_ZERO : (beta == 1.0 ? BETA_ONE : BETA_MIXED); }

KParams make_kparams(const lb_params& p, long long pitch, long long plane, int* err) {
    KParams k;
    std::memset(&k, 0, sizeof(k));
    k.nx = p.nx;
    k.ny = p.ny;
    k.pitch = pitch;
    k.plane = plane;
    k.omega_f = 1.0 / p.tau_f;
    k.omega_g = 1.0 / p.tau_g;
    k.guo_pre = 1.0 - 1.0 / (2.0 * p.tau_f);
    k.corr_pre = 1.0 - 1.0 / (2.0 * p.tau_g);
    k.G = p.G;
    k.two_over_G = 2.0 / p.G;
    k.beta = p.beta;
    k.half_1mbeta = 0.5 * (1.0 - p.beta);
    k.eos = p.eos;
    k.psi_local_T = p.psi_uses_local_T;
    k.a = p.a;
    k.b = p.b;
    k.R = p.R;
    k.cv = p.cv;
    k.inv_cv = 1.0 / p.cv;
    k.T_psi = p.T_psi;
    k.walls = p.walls;
    k.adiabatic_bottom = p.adiabatic_bottom ? 1 : 0;
    k.T_hot = p.T_hot;
    k.T_cold = p.T_cold;
    k.g_grav = p.g_grav;
    k.T_in = p.T_in;
    k.T_w = p.T_w;
    k.U_in = p.U_in;
    const bool dev = p.precision == LB_PREC_FP16_DEV || p.precision == LB_PREC_BF16_DEV;
    for (int i = 0; i < 9; ++i) {
        k.base_f[i] = dev ? (float)(wd(i) * p.rho0) : 0.0f;
        k.base_g[i] = dev ? (float)(wd(i) * p.rho0 * p.cv * p.T0) : 0.0f;
    }
    if (dev) {
        // constants of the deviation-variable collision (collide_dev): sums of
        // the stored bases (exact in double), their offsets from rho0 and
        // rho0 c_v T0, and the rounding of each base
        const double e0 = p.rho0 * p.cv * p.T0;
        double sf = 0.0, sg = 0.0;
        for (int i = 0; i < 9; ++i) {
            sf += (double)k.base_f[i];
            sg += (double)k.base_g[i];
        }
        k.sum_bf = (float)sf;
        k.sum_bg = (float)sg;
        k.dsum_f = (float)(sf - p.rho0);
        k.dsum_g = (float)(sg - e0);
        const int rep[3] = {0, 1, 5};  // rest, axis, diagonal
        for (int q = 0; q < 3; ++q) {
            k.cw_f[q] = (float)(wd(rep[q]) * p.rho0 - (double)k.base_f[rep[q]]);
            k.cw_g[q] = (float)(wd(rep[q]) * e0 - (double)k.base_g[rep[q]]);
        }
    }
    k.err = err;
    k.wait_cycles = WAIT_CYCLES_DEFAULT;
    k.halo_rows = p.halo_rows;
    kp_fill_float(k);
    return k;
}

cudaError_t dispatch_step(const lb_ctx* c, const void* src, void* dst) {
    StepLaunch L;
    L.src = src;
    L.dst = dst;
    L.kp = c->kp;
    L.eq24 = c->p.thermal == LB_THERMAL_EQ24;
    L.bmode = bmode_of(c->p.beta);
    L.bx = c->p.tile_x;
    L.by = c->p.tile_y;
    L.nchunks = c->nchunks;
    L.stream = c->stream;
    if (c->have_out_map) L.dst_map = &c->out_map[dst == c->buf[0] ? 0 : 1];
    if (c->p.walls == LB_WALLS_CHANNEL)
        return c->p.precision == LB_PREC_FP64 ? launch_step_channel_fp64(L) : launch_step_channel_fp32(L);
    if (c->kp.walls)
        return c->p.precision == LB_PREC_FP64 ? launch_step_cavity_fp64(L) : launch_step_cavity_fp32(L);
    switch (c->p.precision) {
        case LB_PREC_FP64: return launch_step_fp64(L);
        case LB_PREC_FP32: return launch_step_fp32(L);
        case LB_PREC_FP16_DEV: return launch_step_fp16(L);
        default: return launch_step_bf16(L);
    }
}

cudaError_t dispatch_moments(const lb_ctx* c, MomentsLaunch& L) {
    L.src = c->buf[c->cur];
    L.kp = c->kp;
    L.bmode = bmode_of(c->p.beta);
    L.stream = c->stream;
    switch (c->p.precision) {
        case LB_PREC_FP64: return launch_moments_fp64(L);
        case LB_PREC_FP32: return launch_moments_fp32(L);
        case LB_PREC_FP16_DEV: return launch_moments_fp16(L);
        default: return launch_moments_bf16(L);
    }
}

cudaError_t dispatch_init(const lb_ctx* c, const double* rho0, const double* T0) {
    void* d = c->buf[c->cur];
    if (c->p.init_balanced) return launch_init_balanced(c->p.precision, d, c->kp, rho0, T0, c->stream);
    switch (c->p.precision) {
        case LB_PREC_FP64: return launch_init_fp64(d, c->kp, rho0, T0, c->stream);
        case LB_PREC_FP32: return launch_init_fp32(d, c->kp, rho0, T0, c->stream);
        case LB_PREC_FP16_DEV: return launch_init_fp16(d, c->kp, rho0, T0, c->stream);
        default: return launch_init_bf16(d, c->kp, rho0, T0, c->stream);
    }
}

cudaError_t dispatch_gather(const lb_ctx* c, double* out) {
    const void* s = c->buf[c->cur];
    switch (c->p.precision) {
        case LB_PREC_FP64: return launch_gather_fp64(s, c->kp, out, c->stream);
        case LB_PREC_FP32: return launch_gather_fp32(s, c->kp, out, c->stream);
        case LB_PREC_FP16_DEV: return launch_gather_fp16(s, c->kp, out, c->stream);
        default: return launch_gather_bf16(s, c->kp, out, c->stream);
    }
}

cudaError_t dispatch_scatter(const lb_ctx* c, const double* in) {
    void* d = c->buf[c->cur];
    switch (c->p.precision) {
        case LB_PREC_FP64: return launch_scatter_fp64(d, c->kp, in, c->stream);
        case LB_PREC_FP32: return launch_scatter_fp32(d, c->kp, in, c->stream);
        case LB_PREC_FP16_DEV: return launch_scatter_fp16(d, c->kp, in, c->stream);
        default: return launch_scatter_bf16(d, c->kp, in, c->stream);
    }
}

FdLaunch fd_launch(const lb_ctx* c) {
    FdLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.kp = c->kp;
    L.bmode = bmode_of(c->p.beta);
    L.chi = (c->p.tau_g - 0.5) * (1.0 / 3.0);
    L.a = c->p.thermal == LB_THERMAL_FD26_PRINTED ? 0.5 : 1.0;
    L.stream = c->stream;
    L.src = c->buf[c->cur];
    L.T = c->Tf[c->tcur];
    L.strip = c->p.tile_y == 0;
    L.nchunks = c->nchunks;
    return L;
}

cudaError_t dispatch_fd_step(lb_ctx* c) {
    FdLaunch L = fd_launch(c);
    L.dst = c->buf[c->cur ^ 1];
    L.T_next = c->Tf[c->tcur ^ 1];
    L.rho = c->fd_rho;
    L.ux = c->fd_ux;
    L.uy = c->fd_uy;
    return c->p.precision == LB_PREC_FP64 ? launch_fd_step_fp64(L) : launch_fd_step_fp32(L);
}

cudaError_t dispatch_fd_moments(lb_ctx* c, double* rho, double* ux, double* uy, double* T) {
    FdLaunch L = fd_launch(c);
    L.m_rho = rho;
    L.m_ux = ux;
    L.m_uy = uy;
    L.m_T = T;
    return c->p.precision == LB_PREC_FP64 ? launch_fd_moments_fp64(L) : launch_fd_moments_fp32(L);
}

cudaError_t dispatch_fd_set_T(lb_ctx* c, const double* d_T0) {
    return c->p.precision == LB_PREC_FP64 ? launch_fd_set_T_fp64(c->Tf[c->tcur], d_T0, c->kp, c->stream)
                                          : launch_fd_set_T_fp32(c->Tf[c->tcur], d_T0, c->kp, c->stream);
}

void release(lb_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->alloc[0]);
    cudaFree(c->alloc[1]);
    cudaFree(c->d_err);
    cudaFree(c->d_ref);
    cudaFree(c->d_snap);
    cudaFree(c->d_part);
    cudaFree(c->d_out8);
    cudaFree(c->Tf_alloc[0]);
    cudaFree(c->Tf_alloc[1]);
    cudaFree(c->fd_rho);
    cudaFree(c->fd_ux);
    cudaFree(c->fd_uy);
    cudaFree(c->fd_u2);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// Read and clear the device error word (synchronises the stream).
lb_status check_device_error(lb_ctx* c) {
    int h = 0;
    CU(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read error word");
    CU(cudaStreamSynchronize(c->stream), "synchronize");
    if (h) {
        CU(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "clear error word");
        CU(cudaStreamSynchronize(c->stream), "synchronize");
        if (h & (1 << LB_ERR_PSI_DOMAIN))
            return fail(LB_ERR_PSI_DOMAIN,
                        "psi^2 = 2 (p_EOS - rho cs^2)/G became negative with beta != 0");
        if (h & (1 << LB_ERR_NONFINITE)) return fail(LB_ERR_NONFINITE, "rho or T became non-finite");
        if (h & (1 << LB_ERR_TIMEOUT))
            return fail(LB_ERR_TIMEOUT, "a bounded device wait of the step kernel gave up (the state is undefined)");
        return fail(LB_ERR_CUDA, "device error word 0x%x", h);
    }
    return LB_OK;
}

lb_status create(const lb_params* p, void* stream, lb_ctx** out) {
    lb_status st = validate(p);
    if (st) return st;
    if (!out) return fail(LB_ERR_ARG, "out is NULL");
    lb_ctx* c = new (std::nothrow) lb_ctx();
    if (!c) return fail(LB_ERR_OOM, "host allocation failed");
    c->p = *p;
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
        // bind the context to the stream's device
        cudaError_t e = cudaStreamGetDevice(c->stream, &c->device);
        if (e == cudaSuccess) e = cudaSetDevice(c->device);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(e, "stream device");
        }
    } else {
        cudaError_t e0 = cudaGetDevice(&c->device);
        if (e0 != cudaSuccess) {
            delete c;
            return cuda_fail(e0, "cudaGetDevice");
        }
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(e, "cudaStreamCreate");
        }
        c->own_stream = true;
    }
    const size_t es = elem_size(p->precision);
    c->fd = p->thermal >= LB_THERMAL_FD26;
    if (c->fd && c->p.tile_y != 0) {
        c->p.tile_x = FD_BX;  // the FD tile front end has one tile shape
        c->p.tile_y = FD_BY;
    }
    if (p->walls != LB_WALLS_PERIODIC) {
        c->p.tile_x = 32;  // the cavity and channel kernels' tile
        c->p.tile_y = 8;
    }
    // kernel choice: the strip-marching TMA kernel where its alignment rules
    // hold, else the tile kernel
    if (c->p.tile_x == 0 && c->p.tile_y == 0) {
        const int bx = p->precision == LB_PREC_FP64 ? 128 : 256;
        // (the FP64 finite-difference step, ALU-bound on the FP64 units, runs
        // faster as the tile front + fused RK2 pair than as the fused strip)
        if (strip_eligible(p->precision, p->nx, pop_layout(p->precision, p->nx, p->ny, true).plane, bx) &&
            (!c->fd || (p->nx >= FD_STRIP_MIN_NX && p->precision == LB_PREC_FP32))) {
            c->p.tile_x = bx;
            c->p.tile_y = 0;
        } else {
            c->p.tile_x = 32;
            c->p.tile_y = 8;
        }
    }
    const bool strip = c->p.tile_y == 0;
    const PopLayout lay = pop_layout(p->precision, p->nx, p->ny, strip);
    const long long pitch = lay.pitch, plane = lay.plane;
    c->buf_bytes = (size_t)plane * pop_planes(p->precision) * es;
    const long long n = (long long)p->nx * p->ny;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&c->alloc[0], c->buf_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->alloc[1], c->buf_bytes);
    if (e == cudaSuccess) {
        c->buf[0] = static_cast<char*>(c->alloc[0]) + lay.origin * es;
        c->buf[1] = static_cast<char*>(c->alloc[1]) + lay.origin * es;
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_ref, sizeof(double) * 2 * n);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_snap, sizeof(double) * 2 * n);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_part, sizeof(double) * 8 * moments_grid_blocks(p->nx, p->ny));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_out8, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    // zero both buffers so the padding never holds uninitialised bits
    if (e == cudaSuccess) e = cudaMemsetAsync(c->alloc[0], 0, c->buf_bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->alloc[1], 0, c->buf_bytes, c->stream);
    if (e != cudaSuccess) {
        release(c);
        return cuda_fail(e, "allocating context buffers");
    }
    if (c->fd) {
        const size_t fb = es * (size_t)n;
        const size_t tb = es * (size_t)plane;  // T in the population plane layout
        cudaError_t e2 = cudaMalloc(&c->Tf_alloc[0], tb);
        if (e2 == cudaSuccess) e2 = cudaMalloc(&c->Tf_alloc[1], tb);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(c->Tf_alloc[0], 0, tb, c->stream);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(c->Tf_alloc[1], 0, tb, c->stream);
        if (e2 == cudaSuccess) {
            c->Tf[0] = static_cast<char*>(c->Tf_alloc[0]) + lay.origin * es;
            c->Tf[1] = static_cast<char*>(c->Tf_alloc[1]) + lay.origin * es;
        }
        if (e2 == cudaSuccess) e2 = cudaMalloc(&c->fd_rho, fb);
        if (e2 == cudaSuccess) e2 = cudaMalloc(&c->fd_ux, fb);
        if (e2 == cudaSuccess) e2 = cudaMalloc(&c->fd_uy, fb);
        if (e2 == cudaSuccess) e2 = cudaMalloc(&c->fd_u2, sizeof(double) * 2 * n);
        if (e2 != cudaSuccess) {
            release(c);
            return cuda_fail(e2, "allocating the finite-difference fields");
        }
    }
    c->kp = make_kparams(c->p, pitch, plane, c->d_err);
    c->kp.ghost = strip ? (c->fd ? FD_GHOST : STRIP_GHOST) : 0;
    c->pitch = pitch;
    c->plane = plane;
    if (strip) {
        // one wave of two resident CTAs per SM: strips x chunks <= 2 x SMs
        // (chunks of at least 8 rows)
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms <= 0)
            sms = 152;
        const int strips = (p->nx + c->p.tile_x - 1) / c->p.tile_x;
        const int rows = p->ny - 2 * p->halo_rows;
        const int max_ch = rows / 8 > 0 ? rows / 8 : 1;
        int nch = (2 * sms) / strips;
        nch = nch < 1 ? 1 : (nch > max_ch ? max_ch : nch);
        c->nchunks = nch;
    }
    if (strip && !c->fd && !c->kp.walls &&
        (p->precision == LB_PREC_FP16_DEV || p->precision == LB_PREC_BF16_DEV)) {
        // the 16-bit strip kernel stores each collided row of a strip with
        // one tensor copy: dims (nx columns, ny rows, planes), box (strip
        // width, 1 row, every plane); columns past nx are clipped by the copy
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (!enc) {
            release(c);
            return fail(LB_ERR_CUDA, "the driver provides no cuTensorMapEncodeTiled");
        }
        const int npl = pop_planes(p->precision);
        const cuuint64_t dims[3] = {(cuuint64_t)p->nx, (cuuint64_t)p->ny, (cuuint64_t)npl};
        const cuuint64_t strides[2] = {(cuuint64_t)(pitch * (long long)es), (cuuint64_t)(plane * (long long)es)};
        const cuuint32_t box[3] = {(cuuint32_t)c->p.tile_x, 1, (cuuint32_t)npl};
        const cuuint32_t estr[3] = {1, 1, 1};
        for (int b = 0; b < 2; ++b) {
            if (enc(&c->out_map[b], CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, c->buf[b], dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
                release(c);
                return fail(LB_ERR_CUDA, "encoding the tensor map of population buffer %d", b);
            }
        }
        c->have_out_map = true;
    }
    *out = c;
    return LB_OK;
}

}  // namespace

extern "C" {

void lb_params_default(lb_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nx = 64;
    p->ny = 64;
    p->eos = LB_EOS_CS;
    p->thermal = LB_THERMAL_EQ24;
    p->precision = LB_PREC_FP32;
    p->psi_uses_local_T = 1;
    p->tile_x = 0;
    p->tile_y = 0;
    p->tau_f = 1.0;
    p->tau_g = 0.8;
    p->G = -1.0;
    p->beta = 1.0;
    p->a = 1.0;
    p->b = 4.0;
    p->R = 1.0;
    p->cv = 1.0;
    p->T_psi = 0.0;
    p->rho0 = 0.12;
    p->T0 = 0.075;
    p->walls = LB_WALLS_PERIODIC;
    p->T_hot = 1.03;
    p->T_cold = 0.97;
    p->g_grav = 0.0;
    p->T_in = 1.03;
    p->T_w = 0.97;
    p->U_in = 0.05;
    p->adiabatic_bottom = 0;
    p->init_balanced = 0;
    p->halo_rows = 0;
}

lb_status lb_init_device(const lb_params* p, const double* d_rho0, const double* d_T0,
                         void* stream, lb_ctx** out) {
    if (!d_rho0 || !d_T0) return fail(LB_ERR_ARG, "rho0/T0 is NULL");
    lb_ctx* c = nullptr;
    lb_status st = create(p, stream, &c);
    if (st) return st;
    cudaError_t e = dispatch_init(c, d_rho0, d_T0);
    if (e == cudaSuccess && c->fd) e = dispatch_fd_set_T(c, d_T0);
    if (e != cudaSuccess) {
        release(c);
        return cuda_fail(e, "init kernel");
    }
    *out = c;
    return LB_OK;
}

lb_status lb_init(const lb_params* p, const double* rho0, const double* T0, void* stream,
                  lb_ctx** out) {
    if (!rho0 || !T0) return fail(LB_ERR_ARG, "rho0/T0 is NULL");
    lb_ctx* c = nullptr;
    lb_status st = create(p, stream, &c);
    if (st) return st;
    const size_t bytes = sizeof(double) * (size_t)p->nx * p->ny;
    // stage the host fields in the residual reference buffer, then build the state
    cudaError_t e = cudaMemcpyAsync(c->d_ref, rho0, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_ref + (size_t)p->nx * p->ny, T0, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = dispatch_init(c, c->d_ref, c->d_ref + (size_t)p->nx * p->ny);
    if (e == cudaSuccess && c->fd) e = dispatch_fd_set_T(c, c->d_ref + (size_t)p->nx * p->ny);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        release(c);
        return cuda_fail(e, "lb_init upload");
    }
    *out = c;
    return LB_OK;
}

lb_status lb_step(lb_ctx* c, int64_t n) {
    if (!c) return fail(LB_ERR_ARG, "ctx is NULL");
    if (n < 0) return fail(LB_ERR_ARG, "n must be >= 0");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    for (int64_t k = 0; k < n; ++k) {
        cudaError_t e = c->fd ? dispatch_fd_step(c) : dispatch_step(c, c->buf[c->cur], c->buf[c->cur ^ 1]);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        c->cur ^= 1;
        if (c->fd) c->tcur ^= 1;
        c->t += 1;
    }
    return LB_OK;
}

lb_status lb_synchronize(lb_ctx* c) {
    if (!c) return fail(LB_ERR_ARG, "ctx is NULL");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    return check_device_error(c);
}

lb_status lb_moments_device(lb_ctx* c, double* d_rho, double* d_ux, double* d_uy, double* d_T) {
    if (!c) return fail(LB_ERR_ARG, "ctx is NULL");
    MomentsLaunch L;
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    std::memset(&L, 0, sizeof(L));
    L.rho = d_rho;
    L.ux = d_ux;
    L.uy = d_uy;
    L.T = d_T;
    cudaError_t e = c->fd ? dispatch_fd_moments(c, d_rho, d_ux, d_uy, d_T) : dispatch_moments(c, L);
    if (e != cudaSuccess) return cuda_fail(e, "moments kernel");
    return LB_OK;
}

lb_status lb_moments(lb_ctx* c, double* rho, double* ux, double* uy, double* T) {
    if (!c) return fail(LB_ERR_ARG, "ctx is NULL");
    const size_t n = (size_t)c->p.nx * c->p.ny;
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    double* d = nullptr;
    CU(cudaMallocAsync(&d, sizeof(double) * 4 * n, c->stream), "moments scratch");
    lb_status st = lb_moments_device(c, d, d + n, d + 2 * n, d + 3 * n);
    double* hs[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4 && st == LB_OK; ++k) {
        if (!hs[k]) continue;
        cudaError_t e = cudaMemcpyAsync(hs[k], d + k * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "moments download");
    }
    cudaFreeAsync(d, c->stream);
    lb_status st2 = check_device_error(c);
    return st ? st : st2;
}

lb_status lb_get_populations(lb_ctx* c, double* f, double* g) {
    if (!c) return fail(LB_ERR_ARG, "ctx is NULL");
    if (c->fd) return fail(LB_ERR_UNSUPPORTED, "the finite-difference treatment has no g populations");
    const size_t n = (size_t)c->p.nx * c->p.ny;
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    double* d = nullptr;
    CU(cudaMallocAsync(&d, sizeof(double) * 18 * n, c->stream), "gather scratch");
    cudaError_t e = dispatch_gather(c, d);
    if (e == cudaSuccess && f) e = cudaMemcpyAsync(f, d, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && g)
        e = cudaMemcpyAsync(g, d + 9 * n, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(d, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lb_get_populations");
    return LB_OK;
}

lb_status lb_set_populations(lb_ctx* c, const double* f, const double* g) {
    if (!c || !f || !g) return fail(LB_ERR_ARG, "NULL argument");
    if (c->fd) return fail(LB_ERR_UNSUPPORTED, "the finite-difference treatment has no g populations");
    const size_t n = (size_t)c->p.nx * c->p.ny;
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    double* d = nullptr;
    CU(cudaMallocAsync(&d, sizeof(double) * 18 * n, c->stream), "scatter scratch");
    cudaError_t e = cudaMemcpyAsync(d, f, sizeof(double) * 9 * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 9 * n, g, sizeof(double) * 9 * n, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = dispatch_scatter(c, d);
    cudaFreeAsync(d, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lb_set_populations");
    c->have_ref = false;
    return LB_OK;
}

lb_status lb_totals(lb_ctx* c, double out[LB_TOTALS_N]) {
    if (!c || !out) return fail(LB_ERR_ARG, "NULL argument");
    const size_t n = (size_t)c->p.nx * c->p.ny;
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    MomentsLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.rho = c->d_snap;
    L.T = c->d_snap + n;
    const bool use_ref = c->have_ref && c->t != c->ref_time;
    L.ref_rho = use_ref ? c->d_ref : nullptr;
    L.ref_T = use_ref ? c->d_ref + n : nullptr;
    L.part = c->d_part;
    cudaError_t e = cudaSuccess;
    if (c->fd) {
        e = dispatch_fd_moments(c, L.rho, c->fd_u2, c->fd_u2 + n, L.T);
        if (e == cudaSuccess)
            e = launch_fd_partials(L.rho, c->fd_u2, c->fd_u2 + n, L.T, L.ref_rho, L.ref_T, (long long)n, c->p.cv,
                                   c->d_part, moments_grid_blocks(c->p.nx, c->p.ny), c->stream);
    } else {
        e = dispatch_moments(c, L);
    }
    if (e != cudaSuccess) return cuda_fail(e, "totals kernel");
    k_reduce_partials<<<1, 256, 0, c->stream>>>(c->d_part, moments_grid_blocks(c->p.nx, c->p.ny), c->d_out8);
    CU(cudaGetLastError(), "reduce kernel");
    double h[8];
    CU(cudaMemcpyAsync(h, c->d_out8, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "totals download");
    lb_status st = check_device_error(c);
    if (st) return st;
    out[0] = h[0];
    out[1] = h[1];
    out[2] = h[2];
    out[3] = h[3];
    out[4] = 0.0;
    if (use_ref) {
        const double K = (double)(c->t - c->ref_time);
        const double r_rho = std::sqrt(h[4]) / (K * std::sqrt(h[5]));
        const double r_T = std::sqrt(h[6]) / (K * std::sqrt(h[7]));
        out[4] = r_rho > r_T ? r_rho : r_T;
    }
    // the snapshot just taken becomes the reference of the next call
    double* tmp = c->d_ref;
    c->d_ref = c->d_snap;
    c->d_snap = tmp;
    c->have_ref = true;
    c->ref_time = c->t;
    return LB_OK;
}

lb_status lb_state_size(const lb_ctx* c, size_t* bytes) {
    if (!c || !bytes) return fail(LB_ERR_ARG, "NULL argument");
    if (c->fd) return fail(LB_ERR_UNSUPPORTED, "the finite-difference treatment has no g populations");
    *bytes = c->buf_bytes + sizeof(int64_t);
    return LB_OK;
}

lb_status lb_save_state(lb_ctx* c, void* host_blob) {
    if (!c || !host_blob) return fail(LB_ERR_ARG, "NULL argument");
    if (c->fd) return fail(LB_ERR_UNSUPPORTED, "the finite-difference treatment has no g populations");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    CU(cudaMemcpyAsync(host_blob, c->alloc[c->cur], c->buf_bytes, cudaMemcpyDeviceToHost, c->stream), "save state");
    CU(cudaStreamSynchronize(c->stream), "synchronize");
    std::memcpy(static_cast<char*>(host_blob) + c->buf_bytes, &c->t, sizeof(int64_t));
    return LB_OK;
}

lb_status lb_load_state(lb_ctx* c, const void* host_blob) {
    if (!c || !host_blob) return fail(LB_ERR_ARG, "NULL argument");
    if (c->fd) return fail(LB_ERR_UNSUPPORTED, "the finite-difference treatment has no g populations");
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    CU(cudaMemcpyAsync(c->alloc[c->cur], host_blob, c->buf_bytes, cudaMemcpyHostToDevice, c->stream), "load state");
    CU(cudaStreamSynchronize(c->stream), "synchronize");
    std::memcpy(&c->t, static_cast<const char*>(host_blob) + c->buf_bytes, sizeof(int64_t));
    c->have_ref = false;
    return LB_OK;
}

int64_t lb_time(const lb_ctx* c) { return c ? c->t : -1; }

lb_status lb_halo_bytes(const lb_ctx* c, size_t* bytes) {
    if (!c || !bytes) return fail(LB_ERR_ARG, "NULL argument");
    if (!c->p.halo_rows) return fail(LB_ERR_ARG, "the context has no ghost rows (halo_rows == 0)");
    *bytes = (size_t)pop_planes(c->p.precision) * c->p.halo_rows * c->pitch * elem_size(c->p.precision);
    return LB_OK;
}

namespace {
// Whole rows [r0, r0 + H) of every plane of the current buffer <-> a dense
// [planes][H][pitch] device buffer (ghost columns included), one 2D copy.
lb_status halo_copy(lb_ctx* c, int32_t face, void* d_buf, bool pack) {
    if (!c || !d_buf) return fail(LB_ERR_ARG, "NULL argument");
    if (!c->p.halo_rows) return fail(LB_ERR_ARG, "the context has no ghost rows (halo_rows == 0)");
    if (face != 0 && face != 1) return fail(LB_ERR_ARG, "face must be 0 (lower) or 1 (upper)");
    const int H = c->p.halo_rows, ny = c->p.ny;
    // pack: the first (face 0) or last (face 1) H updated rows; unpack: the
    // lower (face 0) or upper (face 1) ghost rows
    const int r0 = pack ? (face == 0 ? H : ny - 2 * H) : (face == 0 ? 0 : ny - H);
    const size_t es = elem_size(c->p.precision);
    char* rows = static_cast<char*>(c->alloc[c->cur]) + (size_t)r0 * c->pitch * es;
    const size_t width = (size_t)H * c->pitch * es, spitch = (size_t)c->plane * es;
    const int planes = pop_planes(c->p.precision);
    CU(cudaSetDevice(c->device), "cudaSetDevice");
    cudaError_t e = pack ? cudaMemcpy2DAsync(d_buf, width, rows, spitch, width, planes, cudaMemcpyDeviceToDevice,
                                             c->stream)
                         : cudaMemcpy2DAsync(rows, spitch, d_buf, width, width, planes, cudaMemcpyDeviceToDevice,
                                             c->stream);
    if (e != cudaSuccess) return cuda_fail(e, pack ? "lb_halo_pack" : "lb_halo_unpack");
    return LB_OK;
}
}  // namespace

lb_status lb_halo_pack(lb_ctx* c, int32_t face, void* d_buf) { return halo_copy(c, face, d_buf, true); }

lb_status lb_halo_unpack(lb_ctx* c, int32_t face, const void* d_buf) {
    return halo_copy(c, face, const_cast<void*>(d_buf), false);
}

lb_status lb_set_wait_limit(lb_ctx* c, int64_t cycles) {
    if (!c) return fail(LB_ERR_ARG, "ctx is NULL");
    if (cycles < 0) return fail(LB_ERR_ARG, "cycles must be >= 0 (0 restores the default)");
    c->kp.wait_cycles = cycles == 0 ? WAIT_CYCLES_DEFAULT : (long long)cycles;
    return LB_OK;
}

lb_status lb_get_params(const lb_ctx* c, lb_params* out) {
    if (!c || !out) return fail(LB_ERR_ARG, "NULL argument");
    *out = c->p;
    return LB_OK;
}

lb_status lb_free(lb_ctx* c) {
    release(c);
    return LB_OK;
}

const char* lb_last_error(void) { return g_err; }

const char* lb_version(void) { return "lbgb 0.1 (sm_103a)"; }

}  // extern "C"
