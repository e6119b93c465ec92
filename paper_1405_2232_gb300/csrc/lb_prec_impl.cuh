// lb_prec_impl.cuh -- instantiates the kernels of one storage precision.
// Included by lb_prec_<name>.cu after defining LBGB_PREC (an LB_PREC_*
// value) and LBGB_NAME (the suffix of the launch functions).
#pragma once

#include "lb_cavity.cuh"
#include "lb_fd.cuh"
#include "lb_fd_strip.cuh"
#include "lb_launch.h"
#include "lb_step_strip.cuh"
#include "lb_step_strip_dev.cuh"

namespace lbgb {

#define LBGB_CAT2(a, b) a##b
#define LBGB_CAT(a, b) LBGB_CAT2(a, b)

namespace {

template <int BX, int BY>
cudaError_t step_tile(const StepLaunch& L) {
    using E = typename Store<LBGB_PREC>::elem;
    const dim3 block(BX, BY);
    const dim3 grid((L.kp.nx + BX - 1) / BX, (L.kp.ny - 2 * L.kp.halo_rows + BY - 1) / BY);
    const E* src = static_cast<const E*>(L.src);
    E* dst = static_cast<E*>(L.dst);
    if (L.eq24) {
        switch (L.bmode) {
            case BETA_ZERO: k_step<LBGB_PREC, BX, BY, true, BETA_ZERO><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
            case BETA_ONE: k_step<LBGB_PREC, BX, BY, true, BETA_ONE><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
            default: k_step<LBGB_PREC, BX, BY, true, BETA_MIXED><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
        }
    } else {
        switch (L.bmode) {
            case BETA_ZERO: k_step<LBGB_PREC, BX, BY, false, BETA_ZERO><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
            case BETA_ONE: k_step<LBGB_PREC, BX, BY, false, BETA_ONE><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
            default: k_step<LBGB_PREC, BX, BY, false, BETA_MIXED><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
        }
    }
    return cudaGetLastError();
}

// Everything in this anonymous namespace depends on LBGB_PREC without carrying
// it as a template argument, so it must have internal linkage: each precision
// translation unit gets its own copy (shared weak symbols would let the linker
// pick one precision's launcher for all).

// Stage count per strip width: the deepest ring that still lets two CTAs
// share an SM (228 KB of shared memory).  The 16-bit kernel also holds
// DEV_OUT_BUFS row buffers of the collided rows and a six-row psi ring.
template <int BX>
constexpr int strip_stages() {
    using C = StripCfg<LBGB_PREC>;
    constexpr int NPL = Store<LBGB_PREC>::NPLANES;
    constexpr size_t stage = (size_t)NPL * (BX + 2 * C::HALO) * C::ES;
    constexpr bool DEV = Store<LBGB_PREC>::SPLIT;
    constexpr size_t ring = (size_t)(DEV ? 2 * DEV_PSI_ROWS : 8) * (BX + 2) * sizeof(typename C::real);
    constexpr size_t out = DEV ? (size_t)DEV_OUT_BUFS * NPL * BX * C::ES : 0;
    constexpr size_t budget = 110 * 1024 - 32 - (DEV ? (2 * 12 + 2) * 8 : 0);
    constexpr size_t s = (budget - ring - out) / stage;
    return s > 12 ? 12 : (int)s;
}

// 16-bit deviation storage: k_step_strip_dev; FP32 / FP64: k_step_strip.
template <int BX, int ST, bool EQ24, int BM>
auto strip_kernel() {
    if constexpr (Store<LBGB_PREC>::SPLIT)
        return k_step_strip_dev<LBGB_PREC, BX, ST, EQ24, BM>;
    else
        return k_step_strip<LBGB_PREC, BX, ST, EQ24, BM>;
}

template <int BX, bool EQ24, int BM>
cudaError_t strip_launch(const StepLaunch& L) {
    using E = typename Store<LBGB_PREC>::elem;
    constexpr int ST = strip_stages<BX>();
    static_assert(ST >= 3, "strip kernel needs at least three stages");
    constexpr bool DEV = Store<LBGB_PREC>::SPLIT;
    constexpr size_t smem =
        DEV ? strip_dev_smem_bytes<LBGB_PREC, BX, ST>() : strip_smem_bytes<LBGB_PREC, BX, ST>();
    static_assert(smem <= 110 * 1024, "two CTAs per SM");
    auto kern = strip_kernel<BX, ST, EQ24, BM>();
    static unsigned long long configured = 0;  // per instantiation, one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !(configured >> dev & 1ULL)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) configured |= 1ULL << dev;
    }
    const dim3 grid((L.kp.nx + BX - 1) / BX, L.nchunks);
    if constexpr (DEV) {
        if (!L.dst_map) return cudaErrorInvalidValue;  // the kernel stores through it
        kern<<<grid, strip_threads<BX>(), smem, L.stream>>>(static_cast<const E*>(L.src), static_cast<E*>(L.dst),
                                                             L.kp, L.nchunks, *L.dst_map);
    } else {
        kern<<<grid, strip_threads<BX>(), smem, L.stream>>>(static_cast<const E*>(L.src), static_cast<E*>(L.dst),
                                                             L.kp, L.nchunks);
    }
    return cudaGetLastError();
}

template <int BX>
cudaError_t step_strip(const StepLaunch& L) {
    if (L.eq24) {
        switch (L.bmode) {
            case BETA_ZERO: return strip_launch<BX, true, BETA_ZERO>(L);
            case BETA_ONE: return strip_launch<BX, true, BETA_ONE>(L);
            default: return strip_launch<BX, true, BETA_MIXED>(L);
        }
    }
    switch (L.bmode) {
        case BETA_ZERO: return strip_launch<BX, false, BETA_ZERO>(L);
        case BETA_ONE: return strip_launch<BX, false, BETA_ONE>(L);
        default: return strip_launch<BX, false, BETA_MIXED>(L);
    }
}

}  // namespace

cudaError_t LBGB_CAT(launch_step_, LBGB_NAME)(const StepLaunch& L) {
    if (L.by == 0) {
        if (L.bx == 128) return step_strip<128>(L);
        // (LB_PREC_* are enum constants, invisible to the preprocessor)
        if constexpr (LBGB_PREC != LB_PREC_FP64) {
            if (L.bx == 256) return step_strip<256>(L);
        }
        return cudaErrorInvalidValue;
    }
    if (L.bx == 32 && L.by == 8) return step_tile<32, 8>(L);
    if (L.bx == 32 && L.by == 16) return step_tile<32, 16>(L);
    if (L.bx == 64 && L.by == 4) return step_tile<64, 4>(L);
    return cudaErrorInvalidValue;
}

cudaError_t LBGB_CAT(launch_moments_, LBGB_NAME)(const MomentsLaunch& L) {
    using E = typename Store<LBGB_PREC>::elem;
    const dim3 block(MOM_BX, MOM_BY);
    const dim3 grid((L.kp.nx + MOM_BX - 1) / MOM_BX, (L.kp.ny + MOM_BY - 1) / MOM_BY);
    const E* src = static_cast<const E*>(L.src);
    switch (L.bmode) {
        case BETA_ZERO:
            k_moments<LBGB_PREC, MOM_BX, MOM_BY, BETA_ZERO><<<grid, block, 0, L.stream>>>(
                src, L.kp, L.rho, L.ux, L.uy, L.T, L.ref_rho, L.ref_T, L.part);
            break;
        case BETA_ONE:
            k_moments<LBGB_PREC, MOM_BX, MOM_BY, BETA_ONE><<<grid, block, 0, L.stream>>>(
                src, L.kp, L.rho, L.ux, L.uy, L.T, L.ref_rho, L.ref_T, L.part);
            break;
        default:
            k_moments<LBGB_PREC, MOM_BX, MOM_BY, BETA_MIXED><<<grid, block, 0, L.stream>>>(
                src, L.kp, L.rho, L.ux, L.uy, L.T, L.ref_rho, L.ref_T, L.part);
            break;
    }
    return cudaGetLastError();
}

namespace {
int elementwise_blocks(const KParams& kp) {
    const long long n = (long long)kp.nx * kp.ny;
    long long b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}
}  // namespace

cudaError_t LBGB_CAT(launch_init_, LBGB_NAME)(void* dst, const KParams& kp, const double* rho0,
                                             const double* T0, cudaStream_t st) {
    using E = typename Store<LBGB_PREC>::elem;
    k_init<LBGB_PREC><<<elementwise_blocks(kp), 256, 0, st>>>(static_cast<E*>(dst), kp, rho0, T0);
    return cudaGetLastError();
}

cudaError_t LBGB_CAT(launch_gather_, LBGB_NAME)(const void* src, const KParams& kp, double* out,
                                               cudaStream_t st) {
    using E = typename Store<LBGB_PREC>::elem;
    k_gather<LBGB_PREC><<<elementwise_blocks(kp), 256, 0, st>>>(static_cast<const E*>(src), kp, out);
    return cudaGetLastError();
}

cudaError_t LBGB_CAT(launch_scatter_, LBGB_NAME)(void* dst, const KParams& kp, const double* in,
                                                cudaStream_t st) {
    using E = typename Store<LBGB_PREC>::elem;
    k_scatter<LBGB_PREC><<<elementwise_blocks(kp), 256, 0, st>>>(static_cast<E*>(dst), kp, in);
    return cudaGetLastError();
}

// ------------------------------------------------ cavity (Sec. III B)
cudaError_t LBGB_CAT(launch_step_cavity_, LBGB_NAME)(const StepLaunch& L) {
    if constexpr (LBGB_PREC != LB_PREC_FP64 && LBGB_PREC != LB_PREC_FP32) {
        return cudaErrorNotSupported;
    } else {
        using E = typename Store<LBGB_PREC>::elem;
        const dim3 block(CAV_BX, CAV_BY);
        const dim3 grid((L.kp.nx + CAV_BX - 1) / CAV_BX, (L.kp.ny + CAV_BY - 1) / CAV_BY);
        const E* src = static_cast<const E*>(L.src);
        E* dst = static_cast<E*>(L.dst);
        if (L.eq24) {
            switch (L.bmode) {
                case BETA_ZERO: k_step_cavity<LBGB_PREC, true, BETA_ZERO><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
                case BETA_ONE: k_step_cavity<LBGB_PREC, true, BETA_ONE><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
                default: k_step_cavity<LBGB_PREC, true, BETA_MIXED><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
            }
        } else {
            switch (L.bmode) {
                case BETA_ZERO: k_step_cavity<LBGB_PREC, false, BETA_ZERO><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
                case BETA_ONE: k_step_cavity<LBGB_PREC, false, BETA_ONE><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
                default: k_step_cavity<LBGB_PREC, false, BETA_MIXED><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
            }
        }
        return cudaGetLastError();
    }
}

// ------------------------------------------------ channel (Sec. III A)
cudaError_t LBGB_CAT(launch_step_channel_, LBGB_NAME)(const StepLaunch& L) {
    if constexpr (LBGB_PREC != LB_PREC_FP64 && LBGB_PREC != LB_PREC_FP32) {
        return cudaErrorNotSupported;
    } else {
        using E = typename Store<LBGB_PREC>::elem;
        const dim3 block(CAV_BX, CAV_BY);
        const dim3 grid((L.kp.nx + CAV_BX - 1) / CAV_BX, (L.kp.ny + CAV_BY - 1) / CAV_BY);
        const E* src = static_cast<const E*>(L.src);
        E* dst = static_cast<E*>(L.dst);
        if (L.eq24) {
            switch (L.bmode) {
                case BETA_ZERO: k_step_channel<LBGB_PREC, true, BETA_ZERO><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
                case BETA_ONE: k_step_channel<LBGB_PREC, true, BETA_ONE><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
                default: k_step_channel<LBGB_PREC, true, BETA_MIXED><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
            }
        } else {
            switch (L.bmode) {
                case BETA_ZERO: k_step_channel<LBGB_PREC, false, BETA_ZERO><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
                case BETA_ONE: k_step_channel<LBGB_PREC, false, BETA_ONE><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
                default: k_step_channel<LBGB_PREC, false, BETA_MIXED><<<grid, block, 0, L.stream>>>(src, dst, L.kp); break;
            }
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_channel_outlet<LBGB_PREC><<<(L.kp.ny + 127) / 128, 128, 0, L.stream>>>(dst, L.kp);
        return cudaGetLastError();
    }
}

// ------------------------------------------------ finite-difference T (Eqs. 26-27)
namespace {
constexpr bool kFdSupported = LBGB_PREC == LB_PREC_FP64 || LBGB_PREC == LB_PREC_FP32;

// The whole FD step on a strip context (k_fd_fused).
template <int BM>
cudaError_t fd_fused_launch(const FdLaunch& L) {
    using S = Store<LBGB_PREC>;
    using E = typename S::elem;
    using R = typename S::real;
    constexpr int BX = LBGB_PREC == LB_PREC_FP64 ? 128 : 256;
    constexpr int ST = fd_fused_stages<LBGB_PREC, BX>();
    static_assert(ST >= 3, "FD strip kernel needs at least three stages");
    constexpr size_t smem = fd_fused_smem_bytes<LBGB_PREC, BX, ST>();
    auto kern = k_fd_fused<LBGB_PREC, BX, ST, BM>;
    static unsigned long long configured = 0;  // per instantiation, one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !(configured >> dev & 1ULL)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) configured |= 1ULL << dev;
    }
    const dim3 grid((L.kp.nx + BX - 1) / BX, L.nchunks);
    kern<<<grid, strip_threads<BX>(), smem, L.stream>>>(static_cast<const E*>(L.src), static_cast<E*>(L.dst),
                                                         static_cast<const R*>(L.T), static_cast<R*>(L.T_next),
                                                         L.kp, L.nchunks, (R)L.chi, (R)L.a);
    return cudaGetLastError();
}

template <bool STEP>
cudaError_t fd_front(const FdLaunch& L) {
    if constexpr (!kFdSupported) {
        return cudaErrorNotSupported;
    } else {
        using S = Store<LBGB_PREC>;
        using E = typename S::elem;
        using R = typename S::real;
        const dim3 block(FD_BX, FD_BY);
        const dim3 grid((L.kp.nx + FD_BX - 1) / FD_BX, (L.kp.ny + FD_BY - 1) / FD_BY);
        const E* src = static_cast<const E*>(L.src);
        E* dst = static_cast<E*>(L.dst);
        const R* T = static_cast<const R*>(L.T);
        R *rho = static_cast<R*>(L.rho), *ux = static_cast<R*>(L.ux), *uy = static_cast<R*>(L.uy);
        switch (L.bmode) {
            case BETA_ZERO:
                k_fd_front<LBGB_PREC, BETA_ZERO, STEP><<<grid, block, 0, L.stream>>>(src, dst, T, rho, ux, uy, L.m_rho,
                                                                                   L.m_ux, L.m_uy, L.m_T, L.kp);
                break;
            case BETA_ONE:
                k_fd_front<LBGB_PREC, BETA_ONE, STEP><<<grid, block, 0, L.stream>>>(src, dst, T, rho, ux, uy, L.m_rho,
                                                                                  L.m_ux, L.m_uy, L.m_T, L.kp);
                break;
            default:
                k_fd_front<LBGB_PREC, BETA_MIXED, STEP><<<grid, block, 0, L.stream>>>(src, dst, T, rho, ux, uy,
                                                                                    L.m_rho, L.m_ux, L.m_uy, L.m_T, L.kp);
                break;
        }
        return cudaGetLastError();
    }
}
}  // namespace

cudaError_t LBGB_CAT(launch_fd_step_, LBGB_NAME)(const FdLaunch& L) {
    if constexpr (!kFdSupported) {
        return cudaErrorNotSupported;
    } else {
        using R = typename Store<LBGB_PREC>::real;
        if (L.strip) {
            switch (L.bmode) {
                case BETA_ZERO: return fd_fused_launch<BETA_ZERO>(L);
                case BETA_ONE: return fd_fused_launch<BETA_ONE>(L);
                default: return fd_fused_launch<BETA_MIXED>(L);
            }
        }
        cudaError_t e = fd_front<true>(L);
        if (e != cudaSuccess) return e;
        const dim3 block(FDR_BX, FDR_BY);
        const dim3 grid((L.kp.nx + FDR_BX - 1) / FDR_BX, (L.kp.ny + FDR_BY * FDR_ROWS - 1) / (FDR_BY * FDR_ROWS));
        k_fd_rk2<R><<<grid, block, 0, L.stream>>>(static_cast<const R*>(L.T), static_cast<const R*>(L.rho),
                                                  static_cast<const R*>(L.ux), static_cast<const R*>(L.uy),
                                                  static_cast<R*>(L.T_next), L.kp, (R)L.chi, (R)L.a);
        return cudaGetLastError();
    }
}

cudaError_t LBGB_CAT(launch_fd_moments_, LBGB_NAME)(const FdLaunch& L) { return fd_front<false>(L); }

cudaError_t LBGB_CAT(launch_fd_set_T_, LBGB_NAME)(void* T, const double* T0, const KParams& kp, cudaStream_t st) {
    if constexpr (!kFdSupported) {
        return cudaErrorNotSupported;
    } else {
        using R = typename Store<LBGB_PREC>::real;
        const long long n = (long long)kp.nx * kp.ny;
        long long b = (n + 255) / 256;
        k_fd_set_T<R><<<(int)(b < 2432 ? (b < 1 ? 1 : b) : 2432), 256, 0, st>>>(static_cast<R*>(T), T0, kp);
        return cudaGetLastError();
    }
}

}  // namespace lbgb
