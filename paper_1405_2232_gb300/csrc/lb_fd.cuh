// lb_fd.cuh -- the finite-difference temperature treatment, Eqs. (26)-(27).
//
// The density LBE (Eq. 1 with the force of Eq. 2/4) is stepped as in the
// thermal LB path, with psi taken from a temperature field instead of the g
// populations; then T is advanced by the second-order Runge-Kutta update of
// Eq. (27) applied to Eq. (26):
//   K(T) = -u . grad T + chi (lap T + grad rho . grad T / rho),
//   lambda = rho c_v chi, chi = (tau_g - 1/2) c_s^2,
// with the isotropic central stencils of the D2Q9 lattice
//   grad phi = (1/c_s^2) sum_i w_i e_i phi(x + e_i),
//   lap phi  = (2/c_s^2) sum_i w_i (phi(x + e_i) - phi(x)),
// and rho, u (the velocity of the density LBE, with F/2) held at time n for
// both stages.  T^{n+1} = T^n + (h1 + h2)/2, h1 = K(T^n), h2 = K(T^n + a h1),
// a = 1 (Heun) or 1/2 (the form printed with Eq. 27).
//
// Kernels: k_fd_front (tile + one-site psi ring, as k_step; STEP collides and
// stores f and writes rho^n, u^n; MOMENTS writes rho, u, T), k_fd_stage (one
// RK2 stage per launch, neighbours through L1/L2), k_fd_partials (FP64
// totals of dense fields).  The FP64 mode evaluates every formula in the
// order of its printed form (compiled without contraction).
#pragma once

#include "lb_device.cuh"

namespace lbgb {

constexpr int FD_BX = 32, FD_BY = 8;

// the 9 pre-collision f of site (x, y) (pull)
template <class S>
__device__ __forceinline__ void pull9(const typename S::elem* __restrict__ src, const KParams& kp, int x,
                                      int y, typename S::real f[9]) {
    const int xm = x == 0 ? kp.nx - 1 : x - 1;
    const int xp = x == kp.nx - 1 ? 0 : x + 1;
    const long long r0 = (long long)y * kp.pitch;
    const long long rm = (long long)(y == 0 ? kp.ny - 1 : y - 1) * kp.pitch;
    const long long rp = (long long)(y == kp.ny - 1 ? 0 : y + 1) * kp.pitch;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sx = ex(i) == 1 ? xm : (ex(i) == -1 ? xp : x);
        const long long sr = ey(i) == 1 ? rm : (ey(i) == -1 ? rp : r0);
        f[i] = S::load(src + (long long)i * kp.plane + sr + sx, (typename S::real)kp.base_f[i]);
    }
}

// psi^2 (and psi) of a site with rho from f and T given
template <typename real, int BMODE>
__device__ __forceinline__ void site_psi_T(const KParams& kp, real r, real T, real& psi, real& psi2,
                                           int& flags) {
    const real Te = kp.psi_local_T ? T : (real)kp.T_psi;
    if constexpr (sizeof(real) == 8)
        psi2 = (real)2 * (p_eos<real>(kp, r, Te) - r * (real)(1.0 / 3.0)) / (real)kp.G;
    else
        psi2 = (p_eos<real>(kp, r, Te) - r * (real)(1.0 / 3.0)) * (real)kp.two_over_G;
    psi = (real)0;
    if (BMODE != BETA_ZERO) {
        if (psi2 < (real)0) flags |= 1 << LB_ERR_PSI_DOMAIN;
        psi = sqrt(psi2);
    }
    if (!isfinite(r) || !isfinite(T)) flags |= 1 << LB_ERR_NONFINITE;
}

// Density step (STEP) or moments (!STEP) of the FD treatment.
//   STEP:  f (src, pre-collision at n) -> dst (post-collision, stored at the
//          source site); rho_n, ux_n, uy_n <- rho^n, u^n.
//   !STEP: m_rho, m_ux, m_uy, m_T (FP64, any may be null) <- rho, u, T at n.
template <int PREC, int BMODE, bool STEP>
__global__ void __launch_bounds__(FD_BX* FD_BY)
    k_fd_front(const typename Store<PREC>::elem* __restrict__ src, typename Store<PREC>::elem* __restrict__ dst,
               const typename Store<PREC>::real* __restrict__ Tf, typename Store<PREC>::real* __restrict__ rho_n,
               typename Store<PREC>::real* __restrict__ ux_n, typename Store<PREC>::real* __restrict__ uy_n,
               double* __restrict__ m_rho, double* __restrict__ m_ux, double* __restrict__ m_uy,
               double* __restrict__ m_T, const KParams kp) {
    using S = Store<PREC>;
    using real = typename S::real;
    constexpr int BX = FD_BX, BY = FD_BY, WX = BX + 2, WY = BY + 2, NT = BX * BY;
    __shared__ real s_psi[BMODE != BETA_ZERO ? WX * WY : 1];
    __shared__ real s_psi2[BMODE != BETA_ONE ? WX * WY : 1];
    const int tid = threadIdx.x + threadIdx.y * BX;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    int flags = 0;
    for (int s = tid; s < WX * WY; s += NT) {
        const int ly = s / WX, lx = s - ly * WX;
        const int gx = wrapc(x0 + lx - 1, kp.nx), gy = wrapc(y0 + ly - 1, kp.ny);
        real f[9], psi, psi2;
        pull9<S>(src, kp, gx, gy, f);
        real r = f[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) r += f[i];
        site_psi_T<real, BMODE>(kp, r, Tf[(long long)gy * kp.nx + gx], psi, psi2, flags);
        if (BMODE != BETA_ZERO) s_psi[s] = psi;
        if (BMODE != BETA_ONE) s_psi2[s] = psi2;
    }
    __syncthreads();
    const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
    if (gx < kp.nx && gy < kp.ny) {
        real f[9], g[9];
        pull9<S>(src, kp, gx, gy, f);
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = (real)0;
        real rho = f[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) rho += f[i];
        real Fx, Fy, ux, uy, Tg;
        force_from_window<real, BMODE>(kp, s_psi, s_psi2, (threadIdx.y + 1) * WX + threadIdx.x + 1, WX, Fx, Fy);
        // the f half of the collision; g (zero here) is not used
        collide<real, false>(kp, f, g, rho, Fx, Fy, ux, uy, Tg);
        const long long c = (long long)gy * kp.nx + gx;
        if (STEP) {
            const long long off = (long long)gy * kp.pitch + gx;
#pragma unroll
            for (int i = 0; i < 9; ++i) S::put(dst + (long long)i * kp.plane + off, f[i], (real)kp.base_f[i]);
            rho_n[c] = rho;
            ux_n[c] = ux;
            uy_n[c] = uy;
        } else {
            if (m_rho) m_rho[c] = (double)rho;
            if (m_ux) m_ux[c] = (double)ux;
            if (m_uy) m_uy[c] = (double)uy;
            if (m_T) m_T[c] = (double)Tf[c];
        }
    } else {
        flags = 0;
    }
    if (flags) atomicOr(kp.err, flags);
}

// K(X) of Eq. (26) at (x, y) from the field X and rho, u at time n.
template <typename real>
__device__ __forceinline__ real fd_K(const real* __restrict__ X, const real* __restrict__ rho,
                                     const real* __restrict__ ux, const real* __restrict__ uy, int nx, int ny,
                                     int x, int y, real chi) {
    const long long c = (long long)y * nx + x;
    const int xe = x == nx - 1 ? 0 : x + 1, xw = x == 0 ? nx - 1 : x - 1;
    const int yn = y == ny - 1 ? 0 : y + 1, ys = y == 0 ? ny - 1 : y - 1;
    real gTx = 0, gTy = 0, grx = 0, gry = 0, lap = 0;
    const real Xc = X[c];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int nxi = ex(i) == 1 ? xe : (ex(i) == -1 ? xw : x);
        const int nyi = ey(i) == 1 ? yn : (ey(i) == -1 ? ys : y);
        const long long n = (long long)nyi * nx + nxi;
        const real w = (real)wd(i);
        const real Xn = X[n], rn = rho[n];
        gTx += w * (real)ex(i) * Xn;
        gTy += w * (real)ey(i) * Xn;
        grx += w * (real)ex(i) * rn;
        gry += w * (real)ey(i) * rn;
        lap += w * (Xn - Xc);
    }
    const real cs2 = (real)(1.0 / 3.0);
    gTx /= cs2;
    gTy /= cs2;
    grx /= cs2;
    gry /= cs2;
    lap *= (real)2 / cs2;
    return -(ux[c] * gTx + uy[c] * gTy) + chi * (lap + (grx * gTx + gry * gTy) / rho[c]);
}

// STAGE 1: h1 = K(T), Ts = T + a h1.  STAGE 2: T_next = T + (h1 + K(Ts)) / 2.
template <typename real, int STAGE>
__global__ void k_fd_stage(const real* __restrict__ T, const real* __restrict__ Ts_in,
                           const real* __restrict__ rho, const real* __restrict__ ux,
                           const real* __restrict__ uy, real* __restrict__ h1, real* __restrict__ out, int nx,
                           int ny, real chi, real a, int* err) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long c = (long long)y * nx + x;
    if (STAGE == 1) {
        const real K = fd_K<real>(T, rho, ux, uy, nx, ny, x, y, chi);
        h1[c] = K;
        out[c] = T[c] + a * K;
    } else {
        const real K = fd_K<real>(Ts_in, rho, ux, uy, nx, ny, x, y, chi);
        const real v = T[c] + (real)0.5 * (h1[c] + K);
        out[c] = v;
        if (!isfinite(v)) atomicOr(err, 1 << LB_ERR_NONFINITE);
    }
}

// T field (storage real) <- T0 (FP64)
template <typename real>
__global__ void k_fd_set_T(real* __restrict__ T, const double* __restrict__ T0, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        T[i] = (real)T0[i];
}

}  // namespace lbgb
