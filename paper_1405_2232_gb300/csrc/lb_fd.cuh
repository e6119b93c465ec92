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
// stores f and writes rho^n, u^n; MOMENTS writes rho, u, T), and in
// lb_fd_strip.cuh k_fd_fused (the whole step in one pass on strip contexts)
// and k_fd_rk2 (both RK2 stages in one launch, after the tile front);
// k_fd_partials (FP64 totals of dense fields).  T is stored like one population plane (row pitch kp.pitch, ghost
// columns on strip contexts).  The FP64 mode evaluates every formula in the
// order of its printed form (compiled without contraction).
#pragma once

#include "lb_cavity.cuh"
#include "lb_device.cuh"

namespace lbgb {

constexpr int FD_BX = 32, FD_BY = 8;

// the 9 pre-collision f of site (x, y) (pull)
template <class S>
__device__ __forceinline__ void pull9(const typename S::elem* __restrict__ src, const KParams& kp, int x,
                                      int y, typename S::real f[9]) {
    if (kp.walls) {  // cavity: stored pre-collision at the site
        const long long off = (long long)y * kp.pitch + x;
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[i] = S::load(src + (long long)i * kp.plane + off, (typename S::real)kp.base_f[i]);
        return;
    }
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
    const real Te = kp.psi_local_T ? T : KPR(kp, T_psi);
    if constexpr (sizeof(real) == 8)
        psi2 = (real)2 * (p_eos<real>(kp, r, Te) - r * (real)(1.0 / 3.0)) / KPR(kp, G);
    else
        psi2 = (p_eos<real>(kp, r, Te) - r * (real)(1.0 / 3.0)) * KPR(kp, two_over_G);
    psi = (real)0;
    if (BMODE != BETA_ZERO) {
        if (psi2 < (real)0) flags |= 1 << LB_ERR_PSI_DOMAIN;
        psi = sqrt(psi2);
    }
    if (!isfinite(r) || !isfinite(T)) flags |= 1 << LB_ERR_NONFINITE;
}

// Density step (STEP) or moments (!STEP) of the FD treatment.
//   STEP:  f (src, pre-collision at n) -> dst (post-collision, stored at the
//          source site; cavity: pushed, bounced back at the walls);
//          rho_n, ux_n, uy_n <- rho^n, u^n.
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
        const int gx = ringc(kp, x0 + lx - 1, kp.nx), gy = ringc(kp, y0 + ly - 1, kp.ny);
        real f[9], psi, psi2;
        pull9<S>(src, kp, gx, gy, f);
        real r = f[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) r += f[i];
        site_psi_T<real, BMODE>(kp, r, Tf[(long long)gy * kp.pitch + gx], psi, psi2, flags);
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
        if (kp.walls) Fy += -rho * KPR(kp, g_grav);  // cavity buoyancy
        // the f half of the collision; g (zero here) is not used
        collide<real, false>(kp, f, g, rho, Fx, Fy, ux, uy, Tg);
        const long long c = (long long)gy * kp.nx + gx;
        if (STEP) {
            const long long off = (long long)gy * kp.pitch + gx;
            if (kp.walls) {
                // cavity and channel: push to x + e_i; bounce back from the walls
                // and plates; channel inlet: with the wall velocity; channel
                // outlet: anti-bounce-back at density 1 with the node's velocity
                const real cs2 = (real)(1.0 / 3.0);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int xd = gx + ex(i), yd = gy + ey(i);
                    typename S::elem* pfo = dst + (long long)opp(i) * kp.plane + off;
                    if (xd >= 0 && xd < kp.nx && yd >= 0 && yd < kp.ny) {
                        S::put(dst + (long long)i * kp.plane + (long long)yd * kp.pitch + xd, f[i],
                               (real)kp.base_f[i]);
                    } else if (kp.walls != 2 || yd < 0 || yd >= kp.ny) {
                        S::put(pfo, f[i], (real)kp.base_f[opp(i)]);
                    } else if (xd < 0) {
                        const real eu = (real)ex(i) * KPR(kp, U_in);
                        S::put(pfo, f[i] - (real)2.0 * (real)wd(i) * rho * eu / cs2, (real)kp.base_f[opp(i)]);
                    } else {
                        const real eu = (real)ex(i) * ux + (real)ey(i) * uy;
                        const real fb = -f[i] + (real)2.0 * (real)wd(i) * (real)1.0 *
                                                    ((real)1.0 + (real)0.5 * eu * eu / (cs2 * cs2) -
                                                     (real)0.5 * (ux * ux + uy * uy) / cs2);
                        S::put(pfo, fb, (real)kp.base_f[opp(i)]);
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) S::put(dst + (long long)i * kp.plane + off, f[i], (real)kp.base_f[i]);
            }
            rho_n[c] = rho;
            ux_n[c] = ux;
            uy_n[c] = uy;
        } else {
            if (m_rho) m_rho[c] = (double)rho;
            if (m_ux) m_ux[c] = (double)ux;
            if (m_uy) m_uy[c] = (double)uy;
            if (m_T) m_T[c] = (double)Tf[(long long)gy * kp.pitch + gx];
        }
    } else {
        flags = 0;
    }
    if (flags) atomicOr(kp.err, flags);
}

// T field (storage real, row pitch kp.pitch, ghost columns when kp.ghost)
// <- T0 (FP64, dense [ny][nx])
template <typename real>
__global__ void k_fd_set_T(real* __restrict__ T, const double* __restrict__ T0, const KParams kp) {
    const long long n = (long long)kp.nx * kp.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % kp.nx), y = (int)(i / kp.nx);
        const real v = (real)T0[i];
        real* p = T + (long long)y * kp.pitch + x;
        *p = v;
        if (x < kp.ghost) p[kp.nx] = v;
        if (x >= kp.nx - kp.ghost) p[-kp.nx] = v;
    }
}

}  // namespace lbgb
