// lb_cavity.cuh -- the fused step in the natural-convection cavity of
// Sec. III B and in the plate channel of Sec. III A (walls, an inlet and an
// outlet instead of the periodic lattice).
//
// nx-by-ny fluid nodes inside walls half a lattice spacing outside the
// outermost nodes.  The populations are stored pre-collision at their own
// site and pushed after the collision: a population whose destination lies
// beyond a wall comes back to its node in the opposite direction
// (f: bounce-back on every wall, no slip; g: bounce-back on the adiabatic
// bottom and top walls, anti-bounce-back -g*_i + 2 w_i rho c_v T_w on the
// isothermal side walls, the side-wall rule for a link through a corner).
// psi at a wall node is that of its nearest fluid node, and the buoyancy
// (0, -rho g) is added to the pseudopotential force.  Otherwise the step is
// k_step's: a 32x8 tile, psi for the tile and a one-site ring in shared
// memory, the same force, collision and (FP64) order of operations.
#pragma once

#include "lb_device.cuh"

namespace lbgb {

constexpr int CAV_BX = 32, CAV_BY = 8;

__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}

template <int PREC, bool EQ24, int BMODE>
__global__ void __launch_bounds__(CAV_BX* CAV_BY)
    k_step_cavity(const typename Store<PREC>::elem* __restrict__ src,
                  typename Store<PREC>::elem* __restrict__ dst, const KParams kp) {
    using S = Store<PREC>;
    using real = typename S::real;
    constexpr int BX = CAV_BX, BY = CAV_BY;
    constexpr int WX = BX + 2, WY = BY + 2, NT = BX * BY;
    __shared__ real s_psi[BMODE != BETA_ZERO ? WX * WY : 1];
    __shared__ real s_psi2[BMODE != BETA_ONE ? WX * WY : 1];

    const int nx = kp.nx, ny = kp.ny;
    const int tid = threadIdx.x + threadIdx.y * BX;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    int flags = 0;
    for (int s = tid; s < WX * WY; s += NT) {
        const int ly = s / WX, lx = s - ly * WX;
        const int gx = clampc(x0 + lx - 1, nx), gy = clampc(y0 + ly - 1, ny);
        real f[9], g[9], rho, T, psi, psi2;
        const long long off = (long long)gy * kp.pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = S::load(src + (long long)i * kp.plane + off, (real)kp.base_f[i]);
            g[i] = S::load(src + (long long)(9 + i) * kp.plane + off, (real)kp.base_g[i]);
        }
        site_psi<real, BMODE>(kp, f, g, rho, T, psi, psi2, flags);
        if (BMODE != BETA_ZERO) s_psi[s] = psi;
        if (BMODE != BETA_ONE) s_psi2[s] = psi2;
    }
    __syncthreads();

    const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
    if (gx < nx && gy < ny) {
        real f[9], g[9];
        const long long off = (long long)gy * kp.pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = S::load(src + (long long)i * kp.plane + off, (real)kp.base_f[i]);
            g[i] = S::load(src + (long long)(9 + i) * kp.plane + off, (real)kp.base_g[i]);
        }
        real rho = f[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) rho += f[i];
        real Fx, Fy, ux, uy, T;
        force_from_window<real, BMODE>(kp, s_psi, s_psi2, (threadIdx.y + 1) * WX + threadIdx.x + 1, WX, Fx,
                                       Fy);
        Fy += -rho * KPR(kp, g_grav);
        collide<real, EQ24>(kp, f, g, rho, Fx, Fy, ux, uy, T);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int xd = gx + ex(i), yd = gy + ey(i);
            const bool out_x = xd < 0 || xd >= nx, out_y = yd < 0 || yd >= ny;
            if (!out_x && !out_y) {
                const long long d = (long long)yd * kp.pitch + xd;
                S::put(dst + (long long)i * kp.plane + d, f[i], (real)kp.base_f[i]);
                S::put(dst + (long long)(9 + i) * kp.plane + d, g[i], (real)kp.base_g[i]);
            } else {
                const int o = opp(i);
                S::put(dst + (long long)o * kp.plane + off, f[i], (real)kp.base_f[o]);
                real gb;
                if (out_x) {
                    const real Tw = xd < 0 ? KPR(kp, T_hot) : KPR(kp, T_cold);
                    gb = -g[i] + (real)2.0 * (real)wd(i) * rho * KPR(kp, cv) * Tw;
                } else {
                    gb = g[i];
                }
                S::put(dst + (long long)(9 + o) * kp.plane + off, gb, (real)kp.base_g[o]);
            }
        }
    }
    if (flags) atomicOr(kp.err, flags);
}

// ---------------------------------------------------------------- channel
// The fused step between parallel plates (Sec. III A): the cavity step's
// storage, psi ring and collision; the push applies the plate rules (f
// bounce-back; g anti-bounce-back at T_w, or bounce-back on an adiabatic
// lower plate), the inlet rules (f bounce-back with the wall velocity
// (U_in, 0); g anti-bounce-back at T_in with the symmetric equilibrium at
// u_in) and, for f beyond the outlet, anti-bounce-back at density 1 with
// the node's velocity.  g beyond the outlet is left for k_channel_outlet.
// A link through a corner takes the plate rule.  FP64: the order of
// operations of the printed formulas.
template <int PREC, bool EQ24, int BMODE>
__global__ void __launch_bounds__(CAV_BX* CAV_BY)
    k_step_channel(const typename Store<PREC>::elem* __restrict__ src,
                   typename Store<PREC>::elem* __restrict__ dst, const KParams kp) {
    using S = Store<PREC>;
    using real = typename S::real;
    constexpr int BX = CAV_BX, BY = CAV_BY;
    constexpr int WX = BX + 2, WY = BY + 2, NT = BX * BY;
    __shared__ real s_psi[BMODE != BETA_ZERO ? WX * WY : 1];
    __shared__ real s_psi2[BMODE != BETA_ONE ? WX * WY : 1];

    const int nx = kp.nx, ny = kp.ny;
    const int tid = threadIdx.x + threadIdx.y * BX;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    int flags = 0;
    for (int s = tid; s < WX * WY; s += NT) {
        const int ly = s / WX, lx = s - ly * WX;
        const int gx = clampc(x0 + lx - 1, nx), gy = clampc(y0 + ly - 1, ny);
        real f[9], g[9], rho, T, psi, psi2;
        const long long off = (long long)gy * kp.pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = S::load(src + (long long)i * kp.plane + off, (real)kp.base_f[i]);
            g[i] = S::load(src + (long long)(9 + i) * kp.plane + off, (real)kp.base_g[i]);
        }
        site_psi<real, BMODE>(kp, f, g, rho, T, psi, psi2, flags);
        if (BMODE != BETA_ZERO) s_psi[s] = psi;
        if (BMODE != BETA_ONE) s_psi2[s] = psi2;
    }
    __syncthreads();

    const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
    if (gx < nx && gy < ny) {
        real f[9], g[9];
        const long long off = (long long)gy * kp.pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = S::load(src + (long long)i * kp.plane + off, (real)kp.base_f[i]);
            g[i] = S::load(src + (long long)(9 + i) * kp.plane + off, (real)kp.base_g[i]);
        }
        real rho = f[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) rho += f[i];
        real Fx, Fy, ux, uy, T;
        force_from_window<real, BMODE>(kp, s_psi, s_psi2, (threadIdx.y + 1) * WX + threadIdx.x + 1, WX, Fx,
                                       Fy);
        collide<real, EQ24>(kp, f, g, rho, Fx, Fy, ux, uy, T);
        const real cs2 = (real)(1.0 / 3.0);
        const real uin = KPR(kp, U_in);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int xd = gx + ex(i), yd = gy + ey(i);
            const int o = opp(i);
            typename S::elem* pfo = dst + (long long)o * kp.plane + off;
            typename S::elem* pgo = dst + (long long)(9 + o) * kp.plane + off;
            if (yd < 0 || yd >= ny) {
                // plate
                S::put(pfo, f[i], (real)kp.base_f[o]);
                real gb;
                if (yd < 0 && kp.adiabatic_bottom)
                    gb = g[i];
                else
                    gb = -g[i] + (real)2.0 * (real)wd(i) * rho * KPR(kp, cv) * KPR(kp, T_w);
                S::put(pgo, gb, (real)kp.base_g[o]);
            } else if (xd < 0) {
                // inlet
                const real eu = (real)ex(i) * uin;
                S::put(pfo, f[i] - (real)2.0 * (real)wd(i) * rho * eu / cs2, (real)kp.base_f[o]);
                const real gb = -g[i] + (real)2.0 * (real)wd(i) * rho * KPR(kp, cv) * KPR(kp, T_in) *
                                            ((real)1.0 + (real)0.5 * eu * eu / (cs2 * cs2) -
                                             (real)0.5 * uin * uin / cs2);
                S::put(pgo, gb, (real)kp.base_g[o]);
            } else if (xd < nx) {
                const long long d = (long long)yd * kp.pitch + xd;
                S::put(dst + (long long)i * kp.plane + d, f[i], (real)kp.base_f[i]);
                S::put(dst + (long long)(9 + i) * kp.plane + d, g[i], (real)kp.base_g[i]);
            } else {
                // outlet: f at density 1 with the node's velocity; g by k_channel_outlet
                const real eu = (real)ex(i) * ux + (real)ey(i) * uy;
                const real fb = -f[i] + (real)2.0 * (real)wd(i) * (real)1.0 *
                                            ((real)1.0 + (real)0.5 * eu * eu / (cs2 * cs2) -
                                             (real)0.5 * (ux * ux + uy * uy) / cs2);
                S::put(pfo, fb, (real)kp.base_f[o]);
            }
        }
    }
    if (flags) atomicOr(kp.err, flags);
}

// Outlet of the channel for g: the populations that arrive at column nx - 1
// from beyond the outlet (e_x = -1, source inside the plates) copy those of
// column nx - 2 (zero gradient).  One thread per row; after k_step_channel.
template <int PREC>
__global__ void k_channel_outlet(typename Store<PREC>::elem* __restrict__ buf, const KParams kp) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= kp.ny) return;
    const long long a = (long long)y * kp.pitch + (kp.nx - 1), b = a - 1;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (ex(i) != -1) continue;
        const int ys = y - ey(i);
        if (ys < 0 || ys >= kp.ny) continue;  // set by the plate rule
        buf[(long long)(9 + i) * kp.plane + a] = buf[(long long)(9 + i) * kp.plane + b];
    }
}

}  // namespace lbgb
