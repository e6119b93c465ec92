// lb_init_balanced.cuh -- the initial state at rest under the pseudopotential
// force.
//
// With the forcing scheme of Eq. (1) the velocity of a state is
// u = (sum_i e_i f_i + F/2) / rho, so the state at rest carries the first
// moment sum_i e_i f_i = -F/2.  From given fields rho0, T0 (float64, dense
// [ny][nx]) every site gets
//   psi from rho0 and T (T0, or T_psi when psi does not follow the local T),
//   F of Eq. (4) (Eq. (2) when beta = 1) from the 3x3 neighbourhood,
//   v = -F / (2 rho0),  f_i = f^eq_i(rho0, v),  g_i = c_v T0 f^eq_i(rho0, v).
// The plain start f^eq(rho0, 0) instead moves every interface with F/(2 rho)
// on the first step.  All arithmetic is FP64 in the order of the printed
// formulas (the translation unit is compiled without FMA contraction), then
// rounded once to the storage precision.  Periodic lattices only: the value
// stored at (x, y) for direction i is the one site (x + e_i, y + e_i) pulls.
// One thread per site, nine psi evaluations each (a one-time start; psi is
// recomputed rather than staged).  psi^2 < 0 with beta != 0 sets the
// LB_ERR_PSI_DOMAIN bit of the error word, as the step does.
#pragma once

#include "lb_device.cuh"

namespace lbgb {

template <int BMODE>
__device__ __forceinline__ void psi_of_fields(const KParams& kp, double r, double T, double& psi,
                                              double& psi2, int& flags) {
    const double Te = kp.psi_local_T ? T : kp.T_psi;
    psi2 = 2.0 * (p_eos<double>(kp, r, Te) - r * (1.0 / 3.0)) / kp.G;
    psi = 0.0;
    if (BMODE != BETA_ZERO) {
        if (psi2 < 0.0) flags |= 1 << LB_ERR_PSI_DOMAIN;
        psi = sqrt(psi2);
    }
}

template <int PREC, int BMODE>
__global__ void __launch_bounds__(256)
    k_init_balanced(typename Store<PREC>::elem* __restrict__ dst, const KParams kp,
                    const double* __restrict__ rho0, const double* __restrict__ T0) {
    using S = Store<PREC>;
    using real = typename S::real;
    const int nx = kp.nx, ny = kp.ny;
    const long long n = (long long)nx * ny;
    int flags = 0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % nx), y = (int)(s / nx);
        // 3x3 window, row-major from the row below: index (dy + 1) * 3 + (dx + 1)
        double wpsi[9], wpsi2[9];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const long long q = (long long)wrapc(y + dy, ny) * nx + wrapc(x + dx, nx);
                psi_of_fields<BMODE>(kp, rho0[q], T0[q], wpsi[(dy + 1) * 3 + dx + 1],
                                     wpsi2[(dy + 1) * 3 + dx + 1], flags);
            }
        double Fx, Fy;
        force_from_window<double, BMODE>(kp, wpsi, wpsi2, 4, 3, Fx, Fy);
        const double r = rho0[s], T = T0[s];
        const double vx = -Fx / (2.0 * r);
        const double vy = -Fy / (2.0 * r);
        const double cs2 = 1.0 / 3.0;
        const double usq = vx * vx + vy * vy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double eu = (double)ex(i) * vx + (double)ey(i) * vy;
            const double fe = r * wd(i) * (1.0 + eu / cs2 + 0.5 * eu * eu / (cs2 * cs2) - 0.5 * usq / cs2);
            const double ge = kp.cv * T * fe;
            // stored at the site that streams it here
            const int xs = wrapc(x - ex(i), nx), ys = wrapc(y - ey(i), ny);
            const long long off = (long long)ys * kp.pitch + xs;
            typename S::elem* pf = dst + (long long)i * kp.plane + off;
            typename S::elem* pg = dst + (long long)(9 + i) * kp.plane + off;
            put_pop_ghost<S>(pf, kp.plane, i, xs, kp, (real)fe, (real)kp.base_f[i]);
            put_pop_ghost<S>(pg, kp.plane, 9 + i, xs, kp, (real)ge, (real)kp.base_g[i]);
        }
    }
    if (flags) atomicOr(kp.err, flags);
}

}  // namespace lbgb
