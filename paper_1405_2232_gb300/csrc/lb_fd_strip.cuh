// lb_fd_strip.cuh -- the finite-difference temperature treatment (Eqs. 26-27)
// in one pass over HBM on strip contexts (k_fd_fused), and the fused RK2
// stages used after the tile front on other lattices (k_fd_rk2).
//
// k_fd_fused is k_step_strip (lb_step_strip.cuh) with the g populations
// replaced by the temperature field and the RK2 update of Eq. (27) folded in:
// for every pre-collision row the producer streams the 9 f plane rows and the
// row of T^n (both stored in the ghost-column layout), and the consumer warps
// run four phases on rows lagging behind the newest one, with shared-memory
// row rings for psi, rho, T^n, u^n, h1 and the intermediate T.  Per site it
// reads f and T^n and writes f and T^{n+1} once (80 B in FP32).
//
// k_fd_rk2 evaluates T^{n+1} = T^n + (h1 + K(T^n + a h1))/2, h1 = K(T^n), in
// one launch: a tile stages T^n and rho^n with a two-site ring, u^n with a
// one-site ring, computes h1 and the intermediate T on the tile plus one ring
// in shared memory, then the second stage on the tile (each thread two rows).
//
// K uses the isotropic central stencils of the D2Q9 lattice; in FP64 every
// formula is evaluated in its printed order (compiled without contraction),
// so the fused kernel and the tile front + k_fd_rk2 give the same bits.
#pragma once

#include "lb_fd.cuh"
#include "lb_step_strip.cuh"

namespace lbgb {

// Shared memory of k_fd_fused (elements of real unless noted):
//   stages  STAGES x 10 rows (f_0..f_8, T) x (BX + 2 FD_HALO) elements
//   psi     2 x 4 rows x (BX + 4)          columns -2..W+1
//   rho, T  2 x 8 rows x (BX + 4)          columns -2..W+1
//   u, h1, Ts  4 x 4 rows x (BX + 2)       columns -1..W
template <int PREC, int BX>
constexpr size_t fd_fused_ring_bytes() {
    using C = StripCfg<PREC>;
    return ((size_t)24 * (BX + 4) + (size_t)16 * (BX + 2)) * sizeof(typename C::real);
}
template <int PREC, int BX, int STAGES>
constexpr size_t fd_fused_smem_bytes() {
    using C = StripCfg<PREC>;
    return (size_t)STAGES * 10 * (BX + 2 * FD_HALO) * C::ES + fd_fused_ring_bytes<PREC, BX>() +
           (size_t)2 * STAGES * 8 + 16;
}
template <int PREC, int BX>
constexpr int fd_fused_stages() {
    using C = StripCfg<PREC>;
    constexpr size_t stage = (size_t)10 * (BX + 2 * FD_HALO) * C::ES;
    constexpr size_t s = (110 * 1024 - 32 - fd_fused_ring_bytes<PREC, BX>()) / stage;
    return s > 12 ? 12 : (int)s;
}

// K(X) of Eq. (26) at one site from three row pointers (south, centre, north,
// each at the site's column) of X and of rho.  FP64: the stencil and order of
// operations of the printed form (divisions by c_s^2 included); FP32: the
// same sums with the divisions by c_s^2 = 1/3 taken as products by 3 and the
// division by rho as the fast division.
template <typename real>
__device__ __forceinline__ real fd_K_rows(const real* Xs, const real* Xc, const real* Xn, const real* Rs,
                                          const real* Rc, const real* Rn, real ux, real uy, real chi) {
    real gTx = 0, gTy = 0, grx = 0, gry = 0, lap = 0;
    const real X0 = Xc[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const real w = (real)wd(i);
        const real* xr = ey(i) == 1 ? Xn : (ey(i) == -1 ? Xs : Xc);
        const real* rr = ey(i) == 1 ? Rn : (ey(i) == -1 ? Rs : Rc);
        const real Xv = xr[ex(i)], rn = rr[ex(i)];
        gTx += w * (real)ex(i) * Xv;
        gTy += w * (real)ey(i) * Xv;
        grx += w * (real)ex(i) * rn;
        gry += w * (real)ey(i) * rn;
        lap += w * (Xv - X0);
    }
    if constexpr (sizeof(real) == 8) {
        const real cs2 = (real)(1.0 / 3.0);
        gTx /= cs2;
        gTy /= cs2;
        grx /= cs2;
        gry /= cs2;
        lap *= (real)2 / cs2;
    } else {
        gTx *= (real)3;
        gTy *= (real)3;
        grx *= (real)3;
        gry *= (real)3;
        lap *= (real)6;
    }
    if constexpr (sizeof(real) == 8)
        return -(ux * gTx + uy * gTy) + chi * (lap + (grx * gTx + gry * gTy) / Rc[0]);
    else  // FP32: the fast division (a few ulp; +3% on the issue-bound fused step)
        return -(ux * gTx + uy * gTy) + chi * (lap + __fdividef(grx * gTx + gry * gTy, Rc[0]));
}

// FP32: the same K with the terms that depend only on the site's density and
// velocity folded into a = chi grad(rho) / rho - u, which both RK2 stages
// share (formed once per site in the fused kernel's velocity phase):
// K = a . grad(X) + chi lap(X), the stencil of X alone.
__device__ __forceinline__ float fd_K_rows_a(const float* Xs, const float* Xc, const float* Xn, float ax,
                                             float ay, float chi) {
    float gTx = 0.0f, gTy = 0.0f, lap = 0.0f;
    const float X0 = Xc[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const float w = (float)wd(i);
        const float* xr = ey(i) == 1 ? Xn : (ey(i) == -1 ? Xs : Xc);
        const float Xv = xr[ex(i)];
        gTx += w * (float)ex(i) * Xv;
        gTy += w * (float)ey(i) * Xv;
        lap += w * (Xv - X0);
    }
    return fmaf(ax, 3.0f * gTx, fmaf(ay, 3.0f * gTy, chi * (6.0f * lap)));
}

// a = chi grad(rho) / rho - u at a site (FP32; see fd_K_rows_a), from the
// density rows (south, centre, north, each at the site's column)
__device__ __forceinline__ void fd_a_rows(const float* Rs, const float* Rc, const float* Rn, float ux, float uy,
                                          float chi, float& ax, float& ay) {
    float grx = 0.0f, gry = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const float w = (float)wd(i);
        const float* rr = ey(i) == 1 ? Rn : (ey(i) == -1 ? Rs : Rc);
        const float rn = rr[ex(i)];
        grx += w * (float)ex(i) * rn;
        gry += w * (float)ey(i) * rn;
    }
    const float cr = __fdividef(chi, Rc[0]);
    ax = fmaf(cr, 3.0f * grx, -ux);
    ay = fmaf(cr, 3.0f * gry, -uy);
}

// One whole FD step (Eqs. 1, 26, 27) on a strip context, one pass over HBM:
// f and T^n in, f and T^{n+1} out (both in the ghost-column layout, row
// pitch kp.pitch, kp.ghost = FD_GHOST).  Job k is pre-collision row
// y_start - 2 + k (k = 0 .. rows + 3); rows k = 2 .. rows + 1 are the
// chunk's own.  Iteration j, with one named barrier between A and the rest:
//   A(j)    rho (pulled f), T^n and psi of row j, columns -2..W+1
//   B(j-1)  force and u^n of row j-1, columns -1..W (psi rows j-2..j);
//           own rows also collide f and store it (columns 0..W-1)
//   C(j-2)  stage 1: h1 = K(T^n), Ts = T^n + a h1, columns -1..W
//   D(j-4)  stage 2: T^{n+1} = T^n + (h1 + K(Ts)) / 2, own rows, columns 0..W-1
// Each phase reads only rows finished before the barrier it follows.  Column
// thread t owns column t; the halo warp takes the columns outside 0..W-1.
template <int PREC, int BX, int STAGES, int BMODE>
__global__ void __launch_bounds__(strip_threads<BX>(), 2)
    k_fd_fused(const typename Store<PREC>::elem* __restrict__ src, typename Store<PREC>::elem* __restrict__ dst,
               const typename Store<PREC>::real* __restrict__ Tn, typename Store<PREC>::real* __restrict__ Tnext,
               const KParams kp, int nchunks, typename Store<PREC>::real chi, typename Store<PREC>::real a) {
    using S = Store<PREC>;
    using C = StripCfg<PREC>;
    using elem = typename C::elem;
    using real = typename C::real;
    static_assert(sizeof(elem) == sizeof(real), "the FD treatment stores FP64 or FP32");
    constexpr int HALO = FD_HALO;
    constexpr int SEGW = BX + 2 * HALO;
    constexpr int RA = BX + 4;  // ring rows, columns -2..W+1 at index col + 2
    constexpr int RB = BX + 2;  // ring rows, columns -1..W at index col + 1
    constexpr int ES = C::ES;
    constexpr int NCW = BX / 32;
    constexpr int NP = 10;  // rows per stage: f_0..f_8, T

    extern __shared__ __align__(128) unsigned char smem_raw[];
    elem* stage = reinterpret_cast<elem*>(smem_raw);  // [STAGES][NP][SEGW]
    real* r_psi = reinterpret_cast<real*>(stage + (size_t)STAGES * NP * SEGW);  // [4][RA]
    real* r_psi2 = r_psi + 4 * RA;                                               // [4][RA]
    real* r_rho = r_psi2 + 4 * RA;                                               // [8][RA]
    real* r_T = r_rho + 8 * RA;                                                  // [8][RA]
    real* r_ux = r_T + 8 * RA;                                                   // [4][RB]
    real* r_uy = r_ux + 4 * RB;                                                  // [4][RB]
    real* r_h1 = r_uy + 4 * RB;                                                  // [4][RB]
    real* r_Ts = r_h1 + 4 * RB;                                                  // [4][RB]
    uint64_t* full = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(r_Ts + 4 * RB) + 7) & ~uintptr_t(7));
    uint64_t* empty = full + STAGES;
    __shared__ int s_abort[2];  // one slot per job parity (see the loop)

    const int t = threadIdx.x;
    const int nx = kp.nx, ny = kp.ny;
    const int x0 = blockIdx.x * BX;
    const int W = min(BX, nx - x0);
    const int y_start = (int)((long long)blockIdx.y * ny / nchunks);
    const int y_end = (int)((long long)(blockIdx.y + 1) * ny / nchunks);
    const int njobs = (y_end - y_start) + 4;  // pre-collision rows y_start-2 .. y_end+1
    const uint32_t plane = (uint32_t)kp.plane, pitch = (uint32_t)kp.pitch;
    const int ghost = kp.ghost;

    if (t == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        fence_mbar_init();
        s_abort[0] = 0;
        s_abort[1] = 0;
    }
    __syncthreads();

    if (t >= BX + 32) {
        // ------------------------------------------------ producer warp
        const int lane = t - BX - 32;
        int issued = 0;
        for (int j = 0; j < njobs; ++j) {
            const int s = j % STAGES;
            if (j >= STAGES) {
                // the warp takes one decision (its lanes poll the barrier independently)
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(&empty[s], (uint32_t)(((j / STAGES) - 1) & 1),
                                                               kp.wait_cycles))) {
                    if (lane == 0) atomicOr(kp.err, 1 << LB_ERR_TIMEOUT);
                    break;
                }
            }
            int y = y_start - 2 + j;
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)NP * strip_copy_bytes<ES, HALO>(W));
            __syncwarp();
            if (lane < NP) {
                const elem* row;
                if (lane < 9) {
                    int sy = y - ey(lane);
                    sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                    row = src + (size_t)((uint32_t)lane * plane + (uint32_t)sy * pitch);
                } else {
                    row = reinterpret_cast<const elem*>(Tn) + (size_t)((uint32_t)y * pitch);
                }
                bulk_copy_g2s(stage + ((size_t)s * NP + lane) * SEGW, row + (x0 - HALO),
                              strip_copy_bytes<ES, HALO>(W), &full[s]);
            }
            issued = j + 1;
        }
        if (lane == 0)
            for (int j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j)
                (void)mbar_wait_bounded(&full[j % STAGES], (uint32_t)((j / STAGES) & 1));
        return;
    }

    // ------------------------------------------ column threads and halo warp
    const bool halo = t >= BX;
    const int hl = t & 31;
    // phase A: column (-2..W+1) of this thread, or none
    const int colA = halo ? (hl < 2 ? hl - 2 : (hl < 4 ? W + hl - 2 : -99)) : (t < W ? t : -99);
    // phases B, C: column (-1..W), or none
    const int colB = halo ? (hl == 0 ? -1 : (hl == 1 ? W : -99)) : (t < W ? t : -99);
    const bool own_col = !halo && t < W;
    int flags = 0;
    bool aborted = false;
    for (int j = 0; j < njobs + 2; ++j) {
        // A(j)
        if (j < njobs) {
            const int s = j % STAGES;
            if (!mbar_wait_bounded(&full[s], (uint32_t)((j / STAGES) & 1), kp.wait_cycles)) s_abort[j & 1] = 1;
            if (colA != -99) {
                const elem* st = stage + (size_t)s * NP * SEGW;
                const int c = colA + HALO;
                real f[9], psi, psi2;
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = S::load(st + i * SEGW + c - ex(i), (real)kp.base_f[i]);
                real rho = f[0];
#pragma unroll
                for (int i = 1; i < 9; ++i) rho += f[i];
                const real T = (real)st[9 * SEGW + c];
                site_psi_T<real, BMODE>(kp, rho, T, psi, psi2, flags);
                const int ia = colA + 2;
                if (BMODE != BETA_ZERO) r_psi[(j & 3) * RA + ia] = psi;
                if (BMODE != BETA_ONE) r_psi2[(j & 3) * RA + ia] = psi2;
                r_rho[(j & 7) * RA + ia] = rho;
                r_T[(j & 7) * RA + ia] = T;
            }
        }
        consumer_sync<BX + 32>();
        // (a thread that times out at job j + 1 writes the other slot than the
        // one read here, so every consumer leaves at the same job)
        if (s_abort[j & 1]) {
            aborted = true;
            break;
        }
        // B(k), k = j - 1: force, u; own rows: f collision and store
        {
            const int k = j - 1;
            if (k >= 1 && k <= njobs - 2 && colB != -99) {
                const elem* st = stage + (size_t)(k % STAGES) * NP * SEGW;
                const int c = colB + HALO;
                real f[9], g[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    f[i] = S::load(st + i * SEGW + c - ex(i), (real)kp.base_f[i]);
                    g[i] = (real)0;
                }
                real rho = f[0];
#pragma unroll
                for (int i = 1; i < 9; ++i) rho += f[i];
                const int ia = colB + 2;
                real Fx, Fy, ux, uy, Tg;
                force_from_rows<real, BMODE>(
                    kp, r_psi + ((k - 1) & 3) * RA + ia, r_psi + (k & 3) * RA + ia, r_psi + ((k + 1) & 3) * RA + ia,
                    r_psi2 + ((k - 1) & 3) * RA + ia, r_psi2 + (k & 3) * RA + ia,
                    r_psi2 + ((k + 1) & 3) * RA + ia, Fx, Fy);
                // the f half of the collision; g (zero here) is not used
                // (FP32: the fused multiply-add form, faster in this kernel)
                collide<real, false, true>(kp, f, g, rho, Fx, Fy, ux, uy, Tg);
                if constexpr (sizeof(real) == 4) {
                    // FP32: the rings keep a = chi grad(rho) / rho - u, which
                    // both stages' K share (fd_K_rows_a)
                    real ax, ay;
                    fd_a_rows(r_rho + ((k - 1) & 7) * RA + ia, r_rho + (k & 7) * RA + ia,
                              r_rho + ((k + 1) & 7) * RA + ia, ux, uy, chi, ax, ay);
                    r_ux[(k & 3) * RB + colB + 1] = ax;
                    r_uy[(k & 3) * RB + colB + 1] = ay;
                } else {
                    r_ux[(k & 3) * RB + colB + 1] = ux;
                    r_uy[(k & 3) * RB + colB + 1] = uy;
                }
                if (own_col && k >= 2 && k <= njobs - 3) {
                    int y = y_start - 2 + k;
                    y = y >= ny ? y - ny : y;
                    const int xg = x0 + t;
                    const uint32_t off = (uint32_t)y * pitch + (uint32_t)xg;
                    const bool ghost_lo = xg < ghost, ghost_hi = xg >= nx - ghost;
#pragma unroll
                    for (int i = 0; i < 9; ++i) S::put(dst + ((uint32_t)i * plane + off), f[i], (real)kp.base_f[i]);
                    // the periodic ghost copies: one branch per site, not per plane
                    if (ghost_lo || ghost_hi) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            elem* pf = dst + ((uint32_t)i * plane + off);
                            if (ghost_lo) S::put(pf + nx, f[i], (real)kp.base_f[i]);
                            if (ghost_hi) S::put(pf - nx, f[i], (real)kp.base_f[i]);
                        }
                    }
                }
            }
        }
        // C(k), k = j - 2: stage 1
        {
            const int k = j - 2;
            if (k >= 1 && k <= njobs - 2 && colB != -99) {
                const int ia = colB + 2, ib = colB + 1;
                const real* Ts_ = r_T + ((k - 1) & 7) * RA + ia;
                const real* Tc_ = r_T + (k & 7) * RA + ia;
                const real* Tn_ = r_T + ((k + 1) & 7) * RA + ia;
                real K;
                if constexpr (sizeof(real) == 4)
                    K = fd_K_rows_a(Ts_, Tc_, Tn_, r_ux[(k & 3) * RB + ib], r_uy[(k & 3) * RB + ib], chi);
                else
                    K = fd_K_rows<real>(Ts_, Tc_, Tn_, r_rho + ((k - 1) & 7) * RA + ia, r_rho + (k & 7) * RA + ia,
                                        r_rho + ((k + 1) & 7) * RA + ia, r_ux[(k & 3) * RB + ib],
                                        r_uy[(k & 3) * RB + ib], chi);
                r_h1[(k & 3) * RB + ib] = K;
                r_Ts[(k & 3) * RB + ib] = Tc_[0] + a * K;
            }
        }
        // D(k), k = j - 4: stage 2 on own rows and columns
        {
            const int k = j - 4;
            if (k >= 2 && k <= njobs - 3 && own_col) {
                const int ia = t + 2, ib = t + 1;
                real K;
                if constexpr (sizeof(real) == 4)
                    K = fd_K_rows_a(r_Ts + ((k - 1) & 3) * RB + ib, r_Ts + (k & 3) * RB + ib,
                                    r_Ts + ((k + 1) & 3) * RB + ib, r_ux[(k & 3) * RB + ib], r_uy[(k & 3) * RB + ib],
                                    chi);
                else
                    K = fd_K_rows<real>(r_Ts + ((k - 1) & 3) * RB + ib, r_Ts + (k & 3) * RB + ib,
                                        r_Ts + ((k + 1) & 3) * RB + ib, r_rho + ((k - 1) & 7) * RA + ia,
                                        r_rho + (k & 7) * RA + ia, r_rho + ((k + 1) & 7) * RA + ia,
                                        r_ux[(k & 3) * RB + ib], r_uy[(k & 3) * RB + ib], chi);
                const real v = r_T[(k & 7) * RA + ia] + (real)0.5 * (r_h1[(k & 3) * RB + ib] + K);
                int y = y_start - 2 + k;
                y = y >= ny ? y - ny : y;
                const int xg = x0 + t;
                real* p = Tnext + (long long)y * pitch + xg;
                *p = v;
                if (xg < ghost) p[nx] = v;
                if (xg >= nx - ghost) p[-nx] = v;
                if (!isfinite(v)) flags |= 1 << LB_ERR_NONFINITE;
            }
        }
        // the stage of job j-1 has had its last reader (A at j-1, B at j)
        if (j >= 1 && j <= njobs - 1 && !halo) {
            __syncwarp();
            if ((t & 31) == 0) mbar_arrive(&empty[(j - 1) % STAGES]);
        }
    }
    if (aborted) {
        if (t == 0) atomicOr(kp.err, 1 << LB_ERR_TIMEOUT);
        return;
    }
    if (flags) atomicOr(kp.err, flags);
}

// K(X) of Eq. (26) from shared-memory tiles: X and R (rho) with row strides
// xs and rs, centre indices xc and rc.  FP64: the stencil and order of
// operations of the printed form (divisions by c_s^2 included); FP32:
// the same sums with the divisions by c_s^2 = 1/3 taken as products by 3 and
// the division by rho as the fast division.
template <typename real>
__device__ __forceinline__ real fd_K_tile(const real* X, int xs, int xc, const real* R, int rs, int rc, real ux,
                                          real uy, real chi) {
    real gTx = 0, gTy = 0, grx = 0, gry = 0, lap = 0;
    const real Xc = X[xc];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const real w = (real)wd(i);
        const real Xn = X[xc + ey(i) * xs + ex(i)], rn = R[rc + ey(i) * rs + ex(i)];
        gTx += w * (real)ex(i) * Xn;
        gTy += w * (real)ey(i) * Xn;
        grx += w * (real)ex(i) * rn;
        gry += w * (real)ey(i) * rn;
        lap += w * (Xn - Xc);
    }
    if constexpr (sizeof(real) == 8) {
        const real cs2 = (real)(1.0 / 3.0);
        gTx /= cs2;
        gTy /= cs2;
        grx /= cs2;
        gry /= cs2;
        lap *= (real)2 / cs2;
    } else {
        gTx *= (real)3;
        gTy *= (real)3;
        grx *= (real)3;
        gry *= (real)3;
        lap *= (real)6;
    }
    if constexpr (sizeof(real) == 8)
        return -(ux * gTx + uy * gTy) + chi * (lap + (grx * gTx + gry * gTy) / R[rc]);
    else
        return -(ux * gTx + uy * gTy) + chi * (lap + __fdividef(grx * gTx + gry * gTy, R[rc]));
}

// Ghost value of a temperature-like field X at (rx, ry) outside the lattice
// of a cavity (walls 1) or channel (walls 2) context, from the value Xm at the
// mirror node (the clamped position): reflected about the boundary value,
// 2 T_b - Xm, across an isothermal boundary (cavity side walls; channel
// plates at T_w and inlet at T_in); Xm across an adiabatic one (cavity bottom
// and top, channel lower plate in Case B, channel outlet).  A position outside
// in both directions takes the side-wall rule in the cavity and the plate
// rule in the channel.
template <typename real>
__device__ __forceinline__ real fd_ghost(const KParams& kp, int rx, int ry, real Xm) {
    const int nx = kp.nx, ny = kp.ny;
    if (kp.walls == 1) {
        if (rx < 0) return (real)2.0 * KPR(kp, T_hot) - Xm;
        if (rx >= nx) return (real)2.0 * KPR(kp, T_cold) - Xm;
        return Xm;
    }
    if (ry < 0 || ry >= ny) {
        if (ry < 0 && kp.adiabatic_bottom) return Xm;
        return (real)2.0 * KPR(kp, T_w) - Xm;
    }
    if (rx < 0) return (real)2.0 * KPR(kp, T_in) - Xm;
    return Xm;
}

// tile of k_fd_rk2: FDR_BX x FDR_BY threads, FDR_ROWS rows of sites per thread
constexpr int FDR_BX = 32, FDR_BY = 8, FDR_ROWS = 2;

// Both RK2 stages of Eq. (27): T (T^n) and T_next in the context's T layout
// (row pitch kp.pitch; ghost columns written when kp.ghost), rho, ux, uy dense.
template <typename real>
__global__ void __launch_bounds__(FDR_BX* FDR_BY)
    k_fd_rk2(const real* __restrict__ T, const real* __restrict__ rho, const real* __restrict__ ux,
             const real* __restrict__ uy, real* __restrict__ T_next, const KParams kp, real chi, real a) {
    constexpr int BX = FDR_BX, BY = FDR_BY * FDR_ROWS, NT = FDR_BX * FDR_BY;
    constexpr int W2 = BX + 4, H2 = BY + 4;  // tile + two-site ring (T, rho)
    constexpr int W1 = BX + 2, H1 = BY + 2;  // tile + one-site ring (u, h1, Ts)
    __shared__ real sT[H2 * W2], sR[H2 * W2];
    __shared__ real sUx[H1 * W1], sUy[H1 * W1], sH1[H1 * W1], sTs[H1 * W1];
    const int nx = kp.nx, ny = kp.ny;
    const long long pitch = kp.pitch;
    const int tid = threadIdx.x + threadIdx.y * FDR_BX;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    // cavity and channel (kp.walls): a neighbour outside reads the ghost of
    // fd_ghost (reflected about an isothermal boundary, mirrored across an
    // adiabatic one); rho and u the mirror node's
    const bool walls = kp.walls != 0;
    for (int s = tid; s < H2 * W2; s += NT) {
        const int ly = s / W2, lx = s - ly * W2;
        const int rx = x0 + lx - 2, ry = y0 + ly - 2;
        const int gx = ringc(kp, rx, nx), gy = ringc(kp, ry, ny);
        const real Tv = T[(long long)gy * pitch + gx];
        sT[s] = walls && (rx < 0 || rx >= nx || ry < 0 || ry >= ny) ? fd_ghost<real>(kp, rx, ry, Tv) : Tv;
        sR[s] = rho[(long long)gy * nx + gx];
    }
    for (int s = tid; s < H1 * W1; s += NT) {
        const int ly = s / W1, lx = s - ly * W1;
        const int gx = ringc(kp, x0 + lx - 1, nx), gy = ringc(kp, y0 + ly - 1, ny);
        sUx[s] = ux[(long long)gy * nx + gx];
        sUy[s] = uy[(long long)gy * nx + gx];
    }
    __syncthreads();
    // stage 1 on the tile and its ring: h1 = K(T^n), Ts = T^n + a h1
    for (int s = tid; s < H1 * W1; s += NT) {
        const int ly = s / W1, lx = s - ly * W1;
        const int rx = x0 + lx - 1, ry = y0 + ly - 1;
        if (walls && (rx < 0 || rx >= nx || ry < 0 || ry >= ny)) continue;  // ghost: filled below
        const int c2 = (ly + 1) * W2 + lx + 1;
        const real K = fd_K_tile<real>(sT, W2, c2, sR, W2, c2, sUx[s], sUy[s], chi);
        sH1[s] = K;
        sTs[s] = sT[c2] + a * K;
    }
    __syncthreads();
    if (walls) {
        // intermediate temperature at the ghost sites of the ring, by the same rule
        for (int s = tid; s < H1 * W1; s += NT) {
            const int ly = s / W1, lx = s - ly * W1;
            const int rx = x0 + lx - 1, ry = y0 + ly - 1;
            if (rx >= 0 && rx < nx && ry >= 0 && ry < ny) continue;
            const int mx = clampc(rx, nx) - x0 + 1, my = clampc(ry, ny) - y0 + 1;
            sTs[s] = fd_ghost<real>(kp, rx, ry, sTs[my * W1 + mx]);
        }
        __syncthreads();
    }
    // stage 2 on the tile: T^{n+1} = T^n + (h1 + K(Ts)) / 2
    int flags = 0;
#pragma unroll
    for (int q = 0; q < FDR_ROWS; ++q) {
        const int ly = threadIdx.y + q * FDR_BY;
        const int gx = x0 + threadIdx.x, gy = y0 + ly;
        if (gx < nx && gy < ny) {
            const int c1 = (ly + 1) * W1 + threadIdx.x + 1;
            const int c2 = (ly + 2) * W2 + threadIdx.x + 2;
            const real K = fd_K_tile<real>(sTs, W1, c1, sR, W2, c2, sUx[c1], sUy[c1], chi);
            const real v = sT[c2] + (real)0.5 * (sH1[c1] + K);
            real* p = T_next + (long long)gy * pitch + gx;
            *p = v;
            if (gx < kp.ghost) p[nx] = v;
            if (gx >= nx - kp.ghost) p[-nx] = v;
            if (!isfinite(v)) flags = 1 << LB_ERR_NONFINITE;
        }
    }
    if (flags) atomicOr(kp.err, flags);
}

}  // namespace lbgb
