/*
 * lb_oracle.c -- plain FP64 CPU oracle of the D2Q9 double-distribution
 * thermal pseudopotential lattice Boltzmann step of Li & Luo,
 * "Effect of the forcing term in the pseudopotential lattice Boltzmann
 * modeling of thermal flows" (arXiv:1405.2232).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct reference
 * the GPU path is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant with the CUDA library, and it includes nothing of it.
 *
 * State convention: the arrays hold the PRE-collision populations f_i(x,t)
 * and g_i(x,t) in structure-of-arrays order, index  i*ny*nx + y*nx + x,
 * on a periodic nx-by-ny lattice (the cavity of Sec. III B: or_step_cavity).
 * One step applies, at every site, the
 * collision of Eq. (1) (density) and Eq. (7) or Eq. (24) (temperature) and
 * then streams the post-collision value to x + e_i, giving f_i(x,t+1).
 *
 * The order of operations below follows the paper's formulas as printed;
 * nothing is blocked, fused or reordered beyond them.
 *
 * Readings of passages where the paper is silent (each is listed in the
 * design notes of the repository):
 *   - lattice numbering and weights (Sec. II A names D2Q9 but lists neither):
 *     e0=(0,0); e1..e4=(1,0),(0,1),(-1,0),(0,-1);
 *     e5..e8=(1,1),(-1,1),(-1,-1),(1,-1); omega = 4/9, 1/9, 1/36.
 *   - the forcing term F_i of Eq. (1) is "the scheme of Ref. [21]", read as
 *     Guo, Zheng & Shi (2002):
 *       F_i = (1 - 1/(2 tau_f)) omega_i [ (e_i - u)/cs^2 + (e_i.u) e_i/cs^4 ] . F
 *     with the velocity u = (sum_i e_i f_i + F/2) / rho used in f^eq, g^eq and F_i.
 *   - temperature T = sum_i g_i / (rho c_v), which follows from g^eq = c_v T f^eq.
 *   - psi of Sec. II A is sqrt(2 (p_EOS - rho cs^2) / (G c^2)) with c = 1;
 *     the mixed force Eq. (4) with beta = 0 only needs psi^2, which may be
 *     negative (the single-phase test of Sec. III).
 *   - the pair sums of Eq. (2)/(4) are written as antisymmetric differences
 *     (east minus west, ...), which is the same sum grouped in pairs.
 *   - Carnahan-Starling EOS (not in the paper; used by the workloads):
 *     p = rho R T (1 + eta + eta^2 - eta^3) / (1 - eta)^3 - a rho^2, eta = b rho / 4.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* status codes of the oracle (its own numbering) */
#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NONFINITE 4
#define OR_ERR_PSI_DOMAIN 5

#define OR_EOS_CS 0
#define OR_EOS_VDW 1
#define OR_EOS_IDEAL 2

#define OR_THERMAL_EQ7 0
#define OR_THERMAL_EQ24 1

typedef struct or_params {
    int32_t nx, ny;
    double tau_f, tau_g; /* relaxation times of Eq. (1) and Eq. (7)         */
    double G, beta;      /* interaction strength and mixing of Eq. (2)/(4)  */
    int32_t eos;         /* OR_EOS_*                                        */
    double a, b, R;      /* EOS constants                                   */
    double cv;           /* specific heat at constant volume, g^eq = cv T f^eq */
    int32_t thermal;     /* OR_THERMAL_EQ7 or OR_THERMAL_EQ24               */
    int32_t psi_uses_local_T; /* 1: psi(rho, T(x,t)); 0: psi(rho, T_psi)    */
    double T_psi;
} or_params;

/* D2Q9 lattice (reading of Sec. II A, see header) */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double OMEGA[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                                1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 = c^2/3 with c = 1 (Sec. II A) */

static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* ---------------------------------------------------------------------- */
/* Equations of state.  vdW and ideal: Sec. III.  Carnahan-Starling: see
 * header (not in the paper).                                               */
double or_p_eos(const or_params* P, double rho, double T)
{
    if (P->eos == OR_EOS_IDEAL) {
        return rho * P->R * T;
    }
    if (P->eos == OR_EOS_VDW) {
        return rho * P->R * T / (1.0 - P->b * rho) - P->a * rho * rho;
    }
    /* Carnahan-Starling */
    double eta = P->b * rho / 4.0;
    double num = 1.0 + eta + eta * eta - eta * eta * eta;
    double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
    return rho * P->R * T * num / den - P->a * rho * rho;
}

/* psi^2 = 2 (p_EOS - rho cs^2) / (G c^2), c = 1  (Sec. II A, after Eq. 3) */
double or_psi_sq(const or_params* P, double rho, double T)
{
    double T_eos = P->psi_uses_local_T ? T : P->T_psi;
    return 2.0 * (or_p_eos(P, rho, T_eos) - rho * CS2) / P->G;
}

/* ---------------------------------------------------------------------- */
/* Equilibrium of Sec. II A (after Eq. 1):
 * f_i^eq = rho w_i [1 + (e_i.u)/cs^2 + 0.5 (e_i.u)^2/cs^4 - 0.5 |u|^2/cs^2] */
void or_feq(double rho, double ux, double uy, double feq[9])
{
    double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = rho * OMEGA[i] *
                 (1.0 + eu / CS2 + 0.5 * eu * eu / (CS2 * CS2) - 0.5 * usq / CS2);
    }
}

/* Forcing term F_i of Eq. (1), scheme of Ref. [21] (Guo et al.):
 * F_i = (1 - 1/(2 tau_f)) w_i [ (e_i - u).F / cs^2 + (e_i.u)(e_i.F) / cs^4 ] */
void or_forcing_term(double tau_f, double ux, double uy, double Fx, double Fy,
                     double Fi[9])
{
    double pre = 1.0 - 1.0 / (2.0 * tau_f);
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        double eF = EX[i] * Fx + EY[i] * Fy;
        double emuF = (EX[i] - ux) * Fx + (EY[i] - uy) * Fy;
        Fi[i] = pre * OMEGA[i] * (emuF / CS2 + eu * eF / (CS2 * CS2));
    }
}

/* Correction term of Eq. (25):
 * C_i = (1 - 1/(2 tau_g)) w_i c_v T (e_i.F) / cs^2 */
void or_correction_term(double tau_g, double cv, double T, double Fx, double Fy,
                        double Ci[9])
{
    double pre = 1.0 - 1.0 / (2.0 * tau_g);
    for (int i = 0; i < 9; ++i) {
        double eF = EX[i] * Fx + EY[i] * Fy;
        Ci[i] = pre * OMEGA[i] * cv * T * eF / CS2;
    }
}

/* ---------------------------------------------------------------------- */
/* Density and temperature at every site from the pre-collision
 * populations:  rho = sum_i f_i,  rho c_v T = sum_i g_i.  Then psi^2 and,
 * when beta != 0, psi (which needs psi^2 >= 0).                            */
static int macroscopic_fields(const or_params* P, const double* f, const double* g,
                              double* rho, double* T, double* psi, double* psi2,
                              int nthreads)
{
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    int err = OR_OK;
    (void)nthreads;
#pragma omp parallel for num_threads(nthreads) schedule(static) reduction(max : err)
    for (int64_t s = 0; s < N; ++s) {
        double r = 0.0, e = 0.0;
        for (int i = 0; i < 9; ++i) {
            r += f[i * N + s];
            e += g[i * N + s];
        }
        rho[s] = r;
        T[s] = e / (r * P->cv);
        psi2[s] = or_psi_sq(P, r, T[s]);
        psi[s] = 0.0;
        if (!isfinite(r) || !isfinite(T[s])) {
            if (err < OR_ERR_NONFINITE) err = OR_ERR_NONFINITE;
        }
        if (P->beta != 0.0) {
            if (psi2[s] < 0.0) {
                if (err < OR_ERR_PSI_DOMAIN) err = OR_ERR_PSI_DOMAIN;
                psi[s] = NAN;
            } else {
                psi[s] = sqrt(psi2[s]);
            }
        }
    }
    return err;
}

/* Pseudopotential force at (x, y), Eq. (4) (Eq. (2) when beta = 1):
 * F = -G [ beta psi(x) sum_i w ψ(x+e_i) e_i + (1-beta)/2 sum_i w ψ^2(x+e_i) e_i ]
 * with w(1) = 1/3 on the axes and w(2) = 1/12 on the diagonals.  Each sum is
 * grouped into the pairs of opposite directions.                           */
static void force_sum(const or_params* P, const double* psi, const double* psi2, int64_t C,
                      int64_t E, int64_t W, int64_t N_, int64_t S, int64_t NE, int64_t NW,
                      int64_t SW, int64_t SE, double* Fx, double* Fy)
{
    const double w1 = 1.0 / 3.0, w2 = 1.0 / 12.0;
    double fx = 0.0, fy = 0.0;
    if (P->beta != 0.0) {
        double s1x = w1 * (psi[E] - psi[W]) + w2 * ((psi[NE] - psi[SW]) + (psi[SE] - psi[NW]));
        double s1y = w1 * (psi[N_] - psi[S]) + w2 * ((psi[NE] - psi[SW]) + (psi[NW] - psi[SE]));
        fx += P->beta * psi[C] * s1x;
        fy += P->beta * psi[C] * s1y;
    }
    if (P->beta != 1.0) {
        double s2x = w1 * (psi2[E] - psi2[W]) + w2 * ((psi2[NE] - psi2[SW]) + (psi2[SE] - psi2[NW]));
        double s2y = w1 * (psi2[N_] - psi2[S]) + w2 * ((psi2[NE] - psi2[SW]) + (psi2[NW] - psi2[SE]));
        fx += 0.5 * (1.0 - P->beta) * s2x;
        fy += 0.5 * (1.0 - P->beta) * s2y;
    }
    *Fx = -P->G * fx;
    *Fy = -P->G * fy;
}

static void force_at(const or_params* P, const double* psi, const double* psi2,
                     int x, int y, double* Fx, double* Fy)
{
    const int nx = P->nx, ny = P->ny;
    int xe = wrap(x + 1, nx), xw = wrap(x - 1, nx);
    int yn = wrap(y + 1, ny), ys = wrap(y - 1, ny);
    force_sum(P, psi, psi2, (int64_t)y * nx + x, (int64_t)y * nx + xe, (int64_t)y * nx + xw,
              (int64_t)yn * nx + x, (int64_t)ys * nx + x, (int64_t)yn * nx + xe,
              (int64_t)yn * nx + xw, (int64_t)ys * nx + xw, (int64_t)ys * nx + xe, Fx, Fy);
}

/* Collision of one site: Eq. (1) with F_i for f, and Eq. (7) (or Eq. (24)
 * with C_i of Eq. (25)) for g.  Writes post-collision values fs, gs and the
 * macroscopic velocity.                                                     */
static void collide_site(const or_params* P, const double fl[9], const double gl[9],
                         double rho, double T, double Fx, double Fy,
                         double fs[9], double gs[9], double* ux_out, double* uy_out)
{
    double mx = 0.0, my = 0.0;
    for (int i = 0; i < 9; ++i) {
        mx += EX[i] * fl[i];
        my += EY[i] * fl[i];
    }
    double ux = (mx + 0.5 * Fx) / rho;
    double uy = (my + 0.5 * Fy) / rho;

    double feq[9], Fi[9], Ci[9];
    or_feq(rho, ux, uy, feq);
    or_forcing_term(P->tau_f, ux, uy, Fx, Fy, Fi);
    or_correction_term(P->tau_g, P->cv, T, Fx, Fy, Ci);

    for (int i = 0; i < 9; ++i) {
        fs[i] = fl[i] - (1.0 / P->tau_f) * (fl[i] - feq[i]) + Fi[i];
        double geq = P->cv * T * feq[i];
        gs[i] = gl[i] - (1.0 / P->tau_g) * (gl[i] - geq);
        if (P->thermal == OR_THERMAL_EQ24) gs[i] += Ci[i];
    }
    if (ux_out) *ux_out = ux;
    if (uy_out) *uy_out = uy;
}

static int check_params(const or_params* P)
{
    if (!P || P->nx < 3 || P->ny < 3) return OR_ERR_ARG;
    if (!(P->tau_f > 0.5) || !(P->tau_g > 0.5) || P->G == 0.0 || !(P->cv > 0.0))
        return OR_ERR_ARG;
    if (P->eos < 0 || P->eos > 2 || P->thermal < 0 || P->thermal > 1) return OR_ERR_ARG;
    return OR_OK;
}

/* ---------------------------------------------------------------------- */
/* Natural convection in a square cavity (Sec. III B).  nx-by-ny fluid
 * nodes enclosed by walls half a lattice spacing outside the outermost
 * nodes (so the distance between the side walls is L = nx).  The paper
 * does not state its boundary treatment; readings (listed in the design
 * notes):
 *   - f: halfway bounce-back on every wall (no slip): a population that
 *     would stream into a wall returns to its node with the opposite
 *     direction, f_{-i}(x, t+1) = f*_i(x, t).
 *   - g on the adiabatic bottom and top walls: the same bounce-back (no
 *     energy flux through the wall).
 *   - g on the isothermal side walls (T_h at x = -1/2, T_l at x = nx - 1/2):
 *     anti-bounce-back, g_{-i}(x, t+1) = -g*_i(x, t) + 2 w_i rho(x) c_v T_w,
 *     which holds rho c_v T = rho c_v T_w at the wall to second order.  A
 *     population that reaches a corner (outside in both x and y) takes the
 *     side-wall rule.
 *   - the pseudopotential at a wall node is that of the nearest fluid node
 *     (the force stencil reads psi^2 at clamped coordinates).
 *   - buoyancy: G = (0, -rho g) is added to the pseudopotential force
 *     (Sec. III B: with the ideal EOS no Boussinesq assumption is needed).
 * The step otherwise is or_step: same fields, force, collision.           */
typedef struct or_cavity {
    double T_hot, T_cold; /* side-wall temperatures (left, right) */
    double g_grav;        /* gravity acceleration along -y        */
} or_cavity;

static int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

static void force_at_clamped(const or_params* P, const double* psi, const double* psi2,
                             int x, int y, double* Fx, double* Fy)
{
    const int nx = P->nx, ny = P->ny;
    int xe = clampi(x + 1, nx), xw = clampi(x - 1, nx);
    int yn = clampi(y + 1, ny), ys = clampi(y - 1, ny);
    force_sum(P, psi, psi2, (int64_t)y * nx + x, (int64_t)y * nx + xe, (int64_t)y * nx + xw,
              (int64_t)yn * nx + x, (int64_t)ys * nx + x, (int64_t)yn * nx + xe,
              (int64_t)yn * nx + xw, (int64_t)ys * nx + xw, (int64_t)ys * nx + xe, Fx, Fy);
}

static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* Force at a cavity node: the pseudopotential force with psi at a wall node
 * taken from its nearest fluid node, plus the buoyancy (0, -rho g).       */
static void cavity_force(const or_params* P, const or_cavity* Cv, const double* psi,
                         const double* psi2, const double* rho, int x, int y, double* Fx,
                         double* Fy)
{
    force_at_clamped(P, psi, psi2, x, y, Fx, Fy);
    *Fy += -rho[(int64_t)y * P->nx + x] * Cv->g_grav;
}

/* One cavity step, t -> t+1 (state convention as or_step, walls as above). */
int or_step_cavity(const or_params* P, const or_cavity* Cv, const double* f, const double* g,
                   double* fn, double* gn, int nthreads)
{
    int err = check_params(P);
    if (err) return err;
    if (!Cv) return OR_ERR_ARG;
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* T = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* psi2 = (double*)malloc(sizeof(double) * N);
    if (!rho || !T || !psi || !psi2) {
        free(rho); free(T); free(psi); free(psi2);
        return OR_ERR_ARG;
    }
    if (nthreads < 1) nthreads = 1;
    err = macroscopic_fields(P, f, g, rho, T, psi, psi2, nthreads);

#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t s = (int64_t)y * nx + x;
            double fl[9], gl[9], fs[9], gs[9], Fx, Fy;
            for (int i = 0; i < 9; ++i) {
                fl[i] = f[i * N + s];
                gl[i] = g[i * N + s];
            }
            cavity_force(P, Cv, psi, psi2, rho, x, y, &Fx, &Fy);
            collide_site(P, fl, gl, rho[s], T[s], Fx, Fy, fs, gs, NULL, NULL);
            for (int i = 0; i < 9; ++i) {
                int xd = x + EX[i], yd = y + EY[i];
                int out_x = xd < 0 || xd >= nx, out_y = yd < 0 || yd >= ny;
                if (!out_x && !out_y) {
                    int64_t d = (int64_t)yd * nx + xd;
                    fn[i * N + d] = fs[i];
                    gn[i * N + d] = gs[i];
                } else {
                    int o = OPP[i];
                    fn[o * N + s] = fs[i];
                    if (out_x) {
                        double Tw = xd < 0 ? Cv->T_hot : Cv->T_cold;
                        gn[o * N + s] = -gs[i] + 2.0 * OMEGA[i] * rho[s] * P->cv * Tw;
                    } else {
                        gn[o * N + s] = gs[i];
                    }
                }
            }
        }
    }
    free(rho); free(T); free(psi); free(psi2);
    return err;
}

/* Average Nusselt number at the hot wall (x = -1/2), as Table II reports it:
 * Nu = (L / (T_h - T_l)) < -dT/dx >_y at the wall, L = nx, with dT/dx at the
 * wall from the quadratic through the first three nodes (distances 1/2, 3/2,
 * 5/2 from the wall): dT/dx = -2 T(0) + 3 T(1) - T(2).                     */
double or_nusselt_hot(const or_params* P, const or_cavity* Cv, const double* T)
{
    const int nx = P->nx, ny = P->ny;
    double acc = 0.0;
    for (int y = 0; y < ny; ++y) {
        const int64_t s = (int64_t)y * nx;
        acc += -(-2.0 * T[s] + 3.0 * T[s + 1] - T[s + 2]);
    }
    return (double)nx / (Cv->T_hot - Cv->T_cold) * (acc / ny);
}

/* The same from the energy that crosses the hot-wall links in one step (the
 * method's own flux; it sees lambda_eff of Eq. (23), not lambda): a
 * population g*_i (i = 3, 6, 7, pointing into the wall) leaves node (0, y)
 * and g_{-i} = -g*_i + 2 w_i rho c_v T_h comes back, so the energy entering
 * the fluid is sum_i 2 (g_{-i}(0, y) - w_i rho c_v T_h) over the
 * pre-collision state at steady state.  Nu = <q>_y / (lambda0 (T_h - T_l) / L)
 * with lambda0 = rho0 c_v cs^2 (tau_g - 1/2), rho0 the mean density.      */
double or_nusselt_hot_flux(const or_params* P, const or_cavity* Cv, const double* f, const double* g)
{
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    static const int IN_WALL[3] = {3, 6, 7};
    double mass = 0.0;
    for (int i = 0; i < 9; ++i)
        for (int64_t s = 0; s < N; ++s) mass += f[i * N + s];
    const double rho0 = mass / (double)N;
    double q = 0.0;
    for (int y = 0; y < ny; ++y) {
        const int64_t s = (int64_t)y * nx;
        double rho = 0.0;
        for (int i = 0; i < 9; ++i) rho += f[i * N + s];
        for (int k = 0; k < 3; ++k) {
            const int i = IN_WALL[k];
            q += 2.0 * (g[OPP[i] * N + s] - OMEGA[i] * rho * P->cv * Cv->T_hot);
        }
    }
    const double lambda0 = rho0 * P->cv * CS2 * (P->tau_g - 0.5);
    return (q / ny) / (lambda0 * (Cv->T_hot - Cv->T_cold) / (double)nx);
}

/* ---------------------------------------------------------------------- */
/* One full time step, t -> t+1.  f, g: pre-collision state at t; fn, gn
 * receive the pre-collision state at t+1 (streaming: f_i(x+e_i) <- f*_i(x)).
 * Returns OR_OK, or the worst error seen (the step is still completed).    */
int or_step(const or_params* P, const double* f, const double* g, double* fn,
            double* gn, int nthreads)
{
    int err = check_params(P);
    if (err) return err;
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* T = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* psi2 = (double*)malloc(sizeof(double) * N);
    if (!rho || !T || !psi || !psi2) {
        free(rho); free(T); free(psi); free(psi2);
        return OR_ERR_ARG;
    }
    if (nthreads < 1) nthreads = 1;
    err = macroscopic_fields(P, f, g, rho, T, psi, psi2, nthreads);

#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t s = (int64_t)y * nx + x;
            double fl[9], gl[9], fs[9], gs[9], Fx, Fy;
            for (int i = 0; i < 9; ++i) {
                fl[i] = f[i * N + s];
                gl[i] = g[i * N + s];
            }
            force_at(P, psi, psi2, x, y, &Fx, &Fy);
            collide_site(P, fl, gl, rho[s], T[s], Fx, Fy, fs, gs, NULL, NULL);
            for (int i = 0; i < 9; ++i) {
                int64_t d = (int64_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
                fn[i * N + d] = fs[i];
                gn[i * N + d] = gs[i];
            }
        }
    }
    free(rho); free(T); free(psi); free(psi2);
    return err;
}

/* Macroscopic fields of the pre-collision state at t: rho, u (including the
 * half-force term of the Guo scheme), T, and the force F.  Any output may be
 * NULL.                                                                     */
int or_moments(const or_params* P, const double* f, const double* g, double* rho_out,
               double* ux_out, double* uy_out, double* T_out, double* Fx_out,
               double* Fy_out)
{
    int err = check_params(P);
    if (err) return err;
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* T = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* psi2 = (double*)malloc(sizeof(double) * N);
    if (!rho || !T || !psi || !psi2) {
        free(rho); free(T); free(psi); free(psi2);
        return OR_ERR_ARG;
    }
    err = macroscopic_fields(P, f, g, rho, T, psi, psi2, 1);
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t s = (int64_t)y * nx + x;
            double Fx, Fy, mx = 0.0, my = 0.0;
            force_at(P, psi, psi2, x, y, &Fx, &Fy);
            for (int i = 0; i < 9; ++i) {
                mx += EX[i] * f[i * N + s];
                my += EY[i] * f[i * N + s];
            }
            if (rho_out) rho_out[s] = rho[s];
            if (T_out) T_out[s] = T[s];
            if (ux_out) ux_out[s] = (mx + 0.5 * Fx) / rho[s];
            if (uy_out) uy_out[s] = (my + 0.5 * Fy) / rho[s];
            if (Fx_out) Fx_out[s] = Fx;
            if (Fy_out) Fy_out[s] = Fy;
        }
    }
    free(rho); free(T); free(psi); free(psi2);
    return err;
}

/* Initial state: f = f^eq(rho0, u = 0), g = c_v T0 f^eq(rho0, 0). */
int or_init_equilibrium(const or_params* P, const double* rho0, const double* T0,
                        double* f, double* g)
{
    int err = check_params(P);
    if (err) return err;
    const int64_t N = (int64_t)P->nx * P->ny;
    for (int64_t s = 0; s < N; ++s) {
        double feq[9];
        or_feq(rho0[s], 0.0, 0.0, feq);
        for (int i = 0; i < 9; ++i) {
            f[i * N + s] = feq[i];
            g[i * N + s] = P->cv * T0[s] * feq[i];
        }
    }
    return OR_OK;
}

/* Initial state at rest under the pseudopotential force.  The paper states no
 * initial condition; this start is a reading of the velocity definition of
 * the forcing scheme of Eq. (1): u = (sum_i e_i f_i + F/2) / rho, so a state
 * whose velocity is zero carries the first moment sum_i e_i f_i = -F/2.
 *   psi from rho0 and T0 (Sec. II A), F of Eq. (4) (Eq. (2) when beta = 1),
 *   v = -F / (2 rho0),  f = f^eq(rho0, v),  g = c_v T0 f^eq(rho0, v).
 * Returns OR_ERR_PSI_DOMAIN (state still written, NaN where psi is undefined)
 * when psi^2 < 0 and beta != 0.                                            */
int or_init_balanced(const or_params* P, const double* rho0, const double* T0,
                     double* f, double* g)
{
    int err = check_params(P);
    if (err) return err;
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    double* psi = (double*)malloc(sizeof(double) * N);
    double* psi2 = (double*)malloc(sizeof(double) * N);
    if (!psi || !psi2) {
        free(psi); free(psi2);
        return OR_ERR_ARG;
    }
    for (int64_t s = 0; s < N; ++s) {
        psi2[s] = or_psi_sq(P, rho0[s], T0[s]);
        psi[s] = 0.0;
        if (P->beta != 0.0) {
            if (psi2[s] < 0.0) {
                if (err < OR_ERR_PSI_DOMAIN) err = OR_ERR_PSI_DOMAIN;
                psi[s] = NAN;
            } else {
                psi[s] = sqrt(psi2[s]);
            }
        }
    }
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t s = (int64_t)y * nx + x;
            double Fx, Fy, feq[9];
            force_at(P, psi, psi2, x, y, &Fx, &Fy);
            double vx = -Fx / (2.0 * rho0[s]);
            double vy = -Fy / (2.0 * rho0[s]);
            or_feq(rho0[s], vx, vy, feq);
            for (int i = 0; i < 9; ++i) {
                f[i * N + s] = feq[i];
                g[i * N + s] = P->cv * T0[s] * feq[i];
            }
        }
    }
    free(psi); free(psi2);
    return err;
}

/* The state at t+1 at a list of sites only, from the full state at t.
 * Site x at t+1 receives f*_i(x - e_i), so the collisions of the nine source
 * sites are computed, each with the force from the psi values around it.
 * out_f, out_g: [n_sites][9].  Used to check a large lattice at sampled
 * sites without a full step.                                               */
int or_step_sites(const or_params* P, const double* f, const double* g, int64_t n_sites,
                  const int64_t* sites, double* out_f, double* out_g)
{
    int err = check_params(P);
    if (err) return err;
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    for (int64_t k = 0; k < n_sites; ++k) {
        int64_t d = sites[k];
        if (d < 0 || d >= N) return OR_ERR_ARG;
        int xd = (int)(d % nx), yd = (int)(d / nx);
        for (int i = 0; i < 9; ++i) {
            int xs = wrap(xd - EX[i], nx), ys = wrap(yd - EY[i], ny);
            /* psi, psi^2, rho, T on the 3x3 block around the source site,
             * stored in a local 3x3 lattice so force_at can be reused.    */
            or_params L = *P;
            L.nx = 3;
            L.ny = 3;
            double rho9[9], T9[9], psi9[9], psi29[9];
            for (int by = 0; by < 3; ++by) {
                for (int bx = 0; bx < 3; ++bx) {
                    int64_t s = (int64_t)wrap(ys + by - 1, ny) * nx + wrap(xs + bx - 1, nx);
                    double r = 0.0, e = 0.0;
                    for (int j = 0; j < 9; ++j) {
                        r += f[j * N + s];
                        e += g[j * N + s];
                    }
                    int b = by * 3 + bx;
                    rho9[b] = r;
                    T9[b] = e / (r * P->cv);
                    psi29[b] = or_psi_sq(P, r, T9[b]);
                    psi9[b] = 0.0;
                    if (P->beta != 0.0) {
                        if (psi29[b] < 0.0) {
                            err = OR_ERR_PSI_DOMAIN;
                            psi9[b] = NAN;
                        } else {
                            psi9[b] = sqrt(psi29[b]);
                        }
                    }
                }
            }
            double Fx, Fy, fl[9], gl[9], fs[9], gs[9];
            force_at(&L, psi9, psi29, 1, 1, &Fx, &Fy);
            int64_t s = (int64_t)ys * nx + xs;
            for (int j = 0; j < 9; ++j) {
                fl[j] = f[j * N + s];
                gl[j] = g[j * N + s];
            }
            collide_site(P, fl, gl, rho9[4], T9[4], Fx, Fy, fs, gs, NULL, NULL);
            out_f[k * 9 + i] = fs[i];
            out_g[k * 9 + i] = gs[i];
        }
    }
    return err;
}

/* Neumaier-compensated sum: the accurate reference for the totals. */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum* a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

/* Conserved totals of the pre-collision state: mass sum rho, energy
 * sum rho c_v T (= sum of all g_i), momentum sum rho u (with the half-force
 * term), out[0..3] = mass, energy, px, py.                                  */
int or_totals(const or_params* P, const double* f, const double* g, double out[4])
{
    int err = check_params(P);
    if (err) return err;
    const int64_t N = (int64_t)P->nx * P->ny;
    double* ux = (double*)malloc(sizeof(double) * N);
    double* uy = (double*)malloc(sizeof(double) * N);
    double* rho = (double*)malloc(sizeof(double) * N);
    if (!ux || !uy || !rho) {
        free(ux); free(uy); free(rho);
        return OR_ERR_ARG;
    }
    err = or_moments(P, f, g, rho, ux, uy, NULL, NULL, NULL);
    nsum m = {0, 0}, e = {0, 0}, px = {0, 0}, py = {0, 0};
    for (int64_t s = 0; s < N; ++s) {
        for (int i = 0; i < 9; ++i) {
            nsum_add(&m, f[i * N + s]);
            nsum_add(&e, g[i * N + s]);
        }
        nsum_add(&px, rho[s] * ux[s]);
        nsum_add(&py, rho[s] * uy[s]);
    }
    out[0] = m.s + m.c;
    out[1] = e.s + e.c;
    out[2] = px.s + px.c;
    out[3] = py.s + py.c;
    free(ux); free(uy); free(rho);
    return err;
}

/* Steady-state residual between two density/temperature snapshots taken
 * K steps apart:  r = max over phi in {rho, T} of ||phi1 - phi0||_2 / (K ||phi1||_2). */
double or_residual(int64_t n, const double* rho0, const double* T0, const double* rho1,
                   const double* T1, int64_t K)
{
    nsum dr = {0, 0}, nr = {0, 0}, dT = {0, 0}, nT = {0, 0};
    for (int64_t s = 0; s < n; ++s) {
        nsum_add(&dr, (rho1[s] - rho0[s]) * (rho1[s] - rho0[s]));
        nsum_add(&nr, rho1[s] * rho1[s]);
        nsum_add(&dT, (T1[s] - T0[s]) * (T1[s] - T0[s]));
        nsum_add(&nT, T1[s] * T1[s]);
    }
    double r_rho = sqrt(dr.s + dr.c) / ((double)K * sqrt(nr.s + nr.c));
    double r_T = sqrt(dT.s + dT.c) / ((double)K * sqrt(nT.s + nT.c));
    return r_rho > r_T ? r_rho : r_T;
}

/* Critical point of the EOS: the (rho_c, T_c) where dp/drho = d2p/drho2 = 0.
 * Found by bisection on T of  min_rho dp/drho(rho, T) = 0, the inner minimum
 * by golden-section search.  Derivatives are central differences.           */
static double dp_drho(const or_params* P, double rho, double T)
{
    double h = 1e-6 * (rho > 1e-3 ? rho : 1e-3);
    return (or_p_eos(P, rho + h, T) - or_p_eos(P, rho - h, T)) / (2.0 * h);
}

static double min_dp_drho(const or_params* P, double T, double lo, double hi, double* arg)
{
    const double gr = 0.5 * (sqrt(5.0) - 1.0);
    double a = lo, b = hi;
    double c = b - gr * (b - a), d = a + gr * (b - a);
    for (int it = 0; it < 200; ++it) {
        if (dp_drho(P, c, T) < dp_drho(P, d, T)) b = d;
        else a = c;
        c = b - gr * (b - a);
        d = a + gr * (b - a);
    }
    *arg = 0.5 * (a + b);
    return dp_drho(P, *arg, T);
}

int or_critical_point(const or_params* P, double* Tc, double* rhoc)
{
    if (!P || P->eos == OR_EOS_IDEAL) return OR_ERR_ARG;
    /* rho range inside the EOS's domain: vdW needs b rho < 1, CS eta < 1 */
    double hi = (P->eos == OR_EOS_VDW) ? 0.99 / P->b : 3.96 / P->b;
    double lo = 1e-4 * hi;
    double Tlo = 1e-6, Thi = 10.0 * P->a / (P->b * P->R);
    double arg = 0.0;
    for (int it = 0; it < 200; ++it) {
        double Tm = 0.5 * (Tlo + Thi);
        if (min_dp_drho(P, Tm, lo, hi, &arg) < 0.0) Tlo = Tm;
        else Thi = Tm;
    }
    *Tc = 0.5 * (Tlo + Thi);
    min_dp_drho(P, *Tc, lo, hi, &arg);
    *rhoc = arg;
    return OR_OK;
}

int or_num_threads_available(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Finite-difference temperature treatment, Eqs. (26)-(27).
 *
 * Eq. (26): dT/dt = -u . grad T + (1 / (rho c_v)) div(lambda grad T) = K(T).
 * Readings (the paper gives no more than this):
 *   - lambda = rho c_v chi with chi = (tau_g - 1/2) c_s^2, the diffusivity of
 *     the thermal LB equation, so that the three treatments solve the same
 *     Eq. (6); then K = -u . grad T + chi (lap T + grad rho . grad T / rho).
 *   - u is the velocity of the density LBE, (sum_i e_i f_i + F/2) / rho, and
 *     rho, u are taken at time n for both stages of the update.
 *   - "isotropic central schemes": on the D2Q9 stencil,
 *       grad phi (x) = (1/cs^2) sum_i omega_i e_i phi(x + e_i),
 *       lap  phi (x) = (2/cs^2) sum_i omega_i (phi(x + e_i) - phi(x)).
 * Eq. (27): T^{n+1} = T^n + (dt/2)(h1 + h2), h1 = K(T^n), h2 = K(T^n + a dt h1)
 * with a = 1/2 as printed, or a = 1 (Heun's second-order method, which the
 * printed form is not); dt = 1.                                            */
/* K of Eq. (26) at one site from the values at its 8 neighbours (index i =
 * 1..8 in the lattice order) and at the site itself:
 *   grad phi = (1/cs^2) sum_i w_i e_i phi(x + e_i),
 *   lap phi  = (2/cs^2) sum_i w_i (phi(x + e_i) - phi(x)).                  */
static double fd_K_site(const double Tn[9], const double rn[9], double Tc, double rc, double ux,
                        double uy, double chi)
{
    double gTx = 0.0, gTy = 0.0, grx = 0.0, gry = 0.0, lap = 0.0;
    for (int i = 1; i < 9; ++i) {
        gTx += OMEGA[i] * EX[i] * Tn[i];
        gTy += OMEGA[i] * EY[i] * Tn[i];
        grx += OMEGA[i] * EX[i] * rn[i];
        gry += OMEGA[i] * EY[i] * rn[i];
        lap += OMEGA[i] * (Tn[i] - Tc);
    }
    gTx /= CS2;
    gTy /= CS2;
    grx /= CS2;
    gry /= CS2;
    lap *= 2.0 / CS2;
    return -(ux * gTx + uy * gTy) + chi * (lap + (grx * gTx + gry * gTy) / rc);
}

void or_fd_rhs(const or_params* P, const double* T, const double* rho, const double* ux,
               const double* uy, double* K)
{
    const int nx = P->nx, ny = P->ny;
    const double chi = (P->tau_g - 0.5) * CS2;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            const int64_t c = (int64_t)y * nx + x;
            double Tn[9], rn[9];
            for (int i = 1; i < 9; ++i) {
                const int64_t n = (int64_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
                Tn[i] = T[n];
                rn[i] = rho[n];
            }
            K[c] = fd_K_site(Tn, rn, T[c], rho[c], ux[c], uy[c], chi);
        }
    }
}

/* One Eq. (27) update of T with rho, u fixed; printed != 0 takes a = 1/2. */
int or_fd_rk2(const or_params* P, const double* T, const double* rho, const double* ux,
              const double* uy, int printed, double* Tn)
{
    const int64_t N = (int64_t)P->nx * P->ny;
    double* h1 = (double*)malloc(sizeof(double) * N);
    double* h2 = (double*)malloc(sizeof(double) * N);
    double* Ts = (double*)malloc(sizeof(double) * N);
    if (!h1 || !h2 || !Ts) {
        free(h1); free(h2); free(Ts);
        return OR_ERR_ARG;
    }
    const double a = printed ? 0.5 : 1.0;
    or_fd_rhs(P, T, rho, ux, uy, h1);
    for (int64_t s = 0; s < N; ++s) Ts[s] = T[s] + a * h1[s];
    or_fd_rhs(P, Ts, rho, ux, uy, h2);
    int err = OR_OK;
    for (int64_t s = 0; s < N; ++s) {
        Tn[s] = T[s] + 0.5 * (h1[s] + h2[s]);
        if (!isfinite(Tn[s])) err = OR_ERR_NONFINITE;
    }
    free(h1); free(h2); free(Ts);
    return err;
}

/* One step of the hybrid scheme: f by Eq. (1) with psi(rho, T^n) (or T_psi),
 * then T by Eq. (27).  f: pre-collision populations at n (9 planes), T: T^n;
 * fn, Tn: the state at n + 1.  rho_out, ux_out, uy_out (may be NULL) receive
 * rho^n and u^n. */
int or_step_fd(const or_params* P, const double* f, const double* T, double* fn, double* Tn,
               int printed, double* rho_out, double* ux_out, double* uy_out, int nthreads)
{
    if (!P || P->nx < 3 || P->ny < 3 || !(P->tau_f > 0.5) || !(P->tau_g > 0.5) || P->G == 0.0 ||
        !(P->cv > 0.0) || P->eos < 0 || P->eos > 2)
        return OR_ERR_ARG;
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* psi2 = (double*)malloc(sizeof(double) * N);
    double* ux = (double*)malloc(sizeof(double) * N);
    double* uy = (double*)malloc(sizeof(double) * N);
    if (!rho || !psi || !psi2 || !ux || !uy) {
        free(rho); free(psi); free(psi2); free(ux); free(uy);
        return OR_ERR_ARG;
    }
    if (nthreads < 1) nthreads = 1;
    int err = OR_OK;
    for (int64_t s = 0; s < N; ++s) {
        double r = 0.0;
        for (int i = 0; i < 9; ++i) r += f[i * N + s];
        rho[s] = r;
        const double Te = P->psi_uses_local_T ? T[s] : P->T_psi;
        psi2[s] = or_psi_sq(P, r, Te);
        psi[s] = 0.0;
        if (!isfinite(r) || !isfinite(T[s])) err = err < OR_ERR_NONFINITE ? OR_ERR_NONFINITE : err;
        if (P->beta != 0.0) {
            if (psi2[s] < 0.0) {
                err = OR_ERR_PSI_DOMAIN;
                psi[s] = NAN;
            } else {
                psi[s] = sqrt(psi2[s]);
            }
        }
    }
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            const int64_t s = (int64_t)y * nx + x;
            double fl[9], gl[9], fs[9], gs[9], Fx, Fy;
            for (int i = 0; i < 9; ++i) {
                fl[i] = f[i * N + s];
                gl[i] = 0.0;
            }
            force_at(P, psi, psi2, x, y, &Fx, &Fy);
            collide_site(P, fl, gl, rho[s], T[s], Fx, Fy, fs, gs, &ux[s], &uy[s]);
            for (int i = 0; i < 9; ++i) {
                const int64_t d = (int64_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
                fn[i * N + d] = fs[i];
            }
        }
    }
    const int e2 = or_fd_rk2(P, T, rho, ux, uy, printed, Tn);
    if (e2 > err) err = e2;
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * N);
    if (ux_out) memcpy(ux_out, ux, sizeof(double) * N);
    if (uy_out) memcpy(uy_out, uy, sizeof(double) * N);
    free(rho); free(psi); free(psi2); free(ux); free(uy);
    return err;
}

/* ---------------------------------------------------------------------- */
/* The hybrid scheme (Eqs. 26-27) in the cavity of Sec. III B.  The density
 * LBE takes the cavity rules of or_step_cavity (bounce-back, clamped psi,
 * buoyancy); K of Eq. (26) reads its neighbours through the walls as ghost
 * values (reading listed in the design notes): across a side wall the
 * temperature is reflected about the wall value, 2 T_w - X(mirror node),
 * which puts X = T_w at the wall to second order; across the adiabatic
 * bottom and top walls X(mirror node) (zero normal gradient); rho is
 * mirrored everywhere; a neighbour outside in x takes the side-wall rule.
 * The intermediate temperature of the second stage uses the same rule.     */
static void fd_rhs_cavity(const or_params* P, const or_cavity* Cv, const double* X,
                          const double* rho, const double* ux, const double* uy, double* K)
{
    const int nx = P->nx, ny = P->ny;
    const double chi = (P->tau_g - 0.5) * CS2;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            const int64_t c = (int64_t)y * nx + x;
            double Xn[9], rn[9];
            for (int i = 1; i < 9; ++i) {
                const int xn = x + EX[i], yn = y + EY[i];
                const int64_t m = (int64_t)clampi(yn, ny) * nx + clampi(xn, nx);
                rn[i] = rho[m];
                if (xn < 0 || xn >= nx) {
                    const double Tw = xn < 0 ? Cv->T_hot : Cv->T_cold;
                    Xn[i] = 2.0 * Tw - X[m];
                } else {
                    Xn[i] = X[m];
                }
            }
            K[c] = fd_K_site(Xn, rn, X[c], rho[c], ux[c], uy[c], chi);
        }
    }
}

int or_step_fd_cavity(const or_params* P, const or_cavity* Cv, const double* f, const double* T,
                      double* fn, double* Tn, int printed, double* rho_out, double* ux_out,
                      double* uy_out, int nthreads)
{
    if (!P || !Cv || P->nx < 3 || P->ny < 3 || !(P->tau_f > 0.5) || !(P->tau_g > 0.5) ||
        P->G == 0.0 || !(P->cv > 0.0) || P->eos < 0 || P->eos > 2)
        return OR_ERR_ARG;
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* psi2 = (double*)malloc(sizeof(double) * N);
    double* ux = (double*)malloc(sizeof(double) * N);
    double* uy = (double*)malloc(sizeof(double) * N);
    double* h1 = (double*)malloc(sizeof(double) * N);
    double* h2 = (double*)malloc(sizeof(double) * N);
    double* Ts = (double*)malloc(sizeof(double) * N);
    if (!rho || !psi || !psi2 || !ux || !uy || !h1 || !h2 || !Ts) {
        free(rho); free(psi); free(psi2); free(ux); free(uy); free(h1); free(h2); free(Ts);
        return OR_ERR_ARG;
    }
    if (nthreads < 1) nthreads = 1;
    int err = OR_OK;
    for (int64_t s = 0; s < N; ++s) {
        double r = 0.0;
        for (int i = 0; i < 9; ++i) r += f[i * N + s];
        rho[s] = r;
        const double Te = P->psi_uses_local_T ? T[s] : P->T_psi;
        psi2[s] = or_psi_sq(P, r, Te);
        psi[s] = 0.0;
        if (!isfinite(r) || !isfinite(T[s])) err = err < OR_ERR_NONFINITE ? OR_ERR_NONFINITE : err;
        if (P->beta != 0.0) {
            if (psi2[s] < 0.0) {
                err = OR_ERR_PSI_DOMAIN;
                psi[s] = NAN;
            } else {
                psi[s] = sqrt(psi2[s]);
            }
        }
    }
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            const int64_t s = (int64_t)y * nx + x;
            double fl[9], gl[9], fs[9], gs[9], Fx, Fy;
            for (int i = 0; i < 9; ++i) {
                fl[i] = f[i * N + s];
                gl[i] = 0.0;
            }
            cavity_force(P, Cv, psi, psi2, rho, x, y, &Fx, &Fy);
            collide_site(P, fl, gl, rho[s], T[s], Fx, Fy, fs, gs, &ux[s], &uy[s]);
            for (int i = 0; i < 9; ++i) {
                const int xd = x + EX[i], yd = y + EY[i];
                if (xd >= 0 && xd < nx && yd >= 0 && yd < ny)
                    fn[i * N + (int64_t)yd * nx + xd] = fs[i];
                else
                    fn[OPP[i] * N + s] = fs[i];
            }
        }
    }
    const double a = printed ? 0.5 : 1.0;
    fd_rhs_cavity(P, Cv, T, rho, ux, uy, h1);
    for (int64_t s = 0; s < N; ++s) Ts[s] = T[s] + a * h1[s];
    fd_rhs_cavity(P, Cv, Ts, rho, ux, uy, h2);
    for (int64_t s = 0; s < N; ++s) {
        Tn[s] = T[s] + 0.5 * (h1[s] + h2[s]);
        if (!isfinite(Tn[s])) err = err < OR_ERR_NONFINITE ? OR_ERR_NONFINITE : err;
    }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * N);
    if (ux_out) memcpy(ux_out, ux, sizeof(double) * N);
    if (uy_out) memcpy(uy_out, uy, sizeof(double) * N);
    free(rho); free(psi); free(psi2); free(ux); free(uy); free(h1); free(h2); free(Ts);
    return err;
}

/* Nusselt number at the hot wall of a temperature field with the wall value
 * imposed through the reflected ghost (the FD treatment).  The conductive
 * flux through the wall is lambda dT/dx with lambda = rho c_v cs^2 (tau_g -
 * 1/2) at the first node (the ghost mirrors rho) and dT/dx the central
 * difference across the wall, T(0) - (2 T_h - T(0)); it is normalised by
 * lambda0 (T_h - T_l) / L with the mean density, like or_nusselt_hot_flux.
 * rho may be NULL: the gradient alone (lambda = lambda0).                  */
double or_nusselt_hot_wall(const or_params* P, const or_cavity* Cv, const double* T,
                           const double* rho)
{
    const int nx = P->nx, ny = P->ny;
    double rho0 = 1.0;
    if (rho) {
        double m = 0.0;
        for (int64_t s = 0; s < (int64_t)nx * ny; ++s) m += rho[s];
        rho0 = m / ((double)nx * ny);
    }
    double acc = 0.0;
    for (int y = 0; y < ny; ++y) {
        const double w = rho ? rho[(int64_t)y * nx] / rho0 : 1.0;
        acc += -2.0 * w * (T[(int64_t)y * nx] - Cv->T_hot);
    }
    return (double)nx / (Cv->T_hot - Cv->T_cold) * (acc / ny);
}

/* ---------------------------------------------------------------------- */
/* Thermal flow between parallel plates (Sec. III A): nx-by-ny fluid nodes,
 * plates half a lattice spacing below y = 0 and above y = ny - 1 (gap
 * H = ny), inlet plane half a spacing left of x = 0, outlet plane half a
 * spacing right of x = nx - 1.  The paper gives no boundary scheme;
 * readings (listed in the design notes):
 *   - plates: f halfway bounce-back (no slip); g anti-bounce-back at T_w on
 *     the upper plate and, in Case A, on the lower plate; in Case B the
 *     lower plate is adiabatic (g bounce-back).  A link through a corner
 *     takes the plate rule.
 *   - inlet (uniform U_in, T_in): f bounce-back with the wall velocity,
 *     f_{-i} = f*_i - 2 w_i rho (e_i . u_in) / cs^2; g anti-bounce-back at
 *     T_in with the symmetric part of the equilibrium at u_in,
 *     g_{-i} = -g*_i + 2 w_i rho c_v T_in (1 + (e_i.u_in)^2 / (2 cs^4)
 *     - |u_in|^2 / (2 cs^2)).
 *   - outlet (fully developed, pressure level rho0 = 1): f anti-bounce-back
 *     at the outlet density with the velocity of the node,
 *     f_{-i} = -f*_i + 2 w_i rho0 (1 + (e_i.u)^2 / (2 cs^4) - |u|^2 / (2 cs^2));
 *     g: after streaming, the populations that would come from beyond the
 *     outlet are copied from the column nx - 2 (zero gradient).
 *   - psi at a node outside is that of the nearest fluid node; no gravity.
 * State convention as or_step (pre-collision at the node).                 */
typedef struct or_channel {
    double T_in, T_w, U_in;
    int32_t adiabatic_bottom; /* 0: Case A, 1: Case B */
} or_channel;

int or_step_channel(const or_params* P, const or_channel* Ch, const double* f, const double* g,
                    double* fn, double* gn, int nthreads)
{
    int err = check_params(P);
    if (err) return err;
    if (!Ch || P->nx < 3) return OR_ERR_ARG;
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* T = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* psi2 = (double*)malloc(sizeof(double) * N);
    if (!rho || !T || !psi || !psi2) {
        free(rho); free(T); free(psi); free(psi2);
        return OR_ERR_ARG;
    }
    if (nthreads < 1) nthreads = 1;
    err = macroscopic_fields(P, f, g, rho, T, psi, psi2, nthreads);
    const double uin = Ch->U_in;

#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t s = (int64_t)y * nx + x;
            double fl[9], gl[9], fs[9], gs[9], Fx, Fy;
            for (int i = 0; i < 9; ++i) {
                fl[i] = f[i * N + s];
                gl[i] = g[i * N + s];
            }
            force_at_clamped(P, psi, psi2, x, y, &Fx, &Fy);
            collide_site(P, fl, gl, rho[s], T[s], Fx, Fy, fs, gs, NULL, NULL);
            for (int i = 0; i < 9; ++i) {
                const int xd = x + EX[i], yd = y + EY[i];
                const int o = OPP[i];
                if (yd < 0 || yd >= ny) {
                    /* plate */
                    fn[o * N + s] = fs[i];
                    if (yd < 0 && Ch->adiabatic_bottom)
                        gn[o * N + s] = gs[i];
                    else
                        gn[o * N + s] = -gs[i] + 2.0 * OMEGA[i] * rho[s] * P->cv * Ch->T_w;
                } else if (xd < 0) {
                    /* inlet */
                    const double eu = EX[i] * uin;
                    fn[o * N + s] = fs[i] - 2.0 * OMEGA[i] * rho[s] * eu / CS2;
                    gn[o * N + s] = -gs[i] + 2.0 * OMEGA[i] * rho[s] * P->cv * Ch->T_in *
                                                 (1.0 + 0.5 * eu * eu / (CS2 * CS2) - 0.5 * uin * uin / CS2);
                } else if (xd < nx) {
                    const int64_t d = (int64_t)yd * nx + xd;
                    fn[i * N + d] = fs[i];
                    gn[i * N + d] = gs[i];
                } else {
                    /* outlet: f at the outlet density; g replaced below */
                    double ux, uy;
                    {
                        double mx = 0.0, my = 0.0;
                        for (int k = 0; k < 9; ++k) {
                            mx += EX[k] * fl[k];
                            my += EY[k] * fl[k];
                        }
                        ux = (mx + 0.5 * Fx) / rho[s];
                        uy = (my + 0.5 * Fy) / rho[s];
                    }
                    const double eu = EX[i] * ux + EY[i] * uy;
                    fn[o * N + s] = -fs[i] + 2.0 * OMEGA[i] * 1.0 *
                                                 (1.0 + 0.5 * eu * eu / (CS2 * CS2) - 0.5 * (ux * ux + uy * uy) / CS2);
                }
            }
        }
    }
    /* outlet: g arriving from beyond x = nx - 1 (source right of the outlet
     * and inside the plates) copies column nx - 2 */
    for (int y = 0; y < ny; ++y) {
        for (int i = 0; i < 9; ++i) {
            if (EX[i] != -1) continue;
            const int ys = y - EY[i];
            if (ys < 0 || ys >= ny) continue; /* set by the plate rule */
            const int64_t a = (int64_t)y * nx + (nx - 1), b = (int64_t)y * nx + (nx - 2);
            gn[i * N + a] = gn[i * N + b];
        }
    }
    free(rho); free(T); free(psi); free(psi2);
    return err;
}

/* Local Nusselt number along the channel at column x (Sec. III A):
 * Nu(x) = D_h q_w / (lambda (T_w - T_b)), D_h = 2 H = 2 ny, T_b the bulk
 * temperature sum(rho u_x T) / sum(rho u_x) over the column, q_w the heat
 * the upper plate's links pass into the fluid per step (as
 * or_nusselt_hot_flux) and lambda = rho c_v cs^2 (tau_g - 1/2) with the
 * density of the node next to the plate.  rho, ux, T: moments [ny][nx]. */
double or_channel_nusselt(const or_params* P, const or_channel* Ch, const double* g,
                          const double* rho, const double* ux, const double* T, int x)
{
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    static const int IN_TOP[3] = {2, 5, 6};
    double num = 0.0, den = 0.0;
    for (int y = 0; y < ny; ++y) {
        const int64_t s = (int64_t)y * nx + x;
        num += rho[s] * ux[s] * T[s];
        den += rho[s] * ux[s];
    }
    const double Tb = num / den;
    const int64_t s = (int64_t)(ny - 1) * nx + x;
    double q = 0.0;
    for (int k = 0; k < 3; ++k) {
        const int i = IN_TOP[k];
        q += 2.0 * (g[OPP[i] * N + s] - OMEGA[i] * rho[s] * P->cv * Ch->T_w);
    }
    const double lambda = rho[s] * P->cv * CS2 * (P->tau_g - 0.5);
    return 2.0 * ny * q / (lambda * (Ch->T_w - Tb));
}

/* The same with q_w / lambda replaced by the temperature gradient at the
 * upper plate, from the quadratic through the three nodes next to it
 * (distances 1/2, 3/2, 5/2): dT/dn = -2 T(ny-1) + 3 T(ny-2) - T(ny-3) toward
 * the fluid.  This is the reading under which Eq. (7) reads high.          */
double or_channel_nusselt_grad(const or_params* P, const or_channel* Ch, const double* rho,
                               const double* ux, const double* T, int x)
{
    const int nx = P->nx, ny = P->ny;
    double num = 0.0, den = 0.0;
    for (int y = 0; y < ny; ++y) {
        const int64_t s = (int64_t)y * nx + x;
        num += rho[s] * ux[s] * T[s];
        den += rho[s] * ux[s];
    }
    const double Tb = num / den;
    const double T0 = T[(int64_t)(ny - 1) * nx + x], T1 = T[(int64_t)(ny - 2) * nx + x];
    const double T2 = T[(int64_t)(ny - 3) * nx + x];
    const double dTdn = -2.0 * T0 + 3.0 * T1 - T2; /* d T / d(distance from the plate) */
    /* heat into the fluid per lambda: -dT/dn at the plate (flux along -n) */
    return 2.0 * ny * (-dTdn) / (Ch->T_w - Tb);
}


/* ---------------------------------------------------------------------- */
/* The hybrid scheme (Eqs. 26-27) in the plate channel.  The density LBE
 * takes the channel rules of or_step_channel for f; K of Eq. (26) reads its
 * neighbours through the boundaries as ghosts (reading listed in the design
 * notes): across a plate at T_w (or the inlet at T_in) the temperature is
 * reflected about the boundary value, 2 T_b - X(mirror node); across the
 * adiabatic lower plate of Case B and across the outlet X(mirror node)
 * (zero gradient); rho is mirrored; a neighbour outside in y takes the plate
 * rule.  The intermediate temperature of the second stage takes the same
 * rule.                                                                   */
static double channel_ghost_T(const or_channel* Ch, int xn, int yn, int ny, double Xm)
{
    if (yn < 0 || yn >= ny) {
        if (yn < 0 && Ch->adiabatic_bottom) return Xm;
        return 2.0 * Ch->T_w - Xm;
    }
    if (xn < 0) return 2.0 * Ch->T_in - Xm;
    return Xm; /* outlet */
}

static void fd_rhs_channel(const or_params* P, const or_channel* Ch, const double* X,
                           const double* rho, const double* ux, const double* uy, double* K)
{
    const int nx = P->nx, ny = P->ny;
    const double chi = (P->tau_g - 0.5) * CS2;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            const int64_t c = (int64_t)y * nx + x;
            double Xn[9], rn[9];
            for (int i = 1; i < 9; ++i) {
                const int xn = x + EX[i], yn = y + EY[i];
                const int64_t m = (int64_t)clampi(yn, ny) * nx + clampi(xn, nx);
                rn[i] = rho[m];
                if (xn < 0 || xn >= nx || yn < 0 || yn >= ny)
                    Xn[i] = channel_ghost_T(Ch, xn, yn, ny, X[m]);
                else
                    Xn[i] = X[m];
            }
            K[c] = fd_K_site(Xn, rn, X[c], rho[c], ux[c], uy[c], chi);
        }
    }
}

int or_step_fd_channel(const or_params* P, const or_channel* Ch, const double* f, const double* T,
                       double* fn, double* Tn, int printed, double* rho_out, double* ux_out,
                       double* uy_out, int nthreads)
{
    if (!P || !Ch || P->nx < 3 || P->ny < 3 || !(P->tau_f > 0.5) || !(P->tau_g > 0.5) ||
        P->G == 0.0 || !(P->cv > 0.0) || P->eos < 0 || P->eos > 2)
        return OR_ERR_ARG;
    const int nx = P->nx, ny = P->ny;
    const int64_t N = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* psi = (double*)malloc(sizeof(double) * N);
    double* psi2 = (double*)malloc(sizeof(double) * N);
    double* ux = (double*)malloc(sizeof(double) * N);
    double* uy = (double*)malloc(sizeof(double) * N);
    double* h1 = (double*)malloc(sizeof(double) * N);
    double* h2 = (double*)malloc(sizeof(double) * N);
    double* Ts = (double*)malloc(sizeof(double) * N);
    if (!rho || !psi || !psi2 || !ux || !uy || !h1 || !h2 || !Ts) {
        free(rho); free(psi); free(psi2); free(ux); free(uy); free(h1); free(h2); free(Ts);
        return OR_ERR_ARG;
    }
    if (nthreads < 1) nthreads = 1;
    int err = OR_OK;
    for (int64_t s = 0; s < N; ++s) {
        double r = 0.0;
        for (int i = 0; i < 9; ++i) r += f[i * N + s];
        rho[s] = r;
        const double Te = P->psi_uses_local_T ? T[s] : P->T_psi;
        psi2[s] = or_psi_sq(P, r, Te);
        psi[s] = 0.0;
        if (!isfinite(r) || !isfinite(T[s])) err = err < OR_ERR_NONFINITE ? OR_ERR_NONFINITE : err;
        if (P->beta != 0.0) {
            if (psi2[s] < 0.0) {
                err = OR_ERR_PSI_DOMAIN;
                psi[s] = NAN;
            } else {
                psi[s] = sqrt(psi2[s]);
            }
        }
    }
    const double uin = Ch->U_in;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            const int64_t s = (int64_t)y * nx + x;
            double fl[9], gl[9], fs[9], gs[9], Fx, Fy;
            for (int i = 0; i < 9; ++i) {
                fl[i] = f[i * N + s];
                gl[i] = 0.0;
            }
            force_at_clamped(P, psi, psi2, x, y, &Fx, &Fy);
            collide_site(P, fl, gl, rho[s], T[s], Fx, Fy, fs, gs, &ux[s], &uy[s]);
            for (int i = 0; i < 9; ++i) {
                const int xd = x + EX[i], yd = y + EY[i];
                const int o = OPP[i];
                if (yd < 0 || yd >= ny) {
                    fn[o * N + s] = fs[i];
                } else if (xd < 0) {
                    const double eu = EX[i] * uin;
                    fn[o * N + s] = fs[i] - 2.0 * OMEGA[i] * rho[s] * eu / CS2;
                } else if (xd < nx) {
                    fn[i * N + (int64_t)yd * nx + xd] = fs[i];
                } else {
                    const double eu = EX[i] * ux[s] + EY[i] * uy[s];
                    fn[o * N + s] = -fs[i] + 2.0 * OMEGA[i] * 1.0 *
                                                 (1.0 + 0.5 * eu * eu / (CS2 * CS2) -
                                                  0.5 * (ux[s] * ux[s] + uy[s] * uy[s]) / CS2);
                }
            }
        }
    }
    const double a = printed ? 0.5 : 1.0;
    fd_rhs_channel(P, Ch, T, rho, ux, uy, h1);
    for (int64_t s = 0; s < N; ++s) Ts[s] = T[s] + a * h1[s];
    fd_rhs_channel(P, Ch, Ts, rho, ux, uy, h2);
    for (int64_t s = 0; s < N; ++s) {
        Tn[s] = T[s] + 0.5 * (h1[s] + h2[s]);
        if (!isfinite(Tn[s])) err = err < OR_ERR_NONFINITE ? OR_ERR_NONFINITE : err;
    }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * N);
    if (ux_out) memcpy(ux_out, ux, sizeof(double) * N);
    if (uy_out) memcpy(uy_out, uy, sizeof(double) * N);
    free(rho); free(psi); free(psi2); free(ux); free(uy); free(h1); free(h2); free(Ts);
    return err;
}

/* Local Nusselt number of a temperature field whose plate value enters
 * through the reflected ghost (the FD treatment): q_w / lambda is the
 * central difference across the upper plate, 2 (T_w - T(ny - 1)).         */
double or_channel_nusselt_wall(const or_params* P, const or_channel* Ch, const double* rho,
                               const double* ux, const double* T, int x)
{
    const int nx = P->nx, ny = P->ny;
    double num = 0.0, den = 0.0;
    for (int y = 0; y < ny; ++y) {
        const int64_t s = (int64_t)y * nx + x;
        num += rho[s] * ux[s] * T[s];
        den += rho[s] * ux[s];
    }
    const double Tb = num / den;
    const double q = 2.0 * (Ch->T_w - T[(int64_t)(ny - 1) * nx + x]);
    return 2.0 * ny * q / (Ch->T_w - Tb);
}
