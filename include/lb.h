/*
 * lb.h -- C ABI of the GB300 (sm_103a) fused thermal pseudopotential D2Q9
 * lattice Boltzmann step.
 *
 * Method: Li & Luo, "Effect of the forcing term in the pseudopotential
 * lattice Boltzmann modeling of thermal flows", arXiv:1405.2232.
 *   density LBE ............ Eq. (1), BGK with forcing term F_i (Ref. [21]:
 *                            Guo et al., u = (sum e_i f_i + F/2)/rho)
 *   pseudopotential force .. Eq. (2), mixed form Eq. (4) (parameter beta)
 *   pseudopotential ........ psi = sqrt(2 (p_EOS - rho cs^2)/(G c^2)), Sec. II A
 *   temperature LBE ........ Eq. (7), g^eq = c_v T f^eq   (forcing-term effect)
 *                            Eq. (24) with C_i of Eq. (25) (forcing-free)
 *   equations of state ..... van der Waals and ideal gas (Sec. III),
 *                            Carnahan-Starling
 *
 * Lattice: periodic nx-by-ny D2Q9, site index y*nx + x, c = 1, delta_t = 1,
 * cs^2 = 1/3.  Velocity numbering: e0 = (0,0); e1..e4 = (1,0),(0,1),(-1,0),
 * (0,-1); e5..e8 = (1,1),(-1,1),(-1,-1),(1,-1); weights 4/9, 1/9, 1/36.
 *
 * Host arrays passed to or returned from the library are float64, row-major
 * (y, x); population arrays are [9][ny][nx] and hold the PRE-collision
 * populations f_i(x, t) and g_i(x, t) at the context's current time t.
 *
 * Ownership: the library owns every device buffer of a context (allocated
 * in lb_init, released in lb_free).  Caller arrays are only read or written
 * during the call, except where a function says it is asynchronous.
 *
 * Errors: every function returns an lb_status.  On an argument error nothing
 * changes.  lb_last_error() returns a thread-local message about the last
 * failure.  Numerical trouble on the device (non-finite rho or T, psi^2 < 0
 * when beta != 0) sets a sticky per-context error word that the next
 * synchronising call (lb_synchronize, lb_moments, lb_totals, ...) reports and
 * clears.  Kernels never trap or spin: a bad state is reported, not fatal.
 */
#ifndef LBGB_LB_H
#define LBGB_LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lb_status {
    LB_OK = 0,
    LB_ERR_ARG = 1,         /* invalid argument; nothing was changed            */
    LB_ERR_CUDA = 2,        /* a CUDA runtime call failed                       */
    LB_ERR_OOM = 3,         /* device allocation failed                         */
    LB_ERR_NONFINITE = 4,   /* rho or T became NaN/Inf during a step            */
    LB_ERR_PSI_DOMAIN = 5,  /* 2 (p_EOS - rho cs^2)/G < 0 with beta != 0        */
    LB_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                    */
    LB_ERR_UNSUPPORTED = 7, /* option not built or not available                */
    LB_ERR_NOT_CONVERGED = 8 /* batch domain did not reach the tolerance        */
} lb_status;

/* Equation of state p_EOS(rho, T) used by the pseudopotential (Sec. II A). */
enum {
    LB_EOS_CS = 0,    /* rho R T (1+eta+eta^2-eta^3)/(1-eta)^3 - a rho^2, eta = b rho/4 */
    LB_EOS_VDW = 1,   /* rho R T/(1 - b rho) - a rho^2                      (Sec. III) */
    LB_EOS_IDEAL = 2  /* rho R T                                            (Sec. III) */
};

/* Temperature treatment (Sec. II B). */
enum {
    LB_THERMAL_EQ7 = 0,  /* Eq. (7): g relaxes to c_v T f^eq; recovers Eq. (23)       */
    LB_THERMAL_EQ24 = 1, /* Eq. (24): Eq. (7) + C_i of Eq. (25); recovers Eq. (6)/(A11) */
    /* Eqs. (26)-(27): no g populations; T is a field advanced by a second-order
     * Runge-Kutta step of dT/dt = -u.grad T + (1/(rho c_v)) div(lambda grad T)
     * with lambda = rho c_v (tau_g - 1/2) c_s^2 (the diffusivity of the thermal
     * LBE), the isotropic central D2Q9 stencils for grad and the Laplacian,
     * and rho, u (with F/2) of the density LBE at time n in both stages.
     * FD26: Heun, h2 = K(T^n + dt h1); FD26_PRINTED: h2 = K(T^n + dt/2 h1) as
     * printed with Eq. (27).  Storage FP64 or FP32 only (else
     * LB_ERR_UNSUPPORTED).  Kernels: the whole step in one strip pass
     * (tile (256, 0) in FP32, (128, 0) in FP64; nx >= 8; the FP32 default
     * where the strip rules hold), or the 32x8 tile front followed by one
     * launch of both RK2 stages (any other tile_y != 0 request runs 32x8;
     * the FP64 default); another strip width is LB_ERR_ARG.  Not available
     * in the batched solver; lb_get/set_populations and the state calls
     * return LB_ERR_UNSUPPORTED (there is no g). */
    LB_THERMAL_FD26 = 2,
    LB_THERMAL_FD26_PRINTED = 3
};

/* Storage of the populations in device memory; collision arithmetic is FP64
 * for LB_PREC_FP64 and FP32 otherwise.  The 16-bit modes store the deviation
 * h = f - w_i rho0 (and g - w_i rho0 c_v T0) of the eight moving populations
 * rounded to nearest even, and keep the rest populations f_0, g_0 as FP32
 * deviations (two 16-bit halves, 40 bytes per site and distribution set):
 * after each collision the rest population takes the deviation that keeps the
 * site's stored mass (energy) equal to the mass (energy) it loaded, so the
 * 16-bit modes conserve mass and energy to one FP32 rounding per site and
 * step (Eq. (13); sum C_i = 0 after Eq. (25)), where rounding each moving
 * population on its own changes them coherently. */
enum {
    LB_PREC_FP64 = 0,
    LB_PREC_FP32 = 1,
    LB_PREC_FP16_DEV = 2,
    LB_PREC_BF16_DEV = 3
};

/* Boundaries (Sec. III B).  PERIODIC: the periodic lattice.  CAVITY: the
 * natural-convection cavity: nx-by-ny fluid nodes inside walls half a
 * lattice spacing outside the outermost nodes (side-wall distance L = nx);
 * f bounces back on every wall (no slip); g bounces back on the adiabatic
 * bottom and top walls and anti-bounces back on the side walls, which hold
 * T_hot (left) and T_cold (right): g_{-i}(x, t+1) = -g*_i(x, t) + 2 w_i
 * rho(x, t) c_v T_w (a link that leaves through a corner takes the side-wall
 * rule); psi at a wall node is that of the nearest fluid node; the buoyancy
 * (0, -rho g_grav) is added to the force.  The populations are then stored
 * pre-collision at their site and pushed after the collision.  Cavity
 * contexts: FP64 or FP32, the 32x8 tile kernel (tile_y == 0 is LB_ERR_ARG),
 * not in the batched solver; the finite-difference treatment as below. */
/* CHANNEL (Sec. III A): flow between parallel plates half a spacing below
 * y = 0 and above y = ny - 1 (gap H = ny); f bounces back on the plates; g
 * anti-bounces back at T_w on the upper plate and, in Case A, on the lower
 * one (Case B: lower plate adiabatic, g bounces back); the inlet (half a
 * spacing left of x = 0) bounces f back with the wall velocity (U_in, 0),
 * f_{-i} = f*_i - 2 w_i rho (e_i.u_in)/cs^2, and g anti-bounces back at T_in
 * with the symmetric equilibrium at u_in; the outlet (half a spacing right of
 * x = nx - 1) anti-bounces f back at density 1 with the node's velocity, and
 * copies g from column nx - 2 (zero gradient); psi outside = psi of the
 * nearest node; no gravity.  FP64 or FP32, the 32x8 tile kernel, not in the
 * batched solver.  With the finite-difference treatment (cavity and channel)
 * K of Eq. (26) reads ghosts outside: the temperature reflected about the
 * boundary value (2 T_b - T of the mirror node) across an isothermal
 * boundary, the mirror node's across an adiabatic one or the outlet; rho
 * mirrored. */
enum { LB_WALLS_PERIODIC = 0, LB_WALLS_CAVITY = 1, LB_WALLS_CHANNEL = 2 };

/* Numbers of lb_totals outputs. */
enum { LB_TOTALS_N = 5 };
enum { LB_TUNE_N = 5 };        /* step shapes lb_autotune tries        */
enum { LB_BATCH_TUNE_N = 4 };  /* row-chunk heights lb_batch_autotune tries */

typedef struct lb_params {
    int32_t nx, ny;        /* lattice size, both >= 3                                  */
    int32_t eos;           /* LB_EOS_*                                                 */
    int32_t thermal;       /* LB_THERMAL_*                                             */
    int32_t precision;     /* LB_PREC_*                                                */
    int32_t psi_uses_local_T; /* 1: psi(rho, T(x,t)); 0: psi(rho, T_psi) (T passive)   */
    int32_t tile_x, tile_y;   /* CTA tile of the step kernel; 0 = library default      */
    double tau_f;          /* relaxation time of Eq. (1), > 1/2                        */
    double tau_g;          /* relaxation time of Eq. (7)/(24), > 1/2                   */
    double G;              /* interaction strength of Eq. (2)/(4), != 0                */
    double beta;           /* mixing parameter of Eq. (4); 1 gives Eq. (2)             */
    double a, b, R;        /* EOS constants                                            */
    double cv;             /* specific heat at constant volume (g^eq = c_v T f^eq), > 0 */
    double T_psi;          /* temperature used by psi when psi_uses_local_T == 0       */
    double rho0, T0;       /* deviation base of the 16-bit storage modes               */
    int32_t walls;         /* LB_WALLS_PERIODIC, LB_WALLS_CAVITY or LB_WALLS_CHANNEL   */
    int32_t adiabatic_bottom; /* channel: 0 Case A (both plates at T_w), 1 Case B      */
    double T_hot, T_cold;  /* cavity: left (x = -1/2) and right (x = nx - 1/2) walls   */
    double g_grav;         /* cavity: gravity along -y, buoyancy (0, -rho g) added to F */
    double T_in, T_w, U_in; /* channel: inlet temperature and velocity, plate temperature */
    int32_t init_balanced; /* initial state: 0 at u = 0 in f^eq; 1 at rest under the force (lb_init) */
    int32_t halo_rows;     /* 0: periodic lattice; LB_HALO_ROWS: one y-slab of a decomposed lattice */
} lb_params;

/* Ghost rows per side of a y-slab of a lattice decomposed across ranks.  One
 * fused step at row y reads the post-collision populations of rows y - 2 ..
 * y + 2 (the pull reaches one row, the psi of the force stencil one more), so
 * a slab that owns rows [y0, y1) of the global lattice is a context of
 * ny = (y1 - y0) + 2 LB_HALO_ROWS rows holding global rows
 * [y0 - LB_HALO_ROWS, y1 + LB_HALO_ROWS) (periodic in the global lattice).
 * Its steps update only the owned rows [LB_HALO_ROWS, ny - LB_HALO_ROWS);
 * between steps the caller refreshes the ghost rows from the neighbouring
 * slabs (lb_halo_pack / lb_halo_unpack), after which the owned rows evolve bit
 * for bit as the same rows of the whole lattice.  Periodic in x; lattice
 * Boltzmann treatments (Eq. 7, Eq. 24) only; lb_moments, lb_totals and
 * lb_get_populations cover all ny rows, of which only the owned ones are
 * meaningful. */
enum { LB_HALO_ROWS = 2 };

typedef struct lb_ctx lb_ctx; /* opaque; owned by the library */

/* Fill *p with the defaults: 64x64, CS EOS a=1 b=4 R=1, G=-1, beta=1,
 * tau_f=1, tau_g=0.8, c_v=1, Eq. (24), FP32, psi from the local T,
 * rho0 = 0.12, T0 = 0.075, periodic (cavity fields T_hot = 1.03,
 * T_cold = 0.97, g_grav = 0; channel fields T_in = 1.03, T_w = 0.97,
 * U_in = 0.05, Case A), init_balanced = 0, halo_rows = 0. */
void lb_params_default(lb_params* p);

/* Create a context whose initial state is f = f^eq(rho0, u = 0) and
 * g = c_v T0 f^eq(rho0, 0) (Eq. (1) and Eq. (7) equilibria at rest).
 * With p->init_balanced = 1 the state is instead at rest under the force:
 * with the forcing of Eq. (1) the velocity is u = (sum e_i f_i + F/2)/rho,
 * so f = f^eq(rho0, v) and g = c_v T0 f^eq(rho0, v) with v = -F/(2 rho0),
 * F the Eq. (2)/(4) force of psi(rho0, T0) (T_psi when psi does not follow
 * the local T); evaluated in FP64, rounded once to the storage precision.
 * The plain start moves every interface with F/(2 rho) on its first step;
 * this one does not (fields near a steady state restart without that
 * impulse).  Periodic lattice Boltzmann contexts only: walls or the
 * finite-difference treatment give LB_ERR_UNSUPPORTED; psi^2 < 0 with
 * beta != 0 is reported as LB_ERR_PSI_DOMAIN by the next lb_synchronize.
 * rho0, T0: host float64 arrays [ny][nx], copied during the call.
 * stream: a cudaStream_t for all work of the context, or NULL for a stream
 * the library creates.  *out receives the context.  Returns LB_ERR_ARG for
 * invalid parameters (tau <= 1/2, n < 3, G == 0, c_v <= 0, unknown enum). */
lb_status lb_init(const lb_params* p, const double* rho0, const double* T0,
                  void* stream, lb_ctx** out);

/* As lb_init, but rho0 and T0 are DEVICE float64 arrays [ny][nx]; they are
 * read by kernels on the stream before the call returns.  They must be
 * complete when the call is made: work that writes them on another stream
 * is synchronised by the caller first. */
lb_status lb_init_device(const lb_params* p, const double* d_rho0, const double* d_T0,
                         void* stream, lb_ctx** out);

/* Advance n >= 0 time steps (Eq. (1) for f; Eq. (7) or (24) for g), each one
 * fused kernel launch that reads and writes every population once.
 * Asynchronous on the context's stream. */
lb_status lb_step(lb_ctx* ctx, int64_t n);

/* Wait for the context's stream and report (then clear) the device error word. */
lb_status lb_synchronize(lb_ctx* ctx);

/* Macroscopic fields of the state at time t, as the step computes them:
 * rho = sum f_i, u = (sum e_i f_i + F/2)/rho, T = sum g_i/(rho c_v).
 * Host float64 arrays [ny][nx]; any pointer may be NULL.  Synchronises. */
lb_status lb_moments(lb_ctx* ctx, double* rho, double* ux, double* uy, double* T);

/* Same, into DEVICE float64 arrays [ny][nx]; asynchronous on the stream. */
lb_status lb_moments_device(lb_ctx* ctx, double* d_rho, double* d_ux, double* d_uy,
                            double* d_T);

/* Copy the pre-collision populations at time t to host arrays [9][ny][nx]
 * (any may be NULL).  Synchronises. */
lb_status lb_get_populations(lb_ctx* ctx, double* f, double* g);

/* Replace the state by host populations [9][ny][nx] (pre-collision, time t);
 * values are rounded to the storage precision. */
lb_status lb_set_populations(lb_ctx* ctx, const double* f, const double* g);

/* Global FP64 totals of the state at time t, reduced on the device in a
 * fixed order (deterministic):
 *   out[0] mass   sum_x sum_i f_i
 *   out[1] energy sum_x sum_i g_i  (= sum rho c_v T)
 *   out[2] px     sum_x rho u_x    (with the F/2 term)
 *   out[3] py     sum_x rho u_y
 *   out[4] residual: max over phi in {rho, T} of
 *          ||phi_t - phi_s||_2 / ((t - s) ||phi_t||_2), where s is the time of
 *          the previous lb_totals call (0 on the first call or when t == s).
 * Each call stores (rho, T) at t as the new reference.  Synchronises. */
lb_status lb_totals(lb_ctx* ctx, double out[LB_TOTALS_N]);

/* Raw state for checkpoint/resume: *bytes receives the size of the opaque
 * state blob; lb_save_state copies it to host memory, lb_load_state restores
 * it bit for bit (same params required).  Both synchronise. */
lb_status lb_state_size(const lb_ctx* ctx, size_t* bytes);
lb_status lb_save_state(lb_ctx* ctx, void* host_blob);
lb_status lb_load_state(lb_ctx* ctx, const void* host_blob);

/* Number of steps taken since lb_init (or the loaded state's time). */
int64_t lb_time(const lb_ctx* ctx);

/* Ghost-row exchange of a y-slab context (halo_rows == LB_HALO_ROWS).
 * lb_halo_bytes: size of one face's exchange buffer: every population plane
 * (18; 20 in the 16-bit modes) x LB_HALO_ROWS whole rows of the context's
 * padded row pitch, in the storage type (ghost columns included).
 * lb_halo_pack(face): copy the first (face 0) or last (face 1) LB_HALO_ROWS
 * owned rows of the current state into the DEVICE buffer d_buf, dense
 * [planes][LB_HALO_ROWS][pitch]; face 0 goes to the neighbour below (it
 * becomes that slab's upper ghost rows), face 1 to the neighbour above.
 * lb_halo_unpack(face): write such a buffer into the lower (face 0) or upper
 * (face 1) ghost rows.  Both are asynchronous on the context's stream and
 * allocate nothing; the buffers must not be touched by other streams until
 * the copies are done.  The owned rows of a slab at time t are exact only if
 * its ghost rows hold the neighbours' rows at time t: exchange after every
 * step.  LB_ERR_ARG for a context without ghost rows, a NULL buffer or a face
 * other than 0 or 1.  (Row decomposition of one lattice over GPUs; the paper
 * has no counterpart.) */
lb_status lb_halo_bytes(const lb_ctx* ctx, size_t* bytes);
lb_status lb_halo_pack(lb_ctx* ctx, int32_t face, void* d_buf);
lb_status lb_halo_unpack(lb_ctx* ctx, int32_t face, const void* d_buf);

/* Failure detection (the paper has no counterpart).  The strip-marching step
 * kernels (lattice Boltzmann and finite-difference) hand rows from a copy
 * warp to the compute warps through mbarriers, and every such wait is
 * bounded: after `cycles` SM clock cycles (0: the default, 2e9, about one
 * second at GB300 clocks) the CTA stops, records LB_ERR_TIMEOUT in the
 * context's error word and leaves once the copies it issued have landed (that
 * last wait always takes the default limit).  The next synchronising call
 * reports LB_ERR_TIMEOUT; the state of the step that timed out is undefined
 * (restore it with lb_load_state or lb_set_populations), the context and the
 * device stay usable.  A tiny limit makes the wait give up on purpose (tests
 * of the error path).  Applies to steps launched after the call; the tile
 * kernels and the batched solver do not wait and ignore it.  LB_ERR_ARG for
 * cycles < 0. */
lb_status lb_set_wait_limit(lb_ctx* ctx, int64_t cycles);

/* Parameters the context runs with (tile sizes resolved). */
lb_status lb_get_params(const lb_ctx* ctx, lb_params* out);

/* Release the context and its device memory.  NULL is accepted. */
lb_status lb_free(lb_ctx* ctx);

/* ---------------------------------------------------------------- autotune
 * The fused step (Eqs. 1, 2/4, 7 or 24-25) runs as one of LB_TUNE_N shapes:
 * k = 0, 1: the strip-marching kernel, 256 or 128 columns wide (tile_y == 0;
 * any nx; FP64: 128 only); k = 2..4: the tile
 * kernel with tiles 32x8, 32x16, 64x4.  Results do not depend on the shape
 * (FP64 storage: bit for bit), only the time does.
 *
 * lb_tune_candidate: the (tile_x, tile_y) of shape k.  LB_ERR_ARG if k is out
 * of range.
 * lb_autotune: time every shape valid for *p (its lattice, precision,
 * treatment and force form; p's own tile fields are ignored) over `steps`
 * fused steps after 2 warm-up steps, on a uniform state (rho0, T0 of *p),
 * with CUDA events on `stream` (NULL: a stream of its own).  *best = *p with
 * the fastest tile_x, tile_y; ms_per_step[k] (may be NULL) = each shape's
 * time per step in ms, NaN for shapes not valid here.  Allocates and frees
 * one trial context at a time (two population buffers of the lattice);
 * synchronises.  LB_ERR_ARG for NULL params/best or steps < 1. */
lb_status lb_tune_candidate(int32_t k, int32_t* tile_x, int32_t* tile_y);
lb_status lb_autotune(const lb_params* p, int32_t steps, void* stream, lb_params* best,
                      double ms_per_step[LB_TUNE_N]);

/* ------------------------------------------------------------------ batch
 * Many independent periodic domains (a parameter sweep) advanced together by
 * one persistent fused-step kernel over a device work list of (domain, strip,
 * row chunk) items.  All domains share the storage precision (FP32 or FP64),
 * the temperature treatment and the force form (beta == 0, beta == 1 or
 * mixed); size, tau_f, tau_g, G, beta, EOS and its constants and c_v are per
 * domain; any nx, ny >= 3. */
typedef struct lb_batch lb_batch; /* opaque; owned by the library */

/* Create a batch of n domains; params[d] describes domain d, rho0[d] and T0[d]
 * are its float64 fields [ny][nx], in host or device memory (copied on the
 * batch's stream before the call returns; the copy direction follows from
 * unified addressing; device fields must be complete when the call is made).
 * Initial state as lb_init (params[d].init_balanced chooses it per domain). */
lb_status lb_batch_init(const lb_params* params, int32_t n, const double* const* rho0,
                        const double* const* T0, void* stream, lb_batch** out);

/* Advance every active domain n steps (asynchronous). */
lb_status lb_batch_step(lb_batch* b, int64_t n);

/* Per-domain FP64 check of the active domains (deterministic reduction):
 * residual[d] = max over phi in {rho, T} of ||phi_t - phi_s||_2 / ((t - s) ||phi_t||_2)
 * with s the time of the previous check (0 on the first), mass[d] = sum f,
 * energy[d] = sum g, status[d] = the domain's sticky device error (LB_OK,
 * LB_ERR_PSI_DOMAIN, LB_ERR_NONFINITE, ...).  Any output may be NULL; retired
 * domains report 0.  The check becomes the new reference.  Synchronises. */
lb_status lb_batch_check(lb_batch* b, double* residual, double* mass, double* energy,
                         int32_t* status);

/* Run to steady state: replay a CUDA graph of K fused steps (K even) plus a
 * check until every domain has residual < tol, has failed, or max_steps have
 * passed.  A domain that converges or fails is taken off the work list (its
 * state is kept).  steps_out[d]: steps the domain took; residual_out[d]: its
 * last residual; status_out[d]: LB_OK (converged), LB_ERR_PSI_DOMAIN /
 * LB_ERR_NONFINITE (failed) or LB_ERR_NOT_CONVERGED.  Any output may be NULL.
 * Synchronises. */
lb_status lb_batch_run(lb_batch* b, double tol, int64_t K, int64_t max_steps, int64_t* steps_out,
                       double* residual_out, int32_t* status_out);

/* Host float64 rho and T [ny][nx] of domain d (either may be NULL).  For an
 * active domain this runs a check (the new residual reference).  Synchronises. */
lb_status lb_batch_fields(lb_batch* b, int32_t d, double* rho, double* T);

/* Restart domain d from the float64 fields rho0, T0 [ny][nx] (host or device,
 * copied on the batch's stream before the call returns): its state becomes the
 * initial state of lb_batch_init (init_balanced 0: f^eq at u = 0; 1: at rest
 * under the force), its error word and status are cleared and it is active
 * again (taken back onto the work list if it had converged or failed).  Its
 * step count keeps counting from where it was, so a later lb_batch_run's step
 * cap bounds the domain's steps over both starts; its next residual compares
 * with the fields it restarted from.  This is the fallback of a warm-started
 * solve: a domain whose prediction does not relax restarts from the plain
 * initial fields.  Synchronises.  LB_ERR_ARG for an invalid domain or NULL
 * field. */
lb_status lb_batch_restart(lb_batch* b, int32_t d, const double* rho0, const double* T0,
                           int32_t init_balanced);

/* Steps the batch has taken since lb_batch_init. */
int64_t lb_batch_time(const lb_batch* b);

/* Release the batch.  NULL is accepted. */
lb_status lb_batch_free(lb_batch* b);

/* Work-list granularity: every domain strip is cut into row chunks of about
 * `rows` rows (>= 16; default 64); smaller chunks balance uneven domains over
 * the persistent CTAs, larger ones re-read fewer halo rows.
 * lb_batch_set_chunk_rows rebuilds the lists (synchronises); LB_ERR_ARG for
 * rows < 16.  lb_batch_chunk_rows returns the current height (-1 for NULL).
 * lb_batch_autotune times `steps` batched steps (after 2 warm-up steps) for
 * each of the LB_BATCH_TUNE_N heights 16, 32, 64, 128, keeps the fastest and
 * writes it to *chunk_rows (may be NULL); ms_per_step[k] (may be NULL) gets
 * each height's time per step.  The batch state, its time and its error
 * words are restored afterwards, bit for bit (one temporary device copy of
 * the state is allocated and freed).  Synchronises. */
lb_status lb_batch_set_chunk_rows(lb_batch* b, int32_t rows);
int32_t lb_batch_chunk_rows(const lb_batch* b);
lb_status lb_batch_autotune(lb_batch* b, int32_t steps, int32_t* chunk_rows,
                            double ms_per_step[LB_BATCH_TUNE_N]);

/* Allocation-free FP64 totals of caller-owned device fields.
 *
 * The paper has no counterpart: this is a service for callers that must not
 * have device memory allocated on their behalf -- code running while a stream
 * is captured in a mode that forbids allocation, applications that give all
 * device memory to their own pool, or embedders that fix their memory budget
 * before the run.  lb_totals needs a context, whose buffers lb_init allocates;
 * this entry point allocates nothing (no cudaMalloc, no cudaFree, no allocating
 * library call).  Its scratch is one static device array of 4096 x 8 doubles
 * (256 KB), held by every GPU that loads the library until the process exits.
 *
 * Inputs: d_rho, d_ux, d_uy, d_T -- device float64 [ny][nx] fields (as written
 * by lb_moments_device); d_ref_rho, d_ref_T -- optional device reference fields
 * taken K steps earlier (both NULL: residual 0).  cv: the c_v of the run.
 * Output: d_out -- device float64[LB_TOTALS_N]: sum rho, sum rho c_v T,
 * sum rho u_x, sum rho u_y, residual (same definitions as lb_totals), reduced
 * in a fixed order.  Asynchronous on `stream` (NULL: the default stream).
 *
 * Limits and errors: nx*ny <= 16,777,216 sites (4096^2), else LB_ERR_ARG with
 * a message.  The first call on a device looks up the scratch address (make it
 * before any stream capture) and caches it for the life of the process, which
 * assumes the device is not reset (cudaDeviceReset) meanwhile.  Every call
 * shares the scratch; each call writes all entries it reads, so nothing needs
 * clearing, but calls that overlap on the GPU race on it.  The work runs on the
 * stream's device (the current device for a NULL stream); the calling thread's
 * current device is left as it was. */
lb_status lb_field_totals_noalloc(int32_t nx, int32_t ny, double cv, const double* d_rho,
                                  const double* d_ux, const double* d_uy, const double* d_T,
                                  const double* d_ref_rho, const double* d_ref_T, int64_t K,
                                  double* d_out, void* stream);

/* Thread-local description of the last error ("" if none). */
const char* lb_last_error(void);

/* Library version string. */
const char* lb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBGB_LB_H */
