// lb_launch.h -- host-side launch interface between the C ABI and the
// per-precision kernel translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lb_device.cuh"
#include "lb_fd.cuh"

namespace lbgb {

struct StepLaunch {
    const void* src;
    void* dst;
    KParams kp;
    int eq24;       // 0: Eq. (7), 1: Eq. (24)
    int bmode;      // BetaMode
    int bx, by;     // CTA tile; by == 0: strip kernel of width bx
    int nchunks;    // strip kernel: row chunks per strip
    cudaStream_t stream;
    // 16-bit strip kernel: tensor map of dst (x: nx columns, y: ny rows,
    // z: the planes; box bx x 1 x NPLANES) that its collided rows are stored
    // through; nullptr elsewhere
    const CUtensorMap* dst_map = nullptr;
};

struct MomentsLaunch {
    const void* src;
    KParams kp;
    int bmode;
    double *rho, *ux, *uy, *T;          // may be null
    const double *ref_rho, *ref_T;      // may be null
    double* part;                       // may be null; [grid][8]
    cudaStream_t stream;
};

// One time step (or a moments evaluation) of the finite-difference
// temperature treatment, Eqs. (26)-(27).  Fields are dense [ny][nx] of the
// storage precision's arithmetic type (FP64 or FP32).
struct FdLaunch {
    const void* src;      // f, pre-collision at n
    void* dst;            // f, post-collision (step)
    const void* T;        // T^n
    void* T_next;         // T^{n+1} (step)
    void *rho, *ux, *uy;  // rho^n, u^n (step)
    double *m_rho, *m_ux, *m_uy, *m_T;  // moments outputs (any may be null)
    KParams kp;
    int bmode;
    double chi;           // (tau_g - 1/2) c_s^2
    double a;             // RK2 stage factor: 1 (Heun) or 1/2 (printed form)
    int strip;            // strip context: the step is k_fd_fused
    int nchunks;          // row chunks per strip (strip contexts)
    cudaStream_t stream;
};

cudaError_t launch_fd_partials(const double* rho, const double* ux, const double* uy, const double* T,
                               const double* ref_rho, const double* ref_T, long long n, double cv,
                               double* part, int blocks, cudaStream_t st);

// Tile used by the moments/totals kernel (one fixed shape: deterministic grid).
constexpr int MOM_BX = 32, MOM_BY = 8;

inline int moments_grid_blocks(int nx, int ny) {
    return ((nx + MOM_BX - 1) / MOM_BX) * ((ny + MOM_BY - 1) / MOM_BY);
}

// Supported step tiles (bx, by); every precision instantiates all of them.
// (bx, 0) selects the strip-marching kernel of width bx.
bool step_tile_supported(int bx, int by);

// Planes of a population buffer: 18, plus the low halves of the two rest
// populations in the 16-bit modes (see Store in lb_device.cuh).
inline int pop_planes(int prec) { return (prec == LB_PREC_FP64 || prec == LB_PREC_FP32) ? 18 : 20; }

// Column halo of the strip kernel (16 bytes of elements) and its eligibility:
// a supported width and 32-bit element offsets over all planes (any nx: the
// row copies are rounded up to whole 16-byte units).
inline int strip_halo(int prec) { return prec == LB_PREC_FP64 ? 2 : (prec == LB_PREC_FP32 ? 4 : 8); }
inline bool strip_eligible(int prec, int nx, long long plane, int bx) {
    (void)nx;
    if (prec == LB_PREC_FP64 && bx != 128) return false;
    if (bx != 128 && bx != 256) return false;
    return (long long)pop_planes(prec) * plane < (1LL << 32);
}

// Smallest nx of a finite-difference strip context: the FD_GHOST ghost
// columns on each side must be distinct columns of the row.
constexpr int FD_STRIP_MIN_NX = 8;

// Population buffer layout, in elements: pop_planes planes, rows padded to 128 bytes,
// planes to 256 bytes.  The strip layout also leaves 128 bytes on each side
// of every row for the periodic ghost columns (STRIP_GHOST of them are kept,
// FD_GHOST on finite-difference contexts; the rest is read as halo padding
// and never used); `origin` is the offset of column 0 of row 0 of plane 0
// from the start of the allocation.
struct PopLayout {
    long long pitch, plane, origin;
};
inline PopLayout pop_layout(int prec, int nx, int ny, bool strip) {
    const long long es = prec == LB_PREC_FP64 ? 8 : (prec == LB_PREC_FP32 ? 4 : 2);
    const long long gh = strip ? 128 / es : 0;
    PopLayout L;
    L.pitch = ((2 * gh + nx) * es + 127) / 128 * 128 / es;
    L.plane = (L.pitch * ny * es + 255) / 256 * 256 / es;
    L.origin = gh;
    return L;
}

#define LBGB_DECLARE_PREC(NAME)                                                       \
    cudaError_t launch_step_##NAME(const StepLaunch& L);                               \
    cudaError_t launch_moments_##NAME(const MomentsLaunch& L);                         \
    cudaError_t launch_init_##NAME(void* dst, const KParams& kp, const double* rho0,   \
                                   const double* T0, cudaStream_t st);                 \
    cudaError_t launch_gather_##NAME(const void* src, const KParams& kp, double* out,  \
                                     cudaStream_t st);                                 \
    cudaError_t launch_scatter_##NAME(void* dst, const KParams& kp, const double* in,  \
                                      cudaStream_t st);                                \
    cudaError_t launch_step_cavity_##NAME(const StepLaunch& L);                        \
    cudaError_t launch_step_channel_##NAME(const StepLaunch& L);                       \
    cudaError_t launch_fd_step_##NAME(const FdLaunch& L);                              \
    cudaError_t launch_fd_moments_##NAME(const FdLaunch& L);                           \
    cudaError_t launch_fd_set_T_##NAME(void* T, const double* T0, const KParams& kp, cudaStream_t st);

LBGB_DECLARE_PREC(fp64)
LBGB_DECLARE_PREC(fp32)
LBGB_DECLARE_PREC(fp16)
LBGB_DECLARE_PREC(bf16)

// Start at rest under the force (lb_init_balanced.cu): f = f^eq(rho0, -F/(2 rho0)),
// g = c_v T0 f^eq(rho0, -F/(2 rho0)), for storage precision prec (LB_PREC_*);
// periodic lattices only (cudaErrorInvalidValue for walls).
cudaError_t launch_init_balanced(int prec, void* dst, const KParams& kp, const double* rho0,
                                 const double* T0, cudaStream_t st);

}  // namespace lbgb
