// lb_device.cuh -- device code of the fused thermal pseudopotential D2Q9 step.
//
// Method (Li & Luo, arXiv:1405.2232):
//   f: Eq. (1) BGK + forcing term F_i (Ref. [21], Guo et al.)
//   F: Eq. (2) / mixed Eq. (4), 8-neighbour pseudopotential stencil
//   psi: sqrt(2 (p_EOS - rho cs^2) / G), Sec. II A
//   g: Eq. (7) (g^eq = c_v T f^eq) or Eq. (24) with C_i of Eq. (25)
//
// Storage: structure-of-arrays planes (f_0..f_8, g_0..g_8; the 16-bit modes
// add the low halves of f_0 and g_0, see Store), plane stride `plane`
// elements, row pitch `pitch` elements.  The buffer holds the
// post-collision populations of the previous step at their source site, so
// the pre-collision value f_i(x, t) is read ("pulled") from x - e_i.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lb.h"

namespace lbgb {

// ---------------------------------------------------------------- lattice
__host__ __device__ constexpr int ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
// weights as exact-literal quotients (4/9, 1/9, 1/36)
__host__ __device__ constexpr double wd(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// ---------------------------------------------------------------- storage
// Store<PREC>: element type, arithmetic type and encoding of one storage mode.
// NPLANES planes per buffer.  FP64 / FP32: 18 planes, f_0..f_8 then g_0..g_8.
// 16-bit deviation modes: the eight moving populations of f and of g are
// stored as 16-bit deviations h = f - base (RN-even), while the rest
// populations f_0 and g_0, which carry each site's mass and energy balance,
// are kept as FP32 deviations split into two 16-bit halves: the high half in
// plane 0 (f_0) / 9 (g_0), the low half in plane 18 (f_0) / 19 (g_0), so that
// every plane row has the same element size and alignment.
template <int PREC> struct Store;

template <> struct Store<LB_PREC_FP64> {
    using elem = double;
    using real = double;
    static constexpr int NPLANES = 18;
    static constexpr bool SPLIT = false;
    static __device__ __forceinline__ real load(const elem* p, real) { return *p; }
    static __device__ __forceinline__ void put(elem* p, real v, real) { *p = v; }
};
template <> struct Store<LB_PREC_FP32> {
    using elem = float;
    using real = float;
    static constexpr int NPLANES = 18;
    static constexpr bool SPLIT = false;
    static __device__ __forceinline__ real load(const elem* p, real) { return *p; }
    static __device__ __forceinline__ void put(elem* p, real v, real) { *p = v; }
};
// 16-bit deviation storage: h = f - base, decoded in FP32
template <> struct Store<LB_PREC_FP16_DEV> {
    using elem = __half;
    using real = float;
    static constexpr int NPLANES = 20;
    static constexpr bool SPLIT = true;
    static __device__ __forceinline__ real dec(elem h) { return __half2float(h); }
    // acc + dec(h) in one mixed-precision add (the widening is exact, so this
    // rounds once, as the separate decode and FP32 add do)
    static __device__ __forceinline__ real add_dec(elem h, real acc) {
        asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(acc) : "h"(__half_as_ushort(h)));
        return acc;
    }
    static __device__ __forceinline__ elem enc(real d) { return __float2half_rn(d); }
    static __device__ __forceinline__ unsigned short bits(elem h) { return __half_as_ushort(h); }
    static __device__ __forceinline__ elem from_bits(unsigned short b) { return __ushort_as_half(b); }
    static __device__ __forceinline__ real load(const elem* p, real base) { return base + dec(*p); }
    static __device__ __forceinline__ void put(elem* p, real v, real base) { *p = enc(v - base); }
};
template <> struct Store<LB_PREC_BF16_DEV> {
    using elem = __nv_bfloat16;
    using real = float;
    static constexpr int NPLANES = 20;
    static constexpr bool SPLIT = true;
    static __device__ __forceinline__ real dec(elem h) { return __bfloat162float(h); }
    static __device__ __forceinline__ real add_dec(elem h, real acc) {
        asm("add.rn.f32.bf16 %0, %1, %0;" : "+f"(acc) : "h"(__bfloat16_as_ushort(h)));
        return acc;
    }
    static __device__ __forceinline__ elem enc(real d) { return __float2bfloat16_rn(d); }
    static __device__ __forceinline__ unsigned short bits(elem h) { return __bfloat16_as_ushort(h); }
    static __device__ __forceinline__ elem from_bits(unsigned short b) { return __ushort_as_bfloat16(b); }
    static __device__ __forceinline__ real load(const elem* p, real base) { return base + dec(*p); }
    static __device__ __forceinline__ void put(elem* p, real v, real base) { *p = enc(v - base); }
};

// Planes apart from the high half of a rest population (plane 0 or 9) to its
// low half (plane 18 or 19) in the 16-bit modes.
__host__ __device__ constexpr int rest_lo_offset(int p) { return p == 0 ? 18 : 10; }
__host__ __device__ constexpr bool is_rest_plane(int p) { return p == 0 || p == 9; }

// Deviation of a population: the 16-bit value, or for a rest population of
// a 16-bit mode the FP32 value whose halves sit `lo_off` elements apart.
template <class S>
__device__ __forceinline__ typename S::real dev_of(const typename S::elem* p, int plane_idx, long long lo_off) {
    if constexpr (S::SPLIT) {
        if (is_rest_plane(plane_idx))
            return __uint_as_float(((unsigned)S::bits(p[0]) << 16) | (unsigned)S::bits(p[lo_off]));
        return S::dec(*p);
    } else {
        return *p;
    }
}

// acc + dev_of(p, ...) for a 16-bit mode (the moving populations through the
// mixed-precision add).
template <class S>
__device__ __forceinline__ float acc_dev(const typename S::elem* p, int plane_idx, long long lo_off, float acc) {
    static_assert(S::SPLIT, "deviation storage only");
    if (is_rest_plane(plane_idx))
        return acc + __uint_as_float(((unsigned)S::bits(p[0]) << 16) | (unsigned)S::bits(p[lo_off]));
    return S::add_dec(*p, acc);
}

// Population of plane plane_idx (0..17) at p; `stride` is the distance
// between planes of the container (kp.plane in device memory, the row
// segment width in a shared-memory stage).
template <class S>
__device__ __forceinline__ typename S::real load_pop(const typename S::elem* p, long long stride, int plane_idx,
                                                     typename S::real base) {
    if constexpr (S::SPLIT) {
        if (is_rest_plane(plane_idx)) return base + dev_of<S>(p, plane_idx, rest_lo_offset(plane_idx) * stride);
    }
    return S::load(p, base);
}

// Same, also adding the stored deviation to H (16-bit modes: the exact
// deviation sums of mass and energy that the collision closes on).
template <class S>
__device__ __forceinline__ typename S::real load_pop_acc(const typename S::elem* p, long long stride,
                                                         int plane_idx, typename S::real base,
                                                         typename S::real& H) {
    if constexpr (S::SPLIT) {
        const typename S::real d = dev_of<S>(p, plane_idx, rest_lo_offset(plane_idx) * stride);
        H += d;
        return base + d;
    } else {
        return S::load(p, base);
    }
}

// Write one population value v (absolute) of plane plane_idx at p.
template <class S>
__device__ __forceinline__ void put_pop(typename S::elem* p, long long stride, int plane_idx,
                                        typename S::real v, typename S::real base) {
    if constexpr (S::SPLIT) {
        if (is_rest_plane(plane_idx)) {
            const unsigned b = __float_as_uint(v - base);
            p[0] = S::from_bits((unsigned short)(b >> 16));
            p[rest_lo_offset(plane_idx) * stride] = S::from_bits((unsigned short)(b & 0xffffu));
            return;
        }
    }
    S::put(p, v, base);
}

// ---------------------------------------------------------------- params
// Kernel parameters, derived once on the host from lb_params.
struct KParams {
    int nx, ny;
    long long pitch;   // elements per row
    long long plane;   // elements per plane
    double omega_f;    // 1/tau_f
    double omega_g;    // 1/tau_g
    double guo_pre;    // 1 - 1/(2 tau_f)
    double corr_pre;   // 1 - 1/(2 tau_g)
    double G;
    double two_over_G;
    double beta;
    double half_1mbeta;  // (1 - beta)/2
    int eos;
    int psi_local_T;
    int ghost;         // periodic ghost columns kept on each side of every row (0 or 2)
    int walls;         // 0 periodic; 1 cavity, 2 channel (populations stored pre-collision at their site)
    int adiabatic_bottom;          // channel Case B
    double T_hot, T_cold, g_grav;  // cavity side walls and gravity
    double T_in, T_w, U_in;        // channel inlet and plates
    double a, b, R;
    double cv, inv_cv;
    double T_psi;
    float base_f[9], base_g[9];  // deviation bases of the 16-bit modes
    int* err;                    // sticky device error word (bit per lb_status)
    long long wait_cycles;       // limit of the strip kernels' pipeline waits (<= 0: default)
    int halo_rows;               // 0: periodic in y; H > 0: rows [0, H) and [ny - H, ny) are ghost
                                 // rows of a y-decomposed lattice, the step updates [H, ny - H)
    // 16-bit modes, collision in deviation variables (collide_dev):
    float sum_bf, sum_bg;        // sum_i base_f[i], sum_i base_g[i]
    float dsum_f, dsum_g;        // sum_i base_f[i] - rho0, sum_i base_g[i] - rho0 c_v T0
    float cw_f[3], cw_g[3];      // w rho0 - base_f, w rho0 c_v T0 - base_g (rest, axis, diagonal)
    // the doubles above rounded to float once on the host (kp_fill_float):
    // the 16-bit kernels read these (KPR, collide_dev), since converting a
    // double at each use runs on the FP64 pipe, which is narrow on this GPU
    struct {
        float omega_f, omega_g, guo_pre, corr_pre, G, two_over_G, beta, half_1mbeta;
        float T_hot, T_cold, g_grav, T_in, T_w, U_in, a, b, R, cv, inv_cv, T_psi;
    } f;
    // factors of the deviation-variable collision (collide_dev) in FMA form,
    // per weight class ([0] axis w = 1/9, [1] diagonal w = 1/36)
    struct {
        float omc_f, omc_g;        // 1 - omega_f, 1 - omega_g
        float wo_f[2], wo_g[2];    // omega_f w, omega_g w
        float ocw_f[2], ocw_g[2];  // omega_f cw_f, omega_g cw_g
        float gw[2], gw9[2], gw3[2];  // guo w, 9 guo w, 3 guo w
        float cw3[2];              // 3 corr w
    } d;
};

// Set KParams::f from the double fields (call after they are final).
inline void kp_fill_float(KParams& k) {
    k.f.omega_f = (float)k.omega_f;
    k.f.omega_g = (float)k.omega_g;
    k.f.guo_pre = (float)k.guo_pre;
    k.f.corr_pre = (float)k.corr_pre;
    k.f.G = (float)k.G;
    k.f.two_over_G = (float)k.two_over_G;
    k.f.beta = (float)k.beta;
    k.f.half_1mbeta = (float)k.half_1mbeta;
    k.f.T_hot = (float)k.T_hot;
    k.f.T_cold = (float)k.T_cold;
    k.f.g_grav = (float)k.g_grav;
    k.f.T_in = (float)k.T_in;
    k.f.T_w = (float)k.T_w;
    k.f.U_in = (float)k.U_in;
    k.f.a = (float)k.a;
    k.f.b = (float)k.b;
    k.f.R = (float)k.R;
    k.f.cv = (float)k.cv;
    k.f.inv_cv = (float)k.inv_cv;
    k.f.T_psi = (float)k.T_psi;
    k.d.omc_f = (float)(1.0 - k.omega_f);
    k.d.omc_g = (float)(1.0 - k.omega_g);
    for (int c = 0; c < 2; ++c) {
        const double w = c == 0 ? 1.0 / 9.0 : 1.0 / 36.0;
        k.d.wo_f[c] = (float)(k.omega_f * w);
        k.d.wo_g[c] = (float)(k.omega_g * w);
        k.d.ocw_f[c] = (float)(k.omega_f * (double)k.cw_f[1 + c]);
        k.d.ocw_g[c] = (float)(k.omega_g * (double)k.cw_g[1 + c]);
        k.d.gw[c] = (float)(k.guo_pre * w);
        k.d.gw9[c] = (float)(9.0 * k.guo_pre * w);
        k.d.gw3[c] = (float)(3.0 * k.guo_pre * w);
        k.d.cw3[c] = (float)(3.0 * k.corr_pre * w);
    }
}

// a parameter in the arithmetic type `real`.  Translation units built with
// LB_KP_FLOAT (the 16-bit storage modes, bound by instruction issue) read the
// float copy when real is float; the others convert the double at the use
// (the same rounding; on the HBM-bound FP32 step this measured faster,
// 403 us against 438 us per 4096^2 launch, with the same registers).
template <typename real>
__device__ __forceinline__ real kpick(double d, float f) {
    if constexpr (sizeof(real) == sizeof(float))
        return f;
    else
        return (real)d;
}
#ifdef LB_KP_FLOAT
#define KPR(kp, name) (::lbgb::kpick<real>((kp).name, (kp).f.name))
#else
#define KPR(kp, name) ((real)(kp).name)
#endif

// Default limit of a bounded device wait, in clock cycles (about one second
// at GB300 clocks).
constexpr long long WAIT_CYCLES_DEFAULT = 2000000000LL;

enum BetaMode { BETA_ZERO = 0, BETA_ONE = 1, BETA_MIXED = 2 };

template <typename real>
__device__ __forceinline__ real p_eos(const KParams& kp, real rho, real T) {
    const real R = KPR(kp, R), a = KPR(kp, a), b = KPR(kp, b);
    if (kp.eos == LB_EOS_IDEAL) return rho * R * T;
    if (kp.eos == LB_EOS_VDW) return rho * R * T / ((real)1 - b * rho) - a * rho * rho;
    // Carnahan-Starling, eta = b rho / 4
    const real eta = b * rho / (real)4;
    if constexpr (sizeof(real) == 8) {
        // FP64 parity mode: the printed polynomial, evaluated term by term
        const real num = (real)1 + eta + eta * eta - eta * eta * eta;
        const real den = ((real)1 - eta) * ((real)1 - eta) * ((real)1 - eta);
        return rho * R * T * num / den - a * rho * rho;
    } else {
        const real num = (real)1 + eta * ((real)1 + eta * ((real)1 - eta));
        const real d = (real)1 - eta;
        return rho * R * T * num / (d * d * d) - a * rho * rho;
    }
}

// Periodic ghost columns kept on each side of a row in the strip layout: the
// column halo of a strip reaches two columns past its edge (the pull, plus
// one more site for psi).
constexpr int STRIP_GHOST = 2;
// The finite-difference step on strip contexts (k_fd_fused) reaches further:
// its second RK2 stage needs K one column out, K needs rho two columns out,
// and rho there needs the pull from three columns out.  Column halo of its
// row copies (elements: 16 or 32 bytes) and ghost columns kept on FD strip
// contexts.
constexpr int FD_HALO = 4;
constexpr int FD_GHOST = 3;

// Periodic ghost columns of the strip layout: the value stored at column x of
// a row is also stored at column x + nx when x < kp.ghost and at x - nx when
// x >= nx - kp.ghost, so that a row segment with its column halo is one
// contiguous copy even at the periodic edges.  p points at column x.
template <class S>
__device__ __forceinline__ void put_ghost(typename S::elem* p, int x, const KParams& kp,
                                          typename S::real v, typename S::real base) {
    if (x < kp.ghost) S::put(p + kp.nx, v, base);
    if (x >= kp.nx - kp.ghost) S::put(p - kp.nx, v, base);
}

// put_pop at p and, in the strip layout, at the periodic ghost copies of column x.
template <class S>
__device__ __forceinline__ void put_pop_ghost(typename S::elem* p, long long stride, int plane_idx, int x,
                                              const KParams& kp, typename S::real v, typename S::real base) {
    put_pop<S>(p, stride, plane_idx, v, base);
    if (x < kp.ghost) put_pop<S>(p + kp.nx, stride, plane_idx, v, base);
    if (x >= kp.nx - kp.ghost) put_pop<S>(p - kp.nx, stride, plane_idx, v, base);
}

// Store one value per plane at d (plane stride `stride`) and, for the few
// threads whose column has a periodic ghost copy, once more nx columns right
// (ghost_lo) or left (ghost_hi): one branch per site, not one per plane.
// The periodic ghost copies of a site's planes (columns within STRIP_GHOST of
// either edge are also written nx columns further in, see put_planes).
template <class S, typename IT>
__device__ __forceinline__ void put_ghost_copies(typename S::elem* d, IT stride, int nx, const typename S::elem* v,
                                                 bool ghost_lo, bool ghost_hi) {
    // (the plane offset is formed in IT, the signed column shift by pointer
    // arithmetic: an unsigned IT must never absorb a negative shift)
    if (ghost_lo || ghost_hi) {
        const int sh = ghost_lo ? nx : -nx;
#pragma unroll
        for (int p = 0; p < S::NPLANES; ++p) {
            typename S::elem* q = d + (IT)p * stride;
            q[sh] = v[p];
        }
        if (ghost_lo && ghost_hi) {  // lattices narrower than twice the ghost width
#pragma unroll
            for (int p = 0; p < S::NPLANES; ++p) {
                typename S::elem* q = d + (IT)p * stride;
                q[-nx] = v[p];
            }
        }
    }
}

template <class S, typename IT>
__device__ __forceinline__ void put_planes(typename S::elem* d, IT stride, int nx, const typename S::elem* v,
                                           bool ghost_lo, bool ghost_hi) {
#pragma unroll
    for (int p = 0; p < S::NPLANES; ++p) d[(IT)p * stride] = v[p];
    put_ghost_copies<S>(d, stride, nx, v, ghost_lo, ghost_hi);
}

// The post-collision populations of one site into storage; d points at the
// site in plane 0, `stride` is the plane stride, and with ghost_lo / ghost_hi
// the values also go to the periodic ghost copies nx columns right / left.
//   FP64, FP32: every value as computed (the FP32 collision has already
//     closed mass and energy through f_0 and g_0).
//   16-bit modes: the moving populations are rounded to their 16-bit
//     deviations first; the rest populations then take the deviations that
//     keep the site's stored deviation sums equal to the loaded ones, Hf and
//     Hg: h_0 = H - sum_{i>=1} h_i, at FP32 precision.  The collision of
//     Eq. (1) conserves mass and Eqs. (7)/(24) energy (the sums of f^eq, F_i,
//     g^eq and C_i), so this is exact up to one FP32 rounding per site, where
//     the rounding of each moving population on its own would change the
//     stored mass coherently, step after step.
template <class S, typename IT>
__device__ __forceinline__ void store_site(typename S::elem* d, IT stride, const KParams& kp,
                                           const typename S::real f[9], const typename S::real g[9],
                                           typename S::real Hf, typename S::real Hg, bool ghost_lo,
                                           bool ghost_hi) {
    using real = typename S::real;
    using elem = typename S::elem;
    elem v[S::NPLANES];
    if constexpr (S::SPLIT) {
        real sf = (real)0, sg = (real)0;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            v[i] = S::enc(f[i] - (real)kp.base_f[i]);
            v[9 + i] = S::enc(g[i] - (real)kp.base_g[i]);
            sf += S::dec(v[i]);
            sg += S::dec(v[9 + i]);
        }
        const unsigned bf = __float_as_uint(Hf - sf), bg = __float_as_uint(Hg - sg);
        v[0] = S::from_bits((unsigned short)(bf >> 16));
        v[18] = S::from_bits((unsigned short)(bf & 0xffffu));
        v[9] = S::from_bits((unsigned short)(bg >> 16));
        v[19] = S::from_bits((unsigned short)(bg & 0xffffu));
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            v[i] = (elem)f[i];
            v[9 + i] = (elem)g[i];
        }
    }
    put_planes<S>(d, stride, kp.nx, v, ghost_lo, ghost_hi);
}

// wrap a coordinate that may lie a few tiles outside [0, n)
__device__ __forceinline__ int wrapc(int v, int n) {
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

// clamp a coordinate into [0, n) (cavity: a wall node takes its nearest fluid node)
__device__ __forceinline__ int clampc(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// ring coordinate of a halo site: periodic wrap, or the nearest fluid node in a cavity
__device__ __forceinline__ int ringc(const KParams& kp, int v, int n) {
    return kp.walls ? clampc(v, n) : wrapc(v, n);
}

// Pull the 18 pre-collision populations of site (x, y).
template <class S>
__device__ __forceinline__ void pull18(const typename S::elem* __restrict__ src,
                                       const KParams& kp, int x, int y,
                                       typename S::real f[9], typename S::real g[9]) {
    if (kp.walls) {  // cavity: populations stored pre-collision at their own site
        const long long off = (long long)y * kp.pitch + x;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = load_pop<S>(src + (long long)i * kp.plane + off, kp.plane, i, (typename S::real)kp.base_f[i]);
            g[i] = load_pop<S>(src + (long long)(9 + i) * kp.plane + off, kp.plane, 9 + i,
                               (typename S::real)kp.base_g[i]);
        }
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
        const long long off = sr + sx;
        f[i] = load_pop<S>(src + (long long)i * kp.plane + off, kp.plane, i, (typename S::real)kp.base_f[i]);
        g[i] = load_pop<S>(src + (long long)(9 + i) * kp.plane + off, kp.plane, 9 + i,
                           (typename S::real)kp.base_g[i]);
    }
}

// pull18 of a periodic site that also returns the sums of the stored
// deviations (16-bit modes; zero otherwise), which store_site closes on.
template <class S>
__device__ __forceinline__ void pull18h(const typename S::elem* __restrict__ src, const KParams& kp, int x,
                                        int y, typename S::real f[9], typename S::real g[9],
                                        typename S::real& Hf, typename S::real& Hg) {
    Hf = Hg = (typename S::real)0;
    const int xm = x == 0 ? kp.nx - 1 : x - 1;
    const int xp = x == kp.nx - 1 ? 0 : x + 1;
    const long long r0 = (long long)y * kp.pitch;
    const long long rm = (long long)(y == 0 ? kp.ny - 1 : y - 1) * kp.pitch;
    const long long rp = (long long)(y == kp.ny - 1 ? 0 : y + 1) * kp.pitch;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sx = ex(i) == 1 ? xm : (ex(i) == -1 ? xp : x);
        const long long sr = ey(i) == 1 ? rm : (ey(i) == -1 ? rp : r0);
        const long long off = sr + sx;
        f[i] = load_pop_acc<S>(src + (long long)i * kp.plane + off, kp.plane, i, (typename S::real)kp.base_f[i], Hf);
        g[i] = load_pop_acc<S>(src + (long long)(9 + i) * kp.plane + off, kp.plane, 9 + i,
                               (typename S::real)kp.base_g[i], Hg);
    }
}

// The stored deviations of the 18 pre-collision populations of a periodic
// site (16-bit modes) and their sums Hf, Hg.
template <class S>
__device__ __forceinline__ void pull18_dev(const typename S::elem* __restrict__ src, const KParams& kp, int x,
                                           int y, float h[9], float q[9], float& Hf, float& Hg) {
    Hf = Hg = 0.0f;
    const int xm = x == 0 ? kp.nx - 1 : x - 1;
    const int xp = x == kp.nx - 1 ? 0 : x + 1;
    const long long r0 = (long long)y * kp.pitch;
    const long long rm = (long long)(y == 0 ? kp.ny - 1 : y - 1) * kp.pitch;
    const long long rp = (long long)(y == kp.ny - 1 ? 0 : y + 1) * kp.pitch;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sx = ex(i) == 1 ? xm : (ex(i) == -1 ? xp : x);
        const long long sr = ey(i) == 1 ? rm : (ey(i) == -1 ? rp : r0);
        const long long off = sr + sx;
        h[i] = dev_of<S>(src + (long long)i * kp.plane + off, i, rest_lo_offset(i) * kp.plane);
        q[i] = dev_of<S>(src + (long long)(9 + i) * kp.plane + off, 9 + i, rest_lo_offset(9 + i) * kp.plane);
        Hf += h[i];
        Hg += q[i];
    }
}

// rho, T and the pseudopotential (psi^2, and psi when beta != 0) of one site.
template <typename real, int BMODE>
__device__ __forceinline__ void site_psi(const KParams& kp, const real f[9], const real g[9],
                                         real& rho, real& T, real& psi, real& psi2, int& flags) {
    real r = f[0], e = g[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        r += f[i];
        e += g[i];
    }
    rho = r;
    T = e / (r * KPR(kp, cv));
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

// Eq. (4) force (Eq. (2) when beta = 1) from a shared-memory window with
// row stride W centred at index c.  Pair sums: east-west, north-south and the
// two diagonals, weights w(1) = 1/3, w(2) = 1/12.
template <typename real, int BMODE>
__device__ __forceinline__ void force_from_window(const KParams& kp, const real* s_psi,
                                                  const real* s_psi2, int c, int W,
                                                  real& Fx, real& Fy) {
    const real w1 = (real)(1.0 / 3.0), w2 = (real)(1.0 / 12.0);
    real fx = 0, fy = 0;
    if (BMODE != BETA_ZERO) {
        const real* p = s_psi;
        const real E = p[c + 1], Wv = p[c - 1], N = p[c + W], S = p[c - W];
        const real NE = p[c + W + 1], NW = p[c + W - 1], SE = p[c - W + 1], SW = p[c - W - 1];
        const real d1 = NE - SW, d2 = SE - NW, d3 = NW - SE;
        const real s1x = w1 * (E - Wv) + w2 * (d1 + d2);
        const real s1y = w1 * (N - S) + w2 * (d1 + d3);
        const real pc = (BMODE == BETA_ONE) ? p[c] : KPR(kp, beta) * p[c];
        fx += pc * s1x;
        fy += pc * s1y;
    }
    if (BMODE != BETA_ONE) {
        const real* p = s_psi2;
        const real E = p[c + 1], Wv = p[c - 1], N = p[c + W], S = p[c - W];
        const real NE = p[c + W + 1], NW = p[c + W - 1], SE = p[c - W + 1], SW = p[c - W - 1];
        const real d1 = NE - SW, d2 = SE - NW, d3 = NW - SE;
        const real s2x = w1 * (E - Wv) + w2 * (d1 + d2);
        const real s2y = w1 * (N - S) + w2 * (d1 + d3);
        const real h = (BMODE == BETA_ZERO) ? (real)0.5 : KPR(kp, half_1mbeta);
        fx += h * s2x;
        fy += h * s2y;
    }
    Fx = -KPR(kp, G) * fx;
    Fy = -KPR(kp, G) * fy;
}

// Collision of one site, Eq. (1) + F_i for f and Eq. (7) / (24) for g.
// f, g are overwritten with the post-collision values.
//
// Two evaluations of the same formulas:
//  * FP64 (parity mode): every formula in its printed form and order,
//    divisions by cs^2 included, no contraction (the FP64 translation unit is
//    compiled with --fmad=false), so results are reproducible bit for bit by
//    any literal FP64 implementation;
//  * FP32: multiplications by the constants 3, 4.5, 9 and one reciprocal of
//    rho, contracted to FMAs.
// FMA (FP32 only): the update in fused multiply-add form from the factors in
// kp.d, (1 - omega) f_i + P +- Q (see below); measured faster in the fused
// finite-difference kernel (+2.6%), slower in the strip and batched steps
// (-8% and -0.5%), which keep the direct form.
template <typename real, bool EQ24, bool FMA = false>
__device__ __forceinline__ void collide(const KParams& kp, real f[9], real g[9], real rho,
                                        real Fx, real Fy, real& ux_out, real& uy_out,
                                        real& T_out) {
    if constexpr (sizeof(real) == 8) {
        const double cs2 = 1.0 / 3.0;
        // sum_i e_i f_i in index order
        const double mx = ((((f[1] - f[3]) + f[5]) - f[6]) - f[7]) + f[8];
        const double my = ((((f[2] - f[4]) + f[5]) + f[6]) - f[7]) - f[8];
        double e = g[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) e += g[i];
        const double ux = (mx + 0.5 * Fx) / rho;
        const double uy = (my + 0.5 * Fy) / rho;
        const double T = e / (rho * kp.cv);
        const double usq = ux * ux + uy * uy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double w = wd(i);
            // e_i.u, e_i.F with the zero components dropped (exact)
            const double eu = ex(i) == 0 ? (ey(i) == 0 ? 0.0 : (ey(i) > 0 ? uy : -uy))
                                         : (ey(i) == 0 ? (ex(i) > 0 ? ux : -ux)
                                                       : (ex(i) > 0 ? ux : -ux) + (ey(i) > 0 ? uy : -uy));
            const double eF = ex(i) == 0 ? (ey(i) == 0 ? 0.0 : (ey(i) > 0 ? Fy : -Fy))
                                         : (ey(i) == 0 ? (ex(i) > 0 ? Fx : -Fx)
                                                       : (ex(i) > 0 ? Fx : -Fx) + (ey(i) > 0 ? Fy : -Fy));
            const double emuF = ((double)ex(i) - ux) * Fx + ((double)ey(i) - uy) * Fy;
            const double feq = rho * w * (1.0 + eu / cs2 + 0.5 * eu * eu / (cs2 * cs2) - 0.5 * usq / cs2);
            const double Fi = kp.guo_pre * w * (emuF / cs2 + eu * eF / (cs2 * cs2));
            f[i] = f[i] - kp.omega_f * (f[i] - feq) + Fi;
            const double geq = kp.cv * T * feq;
            double gs = g[i] - kp.omega_g * (g[i] - geq);
            if (EQ24) gs += kp.corr_pre * w * kp.cv * T * eF / cs2;
            g[i] = gs;
        }
        ux_out = ux;
        uy_out = uy;
        T_out = T;
    } else {
        const real mx = (f[1] - f[3]) + ((f[5] - f[7]) + (f[8] - f[6]));
        const real my = (f[2] - f[4]) + ((f[5] - f[7]) + (f[6] - f[8]));
        real e = g[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) e += g[i];
        const real inv_rho = (real)1 / rho;
        const real ux = (mx + (real)0.5 * Fx) * inv_rho;
        const real uy = (my + (real)0.5 * Fy) * inv_rho;
        const real T = e / (rho * KPR(kp, cv));
        const real cvT = KPR(kp, cv) * T;
        if constexpr (FMA) {
            const real m15u2 = (real)-1.5 * fmaf(ux, ux, uy * uy);
            const real uF3 = (real)3 * fmaf(ux, Fx, uy * Fy);
            // Opposite directions i and i' = opposite(i) share the even parts of
            // f^eq and F_i; the odd parts change sign:
            //   f^eq = rho w (1 - 1.5 u^2 + 4.5 (e.u)^2) +- 3 rho w (e.u)
            //   F_i  = guo w (9 (e.u)(e.F) - 3 u.F)      +- 3 guo w (e.F)
            //   C_i  =                                     +- 3 corr w c_v T (e.F)
            // and with c_v T rho = e, c_v T f^eq = e w (...).  The update
            // f_i <- f_i + omega_f (f^eq_i - f_i) + F_i is evaluated as
            // (1 - omega_f) f_i + P +- Q, P = omega_f (even part of f^eq) + (even
            // part of F_i), Q the odd parts, the same for g with C_i: fused
            // multiply-adds of per-site factors (per weight class c: axis, diagonal)
            // and the constants in kp.d.
            real A[2], r45[2], r3[2], B[2], e45[2], e3[2], c3[2];
    #pragma unroll
            for (int c = 0; c < 2; ++c) {
                const real rwo = kp.d.wo_f[c] * rho, ewo = kp.d.wo_g[c] * e;
                A[c] = fmaf(-kp.d.gw[c], uF3, fmaf(rwo, m15u2, rwo));
                r45[c] = (real)4.5 * rwo;
                r3[c] = (real)3 * rwo;
                B[c] = fmaf(ewo, m15u2, ewo);
                e45[c] = (real)4.5 * ewo;
                e3[c] = (real)3 * ewo;
                c3[c] = EQ24 ? kp.d.cw3[c] * cvT : (real)0;
            }
            const real omc_f = kp.d.omc_f, omc_g = kp.d.omc_g;
            // pairs (1,3), (2,4), (5,7), (8,6): e(i) = (dx, dy), e(i') = -(dx, dy)
    #pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int i = p == 0 ? 1 : (p == 1 ? 2 : (p == 2 ? 5 : 8));
                const int k = p == 0 ? 3 : (p == 1 ? 4 : (p == 2 ? 7 : 6));
                const int c = p < 2 ? 0 : 1;
                const real eu = p == 0 ? ux : (p == 1 ? uy : (p == 2 ? ux + uy : ux - uy));
                const real eF = p == 0 ? Fx : (p == 1 ? Fy : (p == 2 ? Fx + Fy : Fx - Fy));
                const real eu2 = eu * eu;
                const real P = fmaf(kp.d.gw9[c], eu * eF, fmaf(r45[c], eu2, A[c]));
                const real Q = fmaf(r3[c], eu, kp.d.gw3[c] * eF);
                f[i] = fmaf(omc_f, f[i], P + Q);
                f[k] = fmaf(omc_f, f[k], P - Q);
                const real Pg = fmaf(e45[c], eu2, B[c]);
                const real Qg = EQ24 ? fmaf(c3[c], eF, e3[c] * eu) : e3[c] * eu;
                g[i] = fmaf(omc_g, g[i], Pg + Qg);
                g[k] = fmaf(omc_g, g[k], Pg - Qg);
            }
        } else {
            const real om_f = KPR(kp, omega_f), om_g = KPR(kp, omega_g);
            const real guo = KPR(kp, guo_pre), corr = KPR(kp, corr_pre);
            const real base = (real)1 - (real)1.5 * (ux * ux + uy * uy);
            const real uF3 = (real)3 * (ux * Fx + uy * Fy);
            // Opposite directions i and i' = opposite(i) share the even parts of
            // f^eq and F_i; the odd parts change sign:
            //   f^eq = rho w (1 - 1.5 u^2 + 4.5 (e.u)^2) +- 3 rho w (e.u)
            //   F_i  = guo w (9 (e.u)(e.F) - 3 u.F)      +- 3 guo w (e.F)
            //   C_i  =                                     +- 3 corr w c_v T (e.F)
            // pairs (1,3), (2,4), (5,7), (8,6): e(i) = (dx, dy), e(i') = -(dx, dy)
    #pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int i = p == 0 ? 1 : (p == 1 ? 2 : (p == 2 ? 5 : 8));
                const int k = p == 0 ? 3 : (p == 1 ? 4 : (p == 2 ? 7 : 6));
                const real w = (real)wd(i);
                const real eu = (real)ex(i) * ux + (real)ey(i) * uy;
                const real eF = (real)ex(i) * Fx + (real)ey(i) * Fy;
                const real rw = rho * w;
                const real feq_even = rw * (base + (real)4.5 * eu * eu);
                const real feq_odd = (real)3 * rw * eu;
                const real F_even = guo * w * ((real)9 * eu * eF - uF3);
                const real F_odd = (real)3 * guo * w * eF;
                const real feq_i = feq_even + feq_odd, feq_k = feq_even - feq_odd;
                f[i] = f[i] + om_f * (feq_i - f[i]) + (F_even + F_odd);
                f[k] = f[k] + om_f * (feq_k - f[k]) + (F_even - F_odd);
                real gi = g[i] + om_g * (cvT * feq_i - g[i]);
                real gk = g[k] + om_g * (cvT * feq_k - g[k]);
                if (EQ24) {
                    const real C_odd = (real)3 * corr * w * cvT * eF;
                    gi += C_odd;
                    gk -= C_odd;
                }
                g[i] = gi;
                g[k] = gk;
            }
        }
        // The collision conserves mass and energy exactly: sum f^eq = rho,
        // sum F_i = 0, sum g^eq = rho c_v T = sum g, sum C_i = 0.  In FP32 the
        // rounded weights alone would add ~7.5e-9 rho per step, coherently, so
        // the rest populations take the exact balance instead.
        real sf = f[1], sg = g[1];
#pragma unroll
        for (int i = 2; i < 9; ++i) {
            sf += f[i];
            sg += g[i];
        }
        f[0] = rho - sf;
        g[0] = e - sg;
        ux_out = ux;
        uy_out = uy;
        T_out = T;
    }
}

// 16-bit modes: the collision of Eq. (1) with F_i and of Eq. (7) / (24) in the
// deviation variables the storage holds, h_i = f_i - base_f[i] and
// q_i = g_i - base_g[i] (base = w_i rho0 and w_i rho0 c_v T0), for the moving
// populations i = 1..8 (the rest populations follow from the closure in
// store_site_dev).  Hf, Hg: the sums of all nine loaded deviations, so that
// rho = sum base_f + Hf and the energy density rho c_v T = sum base_g + Hg.
// The same formulas as collide(): with f^eq_i = w_i rho (1 + 3 e.u + 4.5 (e.u)^2
// - 1.5 u^2) and c_v T rho = e,
//   f^eq_i - base_i = w_i (rho - rho0) + (w_i rho0 - base_i) + w_i rho (4.5 (e.u)^2 - 1.5 u^2) + 3 w_i rho e.u
//   c_v T f^eq_i - base_g,i = w_i (e - e0) + (w_i e0 - base_g,i) + w_i e (4.5 (e.u)^2 - 1.5 u^2) + 3 w_i e e.u
// so no base is added to or subtracted from a population (fewer operations,
// and the small deviations keep their own FP32 precision).  The update
//   h_i <- h_i + omega_f (f^eq_i - base_i - h_i) + F_i
// is evaluated as (1 - omega_f) h_i + P +- Q, with P = omega_f (even part of
// f^eq - base) + (even part of F_i) and Q = omega_f (odd part) + (odd part),
// the same for q_i with C_i of Eq. (25) in its odd part: every term is a
// fused multiply-add of per-site factors and the constants in kp.d.
template <bool EQ24>
__device__ __forceinline__ void collide_dev(const KParams& kp, float h[9], float q[9], float Hf, float Hg,
                                            float Fx, float Fy) {
    const float rho = kp.sum_bf + Hf, e = kp.sum_bg + Hg;
    const float drho = kp.dsum_f + Hf, de = kp.dsum_g + Hg;
    const float mx = (h[1] - h[3]) + ((h[5] - h[7]) + (h[8] - h[6]));
    const float my = (h[2] - h[4]) + ((h[5] - h[7]) + (h[6] - h[8]));
    const float inv_rho = 1.0f / rho;
    const float ux = (mx + 0.5f * Fx) * inv_rho;
    const float uy = (my + 0.5f * Fy) * inv_rho;
    const float cvT = e * inv_rho;
    const float m15u2 = -1.5f * fmaf(ux, ux, uy * uy);
    const float uF3 = 3.0f * fmaf(ux, Fx, uy * Fy);
    // per weight class c (axis, diagonal):
    //   P0 = omega_f (w drho + cw_f) + omega_f w rho (-1.5 u^2) - guo w 3 u.F
    //   P  = P0 + 4.5 omega_f w rho (e.u)^2 + 9 guo w (e.u)(e.F)
    //   Q  = 3 omega_f w rho (e.u) + 3 guo w (e.F)
    //   G0 = omega_g (w de + cw_g) + omega_g w e (-1.5 u^2)
    //   Pg = G0 + 4.5 omega_g w e (e.u)^2,   Qg = 3 omega_g w e (e.u) [+ 3 corr w c_v T (e.F)]
    float P0[2], r45[2], r3[2], G0[2], e45[2], e3[2], c3[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float rwo = kp.d.wo_f[c] * rho, ewo = kp.d.wo_g[c] * e;
        P0[c] = fmaf(-kp.d.gw[c], uF3, fmaf(rwo, m15u2, fmaf(kp.d.wo_f[c], drho, kp.d.ocw_f[c])));
        r45[c] = 4.5f * rwo;
        r3[c] = 3.0f * rwo;
        G0[c] = fmaf(ewo, m15u2, fmaf(kp.d.wo_g[c], de, kp.d.ocw_g[c]));
        e45[c] = 4.5f * ewo;
        e3[c] = 3.0f * ewo;
        c3[c] = EQ24 ? kp.d.cw3[c] * cvT : 0.0f;
    }
    const float omc_f = kp.d.omc_f, omc_g = kp.d.omc_g;
    // pairs of opposite directions (1,3), (2,4), (5,7), (8,6) share the even parts
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = p == 0 ? 1 : (p == 1 ? 2 : (p == 2 ? 5 : 8));
        const int k = p == 0 ? 3 : (p == 1 ? 4 : (p == 2 ? 7 : 6));
        const int c = p < 2 ? 0 : 1;
        const float eu = p == 0 ? ux : (p == 1 ? uy : (p == 2 ? ux + uy : ux - uy));
        const float eF = p == 0 ? Fx : (p == 1 ? Fy : (p == 2 ? Fx + Fy : Fx - Fy));
        const float eu2 = eu * eu;
        const float P = fmaf(kp.d.gw9[c], eu * eF, fmaf(r45[c], eu2, P0[c]));
        const float Q = fmaf(r3[c], eu, kp.d.gw3[c] * eF);
        h[i] = fmaf(omc_f, h[i], P + Q);
        h[k] = fmaf(omc_f, h[k], P - Q);
        const float Pg = fmaf(e45[c], eu2, G0[c]);
        const float Qg = EQ24 ? fmaf(c3[c], eF, e3[c] * eu) : e3[c] * eu;
        q[i] = fmaf(omc_g, q[i], Pg + Qg);
        q[k] = fmaf(omc_g, q[k], Pg - Qg);
    }
}

// The stored form of a site whose deviations collide_dev computed (16-bit
// modes): the moving populations rounded to 16 bits, the rest populations
// closing the stored deviation sums (see store_site), as the NPLANES values of
// the site's planes.
template <class S>
__device__ __forceinline__ void encode_site_dev(const float h[9], const float q[9], float Hf, float Hg,
                                                typename S::elem v[S::NPLANES]) {
    static_assert(S::SPLIT, "deviation storage only");
    float sf = 0.0f, sg = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        v[i] = S::enc(h[i]);
        v[9 + i] = S::enc(q[i]);
        sf = S::add_dec(v[i], sf);
        sg = S::add_dec(v[9 + i], sg);
    }
    const unsigned bf = __float_as_uint(Hf - sf), bg = __float_as_uint(Hg - sg);
    v[0] = S::from_bits((unsigned short)(bf >> 16));
    v[18] = S::from_bits((unsigned short)(bf & 0xffffu));
    v[9] = S::from_bits((unsigned short)(bg >> 16));
    v[19] = S::from_bits((unsigned short)(bg & 0xffffu));
}

// store_site for deviations already computed by collide_dev (16-bit modes).
template <class S, typename IT>
__device__ __forceinline__ void store_site_dev(typename S::elem* d, IT stride, const KParams& kp,
                                               const float h[9], const float q[9], float Hf, float Hg,
                                               bool ghost_lo, bool ghost_hi) {
    typename S::elem v[S::NPLANES];
    encode_site_dev<S>(h, q, Hf, Hg, v);
    put_planes<S>(d, stride, kp.nx, v, ghost_lo, ghost_hi);
}

// ---------------------------------------------------------------- step
// One fused time step.  CTA tile BX x BY; phase 1 computes psi for the tile
// plus a one-site ring from pulled populations (ring pulls hit L2), phase 2
// pulls each tile site again (L1), applies the stencil and both collisions,
// and stores 18 values at the site (the next step pulls them).
template <int PREC, int BX, int BY, bool EQ24, int BMODE>
__global__ void __launch_bounds__(BX* BY)
    k_step(const typename Store<PREC>::elem* __restrict__ src,
           typename Store<PREC>::elem* __restrict__ dst, const KParams kp) {
    using S = Store<PREC>;
    using real = typename S::real;
    constexpr int WX = BX + 2, WY = BY + 2, NT = BX * BY;
    __shared__ real s_psi[BMODE != BETA_ZERO ? WX * WY : 1];
    __shared__ real s_psi2[BMODE != BETA_ONE ? WX * WY : 1];

    const int tid = threadIdx.x + threadIdx.y * BX;
    // rows updated: [H, ny - H) (H = kp.halo_rows; 0 on a periodic lattice)
    const int H = kp.halo_rows;
    const int x0 = blockIdx.x * BX, y0 = H + blockIdx.y * BY;
    int flags = 0;
    for (int s = tid; s < WX * WY; s += NT) {
        const int ly = s / WX, lx = s - ly * WX;
        const int gx = wrapc(x0 + lx - 1, kp.nx), gy = wrapc(y0 + ly - 1, kp.ny);
        real f[9], g[9], rho, T, psi, psi2;
        int fl = 0;
        pull18<S>(src, kp, gx, gy, f, g);
        site_psi<real, BMODE>(kp, f, g, rho, T, psi, psi2, fl);
        // ring rows beyond the updated range (ghost rows' own ring) do not report
        if (y0 + ly - 1 <= kp.ny - H) flags |= fl;
        if (BMODE != BETA_ZERO) s_psi[s] = psi;
        if (BMODE != BETA_ONE) s_psi2[s] = psi2;
    }
    __syncthreads();

    const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
    if (gx < kp.nx && gy < kp.ny - H) {
        real Fx, Fy, ux, uy, T;
        force_from_window<real, BMODE>(kp, s_psi, s_psi2, (threadIdx.y + 1) * WX + threadIdx.x + 1,
                                       WX, Fx, Fy);
        const long long off = (long long)gy * kp.pitch + gx;
        if constexpr (S::SPLIT) {
            float h[9], q[9], Hf, Hg;
            pull18_dev<S>(src, kp, gx, gy, h, q, Hf, Hg);
            collide_dev<EQ24>(kp, h, q, Hf, Hg, Fx, Fy);
            store_site_dev<S>(dst + off, kp.plane, kp, h, q, Hf, Hg, false, false);
        } else {
            real f[9], g[9], Hf, Hg;
            pull18h<S>(src, kp, gx, gy, f, g, Hf, Hg);
            real rho = f[0];
#pragma unroll
            for (int i = 1; i < 9; ++i) rho += f[i];
            collide<real, EQ24>(kp, f, g, rho, Fx, Fy, ux, uy, T);
            store_site<S>(dst + off, kp.plane, kp, f, g, Hf, Hg, false, false);
        }
    } else {
        flags = 0;
    }
    if (flags) atomicOr(kp.err, flags);
}

// ---------------------------------------------------------------- moments
// Same front end as the step; phase 2 writes rho, u (with F/2), T (any
// pointer may be null) and, if `part` is set, reduces FP64 totals per CTA:
//   part[blk*8 + k], k = mass, energy, rho ux, rho uy, |d rho|^2, rho^2, |dT|^2, T^2
// against the reference fields ref_rho/ref_T (may be null).
template <int PREC, int BX, int BY, int BMODE>
__global__ void __launch_bounds__(BX* BY)
    k_moments(const typename Store<PREC>::elem* __restrict__ src, const KParams kp,
              double* __restrict__ o_rho, double* __restrict__ o_ux, double* __restrict__ o_uy,
              double* __restrict__ o_T, const double* __restrict__ ref_rho,
              const double* __restrict__ ref_T, double* __restrict__ part) {
    using S = Store<PREC>;
    using real = typename S::real;
    constexpr int WX = BX + 2, WY = BY + 2, NT = BX * BY;
    __shared__ real s_psi[BMODE != BETA_ZERO ? WX * WY : 1];
    __shared__ real s_psi2[BMODE != BETA_ONE ? WX * WY : 1];
    __shared__ double s_red[NT / 32][8];

    const int tid = threadIdx.x + threadIdx.y * BX;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    int flags = 0;
    for (int s = tid; s < WX * WY; s += NT) {
        const int ly = s / WX, lx = s - ly * WX;
        const int gx = ringc(kp, x0 + lx - 1, kp.nx), gy = ringc(kp, y0 + ly - 1, kp.ny);
        real f[9], g[9], rho, T, psi, psi2;
        pull18<S>(src, kp, gx, gy, f, g);
        site_psi<real, BMODE>(kp, f, g, rho, T, psi, psi2, flags);
        if (BMODE != BETA_ZERO) s_psi[s] = psi;
        if (BMODE != BETA_ONE) s_psi2[s] = psi2;
    }
    __syncthreads();

    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
    if (gx < kp.nx && gy < kp.ny) {
        real f[9], g[9];
        pull18<S>(src, kp, gx, gy, f, g);
        real rho = f[0];
        double m = (double)f[0], e = (double)g[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            rho += f[i];
            m += (double)f[i];
            e += (double)g[i];
        }
        real Fx, Fy, ux, uy, T;
        force_from_window<real, BMODE>(kp, s_psi, s_psi2, (threadIdx.y + 1) * WX + threadIdx.x + 1,
                                       WX, Fx, Fy);
        if (kp.walls) Fy += -rho * KPR(kp, g_grav);  // cavity buoyancy
        collide<real, false>(kp, f, g, rho, Fx, Fy, ux, uy, T);
        const long long idx = (long long)gy * kp.nx + gx;
        if (o_rho) o_rho[idx] = (double)rho;
        if (o_ux) o_ux[idx] = (double)ux;
        if (o_uy) o_uy[idx] = (double)uy;
        if (o_T) o_T[idx] = (double)T;
        if (part) {
            const double dr = (double)rho, dT = (double)T;
            v[0] = m;
            v[1] = e;
            v[2] = dr * (double)ux;
            v[3] = dr * (double)uy;
            if (ref_rho) {
                const double a = dr - ref_rho[idx], b = dT - ref_T[idx];
                v[4] = a * a;
                v[6] = b * b;
            }
            v[5] = dr * dr;
            v[7] = dT * dT;
        }
    } else {
        flags = 0;
    }
    if (flags) atomicOr(kp.err, flags);
    if (!part) return;
    // deterministic block reduction: warp tree, then warps in order
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((tid & 31) == 0) s_red[tid >> 5][k] = x;
    }
    __syncthreads();
    if (tid < 8) {
        double x = 0.0;
        for (int w = 0; w < NT / 32; ++w) x += s_red[w][tid];
        part[(long long)(blockIdx.y * gridDim.x + blockIdx.x) * 8 + tid] = x;
    }
}

// ---------------------------------------------------------------- init / gather
// Initial state f = f^eq(rho0, 0) = w_i rho0, g = c_v T0 w_i rho0, written at
// the source position so the first pull sees it at its own site.
template <int PREC>
__global__ void k_init(typename Store<PREC>::elem* __restrict__ dst, const KParams kp,
                       const double* __restrict__ rho0, const double* __restrict__ T0) {
    using S = Store<PREC>;
    using real = typename S::real;
    const long long n = (long long)kp.nx * kp.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % kp.nx), y = (int)(s / kp.nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            // the value stored at (x, y) is pulled by site (x + e_i, y + e_i)
            // (cavity: stored pre-collision at its own site)
            const int dx = kp.walls ? x : wrapc(x + ex(i), kp.nx), dy = kp.walls ? y : wrapc(y + ey(i), kp.ny);
            const long long d = (long long)dy * kp.nx + dx;
            const double fe = rho0[d] * wd(i);
            const double ge = kp.cv * T0[d] * fe;
            const long long off = (long long)y * kp.pitch + x;
            typename S::elem* pf = dst + (long long)i * kp.plane + off;
            typename S::elem* pg = dst + (long long)(9 + i) * kp.plane + off;
            put_pop_ghost<S>(pf, kp.plane, i, x, kp, (real)fe, (real)kp.base_f[i]);
            put_pop_ghost<S>(pg, kp.plane, 9 + i, x, kp, (real)ge, (real)kp.base_g[i]);
        }
    }
}

// Pre-collision populations at t (pull) -> dense float64 [18][ny][nx].
template <int PREC>
__global__ void k_gather(const typename Store<PREC>::elem* __restrict__ src, const KParams kp,
                         double* __restrict__ out) {
    using S = Store<PREC>;
    using real = typename S::real;
    const long long n = (long long)kp.nx * kp.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % kp.nx), y = (int)(s / kp.nx);
        real f[9], g[9];
        pull18<S>(src, kp, x, y, f, g);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            out[(long long)i * n + s] = (double)f[i];
            out[(long long)(9 + i) * n + s] = (double)g[i];
        }
    }
}

// Dense float64 [18][ny][nx] pre-collision populations -> storage (push to source).
template <int PREC>
__global__ void k_scatter(typename Store<PREC>::elem* __restrict__ dst, const KParams kp,
                          const double* __restrict__ in) {
    using S = Store<PREC>;
    using real = typename S::real;
    const long long n = (long long)kp.nx * kp.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % kp.nx), y = (int)(s / kp.nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            // f_i(x, t) is stored at x - e_i (cavity: at x)
            const int sx = kp.walls ? x : wrapc(x - ex(i), kp.nx), sy = kp.walls ? y : wrapc(y - ey(i), kp.ny);
            const long long off = (long long)sy * kp.pitch + sx;
            typename S::elem* pf = dst + (long long)i * kp.plane + off;
            typename S::elem* pg = dst + (long long)(9 + i) * kp.plane + off;
            const real vf = (real)in[(long long)i * n + s], vg = (real)in[(long long)(9 + i) * n + s];
            put_pop_ghost<S>(pf, kp.plane, i, sx, kp, vf, (real)kp.base_f[i]);
            put_pop_ghost<S>(pg, kp.plane, 9 + i, sx, kp, vg, (real)kp.base_g[i]);
        }
    }
}

}  // namespace lbgb
