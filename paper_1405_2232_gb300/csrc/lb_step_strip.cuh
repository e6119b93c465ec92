// lb_step_strip.cuh -- the fused step as a strip-marching kernel fed by TMA
// bulk copies (sm_90+ cp.async.bulk, mbarrier transaction counts).
//
// Each CTA owns a strip of columns and a chunk of rows and marches up the
// rows.  For every pre-collision row y it needs plane i of source row
// y - e_iy, columns [x0 - HALO, x0 + W + HALO) (HALO * sizeof(elem) = 16
// bytes, so every copy is 16-byte aligned); a producer warp streams these
// 18 row segments into a STAGES-deep shared-memory ring with cp.async.bulk,
// completion tracked by one mbarrier per stage.  Each consumer warp then
//   1. computes rho, T and psi of row y for its 30 columns plus one halo
//      column each side into its own 4-row psi ring,
//   2. collides row y - 1 (Eq. (1) + F_i and Eq. (7)/(24)), whose three psi
//      rows are now complete, reading its populations back from the stage
//      ring and storing the 18 post-collision values with coalesced stores.
// psi is computed for 32 columns per 30 sites (plus 2 rows per chunk), and
// every population is read from HBM once and written once.
//
// Periodic wrap: rows wrap by index; the column halo of the first/last strip
// is fetched from the other end of the row with separate 16-byte copies, so
// the kernel needs nx to be a multiple of HALO (checked on the host).
//
// A dedicated producer warp issues the copies; the consumer warps release a
// stage through a second mbarrier when its last reader is done.  Nothing
// synchronises the whole CTA after set-up.
//
// Every mbarrier wait is bounded: on timeout the CTA records LB_ERR_TIMEOUT,
// the producer waits (again bounded) for the copies it issued, and returns.
#pragma once

#include "lb_device.cuh"

namespace lbgb {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, "
        "p;\n}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait (about one second at GB300 clocks); false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > 2000000000LL) return false;
    }
    return true;
}

// Eq. (4) force from the 3x3 psi neighbourhood given as three row pointers
// (south, centre, north) at the centre column.  Same arithmetic and order as
// force_from_window.
template <typename real, int BMODE>
__device__ __forceinline__ void force_from_rows(const KParams& kp, const real* ps, const real* pc,
                                                const real* pn, const real* qs, const real* qc,
                                                const real* qn, real& Fx, real& Fy) {
    const real w1 = (real)(1.0 / 3.0), w2 = (real)(1.0 / 12.0);
    real fx = 0, fy = 0;
    if (BMODE != BETA_ZERO) {
        const real E = pc[1], Wv = pc[-1], N = pn[0], S = ps[0];
        const real NE = pn[1], NW = pn[-1], SE = ps[1], SW = ps[-1];
        const real d1 = NE - SW, d2 = SE - NW, d3 = NW - SE;
        const real s1x = w1 * (E - Wv) + w2 * (d1 + d2);
        const real s1y = w1 * (N - S) + w2 * (d1 + d3);
        const real c = (BMODE == BETA_ONE) ? pc[0] : (real)kp.beta * pc[0];
        fx += c * s1x;
        fy += c * s1y;
    }
    if (BMODE != BETA_ONE) {
        const real E = qc[1], Wv = qc[-1], N = qn[0], S = qs[0];
        const real NE = qn[1], NW = qn[-1], SE = qs[1], SW = qs[-1];
        const real d1 = NE - SW, d2 = SE - NW, d3 = NW - SE;
        const real s2x = w1 * (E - Wv) + w2 * (d1 + d2);
        const real s2y = w1 * (N - S) + w2 * (d1 + d3);
        const real h = (BMODE == BETA_ZERO) ? (real)0.5 : (real)kp.half_1mbeta;
        fx += h * s2x;
        fy += h * s2y;
    }
    Fx = -(real)kp.G * fx;
    Fy = -(real)kp.G * fy;
}

template <int PREC>
struct StripCfg {
    using elem = typename Store<PREC>::elem;
    using real = typename Store<PREC>::real;
    static constexpr int ES = (int)sizeof(elem);
    static constexpr int HALO = 16 / ES;  // 16-byte halo: 2 (FP64), 4 (FP32), 8 (16-bit)
};

// Columns a consumer warp owns: 30 interior sites, plus one halo column on
// each side for its own psi, so a warp never needs another warp's psi.
constexpr int WARP_COLS = 30;

template <int PREC, int NW, int STAGES>
constexpr size_t strip_smem_bytes() {
    using C = StripCfg<PREC>;
    return (size_t)STAGES * 18 * (NW * WARP_COLS + 2 * C::HALO) * C::ES +
           (size_t)NW * 8 * 32 * sizeof(typename C::real) + (size_t)2 * STAGES * 8 + 16;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Block: NW consumer warps plus one producer warp.  The strip is NW * 30
// columns wide.
//   producer: for every job (pre-collision row) waits until its stage is
//     released, then lane 0 arms the stage's "full" mbarrier with the byte
//     count and lanes 0..17 each issue the copies of one plane-row segment.
//   consumer warp w (interior columns 30w .. 30w+29 of the strip): waits
//     "full", lane l computes psi of column 30w + l - 1 into the warp's own
//     4-row psi ring, __syncwarp, lanes 1..30 collide the row behind, then
//     the warp releases that row's stage on its "empty" mbarrier.  There is
//     no block-wide barrier: warps drift freely within the stage ring.
template <int PREC, int NW, int STAGES, bool EQ24, int BMODE>
__global__ void __launch_bounds__(NW * 32 + 32, 2)
    k_step_strip(const typename Store<PREC>::elem* __restrict__ src,
                 typename Store<PREC>::elem* __restrict__ dst, const KParams kp, int nch_full,
                 int nch_last) {
    using S = Store<PREC>;
    using C = StripCfg<PREC>;
    using elem = typename C::elem;
    using real = typename C::real;
    constexpr int HALO = C::HALO;
    constexpr int BXI = NW * WARP_COLS;  // interior columns of a strip
    constexpr int SEGW = BXI + 2 * HALO;
    constexpr int ES = C::ES;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    elem* stage = reinterpret_cast<elem*>(smem_raw);  // [STAGES][18][SEGW]
    real* rings = reinterpret_cast<real*>(stage + (size_t)STAGES * 18 * SEGW);  // [NW][2][4][32]
    uint64_t* full = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(rings + NW * 8 * 32) + 7) & ~uintptr_t(7));
    uint64_t* empty = full + STAGES;

    const int t = threadIdx.x;
    const int nx = kp.nx, ny = kp.ny;
    // 1-D grid: the full-width strips get nch_full row chunks each, a narrower
    // last strip gets nch_last, so every CTA carries about the same work
    const int full_strips = nx / BXI;
    int strip, chunk, nchunks;
    if ((int)blockIdx.x < full_strips * nch_full) {
        strip = blockIdx.x / nch_full;
        chunk = blockIdx.x - strip * nch_full;
        nchunks = nch_full;
    } else {
        strip = full_strips;
        chunk = blockIdx.x - full_strips * nch_full;
        nchunks = nch_last;
    }
    const int x0 = strip * BXI;
    const int W = min(BXI, nx - x0);
    const int y_start = (int)((long long)chunk * ny / nchunks);
    const int y_end = (int)((long long)(chunk + 1) * ny / nchunks);
    const int njobs = (y_end - y_start) + 2;  // pre-collision rows y_start-1 .. y_end
    const uint32_t plane = (uint32_t)kp.plane, pitch = (uint32_t)kp.pitch;

    if (t == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (t >= NW * 32) {
        // ------------------------------------------------ producer warp
        const int lane = t - NW * 32;
        const bool left_wrap = x0 == 0;
        const bool right_wrap = x0 + W == nx;
        int issued = 0;
        for (int j = 0; j < njobs; ++j) {
            const int s = j % STAGES;
            if (j >= STAGES) {
                // the stage's previous job (j - STAGES) must have been released;
                // on timeout stop issuing (the consumers then time out on "full")
                if (!mbar_wait_bounded(&empty[s], (uint32_t)(((j / STAGES) - 1) & 1))) {
                    if (lane == 0) atomicOr(kp.err, 1 << LB_ERR_TIMEOUT);
                    break;
                }
            }
            int y = y_start - 1 + j;
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)(18 * (W + 2 * HALO) * ES));
            __syncwarp();
            if (lane < 18) {
                const int i = lane;
                const int d = i < 9 ? i : i - 9;
                int sy = y - ey(d);
                sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                const elem* row = src + (size_t)((uint32_t)i * plane + (uint32_t)sy * pitch);
                elem* seg = stage + ((size_t)s * 18 + i) * SEGW;
                if (!left_wrap && !right_wrap) {
                    bulk_copy_g2s(seg, row + (x0 - HALO), (uint32_t)((W + 2 * HALO) * ES), &full[s]);
                } else {
                    bulk_copy_g2s(seg, row + (left_wrap ? nx - HALO : x0 - HALO), HALO * ES, &full[s]);
                    bulk_copy_g2s(seg + HALO, row + x0, (uint32_t)(W * ES), &full[s]);
                    bulk_copy_g2s(seg + HALO + W, row + (right_wrap ? 0 : x0 + W), HALO * ES, &full[s]);
                }
            }
            issued = j + 1;
        }
        // leave only when every copy this CTA issued has landed (bounded)
        if (lane == 0)
            for (int j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j)
                (void)mbar_wait_bounded(&full[j % STAGES], (uint32_t)((j / STAGES) & 1));
        return;
    }

    // ---------------------------------------------------- consumer warps
    const int warp = t >> 5, lane = t & 31;
    const int col = warp * WARP_COLS + lane - 1;    // strip column of this lane's psi site
    const bool has_psi = col <= W;                  // columns -1 .. W are needed
    const bool collides = lane >= 1 && lane <= WARP_COLS && col < W;
    real* rp = rings + (size_t)warp * 8 * 32;        // [4][32] psi
    real* rq = rp + 4 * 32;                          // [4][32] psi^2
    int flags = 0;
    bool abort = false;
    for (int j = 0; j < njobs; ++j) {
        const int s = j % STAGES;
        if (!mbar_wait_bounded(&full[s], (uint32_t)((j / STAGES) & 1))) {
            abort = true;
            break;
        }
        // 1. rho, T, psi of pre-collision row j at this lane's column
        if (has_psi) {
            const elem* st = stage + (size_t)s * 18 * SEGW;
            const int c = col + HALO;  // smem column of the site
            real f[9], g[9], rho, T, psi, psi2;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i] = S::load(st + i * SEGW + c - ex(i), (real)kp.base_f[i]);
                g[i] = S::load(st + (9 + i) * SEGW + c - ex(i), (real)kp.base_g[i]);
            }
            site_psi<real, BMODE>(kp, f, g, rho, T, psi, psi2, flags);
            if (BMODE != BETA_ZERO) rp[(j & 3) * 32 + lane] = psi;
            if (BMODE != BETA_ONE) rq[(j & 3) * 32 + lane] = psi2;
        }
        __syncwarp();
        // 2. collide pre-collision row j-1 (its psi neighbourhood is complete)
        if (j >= 2 && collides) {
            const int sp = (j - 1) % STAGES;
            const elem* st = stage + (size_t)sp * 18 * SEGW;
            const int c = col + HALO;
            real f[9], g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i] = S::load(st + i * SEGW + c - ex(i), (real)kp.base_f[i]);
                g[i] = S::load(st + (9 + i) * SEGW + c - ex(i), (real)kp.base_g[i]);
            }
            real rho = f[0];
#pragma unroll
            for (int i = 1; i < 9; ++i) rho += f[i];
            real Fx, Fy, ux, uy, T;
            force_from_rows<real, BMODE>(
                kp, rp + ((j - 2) & 3) * 32 + lane, rp + ((j - 1) & 3) * 32 + lane,
                rp + (j & 3) * 32 + lane, rq + ((j - 2) & 3) * 32 + lane,
                rq + ((j - 1) & 3) * 32 + lane, rq + (j & 3) * 32 + lane, Fx, Fy);
            collide<real, EQ24>(kp, f, g, rho, Fx, Fy, ux, uy, T);
            int y = y_start + j - 2;
            y = y >= ny ? y - ny : y;
            const uint32_t off = (uint32_t)y * pitch + (uint32_t)(x0 + col);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                S::put(dst + ((uint32_t)i * plane + off), f[i], (real)kp.base_f[i]);
                S::put(dst + ((uint32_t)(9 + i) * plane + off), g[i], (real)kp.base_g[i]);
            }
        }
        // 3. the stage of job j-1 has had its last reader in this warp
        __syncwarp();
        if (j >= 1 && lane == 0) mbar_arrive(&empty[(j - 1) % STAGES]);
    }
    if (abort) {
        if (lane == 0) atomicOr(kp.err, 1 << LB_ERR_TIMEOUT);
        return;
    }
    if (flags) atomicOr(kp.err, flags);
}

}  // namespace lbgb
