// lb_step_strip.cuh -- the fused step as a strip-marching kernel fed by TMA
// bulk copies (sm_90+ cp.async.bulk, mbarrier transaction counts).
//
// Each CTA owns a strip of BX columns and a chunk of rows and marches up the
// rows.  For every pre-collision row y it needs plane i of source row
// y - e_iy, columns [x0 - HALO, x0 + W + HALO) (HALO * sizeof(elem) = 16
// bytes, so every copy is 16-byte aligned); a producer warp streams these
// 18 row segments into a STAGES-deep shared-memory ring with cp.async.bulk,
// completion tracked by one mbarrier per stage.  The consumer warps then
//   1. compute rho, T and psi of row y for columns -1..W (one site of halo on
//      each side, computed by a separate halo warp so that no warp does two
//      sites) into a 4-row psi ring,
//   2. collide row y - 1 (Eq. (1) + F_i and Eq. (7)/(24)), whose three psi
//      rows are now complete, reading its populations back from the stage
//      ring and storing the 18 post-collision values with coalesced stores.
// psi is computed once per site (plus 2 columns per strip and 2 rows per
// chunk), and every population is read from HBM once and written once.
//
// Periodic wrap: rows wrap by index.  Columns wrap through ghost columns: the
// population buffers of a strip context keep STRIP_GHOST periodic copies of
// the first and last columns beside every row (kp.ghost; the layout leaves
// 128 bytes on each side), and this kernel writes them with the row, so the
// first and last strips fetch their halo with the same single copy as every
// other strip.  (Fetching the far end of the row with two extra 16-byte
// copies per plane row made the two edge strips the slowest CTAs of the
// launch.)  Any nx: each plane-row copy is rounded up to whole 16-byte units.
//
// A dedicated producer warp issues the copies; the column warps release a
// stage through a second mbarrier when its last reader is done, so copy issue
// never stalls the consumers' per-row synchronisation.
//
// Every mbarrier wait is bounded: on timeout the CTA records LB_ERR_TIMEOUT,
// the producer waits (again bounded, always with the default limit, so that no
// copy is still in flight when the CTA exits) for the copies it issued, and
// returns.  The limit of the pipeline waits is kp.wait_cycles.
#pragma once

#include "lb_device.cuh"
#include "lb_fd.cuh"

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

__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, "
        "p;\n}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait: false once `limit` clock cycles have passed (the default is
// about one second at GB300 clocks; a limit <= 0 means the default).  With
// the default the polls are try_wait, which may suspend the thread for a
// hardware-chosen time before it returns; a shorter, caller-set limit polls
// with the non-blocking test_wait, so that the limit alone decides.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit = WAIT_CYCLES_DEFAULT) {
    if (limit > 0 && limit < WAIT_CYCLES_DEFAULT) {
        const long long t0 = clock64();
        while (!mbar_test_wait(bar, parity)) {
            if (clock64() - t0 > limit) return false;
        }
        return true;
    }
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > WAIT_CYCLES_DEFAULT) return false;
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
        const real c = (BMODE == BETA_ONE) ? pc[0] : KPR(kp, beta) * pc[0];
        fx += c * s1x;
        fy += c * s1y;
    }
    if (BMODE != BETA_ONE) {
        const real E = qc[1], Wv = qc[-1], N = qn[0], S = qs[0];
        const real NE = qn[1], NW = qn[-1], SE = qs[1], SW = qs[-1];
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

template <int PREC>
struct StripCfg {
    using elem = typename Store<PREC>::elem;
    using real = typename Store<PREC>::real;
    static constexpr int ES = (int)sizeof(elem);
    static constexpr int HALO = 16 / ES;  // 16-byte halo: 2 (FP64), 4 (FP32), 8 (16-bit)
};

// Bytes of one plane-row copy of a strip W columns wide with its column halo,
// rounded up to the 16 bytes a bulk copy moves at a time (for any nx: the
// rounding reads at most HALO - 1 elements more, inside the row's right
// padding, which is never used).
template <int ES, int HALO>
__host__ __device__ constexpr uint32_t strip_copy_bytes(int W) {
    return ((uint32_t)((W + 2 * HALO) * ES) + 15u) & ~15u;
}

template <int PREC, int BX, int STAGES>
constexpr size_t strip_smem_bytes() {
    using C = StripCfg<PREC>;
    return (size_t)STAGES * Store<PREC>::NPLANES * (BX + 2 * C::HALO) * C::ES +
           (size_t)8 * (BX + 2) * sizeof(typename C::real) + (size_t)2 * STAGES * 8 + 16;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// named barrier over the column threads and the halo warp (the producer warp
// never joins)
template <int NT>
__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
}

// Threads per block of k_step_strip: BX column threads, one halo warp, one
// producer warp.
template <int BX>
__host__ __device__ constexpr int strip_threads() {
    return BX + 64;
}

// The producer warp of a strip kernel: for every job j (pre-collision row
// y_start - 1 + j) it waits until the job's stage is released, then lane 0
// arms the stage's "full" mbarrier with the byte count and lanes
// 0..NPLANES-1 each issue the copy of one plane-row segment (columns
// x0 - HALO .. x0 + W + HALO - 1, ghost columns at the lattice edges).  (One
// lane issuing all of them measured slower.)  On a
// timeout of the release wait it records LB_ERR_TIMEOUT and stops issuing
// (the consumers then time out on "full"); it returns only when every copy it
// issued has landed (bounded).
template <class S, int STAGES, int SEGW>
__device__ __forceinline__ void strip_produce(const typename S::elem* __restrict__ src, typename S::elem* stage,
                                              uint64_t* full, uint64_t* empty, const KParams& kp, int lane,
                                              int njobs, int y_start, int x0, int W) {
    using elem = typename S::elem;
    constexpr int ES = (int)sizeof(elem);
    constexpr int HALO = 16 / ES;
    constexpr int NPL = S::NPLANES;
    const int ny = kp.ny;
    const uint32_t plane = (uint32_t)kp.plane, pitch = (uint32_t)kp.pitch;
    const uint32_t cb = strip_copy_bytes<ES, HALO>(W);
    int issued = 0;
    for (int j = 0; j < njobs; ++j) {
        const int s = j % STAGES;
        if (j >= STAGES) {
            // the stage's previous job (j - STAGES) must have been released;
            // the warp takes one decision (its lanes poll the barrier independently)
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&empty[s], (uint32_t)(((j / STAGES) - 1) & 1),
                                                           kp.wait_cycles))) {
                if (lane == 0) atomicOr(kp.err, 1 << LB_ERR_TIMEOUT);
                break;
            }
        }
        int y = y_start - 1 + j;
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)NPL * cb);
        __syncwarp();
        if (lane < NPL) {
            const int i = lane;
            // direction of the plane (planes 18, 19: low halves of the rest populations)
            const int d = i < 9 ? i : (i < 18 ? i - 9 : 0);
            int sy = y - ey(d);
            sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
            const elem* row = src + (size_t)((uint32_t)i * plane + (uint32_t)sy * pitch);
            bulk_copy_g2s(stage + ((size_t)s * NPL + i) * SEGW, row + (x0 - HALO), cb, &full[s]);
        }
        issued = j + 1;
    }
    if (lane == 0)
        for (int j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j)
            (void)mbar_wait_bounded(&full[j % STAGES], (uint32_t)((j / STAGES) & 1));
}

// Block: BX column threads (BX/32 warps), one halo warp and one producer warp.
//   producer: for every job (pre-collision row) waits until its stage is
//     released, then lane 0 arms the stage's "full" mbarrier with the byte
//     count and lanes 0..NPLANES-1 each issue the copy of one plane-row segment.
//   column threads: wait "full", compute psi of their column of the row into
//     the psi ring, sync with the halo warp (named barrier), collide their
//     column of the row behind, then each warp releases the stage of the row
//     behind on its "empty" mbarrier.
//   halo warp: lanes 0 and 1 compute psi of the two halo columns (-1 and W),
//     so that no warp has two psi sites per row, then join the barrier.  It
//     reads a stage only before the barrier of that row, which the column
//     warps pass before they release the stage, so it does not release.
template <int PREC, int BX, int STAGES, bool EQ24, int BMODE>
__global__ void __launch_bounds__(strip_threads<BX>(), 2)
    k_step_strip(const typename Store<PREC>::elem* __restrict__ src,
                 typename Store<PREC>::elem* __restrict__ dst, const KParams kp, int nchunks) {
    using S = Store<PREC>;
    using C = StripCfg<PREC>;
    using elem = typename C::elem;
    using real = typename C::real;
    constexpr int HALO = C::HALO;
    constexpr int SEGW = BX + 2 * HALO;
    constexpr int RW = BX + 2;
    constexpr int ES = C::ES;
    constexpr int NCW = BX / 32;  // consumer warps
    constexpr int NPL = S::NPLANES;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    elem* stage = reinterpret_cast<elem*>(smem_raw);  // [STAGES][NPL][SEGW]
    real* ring_psi = reinterpret_cast<real*>(stage + (size_t)STAGES * NPL * SEGW);  // [4][RW]
    real* ring_psi2 = ring_psi + 4 * RW;                                            // [4][RW]
    uint64_t* full = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(ring_psi2 + 4 * RW) + 7) & ~uintptr_t(7));
    uint64_t* empty = full + STAGES;
    __shared__ int s_abort[2];  // one slot per job parity (see the loop)

    const int t = threadIdx.x;
    const int nx = kp.nx, ny = kp.ny;
    const int x0 = blockIdx.x * BX;
    const int W = min(BX, nx - x0);
    // rows updated: [H, ny - H) (H = kp.halo_rows: ghost rows of a y-decomposed
    // lattice; 0 on a periodic lattice, whose rows wrap)
    const int H = kp.halo_rows, nrows = ny - 2 * H;
    const int y_start = H + (int)((long long)blockIdx.y * nrows / nchunks);
    const int y_end = H + (int)((long long)(blockIdx.y + 1) * nrows / nchunks);
    const int njobs = (y_end - y_start) + 2;  // pre-collision rows y_start-1 .. y_end
    const uint32_t plane = (uint32_t)kp.plane, pitch = (uint32_t)kp.pitch;

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
        strip_produce<S, STAGES, SEGW>(src, stage, full, empty, kp, t - BX - 32, njobs, y_start, x0, W);
        return;
    }

    // ------------------------------------------ column threads and halo warp
    // ring column r holds strip column r - 1: column thread t owns r = t + 1,
    // halo lanes 0 and 1 own r = 0 and r = W + 1
    const bool halo = t >= BX;
    const int r_psi = halo ? ((t & 31) == 0 ? 0 : W + 1) : t + 1;
    const bool has_psi = halo ? (t & 31) < 2 : t < W;
    int flags = 0;
    bool aborted = false;
    for (int j = 0; j < njobs; ++j) {
        const int s = j % STAGES;
        if (!mbar_wait_bounded(&full[s], (uint32_t)((j / STAGES) & 1), kp.wait_cycles)) s_abort[j & 1] = 1;
        // 1. rho, T, psi of pre-collision row j at ring column r_psi
        if (has_psi) {
            const elem* st = stage + (size_t)s * NPL * SEGW;
            real* rp = ring_psi + (j & 3) * RW;
            real* rq = ring_psi2 + (j & 3) * RW;
            {
                const int r = r_psi;
                const int c = r - 1 + HALO;  // smem column of the site
                real rho, T, psi, psi2;
                if constexpr (S::SPLIT) {
                    // rho and the energy density from the sums of the stored deviations
                    float Hf = 0.0f, Hg = 0.0f;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        Hf += dev_of<S>(st + i * SEGW + c - ex(i), i, rest_lo_offset(i) * SEGW);
                        Hg += dev_of<S>(st + (9 + i) * SEGW + c - ex(i), 9 + i, rest_lo_offset(9 + i) * SEGW);
                    }
                    rho = kp.sum_bf + Hf;
                    T = (kp.sum_bg + Hg) / (rho * KPR(kp, cv));
                    site_psi_T<real, BMODE>(kp, rho, T, psi, psi2, flags);
                } else {
                    real f[9], g[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        f[i] = load_pop<S>(st + i * SEGW + c - ex(i), SEGW, i, (real)kp.base_f[i]);
                        g[i] = load_pop<S>(st + (9 + i) * SEGW + c - ex(i), SEGW, 9 + i, (real)kp.base_g[i]);
                    }
                    site_psi<real, BMODE>(kp, f, g, rho, T, psi, psi2, flags);
                }
                if (BMODE != BETA_ZERO) rp[r] = psi;
                if (BMODE != BETA_ONE) rq[r] = psi2;
            }
        }
        consumer_sync<BX + 32>();
        // (a thread that times out at job j + 1 writes the other slot than the
        // one read here, so every consumer leaves at the same job)
        if (s_abort[j & 1]) {
            aborted = true;
            break;
        }
        if (halo) continue;
        // 2. collide pre-collision row j-1 (its psi neighbourhood is complete)
        if (j >= 2 && t < W) {
            const int sp = (j - 1) % STAGES;
            const elem* st = stage + (size_t)sp * NPL * SEGW;
            const int c = t + HALO;
            const int r = t + 1;
            real Fx, Fy;
            force_from_rows<real, BMODE>(
                kp, ring_psi + ((j - 2) & 3) * RW + r, ring_psi + ((j - 1) & 3) * RW + r,
                ring_psi + (j & 3) * RW + r, ring_psi2 + ((j - 2) & 3) * RW + r,
                ring_psi2 + ((j - 1) & 3) * RW + r, ring_psi2 + (j & 3) * RW + r, Fx, Fy);
            int y = y_start + j - 2;
            y = y >= ny ? y - ny : y;
            const int xg = x0 + t;
            const uint32_t off = (uint32_t)y * pitch + (uint32_t)xg;
            if constexpr (S::SPLIT) {
                float h[9], q[9], Hf = 0.0f, Hg = 0.0f;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    h[i] = dev_of<S>(st + i * SEGW + c - ex(i), i, rest_lo_offset(i) * SEGW);
                    q[i] = dev_of<S>(st + (9 + i) * SEGW + c - ex(i), 9 + i, rest_lo_offset(9 + i) * SEGW);
                    Hf += h[i];
                    Hg += q[i];
                }
                collide_dev<EQ24>(kp, h, q, Hf, Hg, Fx, Fy);
                store_site_dev<S>(dst + off, plane, kp, h, q, Hf, Hg, xg < STRIP_GHOST, xg >= nx - STRIP_GHOST);
            } else {
                real f[9], g[9], Hf = (real)0, Hg = (real)0;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    f[i] = load_pop_acc<S>(st + i * SEGW + c - ex(i), SEGW, i, (real)kp.base_f[i], Hf);
                    g[i] = load_pop_acc<S>(st + (9 + i) * SEGW + c - ex(i), SEGW, 9 + i, (real)kp.base_g[i], Hg);
                }
                real rho = f[0];
#pragma unroll
                for (int i = 1; i < 9; ++i) rho += f[i];
                real ux, uy, T;
                collide<real, EQ24>(kp, f, g, rho, Fx, Fy, ux, uy, T);
                store_site<S>(dst + off, plane, kp, f, g, Hf, Hg, xg < STRIP_GHOST, xg >= nx - STRIP_GHOST);
            }
        }
        // 3. the stage of job j-1 has had its last reader (psi at j-1, collision at j)
        if (j >= 1) {
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

}  // namespace lbgb
