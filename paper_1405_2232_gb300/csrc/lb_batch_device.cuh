// lb_batch_device.cuh -- device code of the batched solver: many independent
// periodic domains of different sizes and parameters advanced together.
//
// The fused step is the strip-marching kernel of lb_step_strip.cuh made
// persistent: a fixed grid of CTAs walks a device-side list of work items
// (domain, strip, row chunk) sorted longest first; CTA b starts with item b
// and its producer warp takes every further item from a global counter, so
// the CTAs finish together (a static deal by estimated cost left the last CTA
// 14% behind the mean).  The producer passes each item's index to the consumer
// warps through a small shared-memory queue (written before it arms the
// item's first stage, read after that stage's barrier), and after the last
// item an end mark: a stage completed without data whose queue entry is -1.
// The producer and the consumers keep one job counter across items, so the
// producer streams the next item's rows while the consumers still work on
// the current one.  The list and its length are read from device memory at
// launch.  A launch over n items and G CTAs takes from the counter exactly
// max(0, n - G) + min(G, n) times (every further item, and one failed take
// per CTA that had an item), so the take that returns the last of those
// values resets the counter for the next launch: a captured CUDA graph
// replays the step with no reset node, CTAs without an item touch no atomic,
// and the graph stays valid while converged domains are taken off the list.
//
// Half items: a strip at most BX/2 columns wide (a narrow domain, or the
// remainder strip of a wider one) would leave most column threads idle, so
// its rows are split between the two halves of the CTA, which march them in
// lockstep: column threads [0, BX/2) take rows [y0, ym) and [BX/2, BX) rows
// [ym, y1).  The stage and psi-ring rows hold one segment per half, the
// producer copies both halves' plane rows for a job, the halo warp's lanes
// 0, 1 and 2, 3 compute the halo psi columns of the two halves; when the
// right half has one row fewer it sits out the left half's last job.
//
// As in the single-lattice kernel, every domain is stored in the ghost-column
// layout (one bulk copy per plane row, ghost copies written with the row) and
// a halo warp computes the halo psi columns.
#pragma once

#include "lb_step_strip.cuh"

namespace lbgb {

// Item indices the producer may run ahead of the consumers (it is at most
// STAGES jobs ahead, and every item has at least three jobs).
constexpr int BATCH_QN = 16;

// One domain of a batch.
struct BatchDomain {
    KParams kp;          // physics, sizes, pitch/plane (elements) and error word
    long long off;       // element offset of the domain's 18 planes in each buffer
    long long fld_off;   // site offset of the domain in the dense field arrays
};

// One work item of the persistent step kernel.
struct BatchItem {
    int domain;
    int strip;    // column strip (width BX)
    int y0, y1;   // rows [y0, y1) collided by this item
    int half;     // 1: strip at most BX/2 wide, rows split between the CTA's halves
};

// Rows of the left half of a half item: [y0, batch_split(y0, y1)).
__host__ __device__ inline int batch_split(int y0, int y1) { return y0 + (y1 - y0 + 1) / 2; }

// Row pitches of the batched step's stage and psi ring: room for one full
// strip (BX + 2 HALO, BX + 2) or two half strips (2 (BX/2 + 2 HALO), 2 (BX/2 + 2)).
template <int PREC, int BX>
__host__ __device__ constexpr int batch_segw() {
    return BX + 4 * StripCfg<PREC>::HALO;
}
template <int BX>
__host__ __device__ constexpr int batch_rw() {
    return BX + 4;
}

// Stage count of the batched step: the deepest ring that lets two CTAs share an SM.
template <int PREC, int BX>
constexpr int batch_stages() {
    constexpr size_t stage = (size_t)18 * batch_segw<PREC, BX>() * StripCfg<PREC>::ES;
    constexpr size_t ring = (size_t)8 * batch_rw<BX>() * sizeof(typename StripCfg<PREC>::real);
    constexpr size_t s = (110 * 1024 - 32 - ring) / stage;
    return s > 12 ? 12 : (int)s;
}
template <int PREC, int BX, int STAGES>
constexpr size_t batch_smem_bytes() {
    return (size_t)STAGES * 18 * batch_segw<PREC, BX>() * StripCfg<PREC>::ES +
           (size_t)8 * batch_rw<BX>() * sizeof(typename StripCfg<PREC>::real) + (size_t)2 * STAGES * 8 + 16;
}

template <int PREC, int BX, int STAGES, bool EQ24, int BMODE>
__global__ void __launch_bounds__(strip_threads<BX>(), 2)
    k_batch_step(const typename Store<PREC>::elem* __restrict__ src_base,
                 typename Store<PREC>::elem* __restrict__ dst_base,
                 const BatchDomain* __restrict__ doms, const BatchItem* __restrict__ items,
                 const int* __restrict__ n_items_ptr, int* __restrict__ next_item) {
    // next_item[0]: takes from the counter so far (item G + value)
    using S = Store<PREC>;
    using C = StripCfg<PREC>;
    using elem = typename C::elem;
    using real = typename C::real;
    constexpr int HALO = C::HALO;
    constexpr int SEGW = batch_segw<PREC, BX>();  // stage row pitch
    constexpr int RW = batch_rw<BX>();            // psi ring row pitch
    constexpr int HW = BX / 2;                    // columns of a half strip
    constexpr int SEGW2 = HW + 2 * HALO;          // stage offset of the right half
    constexpr int RW2 = HW + 2;                   // ring offset of the right half
    constexpr int ES = C::ES;
    constexpr int NCW = BX / 32;
    static_assert(HW % 32 == 0, "a half strip is whole warps");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    elem* stage = reinterpret_cast<elem*>(smem_raw);  // [STAGES][18][SEGW]
    real* ring_psi = reinterpret_cast<real*>(stage + (size_t)STAGES * 18 * SEGW);  // [4][RW]
    real* ring_psi2 = ring_psi + 4 * RW;                                            // [4][RW]
    uint64_t* full = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(ring_psi2 + 4 * RW) + 7) & ~uintptr_t(7));
    uint64_t* empty = full + STAGES;
    __shared__ int s_abort[2];  // one slot per job parity (see the loop)
    __shared__ int s_items[BATCH_QN];  // item index of the q-th item this CTA took (-1: no more)

    const int t = threadIdx.x;
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
        const int n_items = *n_items_ptr;
        long long jg = 0;  // job counter across this CTA's items
        int q = 0;         // items taken
        bool timed_out = false;
        const int G = (int)gridDim.x;
        const int takes = max(0, n_items - G) + min(G, n_items);
        for (;; ++q) {
            int it = (int)blockIdx.x;  // the first item: no counter
            if (q > 0) {
                int x = 0;
                if (lane == 0) {
                    x = atomicAdd(next_item, 1);
                    if (x == takes - 1) *next_item = 0;  // the launch's last take
                }
                it = G + __shfl_sync(0xffffffffu, x, 0);
            }
            if (it >= n_items) break;
            const BatchItem item = items[it];
            const BatchDomain& D = doms[item.domain];
            const int nx = D.kp.nx, ny = D.kp.ny;
            const uint32_t plane = (uint32_t)D.kp.plane, pitch = (uint32_t)D.kp.pitch;
            const int x0 = item.strip * BX;
            const int W = min(BX, nx - x0);
            // a half item: the left half's rows set the job count, the right
            // half (rows from ym) has as many or one fewer
            const int ym = item.half ? batch_split(item.y0, item.y1) : item.y1;
            const int njobs = ym - item.y0 + 2;
            const int njobs1 = item.half ? item.y1 - ym + 2 : 0;
            const elem* src = src_base + D.off;
            const uint32_t cb = strip_copy_bytes<ES, HALO>(W);
            for (int j = 0; j < njobs; ++j, ++jg) {
                const int s = (int)(jg % STAGES);
                if (jg >= STAGES) {
                    // the warp takes one decision (its lanes poll the barrier independently)
                    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&empty[s], (uint32_t)(((jg / STAGES) - 1) & 1)))) {
                        if (lane == 0) atomicOr(D.kp.err, 1 << LB_ERR_TIMEOUT);
                        timed_out = true;  // consumers then time out on "full" and leave
                        break;
                    }
                }
                const bool two = j < njobs1;  // the right half of a half item has this job
                if (lane == 0) {
                    // the item's index, published by the arrive below
                    if (j == 0) s_items[q % BATCH_QN] = it;
                    mbar_arrive_expect_tx(&full[s], (uint32_t)(two ? 36 : 18) * cb);
                }
                __syncwarp();
                if (lane < 18) {
                    const int i = lane;
                    const int d = i < 9 ? i : i - 9;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h == 1 && !two) break;
                        int sy = (h == 0 ? item.y0 : ym) - 1 + j - ey(d);
                        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                        const elem* row = src + (size_t)((uint32_t)i * plane + (uint32_t)sy * pitch);
                        // columns x0 - HALO .. x0 + W + HALO - 1 (ghost columns at the edges)
                        bulk_copy_g2s(stage + ((size_t)s * 18 + i) * SEGW + h * SEGW2, row + (x0 - HALO), cb,
                                      &full[s]);
                    }
                }
            }
            if (timed_out) break;
        }
        // every copy this CTA issued has landed (bounded) before the end mark
        // completes the next phase of a stage's barrier, and before the CTA exits
        if (lane == 0)
            for (long long j = (jg > STAGES ? jg - STAGES : 0); j < jg; ++j)
                (void)mbar_wait_bounded(&full[j % STAGES], (uint32_t)((j / STAGES) & 1));
        __syncwarp();
        // the end mark: the next stage completes without data, its queue entry -1
        const int s = (int)(jg % STAGES);
        if (!timed_out && jg >= STAGES &&
            !__all_sync(0xffffffffu, mbar_wait_bounded(&empty[s], (uint32_t)(((jg / STAGES) - 1) & 1)))) {
            if (lane == 0) atomicOr(doms[0].kp.err, 1 << LB_ERR_TIMEOUT);
            timed_out = true;  // consumers then time out on "full" and leave
        }
        if (lane == 0 && !timed_out) {
            s_items[q % BATCH_QN] = -1;
            mbar_arrive(&full[s]);
        }
        return;
    }

    // ------------------------------------------ column threads and halo warp
    // (ring column r holds strip column r - 1; see k_step_strip)
    const bool halo = t >= BX;
    long long jg = 0;
    bool aborted = false;
    for (int q = 0;; ++q) {
        // the first stage of the q-th item this CTA's producer took (or its
        // end mark); one barrier so that every consumer reads the same entry
        // and abort flag
        if (!mbar_wait_bounded(&full[(int)(jg % STAGES)], (uint32_t)((jg / STAGES) & 1))) s_abort[jg & 1] = 1;
        consumer_sync<BX + 32>();
        if (s_abort[jg & 1]) {
            aborted = true;
            break;
        }
        const int it = s_items[q % BATCH_QN];
        if (it < 0) break;
        const BatchItem item = items[it];
        const BatchDomain& D = doms[item.domain];
        const KParams kp = D.kp;
        const int nx = kp.nx, ny = kp.ny;
        const uint32_t plane = (uint32_t)kp.plane, pitch = (uint32_t)kp.pitch;
        const int x0 = item.strip * BX;
        const int W = min(BX, nx - x0);
        // this thread's half: h = 1 for the right half of a half item (column
        // threads from BX/2, halo lanes 2 and 3); its rows start at yh, its
        // stage and ring segments at soff, roff, its column in the strip is tl
        const int ym = item.half ? batch_split(item.y0, item.y1) : item.y1;
        const int njobs = ym - item.y0 + 2;
        const int lane = t & 31;
        const int h = item.half ? (halo ? (lane >> 1) & 1 : (t >= HW ? 1 : 0)) : 0;
        const int tl = t - h * HW;
        const int yh = h ? ym : item.y0;
        const int njobs_h = h ? item.y1 - ym + 2 : njobs;
        const int soff = h * SEGW2, roff = h * RW2;
        elem* dst = dst_base + D.off;
        const int r_psi = halo ? ((lane & 1) == 0 ? 0 : W + 1) : tl + 1;
        const bool has_psi = halo ? lane < (item.half ? 4 : 2) : tl < W;
        int flags = 0;
        for (int j = 0; j < njobs; ++j, ++jg) {
            const int s = (int)(jg % STAGES);
            // (the first job's stage was waited for above)
            if (j > 0 && !mbar_wait_bounded(&full[s], (uint32_t)((jg / STAGES) & 1))) s_abort[jg & 1] = 1;
            if (has_psi && j < njobs_h) {
                const elem* st = stage + (size_t)s * 18 * SEGW + soff;
                real* rp = ring_psi + (int)(jg & 3) * RW + roff;
                real* rq = ring_psi2 + (int)(jg & 3) * RW + roff;
                {
                    const int r = r_psi;
                    const int c = r - 1 + HALO;
                    real f[9], g[9], rho, T, psi, psi2;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        f[i] = S::load(st + i * SEGW + c - ex(i), (real)kp.base_f[i]);
                        g[i] = S::load(st + (9 + i) * SEGW + c - ex(i), (real)kp.base_g[i]);
                    }
                    site_psi<real, BMODE>(kp, f, g, rho, T, psi, psi2, flags);
                    if (BMODE != BETA_ZERO) rp[r] = psi;
                    if (BMODE != BETA_ONE) rq[r] = psi2;
                }
            }
            consumer_sync<BX + 32>();
            // (a thread that times out at the next job writes the other slot
            // than the one read here, so every consumer leaves at the same job)
            if (s_abort[jg & 1]) {
                aborted = true;
                break;
            }
            if (halo) continue;
            if (j >= 2 && j < njobs_h && tl < W) {
                const int sp = (int)((jg - 1) % STAGES);
                const elem* st = stage + (size_t)sp * 18 * SEGW + soff;
                const int c = tl + HALO;
                real f[9], g[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    f[i] = S::load(st + i * SEGW + c - ex(i), (real)kp.base_f[i]);
                    g[i] = S::load(st + (9 + i) * SEGW + c - ex(i), (real)kp.base_g[i]);
                }
                real rho = f[0];
#pragma unroll
                for (int i = 1; i < 9; ++i) rho += f[i];
                const int r = roff + tl + 1;
                real Fx, Fy, ux, uy, T;
                force_from_rows<real, BMODE>(
                    kp, ring_psi + (int)((jg - 2) & 3) * RW + r, ring_psi + (int)((jg - 1) & 3) * RW + r,
                    ring_psi + (int)(jg & 3) * RW + r, ring_psi2 + (int)((jg - 2) & 3) * RW + r,
                    ring_psi2 + (int)((jg - 1) & 3) * RW + r, ring_psi2 + (int)(jg & 3) * RW + r, Fx, Fy);
                collide<real, EQ24>(kp, f, g, rho, Fx, Fy, ux, uy, T);
                const int y = yh + j - 2;
                const int xg = x0 + tl;
                const uint32_t off = (uint32_t)y * pitch + (uint32_t)xg;
                // FP32 / FP64 storage, the values as computed; each plane's ghost
                // copy right after its value (the one-branch-per-site form of
                // store_site keeps all 18 values live past the main stores, which
                // spills at this kernel's register budget of 2 CTAs per SM)
                const bool ghost_lo = xg < STRIP_GHOST, ghost_hi = xg >= nx - STRIP_GHOST;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    elem* pf = dst + ((uint32_t)i * plane + off);
                    elem* pg = dst + ((uint32_t)(9 + i) * plane + off);
                    *pf = (elem)f[i];
                    *pg = (elem)g[i];
                    if (ghost_lo) {
                        pf[nx] = (elem)f[i];
                        pg[nx] = (elem)g[i];
                    }
                    if (ghost_hi) {
                        pf[-nx] = (elem)f[i];
                        pg[-nx] = (elem)g[i];
                    }
                }
            }
            // the job before this one has had its last reader in this warp
            if (j >= 1) {
                __syncwarp();
                if ((t & 31) == 0) mbar_arrive(&empty[(int)((jg - 1) % STAGES)]);
            }
        }
        if (aborted) break;
        // the item's last job (a halo row, never collided) is released too, so
        // the producer may reuse its stage for the next item (column warps
        // only: the halo warp never releases)
        __syncwarp();
        if (!halo && (t & 31) == 0) mbar_arrive(&empty[(int)((jg - 1) % STAGES)]);
        if (flags) atomicOr(kp.err, flags);
    }
    if (aborted && t == 0) atomicOr(doms[0].kp.err, 1 << LB_ERR_TIMEOUT);
}

// Per-domain partial sums over tiles of 256 sites: rho, rho c_v T (sum g),
// |d rho|^2, rho^2, |dT|^2, T^2 against the reference fields, and the new
// reference fields are written.  One CTA per (domain, tile) item.
struct BatchTile {
    int domain;
    int first;   // first site (row-major) of the tile in the domain
};

template <int PREC>
__global__ void __launch_bounds__(256)
    k_batch_check(const typename Store<PREC>::elem* __restrict__ src_base,
                  const BatchDomain* __restrict__ doms, const BatchTile* __restrict__ tiles,
                  const int* __restrict__ n_tiles_ptr, double* __restrict__ ref_rho,
                  double* __restrict__ ref_T, int have_ref, double* __restrict__ part) {
    using S = Store<PREC>;
    using real = typename S::real;
    __shared__ double s_red[8][6];
    const int b = blockIdx.x;
    if (b >= *n_tiles_ptr) return;  // the grid covers the longest list
    const BatchTile tile = tiles[b];
    const BatchDomain& D = doms[tile.domain];
    const KParams& kp = D.kp;
    const int n = kp.nx * kp.ny;
    const int s = tile.first + (int)threadIdx.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (s < n) {
        const int x = s % kp.nx, y = s / kp.nx;
        real f[9], g[9];
        pull18<S>(src_base + D.off, kp, x, y, f, g);
        real rho = f[0], e = g[0];
        double m = (double)f[0], en = (double)g[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            rho += f[i];
            e += g[i];
            m += (double)f[i];
            en += (double)g[i];
        }
        const double r = (double)rho, T = (double)(e / (rho * KPR(kp, cv)));
        const long long fo = D.fld_off + s;
        v[0] = m;
        v[1] = en;
        if (have_ref) {
            const double a = r - ref_rho[fo], c = T - ref_T[fo];
            v[2] = a * a;
            v[4] = c * c;
        }
        v[3] = r * r;
        v[5] = T * T;
        ref_rho[fo] = r;
        ref_T[fo] = T;
        if (!isfinite(r) || !isfinite(T)) atomicOr(kp.err, 1 << LB_ERR_NONFINITE);
    }
    const int tid = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((tid & 31) == 0) s_red[tid >> 5][k] = x;
    }
    __syncthreads();
    if (tid < 6) {
        double x = 0.0;
        for (int w = 0; w < 8; ++w) x += s_red[w][tid];
        part[(long long)b * 6 + tid] = x;
    }
}

// Folds each domain's tile partials (contiguous, in order) into its totals.
static __global__ void k_batch_fold(const double* __restrict__ part, const int* __restrict__ tile_begin,
                             int n_domains, double* __restrict__ out6) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n_domains) return;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = tile_begin[d]; b < tile_begin[d + 1]; ++b)
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] += part[(long long)b * 6 + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) out6[(long long)d * 6 + k] = acc[k];
}

}  // namespace lbgb
