// lb_step_strip_dev.cuh -- the strip-marching step for the 16-bit deviation
// storage modes (FP16 / BF16 deviations, FP32 rest populations in two halves).
//
// The pipeline of k_step_strip (producer warp streaming plane-row segments
// into a stage ring, column threads computing psi into a ring of psi rows
// and colliding the rows whose psi neighbourhood is complete, halo warp for
// the two halo psi columns), changed where these modes, which are bound by
// instruction issue rather than by HBM bandwidth, spent instructions:
//   - two rows per iteration: psi of jobs 2k and 2k + 1, one barrier, then
//     the collisions of jobs 2k - 1 and 2k (their stencils share the psi rows
//     2k - 1 and 2k), so the per-row bookkeeping, waits and barrier are
//     paid once per two sites;
//   - the collided rows are written to shared-memory row buffers (job m
//     into buffer m mod 3, laid out [plane][column]) and leave the CTA as
//     one tensor copy each (cp.async.bulk.tensor.3d shared -> global through
//     the map of the destination buffer: x the column, y the row, z the
//     plane; the copy clips the columns past nx), so no thread forms twenty
//     64-bit store addresses per site; the periodic ghost copies of the edge
//     columns are stored by their threads directly.  Lane 0 of the halo warp
//     issues the copies (twenty per-plane bulk copies, whose operands are
//     uniform registers, made the issuing warp step through its lanes one by
//     one, which loaded its SM sub-partition more than the others): after
//     the barrier of iteration k it copies the row collided second in
//     iteration k - 1, then waits on an mbarrier on which the column warps
//     arrive once the first row of iteration k is written (and fenced for
//     the async proxy) and copies that one, and before the next barrier
//     waits until both copies have read their buffers (waiting for the
//     second row within the iteration put the halo warp, which also computes
//     two psi sites per iteration, last at every barrier; two buffers with an
//     mbarrier that frees the second before it is rewritten measured slower
//     than three);
//   - the deviation sums Hf, Hg of a site, formed when psi of its row is
//     computed, are kept in registers until the site collides (the same sums
//     in the same order, so the result does not change);
//   - stage, parity and ring indices advance incrementally.
//
// The abort flag has one slot per iteration parity: a thread that times out
// at iteration k + 1 writes the other slot than the one a slower thread
// still reads after the barrier of iteration k, so every consumer leaves the
// loop at the same iteration.
#pragma once

#include <cuda.h>

#include "lb_step_strip.cuh"

namespace lbgb {

constexpr int DEV_OUT_BUFS = 3;  // row buffers: job m collides into buffer m mod 3

// 3D tensor copy shared -> global of the box at (x, y, z) (bulk async group
// of the issuing thread)
__device__ __forceinline__ void tensor_store_3d(const CUtensorMap* map, const void* ssrc, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(ssrc)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit_group() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// wait until at most N of this thread's bulk groups still read shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_group_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// wait until every bulk group of this thread has completed
__device__ __forceinline__ void bulk_wait_group_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// psi rows held by the ring: the four rows two collisions read plus the two
// rows a thread one iteration ahead writes
constexpr int DEV_PSI_ROWS = 6;

template <int PREC, int BX, int STAGES>
constexpr size_t strip_dev_smem_bytes() {
    using C = StripCfg<PREC>;
    constexpr int NPL = Store<PREC>::NPLANES;
    return (size_t)STAGES * NPL * (BX + 2 * C::HALO) * C::ES + (size_t)DEV_OUT_BUFS * NPL * BX * C::ES +
           (size_t)2 * DEV_PSI_ROWS * (BX + 2) * sizeof(float) + (size_t)(2 * STAGES + 1) * 8 + 16;
}

// rho, T and psi (Eq. 3 / 4) of one site from its pulled deviations in a
// stage (smem column c), with the deviation sums kept for its collision
template <class S, int SEGW, int BMODE>
__device__ __forceinline__ void dev_psi_site(const KParams& kp, const typename S::elem* st, int c, float& Hf,
                                             float& Hg, float* rp, float* rq, int& flags) {
    float hf = 0.0f, hg = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        hf = acc_dev<S>(st + i * SEGW + c - ex(i), i, rest_lo_offset(i) * SEGW, hf);
        hg = acc_dev<S>(st + (9 + i) * SEGW + c - ex(i), 9 + i, rest_lo_offset(9 + i) * SEGW, hg);
    }
    const float rho = kp.sum_bf + hf;
    const float T = (kp.sum_bg + hg) / (rho * kp.f.cv);
    float psi, psi2;
    site_psi_T<float, BMODE>(kp, rho, T, psi, psi2, flags);
    if (BMODE != BETA_ZERO) *rp = psi;
    if (BMODE != BETA_ONE) *rq = psi2;
    Hf = hf;
    Hg = hg;
}

// Eq. (1) + F_i and Eq. (7) / (24) for one site: its stored form into row
// buffer column o (fenced for the tensor copy), the ghost copies of an edge
// column straight to its planes at d.
template <class S, int SEGW, int BX, bool EQ24>
__device__ __forceinline__ void dev_collide_site(const KParams& kp, const typename S::elem* st, int c, float Hf,
                                                 float Hg, float Fx, float Fy, typename S::elem* d,
                                                 typename S::elem* o, uint32_t plane, bool ghost_lo,
                                                 bool ghost_hi) {
    constexpr int NPL = S::NPLANES;
    float h[9], q[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        h[i] = dev_of<S>(st + i * SEGW + c - ex(i), i, rest_lo_offset(i) * SEGW);
        q[i] = dev_of<S>(st + (9 + i) * SEGW + c - ex(i), 9 + i, rest_lo_offset(9 + i) * SEGW);
    }
    collide_dev<EQ24>(kp, h, q, Hf, Hg, Fx, Fy);
    typename S::elem v[NPL];
    encode_site_dev<S>(h, q, Hf, Hg, v);
#pragma unroll
    for (int p = 0; p < NPL; ++p) o[p * BX] = v[p];
    fence_proxy_async_smem();
    put_ghost_copies<S>(d, plane, kp.nx, v, ghost_lo, ghost_hi);
}

template <int PREC, int BX, int STAGES, bool EQ24, int BMODE>
__global__ void __launch_bounds__(strip_threads<BX>(), 2)
    k_step_strip_dev(const typename Store<PREC>::elem* __restrict__ src,
                     typename Store<PREC>::elem* __restrict__ dst, const KParams kp, int nchunks,
                     const __grid_constant__ CUtensorMap dst_map) {
    using S = Store<PREC>;
    static_assert(S::SPLIT, "16-bit deviation storage only");
    using C = StripCfg<PREC>;
    using elem = typename C::elem;
    using real = float;  // (KPR reads the float copies of the parameters)
    constexpr int HALO = C::HALO;
    constexpr int SEGW = BX + 2 * HALO;
    constexpr int RW = BX + 2;
    constexpr int NPL = S::NPLANES;
    constexpr int ES = C::ES;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    elem* stage = reinterpret_cast<elem*>(smem_raw);                 // [STAGES][NPL][SEGW]
    elem* outb = stage + (size_t)STAGES * NPL * SEGW;                 // [DEV_OUT_BUFS][NPL][BX]
    float* ring_psi = reinterpret_cast<float*>(outb + (size_t)DEV_OUT_BUFS * NPL * BX);  // [6][RW]
    float* ring_psi2 = ring_psi + DEV_PSI_ROWS * RW;                                     // [6][RW]
    uint64_t* full = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(ring_psi2 + DEV_PSI_ROWS * RW) + 7) & ~uintptr_t(7));
    uint64_t* empty = full + STAGES;
    uint64_t* written = empty + STAGES;  // the first row collided in an iteration is complete
    __shared__ int s_abort[2];

    const int t = threadIdx.x;
    const int nx = kp.nx, ny = kp.ny;
    const int x0 = blockIdx.x * BX;
    const int W = min(BX, nx - x0);
    // rows updated: [H, ny - H) (H = kp.halo_rows; 0 on a periodic lattice)
    const int H = kp.halo_rows, nrows = ny - 2 * H;
    const int y_start = H + (int)((long long)blockIdx.y * nrows / nchunks);
    const int y_end = H + (int)((long long)(blockIdx.y + 1) * nrows / nchunks);
    // jobs: pre-collision rows y_start - 1 + j, j = 0 .. njobs - 1; jobs
    // 1 .. njobs - 2 (rows y_start .. y_end - 1) collide
    const int njobs = (y_end - y_start) + 2;

    if (t == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], BX / 32);
        }
        mbar_init(written, BX / 32);
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
    const uint32_t plane = (uint32_t)kp.plane, pitch = (uint32_t)kp.pitch;
    const bool halo = t >= BX;
    const int lane = t & 31;
    // ring column r holds strip column r - 1: column thread t owns r = t + 1,
    // halo lanes 0 and 1 own r = 0 and r = W + 1 (for both jobs: splitting
    // the four halo sites over lanes 0..3 measured slower)
    const int r_psi = halo ? (lane == 0 ? 0 : W + 1) : t + 1;
    const bool has_psi = halo ? lane < 2 : t < W;
    const int c_psi = r_psi - 1 + HALO;   // smem column of the psi site
    const bool issuer = halo && lane == 0;  // copies the collided rows out
    const int xg = x0 + t;
    const bool ghost_lo = xg < STRIP_GHOST, ghost_hi = xg >= nx - STRIP_GHOST;
    const int c = t + HALO;               // smem column of the collided site
    int flags = 0;
    float Hf_p = 0.0f, Hg_p = 0.0f;       // deviation sums of job 2k - 1 (from the iteration before)
    int s0 = 0;                           // stage of job 2k
    uint32_t ph0 = 0;                     // its "full" parity
    int sm = STAGES - 1;                  // stage of job 2k - 1
    int q = 0;                            // psi ring row of job 2k: 2k mod 6
    int b0 = 0;                           // row buffer of job 2k: 2k mod 3
    const int iters = (njobs + 1) / 2;
    bool aborted = false;
    for (int k = 0; k < iters; ++k) {
        const int j0 = 2 * k;
        const bool has1 = j0 + 1 < njobs;
        const int s1 = s0 + 1 == STAGES ? 0 : s0 + 1;
        const uint32_t ph1 = s0 + 1 == STAGES ? ph0 ^ 1u : ph0;
        // 1. psi of jobs 2k and 2k + 1
        bool ok = mbar_wait_bounded(&full[s0], ph0, kp.wait_cycles);
        if (ok && has1) ok = mbar_wait_bounded(&full[s1], ph1, kp.wait_cycles);
        if (!ok) s_abort[k & 1] = 1;
        float Hf_0 = 0.0f, Hg_0 = 0.0f, Hf_1 = 0.0f, Hg_1 = 0.0f;
        if (has_psi && ok) {
            dev_psi_site<S, SEGW, BMODE>(kp, stage + s0 * (NPL * SEGW), c_psi, Hf_0, Hg_0,
                                         ring_psi + q * RW + r_psi, ring_psi2 + q * RW + r_psi, flags);
            if (has1)
                dev_psi_site<S, SEGW, BMODE>(kp, stage + s1 * (NPL * SEGW), c_psi, Hf_1, Hg_1,
                                             ring_psi + (q + 1) * RW + r_psi, ring_psi2 + (q + 1) * RW + r_psi,
                                             flags);
        }
        consumer_sync<BX + 32>();
        if (s_abort[k & 1]) {
            aborted = true;
            break;
        }
        // 2. collide jobs 2k - 1 (into row buffer X) and 2k (into Y)
        const int m0 = j0 - 1, m1 = j0;
        const bool c0 = m0 >= 1 && m0 <= njobs - 2, c1 = m1 >= 1 && m1 <= njobs - 2;
        const int bA = b0 == 0 ? DEV_OUT_BUFS - 1 : b0 - 1;  // row buffer of job 2k - 1
        if (halo) {
            // the row collided second in the iteration before is complete
            // since the barrier (its writers fenced before arriving)
            const int mp = j0 - 2;
            if (issuer && k >= 1 && mp >= 1 && mp <= njobs - 2) {
                const int bP = b0 + 1 == DEV_OUT_BUFS ? 0 : b0 + 1;  // (2k - 2) mod 3
                tensor_store_3d(&dst_map, outb + (size_t)bP * NPL * BX, x0, y_start - 1 + mp, 0);
                bulk_commit_group();
            }
            // the first row of this iteration, once every column warp has written it
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(written, (uint32_t)(k & 1), kp.wait_cycles))) {
                s_abort[(k + 1) & 1] = 1;  // every consumer leaves after the next barrier
            } else if (issuer && c0) {
                tensor_store_3d(&dst_map, outb + (size_t)bA * NPL * BX, x0, y_start - 1 + m0, 0);
                bulk_commit_group();
            }
            // both buffers copied here are written again from the next iteration on
            if (issuer) bulk_wait_group_read<0>();
        } else {
            const int qm2 = q == 0 ? DEV_PSI_ROWS - 2 : q - 2;  // ring row of job 2k - 2
            const int qm1 = qm2 + 1;                            // of job 2k - 1
            const int r = t + 1;
            if (t < W && (c0 || c1)) {
                // the stencils of both collisions (rows 2k-2 .. 2k and 2k-1 .. 2k+1)
                float FxA, FyA, FxB, FyB;
                force_from_rows<float, BMODE>(
                    kp, ring_psi + qm2 * RW + r, ring_psi + qm1 * RW + r, ring_psi + q * RW + r,
                    ring_psi2 + qm2 * RW + r, ring_psi2 + qm1 * RW + r, ring_psi2 + q * RW + r, FxA, FyA);
                force_from_rows<float, BMODE>(
                    kp, ring_psi + qm1 * RW + r, ring_psi + q * RW + r, ring_psi + (q + 1) * RW + r,
                    ring_psi2 + qm1 * RW + r, ring_psi2 + q * RW + r, ring_psi2 + (q + 1) * RW + r, FxB, FyB);
                if (c0) {
                    const int y = y_start - 1 + m0;
                    dev_collide_site<S, SEGW, BX, EQ24>(kp, stage + sm * (NPL * SEGW), c, Hf_p, Hg_p, FxA, FyA,
                                                        dst + ((size_t)y * pitch + (size_t)xg),
                                                        outb + (size_t)bA * NPL * BX + t, plane,
                                                        ghost_lo, ghost_hi);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(written);
                if (c1) {
                    const int y = y_start - 1 + m1;
                    dev_collide_site<S, SEGW, BX, EQ24>(kp, stage + s0 * (NPL * SEGW), c, Hf_0, Hg_0, FxB, FyB,
                                                        dst + ((size_t)y * pitch + (size_t)xg),
                                                        outb + (size_t)b0 * NPL * BX + t, plane,
                                                        ghost_lo, ghost_hi);
                }
            } else {
                __syncwarp();
                if (lane == 0) mbar_arrive(written);
            }
            __syncwarp();
            if (lane == 0) {
                // 3. the stages of jobs 2k - 1 and 2k have had their last readers
                if (k >= 1) mbar_arrive(&empty[sm]);
                mbar_arrive(&empty[s0]);
            }
        }
        Hf_p = Hf_1;
        Hg_p = Hg_1;
        sm = s1;
        s0 = s1 + 1 == STAGES ? 0 : s1 + 1;
        ph0 = s1 + 1 == STAGES ? ph1 ^ 1u : ph1;
        q = q + 2 == DEV_PSI_ROWS ? 0 : q + 2;
        b0 = b0 + 2 >= DEV_OUT_BUFS ? b0 + 2 - DEV_OUT_BUFS : b0 + 2;
    }
    if (!aborted) {
        // the row collided second in the last iteration
        consumer_sync<BX + 32>();
        const int mp = 2 * iters - 2;
        if (issuer && mp >= 1 && mp <= njobs - 2) {
            const int bP = b0 + 1 == DEV_OUT_BUFS ? 0 : b0 + 1;  // mp mod 3
            tensor_store_3d(&dst_map, outb + (size_t)bP * NPL * BX, x0, y_start - 1 + mp, 0);
            bulk_commit_group();
        }
    }
    // no copy may still read shared memory or be unwritten when the CTA exits
    if (issuer) bulk_wait_group_all();
    if (aborted) {
        if (t == 0) atomicOr(kp.err, 1 << LB_ERR_TIMEOUT);
        return;
    }
    if (flags) atomicOr(kp.err, flags);
}

}  // namespace lbgb
