// lb_step_strip_dev.cuh -- the strip-marching step for the 16-bit deviation
// storage modes (FP16 / BF16 deviations, FP32 rest populations in two halves).
//
// The same pipeline as k_step_strip (producer warp streaming plane-row
// segments into a stage ring, column threads computing psi of row y into a
// 4-row ring and colliding row y - 1, halo warp for the two halo psi columns),
// with three changes that cut the per-site instruction count of these modes,
// which are bound by instruction issue rather than by HBM bandwidth:
//   - the collided row is written to a shared-memory row buffer and leaves
//     the CTA as one bulk copy per plane row (cp.async.bulk shared -> global),
//     so no thread forms twenty 64-bit store addresses per site; columns past
//     the last whole 16-byte unit of the strip and the periodic ghost copies
//     of the edge columns are stored by their threads directly.  Lanes
//     0..NPLANES-1 of the halo warp issue the copies while the column warps
//     collide the next row: a copy's operands are uniform registers, so a
//     warp issuing twenty of them steps through its lanes one by one, which
//     in a column warp delayed every row's barrier (one lane issuing all
//     twenty measured slower still);
//   - the deviation sums Hf, Hg of a site, formed when psi of its row is
//     computed, are kept in registers until the site collides one row later
//     (the same sums in the same order, so the result does not change);
//   - stage, parity and row-buffer indices advance incrementally.
// DEV_OUT_BUFS row buffers rotate; before a buffer is written again, the
// lanes that copied it out wait for their copies to finish reading it (two
// buffers and seven stages measured as fast as three buffers and six stages
// at a 256-column strip).
//
// The abort flag has one slot per job parity: a thread that times out at job
// j + 1 writes the other slot than the one a slower thread still reads after
// the barrier of job j, so every consumer leaves the loop at the same job.
#pragma once

#include "lb_step_strip.cuh"

namespace lbgb {

constexpr int DEV_OUT_BUFS = 2;

__device__ __forceinline__ void bulk_copy_s2g(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_u32(ssrc)), "r"(bytes)
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

template <int PREC, int BX, int STAGES>
constexpr size_t strip_dev_smem_bytes() {
    using C = StripCfg<PREC>;
    constexpr int NPL = Store<PREC>::NPLANES;
    return (size_t)STAGES * NPL * (BX + 2 * C::HALO) * C::ES + (size_t)DEV_OUT_BUFS * NPL * BX * C::ES +
           (size_t)8 * (BX + 2) * sizeof(float) + (size_t)2 * STAGES * 8 + 16;
}

template <int PREC, int BX, int STAGES, bool EQ24, int BMODE>
__global__ void __launch_bounds__(strip_threads<BX>(), 2)
    k_step_strip_dev(const typename Store<PREC>::elem* __restrict__ src,
                     typename Store<PREC>::elem* __restrict__ dst, const KParams kp, int nchunks) {
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
    static_assert(NPL <= 32, "one issuing lane per plane in the halo warp");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    elem* stage = reinterpret_cast<elem*>(smem_raw);                 // [STAGES][NPL][SEGW]
    elem* outb = stage + (size_t)STAGES * NPL * SEGW;                 // [DEV_OUT_BUFS][NPL][BX]
    float* ring_psi = reinterpret_cast<float*>(outb + (size_t)DEV_OUT_BUFS * NPL * BX);  // [4][RW]
    float* ring_psi2 = ring_psi + 4 * RW;                                                // [4][RW]
    uint64_t* full = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(ring_psi2 + 4 * RW) + 7) & ~uintptr_t(7));
    uint64_t* empty = full + STAGES;
    __shared__ int s_abort[2];

    const int t = threadIdx.x;
    const int nx = kp.nx, ny = kp.ny;
    const int x0 = blockIdx.x * BX;
    const int W = min(BX, nx - x0);
    // rows updated: [H, ny - H) (H = kp.halo_rows; 0 on a periodic lattice)
    const int H = kp.halo_rows, nrows = ny - 2 * H;
    const int y_start = H + (int)((long long)blockIdx.y * nrows / nchunks);
    const int y_end = H + (int)((long long)(blockIdx.y + 1) * nrows / nchunks);
    const int njobs = (y_end - y_start) + 2;  // pre-collision rows y_start-1 .. y_end

    if (t == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], BX / 32);
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
    const uint32_t plane = (uint32_t)kp.plane, pitch = (uint32_t)kp.pitch;
    const bool halo = t >= BX;
    const int lane = t & 31;
    // ring column r holds strip column r - 1: column thread t owns r = t + 1,
    // halo lanes 0 and 1 own r = 0 and r = W + 1
    const int r_psi = halo ? (lane == 0 ? 0 : W + 1) : t + 1;
    const bool has_psi = halo ? lane < 2 : t < W;
    const int Wb = W & ~(16 / ES - 1);    // columns leaving by bulk copy (whole 16-byte units)
    const uint32_t out_bytes = (uint32_t)Wb * ES;
    const bool issuer = halo && lane < NPL;  // halo lane p copies plane p of each collided row out
    const int xg = x0 + t;
    const bool ghost_lo = xg < STRIP_GHOST, ghost_hi = xg >= nx - STRIP_GHOST;
    int flags = 0;
    float Hf_c = 0.0f, Hg_c = 0.0f;       // deviation sums of this thread's site in the row behind
    int s = 0, sp = STAGES - 1;           // stage of job j and of job j - 1
    uint32_t ph = 0;                      // parity of stage s's "full" barrier at job j
    int ob = 0;                           // row buffer of the collision in job j
    bool aborted = false;
    for (int j = 0; j < njobs; ++j) {
        if (!mbar_wait_bounded(&full[s], ph, kp.wait_cycles)) s_abort[j & 1] = 1;
        // 1. rho, T, psi of pre-collision row j at ring column r_psi
        float Hf_n = 0.0f, Hg_n = 0.0f;
        if (has_psi) {
            const elem* st = stage + s * (NPL * SEGW);
            const int c = r_psi - 1 + HALO;  // smem column of the site
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                Hf_n = acc_dev<S>(st + i * SEGW + c - ex(i), i, rest_lo_offset(i) * SEGW, Hf_n);
                Hg_n = acc_dev<S>(st + (9 + i) * SEGW + c - ex(i), 9 + i, rest_lo_offset(9 + i) * SEGW, Hg_n);
            }
            const float rho = kp.sum_bf + Hf_n;
            const float T = (kp.sum_bg + Hg_n) / (rho * kp.f.cv);
            float psi, psi2;
            site_psi_T<float, BMODE>(kp, rho, T, psi, psi2, flags);
            if (BMODE != BETA_ZERO) ring_psi[(j & 3) * RW + r_psi] = psi;
            if (BMODE != BETA_ONE) ring_psi2[(j & 3) * RW + r_psi] = psi2;
        }
        // the row buffer of this job was copied out DEV_OUT_BUFS - 1 jobs ago
        if (issuer) bulk_wait_group_read<DEV_OUT_BUFS - 2>();
        consumer_sync<BX + 32>();
        if (s_abort[j & 1]) {
            aborted = true;
            break;
        }
        // the row collided in job j - 1 is complete in its buffer (every
        // writer fenced its stores before the barrier): copy it out
        if (issuer && j >= 3 && out_bytes > 0) {
            const int bprev = ob == 0 ? DEV_OUT_BUFS - 1 : ob - 1;
            const int y = y_start + j - 3;
            bulk_copy_s2g(dst + ((size_t)lane * plane + (size_t)y * pitch + (size_t)x0),
                          outb + ((size_t)bprev * NPL + lane) * BX, out_bytes);
            bulk_commit_group();
        }
        if (!halo) {
            // 2. collide pre-collision row j-1 (its psi neighbourhood is complete)
            if (j >= 2 && t < W) {
                const elem* st = stage + sp * (NPL * SEGW);
                const int c = t + HALO;
                const int r = t + 1;
                float Fx, Fy;
                force_from_rows<float, BMODE>(
                    kp, ring_psi + ((j - 2) & 3) * RW + r, ring_psi + ((j - 1) & 3) * RW + r,
                    ring_psi + (j & 3) * RW + r, ring_psi2 + ((j - 2) & 3) * RW + r,
                    ring_psi2 + ((j - 1) & 3) * RW + r, ring_psi2 + (j & 3) * RW + r, Fx, Fy);
                float h[9], q[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    h[i] = dev_of<S>(st + i * SEGW + c - ex(i), i, rest_lo_offset(i) * SEGW);
                    q[i] = dev_of<S>(st + (9 + i) * SEGW + c - ex(i), 9 + i, rest_lo_offset(9 + i) * SEGW);
                }
                collide_dev<EQ24>(kp, h, q, Hf_c, Hg_c, Fx, Fy);
                elem v[NPL];
                encode_site_dev<S>(h, q, Hf_c, Hg_c, v);
                const int y = y_start + j - 2;
                elem* d = dst + ((size_t)y * pitch + (size_t)xg);
                if (t < Wb) {
                    elem* o = outb + (size_t)ob * NPL * BX + t;
#pragma unroll
                    for (int p = 0; p < NPL; ++p) o[p * BX] = v[p];
                    fence_proxy_async_smem();
                    put_ghost_copies<S>(d, plane, nx, v, ghost_lo, ghost_hi);
                } else {
                    put_planes<S>(d, plane, nx, v, ghost_lo, ghost_hi);
                }
            }
            // 3. the stage of job j-1 has had its last reader (psi at j-1, collision at j)
            if (j >= 1) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[sp]);
            }
        }
        Hf_c = Hf_n;
        Hg_c = Hg_n;
        sp = s;
        if (++s == STAGES) {
            s = 0;
            ph ^= 1u;
        }
        if (++ob == DEV_OUT_BUFS) ob = 0;
    }
    if (!aborted) {
        // the last collided row: every writer has fenced its stores
        consumer_sync<BX + 32>();
        if (issuer && njobs >= 3 && out_bytes > 0) {
            const int bprev = ob == 0 ? DEV_OUT_BUFS - 1 : ob - 1;
            const int y = y_start + njobs - 3;
            bulk_copy_s2g(dst + ((size_t)lane * plane + (size_t)y * pitch + (size_t)x0),
                          outb + ((size_t)bprev * NPL + lane) * BX, out_bytes);
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
