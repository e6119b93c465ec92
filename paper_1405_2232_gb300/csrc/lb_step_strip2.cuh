// lb_step_strip2.cuh -- two fused time steps per launch (temporal blocking)
// of the strip-marching kernel, FP32 storage.
//
// A CTA owns a strip of W = BX - 8 columns and a chunk of rows.  As in
// k_step_strip, a producer warp streams each pre-collision row of step t (the
// 18 plane rows, 4 columns of halo on each side) into a stage ring with
// cp.async.bulk.  The consumer warps then run both steps without a trip
// through HBM in between:
//   level 1 (step t):   psi of row r, collision of row r - 1, whose
//                       post-collision populations go to a 6-row ring in
//                       shared memory (columns x0 - 2 .. x0 + W + 1);
//   level 2 (step t+1): the pre-collision populations of step t + 1 are
//                       pulled from that ring, psi of row r - 4, collision of
//                       row r - 5, stored to HBM.
// Per job (one row of step t arriving) a thread does one site of each of the
// four phases; one named barrier per job separates the psi phases from the
// collision phases.  The level-2 rows lag the level-1 rows so that every
// ring slot a phase reads was written before the previous barrier:
//   phase A: psi1(r) from stage j,   psi2(r - 4) from ring rows r-5..r-3
//   barrier
//   phase B: collide1(r - 1) from stage j-1 and psi1 rows r-2..r -> ring row r-1,
//            collide2(r - 5) from ring rows r-6..r-4 and psi2 rows r-6..r-4 -> HBM
// Ring slots are indexed by job (row - (y_start - 3)), mod 6 for the
// population ring and mod 4 for the psi rings.  The arithmetic of each site
// and step is that of k_step_strip, and the ring holds the FP32 values the
// single-step kernel would store and reload, so two fused steps equal two
// single steps bit for bit.
//
// Column ranges per strip (W' = the strip's width, x0 its first column):
//   stage:     x0 - 4 .. x0 + W' + 3   (W' + 8 <= BX columns, 16-byte aligned)
//   psi1:      x0 - 3 .. x0 + W' + 2   (W' + 6 sites)
//   collide1:  x0 - 2 .. x0 + W' + 1   (W' + 4 sites, the ring's columns)
//   psi2:      x0 - 1 .. x0 + W'       (W' + 2 sites)
//   collide2:  x0     .. x0 + W' - 1   (W' sites)
// Rows: a chunk [y_start, y_end) loads rows y_start - 3 .. y_end + 2 of step t.
#pragma once

#include "lb_step_strip.cuh"

namespace lbgb {

template <int BX>
__host__ __device__ constexpr int strip2_width() {
    return BX - 8;
}

template <int BX, int STAGES>
constexpr size_t strip2_smem_bytes() {
    return (size_t)STAGES * 18 * BX * 4 + (size_t)6 * 18 * (strip2_width<BX>() + 4) * 4 +
           (size_t)16 * (BX + 2) * 4 + (size_t)2 * STAGES * 8 + 16;
}

template <int BX, int STAGES, bool EQ24, int BMODE>
__global__ void __launch_bounds__(BX + 32, 3)
    k_step_strip2(const float* __restrict__ src, float* __restrict__ dst, const KParams kp, int nchunks) {
    using S = Store<LB_PREC_FP32>;
    using real = float;
    constexpr int SEGW = BX;                      // stage row: W + 8 columns
    constexpr int WMAX = strip2_width<BX>();
    constexpr int P1W = WMAX + 4;                 // ring row: W + 4 columns
    constexpr int RW = BX + 2;                    // psi ring row
    constexpr int NCW = BX / 32;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stage = reinterpret_cast<float*>(smem_raw);             // [STAGES][18][SEGW]
    float* p1 = stage + (size_t)STAGES * 18 * SEGW;                // [6][18][P1W]
    float* ps1 = p1 + (size_t)6 * 18 * P1W;                        // [4][RW] psi, level 1
    float* qs1 = ps1 + 4 * RW;                                     // [4][RW] psi^2, level 1
    float* ps2 = qs1 + 4 * RW;                                     // [4][RW] psi, level 2
    float* qs2 = ps2 + 4 * RW;                                     // [4][RW] psi^2, level 2
    uint64_t* full = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(qs2 + 4 * RW) + 7) & ~uintptr_t(7));
    uint64_t* empty = full + STAGES;
    __shared__ int s_abort;

    const int t = threadIdx.x;
    const int nx = kp.nx, ny = kp.ny;
    const int x0 = blockIdx.x * WMAX;
    const int W = min(WMAX, nx - x0);
    const int y_start = (int)((long long)blockIdx.y * ny / nchunks);
    const int y_end = (int)((long long)(blockIdx.y + 1) * ny / nchunks);
    const int njobs_load = (y_end - y_start) + 6;   // step-t rows y_start-3 .. y_end+2
    const int njobs = njobs_load + 2;               // two more jobs finish level 2
    const uint32_t plane = (uint32_t)kp.plane, pitch = (uint32_t)kp.pitch;

    if (t == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    if (t >= BX) {
        // ------------------------------------------------ producer warp
        const int lane = t - BX;
        const bool left_wrap = x0 == 0;
        const bool right_wrap = x0 + W == nx;
        int issued = 0;
        for (int j = 0; j < njobs_load; ++j) {
            const int s = j % STAGES;
            if (j >= STAGES) {
                if (!mbar_wait_bounded(&empty[s], (uint32_t)(((j / STAGES) - 1) & 1))) {
                    if (lane == 0) atomicOr(kp.err, 1 << LB_ERR_TIMEOUT);
                    break;
                }
            }
            int y = y_start - 3 + j;
            while (y < 0) y += ny;
            while (y >= ny) y -= ny;
            if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)(18 * (W + 8) * 4));
            __syncwarp();
            if (lane < 18) {
                const int i = lane;
                const int d = i < 9 ? i : i - 9;
                int sy = y - ey(d);
                sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                const float* row = src + (size_t)((uint32_t)i * plane + (uint32_t)sy * pitch);
                float* seg = stage + ((size_t)s * 18 + i) * SEGW;
                if (!left_wrap && !right_wrap) {
                    bulk_copy_g2s(seg, row + (x0 - 4), (uint32_t)((W + 8) * 4), &full[s]);
                } else {
                    bulk_copy_g2s(seg, row + (left_wrap ? nx - 4 : x0 - 4), 16u, &full[s]);
                    bulk_copy_g2s(seg + 4, row + x0, (uint32_t)(W * 4), &full[s]);
                    bulk_copy_g2s(seg + 4 + W, row + (right_wrap ? 0 : x0 + W), 16u, &full[s]);
                }
            }
            issued = j + 1;
        }
        if (lane == 0)
            for (int j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j)
                (void)mbar_wait_bounded(&full[j % STAGES], (uint32_t)((j / STAGES) & 1));
        return;
    }

    // ---------------------------------------------------- consumer warps
    int flags = 0;
    for (int j = 0; j < njobs; ++j) {
        const bool load = j < njobs_load;
        // ---- phase A: psi of the newest row of each level
        if (load) {
            const int s = j % STAGES;
            if (!mbar_wait_bounded(&full[s], (uint32_t)((j / STAGES) & 1))) s_abort = 1;
            const float* st = stage + (size_t)s * 18 * SEGW;
            if (t < W + 6) {
                const int c = t + 1;  // stage column of site x0 - 3 + t
                real f[9], g[9], rho, T, psi, psi2;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    f[i] = st[i * SEGW + c - ex(i)];
                    g[i] = st[(9 + i) * SEGW + c - ex(i)];
                }
                site_psi<real, BMODE>(kp, f, g, rho, T, psi, psi2, flags);
                if (BMODE != BETA_ZERO) ps1[(j & 3) * RW + t] = psi;
                if (BMODE != BETA_ONE) qs1[(j & 3) * RW + t] = psi2;
            }
        }
        if (j >= 6 && t < W + 2) {
            // pre-collision row (job j - 4) of step t + 1, pulled from the ring
            const int p = t + 1;  // ring column of site x0 - 1 + t
            real f[9], g[9], rho, T, psi, psi2;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float* slot = p1 + (size_t)((j - 4 - ey(i)) % 6) * 18 * P1W;
                f[i] = slot[i * P1W + p - ex(i)];
                g[i] = slot[(9 + i) * P1W + p - ex(i)];
            }
            site_psi<real, BMODE>(kp, f, g, rho, T, psi, psi2, flags);
            if (BMODE != BETA_ZERO) ps2[(j & 3) * RW + t] = psi;
            if (BMODE != BETA_ONE) qs2[(j & 3) * RW + t] = psi2;
        }
        consumer_sync<BX>();
        if (s_abort) break;
        // ---- phase B: level-1 collision into the ring, level-2 collision to HBM
        if (j >= 2 && j - 1 < njobs_load && t < W + 4) {
            const float* st = stage + (size_t)((j - 1) % STAGES) * 18 * SEGW;
            const int c = t + 2;  // stage column of site x0 - 2 + t
            real f[9], g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i] = st[i * SEGW + c - ex(i)];
                g[i] = st[(9 + i) * SEGW + c - ex(i)];
            }
            real rho = f[0];
#pragma unroll
            for (int i = 1; i < 9; ++i) rho += f[i];
            const int r = t + 1;  // psi1 column of the site
            real Fx, Fy, ux, uy, T;
            force_from_rows<real, BMODE>(kp, ps1 + ((j - 2) & 3) * RW + r, ps1 + ((j - 1) & 3) * RW + r,
                                         ps1 + (j & 3) * RW + r, qs1 + ((j - 2) & 3) * RW + r,
                                         qs1 + ((j - 1) & 3) * RW + r, qs1 + (j & 3) * RW + r, Fx, Fy);
            collide<real, EQ24>(kp, f, g, rho, Fx, Fy, ux, uy, T);
            float* slot = p1 + (size_t)((j - 1) % 6) * 18 * P1W;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                slot[i * P1W + t] = f[i];
                slot[(9 + i) * P1W + t] = g[i];
            }
        }
        if (j >= 8 && t < W) {
            const int p = t + 2;  // ring column of site x0 + t
            real f[9], g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float* slot = p1 + (size_t)((j - 5 - ey(i)) % 6) * 18 * P1W;
                f[i] = slot[i * P1W + p - ex(i)];
                g[i] = slot[(9 + i) * P1W + p - ex(i)];
            }
            real rho = f[0];
#pragma unroll
            for (int i = 1; i < 9; ++i) rho += f[i];
            const int r = t + 1;  // psi2 column of the site
            real Fx, Fy, ux, uy, T;
            force_from_rows<real, BMODE>(kp, ps2 + ((j - 2) & 3) * RW + r, ps2 + ((j - 1) & 3) * RW + r,
                                         ps2 + (j & 3) * RW + r, qs2 + ((j - 2) & 3) * RW + r,
                                         qs2 + ((j - 1) & 3) * RW + r, qs2 + (j & 3) * RW + r, Fx, Fy);
            collide<real, EQ24>(kp, f, g, rho, Fx, Fy, ux, uy, T);
            int y = y_start + j - 8;
            y = y >= ny ? y - ny : y;
            const uint32_t off = (uint32_t)y * pitch + (uint32_t)(x0 + t);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                S::put(dst + ((uint32_t)i * plane + off), f[i], 0.0f);
                S::put(dst + ((uint32_t)(9 + i) * plane + off), g[i], 0.0f);
            }
        }
        // the stage of job j - 1 has had its last reader (collide1 at job j)
        if (j >= 1 && j - 1 < njobs_load) {
            __syncwarp();
            if ((t & 31) == 0) mbar_arrive(&empty[(j - 1) % STAGES]);
        }
    }
    if (s_abort) {
        if (t == 0) atomicOr(kp.err, 1 << LB_ERR_TIMEOUT);
        return;
    }
    if (flags) atomicOr(kp.err, flags);
}

}  // namespace lbgb
