// unet_tcs.cuh -- the 3x3 circular convolution on the tcgen05 tensor cores for
// the layers whose weights do not fit in shared memory (up to 9 x 384 x 384
// BF16 values): the coarse levels of the network (images 16 .. 128 wide),
// the wide level-1 decoder layer and the input gradients with 64 .. 384
// output channels.  Same implicit GEMM as k_conv3_tc,
//   out[p][co] = sum_{tap, ci} in[shift_tap(p)][ci] W[co][tap][ci],
// with M = 128 pixels of one image row (rows narrower than 128 leave the
// remaining accumulator rows unused), N = NB output channels of one block
// (NB = 128 or 64) and K = 9 taps x Cin, walked in chunks of 16 channels.
//
// A tile is R = 256 / NB consecutive rows of one image (one 128-pixel segment
// of each) for one block of NB output channels; the R rows share every weight
// stage.  Per 16-channel chunk a stage holds
//   A: the (R + 2)-row input halo, 2 channel groups, in the core-matrix layout
//      of k_conv3_tc: group g, halo row h, slot q ->
//      g * TS_GSTR(R) + (h * TC_HROW + q) * 16, the row segment at slots
//      8 .. 8 + segw - 1 (one TMA box per group and row), the wrapped
//      neighbours at slots 7 and 8 + segw (16-byte cp.async copies);
//   B: the chunk's weights of the block for all 9 taps, one contiguous image
//      (blocked_at) moved by one bulk copy: tap t, output-channel group j,
//      input-channel group k -> t * NB * 32 + (2 j + k) * 128 bytes.
// The MMA view of tap (dy, dx) for tile row r starts at halo row r + dy,
// slot 7 + dx.
//
// Roles as in k_conv3_tc: warp 0 produces (elected lane: barrier byte count,
// tensor copies, weight copy; lanes 0 .. 4 (R + 2) - 1: edge pixels, each
// arriving on the stage barrier when it lands), warp 9 runs the MMA loop
// (elected lane issues), warps 1-8 are two epilogue groups taking alternate
// tiles; the accumulators of a tile occupy R x NB = 256 TMEM columns, double
// buffered.  Tiles are ordered with the channel block outermost, so the CTAs
// stream the same weights at the same time (L2 reuse).  Every wait is bounded
// (bit 6 of *a.err on a timeout).
#pragma once

#include "unet_tc.cuh"

namespace unk {

constexpr int TS_STAGES = 4;
constexpr int TS_THREADS = 320;
constexpr int TS_MMA_WARP = 9;

__host__ __device__ constexpr int ts_rows(int NB) { return 256 / NB; }
__host__ __device__ constexpr int ts_gstr(int R) { return (R + 2) * TC_HROW * 16; }           // one channel group
__host__ __device__ constexpr int ts_abytes(int R) { return 2 * ts_gstr(R); }
__host__ __device__ constexpr int ts_bbytes(int NB) { return 9 * NB * 32; }
__host__ __device__ constexpr int ts_stage_bytes(int NB) { return ts_abytes(ts_rows(NB)) + ts_bbytes(NB); }
__host__ __device__ constexpr size_t ts_smem_bytes(int NB) {
    // stages, bias (384 floats), barriers, alignment slack
    return (size_t)TS_STAGES * ts_stage_bytes(NB) + 1536 + 256 + 1024;
}
// output-channel block of a layer (0: not for this kernel)
__host__ __device__ constexpr int ts_block(int Cout) { return Cout % 128 == 0 ? 128 : (Cout % 64 == 0 ? 64 : 0); }

// one MMA from the elected lane of the (converged) warp
__device__ __forceinline__ void ts_mma1(uint32_t d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                        uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n"
        ".reg .pred p, e;\n .reg .b32 el;\n .reg .b64 a, b;\n"
        "setp.ne.b32 p, %5, 0;\n"
        "mov.b64 a, {%1, %2};\n mov.b64 b, {%3, %4};\n"
        "elect.sync el|e, 0xffffffff;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %6, p;\n"
        "}\n" ::"r"(d),
        "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(acc), "r"(idesc)
        : "memory");
}

// from the elected lane: arm bar with `bytes`, then the weight image of the
// stage (one bulk copy of wbytes)
__device__ __forceinline__ void ts_arm_and_copy_w(uint32_t bar, uint32_t bytes, uint32_t dst, const void* src,
                                                  uint32_t wbytes) {
    asm volatile(
        "{\n"
        ".reg .pred e;\n .reg .b32 el;\n"
        "elect.sync el|e, 0xffffffff;\n"
        "@e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
        "@e cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%2], [%3], %4, [%0];\n"
        "}\n" ::"r"(bar),
        "r"(bytes), "r"(dst), "l"(src), "r"(wbytes)
        : "memory");
}

// from the elected lane: one tensor copy (box of the map) to dst
__device__ __forceinline__ void ts_tma(const CUtensorMap* map, uint32_t dst, uint32_t bar, int c1, int c2, int c3) {
    asm volatile(
        "{\n"
        ".reg .pred e;\n .reg .b32 el, z;\n"
        "mov.u32 z, 0;\n"
        "elect.sync el|e, 0xffffffff;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%1], [%0, {z, %3, %4, "
        "%5}], [%2];\n"
        "}\n" ::"l"(reinterpret_cast<uint64_t>(map)),
        "r"(dst), "r"(bar), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

template <int NB>
__global__ void __launch_bounds__(TS_THREADS, 1)
    k_conv3_tcs(ConvArgs a, const __grid_constant__ CUtensorMap xmap, const bf16* __restrict__ wimg) {
    constexpr int R = ts_rows(NB);
    constexpr int GSTR = ts_gstr(R);
    constexpr int ABYTES = ts_abytes(R);
    constexpr int BBYTES = ts_bbytes(NB);
    constexpr int SBYTES = ABYTES + BBYTES;
    constexpr int EDGES = 2 * (R + 2) * 2;               // groups x halo rows x sides
    constexpr uint32_t COLS = 512;                       // 2 buffers x R x NB
    static_assert(R * NB == 256 && EDGES <= 32, "tile shape");
    extern __shared__ __align__(1024) uint8_t ts_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ts_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sS = base;                                                       // [TS_STAGES][SBYTES]
    float* sBias = reinterpret_cast<float*>(sS + (size_t)TS_STAGES * SBYTES);  // [Cout <= 384]
    uint64_t* full = reinterpret_cast<uint64_t*>(sBias + 384);
    uint64_t* empty = full + TS_STAGES;
    uint64_t* accf = empty + TS_STAGES;  // [2]
    uint64_t* acce = accf + 2;           // [2]
    uint64_t* mdone = acce + 2;
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(mdone + 1);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W;
    const int segw = W < TC_M ? W : TC_M;                // pixels of a row segment
    const int segs = W / segw;
    const int rblocks = H / R;
    const int nblocks = a.Cout / NB;
    const int per_block = a.N * rblocks * segs;          // tiles of one channel block
    const int ntiles = nblocks * per_block;              // the host keeps this below 2^31
    const int nchunks = a.Cin / 16;

    if (tid == 0) {
        for (int s = 0; s < TS_STAGES; ++s) {
            tc_bar_init(&full[s], 1 + EDGES);
            tc_bar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc_bar_init(&accf[b], 1);
            tc_bar_init(&acce[b], 128);
        }
        tc_bar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int q = tid; q < a.Cout; q += TS_THREADS) sBias[q] = a.bias ? a.bias[q] : 0.0f;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        // ------------------------------------------------ producer warp
        // this lane's edge pixel: channel group, halo row, side (0 left, 1 right)
        const int eg = lane / (2 * (R + 2)), ehr = (lane % (2 * (R + 2))) >> 1, eside = lane & 1;
        const bool edge = lane < EDGES;
        int s = 0;
        uint32_t ph = 0;  // (job / TS_STAGES) & 1
        long long j = 0;
        for (int tile = blockIdx.x; tile < ntiles && __shfl_sync(0xffffffffu, *s_abort, 0) == 0;
             tile += gridDim.x) {
            const int nb = tile / per_block;
            int rem = tile - nb * per_block;
            const int seg = rem % segs;
            rem /= segs;
            const int y0 = (rem % rblocks) * R;
            const int n = rem / rblocks;
            const int x0 = seg * segw;
            const int xl = wrap(x0 - 1, W), xr = wrap(x0 + segw, W);
            const bf16* wsrc = wimg + (size_t)nb * nchunks * (BBYTES / 2);
            bool stop = false;
            for (int c = 0; c < nchunks; ++c, ++j) {
                if (j >= TS_STAGES && !__all_sync(0xffffffffu, tc_bar_wait(&empty[s], ph ^ 1u))) {
                    if (lane == 0) {
                        *s_abort = 1;
                        if (a.err) atomicOr(a.err, 1 << 6);
                    }
                    stop = true;
                    break;
                }
                const uint32_t st = smem_addr(sS + (size_t)s * SBYTES);
                const uint32_t fb = smem_addr(&full[s]);
                const int cg = (a.xoff + c * 16) / 8;  // first channel group of the chunk
                ts_arm_and_copy_w(fb, (uint32_t)(2 * (R + 2) * segw * 16 + BBYTES), st + ABYTES,
                                  wsrc + (size_t)c * (BBYTES / 2), (uint32_t)BBYTES);
#pragma unroll
                for (int g = 0; g < 2; ++g)
#pragma unroll
                    for (int hr = 0; hr < R + 2; ++hr)
                        ts_tma(&xmap, st + g * GSTR + (hr * TC_HROW + TC_BODY) * 16, fb, x0 / 8, cg + g,
                               n * H + wrap(y0 + hr - 1, H));
                if (edge) {
                    // the copy arrives on the stage's barrier by itself once it has landed
                    const int yy = wrap(y0 + ehr - 1, H);
                    cp_async16(sS + (size_t)s * SBYTES + eg * GSTR +
                                   (ehr * TC_HROW + (eside ? TC_BODY + segw : TC_BODY - 1)) * 16,
                               a.x + act_at((long long)n * H + yy, eside ? xr : xl, cg * 8 + eg * 8, a.xC, W), true);
                    tc_cp_async_arrive(&full[s]);
                }
                if (++s == TS_STAGES) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (stop) break;
        }
        // every copy issued has landed before leaving (waits with the default limit)
        cp_async_wait<0>();
        if (lane == 0)
            for (long long k = (j > TS_STAGES ? j - TS_STAGES : 0); k < j; ++k)
                (void)tc_bar_wait(&full[(int)(k % TS_STAGES)], (uint32_t)((k / TS_STAGES) & 1));
        __syncwarp();
    } else if (warp == TS_MMA_WARP) {
        // ------------------------------------------------ MMA issue (warp-wide, elected lane issues)
        constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NB >> 3) << 17) |
                                   ((uint32_t)(TC_M >> 4) << 24);
        const uint64_t da0 = tc_mdesc(smem_addr(sS) + (uint32_t)((TC_BODY - 1) * 16), (uint32_t)GSTR, 128);
        const uint64_t db0 = tc_mdesc(smem_addr(sS) + (uint32_t)ABYTES, 128, 256);
        const uint32_t ahi = (uint32_t)(da0 >> 32), bhi = (uint32_t)(db0 >> 32);
        int s = 0, b = 0, t = 0;
        uint32_t fph = 0, rnd = 0;  // (job / TS_STAGES) & 1, (t / 2) & 1
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok && __shfl_sync(0xffffffffu, *s_abort, 0) == 0;
             tile += gridDim.x, ++t) {
            if (t >= 2 && !__all_sync(0xffffffffu, tc_bar_wait(&acce[b], rnd ^ 1u))) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dacc = tmem + (uint32_t)(b * R * NB);
            for (int c = 0; c < nchunks; ++c) {
                const uint32_t a_lo = (uint32_t)da0 + (uint32_t)s * (uint32_t)(SBYTES >> 4);
                const uint32_t b_lo = (uint32_t)db0 + (uint32_t)s * (uint32_t)(SBYTES >> 4);
                if (!__all_sync(0xffffffffu, tc_bar_wait(&full[s], fph))) {
                    ok = false;
                    break;
                }
                // edge pixels came through cp.async (generic proxy); the MMAs read via the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap % 3;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        ts_mma1(dacc + (uint32_t)(r * NB), a_lo + (uint32_t)((r + dy) * TC_HROW + dx), ahi,
                                b_lo + (uint32_t)(tap * 2 * NB), bhi, IDESC, (c > 0 || tap > 0) ? 1u : 0u);
                }
                tc_commit_one(&empty[s]);  // the stage is free again once these MMAs have read it
                if (++s == TS_STAGES) {
                    s = 0;
                    fph ^= 1u;
                }
            }
            if (!ok) break;
            tc_commit_one(&accf[b]);
            if (++b == 2) {
                b = 0;
                rnd ^= 1u;
            }
        }
        if (!ok && lane == 0) {
            *s_abort = 1;
            if (a.err) atomicOr(a.err, 1 << 6);
        }
        // every MMA issued has completed before TMEM is released
        tc_commit_one(mdone);
        if (!__all_sync(0xffffffffu, tc_bar_wait(mdone, 0u)) && lane == 0 && a.err) atomicOr(a.err, 1 << 6);
    } else {
        // ------------------------------------------------ epilogue (warps 1-8)
        // group grp takes the CTA's tiles t = grp, grp + 2, ...: buffer grp,
        // phase (k-th own tile) k & 1
        const int grp = (warp - 1) >> 2;
        const int q = warp & 3;                  // TMEM lanes 32 q .. 32 q + 31
        const int px = q * 32 + lane;            // pixel of the row segment
        const bool warp_live = q * 32 < segw;    // the warp has pixels of the image
        const bool live = px < segw;
        uint32_t ph = 0;
        for (int tile = blockIdx.x + grp * (int)gridDim.x; tile < ntiles; tile += 2 * (int)gridDim.x) {
            const int nb = tile / per_block;
            int rem = tile - nb * per_block;
            const int seg = rem % segs;
            rem /= segs;
            const int y0 = (rem % rblocks) * R;
            const int n = rem / rblocks;
            const int x = seg * segw + px;
            const int co0 = nb * NB;
            if (!__all_sync(0xffffffffu, tc_bar_wait(&accf[grp], ph))) {
                *s_abort = 1;
                if (a.err) atomicOr(a.err, 1 << 6);
                break;
            }
            ph ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (warp_live) {
#pragma unroll 1
                for (int r = 0; r < R; ++r) {
                    const long long row = (long long)n * H + y0 + r;
#pragma unroll 1
                    for (int cc = 0; cc < NB; cc += 32) {
                        uint4 mraw[4];
                        if (a.mask && live)
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                mraw[k] = __ldg(reinterpret_cast<const uint4*>(
                                    a.mask + act_at(row, x, a.moff + co0 + cc + 8 * k, a.mC, W)));
                        uint32_t v[32];
                        const uint32_t taddr =
                            tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(grp * R * NB + r * NB + cc);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                            "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
                              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
                              "=r"(v[31])
                            : "r"(taddr));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        if (live) {
#pragma unroll
                            for (int j8 = 0; j8 < 4; ++j8) {
                                const int co = co0 + cc + j8 * 8;
                                float f8[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e) f8[e] = __uint_as_float(v[j8 * 8 + e]) + sBias[co + e];
                                if (a.relu)
#pragma unroll
                                    for (int e = 0; e < 8; ++e) f8[e] = fmaxf(f8[e], 0.0f);
                                if (a.mask) {
                                    float mk[8];
                                    unpack8(mraw[j8], mk);
#pragma unroll
                                    for (int e = 0; e < 8; ++e) f8[e] = mk[e] > 0.0f ? f8[e] : 0.0f;
                                }
                                const uint4 u = pack8(f8);
                                if (!a.up) {
                                    *reinterpret_cast<uint4*>(a.y + act_at(row, x, a.yoff + co, a.yC, W)) = u;
                                } else {
#pragma unroll
                                    for (int uy = 0; uy < 2; ++uy)
#pragma unroll
                                        for (int ux = 0; ux < 2; ++ux)
                                            *reinterpret_cast<uint4*>(a.y + act_at(2 * row + uy, 2 * x + ux,
                                                                                   a.yoff + co, a.yC, 2 * W)) = u;
                                }
                            }
                        }
                    }
                }
            }
            // this thread has read its lanes of buffer grp
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            tc_bar_arrive(&acce[grp]);
            if (__any_sync(0xffffffffu, *s_abort != 0)) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
}

}  // namespace unk
