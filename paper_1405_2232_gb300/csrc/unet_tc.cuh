// unet_tc.cuh -- the 3x3 circular convolution of the warm-start network on the
// fifth-generation tensor cores: tcgen05.mma with BF16 operands read from
// shared memory through matrix descriptors and the FP32 accumulator in tensor
// memory (TMEM), for images whose width is a multiple of 128 (the two finest
// levels of the network, half of its convolution work).
//
// Implicit GEMM, as in k_conv3 / k_conv3_halo:
//   out[p][co] = sum_{tap, ci} in[shift_tap(p)][ci] W[co][tap][ci]
// with M = 128 pixels (one 128-wide segment of one image row), N = Cout (32,
// 64 or 96) and K = 9 taps x Cin.
//
// Reuse: the CTA stages, per 32-channel chunk, the 3-row x 130-pixel input
// halo of its row segment once, in the no-swizzle K-major core-matrix layout
// with the pixels of a halo row 16 bytes apart inside each 8-channel group:
//   group g (8 channels), halo row r, slot h -> g * TC_KG + (r * TC_HROW + h) * 16
// where slots 8 .. 135 hold the segment's 128 pixels (written by one TMA
// tensor copy per group and row, 128-byte aligned) and slots 7 and 136 the
// wrapped neighbours left and right (plain 16-byte copies: circular padding).
// The A operand of tap (dy, dx) is then the same bytes seen through a matrix
// descriptor that starts at halo row dy + 1, slot 7 + dx + 1 (core matrices of
// 8 consecutive pixels 128 bytes apart along M, 8-channel groups TC_KG bytes
// apart along K), so the nine taps are nine descriptors over one staged halo.
// The weights of the layer (9 x Cout x Cin, at most TC_MAX_WBYTES) stay
// resident in shared memory for the CTA's lifetime, per tap in the K-major
// core-matrix layout (8 output channels x 8 input channels per core matrix).
//
// Persistent, warp-specialised CTAs (one per SM, tiles dealt round-robin):
//   warp 0     producer: lane 0 arms the stage's "full" mbarrier with the
//              byte count and issues the 12 TMA tensor copies (4 channel
//              groups x 3 rows, cp.async.bulk.tensor, completion by
//              transaction count); lanes 0..23 copy the 24 wrapped edge
//              pixels and arrive once their copies have landed (after
//              fence.proxy.async); the ring is `stages` deep (up to 8);
//   warp 5     one thread issues the 9 x (32 / 16) MMAs of a stage into the
//              tile's accumulator and tcgen05.commit's the stage's "empty"
//              mbarrier; after the tile's last chunk it commits "acc full";
//   warps 1-4  epilogue: wait "acc full", tcgen05.ld the tile (TMEM lane =
//              pixel, column = output channel), add the bias, apply ReLU and
//              the gradient mask, round to BF16 and store (or store each
//              pixel to its 2 x 2 block for the upsampling), then arrive on
//              "acc empty".
// Two accumulator buffers (2 N TMEM columns, allocated once per CTA) let the
// MMAs of tile t + 1 run while the epilogue drains tile t.
//
// Every mbarrier wait is bounded (about one second); a wait that gives up
// sets bit LB_ERR_TIMEOUT (6) of *a.err and the CTA winds down: no role
// waits unboundedly on another, the producer waits (with the default limit)
// for every copy it issued before leaving, and TMEM is released after a
// block-wide barrier once the MMAs issued have completed.
#pragma once

#include <cuda.h>

#include "unet_kernels.cuh"

namespace unk {

constexpr int TC_M = 128;                       // pixels per tile (UMMA M)
constexpr int TC_KC = 32;                       // input channels per stage
constexpr int TC_HROW = 144;                    // halo row slots (16 bytes each): pixels at 7 .. 136
constexpr int TC_BODY = 8;                      // slot of the segment's first pixel (128-byte aligned)
constexpr int TC_KG = 3 * TC_HROW * 16;         // bytes of one 8-channel group of a halo (6912)
constexpr int TC_ASTRIDE = (TC_KC / 8) * TC_KG; // bytes of one halo stage (27648, a multiple of 128)
constexpr int TC_TMA_BYTES = (TC_KC / 8) * 3 * TC_M * 16;  // bytes the 12 tensor copies deliver
constexpr int TC_EDGES = (TC_KC / 8) * 3 * 2;   // wrapped edge pixels per stage (24)
constexpr int TC_MAX_STAGES = 8;
constexpr int TC_THREADS = 192;                 // producer warp, 4 epilogue warps, MMA warp
constexpr int TC_MAX_WBYTES = 100 * 1024;       // resident weights per layer
constexpr size_t TC_SMEM_LIMIT = 232448;        // dynamic shared memory per CTA
constexpr long long TC_WAIT = 2000000000LL;     // bounded-wait limit (clock cycles)

__host__ __device__ constexpr size_t tc_wbytes(int N, int Cin) { return (size_t)9 * N * Cin * 2; }
__host__ __device__ constexpr size_t tc_fixed_bytes(int N, int Cin) {
    // weights (rounded to 1 KB), barriers + TMEM slot + flag, alignment slack
    return (tc_wbytes(N, Cin) + 1023) / 1024 * 1024 + 256 + 1024;
}
// ring depth that fits the shared memory next to the layer's weights
__host__ __device__ constexpr int tc_stages(int N, int Cin) {
    const size_t room = TC_SMEM_LIMIT - tc_fixed_bytes(N, Cin);
    const size_t s = room / TC_ASTRIDE;
    return s > TC_MAX_STAGES ? TC_MAX_STAGES : (int)s;
}
__host__ __device__ constexpr size_t tc_smem_bytes(int N, int Cin) {
    return tc_fixed_bytes(N, Cin) + (size_t)tc_stages(N, Cin) * TC_ASTRIDE;
}
// whether a layer runs on this kernel (the host checks the image width too)
__host__ __device__ constexpr bool tc_layer_ok(int N, int Cin) {
    return (N == 32 || N == 64 || N == 96) && Cin % TC_KC == 0 && tc_wbytes(N, Cin) <= (size_t)TC_MAX_WBYTES &&
           tc_stages(N, Cin) >= 3;
}

__device__ __forceinline__ void tc_bar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// TMA tensor copy of one box of a 4-D tensor map into shared memory, completion
// counted on an mbarrier in bytes
__device__ __forceinline__ void tc_tma_load4(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                             uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tc_bar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void tc_bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool tc_bar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool tc_bar_wait(uint64_t* bar, uint32_t parity) {
    if (tc_bar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!tc_bar_try(bar, parity))
        if (clock64() - t0 > TC_WAIT) return false;
    return true;
}
// shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets, each >> 4 in 14 bits; descriptor version 1 (bit 46); no swizzle
__device__ __forceinline__ uint64_t tc_mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
template <int N>
__host__ __device__ constexpr uint32_t tc_idesc_n() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}
template <int N>
__host__ __device__ constexpr uint32_t tc_tmem_cols() {
    return 2 * N <= 64 ? 64u : (2 * N <= 128 ? 128u : 256u);
}

template <int N>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv3_tc(ConvArgs a, const __grid_constant__ CUtensorMap xmap, int stages) {
    extern __shared__ __align__(1024) uint8_t tc_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
    const int Cin = a.Cin;
    const size_t wround = (tc_wbytes(N, Cin) + 1023) / 1024 * 1024;
    uint8_t* sW = base;                       // [9][N/8][Cin/8] core matrices
    uint8_t* sA = base + wround;              // [stages][TC_ASTRIDE], 1024-byte aligned
    uint64_t* full = reinterpret_cast<uint64_t*>(sA + (size_t)stages * TC_ASTRIDE);
    uint64_t* empty = full + TC_MAX_STAGES;
    uint64_t* accf = empty + TC_MAX_STAGES;   // [2]
    uint64_t* acce = accf + 2;                // [2]
    uint64_t* mdone = acce + 2;               // the MMA thread's last commit
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(mdone + 1);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W;
    const int segs = W / TC_M;
    const long long ntiles = (long long)a.N * H * segs;
    const int nchunks = Cin / TC_KC;
    const int SBO_W = (Cin / 8) * 128;                  // weights: 8-row (output channel) groups
    const uint32_t wplane = (uint32_t)N * (uint32_t)Cin * 2u;

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            tc_bar_init(&full[s], 1 + TC_EDGES);     // the armed byte count + the edge copies
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
                     "r"(tc_tmem_cols<N>())
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the layer's weights, resident: 16-byte chunks (co, tap, 8 input channels)
    for (int q = tid; q < 9 * N * (Cin / 8); q += TC_THREADS) {
        const int k8 = q % (Cin / 8);
        const int row = q / (Cin / 8);             // tap * N + co
        const int tap = row / N, co = row - tap * N;
        uint8_t* d = sW + (size_t)tap * wplane + (co >> 3) * SBO_W + k8 * 128 + (co & 7) * 16;
        cp_async16(d, a.w + ((long long)co * 9 + tap) * Cin + k8 * 8, true);
    }
    cp_async_commit();
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        // ------------------------------------------------ producer warp
        constexpr int D = 2;  // edge-copy groups in flight before their arrival
        // this lane's edge pixel: channel group g, halo row hr, side (0 left, 1 right)
        const int eg = lane / 6, ehr = (lane % 6) >> 1, eside = lane & 1;
        const bool edge = lane < TC_EDGES;
        long long j = 0;
        for (long long tile = blockIdx.x; tile < ntiles && !*s_abort; tile += gridDim.x) {
            const int seg = (int)(tile % segs);
            const long long r = tile / segs;
            const int y = (int)(r % H);
            const int n = (int)(r / H);
            const int x0 = seg * TC_M;
            bool stop = false;
            for (int c = 0; c < nchunks; ++c, ++j) {
                const int s = (int)(j % stages);
                // one decision per warp (its lanes poll the barrier independently)
                if (j >= stages &&
                    !__all_sync(0xffffffffu, tc_bar_wait(&empty[s], (uint32_t)(((j / stages) - 1) & 1)))) {
                    if (lane == 0) {
                        *s_abort = 1;
                        if (a.err) atomicOr(a.err, 1 << 6);
                    }
                    stop = true;
                    break;
                }
                uint8_t* st = sA + (size_t)s * TC_ASTRIDE;
                const int cbase = a.xoff + c * TC_KC;
                if (lane == 0) {
                    tc_bar_arrive_tx(&full[s], (uint32_t)TC_TMA_BYTES);
#pragma unroll
                    for (int g = 0; g < TC_KC / 8; ++g)
#pragma unroll
                        for (int hr = 0; hr < 3; ++hr)
                            tc_tma_load4(st + g * TC_KG + (hr * TC_HROW + TC_BODY) * 16, &xmap, cbase + g * 8, x0,
                                         wrap(y + hr - 1, H), n, &full[s]);
                }
                if (edge) {
                    const int yy = wrap(y + ehr - 1, H);
                    const int xx = eside ? wrap(x0 + TC_M, W) : wrap(x0 - 1, W);
                    const long long pix = ((long long)n * H + yy) * W + xx;
                    cp_async16(st + eg * TC_KG + (ehr * TC_HROW + (eside ? TC_BODY + TC_M : TC_BODY - 1)) * 16,
                               a.x + pix * a.xC + cbase + eg * 8, true);
                }
                cp_async_commit();
                if (j >= D) {
                    cp_async_wait<D>();
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (edge) tc_bar_arrive(&full[(int)((j - D) % stages)]);
                }
            }
            if (stop) break;
        }
        // the last jobs' edge copies, then their arrivals; then every tensor
        // copy issued has landed (waits with the default limit) before leaving
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (edge)
            for (long long k = (j > D ? j - D : 0); k < j; ++k) tc_bar_arrive(&full[(int)(k % stages)]);
        if (lane == 0)
            for (long long k = (j > stages ? j - stages : 0); k < j; ++k)
                (void)tc_bar_wait(&full[(int)(k % stages)], (uint32_t)((k / stages) & 1));
        __syncwarp();
    } else if (warp == 5) {
        // ------------------------------------------------ MMA issue (one thread)
        if (lane == 0) {
            constexpr uint32_t IDESC = tc_idesc_n<N>();
            const uint32_t aW = smem_addr(sW);
            long long j = 0, t = 0;
            bool ok = true;
            for (long long tile = blockIdx.x; tile < ntiles && ok && !*s_abort; tile += gridDim.x, ++t) {
                const int b = (int)(t & 1);
                if (t >= 2 && !tc_bar_wait(&acce[b], (uint32_t)(((t / 2) - 1) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dacc = tmem + (uint32_t)(b * N);
                for (int c = 0; c < nchunks; ++c, ++j) {
                    const int s = (int)(j % stages);
                    if (!tc_bar_wait(&full[s], (uint32_t)((j / stages) & 1))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t aA = smem_addr(sA + (size_t)s * TC_ASTRIDE);
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int dy = tap / 3, dx = tap % 3;  // halo row and column offset of the view
#pragma unroll
                        for (int kk = 0; kk < TC_KC / 16; ++kk) {
                            const uint64_t da = tc_mdesc(
                                aA + (uint32_t)(2 * kk * TC_KG + (dy * TC_HROW + TC_BODY - 1 + dx) * 16), TC_KG, 128);
                            const uint64_t db = tc_mdesc(
                                aW + (uint32_t)tap * wplane + (uint32_t)((c * (TC_KC / 8) + 2 * kk) * 128), 128,
                                (uint32_t)SBO_W);
                            const uint32_t accum = (c > 0 || tap > 0 || kk > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc),
                                "l"(da), "l"(db), "r"(IDESC), "r"(accum)
                                : "memory");
                        }
                    }
                    // the stage is free again once these MMAs have read it
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_addr(&empty[s]))
                        : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_addr(&accf[b]))
                             : "memory");
            }
            if (!ok) {
                *s_abort = 1;
                if (a.err) atomicOr(a.err, 1 << 6);
            }
            // every MMA this thread issued has completed before TMEM is released
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(mdone))
                         : "memory");
            if (!tc_bar_wait(mdone, 0u) && a.err) atomicOr(a.err, 1 << 6);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue (warps 1-4)
        const int q = warp & 3;                  // TMEM lanes 32 q .. 32 q + 31
        const int px = q * 32 + lane;            // pixel of the tile
        long long t = 0;
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++t) {
            const int b = (int)(t & 1);
            // one decision per warp (the TMEM loads below are warp-wide)
            if (!__all_sync(0xffffffffu, tc_bar_wait(&accf[b], (uint32_t)((t / 2) & 1)))) {
                *s_abort = 1;
                if (a.err) atomicOr(a.err, 1 << 6);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int seg = (int)(tile % segs);
            const long long r = tile / segs;
            const int y = (int)(r % H);
            const int n = (int)(r / H);
            const int x = seg * TC_M + px;
            const long long m = ((long long)n * H + y) * W + x;
#pragma unroll
            for (int cc = 0; cc < N; cc += 32) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * N + cc);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                      "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                      "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j8 = 0; j8 < 4; ++j8) {
                    const int co = cc + j8 * 8;
                    float f8[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) f8[k] = __uint_as_float(v[j8 * 8 + k]);
                    if (a.bias) {
                        const float4 b0 = *reinterpret_cast<const float4*>(a.bias + co);
                        const float4 b1 = *reinterpret_cast<const float4*>(a.bias + co + 4);
                        f8[0] += b0.x; f8[1] += b0.y; f8[2] += b0.z; f8[3] += b0.w;
                        f8[4] += b1.x; f8[5] += b1.y; f8[6] += b1.z; f8[7] += b1.w;
                    }
                    if (a.relu)
#pragma unroll
                        for (int k = 0; k < 8; ++k) f8[k] = fmaxf(f8[k], 0.0f);
                    if (a.mask) {
                        float mk[8];
                        unpack8(*reinterpret_cast<const uint4*>(a.mask + m * a.mC + a.moff + co), mk);
#pragma unroll
                        for (int k = 0; k < 8; ++k) f8[k] = mk[k] > 0.0f ? f8[k] : 0.0f;
                    }
                    const uint4 u = pack8(f8);
                    if (!a.up) {
                        *reinterpret_cast<uint4*>(a.y + m * a.yC + a.yoff + co) = u;
                    } else {
#pragma unroll
                        for (int uy = 0; uy < 2; ++uy)
#pragma unroll
                            for (int ux = 0; ux < 2; ++ux) {
                                const long long pix = ((long long)n * 2 * H + 2 * y + uy) * (2 * W) + 2 * x + ux;
                                *reinterpret_cast<uint4*>(a.y + pix * a.yC + a.yoff + co) = u;
                            }
                    }
                }
            }
            // this thread has read its lanes of buffer b
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            tc_bar_arrive(&acce[b]);
            if (__any_sync(0xffffffffu, *s_abort != 0)) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc_tmem_cols<N>())
                     : "memory");
}

}  // namespace unk
