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
// tensor copy per group and row, 128-byte aligned; in the activation layout
// of act_at the source is one contiguous 2 KB block, which the tensor map
// moves as 16 rows of 128 bytes) and slots 7 and 136 the
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
//              pixels (cp.async), each arriving on the same barrier when it
//              lands (cp.async.mbarrier.arrive; the MMA thread issues the
//              proxy fence after its wait); the ring is `stages` deep (up
//              to 8) and the producer never waits on its own copies;
//   warp 9     runs the MMA loop warp-wide; one elected lane issues the
//              9 x (32 / 16) MMAs of a stage into the
//              tile's accumulator and tcgen05.commit's the stage's "empty"
//              mbarrier; after the tile's last chunk it commits "acc full";
//   warps 1-8  epilogue, two groups of four warps taking alternate tiles:
//              wait "acc full", tcgen05.ld the tile (TMEM lane =
//              pixel, column = output channel), add the bias, apply ReLU and
//              the gradient mask, round to BF16 and store (or store each
//              pixel to its 2 x 2 block for the upsampling), then arrive on
//              "acc empty".
// TC_NACC accumulator buffers (TC_NACC x N TMEM columns, allocated once per
// CTA) let the MMAs of the next tiles run while the epilogue drains earlier
// ones; the bias sits in shared memory.
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
constexpr int TC_THREADS = 320;                 // producer warp, 2 x 4 epilogue warps, MMA warp
constexpr int TC_NACC = 4;                      // accumulator buffers in TMEM
constexpr int TC_MMA_WARP = 9;
constexpr int TC_MAX_WBYTES = 100 * 1024;       // resident weights per layer
constexpr size_t TC_SMEM_LIMIT = 232448;        // dynamic shared memory per CTA
constexpr long long TC_WAIT = 2000000000LL;     // bounded-wait limit (clock cycles)

__host__ __device__ constexpr size_t tc_wbytes(int N, int Cin) { return (size_t)9 * N * Cin * 2; }
__host__ __device__ constexpr size_t tc_fixed_bytes(int N, int Cin) {
    // weights (rounded to 1 KB), bias, barriers + TMEM slot + flag, alignment slack
    return (tc_wbytes(N, Cin) + 1023) / 1024 * 1024 + 1024 + 512 + 1024;
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
// One stage of the halo, issued by one elected lane of the (converged)
// producer warp: arm the stage's barrier with TC_TMA_BYTES, then the 12 tensor
// copies (channel group g = 0..3 of the chunk starting at group cg0, halo row
// hr = 0..2 of image rows r0, r1, r2; 128 pixels from 8 xb) into the stage at
// st: group g, row hr -> st + g TC_KG + (hr TC_HROW + TC_BODY) 16.
static_assert(TC_KC == 32 && TC_KG == 6912 && TC_HROW == 144 && TC_BODY == 8, "offsets below");
__device__ __forceinline__ void tc_produce_stage(const CUtensorMap* map, uint32_t st, uint32_t bar, int xb, int cg0,
                                                 int r0, int r1, int r2) {
    asm volatile(
        "{\n"
        ".reg .pred e;\n .reg .b32 el, d, c, z;\n"
        "mov.u32 z, 0;\n"
        "elect.sync el|e, 0xffffffff;\n"
        "@e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%2], %3;\n"
        "add.u32 d, %1, 128;\n add.u32 c, %5, 0;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %6}], [%2];\n"
        "add.u32 d, %1, 2432;\n add.u32 c, %5, 0;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %7}], [%2];\n"
        "add.u32 d, %1, 4736;\n add.u32 c, %5, 0;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %8}], [%2];\n"
        "add.u32 d, %1, 7040;\n add.u32 c, %5, 1;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %6}], [%2];\n"
        "add.u32 d, %1, 9344;\n add.u32 c, %5, 1;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %7}], [%2];\n"
        "add.u32 d, %1, 11648;\n add.u32 c, %5, 1;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %8}], [%2];\n"
        "add.u32 d, %1, 13952;\n add.u32 c, %5, 2;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %6}], [%2];\n"
        "add.u32 d, %1, 16256;\n add.u32 c, %5, 2;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %7}], [%2];\n"
        "add.u32 d, %1, 18560;\n add.u32 c, %5, 2;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %8}], [%2];\n"
        "add.u32 d, %1, 20864;\n add.u32 c, %5, 3;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %6}], [%2];\n"
        "add.u32 d, %1, 23168;\n add.u32 c, %5, 3;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %7}], [%2];\n"
        "add.u32 d, %1, 25472;\n add.u32 c, %5, 3;\n"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [d], [%0, {z, %4, c, %8}], [%2];\n"
        "}\n" ::"l"(reinterpret_cast<uint64_t>(map)),
        "r"(st), "r"(bar), "r"((uint32_t)TC_TMA_BYTES), "r"(xb), "r"(cg0), "r"(r0), "r"(r1), "r"(r2)
        : "memory");
}

// arrive on an mbarrier once all of this thread's prior cp.async copies have
// landed (the arrival counts towards the barrier's expected count)
__device__ __forceinline__ void tc_cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// nine MMAs into accumulator d, issued by one elected lane of the (converged)
// warp: view i has the descriptors {alo[i], ahi} and {blo[i], bhi}; the first
// accumulates onto d iff acc0 != 0, the rest always
__device__ __forceinline__ void tc_mma9(uint32_t d, uint32_t idesc, const uint32_t (&alo)[9], uint32_t ahi,
                                        const uint32_t (&blo)[9], uint32_t bhi, uint32_t acc0) {
    asm volatile(
        "{\n"
        ".reg .pred p0, p1, e;\n"
        ".reg .b32 el;\n"
        ".reg .b64 a0, a1, a2, a3, a4, a5, a6, a7, a8, b0, b1, b2, b3, b4, b5, b6, b7, b8;\n"
        "setp.ne.b32 p0, %22, 0;\n"
        "setp.eq.b32 p1, %1, %1;\n"
        "elect.sync el|e, 0xffffffff;\n"
        "mov.b64 a0, {%2, %11};\n mov.b64 a1, {%3, %11};\n mov.b64 a2, {%4, %11};\n"
        "mov.b64 a3, {%5, %11};\n mov.b64 a4, {%6, %11};\n mov.b64 a5, {%7, %11};\n"
        "mov.b64 a6, {%8, %11};\n mov.b64 a7, {%9, %11};\n mov.b64 a8, {%10, %11};\n"
        "mov.b64 b0, {%12, %21};\n mov.b64 b1, {%13, %21};\n mov.b64 b2, {%14, %21};\n"
        "mov.b64 b3, {%15, %21};\n mov.b64 b4, {%16, %21};\n mov.b64 b5, {%17, %21};\n"
        "mov.b64 b6, {%18, %21};\n mov.b64 b7, {%19, %21};\n mov.b64 b8, {%20, %21};\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a0, b0, %1, p0;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %1, p1;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a2, b2, %1, p1;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a3, b3, %1, p1;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a4, b4, %1, p1;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a5, b5, %1, p1;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a6, b6, %1, p1;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a7, b7, %1, p1;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a8, b8, %1, p1;\n"
        "}\n" ::"r"(d),
        "r"(idesc), "r"(alo[0]), "r"(alo[1]), "r"(alo[2]), "r"(alo[3]), "r"(alo[4]), "r"(alo[5]), "r"(alo[6]),
        "r"(alo[7]), "r"(alo[8]), "r"(ahi), "r"(blo[0]), "r"(blo[1]), "r"(blo[2]), "r"(blo[3]), "r"(blo[4]),
        "r"(blo[5]), "r"(blo[6]), "r"(blo[7]), "r"(blo[8]), "r"(bhi), "r"(acc0)
        : "memory");
}

// tcgen05.commit from one elected lane of the (converged) warp: the mbarrier
// receives one arrival once every MMA issued before it has completed
__device__ __forceinline__ void tc_commit_one(uint64_t* bar) {
    asm volatile(
        "{\n .reg .pred e;\n .reg .b32 el;\n elect.sync el|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(smem_addr(bar))
        : "memory");
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
    return TC_NACC * N <= 64 ? 64u : (TC_NACC * N <= 128 ? 128u : (TC_NACC * N <= 256 ? 256u : 512u));
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
    float* sBias = reinterpret_cast<float*>(sA + (size_t)stages * TC_ASTRIDE);  // [N <= 96]
    uint64_t* full = reinterpret_cast<uint64_t*>(sBias + 128);
    uint64_t* empty = full + TC_MAX_STAGES;
    uint64_t* accf = empty + TC_MAX_STAGES;   // [TC_NACC]
    uint64_t* acce = accf + TC_NACC;          // [TC_NACC]
    uint64_t* mdone = acce + TC_NACC;         // the MMA thread's last commit
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(mdone + 1);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int H = a.H, W = a.W;
    const int segs = W / TC_M;
    const int ntiles = a.N * H * segs;  // the host keeps this below 2^31
    const int nchunks = Cin / TC_KC;
    const int SBO_W = (Cin / 8) * 128;                  // weights: 8-row (output channel) groups
    const uint32_t wplane = (uint32_t)N * (uint32_t)Cin * 2u;

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            tc_bar_init(&full[s], 1 + TC_EDGES);     // the armed byte count + the edge copies
            tc_bar_init(&empty[s], 1);
        }
        for (int b = 0; b < TC_NACC; ++b) {
            tc_bar_init(&accf[b], 1);
            tc_bar_init(&acce[b], 128);    // the four warps of the epilogue group of the tile
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
    for (int q = tid; q < N; q += TC_THREADS) sBias[q] = a.bias ? a.bias[q] : 0.0f;
    cp_async_commit();
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        // ------------------------------------------------ producer warp
        // this lane's edge pixel: channel group g, halo row hr, side (0 left, 1 right)
        const int eg = lane / 6, ehr = (lane % 6) >> 1, eside = lane & 1;
        const bool edge = lane < TC_EDGES;
        int j = 0, s = 0;                                // jobs issued, their stage
        uint32_t ph = 0;                                 // (j / stages) & 1
        // (the abort flag is read once per warp: every decision here is warp-uniform)
        for (int tile = blockIdx.x; tile < ntiles && __shfl_sync(0xffffffffu, *s_abort, 0) == 0;
             tile += gridDim.x) {
            const int seg = tile % segs;
            const int r = tile / segs;
            const int y = r % H;
            const int n = r / H;
            const int x0 = seg * TC_M;
            const int rr0 = n * H + wrap(y - 1, H), rr1 = n * H + y, rr2 = n * H + wrap(y + 1, H);
            bool stop = false;
            for (int c = 0; c < nchunks; ++c) {
                // one decision per warp (its lanes poll the barrier independently)
                if (j >= stages && !__all_sync(0xffffffffu, tc_bar_wait(&empty[s], ph ^ 1u))) {
                    if (lane == 0) {
                        *s_abort = 1;
                        if (a.err) atomicOr(a.err, 1 << 6);
                    }
                    stop = true;
                    break;
                }
                uint8_t* st = sA + (size_t)s * TC_ASTRIDE;
                const int cbase = a.xoff + c * TC_KC;
                tc_produce_stage(&xmap, smem_addr(st), smem_addr(&full[s]), x0 / 8, cbase / 8, rr0, rr1, rr2);
                if (edge) {
                    // the copy arrives on the stage's barrier by itself once it has landed
                    const int yy = wrap(y + ehr - 1, H);
                    const int xx = eside ? wrap(x0 + TC_M, W) : wrap(x0 - 1, W);
                    cp_async16(st + eg * TC_KG + (ehr * TC_HROW + (eside ? TC_BODY + TC_M : TC_BODY - 1)) * 16,
                               a.x + act_at((long long)n * H + yy, xx, cbase + eg * 8, a.xC, W), true);
                    tc_cp_async_arrive(&full[s]);
                }
                ++j;
                if (++s == stages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (stop) break;
        }
        // every copy issued has landed before leaving (the full barriers of
        // the last jobs complete only then; waits with the default limit)
        cp_async_wait<0>();
        if (lane == 0)
            for (int k = (j > stages ? j - stages : 0); k < j; ++k)
                (void)tc_bar_wait(&full[k % stages], (uint32_t)((k / stages) & 1));
        __syncwarp();
    } else if (warp == TC_MMA_WARP) {
        // ------------------------------------------------ MMA issue
        // The whole warp runs this loop (warp-uniform control flow keeps the
        // descriptors in the uniform datapath); one elected lane issues each
        // MMA and commit.  The low word (start address >> 4) of every view
        // of a stage is a constant offset from the stage's base; the high
        // words (LBO, SBO, version) never change.
        constexpr uint32_t IDESC = tc_idesc_n<N>();
        const uint64_t da0 = tc_mdesc(smem_addr(sA) + (uint32_t)((TC_BODY - 1) * 16), TC_KG, 128);
        const uint64_t db0 = tc_mdesc(smem_addr(sW), 128, (uint32_t)SBO_W);
        const uint32_t ahi = (uint32_t)(da0 >> 32), bhi = (uint32_t)(db0 >> 32);
        const uint32_t wp16 = wplane >> 4;
        int s = 0, b = 0, t = 0;
        uint32_t fph = 0, rnd = 0;  // (job / stages) & 1, (t / TC_NACC) & 1
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok && __shfl_sync(0xffffffffu, *s_abort, 0) == 0;
             tile += gridDim.x, ++t) {
            if (t >= TC_NACC && !__all_sync(0xffffffffu, tc_bar_wait(&acce[b], rnd ^ 1u))) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dacc = tmem + (uint32_t)(b * N);
            for (int c = 0; c < nchunks; ++c) {
                // views of tap (dy, dx): halo row dy, slot TC_BODY - 1 + dx; kk = 1 is TC_KG * 2 bytes on
                const uint32_t a_lo = (uint32_t)da0 + (uint32_t)s * (uint32_t)(TC_ASTRIDE >> 4);
                const uint32_t b_lo = (uint32_t)db0 + (uint32_t)c * (uint32_t)((TC_KC / 8) * 128 >> 4);
                uint32_t a0[9], a1[9], b0[9], b1[9];
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    a0[tap] = a_lo + (uint32_t)((tap / 3) * TC_HROW + tap % 3);
                    a1[tap] = a0[tap] + (uint32_t)(2 * TC_KG >> 4);
                    b0[tap] = b_lo + (uint32_t)tap * wp16;
                    b1[tap] = b0[tap] + 16u;
                }
                if (!__all_sync(0xffffffffu, tc_bar_wait(&full[s], fph))) {
                    ok = false;
                    break;
                }
                // the edge pixels were written by cp.async (generic proxy), the
                // MMAs read the stage through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                tc_mma9(dacc, IDESC, a0, ahi, b0, bhi, c > 0 ? 1u : 0u);
                tc_mma9(dacc, IDESC, a1, ahi, b1, bhi, 1u);
                tc_commit_one(&empty[s]);  // the stage is free again once these MMAs have read it
                if (++s == stages) {
                    s = 0;
                    fph ^= 1u;
                }
            }
            if (!ok) break;
            tc_commit_one(&accf[b]);
            if (++b == TC_NACC) {
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
        // two groups of four warps take alternate tiles, so that one group's
        // loads and stores overlap the other's; the k-th tile of group grp is
        // the CTA's tile t = grp + 2 k: buffer t % 4 = grp + 2 (k % 2), phase
        // (t / 4) % 2 = (k / 2) % 2
        const int grp = (warp - 1) >> 2;         // 0: warps 1-4, 1: warps 5-8
        const int q = warp & 3;                  // TMEM lanes 32 q .. 32 q + 31
        const int px = q * 32 + lane;            // pixel of the tile
        int k = 0;
        for (int tile = blockIdx.x + grp * (int)gridDim.x; tile < ntiles; tile += 2 * (int)gridDim.x, ++k) {
            const int b = grp + 2 * (k & 1);
            const uint32_t rnd = (uint32_t)(k >> 1) & 1u;
            const int seg = tile % segs;
            const long long row = tile / segs;   // n H + y
            const int x = seg * TC_M + px;
            // the gradient mask of this pixel, loaded before the accumulator is ready
            uint4 mraw[N / 8];
            if (a.mask)
#pragma unroll
                for (int kk = 0; kk < N / 8; ++kk)
                    mraw[kk] = __ldg(reinterpret_cast<const uint4*>(a.mask + act_at(row, x, a.moff + 8 * kk, a.mC, W)));
            // one decision per warp (the TMEM loads below are warp-wide)
            if (!__all_sync(0xffffffffu, tc_bar_wait(&accf[b], rnd))) {
                *s_abort = 1;
                if (a.err) atomicOr(a.err, 1 << 6);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
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
                    for (int e = 0; e < 8; ++e) f8[e] = __uint_as_float(v[j8 * 8 + e]) + sBias[co + e];
                    if (a.relu)
#pragma unroll
                        for (int e = 0; e < 8; ++e) f8[e] = fmaxf(f8[e], 0.0f);
                    if (a.mask) {
                        float mk[8];
                        unpack8(mraw[co / 8], mk);
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
                                *reinterpret_cast<uint4*>(a.y + act_at(2 * row + uy, 2 * x + ux, a.yoff + co, a.yC,
                                                                       2 * W)) = u;
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
