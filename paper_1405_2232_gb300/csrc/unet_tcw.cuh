// unet_tcw.cuh -- weight (and bias) gradient of the 3x3 circular convolution
// on the tcgen05 tensor cores, for layers with at least 64 output channels
// (levels 1 .. 3 of the network):
//   dW[co][tap][ci] = sum_p g[p][co] x[p + shift_tap][ci],   db[co] = sum_p g[p][co]
// as one GEMM per tap with M = 128 output channels (a block; rows past Cout
// are computed and dropped), N = NBW input channels (a block) and K = pixels.
//
// A CTA owns one output-channel block, one input-channel block, one kernel
// row dy (taps 3 dy .. 3 dy + 2) and a contiguous range of image row segments
// (a split of the pixels; the splits' partial sums are reduced afterwards in
// a fixed order, as for the mma.sync kernel).  With dy fixed, every output row
// y needs exactly one input row, y + dy - 1, so a stage is
//   g: the row segment of the output gradient, MB / 8 channel groups of segw
//      pixels (16 bytes each): group j, pixel p -> j * segw * 16 + p * 16;
//   x: input row y + dy - 1, NBW / 8 channel groups in the halo layout of
//      k_conv3_tc (slots 8 .. 8 + segw - 1, the wrapped neighbours at slots
//      7 and 8 + segw): group k, slot q -> GX + k * TC_HROW * 16 + q * 16.
// Both operands are read MN-major (8 channels of one pixel are one 16-byte
// core-matrix row; 8 pixels of a K step are 128 contiguous bytes): A = g with
// its channel groups segw * 16 bytes apart, B = x with tap dx's view starting
// at slot 7 + dx.  The three accumulators (dx = 0, 1, 2; NBW TMEM columns
// each) stay in TMEM for the CTA's whole range.
//
// With XM (layers with 32 output channels and at least 64 input channels)
// the roles of the operands swap: A = x with M = 128 input channels, B = g
// with N = NA = Cout, so the 128 MMA rows are the wider side (with M = 32
// output channels three quarters of every MMA would be empty); the
// accumulators are D[ci][co] and the partial sums are written with TMEM lane
// = input channel.
//
// Roles: warp 0 produces (elected lane: barrier byte count and the tensor
// copies; lanes: the wrapped neighbours, arriving when they land), warp 5
// issues the MMAs (warp-wide loop, elected lane), warps 1-4 sum g for the bias
// gradient while the MMAs run (CTAs of input block 0 and dy = 1 only; their
// arrivals release the stage together with the MMA commit) and write the
// partial sums at the end (TMEM lane = output channel).  Every wait is bounded
// (bit 6 of *err on a timeout).
#pragma once

#include "unet_tcs.cuh"  // ts_tma, ts_mma1

namespace unk {

constexpr int TW_THREADS = 192;
constexpr int TW_MMA_WARP = 5;
constexpr int TW_MB = 128;

struct WgradTcArgs {
    const bf16* g;  // gradient at the conv output: channels goff .. of a tensor of gC
    int gC, goff;
    const bf16* x;  // conv input: channels xoff .. of a tensor of xC
    int xC, xoff;
    int Cout, Cin, N, H, W;
    int splits, items_per_split;  // row segments per split
    float* part;                  // [splits][Cout][9][Cin]
    float* bpart;                 // [splits][Cout]
    int* err;
};

__host__ __device__ constexpr int tw_segw(int W) { return W < TC_M ? W : TC_M; }
// channel groups staged per stage: g (output channels) and x (input channels)
__host__ __device__ constexpr int tw_gplanes(int NA, bool XM) { return XM ? NA / 8 : TW_MB / 8; }
__host__ __device__ constexpr int tw_xplanes(int NA, bool XM) { return XM ? TW_MB / 8 : NA / 8; }
__host__ __device__ constexpr int tw_gbytes(int NA, bool XM, int segw) { return tw_gplanes(NA, XM) * segw * 16; }
__host__ __device__ constexpr int tw_xbytes(int NA, bool XM) { return tw_xplanes(NA, XM) * TC_HROW * 16; }
__host__ __device__ constexpr int tw_stage_bytes(int NA, bool XM, int segw) {
    return tw_gbytes(NA, XM, segw) + tw_xbytes(NA, XM);
}
__host__ __device__ constexpr int tw_stages(int NA, bool XM, int segw) {
    return (int)((232448 - 1024 - 512) / tw_stage_bytes(NA, XM, segw)) > 6
               ? 6
               : (int)((232448 - 1024 - 512) / tw_stage_bytes(NA, XM, segw));
}
__host__ __device__ constexpr size_t tw_smem_bytes(int NA, bool XM, int segw) {
    return (size_t)tw_stages(NA, XM, segw) * tw_stage_bytes(NA, XM, segw) + 512 + 1024;
}
// input-channel block of a layer (0: not for this kernel)
__host__ __device__ constexpr int tw_block(int Cin) {
    return Cin % 128 == 0 ? 128 : (Cin % 64 == 0 ? 64 : (Cin % 32 == 0 ? 32 : 0));
}

template <int NA, bool XM>
__global__ void __launch_bounds__(TW_THREADS, 1)
    k_wgrad_tc(WgradTcArgs a, const __grid_constant__ CUtensorMap gmap, const __grid_constant__ CUtensorMap xmap,
               int stages) {
    // NA: N of the MMA (input-channel block; with XM the output channels)
    constexpr int NBW = XM ? TW_MB : NA;            // input channels of a block
    constexpr int XG = tw_xplanes(NA, XM);          // input channel groups staged
    constexpr uint32_t COLS = 3 * NA <= 128 ? 128u : (3 * NA <= 256 ? 256u : 512u);
    static_assert(2 * XG <= 32, "one edge copy per producer lane");
    extern __shared__ __align__(1024) uint8_t tw_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tw_raw) + 1023) & ~uintptr_t(1023));
    const int H = a.H, W = a.W;
    const int segw = tw_segw(W);
    const int segs = W / segw;
    const int GB = tw_gbytes(NA, XM, segw);
    const int SB = GB + tw_xbytes(NA, XM);
    uint8_t* sS = base;                                                     // [stages][SB]
    uint64_t* full = reinterpret_cast<uint64_t*>(sS + (size_t)stages * SB);  // [stages]
    uint64_t* empty = full + 6;                                             // [stages]
    uint64_t* mdone = empty + 6;
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(mdone + 1);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // unit: output block, input block, dy, split (split outermost: the CTAs
    // working on the same pixels run together)
    const int ncob = XM ? 1 : (a.Cout + TW_MB - 1) / TW_MB;
    const int ncib = (a.Cin + NBW - 1) / NBW;
    int u = blockIdx.x;
    const int cob = u % ncob;
    u /= ncob;
    const int cib = u % ncib;
    u /= ncib;
    const int dy = u % 3;
    const int split = u / 3;
    const int items = a.N * H * segs;
    const int it0 = split * a.items_per_split;
    const int it1 = min(it0 + a.items_per_split, items);
    const int nitems = it1 > it0 ? it1 - it0 : 0;
    const bool do_bias = cib == 0 && dy == 1;
    const int cg0 = (a.goff + cob * TW_MB) / 8;         // first g channel group of the block
    const int gvalid = XM ? a.Cout / 8 : min(TW_MB, a.Cout - cob * TW_MB) / 8;  // g groups that exist
    const int xg0 = (a.xoff + cib * NBW) / 8;
    const int xvalid = min(NBW, a.Cin - cib * NBW) / 8;  // x groups that exist
    const int EDGES = 2 * xvalid;                        // wrapped neighbours per stage

    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            tc_bar_init(&full[s], 1 + EDGES);
            tc_bar_init(&empty[s], do_bias ? 1 + 4 : 1);
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
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        // ------------------------------------------------ producer
        const int ek = lane >> 1, eside = lane & 1;  // edge: input group, side
        const bool edge = lane < EDGES;
        int s = 0;
        uint32_t ph = 0;
        int j = 0;
        for (int i = 0; i < nitems && __shfl_sync(0xffffffffu, *s_abort, 0) == 0; ++i, ++j) {
            const int item = it0 + i;
            const int seg = item % segs;
            const int row = item / segs;  // n H + y
            const int y = row % H, n = row / H;
            const int xrow = n * H + wrap(y + dy - 1, H);
            const int x0 = seg * segw;
            if (j >= stages && !__all_sync(0xffffffffu, tc_bar_wait(&empty[s], ph ^ 1u))) {
                if (lane == 0) {
                    *s_abort = 1;
                    if (a.err) atomicOr(a.err, 1 << 6);
                }
                break;
            }
            const uint32_t st = smem_addr(sS + (size_t)s * SB);
            const uint32_t fb = smem_addr(&full[s]);
            {
                // arm with every byte of the stage's tensor copies
                const uint32_t bytes = (uint32_t)((gvalid + xvalid) * segw * 16);
                asm volatile(
                    "{\n .reg .pred e;\n .reg .b32 el;\n elect.sync el|e, 0xffffffff;\n"
                    " @e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n}\n" ::"r"(fb),
                    "r"(bytes)
                    : "memory");
            }
            for (int k = 0; k < gvalid; ++k) ts_tma(&gmap, st + k * segw * 16, fb, x0 / 8, cg0 + k, row);
            for (int k = 0; k < xvalid; ++k)
                ts_tma(&xmap, st + GB + (k * TC_HROW + TC_BODY) * 16, fb, x0 / 8, xg0 + k, xrow);
            if (edge) {
                const int xx = eside ? wrap(x0 + segw, W) : wrap(x0 - 1, W);
                cp_async16(sS + (size_t)s * SB + GB + (ek * TC_HROW + (eside ? TC_BODY + segw : TC_BODY - 1)) * 16,
                           a.x + act_at(xrow, xx, (xg0 + ek) * 8, a.xC, W), true);
                tc_cp_async_arrive(&full[s]);
            }
            if (++s == stages) {
                s = 0;
                ph ^= 1u;
            }
        }
        cp_async_wait<0>();
        if (lane == 0)
            for (int k = (j > stages ? j - stages : 0); k < j; ++k)
                (void)tc_bar_wait(&full[k % stages], (uint32_t)((k / stages) & 1));
        __syncwarp();
    } else if (warp == TW_MMA_WARP) {
        // ------------------------------------------------ MMA issue
        // kind::f16, D FP32, A and B BF16, both MN-major (bits 15, 16)
        constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                   ((uint32_t)(NA >> 3) << 17) | ((uint32_t)(TW_MB >> 4) << 24);
        // no-swizzle MN-major operands: the leading byte offset is the stride
        // between K groups (8 pixels: 128 bytes), the stride byte offset the
        // stride between MN groups (8 channels)
        // g: channel groups segw * 16 bytes apart
        const uint64_t dg0 = tc_mdesc(smem_addr(sS), 128, (uint32_t)(segw * 16));
        // x: channel groups one halo row (TC_HROW * 16 bytes) apart
        const uint64_t dx0 = tc_mdesc(smem_addr(sS) + (uint32_t)(GB + (TC_BODY - 1) * 16), 128, TC_HROW * 16);
        const uint64_t da0 = XM ? dx0 : dg0, db0 = XM ? dg0 : dx0;
        const uint32_t ahi = (uint32_t)(da0 >> 32), bhi = (uint32_t)(db0 >> 32);
        const int ksteps = segw / 16;
        int s = 0;
        uint32_t fph = 0;
        bool ok = true;
        for (int i = 0; i < nitems && __shfl_sync(0xffffffffu, *s_abort, 0) == 0; ++i) {
            const uint32_t a_lo = (uint32_t)da0 + (uint32_t)s * (uint32_t)(SB >> 4);
            const uint32_t b_lo = (uint32_t)db0 + (uint32_t)s * (uint32_t)(SB >> 4);
            if (!__all_sync(0xffffffffu, tc_bar_wait(&full[s], fph))) {
                ok = false;
                break;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int k = 0; k < ksteps; ++k) {
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
                    // the x view of tap dx starts dx slots further
                    ts_mma1(tmem + (uint32_t)(dx * NA), a_lo + (uint32_t)((XM ? dx : 0) + k * 16), ahi,
                            b_lo + (uint32_t)((XM ? 0 : dx) + k * 16), bhi, IDESC, (i > 0 || k > 0) ? 1u : 0u);
            }
            tc_commit_one(&empty[s]);
            if (++s == stages) {
                s = 0;
                fph ^= 1u;
            }
        }
        if (!ok && lane == 0) {
            *s_abort = 1;
            if (a.err) atomicOr(a.err, 1 << 6);
        }
        tc_commit_one(mdone);  // arrives once every MMA issued has completed
    } else {
        // ------------------------------------------------ warps 1-4: bias sums, then the partials
        const int q = warp & 3;  // TMEM lanes 32 q ..; bias: g groups 4 q .. 4 q + 3
        float bs[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) bs[k] = 0.0f;
        if (do_bias) {
            int s = 0;
            uint32_t fph = 0;
            for (int i = 0; i < nitems; ++i) {
                if (!__all_sync(0xffffffffu, tc_bar_wait(&full[s], fph))) {
                    if (lane == 0) {
                        *s_abort = 1;
                        if (a.err) atomicOr(a.err, 1 << 6);
                    }
                    break;
                }
                const uint8_t* gst = sS + (size_t)s * SB;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int k = 4 * q + jj;
                    if (k < gvalid)
                        for (int p = lane; p < segw; p += 32) {
                            float f[8];
                            unpack8(*reinterpret_cast<const uint4*>(gst + k * segw * 16 + p * 16), f);
#pragma unroll
                            for (int e = 0; e < 8; ++e) bs[jj * 8 + e] += f[e];
                        }
                }
                __syncwarp();
                if (lane == 0) tc_bar_arrive(&empty[s]);
                if (++s == stages) {
                    s = 0;
                    fph ^= 1u;
                }
                if (__any_sync(0xffffffffu, *s_abort != 0)) break;
            }
            // lane sums -> the warp's 32 channels (fixed order)
#pragma unroll
            for (int k = 0; k < 32; ++k)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) bs[k] += __shfl_xor_sync(0xffffffffu, bs[k], o);
            const int co = cob * TW_MB + 32 * q + lane;
            if (32 * q + lane < gvalid * 8) {
                float v = 0.0f;
#pragma unroll
                for (int k = 0; k < 32; ++k) v = (k == lane) ? bs[k] : v;
                a.bpart[(long long)split * a.Cout + co] = v;
            }
        }
        // wait for the last MMAs, then TMEM lane (32 q + lane) = output
        // channel (with XM: input channel)
        const bool done = __all_sync(0xffffffffu, tc_bar_wait(mdone, 0u));
        if (!done && lane == 0 && a.err) atomicOr(a.err, 1 << 6);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int col = 32 * q + lane;
        const int co = cob * TW_MB + col;
        const bool valid = col < (XM ? xvalid : gvalid) * 8 && nitems > 0 && done;
        float* out = XM ? a.part + (long long)split * a.Cout * 9 * a.Cin + cib * NBW + col
                        : a.part + ((long long)split * a.Cout + co) * 9 * a.Cin;
#pragma unroll 1
        for (int dx = 0; dx < 3; ++dx) {
            const int tap = dy * 3 + dx;
#pragma unroll 1
            for (int cc = 0; cc < NA; cc += 32) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(dx * NA + cc);
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
                if (valid && XM) {
                    // column j = output channel cc + j: [co][tap][ci], this lane's ci
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        out[((long long)(cc + j) * 9 + tap) * a.Cin] = __uint_as_float(v[j]);
                } else if (valid) {
                    float4* o4 = reinterpret_cast<float4*>(out + (long long)tap * a.Cin + cib * NBW + cc);
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        o4[k] = make_float4(__uint_as_float(v[4 * k]), __uint_as_float(v[4 * k + 1]),
                                            __uint_as_float(v[4 * k + 2]), __uint_as_float(v[4 * k + 3]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
}

}  // namespace unk
