// unet.cu -- host side of the warm-start network (include/unet.h).
//
// Buffers (BF16 in the row-blocked channel-group layout of act_at, sized for
// max_batch; level l has H>>l x W>>l pixels and C_l = base << l channels):
//   x0            padded input, 32 channels
//   a[l]          first encoder conv output, l = 0..3
//   cat[l]        l = 0..2: channels [0, C_{l+1}) the upsampled output of the
//                 level below (written 2x2 by that conv's epilogue), channels
//                 [C_{l+1}, C_{l+1} + C_l) the skip (second encoder conv of l)
//   p[l]          2x2 average pool of skip l (input of level l + 1)
//   c[l]          first decoder conv output, d0 the head input
// and a gradient buffer for each, plus gup[l] (l = 1..3) and gs[l] (l = 0..2).
// Weight gradients come from the split-pixel wgrad kernel and a fixed-order
// sum, so the gradient is deterministic.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "tensor_map.h"
#include "lb.h"
#include "unet.h"
#include "unet_kernels.cuh"
#include "unet_tc.cuh"
#include "unet_tcs.cuh"
#include "unet_tcw.cuh"

namespace lbgb {
lb_status record_error(lb_status st, const char* msg);
}

using unk::bf16;
using lbgb::tensor_map_encoder;

namespace {

lb_status uerr(lb_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
lb_status uerr(lb_status st, const char* fmt, ...) {
    char msg[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    return lbgb::record_error(st, msg);
}

lb_status ucuda(cudaError_t e, const char* what) {
    return uerr(e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define UCU(call, what)                                 \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return ucuda(e_, what);  \
    } while (0)

struct Layer {
    int cin, cout, k;
    long long woff, boff;  // FP32 flat offsets
    long long qoff;        // offset of its BF16 copies (3x3 layers)
};

bool valid_cfg(const un_config* c) {
    return c && c->H >= 8 && c->W >= 8 && c->H % 8 == 0 && c->W % 8 == 0 && c->max_batch >= 1 &&
           c->base >= 32 && c->base % 32 == 0 && c->base <= 256;
}

// layer table in the flat order e0a e0b ... e3b d2a d2b d1a d1b d0a d0b head
int layer_table(const un_config* c, Layer* L) {
    const int C = c->base;
    int n = 0;
    int cin = UN_IN_PAD;
    for (int l = 0; l < UN_LEVELS; ++l) {
        L[n++] = Layer{cin, C << l, 3, 0, 0, 0};
        L[n++] = Layer{C << l, C << l, 3, 0, 0, 0};
        cin = C << l;
    }
    for (int l = UN_LEVELS - 2; l >= 0; --l) {
        L[n++] = Layer{(C << (l + 1)) + (C << l), C << l, 3, 0, 0, 0};
        L[n++] = Layer{C << l, C << l, 3, 0, 0, 0};
    }
    L[n++] = Layer{C, UN_OUT, 1, 0, 0, 0};
    long long o = 0, q = 0;
    for (int k = 0; k < n; ++k) {
        L[k].woff = o;
        o += (long long)L[k].cout * L[k].k * L[k].k * L[k].cin;
        L[k].boff = o;
        o += L[k].cout;
        L[k].qoff = q;
        if (L[k].k == 3) q += (long long)L[k].cout * 9 * L[k].cin;
    }
    return n;
}

// indices into the layer table
inline int LE(int l, int b) { return 2 * l + b; }                       // encoder l, conv a (0) / b (1)
inline int LD(int l, int b) { return 2 * UN_LEVELS + 2 * (UN_LEVELS - 2 - l) + b; }  // decoder l
constexpr int LHEAD = UN_LAYERS - 1;

}  // namespace

struct un_net {
    un_config cfg;
    int device = 0;
    int sms = 152;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Layer L[UN_LAYERS];
    long long nparam = 0, nq = 0;
    float *p = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    bf16 *wb = nullptr, *wt = nullptr;
    bf16 *wbk = nullptr, *wtk = nullptr;  // wb, wt blocked per stage of k_conv3_tcs (layers it takes)
    long long t = 0;
    int lastN = 0;
    // forward
    bf16* x0 = nullptr;
    bf16* a[UN_LEVELS] = {};
    bf16* cat[UN_LEVELS - 1] = {};
    bf16* pl[UN_LEVELS - 1] = {};
    bf16* c[UN_LEVELS - 1] = {};
    bf16* d0 = nullptr;
    float* y = nullptr;
    // backward
    bf16* gd0 = nullptr;
    bf16* ga[UN_LEVELS] = {};
    bf16* gcat[UN_LEVELS - 1] = {};
    bf16* gp[UN_LEVELS - 1] = {};
    bf16* gc[UN_LEVELS - 1] = {};
    bf16* gup[UN_LEVELS] = {};   // index 1..3
    bf16* gs[UN_LEVELS - 1] = {};
    // reductions
    float* wpart = nullptr;
    long long wpart_cap = 0;
    float* bpart = nullptr;   // [1024][256]
    float* hpart = nullptr;   // [hblocks][2C + 2]
    double* lpart = nullptr;  // [hblocks]
    double* d_loss = nullptr;
    int* d_err = nullptr;     // sticky error word of the tcgen05 convolution
    int hblocks = 0;
    std::vector<void*> allocs;
};

namespace {

inline int Hl(const un_net* n, int l) { return n->cfg.H >> l; }
inline int Wl(const un_net* n, int l) { return n->cfg.W >> l; }
inline int Cl(const un_net* n, int l) { return n->cfg.base << l; }
inline long long Pl(const un_net* n, int l, int N) { return (long long)N * Hl(n, l) * Wl(n, l); }

void release(un_net* n) {
    if (!n) return;
    cudaSetDevice(n->device);
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (void* p : n->allocs) cudaFree(p);
    if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
    delete n;
}

template <typename T>
cudaError_t alloc(un_net* n, T** p, long long count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (size_t)count * sizeof(T) > 0 ? (size_t)count * sizeof(T) : 16);
    if (e == cudaSuccess) n->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return e;
}

int grid_for(long long work, int per_block = 256) {
    long long b = (work + per_block - 1) / per_block;
    return (int)(b < 1 ? 1 : (b > 1 << 20 ? 1 << 20 : b));
}

// blocks of k_sum_splits for n outputs (32 per block, grid-stride beyond)
int sum_grid(long long n) {
    const long long b = (n + 31) / 32;
    return (int)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

// splits of the weight-gradient kernel for a layer at M pixels
void wgrad_shape(const un_net* n, const Layer& L, long long M, int* MT, int* NT, int* tiles, int* splits,
                 int* cps) {
    *MT = L.cout % 64 ? 32 : 64;
    *NT = L.cin % 64 ? 32 : 64;
    *tiles = (L.cout / *MT) * (L.cin / *NT) * 9;
    const long long nchunks = (M + 31) / 32;
    long long s = (4LL * n->sms + *tiles - 1) / *tiles;
    const long long smax = nchunks / 8 > 0 ? nchunks / 8 : 1;
    if (s > smax) s = smax;
    if (s < 1) s = 1;
    const long long c = (nchunks + s - 1) / s;
    *cps = (int)c;
    *splits = (int)((nchunks + c - 1) / c);
}

// Tensor map of a BF16 activation tensor (layout of act_at) for k_conv3_tc:
// dims (64 values = 8 pixels x 8 channels, W / 8 pixel blocks, xC / 8
// channel groups, N H rows), box (64, 16, 1, 1): one box is 128 pixels of one
// channel group of one row, a contiguous 2 KB block moved as 16 rows of 128
// bytes.  The view's first channel group is applied in the coordinates.
bool conv_tensor_map(const bf16* x, int xC, int W, int H, int N, CUtensorMap* map, int boxw = unk::TC_M) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[4] = {64, (cuuint64_t)(W / 8), (cuuint64_t)(xC / 8), (cuuint64_t)N * H};
    const cuuint64_t strides[3] = {128, (cuuint64_t)W * 16, (cuuint64_t)xC * W * 2};
    const cuuint32_t box[4] = {64, (cuuint32_t)boxw / 8, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(x), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the stage images of k_conv3_tcs for weights w (a layer's copy in wb or wt)
const bf16* blocked_of(const un_net* n, const bf16* w) {
    if (w >= n->wb && w < n->wb + n->nq) return n->wbk + (w - n->wb);
    if (w >= n->wt && w < n->wt + n->nq) return n->wtk + (w - n->wt);
    return nullptr;
}

cudaError_t conv(un_net* n, const bf16* x, int xC, int xoff, int Cin, const bf16* w, const float* bias, int Cout,
                 bf16* y, int yC, int yoff, const bf16* mask, int mC, int moff, int N, int l, int relu, int up) {
    unk::ConvArgs a;
    a.x = x;
    a.xC = xC;
    a.xoff = xoff;
    a.Cin = Cin;
    a.w = w;
    a.bias = bias;
    a.Cout = Cout;
    a.y = y;
    a.yC = yC;
    a.yoff = yoff;
    a.mask = mask;
    a.mC = mC;
    a.moff = moff;
    a.N = N;
    a.H = Hl(n, l);
    a.W = Wl(n, l);
    a.relu = relu;
    a.up = up;
    a.err = n->d_err;
    const long long M = (long long)N * a.H * a.W;
    CUtensorMap xmap;
    if (a.W % unk::TC_M == 0 && M / unk::TC_M < (1LL << 31) && unk::tc_layer_ok(Cout, Cin) &&
        conv_tensor_map(x, xC, a.W, a.H, N, &xmap)) {
        // fifth-generation tensor cores: persistent CTAs, one per SM at most
        const long long tiles = (long long)N * a.H * (a.W / unk::TC_M);
        const int grid = (int)(tiles < n->sms ? tiles : n->sms);
        const size_t smem = unk::tc_smem_bytes(Cout, Cin);
        const int stages = unk::tc_stages(Cout, Cin);
        switch (Cout) {
            case 32: unk::k_conv3_tc<32><<<grid, unk::TC_THREADS, smem, n->stream>>>(a, xmap, stages); break;
            case 64: unk::k_conv3_tc<64><<<grid, unk::TC_THREADS, smem, n->stream>>>(a, xmap, stages); break;
            default: unk::k_conv3_tc<96><<<grid, unk::TC_THREADS, smem, n->stream>>>(a, xmap, stages); break;
        }
        return cudaGetLastError();
    }
    const int NB = unk::ts_block(Cout);
    const int segw = a.W < unk::TC_M ? a.W : unk::TC_M;
    const bf16* wimg = blocked_of(n, w);
    if (NB && wimg && Cin % 16 == 0 && Cout <= 384 && a.W % 16 == 0 && a.W % segw == 0 &&
        a.H % unk::ts_rows(NB) == 0 && (M / segw) * (Cout / NB) < (1LL << 31) &&
        conv_tensor_map(x, xC, a.W, a.H, N, &xmap, segw)) {
        // fifth-generation tensor cores, weights streamed per 16-channel chunk
        const long long tiles = (M / segw) / unk::ts_rows(NB) * (Cout / NB);
        const int grid = (int)(tiles < n->sms ? tiles : n->sms);
        if (NB == 128)
            unk::k_conv3_tcs<128><<<grid, unk::TS_THREADS, unk::ts_smem_bytes(128), n->stream>>>(a, xmap, wimg);
        else
            unk::k_conv3_tcs<64><<<grid, unk::TS_THREADS, unk::ts_smem_bytes(64), n->stream>>>(a, xmap, wimg);
        return cudaGetLastError();
    }
    if (a.W % unk::HT_W == 0 && a.H % unk::HT_H == 0 && Cout % unk::HT_NT == 0) {
        // halo-tile form: one staged input halo serves all nine taps
        const unsigned tiles = (unsigned)((long long)N * (a.H / unk::HT_H) * (a.W / unk::HT_W));
        unk::k_conv3_halo<<<dim3(tiles, Cout / unk::HT_NT), 256, unk::halo_smem_bytes(), n->stream>>>(a);
        return cudaGetLastError();
    }
    const unsigned gx = (unsigned)((M + unk::CV_MT - 1) / unk::CV_MT);
    if (Cout % 64 == 0)
        unk::k_conv3<64><<<dim3(gx, Cout / 64), 256, 0, n->stream>>>(a);
    else
        unk::k_conv3<32><<<dim3(gx, Cout / 32), 256, 0, n->stream>>>(a);
    return cudaGetLastError();
}

// weight and bias gradient of layer k: g (gradient at its output) and x (its input)
cudaError_t wgrad(un_net* n, int k, const bf16* g, int gC, int goff, const bf16* x, int xC, int xoff, int N, int l) {
    const Layer& L = n->L[k];
    const long long M = Pl(n, l, N);
    const long long nw = (long long)L.cout * 9 * L.cin;
    // the swapped orientation (M = input channels) for 32 output channels
    // and at least 64 input channels; otherwise M = output channels
    const bool xm = L.cout == 32 && L.cin >= 64 && L.cin % 32 == 0;
    const int NBW = xm ? unk::TW_MB : unk::tw_block(L.cin);
    const int W = Wl(n, l), H = Hl(n, l);
    const int segw = unk::tw_segw(W);
    CUtensorMap gmap, xmap;
    if ((xm || (L.cout % 64 == 0 && L.cout <= 384 && NBW)) && W % 16 == 0 && W % segw == 0 &&
        M / segw < (1LL << 30) && conv_tensor_map(g, gC, W, H, N, &gmap, segw) &&
        conv_tensor_map(x, xC, W, H, N, &xmap, segw)) {
        // fifth-generation tensor cores: (output block, input block, kernel row, pixel split) per CTA
        const int units = (xm ? 1 : (L.cout + unk::TW_MB - 1) / unk::TW_MB) * ((L.cin + NBW - 1) / NBW) * 3;
        const long long items = M / segw;
        long long S = n->sms / units;
        if (S < 1) S = 1;
        if (S > items) S = items;
        const long long cap = n->wpart_cap / nw;
        if (S > cap) S = cap;
        if (S > 1024LL * 256 / L.cout) S = 1024LL * 256 / L.cout;
        if (S >= 1) {
            const long long per = (items + S - 1) / S;
            const int splits = (int)((items + per - 1) / per);
            unk::WgradTcArgs a;
            a.g = g;
            a.gC = gC;
            a.goff = goff;
            a.x = x;
            a.xC = xC;
            a.xoff = xoff;
            a.Cout = L.cout;
            a.Cin = L.cin;
            a.N = N;
            a.H = H;
            a.W = W;
            a.splits = splits;
            a.items_per_split = (int)per;
            a.part = n->wpart;
            a.bpart = n->bpart;
            a.err = n->d_err;
            const int na = xm ? 32 : NBW;
            const int stages = unk::tw_stages(na, xm, segw);
            const size_t smem = unk::tw_smem_bytes(na, xm, segw);
            const unsigned grid = (unsigned)(units * splits);
            if (xm)
                unk::k_wgrad_tc<32, true><<<grid, unk::TW_THREADS, smem, n->stream>>>(a, gmap, xmap, stages);
            else if (NBW == 128)
                unk::k_wgrad_tc<128, false><<<grid, unk::TW_THREADS, smem, n->stream>>>(a, gmap, xmap, stages);
            else if (NBW == 64)
                unk::k_wgrad_tc<64, false><<<grid, unk::TW_THREADS, smem, n->stream>>>(a, gmap, xmap, stages);
            else
                unk::k_wgrad_tc<32, false><<<grid, unk::TW_THREADS, smem, n->stream>>>(a, gmap, xmap, stages);
            unk::k_sum_splits<<<sum_grid(nw), dim3(32, 8), 0, n->stream>>>(n->wpart, splits, nw, n->grad + L.woff);
            unk::k_sum_splits_wide<<<L.cout, 256, 0, n->stream>>>(n->bpart, splits, L.cout, n->grad + L.boff);
            return cudaGetLastError();
        }
    }
    if (W % unk::HT_W == 0 && H % unk::HT_H == 0) {
        // halo-tile form: one staged gradient tile and input halo per 128 pixels, all taps
        unk::WgradHaloArgs a;
        a.g = g;
        a.gC = gC;
        a.goff = goff;
        a.x = x;
        a.xC = xC;
        a.xoff = xoff;
        a.Cout = L.cout;
        a.Cin = L.cin;
        a.N = N;
        a.H = Hl(n, l);
        a.W = Wl(n, l);
        const int blocks = (L.cout / 32) * (L.cin / 32);
        const long long n_tiles = M / (unk::HT_H * unk::HT_W);
        long long sp = (4LL * n->sms + blocks - 1) / blocks;
        if (sp > n_tiles) sp = n_tiles;
        if (sp < 1) sp = 1;
        const long long tps = (n_tiles + sp - 1) / sp;
        const int splits = (int)((n_tiles + tps - 1) / tps);
        a.tiles_per_split = (int)tps;
        a.part = n->wpart;
        a.bpart = n->bpart;
        unk::k_wgrad_halo<<<dim3(blocks, splits), 256, unk::wgrad_halo_smem_bytes(), n->stream>>>(a);
        unk::k_sum_splits<<<sum_grid(nw), dim3(32, 8), 0, n->stream>>>(n->wpart, splits, nw, n->grad + L.woff);
        unk::k_sum_splits_wide<<<L.cout, 256, 0, n->stream>>>(n->bpart, splits, L.cout, n->grad + L.boff);
        return cudaGetLastError();
    }
    int MT, NT, tiles, splits, cps;
    wgrad_shape(n, L, M, &MT, &NT, &tiles, &splits, &cps);
    unk::WgradArgs a;
    a.g = g;
    a.gC = gC;
    a.goff = goff;
    a.x = x;
    a.xC = xC;
    a.xoff = xoff;
    a.Cout = L.cout;
    a.Cin = L.cin;
    a.N = N;
    a.H = Hl(n, l);
    a.W = Wl(n, l);
    a.chunks_per_split = cps;
    a.part = n->wpart;
    a.bpart = n->bpart;
    const dim3 grid(tiles, splits);
    if (MT == 32 && NT == 32) unk::k_wgrad<32, 32><<<grid, 256, 0, n->stream>>>(a);
    else if (MT == 32) unk::k_wgrad<32, 64><<<grid, 256, 0, n->stream>>>(a);
    else if (NT == 32) unk::k_wgrad<64, 32><<<grid, 256, 0, n->stream>>>(a);
    else unk::k_wgrad<64, 64><<<grid, 256, 0, n->stream>>>(a);
    unk::k_sum_splits<<<sum_grid(nw), dim3(32, 8), 0, n->stream>>>(n->wpart, splits, nw, n->grad + L.woff);
    // bias: partials of the centre-tap CTAs, summed over the splits in order
    unk::k_sum_splits_wide<<<L.cout, 256, 0, n->stream>>>(n->bpart, splits, L.cout, n->grad + L.boff);
    return cudaGetLastError();
}

const bf16* Wb(const un_net* n, int k) { return n->wb + n->L[k].qoff; }
const bf16* Wt(const un_net* n, int k) { return n->wt + n->L[k].qoff; }
const float* Bias(const un_net* n, int k) { return n->p + n->L[k].boff; }

// the Adam update (adam != 0) and every BF16 copy of the 3x3 weights, one launch
cudaError_t adam_refresh(un_net* n, int adam, float lr, float b1, float b2, float eps, float c1, float c2) {
    unk::AdamRefreshArgs a;
    a.p = n->p;
    a.m = n->m;
    a.v = n->v;
    a.g = n->grad;
    a.n = n->nparam;
    a.lr = lr;
    a.b1 = b1;
    a.b2 = b2;
    a.eps = eps;
    a.c1 = c1;
    a.c2 = c2;
    a.adam = adam;
    a.wb = n->wb;
    a.wt = n->wt;
    a.wbk = n->wbk;
    a.wtk = n->wtk;
    a.nl = 0;
    for (int k = 0; k < UN_LAYERS && a.nl < unk::AR_MAX_LAYERS; ++k) {
        const Layer& L = n->L[k];
        if (L.k != 3) continue;
        a.woff[a.nl] = L.woff;
        a.qoff[a.nl] = L.qoff;
        a.cout[a.nl] = L.cout;
        a.cin[a.nl] = L.cin;
        // stage images for the streamed tensor-core convolution (forward: Cout
        // output channels; input gradient: Cin)
        a.nbf[a.nl] = L.cin % 16 == 0 ? unk::ts_block(L.cout) : 0;
        a.nbt[a.nl] = L.cout % 16 == 0 ? unk::ts_block(L.cin) : 0;
        ++a.nl;
    }
    unk::k_adam_refresh<<<grid_for(n->nparam), 256, 0, n->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t refresh_weights(un_net* n) { return adam_refresh(n, 0, 0.0f, 0.0f, 0.0f, 1.0f, 1.0f, 1.0f); }

cudaError_t forward(un_net* n, int N, const float* d_in) {
    const int LV = UN_LEVELS;
    unk::k_input<<<grid_for(Pl(n, 0, N) * 4), 256, 0, n->stream>>>(d_in, (long long)N * Hl(n, 0), Wl(n, 0), n->x0);
    for (int l = 0; l < LV; ++l) {
        const bf16* src = l == 0 ? n->x0 : n->pl[l - 1];
        const int sC = l == 0 ? UN_IN_PAD : Cl(n, l - 1);
        conv(n, src, sC, 0, sC, Wb(n, LE(l, 0)), Bias(n, LE(l, 0)), Cl(n, l), n->a[l], Cl(n, l), 0, nullptr, 0, 0, N,
             l, 1, 0);
        if (l < LV - 1) {
            const int catC = Cl(n, l + 1) + Cl(n, l);
            conv(n, n->a[l], Cl(n, l), 0, Cl(n, l), Wb(n, LE(l, 1)), Bias(n, LE(l, 1)), Cl(n, l), n->cat[l], catC,
                 Cl(n, l + 1), nullptr, 0, 0, N, l, 1, 0);
            unk::k_pool<<<grid_for(Pl(n, l + 1, N) * Cl(n, l) / 8), 256, 0, n->stream>>>(
                n->cat[l], catC, Cl(n, l + 1), Cl(n, l), N, Hl(n, l), Wl(n, l), n->pl[l]);
        } else {
            // bottleneck output, upsampled into cat[LV - 2]
            const int catC = Cl(n, l) + Cl(n, l - 1);
            conv(n, n->a[l], Cl(n, l), 0, Cl(n, l), Wb(n, LE(l, 1)), Bias(n, LE(l, 1)), Cl(n, l), n->cat[l - 1], catC,
                 0, nullptr, 0, 0, N, l, 1, 1);
        }
    }
    for (int l = LV - 2; l >= 0; --l) {
        const int catC = Cl(n, l + 1) + Cl(n, l);
        conv(n, n->cat[l], catC, 0, catC, Wb(n, LD(l, 0)), Bias(n, LD(l, 0)), Cl(n, l), n->c[l], Cl(n, l), 0, nullptr,
             0, 0, N, l, 1, 0);
        if (l > 0)
            conv(n, n->c[l], Cl(n, l), 0, Cl(n, l), Wb(n, LD(l, 1)), Bias(n, LD(l, 1)), Cl(n, l), n->cat[l - 1],
                 Cl(n, l) + Cl(n, l - 1), 0, nullptr, 0, 0, N, l, 1, 1);
        else
            conv(n, n->c[0], Cl(n, 0), 0, Cl(n, 0), Wb(n, LD(0, 1)), Bias(n, LD(0, 1)), Cl(n, 0), n->d0, Cl(n, 0), 0,
                 nullptr, 0, 0, N, 0, 1, 0);
    }
    return cudaGetLastError();
}

cudaError_t head_fwd(un_net* n, int N, float* out) {
    const Layer& H = n->L[LHEAD];
    const long long P = Pl(n, 0, N);
    const int C = n->cfg.base;
    const int g = grid_for(P);
    switch (C) {
        case 32:
            unk::k_head_fwd<32><<<g, 256, 0, n->stream>>>(n->d0, n->p + H.woff, n->p + H.boff, P, Wl(n, 0), out);
            break;
        case 64:
            unk::k_head_fwd<64><<<g, 256, 0, n->stream>>>(n->d0, n->p + H.woff, n->p + H.boff, P, Wl(n, 0), out);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t backward(un_net* n, int N, const float* d_target) {
    const int LV = UN_LEVELS;
    const Layer& H = n->L[LHEAD];
    const long long P = Pl(n, 0, N);
    const int C = n->cfg.base;
    const int rows = (int)((P + n->hblocks - 1) / n->hblocks);
    const int hb = (int)((P + rows - 1) / rows);
    const float inv2 = (float)(2.0 / ((double)P * UN_OUT));
    switch (C) {
        case 32:
            unk::k_head_bwd<32><<<hb, 256, 0, n->stream>>>(n->d0, n->p + H.woff, n->p + H.boff, d_target, P, Wl(n, 0),
                                                           rows, inv2, n->gd0, n->hpart, n->lpart);
            break;
        case 64:
            unk::k_head_bwd<64><<<hb, 256, 0, n->stream>>>(n->d0, n->p + H.woff, n->p + H.boff, d_target, P, Wl(n, 0),
                                                           rows, inv2, n->gd0, n->hpart, n->lpart);
            break;
        default: return cudaErrorInvalidValue;
    }
    unk::k_sum_splits_wide<<<2 * C + 2, 256, 0, n->stream>>>(n->hpart, hb, 2LL * C + 2, n->grad + H.woff);
    unk::k_sum_doubles<<<1, 256, 0, n->stream>>>(n->lpart, hb, n->d_loss);
    // decoder, finest level first
    for (int l = 0; l < LV - 1; ++l) {
        const bf16* gin = l == 0 ? n->gd0 : n->gup[l];
        const int c = Cl(n, l), catC = Cl(n, l + 1) + Cl(n, l);
        wgrad(n, LD(l, 1), gin, c, 0, n->c[l], c, 0, N, l);
        conv(n, gin, c, 0, c, Wt(n, LD(l, 1)), nullptr, c, n->gc[l], c, 0, n->c[l], c, 0, N, l, 0, 0);
        wgrad(n, LD(l, 0), n->gc[l], c, 0, n->cat[l], catC, 0, N, l);
        conv(n, n->gc[l], c, 0, c, Wt(n, LD(l, 0)), nullptr, catC, n->gcat[l], catC, 0, nullptr, 0, 0, N, l, 0, 0);
        const int cu = Cl(n, l + 1);
        unk::k_up_bwd<<<grid_for(Pl(n, l + 1, N) * cu / 8), 256, 0, n->stream>>>(
            n->gcat[l], catC, 0, n->cat[l], catC, 0, cu, N, Hl(n, l), Wl(n, l), n->gup[l + 1]);
    }
    // encoder, coarsest level first
    for (int l = LV - 1; l >= 0; --l) {
        const bf16* gin = l == LV - 1 ? n->gup[LV - 1] : n->gs[l];
        const int c = Cl(n, l);
        wgrad(n, LE(l, 1), gin, c, 0, n->a[l], c, 0, N, l);
        conv(n, gin, c, 0, c, Wt(n, LE(l, 1)), nullptr, c, n->ga[l], c, 0, n->a[l], c, 0, N, l, 0, 0);
        const bf16* src = l == 0 ? n->x0 : n->pl[l - 1];
        const int sC = l == 0 ? UN_IN_PAD : Cl(n, l - 1);
        wgrad(n, LE(l, 0), n->ga[l], c, 0, src, sC, 0, N, l);
        if (l > 0) {
            const int cp = Cl(n, l - 1), catC = c + cp;
            conv(n, n->ga[l], c, 0, c, Wt(n, LE(l, 0)), nullptr, cp, n->gp[l - 1], cp, 0, nullptr, 0, 0, N, l, 0, 0);
            unk::k_skip_bwd<<<grid_for(Pl(n, l - 1, N) * cp / 8), 256, 0, n->stream>>>(
                n->gp[l - 1], n->gcat[l - 1], catC, c, n->cat[l - 1], catC, c, cp, N, Hl(n, l - 1), Wl(n, l - 1),
                n->gs[l - 1]);
        }
    }
    return cudaGetLastError();
}

// tensor table for un_get_tensor: pointer, element count at N, channels and
// image width of the tensor
bool tensor_of(const un_net* n, int id, int N, const bf16** ptr, long long* count, int* chans, int* width) {
    const int LV = UN_LEVELS;
    const bool grad = id >= UN_T_GRAD;
    const int b = grad ? id - UN_T_GRAD : id;
    const int kind = b / 10 * 10, l = b % 10;
    const bf16* p = nullptr;
    long long cnt = 0;
    switch (kind) {
        case UN_T_X0:
            if (l != 0 || grad) return false;
            p = n->x0;
            cnt = Pl(n, 0, N) * UN_IN_PAD;
            break;
        case UN_T_A:
            if (l >= LV) return false;
            p = grad ? n->ga[l] : n->a[l];
            cnt = Pl(n, l, N) * Cl(n, l);
            break;
        case UN_T_CAT:
            if (l >= LV - 1) return false;
            p = grad ? n->gcat[l] : n->cat[l];
            cnt = Pl(n, l, N) * (Cl(n, l + 1) + Cl(n, l));
            break;
        case UN_T_P:
            if (l >= LV - 1) return false;
            p = grad ? n->gp[l] : n->pl[l];
            cnt = Pl(n, l + 1, N) * Cl(n, l);
            break;
        case UN_T_C:
            if (l >= LV - 1) return false;
            p = grad ? n->gc[l] : n->c[l];
            cnt = Pl(n, l, N) * Cl(n, l);
            break;
        case UN_T_D0:
            if (l != 0) return false;
            p = grad ? n->gd0 : n->d0;
            cnt = Pl(n, 0, N) * Cl(n, 0);
            break;
        case UN_T_UP:
            if (!grad || l < 1 || l >= LV) return false;
            p = n->gup[l];
            cnt = Pl(n, l, N) * Cl(n, l);
            break;
        case UN_T_SKIP:
            if (!grad || l >= LV - 1) return false;
            p = n->gs[l];
            cnt = Pl(n, l, N) * Cl(n, l);
            break;
        default: return false;
    }
    *ptr = p;
    *count = cnt;
    const int lev = kind == UN_T_P ? l + 1 : l;
    *width = Wl(n, lev);
    *chans = (int)(cnt / Pl(n, lev, N));
    return true;
}

}  // namespace

extern "C" {

int64_t un_param_count(const un_config* cfg) {
    if (!valid_cfg(cfg)) return -1;
    Layer L[UN_LAYERS];
    layer_table(cfg, L);
    return L[UN_LAYERS - 1].boff + L[UN_LAYERS - 1].cout;
}

lb_status un_layer_info(const un_config* cfg, int32_t k, int32_t* cin, int32_t* cout, int32_t* ksize,
                        int64_t* offset) {
    if (!valid_cfg(cfg) || k < 0 || k >= UN_LAYERS) return uerr(LB_ERR_ARG, "un_layer_info: bad config or k");
    Layer L[UN_LAYERS];
    layer_table(cfg, L);
    if (cin) *cin = L[k].cin;
    if (cout) *cout = L[k].cout;
    if (ksize) *ksize = L[k].k;
    if (offset) *offset = L[k].woff;
    return LB_OK;
}

lb_status un_create(const un_config* cfg, void* stream, un_net** out) {
    if (!out) return uerr(LB_ERR_ARG, "un_create: out is NULL");
    if (!valid_cfg(cfg))
        return uerr(LB_ERR_ARG, "un_create: H, W must be multiples of 8, base a multiple of 32 (<= 256), max_batch >= 1");
    if (cfg->base != 32 && cfg->base != 64) return uerr(LB_ERR_UNSUPPORTED, "un_create: head kernel built for base 32, 64");
    un_net* n = new (std::nothrow) un_net();
    if (!n) return uerr(LB_ERR_OOM, "host allocation failed");
    n->cfg = *cfg;
    layer_table(cfg, n->L);
    n->nparam = n->L[UN_LAYERS - 1].boff + n->L[UN_LAYERS - 1].cout;
    for (int k = 0; k < UN_LAYERS; ++k)
        if (n->L[k].k == 3) n->nq = n->L[k].qoff + (long long)n->L[k].cout * 9 * n->L[k].cin;
    cudaError_t e = cudaSuccess;
    if (stream) {
        n->stream = static_cast<cudaStream_t>(stream);
        e = cudaStreamGetDevice(n->stream, &n->device);
    } else {
        e = cudaGetDevice(&n->device);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
        n->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaSetDevice(n->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, n->device);
    const int N = cfg->max_batch, LV = UN_LEVELS;
    if (e == cudaSuccess) e = alloc(n, &n->p, n->nparam);
    if (e == cudaSuccess) e = alloc(n, &n->m, n->nparam);
    if (e == cudaSuccess) e = alloc(n, &n->v, n->nparam);
    if (e == cudaSuccess) e = alloc(n, &n->grad, n->nparam);
    if (e == cudaSuccess) e = alloc(n, &n->wb, n->nq);
    if (e == cudaSuccess) e = alloc(n, &n->wt, n->nq);
    if (e == cudaSuccess) e = alloc(n, &n->wbk, n->nq);
    if (e == cudaSuccess) e = alloc(n, &n->wtk, n->nq);
    if (e == cudaSuccess) e = alloc(n, &n->x0, Pl(n, 0, N) * UN_IN_PAD);
    for (int l = 0; l < LV && e == cudaSuccess; ++l) {
        e = alloc(n, &n->a[l], Pl(n, l, N) * Cl(n, l));
        if (e == cudaSuccess) e = alloc(n, &n->ga[l], Pl(n, l, N) * Cl(n, l));
        if (e == cudaSuccess && l >= 1) e = alloc(n, &n->gup[l], Pl(n, l, N) * Cl(n, l));
        if (l < LV - 1 && e == cudaSuccess) {
            const long long catn = Pl(n, l, N) * (Cl(n, l + 1) + Cl(n, l));
            e = alloc(n, &n->cat[l], catn);
            if (e == cudaSuccess) e = alloc(n, &n->gcat[l], catn);
            if (e == cudaSuccess) e = alloc(n, &n->pl[l], Pl(n, l + 1, N) * Cl(n, l));
            if (e == cudaSuccess) e = alloc(n, &n->gp[l], Pl(n, l + 1, N) * Cl(n, l));
            if (e == cudaSuccess) e = alloc(n, &n->c[l], Pl(n, l, N) * Cl(n, l));
            if (e == cudaSuccess) e = alloc(n, &n->gc[l], Pl(n, l, N) * Cl(n, l));
            if (e == cudaSuccess) e = alloc(n, &n->gs[l], Pl(n, l, N) * Cl(n, l));
        }
    }
    if (e == cudaSuccess) e = alloc(n, &n->d0, Pl(n, 0, N) * Cl(n, 0));
    if (e == cudaSuccess) e = alloc(n, &n->gd0, Pl(n, 0, N) * Cl(n, 0));
    if (e == cudaSuccess) e = alloc(n, &n->y, Pl(n, 0, N) * UN_OUT);
    // weight-gradient partials: the largest split count any layer can use
    // (the split count grows with the pixel count, so max_batch bounds it)
    long long cap = 0;
    for (int k = 0; k < UN_LAYERS; ++k) {
        if (n->L[k].k != 3) continue;
        int MT, NT, tiles, splits, cps;
        const int lev = k < 2 * LV ? k / 2 : (UN_LEVELS - 2) - (k - 2 * LV) / 2;
        wgrad_shape(n, n->L[k], Pl(n, lev, N), &MT, &NT, &tiles, &splits, &cps);
        // the split count never exceeds ceil(4 SMs / tiles) at any N
        // (the halo-tile form splits (cout/32)(cin/32) blocks the same way)
        const long long hblocks = (long long)(n->L[k].cout / 32) * (n->L[k].cin / 32);
        long long smax = (4LL * n->sms + tiles - 1) / tiles;
        const long long smax_h = (4LL * n->sms + hblocks - 1) / hblocks;
        if (smax_h > smax) smax = smax_h;
        // the tcgen05 weight gradient: one split per SM's share of its units
        const bool xm = n->L[k].cout == 32 && n->L[k].cin >= 64 && n->L[k].cin % 32 == 0;
        const int nbw = xm ? unk::TW_MB : unk::tw_block(n->L[k].cin);
        if (xm || (n->L[k].cout % 64 == 0 && nbw)) {
            const long long units = (xm ? 1 : (n->L[k].cout + unk::TW_MB - 1) / unk::TW_MB) *
                                    ((n->L[k].cin + nbw - 1) / nbw) * 3;
            const long long s_tc = n->sms / units > 1 ? n->sms / units : 1;
            if (s_tc > smax) smax = s_tc;
        }
        const long long need = smax * n->L[k].cout * 9 * n->L[k].cin;
        if (need > cap) cap = need;
    }
    n->wpart_cap = cap;
    if (e == cudaSuccess) e = alloc(n, &n->wpart, cap);
    if (e == cudaSuccess) e = alloc(n, &n->bpart, 1024LL * 256);
    n->hblocks = 2 * n->sms;
    if (e == cudaSuccess) e = alloc(n, &n->hpart, (long long)n->hblocks * (2 * cfg->base + 2));
    if (e == cudaSuccess) e = alloc(n, &n->lpart, n->hblocks);
    if (e == cudaSuccess) e = alloc(n, &n->d_loss, 1);
    if (e == cudaSuccess) e = alloc(n, &n->d_err, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->d_err, 0, sizeof(int), n->stream);
    // the tcgen05 convolution: the largest dynamic shared memory any layer asks
    if (e == cudaSuccess) e = cudaFuncSetAttribute(unk::k_conv3_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(unk::k_conv3_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(unk::k_conv3_tc<96>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(unk::k_conv3_tcs<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)unk::ts_smem_bytes(128));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(unk::k_conv3_tcs<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)unk::ts_smem_bytes(64));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(unk::k_wgrad_tc<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(unk::k_wgrad_tc<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(unk::k_wgrad_tc<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(unk::k_wgrad_tc<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(unk::k_conv3_halo, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)unk::halo_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(unk::k_wgrad_halo, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)unk::wgrad_halo_smem_bytes());

    if (e == cudaSuccess) e = cudaMemsetAsync(n->p, 0, sizeof(float) * n->nparam, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, sizeof(float) * n->nparam, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, sizeof(float) * n->nparam, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->grad, 0, sizeof(float) * n->nparam, n->stream);
    if (e == cudaSuccess) e = refresh_weights(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) {
        release(n);
        return ucuda(e, "un_create");
    }
    *out = n;
    return LB_OK;
}

lb_status un_set_params(un_net* n, const float* params, int64_t count) {
    if (!n || !params || count != n->nparam) return uerr(LB_ERR_ARG, "un_set_params: NULL or wrong count");
    UCU(cudaSetDevice(n->device), "cudaSetDevice");
    UCU(cudaMemcpyAsync(n->p, params, sizeof(float) * count, cudaMemcpyDefault, n->stream), "params upload");
    UCU(cudaMemsetAsync(n->m, 0, sizeof(float) * count, n->stream), "adam reset");
    UCU(cudaMemsetAsync(n->v, 0, sizeof(float) * count, n->stream), "adam reset");
    n->t = 0;
    UCU(refresh_weights(n), "weight refresh");
    UCU(cudaStreamSynchronize(n->stream), "synchronize");
    return LB_OK;
}

lb_status un_get_params(un_net* n, float* params, int64_t count) {
    if (!n || !params || count != n->nparam) return uerr(LB_ERR_ARG, "un_get_params: NULL or wrong count");
    UCU(cudaSetDevice(n->device), "cudaSetDevice");
    UCU(cudaMemcpyAsync(params, n->p, sizeof(float) * count, cudaMemcpyDefault, n->stream), "params download");
    UCU(cudaStreamSynchronize(n->stream), "synchronize");
    return LB_OK;
}

lb_status un_get_grads(un_net* n, float* grads, int64_t count) {
    if (!n || !grads || count != n->nparam) return uerr(LB_ERR_ARG, "un_get_grads: NULL or wrong count");
    UCU(cudaSetDevice(n->device), "cudaSetDevice");
    UCU(cudaMemcpyAsync(grads, n->grad, sizeof(float) * count, cudaMemcpyDefault, n->stream), "grads download");
    UCU(cudaStreamSynchronize(n->stream), "synchronize");
    return LB_OK;
}

lb_status un_forward(un_net* n, int32_t N, const float* d_in, float* d_out) {
    if (!n || !d_in || !d_out || N < 1 || N > n->cfg.max_batch)
        return uerr(LB_ERR_ARG, "un_forward: NULL pointer or N outside 1..max_batch");
    UCU(cudaSetDevice(n->device), "cudaSetDevice");
    n->lastN = N;
    UCU(forward(n, N, d_in), "forward");
    UCU(head_fwd(n, N, d_out), "head");
    return LB_OK;
}

lb_status un_loss_grad(un_net* n, int32_t N, const float* d_in, const float* d_target, double* loss) {
    if (!n || !d_in || !d_target || N < 1 || N > n->cfg.max_batch)
        return uerr(LB_ERR_ARG, "un_loss_grad: NULL pointer or N outside 1..max_batch");
    UCU(cudaSetDevice(n->device), "cudaSetDevice");
    n->lastN = N;
    UCU(forward(n, N, d_in), "forward");
    UCU(backward(n, N, d_target), "backward");
    if (loss) {
        double s = 0.0;
        UCU(cudaMemcpyAsync(&s, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream), "loss download");
        UCU(cudaStreamSynchronize(n->stream), "synchronize");
        *loss = s / ((double)Pl(n, 0, N) * UN_OUT);
    }
    return LB_OK;
}

lb_status un_adam_step(un_net* n, double lr, double beta1, double beta2, double eps) {
    if (!n || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return uerr(LB_ERR_ARG, "un_adam_step: invalid hyper-parameters");
    UCU(cudaSetDevice(n->device), "cudaSetDevice");
    n->t += 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow(beta1, (double)n->t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(beta2, (double)n->t)));
    UCU(adam_refresh(n, 1, (float)lr, (float)beta1, (float)beta2, (float)eps, c1, c2), "adam");
    return LB_OK;
}

lb_status un_train_step(un_net* n, int32_t N, const float* d_in, const float* d_target, double lr, double* loss) {
    lb_status st = un_loss_grad(n, N, d_in, d_target, loss);
    if (st) return st;
    return un_adam_step(n, lr, 0.9, 0.999, 1e-8);
}

lb_status un_get_tensor(un_net* n, int32_t id, float* host, int64_t count) {
    if (!n || !host) return uerr(LB_ERR_ARG, "un_get_tensor: NULL argument");
    const bf16* p = nullptr;
    long long cnt = 0;
    int C = 0, W = 0;
    if (n->lastN < 1 || !tensor_of(n, id, n->lastN, &p, &cnt, &C, &W) || cnt != count)
        return uerr(LB_ERR_ARG, "un_get_tensor: unknown id %d or wrong size", id);
    UCU(cudaSetDevice(n->device), "cudaSetDevice");
    std::vector<uint16_t> h((size_t)cnt);
    UCU(cudaMemcpyAsync(h.data(), p, sizeof(uint16_t) * cnt, cudaMemcpyDeviceToHost, n->stream), "tensor download");
    UCU(cudaStreamSynchronize(n->stream), "synchronize");
    // row-blocked channel groups -> NHWC
    const long long rows = cnt / ((long long)C * W);
    for (long long r = 0; r < rows; ++r)
        for (int x = 0; x < W; ++x)
            for (int c = 0; c < C; ++c) {
                const uint32_t bits = (uint32_t)h[(size_t)unk::act_at(r, x, c, C, W)] << 16;
                std::memcpy(host + (r * W + x) * C + c, &bits, 4);
            }
    return LB_OK;
}

lb_status un_synchronize(un_net* n) {
    if (!n) return uerr(LB_ERR_ARG, "un_synchronize: NULL net");
    UCU(cudaSetDevice(n->device), "cudaSetDevice");
    int h = 0;
    UCU(cudaMemcpyAsync(&h, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream), "read error word");
    UCU(cudaStreamSynchronize(n->stream), "synchronize");
    if (h) {
        UCU(cudaMemsetAsync(n->d_err, 0, sizeof(int), n->stream), "clear error word");
        UCU(cudaStreamSynchronize(n->stream), "synchronize");
        return uerr(LB_ERR_TIMEOUT, "a bounded wait of the tensor-core convolution gave up (error word 0x%x)", h);
    }
    return LB_OK;
}

lb_status un_free(un_net* n) {
    release(n);
    return LB_OK;
}

lb_status un_warm_fields(int32_t N, int32_t H, int32_t W, const float* d_pred, double rho_dev_scale,
                         double rho_floor, double t_dev_scale, const double* d_rho0, const double* d_T0,
                         double* d_rho, double* d_T, void* stream) {
    if (N < 1 || H < 1 || W < 1 || !d_pred || !d_rho0 || !d_T0 || !d_rho || !d_T)
        return uerr(LB_ERR_ARG, "un_warm_fields: invalid argument");
    unk::WarmArgs a;
    a.pred = d_pred;
    a.rho_dev_scale = rho_dev_scale;
    a.rho_floor = rho_floor;
    a.t_dev_scale = t_dev_scale;
    a.rho0 = d_rho0;
    a.T0 = d_T0;
    a.rho = d_rho;
    a.T = d_T;
    a.P = (long long)H * W;
    unk::k_warm<<<N, 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
    UCU(cudaGetLastError(), "un_warm_fields");
    return LB_OK;
}

}  // extern "C"
