// lb_batch.cu -- host side of the batched solver (lb_batch_* in include/lb.h).
//
// All domains of a batch share the storage precision, the temperature
// treatment and the force form (beta == 0, beta == 1, or mixed); every other
// parameter (size, tau_f, tau_g, G, beta, EOS and its constants, c_v) is per
// domain.  Domains are stored back to back in two ping-pong buffers.  A run
// replays a CUDA graph of K fused steps plus a per-domain residual check, then
// takes converged or failed domains off the device work list; the graph reads
// the list lengths from device memory, so it stays valid.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lb.h"
#include "lb_batch_device.cuh"
#include "lb_launch.h"

namespace lbgb {
lb_status record_error(lb_status st, const char* msg);
// FP64 batch step: its own translation unit, compiled without contraction
cudaError_t launch_batch_step_fp64(const void* src, void* dst, const BatchDomain* doms,
                                   const BatchItem* items, const int* n_items, int* next_item, int eq24,
                                   int bmode, int grid, cudaStream_t stream);
}

using namespace lbgb;

namespace {

constexpr int BATCH_BX_FP32 = 256;
constexpr int BATCH_BX_FP64 = 128;
// row-chunk heights the autotuner tries; the work list is sized for the smallest
constexpr int kChunkCand[LB_BATCH_TUNE_N] = {16, 32, 64, 128};
constexpr int MIN_CHUNK_ROWS = 16;

lb_status err(lb_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
lb_status err(lb_status st, const char* fmt, ...) {
    char msg[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    return record_error(st, msg);
}

lb_status cuerr(cudaError_t e, const char* what) {
    return err(e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, "%s: %s", what,
               cudaGetErrorString(e));
}

#define BCU(call, what)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuerr(e_, what);   \
    } while (0)

int bmode_of(double beta) { return beta == 0.0 ? BETA_ZERO : (beta == 1.0 ? BETA_ONE : BETA_MIXED); }

}  // namespace

struct lb_batch {
    int n = 0;
    int prec = LB_PREC_FP32;
    int eq24 = 1;
    int bmode = BETA_ONE;
    int bx = BATCH_BX_FP32;
    int chunk_rows = 64;
    int device = 0;
    int sms = 152;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<lb_params> params;
    std::vector<BatchDomain> doms;
    std::vector<int> frozen;      // -1: active; else the buffer index holding its state
    std::vector<int> status;      // per-domain lb_status of the run
    std::vector<int64_t> steps;   // steps taken by each domain
    BatchDomain* d_doms = nullptr;
    void* buf[2] = {nullptr, nullptr};
    size_t buf_bytes = 0;
    int cur = 0;
    int* d_err = nullptr;
    // work lists
    BatchItem* d_items = nullptr;
    int* d_counts = nullptr;      // [0] items, [1] tiles
    int* d_next = nullptr;        // takes from the work counter in the current step (the step resets it)
    int max_items = 0;
    BatchTile* d_tiles = nullptr;
    int* d_tile_begin = nullptr;  // [n + 1]
    int max_tiles = 0;
    double* d_part = nullptr;     // [max_tiles][6]
    double* d_out6 = nullptr;     // [n][6]
    double* d_ref_rho = nullptr;  // dense reference fields (all domains)
    double* d_ref_T = nullptr;
    long long n_sites = 0;
    double* h_out6 = nullptr;     // pinned
    int* h_err = nullptr;         // pinned
    int have_ref = 0;
    int64_t t = 0;
    int64_t ref_time = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_k = 0;
    int graph_cur = -1;
};

namespace {

// Launch one batched step src -> dst; with src == nullptr only set the
// kernel's shared-memory attribute (done once, outside any stream capture).
cudaError_t launch_batch_step(lb_batch* b, const void* src, void* dst) {
    const int grid = 2 * b->sms;
    if (b->prec == LB_PREC_FP32) {
        using E = float;
        constexpr int BX = BATCH_BX_FP32, ST = batch_stages<LB_PREC_FP32, BX>();
        constexpr size_t smem = batch_smem_bytes<LB_PREC_FP32, BX, ST>();
        static_assert(smem <= 110 * 1024, "two CTAs per SM");
        auto pick = [&]() -> void (*)(const E*, E*, const BatchDomain*, const BatchItem*, const int*, int*) {
            if (b->eq24) {
                if (b->bmode == BETA_ZERO) return k_batch_step<LB_PREC_FP32, BX, ST, true, BETA_ZERO>;
                if (b->bmode == BETA_ONE) return k_batch_step<LB_PREC_FP32, BX, ST, true, BETA_ONE>;
                return k_batch_step<LB_PREC_FP32, BX, ST, true, BETA_MIXED>;
            }
            if (b->bmode == BETA_ZERO) return k_batch_step<LB_PREC_FP32, BX, ST, false, BETA_ZERO>;
            if (b->bmode == BETA_ONE) return k_batch_step<LB_PREC_FP32, BX, ST, false, BETA_ONE>;
            return k_batch_step<LB_PREC_FP32, BX, ST, false, BETA_MIXED>;
        };
        auto k = pick();
        if (!src) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, strip_threads<BX>(), smem, b->stream>>>(static_cast<const E*>(src), static_cast<E*>(dst),
                                                           b->d_doms, b->d_items, b->d_counts, b->d_next);
        return cudaGetLastError();
    }
    return launch_batch_step_fp64(src, dst, b->d_doms, b->d_items, b->d_counts, b->d_next, b->eq24, b->bmode,
                                  grid, b->stream);
}

cudaError_t launch_batch_check(lb_batch* b) {
    const int grid = b->max_tiles > 0 ? b->max_tiles : 1;
    if (b->prec == LB_PREC_FP32)
        k_batch_check<LB_PREC_FP32><<<grid, 256, 0, b->stream>>>(
            static_cast<const float*>(b->buf[b->cur]), b->d_doms, b->d_tiles, b->d_counts + 1,
            b->d_ref_rho, b->d_ref_T, b->have_ref, b->d_part);
    else
        k_batch_check<LB_PREC_FP64><<<grid, 256, 0, b->stream>>>(
            static_cast<const double*>(b->buf[b->cur]), b->d_doms, b->d_tiles, b->d_counts + 1,
            b->d_ref_rho, b->d_ref_T, b->have_ref, b->d_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_batch_fold<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->d_part, b->d_tile_begin, b->n, b->d_out6);
    return cudaGetLastError();
}

// Rebuild the step work list and the check tile list from the active set.
lb_status rebuild_lists(lb_batch* b) {
    std::vector<BatchItem> items;
    std::vector<BatchTile> tiles;
    std::vector<int> begin(b->n + 1, 0);
    for (int d = 0; d < b->n; ++d) {
        begin[d] = (int)tiles.size();
        if (b->frozen[d] >= 0) continue;
        const int nx = b->params[d].nx, ny = b->params[d].ny;
        const int strips = (nx + b->bx - 1) / b->bx;
        const int chunks = (ny + b->chunk_rows - 1) / b->chunk_rows;
        for (int s = 0; s < strips; ++s) {
            // a strip at most half the kernel's width runs as half items: the
            // chunk's rows split between the two halves of the CTA, so the item
            // takes half the jobs (twice the chunk's rows per item measured
            // slower: fewer items than CTAs on batches of small domains)
            const int w = std::min(b->bx, nx - s * b->bx);
            const int half = 2 * w <= b->bx ? 1 : 0;
            for (int c = 0; c < chunks; ++c) {
                BatchItem it;
                it.domain = d;
                it.strip = s;
                it.y0 = (int)((long long)c * ny / chunks);
                it.y1 = (int)((long long)(c + 1) * ny / chunks);
                it.half = half;
                items.push_back(it);
            }
        }
        for (int first = 0; first < nx * ny; first += 256) tiles.push_back(BatchTile{d, first});
    }
    begin[b->n] = (int)tiles.size();
    if ((int)items.size() > b->max_items || (int)tiles.size() > b->max_tiles)
        return err(LB_ERR_ARG, "batch work list larger than allocated");
    // Longest item first: the persistent CTAs take items in this order from a
    // global counter, so the short items fill in at the end.  Cost of an item:
    // its jobs (rows plus the two halo rows; a half item's two halves march
    // together, so the left half's rows) times the columns they keep busy
    // plus a per-row constant (a narrow strip still pays the row's barrier
    // and latencies).
    auto cost = [&](const BatchItem& a) {
        const long long w = std::min(b->bx, b->params[a.domain].nx - a.strip * b->bx);
        if (a.half) return (long long)(batch_split(a.y0, a.y1) - a.y0 + 2) * (2 * w + 64);
        return (long long)(a.y1 - a.y0 + 2) * (w + 64);
    };
    std::stable_sort(items.begin(), items.end(),
                     [&](const BatchItem& a, const BatchItem& c) { return cost(a) > cost(c); });
    int counts[2] = {(int)items.size(), (int)tiles.size()};
    if (!items.empty())
        BCU(cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(),
                            cudaMemcpyHostToDevice, b->stream), "work list upload");
    if (!tiles.empty())
        BCU(cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(),
                            cudaMemcpyHostToDevice, b->stream), "tile list upload");
    BCU(cudaMemcpyAsync(b->d_tile_begin, begin.data(), sizeof(int) * begin.size(),
                        cudaMemcpyHostToDevice, b->stream), "tile index upload");
    BCU(cudaMemcpyAsync(b->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, b->stream),
        "list length upload");
    // (each step leaves the work counter at zero; reset it here as well, so a
    // step that stopped on an error cannot leave it behind)
    BCU(cudaMemsetAsync(b->d_next, 0, sizeof(int) * 2, b->stream), "work counter reset");
    BCU(cudaStreamSynchronize(b->stream), "synchronize");
    return LB_OK;
}

void release(lb_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->d_doms);
    cudaFree(b->buf[0]);
    cudaFree(b->buf[1]);
    cudaFree(b->d_err);
    cudaFree(b->d_items);
    cudaFree(b->d_counts);
    cudaFree(b->d_next);
    cudaFree(b->d_tiles);
    cudaFree(b->d_tile_begin);
    cudaFree(b->d_part);
    cudaFree(b->d_out6);
    cudaFree(b->d_ref_rho);
    cudaFree(b->d_ref_T);
    cudaFreeHost(b->h_out6);
    cudaFreeHost(b->h_err);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Residual of domain d from the folded sums (0 without a reference).
double residual_of(const lb_batch* b, int d, int64_t K) {
    if (K <= 0) return 0.0;
    const double* v = b->h_out6 + (size_t)d * 6;
    const double r_rho = std::sqrt(v[2]) / ((double)K * std::sqrt(v[3]));
    const double r_T = std::sqrt(v[4]) / ((double)K * std::sqrt(v[5]));
    return r_rho > r_T ? r_rho : r_T;
}

// Read the folded sums and error words to the host (pinned) and wait.
lb_status fetch_check(lb_batch* b) {
    BCU(cudaMemcpyAsync(b->h_out6, b->d_out6, sizeof(double) * 6 * b->n, cudaMemcpyDeviceToHost, b->stream),
        "check download");
    BCU(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->stream),
        "error words download");
    BCU(cudaStreamSynchronize(b->stream), "synchronize");
    return LB_OK;
}

lb_status status_of_word(int w) {
    if (w & (1 << LB_ERR_PSI_DOMAIN)) return LB_ERR_PSI_DOMAIN;
    if (w & (1 << LB_ERR_NONFINITE)) return LB_ERR_NONFINITE;
    if (w & (1 << LB_ERR_TIMEOUT)) return LB_ERR_TIMEOUT;
    return w ? LB_ERR_CUDA : LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_batch_init(const lb_params* params, int32_t n, const double* const* rho0,
                        const double* const* T0, void* stream, lb_batch** out) {
    if (!params || !rho0 || !T0 || !out || n < 1) return err(LB_ERR_ARG, "lb_batch_init: NULL argument or n < 1");
    const int prec = params[0].precision;
    if (prec != LB_PREC_FP32 && prec != LB_PREC_FP64)
        return err(LB_ERR_UNSUPPORTED, "batched solver supports FP32 and FP64 storage");
    for (int d = 0; d < n; ++d) {
        const lb_params& p = params[d];
        if (!rho0[d] || !T0[d]) return err(LB_ERR_ARG, "domain %d: NULL field", d);
        if (p.precision != prec || p.thermal != params[0].thermal ||
            bmode_of(p.beta) != bmode_of(params[0].beta))
            return err(LB_ERR_ARG, "domain %d: precision, thermal treatment and force form must match domain 0", d);
        if (p.nx < 3 || p.ny < 3)
            return err(LB_ERR_ARG, "domain %d: nx and ny must be >= 3", d);
        if (p.walls != LB_WALLS_PERIODIC || p.halo_rows != 0)
            return err(LB_ERR_UNSUPPORTED, "domain %d: the batched solver runs periodic domains", d);
        if (!(p.tau_f > 0.5) || !(p.tau_g > 0.5) || p.G == 0.0 || !(p.cv > 0.0) || p.eos < 0 || p.eos > 2 ||
            p.thermal < 0 || p.thermal > 1 || p.init_balanced < 0 || p.init_balanced > 1)
            return err(LB_ERR_ARG, "domain %d: invalid parameters", d);
    }
    lb_batch* b = new (std::nothrow) lb_batch();
    if (!b) return err(LB_ERR_OOM, "host allocation failed");
    b->n = n;
    b->prec = prec;
    b->eq24 = params[0].thermal == LB_THERMAL_EQ24;
    b->bmode = bmode_of(params[0].beta);
    b->bx = prec == LB_PREC_FP64 ? BATCH_BX_FP64 : BATCH_BX_FP32;
    b->params.assign(params, params + n);
    b->frozen.assign(n, -1);
    b->status.assign(n, LB_OK);
    b->steps.assign(n, 0);
    cudaError_t e = cudaSuccess;
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
        e = cudaStreamGetDevice(b->stream, &b->device);
    } else {
        e = cudaGetDevice(&b->device);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
        release(b);
        return cuerr(e, "lb_batch_init device");
    }
    const size_t es = prec == LB_PREC_FP64 ? 8 : 4;
    // layout: each domain's 18 planes back to back in the strip layout (rows
    // padded to 128 B with periodic ghost columns, planes to 256 B); dense
    // field offsets for the reference fields
    long long off = 0, fld = 0;
    int max_items = 0, max_tiles = 0;
    b->doms.resize(n);
    for (int d = 0; d < n; ++d) {
        const lb_params& p = params[d];
        // the strip layout with periodic ghost columns (pop_layout)
        const PopLayout lay = pop_layout(prec, p.nx, p.ny, true);
        const long long pitch = lay.pitch, plane = lay.plane;
        BatchDomain& D = b->doms[d];
        std::memset(&D, 0, sizeof(D));
        KParams& k = D.kp;
        k.nx = p.nx;
        k.ny = p.ny;
        k.pitch = pitch;
        k.plane = plane;
        k.omega_f = 1.0 / p.tau_f;
        k.omega_g = 1.0 / p.tau_g;
        k.guo_pre = 1.0 - 1.0 / (2.0 * p.tau_f);
        k.corr_pre = 1.0 - 1.0 / (2.0 * p.tau_g);
        k.G = p.G;
        k.two_over_G = 2.0 / p.G;
        k.beta = p.beta;
        k.half_1mbeta = 0.5 * (1.0 - p.beta);
        k.eos = p.eos;
        k.psi_local_T = p.psi_uses_local_T;
        k.a = p.a;
        k.b = p.b;
        k.R = p.R;
        k.cv = p.cv;
        k.inv_cv = 1.0 / p.cv;
        k.T_psi = p.T_psi;
        k.ghost = STRIP_GHOST;
        kp_fill_float(k);
        D.off = off + lay.origin;
        D.fld_off = fld;
        off += 18 * plane;
        fld += (long long)p.nx * p.ny;
        max_items += ((p.nx + b->bx - 1) / b->bx) * ((p.ny + MIN_CHUNK_ROWS - 1) / MIN_CHUNK_ROWS);
        max_tiles += (p.nx * p.ny + 255) / 256;
    }
    b->n_sites = fld;
    b->buf_bytes = (size_t)off * es;
    b->max_items = max_items;
    b->max_tiles = max_tiles;
    if (e == cudaSuccess) e = cudaMalloc(&b->buf[0], b->buf_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->buf[1], b->buf_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_doms, sizeof(BatchDomain) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(BatchItem) * (max_items > 0 ? max_items : 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counts, sizeof(int) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(int) * 2);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_next, 0, sizeof(int) * 2, b->stream);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, sizeof(BatchTile) * (max_tiles > 0 ? max_tiles : 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tile_begin, sizeof(int) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_part, sizeof(double) * 6 * (max_tiles > 0 ? max_tiles : 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_out6, sizeof(double) * 6 * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ref_rho, sizeof(double) * fld);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ref_T, sizeof(double) * fld);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_out6, sizeof(double) * 6 * n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_err, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int) * n, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->buf[0], 0, b->buf_bytes, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->buf[1], 0, b->buf_bytes, b->stream);
    if (e != cudaSuccess) {
        release(b);
        return cuerr(e, "allocating batch buffers");
    }
    for (int d = 0; d < n; ++d) b->doms[d].kp.err = b->d_err + d;
    e = cudaMemcpyAsync(b->d_doms, b->doms.data(), sizeof(BatchDomain) * n, cudaMemcpyHostToDevice, b->stream);
    // initial state of each domain: f = f^eq(rho0, 0), g = c_v T0 f^eq(rho0, 0)
    // (or at rest under the force, init_balanced), built from the fields staged
    // in the reference buffers
    for (int d = 0; d < n && e == cudaSuccess; ++d) {
        const size_t nb = sizeof(double) * (size_t)params[d].nx * params[d].ny;
        double* r = b->d_ref_rho + b->doms[d].fld_off;
        double* tt = b->d_ref_T + b->doms[d].fld_off;
        // host or device sources (unified addressing decides the direction)
        e = cudaMemcpyAsync(r, rho0[d], nb, cudaMemcpyDefault, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tt, T0[d], nb, cudaMemcpyDefault, b->stream);
        if (e == cudaSuccess) {
            const KParams& k = b->doms[d].kp;
            if (params[d].init_balanced) {
                void* dst = prec == LB_PREC_FP32 ? static_cast<void*>(static_cast<float*>(b->buf[0]) + b->doms[d].off)
                                                 : static_cast<void*>(static_cast<double*>(b->buf[0]) + b->doms[d].off);
                e = launch_init_balanced(prec, dst, k, r, tt, b->stream);
            } else {
                if (prec == LB_PREC_FP32)
                    k_init<LB_PREC_FP32><<<64, 256, 0, b->stream>>>(static_cast<float*>(b->buf[0]) + b->doms[d].off, k, r, tt);
                else
                    k_init<LB_PREC_FP64><<<64, 256, 0, b->stream>>>(static_cast<double*>(b->buf[0]) + b->doms[d].off, k, r, tt);
                e = cudaGetLastError();
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        release(b);
        return cuerr(e, "batch initial state");
    }
    e = launch_batch_step(b, nullptr, nullptr);
    if (e != cudaSuccess) {
        release(b);
        return cuerr(e, "batch kernel attributes");
    }
    lb_status st = rebuild_lists(b);
    if (st != LB_OK) {
        release(b);
        return st;
    }
    *out = b;
    return LB_OK;
}

lb_status lb_batch_step(lb_batch* b, int64_t n) {
    if (!b || n < 0) return err(LB_ERR_ARG, "lb_batch_step: invalid argument");
    BCU(cudaSetDevice(b->device), "cudaSetDevice");
    for (int64_t k = 0; k < n; ++k) {
        BCU(launch_batch_step(b, b->buf[b->cur], b->buf[b->cur ^ 1]), "batch step launch");
        b->cur ^= 1;
        b->t += 1;
    }
    for (int d = 0; d < b->n; ++d)
        if (b->frozen[d] < 0) b->steps[d] += n;
    return LB_OK;
}

lb_status lb_batch_check(lb_batch* b, double* residual, double* mass, double* energy, int32_t* status) {
    if (!b) return err(LB_ERR_ARG, "lb_batch_check: NULL batch");
    BCU(cudaSetDevice(b->device), "cudaSetDevice");
    BCU(launch_batch_check(b), "batch check");
    lb_status st = fetch_check(b);
    if (st) return st;
    const int64_t K = b->have_ref ? b->t - b->ref_time : 0;
    for (int d = 0; d < b->n; ++d) {
        if (residual) residual[d] = b->frozen[d] < 0 ? residual_of(b, d, K) : 0.0;
        if (mass) mass[d] = b->h_out6[(size_t)d * 6 + 0];
        if (energy) energy[d] = b->h_out6[(size_t)d * 6 + 1];
        if (status) status[d] = status_of_word(b->h_err[d]);
    }
    b->have_ref = 1;
    b->ref_time = b->t;
    return LB_OK;
}

lb_status lb_batch_run(lb_batch* b, double tol, int64_t K, int64_t max_steps, int64_t* steps_out,
                       double* residual_out, int32_t* status_out) {
    if (!b || K < 2 || K % 2 || !(tol > 0.0))
        return err(LB_ERR_ARG, "lb_batch_run: need an even K >= 2 and tol > 0");
    BCU(cudaSetDevice(b->device), "cudaSetDevice");
    std::vector<double> resid(b->n, 0.0);
    // a fresh reference at the start
    lb_status st = lb_batch_check(b, nullptr, nullptr, nullptr, nullptr);
    if (st) return st;
    const int64_t t_start = b->t;
    while (true) {
        int active = 0;
        for (int d = 0; d < b->n; ++d) active += b->frozen[d] < 0;
        if (!active || b->t - t_start >= max_steps) break;
        // (re)capture the graph of K steps + check when the buffer parity changed
        if (!b->graph || b->graph_k != K || b->graph_cur != b->cur) {
            if (b->graph) {
                cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            BCU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t e = cudaSuccess;
            const int c0 = b->cur;
            for (int64_t k = 0; k < K && e == cudaSuccess; ++k) {
                e = launch_batch_step(b, b->buf[b->cur], b->buf[b->cur ^ 1]);
                b->cur ^= 1;
            }
            b->have_ref = 1;  // the captured check compares with the reference
            if (e == cudaSuccess) e = launch_batch_check(b);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            b->cur = c0;
            if (e != cudaSuccess) return cuerr(e, "capturing the batch graph");
            if (e2 != cudaSuccess) return cuerr(e2, "capturing the batch graph");
            e = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuerr(e, "instantiating the batch graph");
            b->graph_k = (int)K;
            b->graph_cur = b->cur;
        }
        BCU(cudaGraphLaunch(b->graph, b->stream), "graph launch");
        b->t += K;  // K is even: the state is back in buf[cur]
        for (int d = 0; d < b->n; ++d)
            if (b->frozen[d] < 0) b->steps[d] += K;
        st = fetch_check(b);
        if (st) return st;
        const int64_t Kr = b->t - b->ref_time;
        b->ref_time = b->t;
        bool changed = false;
        for (int d = 0; d < b->n; ++d) {
            if (b->frozen[d] >= 0) continue;
            resid[d] = residual_of(b, d, Kr);
            const lb_status s = status_of_word(b->h_err[d]);
            if (s != LB_OK || !std::isfinite(resid[d])) {
                b->status[d] = s != LB_OK ? s : LB_ERR_NONFINITE;
            } else if (resid[d] < tol) {
                b->status[d] = LB_OK;
            } else {
                continue;
            }
            b->frozen[d] = b->cur;
            changed = true;
        }
        if (changed) {
            st = rebuild_lists(b);
            if (st) return st;
        }
    }
    for (int d = 0; d < b->n; ++d) {
        if (b->frozen[d] < 0) b->status[d] = LB_ERR_NOT_CONVERGED;
        if (steps_out) steps_out[d] = b->steps[d];
        if (residual_out) residual_out[d] = resid[d];
        if (status_out) status_out[d] = b->status[d];
    }
    return LB_OK;
}

lb_status lb_batch_fields(lb_batch* b, int32_t d, double* rho, double* T) {
    if (!b || d < 0 || d >= b->n) return err(LB_ERR_ARG, "lb_batch_fields: invalid domain");
    BCU(cudaSetDevice(b->device), "cudaSetDevice");
    // a check refreshes the reference fields, which are rho and T of every
    // active domain; frozen domains keep the fields of their last check
    if (b->frozen[d] < 0) {
        BCU(launch_batch_check(b), "batch fields");
        b->have_ref = 1;
        b->ref_time = b->t;
    }
    const size_t nb = sizeof(double) * (size_t)b->params[d].nx * b->params[d].ny;
    if (rho) BCU(cudaMemcpyAsync(rho, b->d_ref_rho + b->doms[d].fld_off, nb, cudaMemcpyDeviceToHost, b->stream), "fields download");
    if (T) BCU(cudaMemcpyAsync(T, b->d_ref_T + b->doms[d].fld_off, nb, cudaMemcpyDeviceToHost, b->stream), "fields download");
    BCU(cudaStreamSynchronize(b->stream), "synchronize");
    return LB_OK;
}

lb_status lb_batch_restart(lb_batch* b, int32_t d, const double* rho0, const double* T0, int32_t init_balanced) {
    if (!b || d < 0 || d >= b->n || !rho0 || !T0)
        return err(LB_ERR_ARG, "lb_batch_restart: invalid domain or NULL field");
    if (init_balanced != 0 && init_balanced != 1) return err(LB_ERR_ARG, "lb_batch_restart: init_balanced must be 0 or 1");
    BCU(cudaSetDevice(b->device), "cudaSetDevice");
    const BatchDomain& D = b->doms[d];
    const size_t nb = sizeof(double) * (size_t)b->params[d].nx * b->params[d].ny;
    double* r = b->d_ref_rho + D.fld_off;
    double* tt = b->d_ref_T + D.fld_off;
    // the fields are staged in the domain's residual reference (its next
    // residual compares with them), then the state is built in the buffer the
    // active domains currently hold
    BCU(cudaMemcpyAsync(r, rho0, nb, cudaMemcpyDefault, b->stream), "restart fields");
    BCU(cudaMemcpyAsync(tt, T0, nb, cudaMemcpyDefault, b->stream), "restart fields");
    void* dst = b->prec == LB_PREC_FP32 ? static_cast<void*>(static_cast<float*>(b->buf[b->cur]) + D.off)
                                       : static_cast<void*>(static_cast<double*>(b->buf[b->cur]) + D.off);
    cudaError_t e;
    if (init_balanced) {
        e = launch_init_balanced(b->prec, dst, D.kp, r, tt, b->stream);
    } else {
        if (b->prec == LB_PREC_FP32)
            k_init<LB_PREC_FP32><<<64, 256, 0, b->stream>>>(static_cast<float*>(dst), D.kp, r, tt);
        else
            k_init<LB_PREC_FP64><<<64, 256, 0, b->stream>>>(static_cast<double*>(dst), D.kp, r, tt);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuerr(e, "restart initial state");
    BCU(cudaMemsetAsync(b->d_err + d, 0, sizeof(int), b->stream), "restart error word");
    BCU(cudaStreamSynchronize(b->stream), "synchronize");
    const bool was_frozen = b->frozen[d] >= 0;
    b->frozen[d] = -1;
    b->status[d] = LB_OK;
    b->params[d].init_balanced = init_balanced;
    return was_frozen ? rebuild_lists(b) : LB_OK;
}

int64_t lb_batch_time(const lb_batch* b) { return b ? b->t : -1; }

lb_status lb_batch_set_chunk_rows(lb_batch* b, int32_t rows) {
    if (!b || rows < MIN_CHUNK_ROWS || rows > 1 << 20)
        return err(LB_ERR_ARG, "lb_batch_set_chunk_rows: rows must be >= %d", MIN_CHUNK_ROWS);
    BCU(cudaSetDevice(b->device), "cudaSetDevice");
    b->chunk_rows = rows;
    return rebuild_lists(b);
}

int32_t lb_batch_chunk_rows(const lb_batch* b) { return b ? b->chunk_rows : -1; }

lb_status lb_batch_autotune(lb_batch* b, int32_t steps, int32_t* chunk_rows,
                            double ms_per_step[LB_BATCH_TUNE_N]) {
    if (!b || steps < 1) return err(LB_ERR_ARG, "lb_batch_autotune: NULL batch or steps < 1");
    BCU(cudaSetDevice(b->device), "cudaSetDevice");
    // snapshot: the current buffer (active and frozen domains) and the error words
    void* snap = nullptr;
    BCU(cudaMalloc(&snap, b->buf_bytes), "autotune snapshot");
    std::vector<int> errw(b->n, 0);
    cudaError_t e = cudaMemcpyAsync(snap, b->buf[b->cur], b->buf_bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(errw.data(), b->d_err, sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    const int cur0 = b->cur, rows0 = b->chunk_rows;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    lb_status st = LB_OK;
    double best = INFINITY;
    int best_rows = rows0;
    for (int k = 0; k < LB_BATCH_TUNE_N && e == cudaSuccess && st == LB_OK; ++k) {
        if (ms_per_step) ms_per_step[k] = NAN;
        b->chunk_rows = kChunkCand[k];
        st = rebuild_lists(b);
        if (st != LB_OK) break;
        for (int w = 0; w < 2 && e == cudaSuccess; ++w) {
            e = launch_batch_step(b, b->buf[b->cur], b->buf[b->cur ^ 1]);
            b->cur ^= 1;
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], b->stream);
        for (int s = 0; s < steps && e == cudaSuccess; ++s) {
            e = launch_batch_step(b, b->buf[b->cur], b->buf[b->cur ^ 1]);
            b->cur ^= 1;
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e != cudaSuccess) break;
        const double per = (double)ms / steps;
        if (ms_per_step) ms_per_step[k] = per;
        if (per < best) {
            best = per;
            best_rows = kChunkCand[k];
        }
    }
    // restore the snapshot, whatever happened
    b->cur = cur0;
    cudaError_t e2 = cudaMemcpyAsync(b->buf[cur0], snap, b->buf_bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e2 == cudaSuccess)
        e2 = cudaMemcpyAsync(b->d_err, errw.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, b->stream);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(b->stream);
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    cudaFree(snap);
    if (e != cudaSuccess) return cuerr(e, "batch autotune");
    if (e2 != cudaSuccess) return cuerr(e2, "batch autotune restore");
    if (st != LB_OK) return st;
    b->chunk_rows = st == LB_OK && std::isfinite(best) ? best_rows : rows0;
    st = rebuild_lists(b);
    if (st == LB_OK && chunk_rows) *chunk_rows = b->chunk_rows;
    return st;
}

lb_status lb_batch_free(lb_batch* b) {
    release(b);
    return LB_OK;
}

}  // extern "C"
