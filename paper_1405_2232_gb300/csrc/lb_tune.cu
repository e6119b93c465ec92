// lb_tune.cu -- the step-shape autotuner (lb_tune_candidate, lb_autotune).
//
// Every shape the fused step can run with is timed on a uniform state of the
// caller's lattice, parameters and precision; the fastest wins.  The state is
// uniform so that no candidate can leave the psi domain while it is timed, and
// the timing uses CUDA events on the stream the trial contexts run on.  Results
// do not depend on the shape (FP64: bit for bit), so the choice is free.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "lb.h"

namespace lbgb {
lb_status record_error(lb_status st, const char* msg);
}

namespace {

// (tile_x, tile_y); tile_y == 0 selects the strip-marching kernel
constexpr int kCand[LB_TUNE_N][2] = {{256, 0}, {128, 0}, {32, 8}, {32, 16}, {64, 4}};

lb_status tune_fail(lb_status st, const char* what, cudaError_t e) {
    char msg[300];
    snprintf(msg, sizeof(msg), "lb_autotune: %s: %s", what, cudaGetErrorString(e));
    return lbgb::record_error(st, msg);
}

}  // namespace

extern "C" {

lb_status lb_tune_candidate(int32_t k, int32_t* tile_x, int32_t* tile_y) {
    if (k < 0 || k >= LB_TUNE_N || !tile_x || !tile_y)
        return lbgb::record_error(LB_ERR_ARG, "lb_tune_candidate: index out of range or NULL output");
    *tile_x = kCand[k][0];
    *tile_y = kCand[k][1];
    return LB_OK;
}

lb_status lb_autotune(const lb_params* p, int32_t steps, void* stream, lb_params* best,
                      double ms_per_step[LB_TUNE_N]) {
    if (!p || !best || steps < 1)
        return lbgb::record_error(LB_ERR_ARG, "lb_autotune: NULL params/best or steps < 1");
    const size_t n = (size_t)p->nx * (size_t)(p->ny > 0 ? p->ny : 0);
    if (p->nx < 3 || p->ny < 3)
        return lbgb::record_error(LB_ERR_ARG, "lb_autotune: nx, ny must be >= 3");
    std::vector<double> rho(n, p->rho0), T(n, p->T0);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool own = false;
    cudaError_t e = cudaSuccess;
    if (st) {
        int dev = 0;
        e = cudaStreamGetDevice(st, &dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);
    } else {
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        own = e == cudaSuccess;
    }
    if (e != cudaSuccess) return tune_fail(LB_ERR_CUDA, "stream", e);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    lb_status result = LB_OK;
    double best_ms = INFINITY;
    int best_k = -1;
    for (int k = 0; k < LB_TUNE_N && e == cudaSuccess; ++k) {
        if (ms_per_step) ms_per_step[k] = NAN;
        lb_params q = *p;
        q.tile_x = kCand[k][0];
        q.tile_y = kCand[k][1];
        lb_ctx* c = nullptr;
        lb_status s = lb_init(&q, rho.data(), T.data(), st, &c);
        if (s == LB_ERR_ARG) continue;  // shape not valid for this lattice/precision
        if (s != LB_OK) {
            result = s;
            break;
        }
        s = lb_step(c, 2);  // warm-up
        if (s == LB_OK) e = cudaEventRecord(ev[0], st);
        if (s == LB_OK && e == cudaSuccess) s = lb_step(c, steps);
        if (s == LB_OK && e == cudaSuccess) e = cudaEventRecord(ev[1], st);
        if (s == LB_OK && e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.0f;
        if (s == LB_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (s == LB_OK && e == cudaSuccess) s = lb_synchronize(c);
        lb_free(c);
        if (s != LB_OK) {
            result = s;
            break;
        }
        if (e != cudaSuccess) break;
        const double per = (double)ms / steps;
        if (ms_per_step) ms_per_step[k] = per;
        if (per < best_ms) {
            best_ms = per;
            best_k = k;
        }
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (own) cudaStreamDestroy(st);
    if (e != cudaSuccess) return tune_fail(LB_ERR_CUDA, "timing", e);
    if (result != LB_OK) return result;
    if (best_k < 0) return lbgb::record_error(LB_ERR_UNSUPPORTED, "lb_autotune: no step shape is valid");
    *best = *p;
    best->tile_x = kCand[best_k][0];
    best->tile_y = kCand[best_k][1];
    return LB_OK;
}

}  // extern "C"
