// sg_tune (declared in include/smolyak.h): measured choice of the fast path's
// term schedule for one context.
//
// The schedule knob is the slicing target: a term whose grid leaves room for
// fewer than that many vectors per chunk is sliced over its leading outer
// positions (smaller slices, fewer chunks), else it runs unsliced in more,
// smaller chunks.  Which is faster depends on the problem's term shapes and on
// the block size in vectors the caller applies, so the context is re-planned
// for every candidate and timed on real applies.  Only the slicing depths in the
// term records change (and with them the layout of the per-term potential
// tables, rebuilt for each): images, M^B and capacities stay as they are.
#include <algorithm>
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "sg_internal.h"

extern "C" sg_status sg_tune(sg_ctx *ctx, int nvec, int *slice_vt, double *ms_out, void *stream)
{
    if (!ctx) return SG_EINVAL;
    if (!ctx->has_device) { ctx->last_error = "sg_tune: context was made by sg_plan"; return SG_EINVAL; }
    if (!sg_on_ctx_device(ctx)) { ctx->last_error = std::string("sg_tune: ") + "the current CUDA device is not the one the context was made on"; return SG_EINVAL; }
    if (nvec < 1 || nvec > 64) { ctx->last_error = "sg_tune: need 1 <= nvec <= 64"; return SG_EINVAL; }
    sg::HostTables &T = ctx->host;
    if (!ctx->kp.fast.enabled) {  // generic kernel: no schedule to choose
        if (slice_vt) *slice_vt = 0;
        if (ms_out) *ms_out = 0.0;
        return SG_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) { ctx->last_error = "sg_tune: stream synchronize"; return SG_ECUDA; }
    const size_t n = (size_t)T.n_cs * nvec;
    double *x = nullptr, *y = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&x, n * sizeof(double))) != cudaSuccess || (e = cudaMalloc(&y, n * sizeof(double))) != cudaSuccess) {
        if (x) cudaFree(x);
        ctx->last_error = std::string("sg_tune: cudaMalloc: ") + cudaGetErrorString(e);
        return SG_ENOMEM;
    }
    {
        std::vector<double> h(n);
        for (size_t i = 0; i < n; i++) h[i] = 1.0 / (1.0 + (double)(i % 977)) - 0.25;
        e = cudaMemcpy(x, h.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    }
    const size_t rec_bytes = T.fdesc.size() * sizeof(int4);
    const std::vector<int4> original = T.fdesc;
    const int original_vt = T.slice_vt;
    std::vector<int4> best_desc;
    int best_vt = 0;
    double best_ms = std::numeric_limits<double>::infinity();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    sg_status st = e == cudaSuccess ? SG_OK : SG_ECUDA;
    for (int vt : {1, 2, 4}) {
        if (st != SG_OK) break;
        T.slice_vt = vt;
        const std::string err = sg::build_fast_descs(ctx->prob, ctx->fp32, &T, T.fbudget, ctx->fp32 ? 4 : 8);
        if (!err.empty() || !T.fast || T.fdesc.size() * sizeof(int4) != rec_bytes ||
            T.fn_big != ctx->kp.fast.n_big) {
            T.fast = true;  // this target cannot plan every term: skip it
            continue;
        }
        if ((e = cudaMemcpy(const_cast<int4 *>(ctx->kp.fast.desc), T.fdesc.data(), rec_bytes,
                            cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = sg::launch_build_mtab(ctx->kp, ctx->fp32, s)) != cudaSuccess ||  // layout follows the slicing
            (e = cudaStreamSynchronize(s)) != cudaSuccess) { st = SG_ECUDA; break; }
        // one untimed apply, then the median of three
        std::vector<float> t;
        for (int k = 0; k < 4 && st == SG_OK; k++) {
            if ((e = cudaEventRecord(e0, s)) != cudaSuccess) { st = SG_ECUDA; break; }
            st = sg_apply_H(ctx, x, y, nvec, stream);
            if (st == SG_OK && (e = cudaEventRecord(e1, s)) != cudaSuccess) st = SG_ECUDA;
            if (st == SG_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) st = SG_ECUDA;
            float ms = 0.f;
            if (st == SG_OK) cudaEventElapsedTime(&ms, e0, e1);
            if (k > 0) t.push_back(ms);
        }
        if (st != SG_OK) break;
        std::sort(t.begin(), t.end());
        if (t[1] < best_ms) { best_ms = t[1]; best_vt = vt; best_desc = T.fdesc; }
    }
    // keep the fastest plan (or the original one if none could be timed)
    T.fdesc = best_vt ? best_desc : original;
    T.slice_vt = best_vt ? best_vt : original_vt;
    T.fast = true;
    cudaError_t e2 = cudaMemcpy(const_cast<int4 *>(ctx->kp.fast.desc), T.fdesc.data(), rec_bytes,
                                cudaMemcpyHostToDevice);
    if (e2 == cudaSuccess) e2 = sg::launch_build_mtab(ctx->kp, ctx->fp32, s);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
    if (st == SG_OK && e2 != cudaSuccess) { st = SG_ECUDA; e = e2; }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    if (st != SG_OK) {
        // a failed apply has set its own message; CUDA errors of the tuner set this one
        if (st == SG_ECUDA && e != cudaSuccess) ctx->last_error = std::string("sg_tune: ") + cudaGetErrorString(e);
        return st;
    }
    if (slice_vt) *slice_vt = best_vt;
    if (ms_out) *ms_out = best_ms;
    return SG_OK;
}
