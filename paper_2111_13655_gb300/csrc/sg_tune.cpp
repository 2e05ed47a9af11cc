// sg_tune (declared in include/smolyak.h): measured choice of the fast path's
// term schedule for one context.
//
// Three knobs of the host plan, searched one after another (coordinate
// descent: each in turn over its candidates with the others at their best so
// far), every candidate timed on real applies of the caller's block size:
//   1. the slicing target: a term whose grid leaves room for fewer than that
//      many vectors per chunk is sliced over its leading outer positions
//      (smaller slices, fewer chunks), else it runs unsliced in more, smaller
//      chunks;
//   2. the block/warp split: terms that fit a quarter of a block's shared
//      memory with that many vectors per chunk run one per warp (no block
//      barriers, four terms per block), the larger ones one per block;
//   3. the shared-memory budget of a block (the group size in memory): more
//      per block means more vectors per chunk and fewer resident blocks.
// Only the term records (slicing depths), the split point and the work-area
// capacities change; M^B, the term images and the sizes of the inner-block
// tables do not (the tables' layout follows the slicing and is rebuilt for
// each candidate).
#include <algorithm>
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "sg_internal.h"

namespace {

struct Plan {
    int slice_vt, warp_vt, smem_kb;
};

struct Tuner {
    sg_ctx *ctx;
    cudaStream_t s;
    const double *x;
    double *y;
    int nvec;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaSuccess;

    // Re-plans the records for p and installs them (records, split, capacities,
    // inner-block tables).  False when the plan cannot hold every term.
    bool install(const Plan &p, size_t rec_bytes)
    {
        sg::HostTables &T = ctx->host;
        T.slice_vt = p.slice_vt;
        T.warp_vt = p.warp_vt;
        const int rb = ctx->fp32 ? 4 : 8;
        const int budget = p.smem_kb * 1024;
        const std::string e = sg::build_fast_descs(ctx->prob, ctx->fp32, &T, budget, rb);
        if (!e.empty() || !T.fast || T.fdesc.size() * sizeof(int4) != rec_bytes) {
            T.fast = true;
            return false;
        }
        sg::FastParams &F = ctx->kp.fast;
        T.fbudget = budget;
        F.n_big = T.fn_big;
        F.work_cta = T.fwork_cta;
        F.work_warp = T.fwork_warp;
        ctx->smem_bytes = sg::fast_smem_bytes(ctx->kp, ctx->fp32);
        if ((err = cudaMemcpy(const_cast<int4 *>(F.desc), T.fdesc.data(), rec_bytes, cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (err = sg::launch_build_mtab(ctx->kp, ctx->fp32, s)) != cudaSuccess ||
            (err = cudaStreamSynchronize(s)) != cudaSuccess)
            return false;
        ctx->plan_version++;
        return true;
    }

    // Median of three timed applies after one untimed; negative on failure.
    double time_apply(sg_status *st)
    {
        std::vector<float> t;
        for (int k = 0; k < 4 && *st == SG_OK; k++) {
            if ((err = cudaEventRecord(e0, s)) != cudaSuccess) { *st = SG_ECUDA; break; }
            *st = sg_apply_H(ctx, x, y, nvec, s);
            if (*st == SG_OK && (err = cudaEventRecord(e1, s)) != cudaSuccess) *st = SG_ECUDA;
            if (*st == SG_OK && (err = cudaEventSynchronize(e1)) != cudaSuccess) *st = SG_ECUDA;
            float ms = 0.f;
            if (*st == SG_OK) cudaEventElapsedTime(&ms, e0, e1);
            if (k > 0) t.push_back(ms);
        }
        if (*st != SG_OK) return -1.0;
        std::sort(t.begin(), t.end());
        return t[1];
    }
};

}  // namespace

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
    Tuner tu{ctx, s, x, y, nvec};
    if (e == cudaSuccess) e = cudaEventCreate(&tu.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&tu.e1);
    sg_status st = e == cudaSuccess ? SG_OK : SG_ECUDA;
    const size_t rec_bytes = T.fdesc.size() * sizeof(int4);
    const Plan original{T.slice_vt > 0 ? T.slice_vt : (ctx->fp32 ? SG_F32_SLICE_VT : SG_F64_SLICE_VT),
                        T.warp_vt > 0 ? T.warp_vt : SG_WARP_VT, T.fbudget / 1024};
    Plan best = original;
    double best_ms = std::numeric_limits<double>::infinity();
    std::vector<Plan> tried;
    auto evaluate = [&](const Plan &p) {
        for (const Plan &q : tried)
            if (q.slice_vt == p.slice_vt && q.warp_vt == p.warp_vt && q.smem_kb == p.smem_kb) return;
        tried.push_back(p);
        if (st != SG_OK || !tu.install(p, rec_bytes)) {
            if (tu.err != cudaSuccess) st = SG_ECUDA;
            return;
        }
        const double ms = tu.time_apply(&st);
        if (st == SG_OK && ms >= 0.0 && ms < best_ms) { best_ms = ms; best = p; }
    };
    evaluate(original);
    for (int v : {1, 2, 4}) evaluate(Plan{v, best.warp_vt, best.smem_kb});
    for (int v : {1, 2, 4}) evaluate(Plan{best.slice_vt, v, best.smem_kb});
    for (int kb : ctx->fp32 ? std::vector<int>{52, 70, 104} : std::vector<int>{70, 104})
        evaluate(Plan{best.slice_vt, best.warp_vt, kb});
    // keep the fastest plan (the original one if none could be timed)
    const bool ok = std::isfinite(best_ms);
    const cudaError_t keep_err = tu.err;
    tu.err = cudaSuccess;
    if (!tu.install(ok ? best : original, rec_bytes) && st == SG_OK) {
        st = tu.err != cudaSuccess ? SG_ECUDA : SG_EINVAL;
        if (st == SG_EINVAL) ctx->last_error = "sg_tune: the kept plan could not be installed";
    }
    if (tu.e0) cudaEventDestroy(tu.e0);
    if (tu.e1) cudaEventDestroy(tu.e1);
    cudaFree(x);
    cudaFree(y);
    if (st != SG_OK) {
        // a failed apply has set its own message; CUDA errors of the tuner set this one
        const cudaError_t ce = tu.err != cudaSuccess ? tu.err : keep_err != cudaSuccess ? keep_err : e;
        if (st == SG_ECUDA && ce != cudaSuccess) ctx->last_error = std::string("sg_tune: ") + cudaGetErrorString(ce);
        return st;
    }
    if (slice_vt) *slice_vt = ok ? best.slice_vt : 0;
    if (ms_out) *ms_out = ok ? best_ms : 0.0;
    return SG_OK;
}

extern "C" sg_status sg_tune_plan(const sg_ctx *ctx, int *slice_vt, int *warp_vt, int *smem_kb)
{
    if (!ctx) return SG_EINVAL;
    const sg::HostTables &T = ctx->host;
    const bool fast = ctx->kp.fast.enabled || (!ctx->has_device && T.fast);
    if (slice_vt) *slice_vt = fast ? (T.slice_vt > 0 ? T.slice_vt : (ctx->fp32 ? SG_F32_SLICE_VT : SG_F64_SLICE_VT)) : 0;
    if (warp_vt) *warp_vt = fast ? (T.warp_vt > 0 ? T.warp_vt : SG_WARP_VT) : 0;
    if (smem_kb) *smem_kb = fast ? T.fbudget / 1024 : 0;
    return SG_OK;
}
