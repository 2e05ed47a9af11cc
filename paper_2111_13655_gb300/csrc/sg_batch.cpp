// Many Smolyak problems per apply (declared in include/smolyak.h): the terms
// of all problems of one kernel variant go to the device in one launch per
// form (block / warp), ordered by estimated cost over all problems, so a
// batch of small and large problems keeps every SM busy until the end.
#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "sg_internal.h"

// Order of the batched work items: 0 = by term cost over all problems,
// 1 = problem-major (problems by total cost, then their terms by cost).
#ifndef SG_BATCH_ORDER
#define SG_BATCH_ORDER 0
#endif
// A fast-path problem with at least this many block-form terms fills the GPU
// for several waves by itself: it runs as its own launches (parameters in the
// kernel's parameter bank, as in sg_apply_H) inside the batch's sequence, and
// only the smaller problems share the packed launches.
#ifndef SG_BATCH_SOLO_TERMS
#define SG_BATCH_SOLO_TERMS 16384
#endif

struct sg_batch {
    std::vector<sg_ctx *> ctxs;
    std::vector<int> plan_versions;    // of the contexts when the batch was made
    int device = 0;
    bool fp32 = false;
    std::vector<long long> cs_prefix;  // host copy
    int64_t n_terms = 0, max_ncs = 0;
    const long long *d_cs_prefix = nullptr;
    const sg::KParams *d_kps = nullptr;
    struct Group {
        sg::KParams kp_any;
        sg::FastBatchGroup g;
    };
    std::vector<Group> groups;
    std::vector<int> generic;          // problems outside the fast path: one launch each
    std::vector<int> solo;             // large fast-path problems: their own launches
    std::vector<void *> allocations;
    std::vector<sg::KParams> h_kps;    // host copy of d_kps (the input-copy pointers change with the workspace)
    unsigned long long *acc = nullptr;
    long long *maxbits = nullptr;
    void *xs = nullptr;                // entry-major input copies of the fast-path problems
    int acc_nvec = 0;
    // the apply's launch sequence captured as a graph, for the last (x, y, nvec, stream)
    cudaGraphExec_t graph = nullptr;
    const double *gx = nullptr;
    double *gy = nullptr;
    int gnvec = 0;
    cudaStream_t gstream = nullptr;
    int64_t graph_launches = 0;
    std::string last_error;
};

namespace {

sg_status bfail(sg_batch *b, sg_status st, const std::string &msg)
{
    if (b) b->last_error = msg;
    return st;
}

template <typename T>
sg_status bupload(sg_batch *b, const std::vector<T> &v, const T **dst)
{
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return bfail(b, SG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    b->allocations.push_back(p);
    if (!v.empty() && (e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bfail(b, SG_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    *dst = static_cast<const T *>(p);
    return SG_OK;
}

void drop_graph(sg_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->gx = nullptr;
    b->gy = nullptr;
    b->gnvec = 0;
    b->gstream = nullptr;
}

void free_all(sg_batch *b)
{
    drop_graph(b);
    for (void *p : b->allocations) cudaFree(p);
    b->allocations.clear();
    if (b->acc) cudaFree(b->acc);
    if (b->maxbits) cudaFree(b->maxbits);
    if (b->xs) cudaFree(b->xs);
    b->acc = nullptr;
    b->maxbits = nullptr;
    b->xs = nullptr;
}

}  // namespace

extern "C" sg_status sg_batch_create(sg_ctx *const *ctxs, int n, sg_batch **out)
{
    if (!out) return SG_EINVAL;
    *out = nullptr;
    if (!ctxs || n < 1 || n > 65535) return SG_EINVAL;
    sg_batch *b = new (std::nothrow) sg_batch;
    if (!b) return SG_ENOMEM;
    for (int j = 0; j < n; j++) {
        sg_ctx *c = ctxs[j];
        if (!c || !c->has_device) { delete b; return SG_EINVAL; }
        if (c->kp.fast.df) { delete b; return SG_EUNSUPPORTED; }  // double-float contexts are applied one by one
        if (j > 0 && (c->device != b->device || c->fp32 != b->fp32)) { delete b; return SG_EINVAL; }
        b->device = c->device;
        b->fp32 = c->fp32;
        b->ctxs.push_back(c);
        b->plan_versions.push_back(c->plan_version);
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != b->device) { delete b; return SG_EINVAL; }

    b->cs_prefix.assign(n + 1, 0);
    std::vector<sg::KParams> kps(n);
    for (int j = 0; j < n; j++) {
        const sg_ctx *c = ctxs[j];
        b->cs_prefix[j + 1] = b->cs_prefix[j] + c->host.n_cs;
        b->max_ncs = std::max<int64_t>(b->max_ncs, c->host.n_cs);
        b->n_terms += c->host.n_terms;
        kps[j] = c->kp;
        kps[j].acc = nullptr;  // the batch kernels take the batch's accumulators explicitly
        kps[j].xs = nullptr;   // set with the workspace (the batch's own input copies)
        kps[j].xs_nvec = 0;
    }

    // every fast-path problem (of the batch's one precision) shares the launches
    std::map<int, std::vector<int>> by_variant;
    for (int j = 0; j < n; j++) {
        const sg::KParams &kp = ctxs[j]->kp;
        if (!kp.fast.enabled) b->generic.push_back(j);
        else if (kp.fast.n_big >= SG_BATCH_SOLO_TERMS) b->solo.push_back(j);
        else by_variant[0].push_back(j);
    }
    sg_status st;
    b->h_kps = kps;
    if ((st = bupload(b, kps, &b->d_kps)) != SG_OK || (st = bupload(b, b->cs_prefix, &b->d_cs_prefix)) != SG_OK) {
        free_all(b);
        delete b;
        return st;
    }
    for (auto &kv : by_variant) {
        sg_batch::Group G{};
        G.kp_any = ctxs[kv.second[0]]->kp;
        G.kp_any.xs = nullptr;
        G.g.kps = b->d_kps;
        for (int f = 0; f < 2; f++) {
            struct Item { int64_t cost; int j, p; };
            std::vector<Item> it;
            size_t part = 0;
            for (int j : kv.second) {
                const sg::HostTables &T = ctxs[j]->host;
                const int nb = ctxs[j]->kp.fast.n_big;
                const int64_t p0 = f == 0 ? 0 : nb, p1 = f == 0 ? nb : T.n_terms;
                if (p1 > p0) part = std::max(part, sg::fast_part_bytes(ctxs[j]->kp, b->fp32, f == 1));
                for (int64_t p = p0; p < p1; p++) it.push_back({T.pcost[p], j, (int)p});
            }
            if (SG_BATCH_ORDER == 0) {
                std::stable_sort(it.begin(), it.end(), [](const Item &a, const Item &c) { return a.cost > c.cost; });
            } else {
                // problem-major: problems by decreasing total cost, each problem's
                // terms by decreasing cost (a few problems in flight at a time)
                std::map<int, int64_t> tot;
                for (const Item &t : it) tot[t.j] += t.cost;
                std::stable_sort(it.begin(), it.end(), [&](const Item &a, const Item &c) {
                    if (a.j != c.j) return tot[a.j] != tot[c.j] ? tot[a.j] > tot[c.j] : a.j < c.j;
                    return a.cost > c.cost;
                });
            }
            std::vector<int2> items(it.size());
            for (size_t q = 0; q < it.size(); q++) items[q] = make_int2(it[q].j, it[q].p);
            if (it.size() > (size_t)0x7FFFFFFF) { free_all(b); delete b; return SG_EUNSUPPORTED; }
            G.g.count[f] = (int)it.size();
            G.g.part[f] = (int)part;
            if ((st = bupload(b, items, &G.g.items[f])) != SG_OK) { free_all(b); delete b; return st; }
        }
        cudaError_t e = sg::configure_fast_batch(G.kp_any, b->fp32, G.g);
        if (e != cudaSuccess) { free_all(b); delete b; return SG_ECUDA; }
        b->groups.push_back(G);
    }
    *out = b;
    return SG_OK;
}

extern "C" sg_status sg_batch_size(const sg_batch *b, int64_t *n_cs_total, int64_t *n_terms_total,
                                   int *launches_per_apply)
{
    if (!b) return SG_EINVAL;
    if (n_cs_total) *n_cs_total = b->cs_prefix.back();
    if (n_terms_total) *n_terms_total = b->n_terms;
    if (launches_per_apply) {
        // max|x|, finalisation, the input copies
        int l = 2 + (SG_STAGE_X && (!b->groups.empty() || !b->solo.empty()));
        for (const auto &G : b->groups) l += (G.g.count[0] > 0) + (G.g.count[1] > 0);
        for (int j : b->solo) {
            const sg::KParams &kp = b->ctxs[j]->kp;
            l += (kp.fast.n_big > 0) + (kp.n_terms > kp.fast.n_big);
        }
        for (int j : b->generic) {
            const sg::KParams &kp = b->ctxs[j]->kp;
            l += kp.n_terms > 0;
        }
        *launches_per_apply = l;
    }
    return SG_OK;
}

sg_status enqueue_apply(sg_batch *b, const double *x, double *y, int nvec, cudaStream_t s);

extern "C" sg_status sg_apply_H_batch(sg_batch *b, const double *x, double *y, int nvec, void *stream)
{
    if (!b) return SG_EINVAL;
    if (!x || !y) return bfail(b, SG_EINVAL, "x or y is NULL");
    if (nvec < 1) return bfail(b, SG_EINVAL, "nvec must be >= 1");
    const int nprob = (int)b->ctxs.size();
    const size_t total = (size_t)b->cs_prefix.back() * (size_t)nvec;
    if ((x < y + total) && (y < x + total)) return bfail(b, SG_EINVAL, "x and y overlap");
    if ((size_t)nprob * nvec > 65535u * 65535u) return bfail(b, SG_EUNSUPPORTED, "too many vectors");
    if (nvec > 65535) return bfail(b, SG_EUNSUPPORTED, "nvec > 65535");
    for (int j = 0; j < nprob; j++)
        if (b->ctxs[j]->plan_version != b->plan_versions[j])
            return bfail(b, SG_EINVAL, "problem " + std::to_string(j) +
                                           " was re-planned by sg_tune after the batch was made: recreate the batch");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (nvec > b->acc_nvec) {
        drop_graph(b);  // it names the old workspace
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
            return bfail(b, SG_ECUDA, std::string("stream synchronize: ") + cudaGetErrorString(e));
        if (b->acc) cudaFree(b->acc);
        if (b->maxbits) cudaFree(b->maxbits);
        if (b->xs) cudaFree(b->xs);
        b->acc = nullptr;
        b->maxbits = nullptr;
        b->xs = nullptr;
        b->acc_nvec = 0;
        const size_t words = total * sg::acc_words(b->fp32);
        if ((e = cudaMalloc(&b->acc, words * sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaMalloc(&b->maxbits, sizeof(long long) * (size_t)nprob * nvec)) != cudaSuccess)
            return bfail(b, SG_ENOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
#if SG_STAGE_X
        if (!b->groups.empty() || !b->solo.empty()) {
            // the fast-path problems gather from entry-major copies, problem j's rows from cs_prefix[j]
            const size_t rb = b->fp32 ? 4 : 8, stride = (size_t)sg::xs_stride(nvec);
            if ((e = cudaMalloc(&b->xs, (size_t)b->cs_prefix.back() * stride * rb)) != cudaSuccess)
                return bfail(b, SG_ENOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
            for (int j = 0; j < nprob; j++) {
                if (!b->ctxs[j]->kp.fast.enabled) continue;
                b->h_kps[j].xs = static_cast<unsigned char *>(b->xs) + (size_t)b->cs_prefix[j] * stride * rb;
                b->h_kps[j].xs_nvec = nvec;
            }
            if ((e = cudaMemcpy(const_cast<sg::KParams *>(b->d_kps), b->h_kps.data(),
                                sizeof(sg::KParams) * b->h_kps.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
                return bfail(b, SG_ECUDA, std::string("parameter upload: ") + cudaGetErrorString(e));
        }
#endif
        if ((e = cudaMemsetAsync(b->acc, 0, words * sizeof(unsigned long long), s)) != cudaSuccess)
            return bfail(b, SG_ECUDA, std::string("workspace memset: ") + cudaGetErrorString(e));
        b->acc_nvec = nvec;
    }
    // Replay the captured launch sequence when the same buffers, block size and
    // stream come back; capture it on first use.  Not on the legacy default
    // stream (it cannot be captured) nor while the caller is capturing the
    // stream itself (the launches then go into the caller's graph).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s != nullptr && (e = cudaStreamIsCapturing(s, &cs)) != cudaSuccess)
        return bfail(b, SG_ECUDA, std::string("stream capture query: ") + cudaGetErrorString(e));
    if (s != nullptr && cs == cudaStreamCaptureStatusNone) {
        if (!(b->graph && b->gx == x && b->gy == y && b->gnvec == nvec && b->gstream == s)) {
            drop_graph(b);
            cudaGraph_t g = nullptr;
            if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return bfail(b, SG_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
            const sg_status st = enqueue_apply(b, x, y, nvec, s);
            e = cudaStreamEndCapture(s, &g);
            if (st != SG_OK) { if (g) cudaGraphDestroy(g); return st; }
            if (e != cudaSuccess) return bfail(b, SG_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { b->graph = nullptr; return bfail(b, SG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)); }
            b->gx = x; b->gy = y; b->gnvec = nvec; b->gstream = s;
        }
        if ((e = cudaGraphLaunch(b->graph, s)) != cudaSuccess)
            return bfail(b, SG_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        b->graph_launches++;
        return SG_OK;
    }
    return enqueue_apply(b, x, y, nvec, s);
}

// The launch sequence of one batched apply: max|x|, term kernels, finalisation.
sg_status enqueue_apply(sg_batch *b, const double *x, double *y, int nvec, cudaStream_t s)
{
    const int nprob = (int)b->ctxs.size();
    cudaError_t e;
    if ((e = sg::launch_maxabs_batch(x, b->d_cs_prefix, nprob, b->max_ncs, nvec, b->maxbits, s)) != cudaSuccess)
        return bfail(b, SG_ECUDA, std::string("max|x| launch: ") + cudaGetErrorString(e));
    if (b->xs && (e = sg::launch_stage_x_batch(b->fp32, x, b->d_cs_prefix, nprob, b->max_ncs, nvec, b->acc_nvec,
                                               b->xs, s)) != cudaSuccess)
        return bfail(b, SG_ECUDA, std::string("input copy launch: ") + cudaGetErrorString(e));
    for (int j : b->solo) {
        sg::KParams kp = b->h_kps[j];  // with the batch's input copy of problem j
        const size_t off = (size_t)nvec * (size_t)b->cs_prefix[j];
        kp.acc = b->acc + off * sg::acc_words(b->fp32);
        if (!kp.xs || nvec > kp.xs_nvec) kp.xs = nullptr;
        if ((e = sg::launch_apply_fast(kp, b->fp32, x + off, nvec, b->maxbits + (size_t)j * nvec, s)) != cudaSuccess)
            return bfail(b, SG_ECUDA, std::string("term launch: ") + cudaGetErrorString(e));
    }
    for (const auto &G : b->groups)
        if ((e = sg::launch_fast_batch(G.kp_any, b->fp32, G.g, x, b->acc, b->maxbits, b->d_cs_prefix, nvec, s)) !=
            cudaSuccess)
            return bfail(b, SG_ECUDA, std::string("batched term launch: ") + cudaGetErrorString(e));
    for (int j : b->generic) {
        sg::KParams kp = b->ctxs[j]->kp;
        const size_t off = (size_t)nvec * (size_t)b->cs_prefix[j];
        kp.acc = b->acc + off * sg::acc_words(b->fp32);
        kp.xs = nullptr;  // the context's own input copy is not the batch's
        if ((e = sg::launch_apply_terms(kp, b->fp32, x + off, b->maxbits + (size_t)j * nvec, nvec, s)) !=
            cudaSuccess)
            return bfail(b, SG_ECUDA, std::string("term launch: ") + cudaGetErrorString(e));
    }
    if ((e = sg::launch_finalize_batch(b->d_kps, b->d_cs_prefix, nprob, b->max_ncs, x, y, b->acc,
                                       b->maxbits, nvec, b->fp32, s)) != cudaSuccess)
        return bfail(b, SG_ECUDA, std::string("finalise launch: ") + cudaGetErrorString(e));
    return SG_OK;
}

extern "C" const char *sg_batch_last_error(const sg_batch *b)
{
    return b ? b->last_error.c_str() : "";
}

extern "C" void sg_batch_destroy(sg_batch *b)
{
    if (!b) return;
    free_all(b);
    delete b;
}
