// Request server (declared in include/smolyak.h): continuous batching of
// Chebyshev propagation requests and block-Davidson eigen requests of
// different D, L and basis sizes.
//
// Each engine iteration
//   1. retires requests whose last step has ended (psi and logs to the host),
//   2. admits queued requests, first come first served, while their planned
//      device memory fits the budget (context tables, M^B, state vectors,
//      batch workspace): builds the context, the spectral interval and the
//      Chebyshev weights,
//   3. on any change of the active set, rebuilds the batch over the active
//      contexts and moves the surviving states to the new layout,
//   4. applies H_S to every active request's current Chebyshev vector in one
//      sg_apply_H_batch (all requests' terms in one launch per kernel form),
//   5. advances every request's recurrence by one term in one fused kernel.
// A request's arithmetic is the same whatever else is in the batch (batched
// applies are bitwise those of the request's own context, the update is
// elementwise, the logged sums run over the request's own entries in a fixed
// order), so its results do not depend on the mix.
//
// Eigen requests: each runs the block Davidson of sg_eigs on a host thread of
// its own, with its vector algebra on its own stream.  Its applications of
// H_S are handed to the engine: a request's block occupies (block + 1) / 2
// two-vector slots of the batch (its context repeated), so every engine
// iteration applies the waiting blocks of all eigen requests together with
// the propagation requests' Chebyshev vectors in one batched apply.  While
// eigen requests are active the engine runs one iteration at a time (it
// waits for their blocks); otherwise pairs of iterations replay as a graph.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "sg_internal.h"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum ReqKind { kProp = 0, kEig = 1 };
// phases of an eigen request's hand-off with the engine
enum EigPhase { kRunning = 0, kPosted = 1, kApplied = 2, kFinished = 3 };

struct Req {
    int64_t id = 0;
    int kind = kProp;
    int state = SG_REQ_QUEUED;
    // problem (deep copy of the request)
    int D = 0, L = 0;
    std::vector<sg_basis> basis;
    std::vector<sg_grid> grids;
    std::vector<double> omega, coef;
    std::vector<int> nfac, mode, power;
    std::vector<double> psi0;  // 2 * n_cs: real part, imaginary part
    double dt = 0;
    int nsteps = 0, order = 0;
    int64_t n_cs = 0, bytes = 0;
    // while active
    sg_ctx *ctx = nullptr;
    double ebar = 0, de = 1, cph = 1, sph = 0;
    std::vector<double> c;     // (2 - delta_k0) J_k, k = 0..K
    int K = 1, step = 0, k = 0;
    double *d_log = nullptr;   // [nsteps][norm, energy]
    double *d_c = nullptr;     // device copy of c
    bool fresh = false;        // psi0 not yet in the state buffers
    int64_t off = 0;           // complex-entry offset in the current layout
    // results
    std::vector<double> psi, log;
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::string error;
    // eigen requests
    int nev = 0, block = 0, eig_max_it = 0, want_vectors = 0;
    double tol = 0;
    int nslots = 1;            // two-vector batch slots (propagation: 1)
    std::thread worker;
    int phase = kRunning;      // guarded by the server's mutex
    const double *ex = nullptr;
    double *ey = nullptr;
    int er = 0;                // vectors of the posted block
    sg_status apply_status = SG_OK, eig_status = SG_OK;
    int nconv = 0;
    std::vector<double> evals, resid, evecs;
};

}  // namespace

struct sg_server {
    sg_precision prec = SG_FP64;
    int device = 0;
    int64_t budget = 0, used = 0;
    cudaStream_t stream = nullptr;
    int64_t next_id = 1;
    std::map<int64_t, Req *> all;
    std::deque<Req *> queue;
    std::vector<Req *> active;
    sg_batch *batch = nullptr;
    bool dirty = false;
    // state buffers over the active requests (batch layout, nvec = 2)
    double *X = nullptr, *Y = nullptr, *P = nullptr, *A = nullptr;
    int64_t total = 0;
    int nslots = 0;
    sg::ChebState *d_state = nullptr;
    long long *d_prefix = nullptr;
    // two engine iterations (roles X -> P, then back), replayed between changes of
    // the active set; one graph per assignment of the two buffers to X
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
    const double *graph_x[2] = {nullptr, nullptr};
    int64_t iterations = 0, applications = 0;
    std::string last_error;
    // hand-off with the eigen requests' threads
    std::mutex mu;
    std::condition_variable cv;
    bool aborting = false;
};

namespace {

sg_status sfail(sg_server *s, sg_status st, const std::string &m)
{
    s->last_error = m;
    return st;
}

void free_state(sg_server *s)
{
    for (double **p : {&s->X, &s->Y, &s->P, &s->A})
        if (*p) { cudaFree(*p); *p = nullptr; }
    if (s->d_state) cudaFree(s->d_state);
    if (s->d_prefix) cudaFree(s->d_prefix);
    s->d_state = nullptr;
    s->d_prefix = nullptr;
    s->total = 0;
    for (int g = 0; g < 2; g++) {
        if (s->graph_exec[g]) cudaGraphExecDestroy(s->graph_exec[g]);
        if (s->graph[g]) cudaGraphDestroy(s->graph[g]);
        s->graph_exec[g] = nullptr;
        s->graph[g] = nullptr;
        s->graph_x[g] = nullptr;
    }
}

void release(sg_server *s, Req *r)
{
    if (r->worker.joinable()) r->worker.join();
    if (r->ctx) sg_destroy(r->ctx);
    r->ctx = nullptr;
    if (r->d_log) cudaFree(r->d_log);
    if (r->d_c) cudaFree(r->d_c);
    r->d_log = nullptr;
    r->d_c = nullptr;
    s->used -= r->bytes;
}

sg_status make_ctx(Req *r, sg_precision prec, bool device, sg_ctx **out)
{
    sg_poly V{(int)r->coef.size(), r->coef.data(), r->nfac.data(), r->mode.data(), r->power.data()};
    sg_hamiltonian H{r->omega.data(), V};
    return device ? sg_create(r->D, r->L, r->basis.data(), r->grids.data(), &H, prec, out)
                  : sg_plan(r->D, r->L, r->basis.data(), r->grids.data(), &H, prec, out);
}

// Spectral interval, Chebyshev weights and per-step constants of an admitted request.
sg_status prepare(sg_server *s, Req *r)
{
    double emin = 0, emax = 0;
    sg_status st = sg::chebyshev_bounds(r->ctx, s->stream, &emin, &emax);
    if (st != SG_OK) return st;
    r->ebar = 0.5 * (emax + emin);
    r->de = 0.5 * (emax - emin);
    const std::vector<double> J = sg::bessel_j(r->order, r->de * r->dt);
    int kend = r->order;  // skip terms whose Bessel weight is below double precision
    while (kend > 1 && kend > r->de * r->dt && std::fabs(J[kend]) < 1e-17) kend--;
    r->K = kend;
    r->c.assign(kend + 1, 0.0);
    for (int k = 0; k <= kend; k++) r->c[k] = (k == 0 ? 1.0 : 2.0) * J[k];
    r->cph = std::cos(r->ebar * r->dt);
    r->sph = -std::sin(r->ebar * r->dt);
    return SG_OK;
}

// New layout over the active requests' batch slots (a propagation request has
// one two-vector slot, an eigen request (block + 1) / 2); copies the surviving
// propagation states and uploads new ones.
sg_status relayout(sg_server *s)
{
    cudaError_t e;
    if (s->batch) { sg_batch_destroy(s->batch); s->batch = nullptr; }
    std::vector<long long> prefix(1, 0);
    std::vector<sg_ctx *> ctxs;
    std::vector<sg::ChebState> state;
    std::vector<int64_t> first_slot(s->active.size());
    for (size_t j = 0; j < s->active.size(); j++) {
        Req *r = s->active[j];
        first_slot[j] = prefix.back();
        for (int q = 0; q < r->nslots; q++) {
            prefix.push_back(prefix.back() + r->n_cs);
            ctxs.push_back(r->ctx);
            if (r->kind == kProp)
                state.push_back(sg::ChebState{r->k, r->K, r->step, r->nsteps, r->ebar, 1.0 / r->de, r->cph, r->sph,
                                              r->d_c, r->d_log});
            else  // never updated: the recurrence passes the slot through
                state.push_back(sg::ChebState{0, 1, 0, 0, 0.0, 1.0, 1.0, 0.0, nullptr, nullptr});
        }
    }
    const int64_t total = prefix.back();
    double *nb[4] = {nullptr, nullptr, nullptr, nullptr};
    if (total > 0) {
        for (double *&p : nb)
            if ((e = cudaMalloc(&p, sizeof(double) * 2 * (size_t)total)) != cudaSuccess) {
                for (double *q : nb) if (q) cudaFree(q);
                return sfail(s, SG_ENOMEM, std::string("server state cudaMalloc: ") + cudaGetErrorString(e));
            }
    }
    double *old[4] = {s->X, s->Y, s->P, s->A};
    for (size_t j = 0; j < s->active.size(); j++) {
        Req *r = s->active[j];
        const int64_t no = first_slot[j];
        if (r->kind == kProp) {
            const size_t bytes = sizeof(double) * 2 * (size_t)r->n_cs;
            if (r->fresh) {
                e = cudaMemcpyAsync(nb[0] + 2 * no, r->psi0.data(), bytes, cudaMemcpyHostToDevice, s->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // psi0 may be released next
                if (e != cudaSuccess) return sfail(s, SG_ECUDA, std::string("psi0 upload: ") + cudaGetErrorString(e));
                r->fresh = false;
                std::vector<double>().swap(r->psi0);
            } else {
                for (int b : {0, 2, 3})
                    if ((e = cudaMemcpyAsync(nb[b] + 2 * no, old[b] + 2 * r->off, bytes, cudaMemcpyDeviceToDevice,
                                             s->stream)) != cudaSuccess)
                        return sfail(s, SG_ECUDA, std::string("state move: ") + cudaGetErrorString(e));
            }
        }
        r->off = no;
    }
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return sfail(s, SG_ECUDA, std::string("relayout sync: ") + cudaGetErrorString(e));
    free_state(s);
    s->X = nb[0]; s->Y = nb[1]; s->P = nb[2]; s->A = nb[3];
    s->total = total;
    s->nslots = (int)state.size();
    const size_t na = std::max<size_t>(1, state.size());
    if ((e = cudaMalloc(&s->d_state, sizeof(sg::ChebState) * na)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_prefix, sizeof(long long) * (na + 1))) != cudaSuccess)
        return sfail(s, SG_ENOMEM, std::string("server tables cudaMalloc: ") + cudaGetErrorString(e));
    if ((e = cudaMemcpy(s->d_prefix, prefix.data(), sizeof(long long) * prefix.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (!state.empty() && (e = cudaMemcpy(s->d_state, state.data(), sizeof(sg::ChebState) * state.size(),
                                           cudaMemcpyHostToDevice)) != cudaSuccess))
        return sfail(s, SG_ECUDA, std::string("server tables upload: ") + cudaGetErrorString(e));
    if (!ctxs.empty()) {
        sg_status st = sg_batch_create(ctxs.data(), (int)ctxs.size(), &s->batch);
        if (st != SG_OK) return sfail(s, st, "sg_batch_create over the active requests failed");
    }
    s->dirty = false;
    return SG_OK;
}

// Whether an active request has finished: a propagation request after its
// last step, an eigen request when its solver thread has ended.
bool finished(sg_server *s, const Req *r)
{
    if (r->kind == kProp) return r->step >= r->nsteps;
    std::lock_guard<std::mutex> lk(s->mu);
    return r->phase == kFinished;
}

void retire(sg_server *s)
{
    bool any = false;
    for (const Req *r : s->active) any |= finished(s, r);
    if (!any) return;
    // the iterations run asynchronously on the server's (non-blocking) stream
    const cudaError_t es = cudaStreamSynchronize(s->stream);
    std::vector<Req *> keep;
    for (Req *r : s->active) {
        if (!finished(s, r)) { keep.push_back(r); continue; }
        if (r->kind == kEig) {
            if (r->worker.joinable()) r->worker.join();
            int derr = 0;
            if (r->eig_status == SG_OK || r->eig_status == SG_ENOCONV) sg_device_error(r->ctx, &derr);
            r->state = (r->eig_status == SG_OK || r->eig_status == SG_ENOCONV) && derr == 0 ? SG_REQ_DONE
                                                                                           : SG_REQ_FAILED;
            if (derr) r->error = "device error " + std::to_string(derr);
            r->t_done = now_s();
            release(s, r);
            s->dirty = true;
            continue;
        }
        r->psi.resize(2 * (size_t)r->n_cs);
        r->log.resize(2 * (size_t)r->nsteps);
        cudaError_t e = es;
        if (e == cudaSuccess)
            e = cudaMemcpy(r->psi.data(), s->X + 2 * r->off, sizeof(double) * r->psi.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && r->nsteps > 0)
            e = cudaMemcpy(r->log.data(), r->d_log, sizeof(double) * r->log.size(), cudaMemcpyDeviceToHost);
        int derr = 0;
        if (e == cudaSuccess) sg_device_error(r->ctx, &derr);
        r->state = (e == cudaSuccess && derr == 0) ? SG_REQ_DONE : SG_REQ_FAILED;
        if (e != cudaSuccess) r->error = cudaGetErrorString(e);
        else if (derr) r->error = "device error " + std::to_string(derr);
        r->t_done = now_s();
        release(s, r);
        s->dirty = true;
    }
    s->active.swap(keep);
}

// Host thread of an eigen request: the block Davidson of sg_eigs on the
// request's context, vector algebra on a stream of its own, every application
// of H_S handed to the engine (at most 2 * nslots vectors per engine
// iteration) and waited for.
void eig_worker(sg_server *s, Req *r)
{
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    sg_status res = SG_OK;
    std::string err;
    double *evecs = nullptr;
    const int64_t n = r->n_cs;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { res = SG_ECUDA; err = "stream"; }
    if (res == SG_OK && r->want_vectors &&
        cudaMalloc(&evecs, sizeof(double) * (size_t)n * r->nev) != cudaSuccess) { res = SG_ENOMEM; err = "eigenvectors"; }
    r->evals.assign(r->nev, 0.0);
    r->resid.assign(r->nev, 0.0);
    if (res == SG_OK) {
        const int cap = 2 * r->nslots;
        sg::ApplyFn fn = [s, r, n, cap](const double *x, double *y, int nr) -> sg_status {
            for (int j0 = 0; j0 < nr; j0 += cap) {
                std::unique_lock<std::mutex> lk(s->mu);
                r->ex = x + (size_t)j0 * n;
                r->ey = y + (size_t)j0 * n;
                r->er = std::min(cap, nr - j0);
                r->phase = kPosted;
                s->cv.notify_all();
                s->cv.wait(lk, [&] { return r->phase == kApplied || s->aborting; });
                if (s->aborting) return SG_ECUDA;
                r->phase = kRunning;
                if (r->apply_status != SG_OK) return r->apply_status;
            }
            return SG_OK;
        };
        int nconv = 0;
        res = sg::davidson_routed(r->ctx, st, fn, r->nev, r->block, r->tol, r->eig_max_it, r->evals.data(),
                                  r->resid.data(), evecs, &nconv, &err);
        r->nconv = nconv;
        if (res == SG_OK && nconv < r->nev) res = SG_ENOCONV;
        if (evecs && (res == SG_OK || res == SG_ENOCONV)) {
            r->evecs.resize((size_t)n * r->nev);
            if (cudaMemcpy(r->evecs.data(), evecs, sizeof(double) * r->evecs.size(), cudaMemcpyDeviceToHost) !=
                cudaSuccess) { res = SG_ECUDA; err = "eigenvector copy"; }
        }
    }
    if (evecs) cudaFree(evecs);
    if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    std::lock_guard<std::mutex> lk(s->mu);
    r->eig_status = res;
    if (res != SG_OK && res != SG_ENOCONV) r->error = err.empty() ? "eigen solver failed" : err;
    r->phase = kFinished;
    s->cv.notify_all();
}

sg_status admit(sg_server *s)
{
    while (!s->queue.empty() && s->used + s->queue.front()->bytes <= s->budget) {
        Req *r = s->queue.front();
        s->queue.pop_front();
        r->t_admit = now_s();
        if (r->kind == kProp && r->nsteps == 0) {  // nothing to propagate: the result is the initial state
            r->psi.swap(r->psi0);
            r->state = SG_REQ_DONE;
            r->t_done = now_s();
            continue;
        }
        s->used += r->bytes;
        sg_status st = make_ctx(r, s->prec, true, &r->ctx);
        if (r->kind == kEig) {
            if (st != SG_OK) {
                r->state = SG_REQ_FAILED;
                r->error = sg_last_error(nullptr);
                r->t_done = now_s();
                release(s, r);
                continue;
            }
            r->state = SG_REQ_ACTIVE;
            r->phase = kRunning;
            r->step = 0;
            s->active.push_back(r);
            s->dirty = true;
            r->worker = std::thread(eig_worker, s, r);
            continue;
        }
        if (st == SG_OK) st = prepare(s, r);
        cudaError_t e = cudaSuccess;
        if (st == SG_OK) {
            e = cudaMalloc(&r->d_log, sizeof(double) * 2 * (size_t)r->nsteps);
            if (e == cudaSuccess) e = cudaMalloc(&r->d_c, sizeof(double) * r->c.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(r->d_c, r->c.data(), sizeof(double) * r->c.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = SG_ENOMEM;
        }
        if (st != SG_OK) {
            r->state = SG_REQ_FAILED;
            r->error = r->ctx ? sg_last_error(r->ctx) : sg_last_error(nullptr);
            if (r->error.empty() && e != cudaSuccess) r->error = cudaGetErrorString(e);
            r->t_done = now_s();
            release(s, r);
            continue;
        }
        r->state = SG_REQ_ACTIVE;
        r->fresh = true;
        r->step = 0;
        r->k = 0;
        s->active.push_back(r);
        s->dirty = true;
    }
    return SG_OK;
}

// One engine iteration with the current roles of X and P: Y = H X over all
// active requests, then logs, recurrence update (into P) and state advance,
// over every two-vector slot (an eigen request holds several).
sg_status enqueue_iteration(sg_server *s, double *X, double *P)
{
    sg_status st = sg_apply_H_batch(s->batch, X, s->Y, 2, s->stream);
    if (st != SG_OK) return sfail(s, st, std::string("batched apply: ") + sg_batch_last_error(s->batch));
    cudaError_t e = sg::launch_cheb_iteration(s->d_state, s->d_prefix, s->nslots, s->total, X, s->Y, P, s->A,
                                              s->stream);
    if (e != cudaSuccess) return sfail(s, SG_ECUDA, std::string("recurrence update: ") + cudaGetErrorString(e));
    return SG_OK;
}

// Runs n iterations over the current active set (none of which passes a
// request's last step): pairs of iterations as one graph launch, a last odd
// one launched directly.  Asynchronous.
sg_status iterate(sg_server *s, int64_t n)
{
    cudaError_t e;
    sg_status st;
    int64_t done = 0;
    int slot = s->graph_x[0] == s->X ? 0 : (s->graph_x[1] == s->X ? 1 : -1);
    if (slot < 0 && n >= 3) {
        if (!s->graph_x[0] && !s->graph_x[1]) {
            // the first iteration sizes the batch workspace outside any capture
            if ((st = enqueue_iteration(s, s->X, s->P)) != SG_OK) return st;
            std::swap(s->X, s->P);
            done = 1;
        }
        slot = s->graph_x[0] ? 1 : 0;
        if ((e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return sfail(s, SG_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
        sg_status s1 = enqueue_iteration(s, s->X, s->P);
        sg_status s2 = s1 == SG_OK ? enqueue_iteration(s, s->P, s->X) : s1;
        e = cudaStreamEndCapture(s->stream, &s->graph[slot]);
        if (s2 != SG_OK) return s2;
        if (e != cudaSuccess) return sfail(s, SG_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
        if ((e = cudaGraphInstantiate(&s->graph_exec[slot], s->graph[slot], 0)) != cudaSuccess)
            return sfail(s, SG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        s->graph_x[slot] = s->X;
    }
    for (; slot >= 0 && done + 2 <= n; done += 2)
        if ((e = cudaGraphLaunch(s->graph_exec[slot], s->stream)) != cudaSuccess)
            return sfail(s, SG_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    for (; done < n; done++) {
        if ((st = enqueue_iteration(s, s->X, s->P)) != SG_OK) return st;
        std::swap(s->X, s->P);
    }
    for (Req *r : s->active)
        for (int64_t i = 0; i < n; i++) {
            if (r->k + 1 == r->K) { r->k = 0; r->step++; }
            else r->k++;
        }
    s->iterations += n;
    s->applications += 2 * (int64_t)s->active.size() * n;  // propagation requests only here
    return SG_OK;
}

// Iterations until the first active propagation request finishes its last step.
int64_t until_first_finish(const sg_server *s)
{
    int64_t m = INT64_MAX;
    for (const Req *r : s->active)
        if (r->kind == kProp) m = std::min<int64_t>(m, (int64_t)(r->nsteps - r->step - 1) * r->K + (r->K - r->k));
    return m;
}

bool has_eig(const sg_server *s)
{
    for (const Req *r : s->active)
        if (r->kind == kEig) return true;
    return false;
}

// Waits (at most 600 s) until every active eigen request has handed over a
// block or finished; *any_finished tells whether some finished.
sg_status wait_eig(sg_server *s, bool *any_finished)
{
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv.wait_for(lk, std::chrono::seconds(600), [&] {
        for (const Req *r : s->active)
            if (r->kind == kEig && r->phase != kPosted && r->phase != kFinished) return false;
        return true;
    });
    if (!ok) return sfail(s, SG_ETIMEOUT, "an eigen request did not hand over its block within 600 s");
    *any_finished = false;
    for (const Req *r : s->active) *any_finished |= r->kind == kEig && r->phase == kFinished;
    return SG_OK;
}

// One engine iteration with eigen requests active: their blocks go into
// their slots of X (unused vectors of a slot zero), one batched apply and
// recurrence update for everyone, the eigen results back to the requests.
sg_status eig_iteration(sg_server *s)
{
    cudaError_t e = cudaSuccess;
    for (const Req *r : s->active) {
        if (r->kind != kEig) continue;
        const size_t n = (size_t)r->n_cs;
        double *dst = s->X + 2 * r->off;
        e = cudaMemcpyAsync(dst, r->ex, sizeof(double) * n * r->er, cudaMemcpyDeviceToDevice, s->stream);
        if (e == cudaSuccess && r->er < 2 * r->nslots)
            e = cudaMemsetAsync(dst + n * r->er, 0, sizeof(double) * n * (2 * r->nslots - r->er), s->stream);
        if (e != cudaSuccess) return sfail(s, SG_ECUDA, std::string("eigen block copy: ") + cudaGetErrorString(e));
    }
    sg_status st = enqueue_iteration(s, s->X, s->P);
    if (st == SG_OK)
        for (const Req *r : s->active)
            if (r->kind == kEig && e == cudaSuccess)
                e = cudaMemcpyAsync(r->ey, s->Y + 2 * r->off, sizeof(double) * (size_t)r->n_cs * r->er,
                                    cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (st == SG_OK && e != cudaSuccess) st = sfail(s, SG_ECUDA, std::string("eigen iteration: ") + cudaGetErrorString(e));
    std::swap(s->X, s->P);
    int64_t apps = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Req *r : s->active) {
            if (r->kind == kProp) {
                apps += 2;
                if (r->k + 1 == r->K) { r->k = 0; r->step++; }
                else r->k++;
            } else {
                apps += r->er;
                r->apply_status = st;
                r->phase = kApplied;
                r->step++;
            }
        }
    }
    s->cv.notify_all();
    s->iterations += 1;
    s->applications += apps;
    return st;
}

}  // namespace

extern "C" {

sg_status sg_server_create(sg_precision prec, int64_t hbm_budget_bytes, sg_server **out)
{
    if (!out) return SG_EINVAL;
    *out = nullptr;
    if ((prec != SG_FP64 && prec != SG_MIXED) || hbm_budget_bytes <= 0) return SG_EINVAL;
    sg_server *s = new (std::nothrow) sg_server;
    if (!s) return SG_ENOMEM;
    s->prec = prec;
    s->budget = hbm_budget_bytes;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return SG_ECUDA;
    }
    *out = s;
    return SG_OK;
}

sg_status sg_server_submit(sg_server *s, const sg_prop_request *q, int64_t *id)
{
    if (!s) return SG_EINVAL;
    if (!q || !id || !q->basis || !q->grids || !q->H || !q->H->omega || q->nsteps < 0 || q->order < 1 ||
        !std::isfinite(q->dt) || (!q->psi0 && !q->factors))
        return sfail(s, SG_EINVAL, "sg_server_submit: invalid request");
    Req *r = new (std::nothrow) Req;
    if (!r) return SG_ENOMEM;
    r->D = q->D;
    r->L = q->L;
    if (r->D < 1 || r->D > sg::kMaxD) { delete r; return sfail(s, SG_EINVAL, "sg_server_submit: D out of range"); }
    r->basis.assign(q->basis, q->basis + r->D);
    r->grids.assign(q->grids, q->grids + r->D);
    r->omega.assign(q->H->omega, q->H->omega + r->D);
    const sg_poly &V = q->H->V;
    int nf = 0;
    for (int m = 0; m < V.nterms; m++) nf += V.nfac[m];
    r->coef.assign(V.coef, V.coef + V.nterms);
    r->nfac.assign(V.nfac, V.nfac + V.nterms);
    r->mode.assign(V.mode, V.mode + nf);
    r->power.assign(V.power, V.power + nf);
    r->dt = q->dt;
    r->nsteps = q->nsteps;
    r->order = q->order;
    sg_ctx *plan = nullptr;
    sg_status st = make_ctx(r, s->prec, false, &plan);
    if (st != SG_OK) {
        delete r;
        return sfail(s, st, std::string("sg_server_submit: ") + sg_last_error(nullptr));
    }
    int64_t n_cs = 0, n_terms = 0;
    sg_size(plan, &n_cs, &n_terms, nullptr, nullptr, nullptr);
    r->n_cs = n_cs;
    r->psi0.assign(2 * (size_t)n_cs, 0.0);
    if (q->psi0) std::copy(q->psi0, q->psi0 + 2 * n_cs, r->psi0.begin());
    else st = sg_product_state(plan, q->factors, q->ld, r->psi0.data());
    // tables + M^B + batch items + 4 state vectors, the batch workspace (2
    // vectors x 4 fixed-point words), the context's own one-vector workspace
    // (left by the spectral-bound run) + logs
    r->bytes = sg::planned_device_bytes(plan) + 8 * n_terms + 2 * n_cs * (4 * 8 + 32) + 32 * n_cs +
               16 * (int64_t)r->nsteps + ((int64_t)1 << 20);
    sg_destroy(plan);
    if (st != SG_OK) { delete r; return sfail(s, st, "sg_server_submit: bad initial-state factors"); }
    if (r->bytes > s->budget) {
        const int64_t b = r->bytes;
        delete r;
        return sfail(s, SG_EBUDGET, "sg_server_submit: request needs " + std::to_string(b) +
                                        " bytes of device memory, over the budget");
    }
    r->id = s->next_id++;
    r->t_submit = now_s();
    s->all[r->id] = r;
    s->queue.push_back(r);
    *id = r->id;
    return SG_OK;
}

sg_status sg_server_submit_eigs(sg_server *s, const sg_eig_request *q, int64_t *id)
{
    if (!s) return SG_EINVAL;
    if (!q || !id || !q->basis || !q->grids || !q->H || !q->H->omega || q->nev < 1 || !(q->tol > 0) ||
        q->max_it < 1)
        return sfail(s, SG_EINVAL, "sg_server_submit_eigs: invalid request");
    if (q->D < 1 || q->D > sg::kMaxD) return sfail(s, SG_EINVAL, "sg_server_submit_eigs: D out of range");
    Req *r = new (std::nothrow) Req;
    if (!r) return SG_ENOMEM;
    r->kind = kEig;
    r->D = q->D;
    r->L = q->L;
    r->basis.assign(q->basis, q->basis + r->D);
    r->grids.assign(q->grids, q->grids + r->D);
    r->omega.assign(q->H->omega, q->H->omega + r->D);
    const sg_poly &V = q->H->V;
    int nf = 0;
    for (int m = 0; m < V.nterms; m++) nf += V.nfac[m];
    r->coef.assign(V.coef, V.coef + V.nterms);
    r->nfac.assign(V.nfac, V.nfac + V.nterms);
    r->mode.assign(V.mode, V.mode + nf);
    r->power.assign(V.power, V.power + nf);
    r->nev = q->nev;
    r->block = q->block <= 0 ? std::min(q->nev, 8) : std::min(q->block, 8);
    r->nslots = (r->block + 1) / 2;
    r->tol = q->tol;
    r->eig_max_it = q->max_it;
    r->want_vectors = q->want_vectors ? 1 : 0;
    sg_ctx *plan = nullptr;
    sg_status st = make_ctx(r, s->prec, false, &plan);
    if (st != SG_OK) {
        delete r;
        return sfail(s, st, std::string("sg_server_submit_eigs: ") + sg_last_error(nullptr));
    }
    int64_t n_cs = 0, n_terms = 0;
    sg_size(plan, &n_cs, &n_terms, nullptr, nullptr, nullptr);
    const int64_t pb = sg::planned_device_bytes(plan);
    sg_destroy(plan);
    r->n_cs = n_cs;
    if (r->nev > n_cs) {
        delete r;
        return sfail(s, SG_EINVAL, "sg_server_submit_eigs: nev exceeds N_cs");
    }
    // tables + M^B + batch items per slot + 4 state vectors and the batch
    // workspace per slot + the Davidson basis and its images (2 kmax vectors),
    // Ritz vectors, residuals and directions, eigenvectors, Gram scratch
    const int64_t kmax = std::max(3 * r->nev, r->nev + 6 * r->block);
    const int64_t vecs = 2 * kmax + 2 * std::max(r->nev, r->block) + r->block + (r->want_vectors ? r->nev : 0);
    r->bytes = pb + r->nslots * (8 * n_terms + 2 * n_cs * (4 * 8 + 32)) + 8 * vecs * n_cs + ((int64_t)4 << 20);
    if (r->bytes > s->budget) {
        const int64_t b = r->bytes;
        delete r;
        return sfail(s, SG_EBUDGET, "sg_server_submit_eigs: request needs " + std::to_string(b) +
                                        " bytes of device memory, over the budget");
    }
    r->id = s->next_id++;
    r->t_submit = now_s();
    s->all[r->id] = r;
    s->queue.push_back(r);
    *id = r->id;
    return SG_OK;
}

sg_status sg_server_eig_result(sg_server *s, int64_t id, double *evals, double *resid, double *evecs_host,
                               double *times, int *converged)
{
    if (!s) return SG_EINVAL;
    auto f = s->all.find(id);
    if (f == s->all.end()) return sfail(s, SG_EINVAL, "sg_server_eig_result: unknown id");
    Req *r = f->second;
    if (r->kind != kEig) return sfail(s, SG_EINVAL, "sg_server_eig_result: a propagation request (sg_server_result)");
    if (r->state == SG_REQ_FAILED) return sfail(s, SG_ECUDA, "request failed: " + r->error);
    if (r->state != SG_REQ_DONE) return sfail(s, SG_EINVAL, "sg_server_eig_result: request not finished");
    if (evecs_host && !r->want_vectors)
        return sfail(s, SG_EINVAL, "sg_server_eig_result: the request did not ask for eigenvectors");
    if (evals) std::copy(r->evals.begin(), r->evals.end(), evals);
    if (resid) std::copy(r->resid.begin(), r->resid.end(), resid);
    if (evecs_host) std::copy(r->evecs.begin(), r->evecs.end(), evecs_host);
    if (times) {
        times[0] = r->t_admit - r->t_submit;
        times[1] = r->t_done - r->t_submit;
    }
    if (converged) *converged = r->nconv;
    return r->eig_status;
}

sg_status sg_server_progress(sg_server *s, int max_iters, int *n_active, int *n_queued)
{
    if (!s || max_iters < 0) return SG_EINVAL;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != s->device)
        return sfail(s, SG_EINVAL, "sg_server_progress: the server's device is not current");
    sg_status st = SG_OK;
    int64_t done = 0;
    while (done < max_iters) {
        retire(s);
        admit(s);
        if (s->dirty && (st = relayout(s)) != SG_OK) break;
        if (s->active.empty()) break;
        if (has_eig(s)) {
            bool fin = false;
            if ((st = wait_eig(s, &fin)) != SG_OK) break;
            if (fin) continue;  // retire the finished eigen requests first
            if ((st = eig_iteration(s)) != SG_OK) break;
            done += 1;
            continue;
        }
        const int64_t n = std::min<int64_t>(max_iters - done, until_first_finish(s));
        if ((st = iterate(s, n)) != SG_OK) break;
        done += n;
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (st == SG_OK && e != cudaSuccess) st = sfail(s, SG_ECUDA, std::string("progress: ") + cudaGetErrorString(e));
    if (st == SG_OK) retire(s);
    if (n_active) *n_active = (int)s->active.size();
    if (n_queued) *n_queued = (int)s->queue.size();
    return st;
}

sg_status sg_server_query(const sg_server *s, int64_t id, int *state, int64_t *n_cs, int *steps_done)
{
    if (!s) return SG_EINVAL;
    auto f = s->all.find(id);
    if (f == s->all.end()) return SG_EINVAL;
    const Req *r = f->second;
    if (state) *state = r->state;
    if (n_cs) *n_cs = r->n_cs;
    if (steps_done) *steps_done = r->step;
    return SG_OK;
}

sg_status sg_server_result(sg_server *s, int64_t id, double *psi_host, double *norm_log, double *energy_log,
                           double *times)
{
    if (!s) return SG_EINVAL;
    auto f = s->all.find(id);
    if (f == s->all.end()) return sfail(s, SG_EINVAL, "sg_server_result: unknown id");
    Req *r = f->second;
    if (r->kind != kProp) return sfail(s, SG_EINVAL, "sg_server_result: an eigen request (sg_server_eig_result)");
    if (r->state == SG_REQ_FAILED) return sfail(s, SG_ECUDA, "request failed: " + r->error);
    if (r->state != SG_REQ_DONE) return sfail(s, SG_EINVAL, "sg_server_result: request not finished");
    if (psi_host) std::copy(r->psi.begin(), r->psi.end(), psi_host);
    for (int k = 0; k < r->nsteps; k++) {
        if (norm_log) norm_log[k] = r->log[2 * (size_t)k];
        if (energy_log) energy_log[k] = r->log[2 * (size_t)k + 1];
    }
    if (times) {
        times[0] = r->t_admit - r->t_submit;
        times[1] = r->t_done - r->t_submit;
    }
    return SG_OK;
}

sg_status sg_server_stats(const sg_server *s, int64_t *iterations, int64_t *applications, int64_t *bytes_in_use)
{
    if (!s) return SG_EINVAL;
    if (iterations) *iterations = s->iterations;
    if (applications) *applications = s->applications;
    if (bytes_in_use) *bytes_in_use = s->used;
    return SG_OK;
}

const char *sg_server_last_error(const sg_server *s)
{
    return s ? s->last_error.c_str() : "";
}

void sg_server_destroy(sg_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->aborting = true;
    }
    s->cv.notify_all();
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (Req *r : s->active) release(s, r);
    if (s->batch) sg_batch_destroy(s->batch);
    free_state(s);
    for (auto &kv : s->all) delete kv.second;
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
