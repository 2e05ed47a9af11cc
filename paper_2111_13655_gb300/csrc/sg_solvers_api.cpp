// C ABI of the solvers: sg_eigs, sg_eigs_refine, sg_propagate, sg_product_state.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "sg_internal.h"

namespace sg {
cudaError_t dev_gram(const double *A, int ka, const double *B, int kb, int64_t n, double *C_dev, double *partial,
                     cudaStream_t s);
size_t gram_partial_doubles(int ka);
cudaError_t dev_combine(const double *V, int k, const double *S_dev, int r, double alpha, double beta, double *out,
                        int64_t n, cudaStream_t s);
cudaError_t dev_axpby(int64_t len, double a, const double *x, double b, double *y, cudaStream_t s);
cudaError_t dev_precond(const double *d, const double *theta_dev, int r, int64_t n, double *x, cudaStream_t s);
void sym_eig(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &Z);
int chol_inverse(int b, std::vector<double> &G);
std::vector<double> bessel_j(int kmax, double x);
}  // namespace sg

namespace {

using namespace sg;

constexpr int kBlk = 8;  // largest block size of the eigensolvers

struct SolverError {
    sg_status st;
    std::string msg;
};

void ck(cudaError_t e, const char *where)
{
    if (e != cudaSuccess) throw SolverError{SG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e)};
}

void ckst(sg_status st, sg_ctx *ctx)
{
    if (st != SG_OK) throw SolverError{st, sg_last_error(ctx)};
}

// device buffer owned by a solver call
struct DBuf {
    double *p = nullptr;
    explicit DBuf(size_t n) { ck(cudaMalloc(&p, std::max<size_t>(1, n) * sizeof(double)), "solver cudaMalloc"); }
    ~DBuf() { if (p) cudaFree(p); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
};

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Solver context: the apply, scratch, and small dense helpers.
struct Solver {
    sg_ctx *ctx;
    cudaStream_t s;
    int64_t n;
    DBuf partial, smalls;  // Gram scratch; small device matrices
    const ApplyFn *apply_fn = nullptr;  // when set, applications of H_S go through it
    Solver(sg_ctx *c, cudaStream_t st, int kmax)
        : ctx(c), s(st), n(c->host.n_cs), partial(gram_partial_doubles(std::max(kmax, 1))),
          smalls((size_t)std::max(kmax, 1) * kBlk * 2 + 64) {}

    void apply(const double *x, double *y, int r)
    {
        if (!apply_fn) { ckst(sg_apply_H(ctx, x, y, r, s), ctx); return; }
        // the routed apply reads x and writes y outside this stream: order both
        ck(cudaStreamSynchronize(s), "apply sync");
        const sg_status st = (*apply_fn)(x, y, r);
        if (st != SG_OK) throw SolverError{st, "routed apply failed"};
    }
    // C (ka x kb host, row-major) = A^T B
    std::vector<double> gram(const double *A, int ka, const double *B, int kb)
    {
        std::vector<double> C((size_t)ka * kb);
        for (int j0 = 0; j0 < kb; j0 += kBlk) {
            const int r = std::min(kBlk, kb - j0);
            ck(dev_gram(A, ka, B + (size_t)j0 * n, r, n, smalls.p, partial.p, s), "gram");
            std::vector<double> tmp((size_t)ka * r);
            ck(cudaMemcpyAsync(tmp.data(), smalls.p, sizeof(double) * ka * r, cudaMemcpyDeviceToHost, s), "gram copy");
            ck(cudaStreamSynchronize(s), "gram sync");
            for (int i = 0; i < ka; i++)
                for (int j = 0; j < r; j++) C[(size_t)i * kb + j0 + j] = tmp[(size_t)i * r + j];
        }
        return C;
    }
    // out (r x n) = beta out + alpha * V (k x n)^T-combination with S (k x r host, row-major)
    void combine(const double *V, int k, const std::vector<double> &S, int r, double alpha, double beta, double *out)
    {
        for (int j0 = 0; j0 < r; j0 += kBlk) {
            const int rr = std::min(kBlk, r - j0);
            std::vector<double> Sj((size_t)k * rr);
            for (int i = 0; i < k; i++)
                for (int j = 0; j < rr; j++) Sj[(size_t)i * rr + j] = S[(size_t)i * r + j0 + j];
            ck(cudaMemcpyAsync(smalls.p, Sj.data(), sizeof(double) * Sj.size(), cudaMemcpyHostToDevice, s), "S copy");
            ck(dev_combine(V, k, smalls.p, rr, alpha, beta, out + (size_t)j0 * n, n, s), "combine");
        }
    }
    // X (r x n) <- X - V V^T X, twice (V: k x n orthonormal)
    void orth_against(const double *V, int k, double *X, int r)
    {
        if (k <= 0) return;
        for (int pass = 0; pass < 2; pass++) {
            std::vector<double> C = gram(V, k, X, r);
            combine(V, k, C, r, -1.0, 1.0, X);
        }
    }
    // orthonormalise the r columns of X (Cholesky QR twice); returns the rank kept
    int orthonormalise(double *X, int r)
    {
        int rank = r;
        for (int pass = 0; pass < 2; pass++) {
            std::vector<double> G = gram(X, rank, X, rank);
            const int rk = chol_inverse(rank, G);
            DBuf tmp((size_t)rank * n);
            // X <- X R^{-1} (first rk columns)
            combine(X, rank, G, rk, 1.0, 0.0, tmp.p);
            ck(cudaMemcpyAsync(X, tmp.p, sizeof(double) * n * rk, cudaMemcpyDeviceToDevice, s), "orth copy");
            rank = rk;
            if (rank == 0) break;
        }
        return rank;
    }
    // Davidson start: unit vectors of the r lowest harmonic energies (the
    // preconditioner's diagonal; ties by index), so the subspace overlaps the
    // low-lying states from the first step.  False when no mode is split.
    bool lowest_diagonal_block(double *X, int r)
    {
        const std::vector<double> &d = ctx->host.esplit;
        if ((int64_t)d.size() != n) return false;
        bool any = false;
        for (double v : d) any |= v != 0.0;
        if (!any) return false;
        std::vector<int64_t> idx(n);
        for (int64_t i = 0; i < n; i++) idx[i] = i;
        std::partial_sort(idx.begin(), idx.begin() + r, idx.end(),
                          [&](int64_t a, int64_t b) { return d[a] < d[b] || (d[a] == d[b] && a < b); });
        std::vector<double> h((size_t)r * n, 0.0);
        for (int j = 0; j < r; j++) h[(size_t)j * n + idx[j]] = 1.0;
        ck(cudaMemcpyAsync(X, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s), "start copy");
        ck(cudaStreamSynchronize(s), "start sync");
        return true;
    }
    void random_block(double *X, int r, uint64_t seed)
    {
        std::vector<double> h((size_t)r * n);
        uint64_t st = seed;
        for (auto &v : h) v = (double)(splitmix(st) >> 11) * 0x1.0p-53 - 0.5;
        ck(cudaMemcpyAsync(X, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s), "random copy");
        ck(cudaStreamSynchronize(s), "random sync");
    }
    std::vector<double> norms(const double *X, int r)
    {
        std::vector<double> out(r);
        for (int j = 0; j < r; j++) {
            std::vector<double> g = gram(X + (size_t)j * n, 1, X + (size_t)j * n, 1);
            out[j] = std::sqrt(std::max(0.0, g[0]));
        }
        return out;
    }
};

// Block Davidson (or, without preconditioner and without restart, a block
// Lanczos-type Krylov method with full reorthogonalisation and Rayleigh-Ritz).
// Returns the number of converged eigenpairs; evals/resid on the host, the
// Ritz vectors in evecs (device, nev x n) when not null.
int block_eigs(Solver &S, int nev, int b, bool davidson, double tol, int max_it, const double *X0, int nx0,
               double *evals, double *evecs, double *resid)
{
    const int64_t n = S.n;
    // basis size: Davidson restarts at max(3 nev, nev + 6 b); the Krylov (Lanczos)
    // form keeps at most 320 vectors (its projected problem is solved densely)
    const int kmax = (int)std::min<int64_t>(n, davidson ? std::max(3 * nev, nev + 6 * b)
                                                        : std::min<int64_t>((int64_t)max_it * b + b, 320));
    DBuf V((size_t)kmax * n), W((size_t)kmax * n), X((size_t)std::max(nev, b) * n), HX((size_t)std::max(nev, b) * n),
        T((size_t)b * n), dd(kBlk + 8);
    std::vector<double> Tm;  // projected matrix, k x k
    int k = 0;
    // initial block
    int r0 = std::min<int64_t>(b, n);
    if (X0 && nx0 > 0) {
        r0 = std::min(nx0, kmax);
        ck(cudaMemcpyAsync(V.p, X0, sizeof(double) * n * r0, cudaMemcpyDeviceToDevice, S.s), "x0 copy");
    } else if (!davidson || !S.lowest_diagonal_block(V.p, r0)) {
        S.random_block(V.p, r0, 0x5eed1234ull);
    }
    r0 = S.orthonormalise(V.p, r0);
    auto extend = [&](int r) {  // V[k..k+r) are new orthonormal vectors: W = H V, grow Tm
        for (int j0 = 0; j0 < r; j0 += kBlk) {
            const int rr = std::min(kBlk, r - j0);
            S.apply(V.p + (size_t)(k + j0) * n, W.p + (size_t)(k + j0) * n, rr);
        }
        std::vector<double> C = S.gram(V.p, k + r, W.p + (size_t)k * n, r);  // (k+r) x r
        std::vector<double> Tn((size_t)(k + r) * (k + r));
        for (int i = 0; i < k; i++)
            for (int j = 0; j < k; j++) Tn[(size_t)i * (k + r) + j] = Tm[(size_t)i * k + j];
        for (int i = 0; i < k + r; i++)
            for (int j = 0; j < r; j++) {
                const double v = C[(size_t)i * r + j];
                Tn[(size_t)i * (k + r) + k + j] = v;
                Tn[(size_t)(k + j) * (k + r) + i] = v;
            }
        for (int i = k; i < k + r; i++)  // symmetrise the new diagonal block
            for (int j = i + 1; j < k + r; j++) {
                const double v = 0.5 * (Tn[(size_t)i * (k + r) + j] + Tn[(size_t)j * (k + r) + i]);
                Tn[(size_t)i * (k + r) + j] = Tn[(size_t)j * (k + r) + i] = v;
            }
        Tm.swap(Tn);
        k += r;
    };
    extend(r0);
    std::vector<double> theta, Z;
    int nconv = 0;
    const int ne = std::min<int64_t>(nev, n);
    for (int it = 0; it < max_it; it++) {
        sym_eig(k, Tm, theta, Z);
        const int nr = std::min(ne, k);
        // Ritz vectors and their images, residuals
        std::vector<double> Zr((size_t)k * nr);
        for (int i = 0; i < k; i++)
            for (int j = 0; j < nr; j++) Zr[(size_t)i * nr + j] = Z[(size_t)i * k + j];
        S.combine(V.p, k, Zr, nr, 1.0, 0.0, X.p);
        S.combine(W.p, k, Zr, nr, 1.0, 0.0, HX.p);
        for (int j = 0; j < nr; j++) ck(dev_axpby(n, -theta[j], X.p + (size_t)j * n, 1.0, HX.p + (size_t)j * n, S.s), "resid");
        std::vector<double> rn = S.norms(HX.p, nr);
        nconv = 0;
        while (nconv < nr && rn[nconv] <= tol * std::max(1.0, std::fabs(theta[nconv]))) nconv++;
        for (int j = 0; j < nr; j++) { evals[j] = theta[j]; if (resid) resid[j] = rn[j]; }
        if (nconv >= ne || k >= n) break;
        // new directions: the residuals of the first unconverged Ritz pairs
        int r = std::min(b, nr - nconv);
        if (r <= 0) r = 1;
        if (!davidson && k + r > kmax) break;
        const int first = std::min(nconv, nr - r);
        ck(cudaMemcpyAsync(T.p, HX.p + (size_t)first * n, sizeof(double) * n * r, cudaMemcpyDeviceToDevice, S.s), "dir copy");
        if (davidson) {
            const double *d = S.ctx->kp.esplit;  // harmonic energies: a diagonal preconditioner
            bool any = false;
            for (int i = 0; i < S.ctx->prob.D; i++) any |= S.ctx->host.harm_mono[i] >= 0;
            if (any) {
                std::vector<double> th(theta.begin() + first, theta.begin() + first + r);
                ck(cudaMemcpyAsync(dd.p, th.data(), sizeof(double) * r, cudaMemcpyHostToDevice, S.s), "theta copy");
                ck(dev_precond(d, dd.p, r, n, T.p, S.s), "precond");
            }
            if (k + r > kmax) {  // restart with the current Ritz vectors
                const int keep = std::min(nr, kmax - r);
                ck(cudaMemcpyAsync(V.p, X.p, sizeof(double) * n * keep, cudaMemcpyDeviceToDevice, S.s), "restart V");
                k = 0;
                Tm.clear();
                extend(S.orthonormalise(V.p, keep));  // recomputes W = H V
            }
        }
        S.orth_against(V.p, k, T.p, r);
        int rk = S.orthonormalise(T.p, r);
        if (rk == 0) {  // the directions lie in the basis: add random ones
            S.random_block(T.p, r, 0x5eed0000ull + (uint64_t)it);
            S.orth_against(V.p, k, T.p, r);
            rk = S.orthonormalise(T.p, r);
            if (rk == 0) break;
        }
        ck(cudaMemcpyAsync(V.p + (size_t)k * n, T.p, sizeof(double) * n * rk, cudaMemcpyDeviceToDevice, S.s), "append");
        extend(rk);
    }
    if (evecs) ck(cudaMemcpyAsync(evecs, X.p, sizeof(double) * n * std::min(ne, k), cudaMemcpyDeviceToDevice, S.s), "evecs");
    ck(cudaStreamSynchronize(S.s), "eigs sync");
    return nconv;
}

// Spectral interval of H_S for the Chebyshev propagator: a 40-vector Krylov
// run (Rayleigh-Ritz), the extreme Ritz values widened by their residual norms
// and by 5% of the range.  Deterministic (fixed start vector, ordered sums).
void spectral_bounds(Solver &S, double &emin, double &emax)
{
    const int64_t n = S.n;
    const int ks = (int)std::min<int64_t>(n, 40);
    {
        DBuf V((size_t)(ks + 1) * n), W((size_t)(ks + 1) * n), Xr(2 * (size_t)n), HXr(2 * (size_t)n);
        S.random_block(V.p, 1, 0xc4eb00ull);
        S.orthonormalise(V.p, 1);
        std::vector<double> Tm;
        int k = 0;
        for (int it = 0; it < ks; it++) {
            S.apply(V.p + (size_t)k * n, W.p + (size_t)k * n, 1);
            std::vector<double> C = S.gram(V.p, k + 1, W.p + (size_t)k * n, 1);
            std::vector<double> Tn((size_t)(k + 1) * (k + 1));
            for (int i = 0; i < k; i++)
                for (int j = 0; j < k; j++) Tn[(size_t)i * (k + 1) + j] = Tm[(size_t)i * k + j];
            for (int i = 0; i <= k; i++) Tn[(size_t)i * (k + 1) + k] = Tn[(size_t)k * (k + 1) + i] = C[i];
            Tm.swap(Tn);
            k++;
            if (k >= ks) break;
            ck(cudaMemcpyAsync(V.p + (size_t)k * n, W.p + (size_t)(k - 1) * n, sizeof(double) * n,
                               cudaMemcpyDeviceToDevice, S.s), "krylov copy");
            S.orth_against(V.p, k, V.p + (size_t)k * n, 1);
            if (S.orthonormalise(V.p + (size_t)k * n, 1) == 0) break;
        }
        std::vector<double> th, Z;
        sym_eig(k, Tm, th, Z);
        double rlo = 0, rhi = 0;
        for (int end = 0; end < 2; end++) {
            const int j = end == 0 ? 0 : k - 1;
            std::vector<double> z(k);
            for (int i = 0; i < k; i++) z[i] = Z[(size_t)i * k + j];
            S.combine(V.p, k, z, 1, 1.0, 0.0, Xr.p);
            S.combine(W.p, k, z, 1, 1.0, 0.0, HXr.p);
            ck(dev_axpby(n, -th[j], Xr.p, 1.0, HXr.p, S.s), "bound resid");
            const double rr = S.norms(HXr.p, 1)[0];
            (end == 0 ? rlo : rhi) = rr;
        }
        const double range = th[k - 1] - th[0];
        emin = th[0] - rlo - 0.05 * range;
        emax = th[k - 1] + rhi + 0.05 * range;
    }
}

}  // namespace

extern "C" {

sg_status sg_eigs(sg_ctx *ctx, int nev, int method, int block, double tol, int max_it, double *evals,
                  double *evecs, double *resid, void *stream)
{
    if (!ctx) return SG_EINVAL;
    if (!ctx->has_device) { ctx->last_error = "context was made by sg_plan"; return SG_EINVAL; }
    if (!sg_on_ctx_device(ctx)) { ctx->last_error = "the current CUDA device is not the one the context was made on"; return SG_EINVAL; }
    if (nev < 1 || nev > ctx->host.n_cs || !evals || !(tol > 0) || max_it < 1 ||
        (method != SG_LANCZOS && method != SG_DAVIDSON)) {
        ctx->last_error = "sg_eigs: need 1 <= nev <= N_cs, tol > 0, max_it >= 1, a known method, evals";
        return SG_EINVAL;
    }
    const int b = block <= 0 ? std::min(nev, kBlk) : std::min(block, kBlk);
    try {
        Solver S(ctx, (cudaStream_t)stream, std::max(3 * nev, nev + 6 * b) + 328);
        const int nconv = block_eigs(S, nev, b, method == SG_DAVIDSON, tol, max_it, nullptr, 0, evals, evecs, resid);
        if (nconv < std::min<int64_t>(nev, ctx->host.n_cs)) {
            ctx->last_error = "sg_eigs: " + std::to_string(nconv) + " of " + std::to_string(nev) + " eigenpairs converged";
            return SG_ENOCONV;
        }
    } catch (const SolverError &e) {
        ctx->last_error = e.msg;
        return e.st;
    }
    return SG_OK;
}

sg_status sg_eigs_refine(sg_ctx *ctx, int nev, double *evecs, double *evals, double *resid, double tol, int max_it,
                         void *stream)
{
    if (!ctx) return SG_EINVAL;
    if (!ctx->has_device || nev < 1 || nev > ctx->host.n_cs || !evecs || !evals || !(tol > 0) || max_it < 1) {
        ctx->last_error = "sg_eigs_refine: invalid arguments";
        return SG_EINVAL;
    }
    if (!sg_on_ctx_device(ctx)) { ctx->last_error = "the current CUDA device is not the one the context was made on"; return SG_EINVAL; }
    const int b = std::min(nev, kBlk);
    try {
        Solver S(ctx, (cudaStream_t)stream, std::max(3 * nev, nev + 6 * b) + 8);
        const int nconv = block_eigs(S, nev, b, true, tol, max_it, evecs, nev, evals, evecs, resid);
        if (nconv < nev) {
            ctx->last_error = "sg_eigs_refine: " + std::to_string(nconv) + " of " + std::to_string(nev) + " converged";
            return SG_ENOCONV;
        }
    } catch (const SolverError &e) {
        ctx->last_error = e.msg;
        return e.st;
    }
    return SG_OK;
}

sg_status sg_product_state(const sg_ctx *ctx, const double *factors, int ld, double *out_host)
{
    if (!ctx || !factors || !out_host || ld < ctx->host.kw) return SG_EINVAL;
    const int D = ctx->prob.D, L = ctx->prob.L, kw = ctx->host.kw;
    const std::vector<uint8_t> &lmin = ctx->host.lmin_tab;
    std::vector<int> k(D, 0), c(D, 0);
    int sum = 0;
    int64_t r = 0;
    for (;;) {
        double v = 1.0;
        for (int i = 0; i < D; i++) v *= factors[(size_t)i * ld + k[i]];
        out_host[r++] = v;
        int i = D - 1;
        while (i >= 0) {
            k[i]++;
            const int lm = k[i] < kw ? lmin[(size_t)i * kw + k[i]] : 255;
            if (lm <= L && sum - c[i] + lm <= L) { sum += lm - c[i]; c[i] = lm; break; }
            sum -= c[i]; c[i] = 0; k[i] = 0; i--;
        }
        if (i < 0) break;
    }
    return r == ctx->host.n_cs ? SG_OK : SG_EINVAL;
}

sg_status sg_propagate(sg_ctx *ctx, double *psi, double dt, int nsteps, int order, double *norm_log,
                       double *energy_log, void *stream)
{
    if (!ctx) return SG_EINVAL;
    if (!ctx->has_device || !psi || nsteps < 0 || order < 1 || !std::isfinite(dt)) {
        ctx->last_error = "sg_propagate: invalid arguments";
        return SG_EINVAL;
    }
    if (!sg_on_ctx_device(ctx)) { ctx->last_error = "the current CUDA device is not the one the context was made on"; return SG_EINVAL; }
    try {
        Solver S(ctx, (cudaStream_t)stream, 48);
        const int64_t n = S.n;
        double emin, emax;
        spectral_bounds(S, emin, emax);
        const double Ebar = 0.5 * (emax + emin), dE = 0.5 * (emax - emin);
        const std::vector<double> J = bessel_j(order, dE * dt);
        int kend = order;  // skip terms whose Bessel weight is below double precision
        while (kend > 1 && kend > dE * dt && std::fabs(J[kend]) < 1e-17) kend--;
        // phi buffers: 2 real vectors (re, im) each
        DBuf p0(2 * (size_t)n), p1(2 * (size_t)n), hp(2 * (size_t)n), acc(2 * (size_t)n);
        const double cph = std::cos(Ebar * dt), sph = -std::sin(Ebar * dt);  // e^{-i Ebar dt}
        for (int step = 0; step < nsteps; step++) {
            // phi_0 = psi, phi_1 = (H - Ebar) psi / dE
            ck(cudaMemcpyAsync(p0.p, psi, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, S.s), "cheb copy");
            S.apply(p0.p, hp.p, 2);
            if (norm_log || energy_log) {
                std::vector<double> a = S.gram(psi, 1, psi, 1), bq = S.gram(psi + n, 1, psi + n, 1);
                std::vector<double> c1 = S.gram(psi, 1, hp.p, 1), c2 = S.gram(psi + n, 1, hp.p + n, 1);
                const double nn = a[0] + bq[0];
                if (norm_log) norm_log[step] = nn;
                if (energy_log) energy_log[step] = (c1[0] + c2[0]) / nn;
            }
            ck(cudaMemcpyAsync(p1.p, hp.p, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, S.s), "cheb copy");
            ck(dev_axpby(2 * n, -Ebar / dE, p0.p, 1.0 / dE, p1.p, S.s), "cheb phi1");
            // acc = J0 phi0 + 2 J1 (-i) phi1
            ck(dev_axpby(2 * n, J[0], p0.p, 0.0, acc.p, S.s), "acc0");
            auto add_term = [&](int kk, const double *ph) {
                const double c = (kk == 0 ? 1.0 : 2.0) * J[kk];
                // (-i)^kk (x + i y): 0: x + iy; 1: y - ix; 2: -x - iy; 3: -y + ix
                const double *x = ph, *y = ph + n;
                double *ar = acc.p, *ai = acc.p + n;
                switch (kk % 4) {
                    case 0: ck(dev_axpby(n, c, x, 1.0, ar, S.s), "t"); ck(dev_axpby(n, c, y, 1.0, ai, S.s), "t"); break;
                    case 1: ck(dev_axpby(n, c, y, 1.0, ar, S.s), "t"); ck(dev_axpby(n, -c, x, 1.0, ai, S.s), "t"); break;
                    case 2: ck(dev_axpby(n, -c, x, 1.0, ar, S.s), "t"); ck(dev_axpby(n, -c, y, 1.0, ai, S.s), "t"); break;
                    default: ck(dev_axpby(n, -c, y, 1.0, ar, S.s), "t"); ck(dev_axpby(n, c, x, 1.0, ai, S.s), "t"); break;
                }
            };
            add_term(1, p1.p);
            double *a0 = p0.p, *a1 = p1.p;
            for (int kk = 2; kk <= kend; kk++) {
                // phi_{k} = 2 (H - Ebar)/dE phi_{k-1} - phi_{k-2}, written over phi_{k-2}
                S.apply(a1, hp.p, 2);
                ck(dev_axpby(2 * n, -2.0 * Ebar / dE, a1, -1.0, a0, S.s), "cheb rec");
                ck(dev_axpby(2 * n, 2.0 / dE, hp.p, 1.0, a0, S.s), "cheb rec");
                std::swap(a0, a1);
                add_term(kk, a1);
            }
            // psi = e^{-i Ebar dt} acc
            ck(dev_axpby(n, cph, acc.p, 0.0, psi, S.s), "phase");
            ck(dev_axpby(n, -sph, acc.p + n, 1.0, psi, S.s), "phase");
            ck(dev_axpby(n, sph, acc.p, 0.0, psi + n, S.s), "phase");
            ck(dev_axpby(n, cph, acc.p + n, 1.0, psi + n, S.s), "phase");
        }
        ck(cudaStreamSynchronize(S.s), "propagate sync");
    } catch (const SolverError &e) {
        ctx->last_error = e.msg;
        return e.st;
    }
    return SG_OK;
}

}  // extern "C"

namespace sg {

sg_status davidson_routed(sg_ctx *ctx, cudaStream_t stream, const ApplyFn &apply, int nev, int block, double tol,
                          int max_it, double *evals, double *resid, double *evecs, int *nconv, std::string *err)
{
    const int b = block <= 0 ? std::min(nev, kBlk) : std::min(block, kBlk);
    try {
        Solver S(ctx, stream, std::max(3 * nev, nev + 6 * b) + 328);
        S.apply_fn = &apply;
        *nconv = block_eigs(S, nev, b, true, tol, max_it, nullptr, 0, evals, evecs, resid);
    } catch (const SolverError &e) {
        if (err) *err = e.msg;
        return e.st;
    }
    return SG_OK;
}

sg_status chebyshev_bounds(sg_ctx *ctx, cudaStream_t stream, double *emin, double *emax)
{
    try {
        Solver S(ctx, stream, 48);
        spectral_bounds(S, *emin, *emax);
        ck(cudaStreamSynchronize(S.s), "bounds sync");
    } catch (const SolverError &e) {
        ctx->last_error = e.msg;
        return e.st;
    }
    return SG_OK;
}

}  // namespace sg
