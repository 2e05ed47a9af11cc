// C ABI of libsmolyak (declared in include/smolyak.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "sg_df.cuh"
#include "sg_internal.h"

namespace {

thread_local std::string g_create_error;

sg_status fail(sg_ctx *ctx, sg_status st, const std::string &msg)
{
    if (ctx) ctx->last_error = msg; else g_create_error = msg;
    return st;
}

sg_status cuda_fail(sg_ctx *ctx, cudaError_t e, const char *where)
{
    return fail(ctx, SG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// FP64 values as double-float pairs (hi = fl32(d), lo = fl32(d - hi))
std::vector<float2> df_pairs(const std::vector<double> &v)
{
    std::vector<float2> out(v.size());
    for (size_t i = 0; i < v.size(); i++) {
        const sg::df2 d(v[i]);
        out[i] = make_float2(d.hi, d.lo);
    }
    return out;
}

template <typename T>
sg_status upload(sg_ctx *ctx, const std::vector<T> &v, const T **dst)
{
    void *p = nullptr;
    size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(ctx, SG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    ctx->allocations.push_back(p);
    ctx->bytes_device += (int64_t)bytes;
    if (!v.empty()) {
        e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy");
    }
    *dst = static_cast<const T *>(p);
    return SG_OK;
}

void free_all(sg_ctx *ctx)
{
    for (void *p : ctx->allocations) cudaFree(p);
    ctx->allocations.clear();
    if (ctx->stage_x) cudaFree(ctx->stage_x);
    if (ctx->stage_y) cudaFree(ctx->stage_y);
    ctx->stage_x = ctx->stage_y = nullptr;
    if (ctx->acc) cudaFree(ctx->acc);
    if (ctx->maxbits) cudaFree(ctx->maxbits);
    if (ctx->xs) cudaFree(ctx->xs);
    ctx->acc = nullptr;
    ctx->maxbits = nullptr;
    ctx->xs = nullptr;
    ctx->acc_nvec = 0;
}

// Apply workspace for nvec vectors: fixed-point accumulators (zeroed here and
// left zeroed by every apply), the per-vector max|x| words and, for the fast
// path, the entry-major input copy.
sg_status ensure_workspace(sg_ctx *ctx, int nvec, cudaStream_t s)
{
    if (nvec <= ctx->acc_nvec) return SG_OK;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    if (ctx->acc) cudaFree(ctx->acc);
    if (ctx->maxbits) cudaFree(ctx->maxbits);
    if (ctx->xs) cudaFree(ctx->xs);
    ctx->acc = nullptr;
    ctx->maxbits = nullptr;
    ctx->xs = nullptr;
    ctx->kp.xs = nullptr;
    ctx->kp.xs_nvec = 0;
    ctx->acc_nvec = 0;
    const size_t words = (size_t)ctx->host.n_cs * nvec * sg::acc_words(ctx->fp32);
    if ((e = cudaMalloc(&ctx->acc, words * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&ctx->maxbits, sizeof(long long) * nvec)) != cudaSuccess)
        return fail(ctx, SG_ENOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
#if SG_STAGE_X
    if (ctx->kp.fast.enabled) {
        const size_t xs_bytes = (size_t)ctx->host.n_cs * sg::xs_stride(nvec) * (ctx->fp32 ? 4 : 8);
        if ((e = cudaMalloc(&ctx->xs, xs_bytes)) != cudaSuccess)
            return fail(ctx, SG_ENOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
        ctx->kp.xs = ctx->xs;
        ctx->kp.xs_nvec = nvec;
    }
#endif
    if ((e = cudaMemsetAsync(ctx->acc, 0, words * sizeof(unsigned long long), s)) != cudaSuccess)
        return cuda_fail(ctx, e, "workspace memset");
    ctx->acc_nvec = nvec;
    ctx->kp.acc = ctx->acc;
    return SG_OK;
}

// Device shared-memory opt-in limit of sm_100-class GPUs, used to size plans
// made without a device (sg_plan).
constexpr int kPlanSmemOptin = 232448;

sg_status plan(int D, int L, const sg_basis *basis, const sg_grid *grids,
                     const sg_hamiltonian *H, sg_precision prec, int smem_optin, sg_ctx **out)
{
    using namespace sg;
    if (!out) return fail(nullptr, SG_EINVAL, "out is NULL");
    *out = nullptr;
    if (D < 1) return fail(nullptr, SG_EINVAL, "D must be >= 1");
    if (D > kMaxD) return fail(nullptr, SG_EUNSUPPORTED, "D > 32");
    if (L < 0) return fail(nullptr, SG_EINVAL, "L must be >= 0");
    if (!basis || !grids || !H || !H->omega) return fail(nullptr, SG_EINVAL, "NULL basis/grids/H/omega");
    if (prec != SG_FP64 && prec != SG_MIXED && prec != SG_DF64) return fail(nullptr, SG_EINVAL, "unknown precision");
    for (int i = 0; i < D; i++) {
        const sg_basis &b = basis[i];
        const sg_grid &g = grids[i];
        if (b.nb_A < 1 || b.nb_B < 0 || g.nq_A < b.nb_A || g.nq_B < b.nb_B)
            return fail(nullptr, SG_EINVAL, "mode rules need nb_A>=1, nb_B>=0, nq_A>=nb_A, nq_B>=nb_B");
        if (!(b.scale > 0) || !std::isfinite(b.scale) || !std::isfinite(b.q0))
            return fail(nullptr, SG_EINVAL, "scale must be finite and > 0, q0 finite");
        if ((int64_t)g.nq_A + (int64_t)g.nq_B * L > kMaxLevelSize)
            return fail(nullptr, SG_EUNSUPPORTED, "nq(L) > 32");
        if (!std::isfinite(H->omega[i])) return fail(nullptr, SG_EINVAL, "omega not finite");
    }
    const sg_poly &V = H->V;
    if (V.nterms < 0) return fail(nullptr, SG_EINVAL, "V.nterms < 0");
    if (V.nterms > kMaxMono) return fail(nullptr, SG_EUNSUPPORTED, "more than 256 monomials");
    if (V.nterms > 0 && (!V.coef || !V.nfac)) return fail(nullptr, SG_EINVAL, "NULL V arrays");

    sg_ctx *ctx = new (std::nothrow) sg_ctx();
    if (!ctx) return fail(nullptr, SG_ENOMEM, "host allocation failed");
    Problem &p = ctx->prob;
    p.D = D; p.L = L; p.prec = prec;
    p.basis.assign(basis, basis + D);
    p.grids.assign(grids, grids + D);
    p.omega.assign(H->omega, H->omega + D);
    p.mfoff.push_back(0);
    for (int m = 0; m < V.nterms; m++) {
        if (V.nfac[m] < 0 || V.nfac[m] > kMaxFac) { delete ctx; return fail(nullptr, SG_EUNSUPPORTED, "monomial with more than 8 factors"); }
        if (!std::isfinite(V.coef[m])) { delete ctx; return fail(nullptr, SG_EINVAL, "V coefficient not finite"); }
        if (V.nfac[m] > 0 && (!V.mode || !V.power)) { delete ctx; return fail(nullptr, SG_EINVAL, "NULL V factor arrays"); }
        p.mcoef.push_back(V.coef[m]);
        p.mnfac.push_back(V.nfac[m]);
        int tot[kMaxD] = {0};
        for (int f = p.mfoff[m]; f < p.mfoff[m] + V.nfac[m]; f++) {
            if (V.mode[f] < 0 || V.mode[f] >= D) { delete ctx; return fail(nullptr, SG_EINVAL, "factor mode out of range"); }
            if (V.power[f] < 1 || V.power[f] > kMaxPow) { delete ctx; return fail(nullptr, SG_EUNSUPPORTED, "factor power outside 1..16"); }
            tot[V.mode[f]] += V.power[f];
            if (tot[V.mode[f]] > kMaxPow) { delete ctx; return fail(nullptr, SG_EUNSUPPORTED, "total power of a mode > 16"); }
            p.mfmode.push_back(V.mode[f]);
            p.mfpow.push_back(V.power[f]);
        }
        p.mfoff.push_back(p.mfoff[m] + V.nfac[m]);
    }
    ctx->fp32 = (prec == SG_MIXED);
    const int budget = std::min(smem_optin - 4096, ctx->fp32 ? 72 * 1024 : 110 * 1024);
    std::string err = build_tables(p, budget, ctx->fp32 ? 4 : 8, &ctx->host);
    if (!err.empty()) { delete ctx; return fail(nullptr, SG_EUNSUPPORTED, err); }
    HostTables &T = ctx->host;
    KParams &kp = ctx->kp;
    kp.D = D; kp.L = L; kp.Dpad = T.Dpad;
    kp.nmono = (int)p.mcoef.size(); kp.pmax = T.pmax; kp.kw = T.kw;
    kp.n_cs = (int)T.n_cs; kp.n_terms = T.n_terms;
    kp.part = 0; kp.nparts = 1;
    kp.cap = T.cap; kp.maxnb = T.maxnb; kp.matcap = T.matcap; kp.vtabcap = T.vtabcap;
    *out = ctx;
    return SG_OK;
}

}  // namespace

namespace sg {

int64_t planned_device_bytes(const sg_ctx *ctx)
{
    const HostTables &T = ctx->host;
    const Problem &p = ctx->prob;
    auto b = [](const auto &v) { return (int64_t)v.size() * (int64_t)sizeof(v[0]); };
    int64_t bytes = b(T.levels) + b(T.coefs) + b(T.order) + b(T.rank_tab) + b(T.lmin_tab) + b(T.lvl) +
                    b(T.tabd) * 3 / 2 + b(p.mcoef) + b(p.mnfac) + b(p.mfoff) + b(p.mfmode) + b(p.mfpow) +
                    b(T.harm_mono) + b(T.esplit);
    if (T.fast)
        bytes += b(T.pair_modes) + b(T.h1off) + b(T.goff) + b(T.ioff) + b(T.soff) + b(T.spoff) + b(T.fsc) +
                 b(T.ftab) * 3 / 2 + b(T.fdesc) + b(T.fdesc_off) + T.franks * (int64_t)sizeof(int) +
                 b(T.fimg) / (ctx->fp32 ? 2 : 1) + b(T.fimg_off) + b(T.fvt_off) + b(T.frank_start) +
                 (T.fvt_off.empty() ? 0 : T.fvt_off.back()) * (ctx->fp32 ? 4 : 8);
    return bytes;
}

}  // namespace sg

extern "C" {

sg_status sg_plan(int D, int L, const sg_basis *basis, const sg_grid *grids,
                  const sg_hamiltonian *H, sg_precision prec, sg_ctx **out)
{
    return plan(D, L, basis, grids, H, prec, kPlanSmemOptin, out);
}

sg_status sg_create(int D, int L, const sg_basis *basis, const sg_grid *grids,
                    const sg_hamiltonian *H, sg_precision prec, sg_ctx **out)
{
    using namespace sg;
    if (!out) return fail(nullptr, SG_EINVAL, "out is NULL");
    *out = nullptr;
    int device = 0, smem_optin = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
    sg_ctx *ctx = nullptr;
    sg_status st0 = plan(D, L, basis, grids, H, prec, smem_optin, &ctx);
    if (st0 != SG_OK) return st0;
    ctx->device = device;
    Problem &p = ctx->prob;
    HostTables &T = ctx->host;
    KParams &kp = ctx->kp;
    std::vector<float> tabf(T.tabd.begin(), T.tabd.end());
    std::vector<float> ftabf(T.ftab.begin(), T.ftab.end());
    std::vector<int> zero(1, 0);
    sg_status st = SG_OK;
    const int *errp = nullptr;
    if ((st = upload(ctx, T.levels, &kp.levels)) != SG_OK ||
        (st = upload(ctx, T.coefs, &kp.coefs)) != SG_OK ||
        (st = upload(ctx, T.order, &kp.order)) != SG_OK ||
        (st = upload(ctx, T.rank_tab, &kp.rank_tab)) != SG_OK ||
        (st = upload(ctx, T.lmin_tab, &kp.lmin_tab)) != SG_OK ||
        (st = upload(ctx, T.lvl, &kp.lvl)) != SG_OK ||
        (st = upload(ctx, T.tabd, &kp.tabd)) != SG_OK ||
        (st = upload(ctx, tabf, &kp.tabf)) != SG_OK ||
        (st = upload(ctx, p.mcoef, &kp.mcoef)) != SG_OK ||
        (st = upload(ctx, p.mnfac, &kp.mnfac)) != SG_OK ||
        (st = upload(ctx, p.mfoff, &kp.mfoff)) != SG_OK ||
        (st = upload(ctx, p.mfmode, &kp.mfmode)) != SG_OK ||
        (st = upload(ctx, p.mfpow, &kp.mfpow)) != SG_OK ||
        (st = upload(ctx, T.harm_mono, &kp.harm_mono)) != SG_OK ||
        (st = upload(ctx, T.esplit, &kp.esplit)) != SG_OK ||
        (st = upload(ctx, zero, &errp)) != SG_OK ||
        (T.fast && ((st = upload(ctx, T.pair_modes, &kp.fast.pair_modes)) != SG_OK ||
                    (st = upload(ctx, T.h1off, &kp.fast.h1off)) != SG_OK ||
                    (st = upload(ctx, T.goff, &kp.fast.goff)) != SG_OK ||
                    (st = upload(ctx, T.ioff, &kp.fast.ioff)) != SG_OK ||
                    (st = upload(ctx, T.soff, &kp.fast.soff)) != SG_OK ||
                    (st = upload(ctx, T.spoff, &kp.fast.spoff)) != SG_OK ||
                    (st = upload(ctx, T.fsc, &kp.fast.sc)) != SG_OK ||
                    (st = upload(ctx, T.ftab, &kp.fast.tabd)) != SG_OK ||
                    (st = upload(ctx, ftabf, &kp.fast.tabf)) != SG_OK ||
                    (st = upload(ctx, T.fdesc, &kp.fast.desc)) != SG_OK ||
                    (st = upload(ctx, T.fdesc_off, &kp.fast.desc_off)) != SG_OK ||
                    (st = upload(ctx, T.fimg_off, &kp.fast.img_off)) != SG_OK ||
                    (st = upload(ctx, T.fvt_off, &kp.fast.mt_off)) != SG_OK ||
                    (st = upload(ctx, T.frank_start, &kp.fast.rank_start)) != SG_OK ||
                    (ctx->fp32 ? (st = upload(ctx, std::vector<float>(T.fimg.begin(), T.fimg.end()),
                                              &kp.fast.imgf)) != SG_OK
                     : p.prec == SG_DF64 ? (st = upload(ctx, df_pairs(T.fimg), &kp.fast.imgx)) != SG_OK
                                         : (st = upload(ctx, T.fimg, &kp.fast.imgd)) != SG_OK)))) {
        g_create_error = ctx->last_error;
        free_all(ctx);
        delete ctx;
        return st;
    }
    kp.err = const_cast<int *>(errp);
    ctx->has_device = true;
    if (p.prec == SG_DF64 && !T.fast) {
        st = fail(nullptr, SG_EUNSUPPORTED,
                  "SG_DF64 needs the fast path (a potential with one- and two-mode monomials of a chain)");
        free_all(ctx);
        delete ctx;
        return st;
    }
    if (T.fast) {
        kp.fast.enabled = 1;
        kp.fast.df = p.prec == SG_DF64;
        kp.fast.nb1 = T.nb1;
        kp.fast.nq1 = T.nq1;
        kp.fast.npairs = (int)T.pair_modes.size() / 2;
        kp.fast.c0const = T.c0const;
        kp.fast.desccap = T.fdesccap;
        kp.fast.gcap = T.fgcap;
        kp.fast.nbocap = T.fnbocap;
        kp.fast.n_big = T.fn_big;
        kp.fast.work_cta = T.fwork_cta;
        kp.fast.work_warp = T.fwork_warp;
        kp.matcap = T.matcap;
        kp.cap = T.fast_cap;
        // M^B in the fast kernel's layout order, built on the device
        void *rp = nullptr;
        e = cudaMalloc(&rp, std::max<size_t>(1, (size_t)T.franks) * sizeof(int));
        if (e != cudaSuccess) {
            st = fail(nullptr, SG_ENOMEM, std::string("cudaMalloc (index maps): ") + cudaGetErrorString(e));
            free_all(ctx);
            delete ctx;
            return st;
        }
        ctx->allocations.push_back(rp);
        ctx->bytes_device += (int64_t)T.franks * (int64_t)sizeof(int);
        kp.fast.ranks = static_cast<const int *>(rp);
        // the inner-block tables of every term with a grid, in the context's precision
        void *vp = nullptr;
        const size_t nvt = std::max<size_t>(1, (size_t)T.fvt_off.back());
        // 16 bytes of padding: the term kernel prefetches 16-byte rounded ranges
        e = cudaMalloc(&vp, nvt * (ctx->fp32 ? sizeof(float) : sizeof(double)) + 16);
        if (e != cudaSuccess) {
            st = fail(nullptr, SG_ENOMEM, std::string("cudaMalloc (inner-block tables): ") + cudaGetErrorString(e));
            free_all(ctx);
            delete ctx;
            return st;
        }
        ctx->allocations.push_back(vp);
        ctx->bytes_device += (int64_t)nvt * (ctx->fp32 ? 4 : 8);
        if (ctx->fp32) kp.fast.mtabf = static_cast<const float *>(vp);
        else if (kp.fast.df) kp.fast.mtabx = static_cast<const float2 *>(vp);
        else kp.fast.mtabd = static_cast<const double *>(vp);
        e = launch_build_ranks(kp, static_cast<int *>(rp), 0);
        if (e == cudaSuccess) e = launch_build_mtab(kp, ctx->fp32, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) {
            ctx->smem_bytes = fast_smem_bytes(kp, ctx->fp32);
            e = configure_fast_kernels(kp, ctx->fp32);
        }
    } else {
        ctx->smem_bytes = apply_smem_bytes(kp, ctx->fp32);
        e = configure_kernels(ctx->smem_bytes, ctx->fp32);
    }
    if (e != cudaSuccess) {
        st = cuda_fail(nullptr, e, "cudaFuncSetAttribute");
        free_all(ctx);
        delete ctx;
        return st;
    }
    *out = ctx;
    return SG_OK;
}

sg_status sg_size(const sg_ctx *ctx, int64_t *n_cs, int64_t *n_terms, int64_t *n_s,
                  int64_t *n_grid, int64_t *bytes_device)
{
    if (!ctx) return SG_EINVAL;
    if (n_cs) *n_cs = ctx->host.n_cs;
    if (n_terms) *n_terms = ctx->host.n_terms;
    if (n_s) *n_s = ctx->host.n_s;
    if (n_grid) *n_grid = ctx->host.n_grid;
    // a context made by sg_plan holds nothing on the device: report what
    // sg_create would allocate for the same problem
    if (bytes_device) *bytes_device = ctx->has_device ? ctx->bytes_device : sg::planned_device_bytes(ctx);
    return SG_OK;
}

sg_status sg_apply_H(sg_ctx *ctx, const double *x, double *y, int nvec, void *stream)
{
    if (!ctx) return SG_EINVAL;
    if (!ctx->has_device) return fail(ctx, SG_EINVAL, "context was made by sg_plan (no device state)");
    if (!sg_on_ctx_device(ctx)) return fail(ctx, SG_EINVAL, "the current CUDA device is not the one the context was made on");
    if (!x || !y) return fail(ctx, SG_EINVAL, "x or y is NULL");
    if (nvec < 1) return fail(ctx, SG_EINVAL, "nvec must be >= 1");
    const size_t n = (size_t)ctx->host.n_cs * nvec;
    if ((x < y + n) && (y < x + n)) return fail(ctx, SG_EINVAL, "x and y overlap");
    sg_status st = ensure_workspace(ctx, nvec, (cudaStream_t)stream);
    if (st != SG_OK) return st;
    cudaError_t e = sg::launch_apply(ctx->kp, ctx->fp32, x, y, nvec, ctx->maxbits, nullptr,
                                     (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "apply launch");
    return SG_OK;
}

sg_status sg_apply_H_part(sg_ctx *ctx, const double *x, int nvec, int part, int nparts, int64_t *acc, void *stream)
{
    if (!ctx) return SG_EINVAL;
    if (!ctx->has_device) return fail(ctx, SG_EINVAL, "context was made by sg_plan (no device state)");
    if (!sg_on_ctx_device(ctx)) return fail(ctx, SG_EINVAL, "the current CUDA device is not the one the context was made on");
    if (!x || !acc) return fail(ctx, SG_EINVAL, "x or acc is NULL");
    if (nvec < 1) return fail(ctx, SG_EINVAL, "nvec must be >= 1");
    if (nparts < 1 || part < 0 || part >= nparts) return fail(ctx, SG_EINVAL, "need 0 <= part < nparts");
    sg_status st = ensure_workspace(ctx, nvec, (cudaStream_t)stream);  // the per-vector exponents
    if (st != SG_OK) return st;
    sg::KParams kp = ctx->kp;
    kp.acc = reinterpret_cast<unsigned long long *>(acc);
    kp.part = part;
    kp.nparts = nparts;
    cudaError_t e = sg::launch_maxabs(kp, x, nvec, ctx->maxbits, (cudaStream_t)stream);
    if (e == cudaSuccess) e = sg::launch_apply_terms(kp, ctx->fp32, x, ctx->maxbits, nvec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "partial apply launch");
    return SG_OK;
}

sg_status sg_apply_H_finish(sg_ctx *ctx, const double *x, int64_t *acc, double *y, int nvec, void *stream)
{
    if (!ctx) return SG_EINVAL;
    if (!ctx->has_device) return fail(ctx, SG_EINVAL, "context was made by sg_plan (no device state)");
    if (!sg_on_ctx_device(ctx)) return fail(ctx, SG_EINVAL, "the current CUDA device is not the one the context was made on");
    if (!x || !y || !acc) return fail(ctx, SG_EINVAL, "x, y or acc is NULL");
    if (nvec < 1) return fail(ctx, SG_EINVAL, "nvec must be >= 1");
    const size_t n = (size_t)ctx->host.n_cs * nvec;
    if ((x < y + n) && (y < x + n)) return fail(ctx, SG_EINVAL, "x and y overlap");
    sg_status st = ensure_workspace(ctx, nvec, (cudaStream_t)stream);
    if (st != SG_OK) return st;
    sg::KParams kp = ctx->kp;
    kp.acc = reinterpret_cast<unsigned long long *>(acc);
    cudaError_t e = sg::launch_maxabs(kp, x, nvec, ctx->maxbits, (cudaStream_t)stream);
    if (e == cudaSuccess) e = sg::launch_finalize(kp, ctx->fp32, x, y, nvec, ctx->maxbits, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "finish launch");
    return SG_OK;
}

sg_status sg_part_size(const sg_ctx *ctx, int part, int nparts, int64_t *n_terms, int64_t *cost)
{
    if (!ctx || nparts < 1 || part < 0 || part >= nparts) return SG_EINVAL;
    const sg::HostTables &T = ctx->host;
    int64_t c = 0, k = 0;
    for (int64_t p = part; p < T.n_terms; p += nparts) {
        c += T.pcost[(size_t)p];
        k++;
    }
    if (n_terms) *n_terms = k;
    if (cost) *cost = c;
    return SG_OK;
}

sg_status sg_apply_H_host(sg_ctx *ctx, const double *x_host, double *y_host, int nvec, void *stream)
{
    if (!ctx) return SG_EINVAL;
    if (!ctx->has_device) return fail(ctx, SG_EINVAL, "context was made by sg_plan (no device state)");
    if (!sg_on_ctx_device(ctx)) return fail(ctx, SG_EINVAL, "the current CUDA device is not the one the context was made on");
    if (!x_host || !y_host) return fail(ctx, SG_EINVAL, "x_host or y_host is NULL");
    if (nvec < 1) return fail(ctx, SG_EINVAL, "nvec must be >= 1");
    const int64_t n = ctx->host.n_cs * (int64_t)nvec;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (n > ctx->stage_elems) {
        if (ctx->stage_x) cudaFree(ctx->stage_x);
        if (ctx->stage_y) cudaFree(ctx->stage_y);
        ctx->stage_x = ctx->stage_y = nullptr;
        ctx->stage_elems = 0;
        if ((e = cudaMalloc(&ctx->stage_x, n * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&ctx->stage_y, n * sizeof(double))) != cudaSuccess)
            return fail(ctx, SG_ENOMEM, std::string("staging cudaMalloc: ") + cudaGetErrorString(e));
        ctx->stage_elems = n;
    }
    if ((e = cudaMemcpyAsync(ctx->stage_x, x_host, n * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "H2D copy");
    sg_status st = ensure_workspace(ctx, nvec, s);
    if (st != SG_OK) return st;
    if ((e = sg::launch_apply(ctx->kp, ctx->fp32, ctx->stage_x, ctx->stage_y, nvec, ctx->maxbits,
                              nullptr, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "apply launch");
    if ((e = cudaMemcpyAsync(y_host, ctx->stage_y, n * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "D2H copy");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    return SG_OK;
}

sg_status sg_term_levels(const sg_ctx *ctx, int64_t t0, int64_t nt, int *levels_host, int *coef_host)
{
    if (!ctx) return SG_EINVAL;
    const sg::HostTables &T = ctx->host;
    if (t0 < 0 || nt < 0 || t0 + nt > T.n_terms || (nt > 0 && !levels_host)) return SG_EINVAL;
    const int D = ctx->prob.D;
    for (int64_t t = 0; t < nt; t++) {
        for (int i = 0; i < D; i++) levels_host[t * D + i] = T.levels[(size_t)(t0 + t) * T.Dpad + i];
        if (coef_host) coef_host[t] = T.coefs[t0 + t];
    }
    return SG_OK;
}

sg_status sg_index_map(sg_ctx *ctx, int64_t t0, int64_t nt, int64_t *offsets_host,
                       int64_t *cs_index_dev, void *stream)
{
    if (!ctx) return SG_EINVAL;
    const sg::HostTables &T = ctx->host;
    if (t0 < 0 || nt < 0 || t0 + nt > T.n_terms || !offsets_host)
        return fail(ctx, SG_EINVAL, "bad term range or NULL offsets");
    const int D = ctx->prob.D, L = ctx->prob.L;
    offsets_host[0] = 0;
    for (int64_t t = 0; t < nt; t++) {
        int64_t nb = 1;
        for (int i = 0; i < D; i++) nb *= T.lvl[(size_t)i * (L + 1) + T.levels[(size_t)(t0 + t) * T.Dpad + i]].nb;
        offsets_host[t + 1] = offsets_host[t] + nb;
    }
    if (!cs_index_dev || nt == 0) return SG_OK;
    if (!ctx->has_device) return fail(ctx, SG_EINVAL, "context was made by sg_plan (no device state)");
    if (!sg_on_ctx_device(ctx)) return fail(ctx, SG_EINVAL, "the current CUDA device is not the one the context was made on");
    int64_t *offs_dev = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&offs_dev, sizeof(int64_t) * (nt + 1));
    if (e != cudaSuccess) return fail(ctx, SG_ENOMEM, "cudaMalloc offsets");
    e = cudaMemcpyAsync(offs_dev, offsets_host, sizeof(int64_t) * (nt + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = sg::launch_index_map(ctx->kp, t0, nt, offs_dev, cs_index_dev, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(offs_dev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "index map");
    return SG_OK;
}

sg_status sg_device_error(sg_ctx *ctx, int *code)
{
    if (!ctx || !code) return SG_EINVAL;
    if (!ctx->has_device) return fail(ctx, SG_EINVAL, "context was made by sg_plan (no device state)");
    if (!sg_on_ctx_device(ctx)) return fail(ctx, SG_EINVAL, "the current CUDA device is not the one the context was made on");
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, ctx->kp.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read error word");
    *code = v;
    if (v) {  // reported once: clear it for the next apply
        int z = 0;
        e = cudaMemcpy(ctx->kp.err, &z, sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "clear error word");
    }
    return SG_OK;
}

sg_status sg_compact_rank(const sg_ctx *ctx, const int *k, int64_t n, int64_t *rank)
{
    if (!ctx || n < 0 || (n > 0 && (!k || !rank))) return SG_EINVAL;
    const sg::HostTables &T = ctx->host;
    const int D = ctx->prob.D, L = ctx->prob.L;
    for (int64_t q = 0; q < n; q++) {
        const int *kq = k + q * D;
        int64_t r = 0;
        int s = 0;
        bool ok = true;
        for (int i = 0; i < D && ok; i++) {
            if (kq[i] < 0 || kq[i] >= T.kw) { ok = false; break; }
            const int lm = T.lmin_tab[(size_t)i * T.kw + kq[i]];
            if (lm > L || s + lm > L) { ok = false; break; }
            r += T.rank_tab[((size_t)i * (L + 1) + s) * T.kw + kq[i]];
            s += lm;
        }
        rank[q] = ok ? r : -1;
    }
    return SG_OK;
}

sg_status sg_mode_tables(const sg_ctx *ctx, int mode, int level, int *nb, int *nq,
                         double *B, double *BW, double *K, double *Q)
{
    if (!ctx || mode < 0 || mode >= ctx->prob.D || level < 0 || level > ctx->prob.L) return SG_EINVAL;
    const sg::HostTables &T = ctx->host;
    const sg::LevelInfo &li = T.lvl[(size_t)mode * (ctx->prob.L + 1) + level];
    if (nb) *nb = li.nb;
    if (nq) *nq = li.nq;
    const double *t = T.tabd.data();
    if (B) std::copy(t + li.offB, t + li.offB + li.nb * li.nq, B);
    if (BW) std::copy(t + li.offBW, t + li.offBW + li.nb * li.nq, BW);
    if (K) std::copy(t + li.offK, t + li.offK + li.nb * li.nb, K);
    if (Q) std::copy(t + li.offQ, t + li.offQ + li.nq, Q);
    return SG_OK;
}

const char *sg_last_error(const sg_ctx *ctx)
{
    return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

void sg_destroy(sg_ctx *ctx)
{
    if (!ctx) return;
    free_all(ctx);
    delete ctx;
}

}  // extern "C"
