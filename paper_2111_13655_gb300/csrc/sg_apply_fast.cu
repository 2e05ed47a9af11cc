// Fast path of the Smolyak operator action: per-context set-up kernels and
// the host entry points; the term kernels are in sg_fast.cuh, instantiated by
// sg_fast_f32.cu and sg_fast_f64.cu.
#include "sg_fast.cuh"

namespace sg {

namespace {

// M^B in layout order: compact index of every basis function of every term
// (built once per context; the same partial-rank arithmetic as the generic kernel).
__global__ void __launch_bounds__(kFT) k_build_ranks(const KParams P, int *__restrict__ ranks)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ FHdr H;
    int4 *buf = reinterpret_cast<int4 *>(smraw);
    if (threadIdx.x < 32) {
        load_record(P, blockIdx.x, buf, H);
        derive_layout(P, 1, 1 << 30, H);
    }
    __syncthreads();
    const int m = H.m, R = H.R, NBo = H.NBo, Lp = P.L + 1;
    for (int e = threadIdx.x; e < H.NB; e += kFT) {
        const int i = e / NBo, o = e - i * NBo;
        int r = 0, s = 0;
        for (int a = 0; a < m; a++) {
            const int j = H.bymode[a];
            const int src = j < R ? i : o;
            const int q = fdiv(src, H.ostride[j], H.smag[j]);
            const int kj = q - fdiv(q, H.nb[j], H.bmag[j]) * H.nb[j];
            const int md = H.mode[j];
            r += P.rank_tab[(md * Lp + s) * P.kw + kj];
            s += P.lmin_tab[md * P.kw + kj];
        }
        ranks[H.rank_off + e] = r;
    }
}


// The coupling potential V = sum_p G_p(u_a, u_b) on each term's collapsed grid,
// once per context, in the order the term kernel's register phase reads it:
// [slice][inner grid point gi][outer grid point g] (g fastest).  Digits: inner
// positions from gi (first position slowest), sliced positions from the slice
// (last fastest), the other outer positions from g.  G tables from the image.
template <typename T>
__global__ void __launch_bounds__(kFT) k_build_vtab(const KParams P, T *__restrict__ vt)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ FHdr H;
    const int p = blockIdx.x;
    const long long v0 = P.fast.vt_off[p], nv = P.fast.vt_off[p + 1] - v0;
    if (nv == 0) return;
    if (threadIdx.x < 32) {
        load_record(P, p, reinterpret_cast<int4 *>(smraw), H);
        derive_layout(P, 1, 1 << 30, H);
    }
    __syncthreads();
    const int m = H.m, R = H.R, s0 = R + H.s, NGs = H.NGs;
    long long NGI = 1;
    for (int j = 0; j < R; j++) NGI *= H.nq[j];
    const T *G = FTab<T>::img(P) + P.fast.img_off[p] + H.matsz;
    for (long long e = threadIdx.x; e < nv; e += kFT) {
        const long long per_slice = NGI * NGs;
        const int sl = (int)(e / per_slice);
        const long long r1 = e - (long long)sl * per_slice;
        const int gi = (int)(r1 / NGs), g = (int)(r1 - (long long)gi * NGs);
        int u[kMaxD];
        int rem = gi;
        for (int j = R - 1; j >= 0; j--) { u[j] = rem % H.nq[j]; rem /= H.nq[j]; }
        rem = sl;
        for (int j = s0 - 1; j >= R; j--) { u[j] = rem % H.nq[j]; rem /= H.nq[j]; }
        for (int j = s0; j < m; j++) u[j] = (g / H.gstride[j]) % H.nq[j];
        T v = T(0);
        for (int q = 0; q < H.npair; q++) {
            const int a = H.pa[q], b = H.pb[q];
            v += G[H.pg[q] + u[a] * H.nq[b] + u[b]];
        }
        vt[v0 + e] = v;
    }
}

}  // namespace

cudaError_t launch_build_vtab(const KParams &kp, bool fp32, cudaStream_t stream)
{
    if (kp.n_terms == 0) return cudaSuccess;
    const size_t smem = 16 * (size_t)kp.fast.desccap;
    if (fp32)
        k_build_vtab<float><<<(unsigned)kp.n_terms, kFT, smem, stream>>>(kp, const_cast<float *>(kp.fast.vtabf));
    else
        k_build_vtab<double><<<(unsigned)kp.n_terms, kFT, smem, stream>>>(kp, const_cast<double *>(kp.fast.vtabd));
    return cudaGetLastError();
}

size_t fast_smem_bytes(const KParams &kp, bool fp32)
{
    const size_t rb = fp32 ? 4 : 8;
    return std::max(part_bytes(kp, rb, kp.fast.work_cta), (size_t)(kFT / 32) * part_bytes(kp, rb, kp.fast.work_warp));
}

size_t fast_part_bytes(const KParams &kp, bool fp32, bool warp_form)
{
    return part_bytes(kp, fp32 ? 4 : 8, warp_form ? kp.fast.work_warp : kp.fast.work_cta);
}

static FastBatchLaunch batch_args(const FastBatchGroup &g, const double *x, unsigned long long *acc,
                                  const long long *maxbits, const long long *cs_prefix, int nvec,
                                  cudaStream_t stream, bool configure)
{
    FastBatchLaunch a{};
    a.kps = g.kps;
    for (int f = 0; f < 2; f++) { a.items[f] = g.items[f]; a.count[f] = g.count[f]; a.part[f] = g.part[f]; }
    a.x = x; a.acc = acc; a.maxbits = maxbits; a.cs_prefix = cs_prefix; a.nvec = nvec;
    a.stream = stream; a.configure = configure;
    return a;
}

cudaError_t configure_fast_batch(const KParams &kp_any, bool fp32, const FastBatchGroup &g)
{
    const FastBatchLaunch a = batch_args(g, nullptr, nullptr, nullptr, nullptr, 0, 0, true);
    return fp32 ? fast_batch_launch_f32(kp_any, a) : fast_batch_launch_f64(kp_any, a);
}

cudaError_t launch_fast_batch(const KParams &kp_any, bool fp32, const FastBatchGroup &g, const double *x,
                              unsigned long long *acc, const long long *maxbits, const long long *cs_prefix,
                              int nvec, cudaStream_t stream)
{
    const FastBatchLaunch a = batch_args(g, x, acc, maxbits, cs_prefix, nvec, stream, false);
    return fp32 ? fast_batch_launch_f32(kp_any, a) : fast_batch_launch_f64(kp_any, a);
}

cudaError_t launch_build_ranks(const KParams &kp, int *ranks, cudaStream_t stream)
{
    if (kp.n_terms == 0) return cudaSuccess;
    const size_t smem = 16 * (size_t)kp.fast.desccap;
    k_build_ranks<<<(unsigned)kp.n_terms, kFT, smem, stream>>>(kp, ranks);
    return cudaGetLastError();
}

cudaError_t configure_fast_kernels(const KParams &kp, bool fp32)
{
    FastLaunch a{nullptr, 0, nullptr, 0, true};
    return fp32 ? fast_launch_f32(kp, a) : fast_launch_f64(kp, a);
}

cudaError_t launch_apply_fast(const KParams &kp, bool fp32, const double *x, int nvec,
                              const long long *maxbits, cudaStream_t stream)
{
    if (kp.n_terms == 0) return cudaSuccess;
    FastLaunch a{x, nvec, maxbits, stream, false};
    return fp32 ? fast_launch_f32(kp, a) : fast_launch_f64(kp, a);
}

}  // namespace sg
