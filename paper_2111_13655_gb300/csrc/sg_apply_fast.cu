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


}  // namespace

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
