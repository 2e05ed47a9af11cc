// Fast path of the Smolyak operator action: per-context set-up kernels (M^B,
// the inner-block tables) and the host entry points; the term kernels are in
// sg_fast.cuh, instantiated by sg_fast_f32.cu, sg_fast_f64.cu and the batch units.
#include "sg_fast.cuh"

namespace sg {

namespace {

// M^B in layout order: compact index of every basis function of every term,
// element e = o * NBI + i (outer site o, inner index i) of the term's list
// (built once per context; the same partial-rank arithmetic as the generic kernel).
__global__ void __launch_bounds__(kFT) k_build_ranks(const KParams P, int *__restrict__ ranks)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ FHdr H;
    int4 *buf = reinterpret_cast<int4 *>(smraw);
    if (threadIdx.x < 32) {
        load_record(P, blockIdx.x, buf, H);
        derive_layout<float>(P, 1, 1 << 30, H);
    }
    __syncthreads();
    const int m = H.m, R = H.R, NBI = H.NBI, Lp = P.L + 1;
    for (int e = threadIdx.x; e < H.NB; e += kFT) {
        const int o = e / NBI, i = e - o * NBI;
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

__host__ __device__ constexpr int ipow(int b, int e) { return e <= 0 ? 1 : b * ipow(b, e - 1); }

// Inner-block table of one term with coupled pairs (FP64 arithmetic, stored in
// T): for every slice and outer grid point g of the slice,
//   M_g[r][c] = sum_{inner grid points u} V(g, u) prod_j w_{u_j} b_{r_j}(u_j) b_{c_j}(u_j)
//             + sum_{inner j} H1_j[r_j][c_j] prod_{i != j} delta(r_i, c_i) + c0 delta(r, c),
// V = sum over the term's active pairs of G_p (the two-mode monomials on the
// pair's grid), H1_j = the single-mode matrix of inner position j with its
// induced parts, c0 = the term's constant.  Indices r, c run over the inner
// basis (first inner position slowest); M_g is stored as its upper triangle,
// row by row, in units of `UE` elements: [slice][unit][g][UE].
template <typename T, int NB1, int R>
__device__ void build_mtab_term(const KParams &P, const FHdr &H, T *__restrict__ mt)
{
    constexpr int NBI = ipow(NB1, R), NE = NBI * (NBI + 1) / 2;
    constexpr int U = vunit<T>(), UE = NBI == 1 ? 1 : U, NEU = (NE + UE - 1) / UE;
    const int m = H.m, ps = R + H.s, NGs = H.NGs, nitems = H.nslice * NGs;
    int NGI = 1;
    for (int j = 0; j < R; j++) NGI *= H.nq[j];
    const double *t1 = P.tabd, *ft = P.fast.tabd;
    for (int it = threadIdx.x; it < nitems; it += kFT) {
        const int sl = it / NGs, g = it - sl * NGs;
        int u[kMaxD];
        int rem = sl;
        for (int j = ps - 1; j >= R; j--) { u[j] = rem % H.nq[j]; rem /= H.nq[j]; }
        for (int j = ps; j < m; j++) u[j] = (g / H.gstride[j]) % H.nq[j];
        double M[NE];
#pragma unroll
        for (int e = 0; e < NE; e++) M[e] = 0.0;
        for (int gi = 0; gi < NGI; gi++) {
            int r2 = gi;
            for (int j = R - 1; j >= 0; j--) { u[j] = r2 % H.nq[j]; r2 /= H.nq[j]; }
            double V = 0.0;
            for (int q = 0; q < H.npair; q++) {
                const int a = H.pa[q], b = H.pb[q];
                V += ft[H.pgg[q] + u[a] * H.nq[b] + u[b]];
            }
            // w[r] = prod_j (B^T W)_j[r_j][u_j], b[c] = prod_j B_j[u_j][c_j]
            double wv[NBI], bv[NBI];
#pragma unroll
            for (int r = 0; r < NBI; r++) {
                double wp = V, bp = 1.0;
                int rr = r;
#pragma unroll
                for (int j = R - 1; j >= 0; j--) {
                    const int kj = rr % NB1;
                    rr /= NB1;
                    wp *= t1[H.gBW[j] + kj * H.nq[j] + u[j]];
                    bp *= t1[H.gB[j] + u[j] * NB1 + kj];
                }
                wv[r] = wp; bv[r] = bp;
            }
#pragma unroll
            for (int r = 0; r < NBI; r++)
#pragma unroll
                for (int c = r; c < NBI; c++) M[tri_index(r, c, NBI)] += wv[r] * bv[c];
        }
        // single-mode matrices of the inner positions (base + induced parts), and c0
#pragma unroll
        for (int j = 0; j < R; j++) {
            const int st = ipow(NB1, R - 1 - j);
#pragma unroll
            for (int r = 0; r < NBI; r++)
#pragma unroll
                for (int c = r; c < NBI; c++) {
                    const int rj = (r / st) % NB1, cj = (c / st) % NB1;
                    if (r - rj * st != c - cj * st) continue;  // other inner digits differ
                    double h = ft[H.gH1[j] + rj * NB1 + cj];
                    for (int q = 0; q < H.nind; q++)
                        if (H.ipos[q] == j) h += ft[H.ioffs[q] + rj * NB1 + cj];
                    M[tri_index(r, c, NBI)] += h;
                }
        }
#pragma unroll
        for (int r = 0; r < NBI; r++) M[tri_index(r, r, NBI)] += H.c0;
#pragma unroll
        for (int q = 0; q < NEU; q++)
#pragma unroll
            for (int e = 0; e < UE; e++) {
                const int idx = q * UE + e;
                mt[((size_t)(sl * NEU + q) * NGs + g) * UE + e] = idx < NE ? (T)M[idx] : T(0);
            }
    }
}

template <typename T, int NB1>
__global__ void __launch_bounds__(kFT) k_build_mtab(const KParams P, T *__restrict__ mt)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ FHdr H;
    const int p = blockIdx.x;
    const long long t0 = P.fast.mt_off[p];
    if (P.fast.mt_off[p + 1] == t0) return;
    if (threadIdx.x < 32) {
        load_record(P, p, reinterpret_cast<int4 *>(smraw), H);
        derive_layout<T>(P, 1, 1 << 30, H);
    }
    __syncthreads();
    if (H.bad) return;
    T *out = mt + t0;
    switch (H.R) {
        case 0: build_mtab_term<T, NB1, 0>(P, H, out); return;
        case 1: if constexpr (NB1 > 1) build_mtab_term<T, NB1, 1>(P, H, out); return;
        case 2: if constexpr (NB1 > 1) build_mtab_term<T, NB1, 2>(P, H, out); return;
        case 3: if constexpr (NB1 == 2) build_mtab_term<T, NB1, 3>(P, H, out); return;
        default: if (threadIdx.x == 0 && P.err) atomicCAS(P.err, 0, 113); return;
    }
}

}  // namespace

cudaError_t launch_build_mtab(const KParams &kp, bool fp32, cudaStream_t stream)
{
    if (kp.n_terms == 0) return cudaSuccess;
    const size_t smem = 16 * (size_t)kp.fast.desccap;
    const unsigned nb = (unsigned)kp.n_terms;
    float *mf = const_cast<float *>(kp.fast.mtabf);
    double *md = const_cast<double *>(kp.fast.mtabd);
    if (kp.fast.df) {
        df2 *mx = reinterpret_cast<df2 *>(const_cast<float2 *>(kp.fast.mtabx));
        switch (fast_inner_nb(kp.fast.nb1)) {
            case 2: k_build_mtab<df2, 2><<<nb, kFT, smem, stream>>>(kp, mx); break;
            case 3: k_build_mtab<df2, 3><<<nb, kFT, smem, stream>>>(kp, mx); break;
            default: k_build_mtab<df2, 1><<<nb, kFT, smem, stream>>>(kp, mx); break;
        }
        return cudaGetLastError();
    }
    // inner positions are level-1 modes of a uniform size nb1 (2 or 3); none otherwise
    switch (fast_inner_nb(kp.fast.nb1)) {
        case 2:
            if (fp32) k_build_mtab<float, 2><<<nb, kFT, smem, stream>>>(kp, mf);
            else k_build_mtab<double, 2><<<nb, kFT, smem, stream>>>(kp, md);
            break;
        case 3:
            if (fp32) k_build_mtab<float, 3><<<nb, kFT, smem, stream>>>(kp, mf);
            else k_build_mtab<double, 3><<<nb, kFT, smem, stream>>>(kp, md);
            break;
        default:
            if (fp32) k_build_mtab<float, 1><<<nb, kFT, smem, stream>>>(kp, mf);
            else k_build_mtab<double, 1><<<nb, kFT, smem, stream>>>(kp, md);
            break;
    }
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
    return fp32 ? fast_launch_f32(kp, a) : kp.fast.df ? fast_launch_df(kp, a) : fast_launch_f64(kp, a);
}

cudaError_t launch_apply_fast(const KParams &kp, bool fp32, const double *x, int nvec,
                              const long long *maxbits, cudaStream_t stream)
{
    if (kp.n_terms == 0) return cudaSuccess;
    FastLaunch a{x, nvec, maxbits, stream, false};
    return fp32 ? fast_launch_f32(kp, a) : kp.fast.df ? fast_launch_df(kp, a) : fast_launch_f64(kp, a);
}

}  // namespace sg
