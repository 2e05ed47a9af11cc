// Device code of the fast path of the Smolyak operator action (sm_103a):
// potentials whose monomials touch at most two modes (the Henon-Heiles family
// of Sec. 4, Eq. (18)).  Included by the units that instantiate it:
// sg_fast_f32.cu / sg_fast_f64.cu (one problem per launch) and
// sg_fast_batch_f32.cu / sg_fast_batch_f64.cu (many problems per launch).
//
// One thread block (or, for small terms, one warp) per Smolyak term, terms
// ordered most-expensive first.  The term operator (Alg. 1 of arXiv
// 2111.13655 with the grid operator split as described in build_fast_tables) is
//     y_l = c0 x_l + sum_j H1_j x_l + (x B^T W) diag(V_l) (x B) x_l,
// V_l(u) = sum over the term's active coupled pairs of G_p(u_a, u_b).
// The basis->grid (Eq. (15)) and grid->basis (Eq. (14)) transfers run mode by
// mode.
//
// Layout of a term tensor: [i][v][o] -- i runs over the "inner" slots (up to
// RMAX slots of level 1, the slowest positions), v over a chunk of vectors,
// o over the "outer" slots in mode order (last fastest).  Outer slots are
// contracted breadth-first in shared memory with the 1D matrix in registers,
// one (fibre, vector) per thread; the inner slots, the potential and their
// back-transfer run in registers, one outer grid point per thread, the
// potential evaluated once for all vectors of the chunk.  Vectors are batched
// inside every phase, so block-wide barriers are shared by the whole chunk.
// The compress-add of D_l * y_l into the compact result is the exact
// fixed-point sum of sg_fixed.cuh.
#pragma once

#include <algorithm>
#include <cstdint>

#include "sg_fixed.cuh"
#include "sg_internal.h"

namespace sg {

// One problem per launch (sg_fast_f32.cu, sg_fast_f64.cu).
struct FastLaunch {
    const double *x;
    int nvec;
    const long long *maxbits;
    cudaStream_t stream;
    bool configure;  // set the kernels' shared-memory limits instead of launching
};
cudaError_t fast_launch_f32(const KParams &kp, const FastLaunch &a);
cudaError_t fast_launch_f64(const KParams &kp, const FastLaunch &a);

// Many problems of one kernel variant per launch (sg_fast_batch_f32.cu,
// sg_fast_batch_f64.cu).  [0]: block-form items, [1]: warp-form items.
struct FastBatchLaunch {
    const KParams *kps;           // device, one per problem
    const int2 *items[2];         // device: (problem, processing position), cost order
    int count[2];
    int part[2];                  // shared-memory partition per term group (bytes)
    const double *x;              // problems' vectors, problem after problem
    unsigned long long *acc;      // their accumulators, same order
    const long long *maxbits;     // [problem][nvec]
    const long long *cs_prefix;   // [n + 1] sums of N_cs
    int nvec;
    cudaStream_t stream;
    bool configure;
};
cudaError_t fast_batch_launch_f32(const KParams &kp_any, const FastBatchLaunch &a);
cudaError_t fast_batch_launch_f64(const KParams &kp_any, const FastBatchLaunch &a);

namespace {

constexpr int kFT = 128;   // threads per term block
constexpr int kMaxVB = 8;  // vectors per chunk

struct FHdr {
    int m, R, NB, NBo, grid, bad, coef;
    int s, vb, NBO, NBrest, NBIn, nslice, NGs;
    int matsz;                                           // elements of the B, B^T W, H1 block
    unsigned nbomag, nbOmag;                             // reciprocals of NBo and NBO
    int npair, nind, gsize;
    double c0;
    long long rank_off;
    int mode[kMaxD], nb[kMaxD], nq[kMaxD];               // by layout position
    int ostride[kMaxD];                                  // stride of a position inside its block (i or o)
    unsigned smag[kMaxD], bmag[kMaxD];                   // reciprocals of ostride and nb
    int oB[kMaxD], oBW[kMaxD], oH[kMaxD];                // shared-memory offsets of B, B^T W, H1
    int gstride[kMaxD];                                  // outer grid strides inside a slice
    unsigned gmag[kMaxD], qmag[kMaxD];                   // reciprocals of gstride and nq
    int bymode[kMaxD];                                   // positions sorted by mode
    int gB[kMaxD], gBW[kMaxD], gH1[kMaxD];               // global offsets of B, B^T W, H1 base
    int uS[kMaxD];                                       // slice indices of the sliced positions
    int pg[kMaxPairs], pgg[kMaxPairs], ioffs[kMaxPairs]; // G offsets (shared, global), induced offsets
    unsigned char pa[kMaxPairs], pb[kMaxPairs], ipos[kMaxPairs];
};
constexpr int kHdrBytes = 4096;  // per-group header budget the host plans with
static_assert(sizeof(FHdr) <= kHdrBytes, "term header too large");

template <int GS>
__device__ __forceinline__ void gsync()
{
    if (GS == 32) __syncwarp(); else __syncthreads();
}

// floor(x / d) for x * d < 2^32, via a 32-bit reciprocal (mag = ceil(2^32 / d), d > 1)
__device__ __forceinline__ unsigned rmag(unsigned d) { return d <= 1 ? 0u : 0xFFFFFFFFu / d + 1u; }
__device__ __forceinline__ int fdiv(int x, int d, unsigned mag)
{
    return d == 1 ? x : (int)__umulhi((unsigned)x, mag);
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of 16)
static __device__ __forceinline__ void l2_prefetch_bulk(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// at most this much of a term's stored potential is prefetched at entry (the
// largest tables are 236 KB in FP32; ~600 resident blocks share the L2)
constexpr int kVtPrefetchBytes = 32768;

template <typename T> struct FTab;
template <> struct FTab<double> {
    static __device__ const double *vt(const KParams &P) { return P.fast.vtabd; }
    static __device__ const double *img(const KParams &P) { return P.fast.imgd; }
    static __device__ const double *f(const KParams &P) { return P.fast.tabd; }
    static __device__ const double *t(const KParams &P) { return P.tabd; }
};
template <> struct FTab<float> {
    static __device__ const float *vt(const KParams &P) { return P.fast.vtabf; }
    static __device__ const float *img(const KParams &P) { return P.fast.imgf; }
    static __device__ const float *f(const KParams &P) { return P.fast.tabf; }
    static __device__ const float *t(const KParams &P) { return P.tabf; }
};

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-term set-up from the term's record (built on the host): warp 0 copies
// the record to shared memory and parses it, lane 0 derives the layout.
__device__ void load_record(const KParams &P, int p, int4 *buf, FHdr &H)
{
    const int lane = threadIdx.x & 31;
    const unsigned lo = P.fast.desc_off[p], hi = P.fast.desc_off[p + 1];
    for (unsigned u = lo + lane; u < hi; u += 32) buf[u - lo] = P.fast.desc[u];
    __syncwarp();
    const FDescHdr *hd = reinterpret_cast<const FDescHdr *>(buf);
    const int m = hd->m, np = hd->npair, ni = hd->nind;
    const FDescPos *ps = reinterpret_cast<const FDescPos *>(buf + 3);
    const FDescPair *pr = reinterpret_cast<const FDescPair *>(buf + 3 + m);
    const FDescInd *in = reinterpret_cast<const FDescInd *>(buf + 3 + m + np);
    for (int j = lane; j < m; j += 32) {
        H.mode[j] = ps[j].mode; H.nb[j] = ps[j].nb; H.nq[j] = ps[j].nq;
        H.gB[j] = ps[j].offB; H.gBW[j] = ps[j].offBW; H.gH1[j] = ps[j].offH1;
    }
    for (int q = lane; q < np; q += 32) { H.pa[q] = pr[q].pa; H.pb[q] = pr[q].pb; H.pg[q] = pr[q].gsm; H.pgg[q] = pr[q].goff; }
    for (int q = lane; q < ni; q += 32) { H.ipos[q] = in[q].pos; H.ioffs[q] = in[q].ioff; }
    if (lane == 0) {
        H.m = m; H.R = hd->R; H.NB = hd->NB; H.coef = hd->coef; H.s = hd->s;
        H.npair = np; H.nind = ni; H.gsize = hd->gsize; H.c0 = hd->c0; H.rank_off = hd->rank_off;
        H.grid = np > 0;
    }
    __syncwarp();
}

// Layout quantities of the term, shared memory only: lane j handles position j.
__device__ void derive_layout(const KParams &P, int nvec, int work, FHdr &H)
{
    const int lane = threadIdx.x & 31;
    const int m = H.m, R = H.R, sv = H.s;
    if (lane < m) {
        const int j = lane, nb = H.nb[j], nq = H.nq[j];
        int off = 0, st = 1, gs = 1, rank = 0;
        for (int i = 0; i < j; i++) off += 2 * H.nq[i] * H.nb[i] + H.nb[i] * H.nb[i];
        const int end = j < R ? R : m;
        for (int i = j + 1; i < end; i++) st *= H.nb[i];
        for (int i = j + 1; i < m; i++) gs *= H.nq[i];
        for (int i = 0; i < m; i++) rank += H.mode[i] < H.mode[j];
        H.oB[j] = off; H.oBW[j] = off + nq * nb; H.oH[j] = off + 2 * nq * nb;
        H.bmag[j] = rmag(nb); H.qmag[j] = rmag(nq);
        H.ostride[j] = st; H.smag[j] = rmag(st);
        H.gstride[j] = gs; H.gmag[j] = rmag(gs);
        H.bymode[rank] = j;
    }
    __syncwarp();
    if (lane != 0) return;
    H.bad = 0;
    int mat = 0, NBIn = 1;
    int64_t stage = 1;
    H.NBO = 1; H.nslice = 1; H.NBrest = 1; H.NGs = 1;
    for (int j = 0; j < m; j++) {
        mat += 2 * H.nq[j] * H.nb[j] + H.nb[j] * H.nb[j];
        if (j < R) NBIn *= H.nb[j];
        else if (j < R + sv) { H.NBO *= H.nb[j]; H.nslice *= H.nq[j]; }
        else { H.NBrest *= H.nb[j]; H.NGs *= H.nq[j]; stage *= H.nq[j]; }
    }
    if (mat > P.matcap || H.gsize > P.fast.gcap || H.NBO > P.fast.nbocap) { H.bad = 1; return; }
    H.matsz = mat;
    H.NBIn = NBIn; H.NBo = H.NB / NBIn;
    H.nbomag = rmag((unsigned)H.NBo);
    H.nbOmag = rmag((unsigned)H.NBO);
    stage *= NBIn;
    const int64_t per_vec = 2 * (int64_t)H.NB + (H.grid ? 2 * stage : 0);
    if (per_vec > work) { H.bad = 2; return; }
    int vb = nvec < kMaxVB ? nvec : kMaxVB;
    while (vb > 1 && per_vec * vb > work) vb--;
    H.vb = vb;
}

// Fibres f = tid, tid + GS, ... of an A x C grid as (a, c) = (f / C, f % C),
// stepped without a division: one division per call for the start and the
// step GS = as * C + cs, then one carry per step.
struct FibreWalk {
    int a, c, as, cs;
    __device__ __forceinline__ void step(int C)
    {
        a += as;
        c += cs;
        if (c >= C) { c -= C; a++; }
    }
};
template <int GS>
__device__ __forceinline__ FibreWalk fibre_walk(int C, int tid)
{
    FibreWalk w;
    w.a = tid / C;
    w.c = tid - w.a * C;
    w.as = GS / C;
    w.cs = GS - w.as * C;
    return w;
}

// out[a][r][c] = sum_k M[r][k] in[a][k][c], matrix in registers, one fibre (a, c) at a time per thread
template <typename T, int N, int RR, int GS>
__device__ __forceinline__ void fcontract_t(const T *__restrict__ in, T *__restrict__ out, int A, int C,
                                            const T *__restrict__ M, int tid)
{
    T mr[RR * N];
#pragma unroll
    for (int i = 0; i < RR * N; i++) mr[i] = M[i];
    for (FibreWalk w = fibre_walk<GS>(C, tid); w.a < A; w.step(C)) {
        const T *ip = in + w.a * N * C + w.c;
        T *op = out + w.a * RR * C + w.c;
        T xv[N];
#pragma unroll
        for (int k = 0; k < N; k++) xv[k] = ip[k * C];
#pragma unroll
        for (int r = 0; r < RR; r++) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < N; k++) acc = fma_t(mr[r * N + k], xv[k], acc);
            op[r * C] = acc;
        }
    }
}

template <typename T, int GS>
__device__ void fcontract_rt(const T *__restrict__ in, T *__restrict__ out, int A, int n, int r, int C,
                             const T *__restrict__ M, int tid)
{
    for (FibreWalk w = fibre_walk<GS>(C, tid); w.a < A; w.step(C)) {
        const T *ip = in + (w.a * n) * C + w.c;
        for (int rr = 0; rr < r; rr++) {
            const T *mp = M + rr * n;
            T acc = T(0);
            for (int k = 0; k < n; k++) acc += mp[k] * ip[k * C];
            out[(w.a * r + rr) * C + w.c] = acc;
        }
    }
}

template <typename T, int GS>
__device__ void fcontract(const T *in, T *out, int A, int n, int r, int C, const T *M, int tid)
{
#define SG_FC(NN, RRR) case (NN) * 64 + (RRR): fcontract_t<T, NN, RRR, GS>(in, out, A, C, M, tid); return;
    switch (n * 64 + r) {
        SG_FC(2, 2) SG_FC(2, 3) SG_FC(3, 2) SG_FC(3, 3) SG_FC(3, 4) SG_FC(4, 3) SG_FC(4, 4) SG_FC(4, 5)
        SG_FC(5, 4) SG_FC(5, 5) SG_FC(5, 6) SG_FC(6, 5) SG_FC(6, 6) SG_FC(6, 7) SG_FC(7, 6)
        default: fcontract_rt<T, GS>(in, out, A, n, r, C, M, tid); return;
    }
#undef SG_FC
}

__host__ __device__ constexpr int cpow(int b, int e) { return e <= 0 ? 1 : b * cpow(b, e - 1); }

// one register stage: out[p][u][q] = sum_k M[u][k] in[p][k][q]
template <typename T, int SZ, int PP, int N, int RR, int Q, int MS>
__device__ __forceinline__ void rstage(const T (&in)[SZ], T (&out)[SZ], const T (&M)[MS])
{
#pragma unroll
    for (int p = 0; p < PP; p++)
#pragma unroll
        for (int u = 0; u < RR; u++)
#pragma unroll
            for (int q = 0; q < Q; q++) {
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < N; k++) acc = fma_t(M[u * N + k], in[(p * N + k) * Q + q], acc);
                out[(p * RR + u) * Q + q] = acc;
            }
}

// Register phase: for every outer grid point g of the slice and every vector
// of the chunk, the inner slots basis -> grid, times the potential, grid ->
// basis, in place in Z[i][v][g].
template <typename T, int R, int NB1, int NQ1, bool UNI, int GS>
__device__ void reg_phase(const FHdr &H, const T *mats, const T *__restrict__ vt, T *Z, const int vb, const int tid)
{
    constexpr int NBI = cpow(NB1, R), NGI = cpow(NQ1, R), SZ = NGI;
    constexpr int RA = R > 0 ? R : 1;
    constexpr int NM = UNI ? 1 : RA;
    T Bm[NM][NQ1 * NB1], BWm[NM][NB1 * NQ1];
#pragma unroll
    for (int b = 0; b < NM; b++)
#pragma unroll
        for (int e = 0; e < NQ1 * NB1; e++) {
            Bm[b][e] = R > 0 ? mats[H.oB[b] + e] : T(0);
            BWm[b][e] = R > 0 ? mats[H.oBW[b] + e] : T(0);
        }
    const int NGs = H.NGs;
    for (int g = tid; g < NGs; g += GS) {
        // the coupling potential at the NGI inner points of outer grid point g
        // (evaluated once per context; vt: this slice's table, [gi][g])
        T V[SZ];
#pragma unroll
        for (int gi = 0; gi < NGI; gi++) V[gi] = __ldg(vt + (size_t)gi * NGs + g);
        for (int v = 0; v < vb; v++) {
            T va[SZ], vw[SZ];
#pragma unroll
            for (int i = 0; i < NBI; i++) va[i] = Z[(i * vb + v) * NGs + g];
            if constexpr (R == 0) {
                va[0] *= V[0];
            } else if constexpr (R == 1) {
                rstage<T, SZ, 1, NB1, NQ1, 1>(va, vw, Bm[0]);
#pragma unroll
                for (int gi = 0; gi < NGI; gi++) vw[gi] *= V[gi];
                rstage<T, SZ, 1, NQ1, NB1, 1>(vw, va, BWm[0]);
            } else if constexpr (R == 2) {
                rstage<T, SZ, 1, NB1, NQ1, NB1>(va, vw, Bm[0]);
                rstage<T, SZ, NQ1, NB1, NQ1, 1>(vw, va, Bm[UNI ? 0 : 1]);
#pragma unroll
                for (int gi = 0; gi < NGI; gi++) va[gi] *= V[gi];
                rstage<T, SZ, NQ1, NQ1, NB1, 1>(va, vw, BWm[UNI ? 0 : 1]);
                rstage<T, SZ, 1, NQ1, NB1, NB1>(vw, va, BWm[0]);
            } else if constexpr (R == 3) {
                rstage<T, SZ, 1, NB1, NQ1, NB1 * NB1>(va, vw, Bm[0]);
                rstage<T, SZ, NQ1, NB1, NQ1, NB1>(vw, va, Bm[UNI ? 0 : 1]);
                rstage<T, SZ, NQ1 * NQ1, NB1, NQ1, 1>(va, vw, Bm[UNI ? 0 : 2]);
#pragma unroll
                for (int gi = 0; gi < NGI; gi++) vw[gi] *= V[gi];
                rstage<T, SZ, NQ1 * NQ1, NQ1, NB1, 1>(vw, va, BWm[UNI ? 0 : 2]);
                rstage<T, SZ, NQ1, NQ1, NB1, NB1>(va, vw, BWm[UNI ? 0 : 1]);
                rstage<T, SZ, 1, NQ1, NB1, NB1 * NB1>(vw, va, BWm[0]);
            }
#pragma unroll
            for (int i = 0; i < NBI; i++) Z[(i * vb + v) * NGs + g] = va[i];
        }
    }
}

// Shared-memory partition of one term group: matrices, G tables, slice
// weights (head), then the work area for X, Y and the two grid buffers.
__host__ __device__ inline size_t part_head_bytes(const KParams &P, size_t rb)
{
    return (((size_t)P.matcap + P.fast.gcap + 2 * (size_t)P.fast.nbocap) * rb + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t part_bytes(const KParams &P, size_t rb, int work)
{
    return (part_head_bytes(P, rb) + (size_t)work * rb + 15) & ~(size_t)15;
}


// Per-chunk element loops, compiled for VB vectors (no predicated lanes for
// small chunks).  Tensor layout [i][v][o] (i: inner slots, v: vector, o: outer).
//   chunk_in:  gather X through M^B (x: the chunk's first vector), a barrier,
//              then the basis part Y = c0 X + sum_j H1_j x_j X, a barrier.
//   chunk_out: the exact compress-add of D_l * Y into the accumulators of the
//              chunk's vectors (acc: the first vector's), a barrier.
// One row of a single-mode matrix applied along a position: acc[v] +=
// sum_kp H[kp] x[kp * st + v * NBo], NK and VB at compile time.
template <typename T, int VB, int NK>
__device__ __forceinline__ void basis_row(T (&acc)[VB], const T *xp, const T *Hr, int st, int NBo)
{
    T hv[NK];
#pragma unroll
    for (int kp = 0; kp < NK; kp++) hv[kp] = Hr[kp];
#pragma unroll
    for (int kp = 0; kp < NK; kp++)
#pragma unroll
        for (int v = 0; v < VB; v++) acc[v] = fma_t(hv[kp], xp[kp * st + v * NBo], acc[v]);
}

template <typename T, int VB, int GS>
__device__ __forceinline__ void chunk_in(FHdr &H, const KParams &P, const double *__restrict__ x,
                                         const int *__restrict__ rk, const T *mats, T *X, T *Y, int tid)
{
    const int NB = H.NB, NBo = H.NBo, m = H.m, R = H.R;
    {
        int rn = tid < NB ? __ldg(rk + tid) : 0;
        for (int e = tid; e < NB; e += GS) {
            const int r = rn;
            if (e + GS < NB) rn = __ldg(rk + e + GS);
            const int i = fdiv(e, NBo, H.nbomag), o = e - i * NBo;
            T xv[VB];
#pragma unroll
            for (int v = 0; v < VB; v++) xv[v] = (T)__ldg(x + (size_t)v * P.n_cs + r);
#pragma unroll
            for (int v = 0; v < VB; v++) X[(i * VB + v) * NBo + o] = xv[v];
        }
    }
    gsync<GS>();
    for (int e = tid; e < NB; e += GS) {
        const int i = fdiv(e, NBo, H.nbomag), o = e - i * NBo;
        const int base0 = i * VB * NBo + o;
        T acc[VB];
#pragma unroll
        for (int v = 0; v < VB; v++) acc[v] = (T)H.c0 * X[base0 + v * NBo];
        for (int j = 0; j < m; j++) {
            const int src = j < R ? i : o;
            const int q = fdiv(src, H.ostride[j], H.smag[j]);
            const int nbj = H.nb[j], kj = q - fdiv(q, nbj, H.bmag[j]) * nbj;
            const int st = j < R ? H.ostride[j] * VB * NBo : H.ostride[j];
            const T *xp = X + base0 - kj * st;
            const T *Hr = mats + H.oH[j] + kj * nbj;
            switch (nbj) {
                case 2: basis_row<T, VB, 2>(acc, xp, Hr, st, NBo); break;
                case 3: basis_row<T, VB, 3>(acc, xp, Hr, st, NBo); break;
                case 4: basis_row<T, VB, 4>(acc, xp, Hr, st, NBo); break;
                case 5: basis_row<T, VB, 5>(acc, xp, Hr, st, NBo); break;
                default:
                    for (int kp = 0; kp < nbj; kp++) {
                        const T hv = Hr[kp];
#pragma unroll
                        for (int v = 0; v < VB; v++) acc[v] = fma_t(hv, xp[kp * st + v * NBo], acc[v]);
                    }
            }
        }
#pragma unroll
        for (int v = 0; v < VB; v++) Y[base0 + v * NBo] = acc[v];
    }
    gsync<GS>();
}

template <typename T, int VB, int GS>
__device__ __forceinline__ void chunk_out(FHdr &H, const KParams &P, const int *__restrict__ rk,
                                          const long long *__restrict__ maxbits, unsigned long long *acc,
                                          const T *Y, int tid)
{
    const int NB = H.NB, NBo = H.NBo;
    int Ev[VB];
#pragma unroll
    for (int v = 0; v < VB; v++) Ev[v] = fx::Acc<T>::unit(maxbits[v]);
    for (int e = tid; e < NB; e += GS) {
        const int i = fdiv(e, NBo, H.nbomag), o = e - i * NBo;
        unsigned long long *a = acc + (size_t)__ldg(rk + e) * fx::Acc<T>::words;
#pragma unroll
        for (int v = 0; v < VB; v++)
            fx::Acc<T>::add_unit(a + (size_t)v * P.n_cs * fx::Acc<T>::words, Y[(i * VB + v) * NBo + o], H.coef,
                                 Ev[v], P.err);
    }
    gsync<GS>();
}

// One Smolyak term (processing position p of problem P) by a group of GS
// threads: GS = 128 (a whole block) or GS = 32 (one warp; no block-wide
// barriers).  `base` is the group's shared-memory partition (part_bytes of P
// with `work_cap` work elements), `accp` the problem's fixed-point
// accumulators, `x` and `maxbits` its input vectors and their exponents.
template <typename T, int NB1, int NQ1, int RMAX, bool UNI, int GS>
__device__ __forceinline__ void fast_term(const KParams &P, const double *__restrict__ x,
                                          unsigned long long *accp, const long long *__restrict__ maxbits,
                                          int nvec, int p, int work_cap, unsigned char *base, FHdr &H,
                                          const int tid)
{
    const size_t rb = sizeof(T);
    T *mats = reinterpret_cast<T *>(base);
    T *WoF = mats + P.matcap + P.fast.gcap;
    T *WoB = WoF + P.fast.nbocap;
    T *work = reinterpret_cast<T *>(base + part_head_bytes(P, rb));

    // the start of the term's stored potential is fetched into L2 now: it is
    // first read after the gather, the basis part and the outer contractions
    if (tid == 0) {
        const long long v0 = P.fast.vt_off[p], v1 = P.fast.vt_off[p + 1];
        if (v1 > v0) {
            // 16-byte aligned and rounded; the table buffer is padded by 16 bytes
            const size_t b0 = ((size_t)v0 * rb) & ~(size_t)15;
            const size_t e1 = ((size_t)v1 * rb + 15) & ~(size_t)15;
            const size_t b1 = e1 - b0 > (size_t)kVtPrefetchBytes ? b0 + (size_t)kVtPrefetchBytes : e1;
            l2_prefetch_bulk(reinterpret_cast<const unsigned char *>(FTab<T>::vt(P)) + b0, (unsigned)(b1 - b0));
        }
    }
    // the term's image (B, B^T W, H1 per position, then its G tables) is copied
    // as it lies while warp 0 decodes the record
    {
        const long long i0 = P.fast.img_off[p];
        const int isz = (int)(P.fast.img_off[p + 1] - i0);
        const T *img = FTab<T>::img(P) + i0;
        if (isz <= P.matcap + P.fast.gcap)
            for (int e = tid; e < isz; e += GS) mats[e] = img[e];
    }
    if (tid < 32) {
        load_record(P, p, reinterpret_cast<int4 *>(work), H);
        derive_layout(P, nvec, work_cap, H);
    }
    gsync<GS>();
    if (H.bad) {
        if (tid == 0 && P.err) atomicCAS(P.err, 0, 110 + H.bad);
        return;
    }
    const int m = H.m, R = H.R, NB = H.NB, NBo = H.NBo;
    const int *rk = P.fast.ranks + H.rank_off;
    const T *gtab = mats + H.matsz;  // the term's G tables follow its matrices

    for (int v0 = 0; v0 < nvec; v0 += H.vb) {
        const int vb = min(H.vb, nvec - v0);
        T *X = work, *Y = work + NB * vb, *bufA = Y + NB * vb;
        // gather X[i][v][o] through M^B, then the basis part Y = c0 X + sum_j H1_j x_j X
        // (element loops compiled for the chunk's vector count)
        switch (vb) {
#define SG_VB(VB) case VB: chunk_in<T, VB, GS>(H, P, x + (size_t)v0 * P.n_cs, rk, mats, X, Y, tid); break;
            SG_VB(1) SG_VB(2) SG_VB(3) SG_VB(4) SG_VB(5) SG_VB(6) SG_VB(7) SG_VB(8)
#undef SG_VB
        }
        if (H.grid) {
            const int ps = R + H.s;
            int vt_ngi = 1;
            for (int j = 0; j < R; j++) vt_ngi *= H.nq[j];
            const int NBIv = H.NBIn * vb;
            T *bufB = bufA + (size_t)H.NBIn * H.NGs * vb;
            for (int sl = 0; sl < H.nslice; sl++) {
                T *cur, *oth, *spare;
                if (H.s > 0) {
                    if (tid == 0) {
                        int rem = sl;
                        for (int j = ps - 1; j >= R; j--) { H.uS[j] = rem % H.nq[j]; rem /= H.nq[j]; }
                    }
                    gsync<GS>();
                    for (int ko = tid; ko < H.NBO; ko += GS) {
                        int rem = ko;
                        T wf = T(1), wb = T(1);
                        for (int j = ps - 1; j >= R; j--) {
                            const int kj = rem % H.nb[j];
                            rem /= H.nb[j];
                            wf *= mats[H.oB[j] + H.uS[j] * H.nb[j] + kj];
                            wb *= mats[H.oBW[j] + kj * H.nq[j] + H.uS[j]];
                        }
                        WoF[ko] = wf; WoB[ko] = wb;
                    }
                    gsync<GS>();
                    // Xs[iv][rest] = sum_ko WoF[ko] X[iv][ko][rest]
                    for (FibreWalk w = fibre_walk<GS>(H.NBrest, tid); w.a < NBIv; w.step(H.NBrest)) {
                        const T *xp = X + (size_t)w.a * NBo + w.c;
                        T acc = T(0);
                        for (int ko = 0; ko < H.NBO; ko++) acc += WoF[ko] * xp[ko * H.NBrest];
                        bufA[w.a * H.NBrest + w.c] = acc;
                    }
                    gsync<GS>();
                    cur = bufA; oth = bufB; spare = bufA;
                } else {
                    cur = X; oth = bufA; spare = bufB;  // X is not needed after the basis part
                }
                // outer basis -> grid (ping-pong between the two grid buffers)
                int A = NBIv;
                for (int j = ps; j < m; j++) {
                    int C = 1;
                    for (int i2 = j + 1; i2 < m; i2++) C *= H.nb[i2];
                    fcontract<T, GS>(cur, oth, A, H.nb[j], H.nq[j], C, mats + H.oB[j], tid);
                    A *= H.nq[j];
                    T *freed = (cur == X) ? spare : cur;
                    cur = oth; oth = freed;
                    gsync<GS>();
                }
                if (cur == X) oth = bufA;
                // inner slots and potential, in registers
                {
                    const T *vts = FTab<T>::vt(P) + P.fast.vt_off[p] + (size_t)sl * H.NGs * (size_t)vt_ngi;
                    switch (R) {
                        case 0: reg_phase<T, 0, NB1, NQ1, UNI, GS>(H, mats, vts, cur, vb, tid); break;
                        case 1: if constexpr (RMAX >= 1) reg_phase<T, 1, NB1, NQ1, UNI, GS>(H, mats, vts, cur, vb, tid); break;
                        case 2: if constexpr (RMAX >= 2) reg_phase<T, 2, NB1, NQ1, UNI, GS>(H, mats, vts, cur, vb, tid); break;
                        case 3: if constexpr (RMAX >= 3) reg_phase<T, 3, NB1, NQ1, UNI, GS>(H, mats, vts, cur, vb, tid); break;
                        default: break;
                    }
                }
                gsync<GS>();
                // outer grid -> basis, reverse order
                for (int j = m - 1; j >= ps; j--) {
                    int Aj = NBIv, C = 1;
                    for (int i2 = ps; i2 < j; i2++) Aj *= H.nq[i2];
                    for (int i2 = j + 1; i2 < m; i2++) C *= H.nb[i2];
                    fcontract<T, GS>(cur, oth, Aj, H.nq[j], H.nb[j], C, mats + H.oBW[j], tid);
                    T *tp = cur; cur = oth; oth = tp;
                    gsync<GS>();
                }
                // Y[iv][ko][rest] += WoB[ko] cur[iv][rest]
                if (H.s > 0) {
                    for (FibreWalk w = fibre_walk<GS>(H.NBrest, tid); w.a < NBIv * H.NBO; w.step(H.NBrest)) {
                        const int iv = fdiv(w.a, H.NBO, H.nbOmag), ko = w.a - iv * H.NBO;
                        Y[w.a * H.NBrest + w.c] += WoB[ko] * cur[iv * H.NBrest + w.c];
                    }
                } else {
                    for (int e = tid; e < NB * vb; e += GS) Y[e] += cur[e];
                }
                gsync<GS>();
            }
        }
        // exact compress-add of D_l * y_l
        switch (vb) {
#define SG_VB(VB) case VB: chunk_out<T, VB, GS>(H, P, rk, maxbits + v0, accp + (size_t)v0 * P.n_cs * fx::Acc<T>::words, Y, tid); break;
            SG_VB(1) SG_VB(2) SG_VB(3) SG_VB(4) SG_VB(5) SG_VB(6) SG_VB(7) SG_VB(8)
#undef SG_VB
        }
    }
}

// Terms [p0, p0 + pcount) of one problem's processing order; NG = 128 / GS
// term groups per block.
template <typename T, int NB1, int NQ1, int RMAX, bool UNI, int GS>
__global__ void __launch_bounds__(kFT, sizeof(T) == 4 ? SG_F32_MINBLOCKS : SG_F64_MINBLOCKS)
    k_apply_fast(const KParams P, const double *__restrict__ x, const long long *__restrict__ maxbits, int nvec,
                 int p0, int pcount, int work_cap)
{
    constexpr int NG = kFT / GS;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ FHdr Hs[NG];
    const int grp = threadIdx.x / GS, tid = threadIdx.x % GS;
    const int pidx = blockIdx.x * NG + grp;
    if (pidx >= pcount) return;
    fast_term<T, NB1, NQ1, RMAX, UNI, GS>(P, x, P.acc, maxbits, nvec, p0 + pidx, work_cap,
                                          smraw + (size_t)grp * part_bytes(P, sizeof(T), work_cap), Hs[grp],
                                          tid);
}

// Many problems in one launch: work item i = (problem, processing position);
// items come ordered by estimated cost over all problems.  Problem j's
// vectors, accumulators and exponents start at nvec * cs_prefix[j] (times
// kAccDigits for the accumulators) and j * nvec.  Every group's shared-memory
// partition is `part` bytes, the largest over the problems.
template <typename T, int NB1, int NQ1, int RMAX, bool UNI, int GS>
__global__ void __launch_bounds__(kFT, sizeof(T) == 4 ? SG_F32_MINBLOCKS : SG_F64_MINBLOCKS)
    k_apply_fast_batch(const KParams *__restrict__ kps, const int2 *__restrict__ items, int count,
                       const double *__restrict__ x, unsigned long long *acc,
                       const long long *__restrict__ maxbits, const long long *__restrict__ cs_prefix, int nvec,
                       int part)
{
    constexpr int NG = kFT / GS;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ FHdr Hs[NG];
    const int grp = threadIdx.x / GS, tid = threadIdx.x % GS;
    const int pidx = blockIdx.x * NG + grp;
    if (pidx >= count) return;
    const int2 it = items[pidx];
    const KParams &P = kps[it.x];
    const size_t off = (size_t)nvec * (size_t)cs_prefix[it.x];
    fast_term<T, NB1, NQ1, RMAX, UNI, GS>(P, x + off, acc + off * fx::Acc<T>::words, maxbits + (size_t)it.x * nvec, nvec,
                                          it.y, GS == kFT ? P.fast.work_cta : P.fast.work_warp,
                                          smraw + (size_t)grp * part, Hs[grp], tid);
}

// Sets a kernel's dynamic shared-memory limit to the most the device allows
// beside the kernel's static shared memory (a property of the kernel, shared
// by every context, so never one context's own need); fails if `need` is more.
template <typename K>
cudaError_t set_smem_limit(K kernel, size_t need)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const long long lim = (long long)optin - (long long)fa.sharedSizeBytes;
    if (lim <= 0 || (long long)need > lim) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
}

template <typename T, int NB1, int NQ1, int RMAX, bool UNI>
cudaError_t launch_t(const KParams &kp, const FastLaunch &a)
{
    const size_t rb = sizeof(T);
    const size_t smem_cta = part_bytes(kp, rb, kp.fast.work_cta);
    const size_t smem_warp = (size_t)(kFT / 32) * part_bytes(kp, rb, kp.fast.work_warp);
    if (a.configure) {
        cudaError_t e = set_smem_limit(k_apply_fast<T, NB1, NQ1, RMAX, UNI, kFT>, smem_cta);
        if (e != cudaSuccess) return e;
        return set_smem_limit(k_apply_fast<T, NB1, NQ1, RMAX, UNI, 32>, smem_warp);
    }
    const int nbig = kp.fast.n_big, nrest = (int)kp.n_terms - nbig;
    if (nbig > 0)
        k_apply_fast<T, NB1, NQ1, RMAX, UNI, kFT><<<(unsigned)nbig, kFT, smem_cta, a.stream>>>(
            kp, a.x, a.maxbits, a.nvec, 0, nbig, kp.fast.work_cta);
    if (nrest > 0) {
        const unsigned blocks = (unsigned)((nrest + kFT / 32 - 1) / (kFT / 32));
        k_apply_fast<T, NB1, NQ1, RMAX, UNI, 32><<<blocks, kFT, smem_warp, a.stream>>>(
            kp, a.x, a.maxbits, a.nvec, nbig, nrest, kp.fast.work_warp);
    }
    return cudaGetLastError();
}

template <typename T, int NB1, int NQ1, int RMAX, bool UNI>
cudaError_t batch_t(const FastBatchLaunch &a)
{
    constexpr int NG = kFT / 32;
    if (a.configure) {
        cudaError_t e = set_smem_limit(k_apply_fast_batch<T, NB1, NQ1, RMAX, UNI, kFT>, (size_t)a.part[0]);
        if (e != cudaSuccess) return e;
        return set_smem_limit(k_apply_fast_batch<T, NB1, NQ1, RMAX, UNI, 32>, (size_t)NG * a.part[1]);
    }
    if (a.count[0] > 0)
        k_apply_fast_batch<T, NB1, NQ1, RMAX, UNI, kFT><<<(unsigned)a.count[0], kFT, (size_t)a.part[0], a.stream>>>(
            a.kps, a.items[0], a.count[0], a.x, a.acc, a.maxbits, a.cs_prefix, a.nvec, a.part[0]);
    if (a.count[1] > 0)
        k_apply_fast_batch<T, NB1, NQ1, RMAX, UNI, 32>
            <<<(unsigned)((a.count[1] + NG - 1) / NG), kFT, (size_t)NG * a.part[1], a.stream>>>(
                a.kps, a.items[1], a.count[1], a.x, a.acc, a.maxbits, a.cs_prefix, a.nvec, a.part[1]);
    return cudaGetLastError();
}

template <typename T_, int NB1_, int NQ1_, int RMAX_, bool UNI_>
struct Variant {
    using T = T_;
    static constexpr int NB1 = NB1_, NQ1 = NQ1_, RMAX = RMAX_;
    static constexpr bool UNI = UNI_;
};

// Calls f(Variant<...>{}) for the kernel variant of kp's fast tables.  The
// register-slot count must be fast_rmax(...): the host built the records with it.
template <typename T, bool UNI, typename F>
cudaError_t for_variant_u(const KParams &kp, F &&f)
{
    constexpr bool F32 = sizeof(T) == 4;
    const int nb1 = kp.fast.nb1, nq1 = kp.fast.nq1;
    if (nb1 == 2 && nq1 == 3) return f(Variant<T, 2, 3, F32 ? SG_F32_RMAX2 : SG_F64_RMAX2, UNI>{});
    if (nb1 == 2 && nq1 == 2) return f(Variant<T, 2, 2, F32 ? SG_F32_RMAX2 : SG_F64_RMAX2, UNI>{});
    if (nb1 == 3 && nq1 == 3) return f(Variant<T, 3, 3, F32 ? SG_F32_RMAX3 : 1, UNI>{});
    return f(Variant<T, 1, 1, 0, UNI>{});
}

template <typename T, typename F>
cudaError_t for_variant(const KParams &kp, F &&f)
{
    return kp.fast.uni1 ? for_variant_u<T, true>(kp, f) : for_variant_u<T, false>(kp, f);
}

}  // namespace

}  // namespace sg
