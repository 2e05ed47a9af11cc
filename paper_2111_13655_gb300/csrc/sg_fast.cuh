// Device code of the fast path of the Smolyak operator action (sm_103a):
// potentials whose monomials touch at most two modes (the Henon-Heiles family
// of Sec. 4, Eq. (18)).  Included by the units that instantiate it:
// sg_fast_f32.cu / sg_fast_f64.cu / sg_fast_df.cu (one problem per launch;
// T = float, double or the double-float pair df2), sg_fast_batch_f32.cu /
// sg_fast_batch_f64.cu (many problems per launch) and sg_apply_fast.cu (the
// per-context set-up kernels).
//
// One thread block (or, for small terms, one warp) per Smolyak term, terms
// ordered most-expensive first.  With the grid operator split as described in
// build_fast_tables, the term operator of Alg. 1 is
//     y_l = c0 x_l + sum_j H1_j x_l + (x_j B_j^T W_j) diag(V_l) (x_j B_j) x_l,
// V_l(u) = sum over the term's active coupled pairs of G_p(u_a, u_b).
//
// Positions of a term: the transformed modes (nb > 1).  Up to three level-1
// modes are "inner" positions, the others "outer".  The basis -> grid
// (Eq. (15)) and grid -> basis (Eq. (14)) transfers of the outer positions
// run mode by mode in shared memory.  The inner positions never go to the
// grid in the term kernel: at every outer grid point g their whole action,
//     M_g = (x_in B^T W) diag(V_l(g, .)) (x_in B) + c0 I + sum_{j inner} H1_j,
// an NBI x NBI symmetric matrix (NBI = product of the inner sizes), is the
// same for every apply.  It is formed once per context in FP64 (k_build_mtab)
// from the quadrature rule, the pair tables and the single-mode matrices, and
// stored per term ("inner-block table").  Because B_j^T W_j B_j = I for nq >= nb
// on the outer positions, applying M_g between the outer transfers gives
// exactly the term operator above (up to rounding).
//
// Shared-memory layout of a term tensor: [outer site][vector][inner index],
// the outer site in canonical order (first outer position slowest).  A site
// holds a contiguous payload of vb * NBI values, moved as 16-byte vectors:
//   forward pass of position j:  [k_j][rest][payload] -> [rest][u_j][payload]
//     (the slowest axis is contracted and becomes the fastest), positions in
//     the order of fewest multiply-adds, ending on the canonical grid order;
//   backward pass of position j: [rest][u_j][payload] -> [k_j][rest][payload]
//     (the fastest axis is contracted and becomes the slowest), positions in
//     reverse order, ending on the canonical basis order.
// The basis part of the outer positions is fused with the exact fixed-point
// compress-add of D_l * y_l (sg_fixed.cuh).
//
// Per term, before the first chunk: the term's image (its 1D matrices and
// pair tables) and its slice of M^B are copied into shared memory while one
// warp decodes the record; one thread issues L2 prefetches of the data of the
// term one residency ahead.  Each chunk gathers its vectors from the
// entry-major copy of x made at the start of the apply (k_stage_x), where the
// vectors of one compact entry are adjacent.
#pragma once

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "sg_fixed.cuh"
#include "sg_internal.h"

namespace sg {

// One problem per launch (sg_fast_f32.cu, sg_fast_f64.cu, sg_fast_df.cu).
struct FastLaunch {
    const double *x;
    int nvec;
    const long long *maxbits;
    cudaStream_t stream;
    bool configure;  // set the kernels' shared-memory limits instead of launching
};
cudaError_t fast_launch_f32(const KParams &kp, const FastLaunch &a);
cudaError_t fast_launch_f64(const KParams &kp, const FastLaunch &a);
cudaError_t fast_launch_df(const KParams &kp, const FastLaunch &a);

// Many problems of one precision per launch (sg_fast_batch_f32.cu,
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
    int m, R, NB, NBI, NBo, grid, bad, coef;
    int s, vb, NBO, NBrest, NGs, nslice;
    int matsz, npair, nind;
    double c0;
    long long rank_off;
    int mode[kMaxD], nb[kMaxD], nq[kMaxD];               // by position
    int ostride[kMaxD];                                  // stride inside the inner index (j < R) or in outer sites
    unsigned smag[kMaxD], bmag[kMaxD];                   // reciprocals of ostride and nb
    int oB[kMaxD], oBW[kMaxD], oH[kMaxD];                // shared-memory offsets of B, B^T W, H1
    int gB[kMaxD], gBW[kMaxD], gH1[kMaxD];               // global offsets of B, B^T W (1D tables), H1 base (fast tables)
    int gstride[kMaxD];                                  // grid strides of the non-sliced outer positions
    int bymode[kMaxD];                                   // positions sorted by mode
    int uS[kMaxD];                                       // slice digits of the sliced positions
    int pgg[kMaxPairs], ioffs[kMaxPairs];                // G-table and induced-matrix offsets (fast tables)
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
__device__ __forceinline__ df2 fma_t(df2 a, df2 b, df2 c) { return df_fma(a, b, c); }

// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of 16)
static __device__ __forceinline__ void l2_prefetch_bulk(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// at most this much of a term's inner-block table is prefetched at entry
constexpr int kMtPrefetchBytes = 32768;
// Bulk prefetch of the 16-byte units inside [p0, p1) bytes of a buffer that
// starts 16-byte aligned (the ends are rounded inwards, never outside it),
// at most `cap` bytes.
static __device__ __forceinline__ void l2_prefetch_span(const void *base, size_t p0, size_t p1, size_t cap)
{
    const size_t b0 = (p0 + 15) & ~(size_t)15, b1 = p1 & ~(size_t)15;
    if (b1 <= b0) return;
    const size_t n = b1 - b0 < cap ? b1 - b0 : cap;
    l2_prefetch_bulk(reinterpret_cast<const unsigned char *>(base) + b0, (unsigned)n);
}
#ifndef SG_LOOKAHEAD
#define SG_LOOKAHEAD 1
#endif


template <typename T> struct FTab;
template <> struct FTab<double> {
    static __device__ const double *mt(const KParams &P) { return P.fast.mtabd; }
    static __device__ const double *img(const KParams &P) { return P.fast.imgd; }
};
template <> struct FTab<float> {
    static __device__ const float *mt(const KParams &P) { return P.fast.mtabf; }
    static __device__ const float *img(const KParams &P) { return P.fast.imgf; }
};
template <> struct FTab<df2> {
    static __device__ const df2 *mt(const KParams &P) { return reinterpret_cast<const df2 *>(P.fast.mtabx); }
    static __device__ const df2 *img(const KParams &P) { return reinterpret_cast<const df2 *>(P.fast.imgx); }
};

// W consecutive elements of T moved as one access (W * sizeof(T) <= 16 bytes)
template <typename T, int W>
struct alignas(sizeof(T) * W) VecT {
    T v[W];
};
template <typename T, int W>
__device__ __forceinline__ VecT<T, W> vld(const T *p)
{
    return *reinterpret_cast<const VecT<T, W> *>(p);
}
template <typename T, int W>
__device__ __forceinline__ void vst(T *p, const VecT<T, W> &a)
{
    *reinterpret_cast<VecT<T, W> *>(p) = a;
}
// read-only global loads of one unit
template <typename T, int W> struct Ldg;
template <> struct Ldg<float, 1> {
    static __device__ __forceinline__ VecT<float, 1> f(const float *p) { return {{__ldg(p)}}; }
};
template <> struct Ldg<float, 4> {
    static __device__ __forceinline__ VecT<float, 4> f(const float *p)
    {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        return {{t.x, t.y, t.z, t.w}};
    }
};
template <> struct Ldg<df2, 1> {
    static __device__ __forceinline__ VecT<df2, 1> f(const df2 *p)
    {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        return {{df2(t.x, t.y)}};
    }
};
template <> struct Ldg<df2, 2> {
    static __device__ __forceinline__ VecT<df2, 2> f(const df2 *p)
    {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        return {{df2(t.x, t.y), df2(t.z, t.w)}};
    }
};
template <> struct Ldg<double, 1> {
    static __device__ __forceinline__ VecT<double, 1> f(const double *p) { return {{__ldg(p)}}; }
};
template <> struct Ldg<double, 2> {
    static __device__ __forceinline__ VecT<double, 2> f(const double *p)
    {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        return {{t.x, t.y}};
    }
};

// elements per 16 bytes
template <typename T> __host__ __device__ constexpr int vunit() { return 16 / (int)sizeof(T); }

__host__ __device__ constexpr int tri_index(int r, int c, int n)
{
    // row r of the upper triangle starts after rows 0..r-1 (n, n-1, ... entries)
    return r <= c ? r * n - r * (r - 1) / 2 + (c - r) : c * n - c * (c - 1) / 2 + (r - c);
}

// Per-term set-up from the term's record (built on the host): warp 0 copies
// the record to shared memory and parses it.
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
    for (int q = lane; q < np; q += 32) { H.pa[q] = pr[q].pa; H.pb[q] = pr[q].pb; H.pgg[q] = pr[q].goff; }
    for (int q = lane; q < ni; q += 32) { H.ipos[q] = in[q].pos; H.ioffs[q] = in[q].ioff; }
    if (lane == 0) {
        H.m = m; H.R = hd->R; H.NB = hd->NB; H.coef = hd->coef; H.s = hd->s;
        H.npair = np; H.nind = ni; H.c0 = hd->c0; H.rank_off = hd->rank_off;
        H.grid = np > 0;
    }
    __syncwarp();
}

// Layout quantities of the term, shared memory only: lane j handles position j.
template <typename T>
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
        H.bmag[j] = rmag(nb);
        H.ostride[j] = st; H.smag[j] = rmag(st);
        H.gstride[j] = gs;
        H.bymode[rank] = j;
    }
    __syncwarp();
    if (lane != 0) return;
    H.bad = 0;
    int mat = 0, NBI = 1;
    H.NBO = 1; H.nslice = 1; H.NBrest = 1; H.NGs = 1;
    for (int j = 0; j < m; j++) {
        mat += 2 * H.nq[j] * H.nb[j] + H.nb[j] * H.nb[j];
        if (j < R) NBI *= H.nb[j];
        else if (j < R + sv) { H.NBO *= H.nb[j]; H.nslice *= H.nq[j]; }
        else { H.NBrest *= H.nb[j]; H.NGs *= H.nq[j]; }
    }
    if (mat > P.matcap || H.NBO > P.fast.nbocap) { H.bad = 1; return; }
    H.matsz = mat;
    H.NBI = NBI; H.NBo = H.NB / NBI;
    constexpr int U = vunit<T>();
    const int64_t stage = (int64_t)NBI * H.NGs;
    if (chunk_need(H.NB, stage, sv > 0, H.grid, 1, U) > work) { H.bad = 2; return; }
    int vb = nvec < kMaxVB ? nvec : kMaxVB;
    while (vb > 1 && chunk_need(H.NB, stage, sv > 0, H.grid, vb, U) > work) vb--;
    H.vb = vb;
}

// ---------------------------------------------------------------------------
// One-position transfers over a tensor of sites with a payload of PW units of
// W elements each (unit-aligned).  M is the nout x nin matrix (row-major) of
// the transfer: B (nq x nb) forward, B^T W (nb x nq) backward.
//
// forward:  in[k][c][pw] -> out[c][u][pw],  c < C, out = sum_k M[u][k] in[k]
// backward: in[c][u][pw] -> out[k][c][pw]
template <typename T, int W, int NI, int NO, int GS>
__device__ __forceinline__ void fwd_pass_t(const T *__restrict__ in, T *__restrict__ out, int C, int PW,
                                           unsigned pwmag, const T *__restrict__ M, int tid)
{
    T mr[NO * NI];
#pragma unroll
    for (int i = 0; i < NO * NI; i++) mr[i] = M[i];
    const int total = C * PW, cpw = C * PW;
    for (int w = tid; w < total; w += GS) {
        const int c = fdiv(w, PW, pwmag), pw = w - c * PW;
        VecT<T, W> xv[NI];
#pragma unroll
        for (int k = 0; k < NI; k++) xv[k] = vld<T, W>(in + (size_t)(k * cpw + w) * W);
        T *op = out + (size_t)((c * NO) * PW + pw) * W;
#pragma unroll
        for (int u = 0; u < NO; u++) {
            VecT<T, W> a;
#pragma unroll
            for (int e = 0; e < W; e++) {
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < NI; k++) acc = fma_t(mr[u * NI + k], xv[k].v[e], acc);
                a.v[e] = acc;
            }
            vst<T, W>(op + (size_t)u * PW * W, a);
        }
    }
}

template <typename T, int W, int NI, int NO, int GS>
__device__ __forceinline__ void bwd_pass_t(const T *__restrict__ in, T *__restrict__ out, int C, int PW,
                                           unsigned pwmag, const T *__restrict__ M, int tid)
{
    T mr[NO * NI];
#pragma unroll
    for (int i = 0; i < NO * NI; i++) mr[i] = M[i];
    const int total = C * PW, cpw = C * PW;
    for (int w = tid; w < total; w += GS) {
        const int c = fdiv(w, PW, pwmag), pw = w - c * PW;
        const T *ip = in + (size_t)((c * NI) * PW + pw) * W;
        VecT<T, W> xv[NI];
#pragma unroll
        for (int u = 0; u < NI; u++) xv[u] = vld<T, W>(ip + (size_t)u * PW * W);
#pragma unroll
        for (int k = 0; k < NO; k++) {
            VecT<T, W> a;
#pragma unroll
            for (int e = 0; e < W; e++) {
                T acc = T(0);
#pragma unroll
                for (int u = 0; u < NI; u++) acc = fma_t(mr[k * NI + u], xv[u].v[e], acc);
                a.v[e] = acc;
            }
            vst<T, W>(out + (size_t)(k * cpw + w) * W, a);
        }
    }
}

// Any sizes (levels beyond the compiled ones): matrix and inputs read from
// shared memory per output.
template <typename T, int W, int GS>
__device__ void pass_rt(const T *__restrict__ in, T *__restrict__ out, int C, int PW, unsigned pwmag, int ni,
                        int no, const T *__restrict__ M, bool forward, int tid)
{
    const int total = C * PW, cpw = C * PW;
    for (int w = tid; w < total; w += GS) {
        const int c = fdiv(w, PW, pwmag), pw = w - c * PW;
        for (int r = 0; r < no; r++) {
            VecT<T, W> a;
#pragma unroll
            for (int e = 0; e < W; e++) a.v[e] = T(0);
            for (int k = 0; k < ni; k++) {
                const T mv = M[r * ni + k];
                const VecT<T, W> xv = forward ? vld<T, W>(in + (size_t)(k * cpw + w) * W)
                                              : vld<T, W>(in + (size_t)((c * ni + k) * PW + pw) * W);
#pragma unroll
                for (int e = 0; e < W; e++) a.v[e] = fma_t(mv, xv.v[e], a.v[e]);
            }
            if (forward) vst<T, W>(out + (size_t)((c * no + r) * PW + pw) * W, a);
            else vst<T, W>(out + (size_t)(r * cpw + w) * W, a);
        }
    }
}

template <typename T, int W, int GS>
__device__ void fwd_pass(const T *in, T *out, int C, int PW, int nb, int nq, const T *M, int tid)
{
    const unsigned mag = rmag((unsigned)PW);
#define SG_FP(NI, NO) case (NI) * 64 + (NO): fwd_pass_t<T, W, NI, NO, GS>(in, out, C, PW, mag, M, tid); return;
    switch (nb * 64 + nq) {
        SG_FP(2, 3) SG_FP(3, 4) SG_FP(4, 5) SG_FP(5, 6) SG_FP(2, 2) SG_FP(3, 3) SG_FP(4, 4) SG_FP(5, 5)
        default: pass_rt<T, W, GS>(in, out, C, PW, mag, nb, nq, M, true, tid); return;
    }
#undef SG_FP
}

template <typename T, int W, int GS>
__device__ void bwd_pass(const T *in, T *out, int C, int PW, int nq, int nb, const T *M, int tid)
{
    const unsigned mag = rmag((unsigned)PW);
#define SG_BP(NI, NO) case (NI) * 64 + (NO): bwd_pass_t<T, W, NI, NO, GS>(in, out, C, PW, mag, M, tid); return;
    switch (nq * 64 + nb) {
        SG_BP(3, 2) SG_BP(4, 3) SG_BP(5, 4) SG_BP(6, 5) SG_BP(2, 2) SG_BP(3, 3) SG_BP(4, 4) SG_BP(5, 5)
        default: pass_rt<T, W, GS>(in, out, C, PW, mag, nq, nb, M, false, tid); return;
    }
#undef SG_BP
}

// Register phase: at every outer grid point g of the slice, every vector's
// inner block z (NBI values) becomes M_g z, in place in Z[g][v][i].  M_g is
// read from the inner-block table tab ([unit][g][unit elements], this slice).
// One (grid point, vector) pair per work item; M_g is read once per item (the
// items of one grid point share its cache lines).  When an inner block spans
// two 16-byte units, they are read and written in an order that alternates
// per group of four threads, which keeps a quarter warp's 16-byte accesses on
// distinct banks.
template <typename T, int NBI, int GS>
__device__ void reg_phase(const T *__restrict__ tab, T *Z, int NGs, int vb, int tid)
{
    constexpr int U = vunit<T>();
    constexpr int UE = NBI == 1 ? 1 : U;
    constexpr int NEU = (NBI * (NBI + 1) / 2 + UE - 1) / UE;
    constexpr bool TWO = NBI == 2 * U;  // the block is exactly two 16-byte units
    constexpr int ZW = (NBI * (int)sizeof(T)) % 16 == 0 ? U : NBI == 2 && sizeof(T) == 4 ? 2 : 1;
    const int total = NGs * vb;
    const unsigned vmag = rmag((unsigned)vb);
    for (int w = tid; w < total; w += GS) {
        const int g = fdiv(w, vb, vmag);
        T mm[NEU * UE];
#pragma unroll
        for (int q = 0; q < NEU; q++) {
            const VecT<T, UE> t = Ldg<T, UE>::f(tab + ((size_t)q * NGs + g) * UE);
#pragma unroll
            for (int e = 0; e < UE; e++) mm[q * UE + e] = t.v[e];
        }
        T *zp = Z + (size_t)w * NBI;
        T z[NBI], y[NBI];
        if constexpr (TWO) {
            const bool h = (w >> 2) & 1;
            const VecT<T, U> a = vld<T, U>(zp + (h ? U : 0)), b = vld<T, U>(zp + (h ? 0 : U));
#pragma unroll
            for (int e = 0; e < U; e++) { z[e] = h ? b.v[e] : a.v[e]; z[U + e] = h ? a.v[e] : b.v[e]; }
        } else {
#pragma unroll
            for (int i = 0; i < NBI; i += ZW) {
                const VecT<T, ZW> t = vld<T, ZW>(zp + i);
#pragma unroll
                for (int e = 0; e < ZW; e++) z[i + e] = t.v[e];
            }
        }
#pragma unroll
        for (int r = 0; r < NBI; r++) {
            T acc = T(0);
#pragma unroll
            for (int c = 0; c < NBI; c++) acc = fma_t(mm[tri_index(r, c, NBI)], z[c], acc);
            y[r] = acc;
        }
        if constexpr (TWO) {
            const bool h = (w >> 2) & 1;
            VecT<T, U> a, b;
#pragma unroll
            for (int e = 0; e < U; e++) { a.v[e] = h ? y[U + e] : y[e]; b.v[e] = h ? y[e] : y[U + e]; }
            vst<T, U>(zp + (h ? U : 0), a);
            vst<T, U>(zp + (h ? 0 : U), b);
        } else {
#pragma unroll
            for (int i = 0; i < NBI; i += ZW) {
                VecT<T, ZW> t;
#pragma unroll
                for (int e = 0; e < ZW; e++) t.v[e] = y[i + e];
                vst<T, ZW>(zp + i, t);
            }
        }
    }
}

// Shared-memory partition of one term group: matrices, slice weights
// (head), then the work area.
__host__ __device__ inline size_t part_head_bytes(const KParams &P, size_t rb)
{
    return (((size_t)P.matcap + P.fast.gcap + 2 * (size_t)P.fast.nbocap) * rb + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t part_bytes(const KParams &P, size_t rb, int work)
{
    return (part_head_bytes(P, rb) + (size_t)work * rb + 15) & ~(size_t)15;
}

// Gather of one chunk: X[o][v][i] = x_v[rank(o, i)] (M^B holds the ranks in
// the order [outer site][inner index]).  The source is either the
// entry-major copy xs (ST: element (r, v) at r * stride + v, in T; the
// threads of consecutive vectors read consecutive words) or x itself (vector
// v at v * n_cs, FP64).
template <typename T, int NBI, int GS, bool ST>
__device__ __forceinline__ void gather_t(const FHdr &H, const void *__restrict__ src, size_t stride,
                                         const int *__restrict__ rk, T *X, int vb, int tid)
{
    constexpr int ZW = (NBI * (int)sizeof(T)) % 16 == 0 ? vunit<T>() : NBI == 2 && sizeof(T) == 4 ? 2 : 1;
    const int NBo = H.NBo, total = NBo * vb;
    const unsigned vmag = rmag((unsigned)vb);
    for (int w = tid; w < total; w += GS) {
        const int o = fdiv(w, vb, vmag), v = w - o * vb;
        const int *rp = rk + (size_t)o * NBI;
        T val[NBI];
        if constexpr (ST) {
            const T *xv = static_cast<const T *>(src) + v;
#pragma unroll
            for (int i = 0; i < NBI; i++) val[i] = Ldg<T, 1>::f(xv + (size_t)rp[i] * stride).v[0];
        } else {
            const double *xv = static_cast<const double *>(src) + (size_t)v * stride;
#pragma unroll
            for (int i = 0; i < NBI; i++) val[i] = (T)__ldg(xv + rp[i]);
        }
        T *dst = X + (size_t)w * NBI;
#pragma unroll
        for (int i = 0; i < NBI; i += ZW) {
            VecT<T, ZW> t;
#pragma unroll
            for (int e = 0; e < ZW; e++) t.v[e] = val[i + e];
            vst<T, ZW>(dst + i, t);
        }
    }
}

template <typename T, int GS, bool ST>
__device__ void gather_rt(const FHdr &H, const void *__restrict__ src, size_t stride, const int *__restrict__ rk,
                          T *X, int vb, int tid)
{
    const int NBI = H.NBI, total = H.NBo * vb;
    const unsigned vmag = rmag((unsigned)vb);
    for (int w = tid; w < total; w += GS) {
        const int o = fdiv(w, vb, vmag), v = w - o * vb;
        for (int i = 0; i < NBI; i++) {
            const size_t r = (size_t)rk[(size_t)o * NBI + i];
            X[(size_t)w * NBI + i] = ST ? Ldg<T, 1>::f(static_cast<const T *>(src) + r * stride + v).v[0]
                                        : (T)__ldg(static_cast<const double *>(src) + (size_t)v * stride + r);
        }
    }
}

template <typename T, int GS, bool ST>
__device__ void gather_s(const FHdr &H, const void *src, size_t stride, const int *rk, T *X, int vb, int tid)
{
    switch (H.NBI) {
        case 1: gather_t<T, 1, GS, ST>(H, src, stride, rk, X, vb, tid); return;
        case 2: gather_t<T, 2, GS, ST>(H, src, stride, rk, X, vb, tid); return;
        case 4: gather_t<T, 4, GS, ST>(H, src, stride, rk, X, vb, tid); return;
        case 8: gather_t<T, 8, GS, ST>(H, src, stride, rk, X, vb, tid); return;
        default: gather_rt<T, GS, ST>(H, src, stride, rk, X, vb, tid); return;
    }
}

// The chunk's vectors v0 .. v0 + vb - 1: from the problem's entry-major copy
// when it has one, else from x.
template <typename T, int GS>
__device__ void gather(const FHdr &H, const KParams &P, const double *x, int v0, const int *rk, T *X, int vb,
                       int tid)
{
    if (P.xs)
        gather_s<T, GS, true>(H, static_cast<const T *>(P.xs) + v0, (size_t)xs_stride(P.xs_nvec), rk, X, vb, tid);
    else
        gather_s<T, GS, false>(H, x + (size_t)v0 * P.n_cs, (size_t)P.n_cs, rk, X, vb, tid);
}

// Final step of a chunk, fused: y = F + (c0 X when the term has no grid) +
// sum over outer positions j of H1_j x_j X, then the exact compress-add of
// D_l * y into the accumulators.  First pass: work item = (outer site o, unit
// of W payload elements); y is written to `dst` in the payload layout
// [o][v][i] (dst = F, each unit in place -- only its own item reads it -- or,
// without a grid, a separate basis-sized area).  A barrier.  Second pass: one
// element per item in the order [o][i][v] (inner index, then vector), so the
// lanes of a warp that share a compact entry add into consecutive words (the
// accumulators are entry-major: entry r, vector v at r * nvec + v).
template <typename T, int W, int GS>
__device__ void combine_add(const FHdr &H, const KParams &P, const int *__restrict__ rk,
                            const long long *__restrict__ maxbits, unsigned long long *acc, int nvec, int v0,
                            const T *X, const T *F, T *dst, const T *mats, int vb, int tid)
{
    const int NBI = H.NBI, Pl = NBI * vb, PW = Pl / W, total = H.NBo * PW;
    const int m = H.m, R = H.R;
    const unsigned pwmag = rmag((unsigned)PW);
    const T c0 = H.grid ? T(0) : (T)H.c0;
    for (int w = tid; w < total; w += GS) {
        const int o = fdiv(w, PW, pwmag), pw = w - o * PW;
        const size_t eoff = (size_t)w * W;  // = o * Pl + pw * W
        T a[W];
        {
            const VecT<T, W> xv = vld<T, W>(X + eoff);
            if (F) {
                const VecT<T, W> fv = vld<T, W>(F + eoff);
#pragma unroll
                for (int e = 0; e < W; e++) a[e] = fma_t(c0, xv.v[e], fv.v[e]);
            } else {
#pragma unroll
                for (int e = 0; e < W; e++) a[e] = c0 * xv.v[e];
            }
        }
        for (int j = R; j < m; j++) {
            const int q = fdiv(o, H.ostride[j], H.smag[j]);
            const int nbj = H.nb[j], kj = q - fdiv(q, nbj, H.bmag[j]) * nbj;
            const int st = H.ostride[j] * Pl;
            const T *xp = X + eoff - (size_t)kj * st;
            const T *hr = mats + H.oH[j] + kj * nbj;
            for (int kp = 0; kp < nbj; kp++) {
                const T hv = hr[kp];
                const VecT<T, W> xv = vld<T, W>(xp + (size_t)kp * st);
#pragma unroll
                for (int e = 0; e < W; e++) a[e] = fma_t(hv, xv.v[e], a[e]);
            }
        }
        VecT<T, W> out;
#pragma unroll
        for (int e = 0; e < W; e++) out.v[e] = a[e];
        vst<T, W>(dst + eoff, out);
    }
    gsync<GS>();
    const int n = H.NB * vb;
    const unsigned nbimag = rmag((unsigned)NBI);
    if (GS % vb == 0) {
        // each thread keeps one vector (and its accumulator unit) for the whole pass
        const int v = tid % vb, step = GS / vb;
        const int E = fx::Acc<T>::unit(maxbits[v0 + v]);
        unsigned long long *av = acc + (size_t)(v0 + v) * fx::Acc<T>::words;
        const T *dv = dst + (size_t)v * NBI;
        for (int oi = tid / vb; oi < H.NB; oi += step) {  // oi = o * NBI + i
            const int o = fdiv(oi, NBI, nbimag), i = oi - o * NBI;
            fx::Acc<T>::add_unit(av + (size_t)rk[oi] * nvec * fx::Acc<T>::words, dv[(size_t)o * Pl + i], H.coef, E,
                                 P.err);
        }
        return;
    }
    const unsigned vmag = rmag((unsigned)vb);
    for (int w = tid; w < n; w += GS) {
        const int oi = fdiv(w, vb, vmag), v = w - oi * vb;  // oi = o * NBI + i
        const int o = fdiv(oi, NBI, nbimag), i = oi - o * NBI;
        const int r = rk[oi];
        fx::Acc<T>::add(acc + ((size_t)r * nvec + v0 + v) * fx::Acc<T>::words, dst[(size_t)o * Pl + v * NBI + i],
                        H.coef, maxbits[v0 + v], P.err);
    }
}

// One Smolyak term (processing position p of problem P) by a group of GS
// threads: GS = 128 (a whole block) or GS = 32 (one warp; no block-wide
// barriers).  `base` is the group's shared-memory partition (part_bytes of P
// with `work_cap` work elements), `accp` the problem's fixed-point
// accumulators (entry-major, nvec vectors), `x` and `maxbits` its input
// vectors and their exponents.
template <typename T, int GS>
__device__ __forceinline__ void fast_term(const KParams &P, const double *__restrict__ x,
                                          unsigned long long *accp, const long long *__restrict__ maxbits,
                                          int nvec, int p, int work_cap, unsigned char *base, FHdr &H,
                                          const int tid, const KParams &PA, int pa)
{
    constexpr int U = vunit<T>();
    const size_t rb = sizeof(T);
    T *mats = reinterpret_cast<T *>(base);
    T *WoF = mats + P.matcap + P.fast.gcap;
    T *WoB = WoF + P.fast.nbocap;
    T *work = reinterpret_cast<T *>(base + part_head_bytes(P, rb));

    // the start of the term's inner-block table is fetched into L2 now: it is
    // first read after the gather and the forward transfers
    if (tid == 0) {
        const long long v0 = P.fast.mt_off[p], v1 = P.fast.mt_off[p + 1];
        if (v1 > v0) {
            // 16-byte aligned and rounded; the table buffer is padded by 16 bytes
            const size_t b0 = ((size_t)v0 * rb) & ~(size_t)15;
            const size_t e1 = ((size_t)v1 * rb + 15) & ~(size_t)15;
            const size_t b1 = e1 - b0 > (size_t)kMtPrefetchBytes ? b0 + (size_t)kMtPrefetchBytes : e1;
            l2_prefetch_bulk(reinterpret_cast<const unsigned char *>(FTab<T>::mt(P)) + b0, (unsigned)(b1 - b0));
        }
    }
    // Look-ahead: the group that will take processing position pa (of problem
    // *PA) about one residency later gets that term's record, image, compact
    // indices and the start of its inner-block table fetched into L2 now; its
    // offsets are read here and the prefetches issued after the prologue.
    // One thread: the first of warp 1 in the block form, lane 0 in the warp form.
    const bool la = SG_LOOKAHEAD && pa >= 0 && tid == (GS == 32 ? 0 : 32);
    unsigned la_d0 = 0, la_d1 = 0;
    long long la_i0 = 0, la_i1 = 0, la_r0 = 0, la_r1 = 0, la_m0 = 0, la_m1 = 0;
    if (la) {
        la_d0 = PA.fast.desc_off[pa]; la_d1 = PA.fast.desc_off[pa + 1];
        la_i0 = PA.fast.img_off[pa]; la_i1 = PA.fast.img_off[pa + 1];
        la_r0 = PA.fast.rank_start[pa]; la_r1 = PA.fast.rank_start[pa + 1];
        la_m0 = PA.fast.mt_off[pa]; la_m1 = PA.fast.mt_off[pa + 1];
    }
    // the term's image (B, B^T W, H1 per position, then its G tables) and its
    // compact indices (M^B) are copied as they lie while warp 0 decodes the
    // record (into a scratch at the end of the work area)
    int *rks = reinterpret_cast<int *>(work);
    const int64_t rec_off = record_scratch_offset((int64_t)work_cap * rb, P.fast.desccap);
    bool rfit;
    {
        const long long i0 = P.fast.img_off[p];
        const int isz = (int)(P.fast.img_off[p + 1] - i0);
        const T *img = FTab<T>::img(P) + i0;
        if (isz <= P.matcap + P.fast.gcap)
            for (int e = tid; e < isz; e += GS) mats[e] = img[e];
        const long long r0 = P.fast.rank_start[p];
        const int nr = (int)(P.fast.rank_start[p + 1] - r0);
        // the indices must stay clear of the record scratch (the planner keeps
        // them apart; a term that breaks this is refused below)
        rfit = 4 * (int64_t)nr <= rec_off;
        if (rfit)
            for (int e = tid; e < nr; e += GS) rks[e] = __ldg(P.fast.ranks + r0 + e);
    }
    if (tid < 32) {
        load_record(P, p, reinterpret_cast<int4 *>(reinterpret_cast<unsigned char *>(work) + rec_off), H);
        derive_layout<T>(P, nvec, work_cap, H);
    }
    gsync<GS>();
    if (la) {
        l2_prefetch_span(PA.fast.desc, 16 * (size_t)la_d0, 16 * (size_t)la_d1, ~(size_t)0);
        l2_prefetch_span(FTab<T>::img(PA), (size_t)la_i0 * rb, (size_t)la_i1 * rb, ~(size_t)0);
        l2_prefetch_span(PA.fast.ranks, 4 * (size_t)la_r0, 4 * (size_t)la_r1, ~(size_t)0);
        l2_prefetch_span(FTab<T>::mt(PA), (size_t)la_m0 * rb, (size_t)la_m1 * rb, (size_t)kMtPrefetchBytes);
    }
    if (H.bad || !rfit) {
        if (tid == 0 && P.err) atomicCAS(P.err, 0, 110 + (rfit ? H.bad : 3));
        return;
    }
    const int m = H.m, R = H.R, NB = H.NB, NBI = H.NBI;
    const int *rk = rks;  // the term's compact indices, in shared memory
    const bool sliced = H.s > 0;
    const int ps = R + H.s;  // first non-sliced outer position

    for (int v0 = 0; v0 < nvec; v0 += H.vb) {
        const int vb = min(H.vb, nvec - v0);
        const int Pl = NBI * vb;                       // payload elements per site
        const int WW = Pl % U == 0 ? U : 1;            // unit of the vector accesses
        const int PW = Pl / WW;
        T *X = work + ranks_elems(NB, U);
        T *Y = X + pad_elems((int64_t)NB * vb, U);
        T *A = sliced ? Y + pad_elems((int64_t)NB * vb, U) : Y;
        T *Bf = A + pad_elems((int64_t)NBI * H.NGs * vb, U);
        gather<T, GS>(H, P, x, v0, rk, X, vb, tid);
        gsync<GS>();
        const T *F = nullptr;
        if (H.grid) {
            for (int sl = 0; sl < H.nslice; sl++) {
                const T *cur;
                int nxt;
                if (sliced) {
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
                    // A[rest][payload] = sum_ko WoF[ko] X[ko][rest][payload]
                    const int nrest = H.NBrest * Pl;
                    for (int e = tid; e < nrest; e += GS) {
                        T acc = T(0);
                        for (int ko = 0; ko < H.NBO; ko++) acc = fma_t(WoF[ko], X[(size_t)ko * nrest + e], acc);
                        A[e] = acc;
                    }
                    gsync<GS>();
                    cur = A; nxt = 1;
                } else {
                    cur = X; nxt = 0;
                }
                // outer basis -> grid, positions ps..m-1 (slowest axis each time)
                int sites = H.NBrest;
                for (int j = ps; j < m; j++) {
                    const int C = sites / H.nb[j];
                    T *out = nxt ? Bf : A;
                    if (WW == U) fwd_pass<T, U, GS>(cur, out, C, PW, H.nb[j], H.nq[j], mats + H.oB[j], tid);
                    else fwd_pass<T, 1, GS>(cur, out, C, PW, H.nb[j], H.nq[j], mats + H.oB[j], tid);
                    sites = C * H.nq[j];
                    cur = out; nxt ^= 1;
                    gsync<GS>();
                }
                // inner blocks at every outer grid point
                {
                    T *Z = const_cast<T *>(cur);
                    const int ue = mt_unit(NBI, U), neu = mt_units(NBI, U);
                    const T *tab = FTab<T>::mt(P) + P.fast.mt_off[p] + (size_t)sl * neu * ue * H.NGs;
                    switch (NBI) {
                        case 1: reg_phase<T, 1, GS>(tab, Z, H.NGs, vb, tid); break;
                        case 2: reg_phase<T, 2, GS>(tab, Z, H.NGs, vb, tid); break;
                        case 3: reg_phase<T, 3, GS>(tab, Z, H.NGs, vb, tid); break;
                        case 4: reg_phase<T, 4, GS>(tab, Z, H.NGs, vb, tid); break;
                        case 8: reg_phase<T, 8, GS>(tab, Z, H.NGs, vb, tid); break;
                        case 9: reg_phase<T, 9, GS>(tab, Z, H.NGs, vb, tid); break;
                        default: break;
                    }
                }
                gsync<GS>();
                // outer grid -> basis, positions m-1..ps (fastest axis each time)
                for (int j = m - 1; j >= ps; j--) {
                    const int C = sites / H.nq[j];
                    T *out = nxt ? Bf : A;
                    if (WW == U) bwd_pass<T, U, GS>(cur, out, C, PW, H.nq[j], H.nb[j], mats + H.oBW[j], tid);
                    else bwd_pass<T, 1, GS>(cur, out, C, PW, H.nq[j], H.nb[j], mats + H.oBW[j], tid);
                    sites = C * H.nb[j];
                    cur = out; nxt ^= 1;
                    gsync<GS>();
                }
                if (sliced) {
                    // Y[ko][rest][payload] (+)= WoB[ko] cur[rest][payload]
                    const int nrest = H.NBrest * Pl;
                    for (int e = tid; e < nrest; e += GS) {
                        const T c = cur[e];
                        for (int ko = 0; ko < H.NBO; ko++) {
                            T *yp = Y + (size_t)ko * nrest + e;
                            *yp = sl == 0 ? WoB[ko] * c : fma_t(WoB[ko], c, *yp);
                        }
                    }
                    gsync<GS>();
                } else {
                    F = cur;
                }
            }
            if (sliced) F = Y;
        }
        // basis part of the outer positions and exact compress-add of D_l * y_l
        // (y in place of F; a term without a grid uses the area after X)
        T *dst = F ? const_cast<T *>(F) : Y;
        if (WW == U) combine_add<T, U, GS>(H, P, rk, maxbits, accp, nvec, v0, X, F, dst, mats, vb, tid);
        else combine_add<T, 1, GS>(H, P, rk, maxbits, accp, nvec, v0, X, F, dst, mats, vb, tid);
        gsync<GS>();
    }
}

// Terms [p0, p0 + pcount) of one problem's processing order; NG = 128 / GS
// term groups per block.
template <typename T, int GS>
__global__ void __launch_bounds__(kFT, sizeof(T) == 4 ? SG_F32_MINBLOCKS : SG_F64_MINBLOCKS)
    k_apply_fast(const KParams P, const double *__restrict__ x, const long long *__restrict__ maxbits, int nvec,
                 int p0, int pcount, int pstride, int work_cap, int ahead)
{
    constexpr int NG = kFT / GS;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ FHdr Hs[NG];
    const int grp = threadIdx.x / GS, tid = threadIdx.x % GS;
    const int pidx = blockIdx.x * NG + grp;
    if (pidx >= pcount) return;
    const int qa = ahead > 0 && pidx + ahead < pcount ? p0 + (pidx + ahead) * pstride : -1;
    fast_term<T, GS>(P, x, P.acc, maxbits, nvec, p0 + pidx * pstride, work_cap,
                     smraw + (size_t)grp * part_bytes(P, sizeof(T), work_cap), Hs[grp], tid, P, qa);
}

// Many problems in one launch: work item i = (problem, processing position);
// items come ordered by estimated cost over all problems.  Problem j's
// vectors, accumulators and exponents start at nvec * cs_prefix[j] (times
// the accumulator words for the accumulators) and j * nvec.  Every group's
// shared-memory partition is `part` bytes, the largest over the problems.
template <typename T, int GS>
__global__ void __launch_bounds__(kFT, sizeof(T) == 4 ? SG_F32_MINBLOCKS : SG_F64_MINBLOCKS)
    k_apply_fast_batch(const KParams *__restrict__ kps, const int2 *__restrict__ items, int count,
                       const double *__restrict__ x, unsigned long long *acc,
                       const long long *__restrict__ maxbits, const long long *__restrict__ cs_prefix, int nvec,
                       int part, int ahead)
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
    const int2 ia = ahead > 0 && pidx + ahead < count ? items[pidx + ahead] : make_int2(it.x, -1);
    fast_term<T, GS>(P, x + off, acc + off * fx::Acc<T>::words, maxbits + (size_t)it.x * nvec, nvec, it.y,
                     GS == kFT ? P.fast.work_cta : P.fast.work_warp, smraw + (size_t)grp * part, Hs[grp], tid,
                     kps[ia.x], ia.y);
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

// Term groups of kernel `kernel` resident on the whole device at `smem` bytes
// of dynamic shared memory per block: the look-ahead distance of its
// prefetches.  Answers are kept (a small table shared by all host threads)
// and first asked when the kernels are configured, so that a launch inside a
// stream capture normally finds its answer there.
struct ResidentEntry {
    const void *k;
    size_t smem;
    int dev, groups;
};
inline std::mutex g_resident_mu;
inline ResidentEntry g_resident[16];
inline int g_resident_next = 0;

template <typename K>
int resident_groups(K kernel, size_t smem, int groups_per_block)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const void *kp = reinterpret_cast<const void *>(kernel);
    {
        std::lock_guard<std::mutex> lk(g_resident_mu);
        for (const ResidentEntry &c : g_resident)
            if (c.k == kp && c.smem == smem && c.dev == dev) return c.groups;
    }
    int nb = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kFT, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    std::lock_guard<std::mutex> lk(g_resident_mu);
    g_resident[g_resident_next] = ResidentEntry{kp, smem, dev, nb * nsm * groups_per_block};
    g_resident_next = (g_resident_next + 1) % 16;
    return nb * nsm * groups_per_block;
}

template <typename T>
cudaError_t launch_t(const KParams &kp, const FastLaunch &a)
{
    const size_t rb = sizeof(T);
    const size_t smem_cta = part_bytes(kp, rb, kp.fast.work_cta);
    const size_t smem_warp = (size_t)(kFT / 32) * part_bytes(kp, rb, kp.fast.work_warp);
    if (a.configure) {
        cudaError_t e = set_smem_limit(k_apply_fast<T, kFT>, smem_cta);
        if (e == cudaSuccess) e = set_smem_limit(k_apply_fast<T, 32>, smem_warp);
        if (e == cudaSuccess) {
            resident_groups(k_apply_fast<T, kFT>, smem_cta, 1);
            resident_groups(k_apply_fast<T, 32>, smem_warp, kFT / 32);
        }
        return e;
    }
    const int nbig = kp.fast.n_big, nrest = (int)kp.n_terms - nbig;
    const int ahead_cta = nbig > 0 ? resident_groups(k_apply_fast<T, kFT>, smem_cta, 1) : 0;
    const int ahead_warp = nrest > 0 ? resident_groups(k_apply_fast<T, 32>, smem_warp, kFT / 32) : 0;
    if (kp.nparts > 1) {
        // one part of a term-sharded apply: positions p = part (mod nparts) of each form
        const int G = kp.nparts, r = kp.part;
        const int cb = nbig > r ? (nbig - r + G - 1) / G : 0;
        const int p1 = nbig + ((r - nbig) % G + G) % G;
        const int cw = (int)kp.n_terms > p1 ? ((int)kp.n_terms - p1 + G - 1) / G : 0;
        if (cb > 0)
            k_apply_fast<T, kFT><<<(unsigned)cb, kFT, smem_cta, a.stream>>>(kp, a.x, a.maxbits, a.nvec, r, cb, G,
                                                                          kp.fast.work_cta, ahead_cta);
        if (cw > 0)
            k_apply_fast<T, 32><<<(unsigned)((cw + kFT / 32 - 1) / (kFT / 32)), kFT, smem_warp, a.stream>>>(
                kp, a.x, a.maxbits, a.nvec, p1, cw, G, kp.fast.work_warp, ahead_warp);
        return cudaGetLastError();
    }
    if (nbig > 0)
        k_apply_fast<T, kFT><<<(unsigned)nbig, kFT, smem_cta, a.stream>>>(kp, a.x, a.maxbits, a.nvec, 0, nbig, 1,
                                                                        kp.fast.work_cta, ahead_cta);
    if (nrest > 0) {
        const unsigned blocks = (unsigned)((nrest + kFT / 32 - 1) / (kFT / 32));
        k_apply_fast<T, 32><<<blocks, kFT, smem_warp, a.stream>>>(kp, a.x, a.maxbits, a.nvec, nbig, nrest, 1,
                                                                kp.fast.work_warp, ahead_warp);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t batch_t(const FastBatchLaunch &a)
{
    constexpr int NG = kFT / 32;
    if (a.configure) {
        cudaError_t e = set_smem_limit(k_apply_fast_batch<T, kFT>, (size_t)a.part[0]);
        if (e == cudaSuccess) e = set_smem_limit(k_apply_fast_batch<T, 32>, (size_t)NG * a.part[1]);
        if (e == cudaSuccess) {
            resident_groups(k_apply_fast_batch<T, kFT>, (size_t)a.part[0], 1);
            resident_groups(k_apply_fast_batch<T, 32>, (size_t)NG * a.part[1], NG);
        }
        return e;
    }
    if (a.count[0] > 0)
        k_apply_fast_batch<T, kFT><<<(unsigned)a.count[0], kFT, (size_t)a.part[0], a.stream>>>(
            a.kps, a.items[0], a.count[0], a.x, a.acc, a.maxbits, a.cs_prefix, a.nvec, a.part[0],
            resident_groups(k_apply_fast_batch<T, kFT>, (size_t)a.part[0], 1));
    if (a.count[1] > 0)
        k_apply_fast_batch<T, 32><<<(unsigned)((a.count[1] + NG - 1) / NG), kFT, (size_t)NG * a.part[1], a.stream>>>(
            a.kps, a.items[1], a.count[1], a.x, a.acc, a.maxbits, a.cs_prefix, a.nvec, a.part[1],
            resident_groups(k_apply_fast_batch<T, 32>, (size_t)NG * a.part[1], NG));
    return cudaGetLastError();
}

}  // namespace

}  // namespace sg
