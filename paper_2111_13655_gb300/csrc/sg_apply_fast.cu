// Smolyak operator action, fast path (sm_103a): potentials whose monomials
// touch at most two modes (the Henon-Heiles family of Sec. 4, Eq. (18)).
//
// One thread block per Smolyak term, terms ordered most-expensive first.  The
// term operator (Alg. 1 of arXiv 2111.13655 with the grid operator split as
// described in build_fast_tables) is
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
#include <algorithm>
#include <cstdint>

#include "sg_fixed.cuh"
#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kFT = 128;   // threads per term block
constexpr int kMaxVB = 8;  // vectors per chunk

struct FHdr {
    int m, R, NB, NBo, grid, bad, coef;
    int s, vb, NBO, NBrest, NBIn, nslice, NGs;
    double c0;
    int mode[kMaxD], lev[kMaxD], nb[kMaxD], nq[kMaxD];  // by layout position
    int ostride[kMaxD];                                  // stride of a position inside its block (i or o)
    unsigned smag[kMaxD], bmag[kMaxD];                   // reciprocals of ostride and nb
    int oB[kMaxD], oBW[kMaxD], oH[kMaxD];                // shared-memory offsets of B, B^T W, H1
    int gstride[kMaxD];                                  // outer grid strides inside a slice
    unsigned gmag[kMaxD], qmag[kMaxD];                   // reciprocals of gstride and nq
    int bymode[kMaxD];                                   // positions sorted by mode
    int pos_of_mode[kMaxD], lev_of_mode[kMaxD];
    int npair, nind;
    int pa[kMaxPairs], pb[kMaxPairs], pg[kMaxPairs];     // active pairs: positions, G offset
    int ipos[kMaxPairs], ioffs[kMaxPairs];               // induced matrices: position, offset
    int uS[kMaxD];                                       // slice indices of the sliced positions
};

// floor(x / d) for x * d < 2^32, via a 32-bit reciprocal (mag = ceil(2^32 / d), d > 1)
__device__ __forceinline__ unsigned rmag(unsigned d) { return d <= 1 ? 0u : 0xFFFFFFFFu / d + 1u; }
__device__ __forceinline__ int fdiv(int x, int d, unsigned mag)
{
    return d == 1 ? x : (int)__umulhi((unsigned)x, mag);
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

template <typename T> struct FTab;
template <> struct FTab<double> {
    static __device__ const double *f(const KParams &P) { return P.fast.tabd; }
    static __device__ const double *t(const KParams &P) { return P.tabd; }
};
template <> struct FTab<float> {
    static __device__ const float *f(const KParams &P) { return P.fast.tabf; }
    static __device__ const float *t(const KParams &P) { return P.tabf; }
};

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-term set-up by warp 0: lane i looks at mode i, lane p at coupled pair p.
template <int NB1, int NQ1, int RMAX>
__device__ void fast_decode(const KParams &P, int t, int nvec, int work, FHdr &H)
{
    const FastParams &F = P.fast;
    const int Lp = P.L + 1, lane = threadIdx.x & 31;
    const uint8_t *lt = P.levels + (size_t)t * P.Dpad;
    int lev = 0, nb = 1, nq = 1;
    double c0 = 0.0;
    if (lane < P.D) {
        lev = lt[lane];
        const LevelInfo li = P.lvl[lane * Lp + lev];
        nb = li.nb; nq = li.nq;
        if (nb <= 1) c0 += F.sc[F.soff[lane * Lp + lev]];
        H.lev_of_mode[lane] = lev;
    }
    const bool active = lane < P.D && nb > 1;
    const bool lvl1 = active && nb == NB1 && nq == NQ1;
    const unsigned am = __ballot_sync(0xffffffffu, active);
    unsigned l1m = __ballot_sync(0xffffffffu, lvl1);
    unsigned im = 0;
    for (int r = 0; r < RMAX && l1m; r++) {  // the last RMAX level-1 modes become inner
        const int hi = 31 - __clz(l1m);
        im |= 1u << hi;
        l1m &= ~(1u << hi);
    }
    const unsigned om = am & ~im;
    const int R = __popc(im), m = __popc(am);
    const unsigned below = (1u << lane) - 1u;
    int pos = -1;
    if (active) pos = ((im >> lane) & 1u) ? __popc(im & below) : R + __popc(om & below);
    if (lane < P.D) H.pos_of_mode[lane] = pos;
    if (active) {
        H.mode[pos] = lane; H.lev[pos] = lev; H.nb[pos] = nb; H.nq[pos] = nq;
        H.bymode[__popc(am & below)] = pos;
    }
    __syncwarp();
    int nact = 0, nind = 0;
    for (int p0 = 0; p0 < F.npairs; p0 += 32) {
        const int p = p0 + lane;
        int a = 0, b = 0, pa = -1, pb = -1;
        if (p < F.npairs) {
            a = F.pair_modes[2 * p]; b = F.pair_modes[2 * p + 1];
            pa = H.pos_of_mode[a]; pb = H.pos_of_mode[b];
        }
        const bool isact = p < F.npairs && pa >= 0 && pb >= 0;
        const bool isind = p < F.npairs && ((pa >= 0) != (pb >= 0));
        const unsigned actm = __ballot_sync(0xffffffffu, isact), indm = __ballot_sync(0xffffffffu, isind);
        if (p < F.npairs) {
            const int la = H.lev_of_mode[a], lb = H.lev_of_mode[b];
            const int key = (p * Lp + la) * Lp + lb;
            if (isact) {
                const int q = nact + __popc(actm & below);
                H.pa[q] = pa; H.pb[q] = pb; H.pg[q] = F.goff[key];
            } else if (isind) {
                const int side = pa >= 0 ? 0 : 1;
                const int lact = side == 0 ? la : lb, lcol = side == 0 ? lb : la;
                const int q = nind + __popc(indm & below);
                H.ipos[q] = side == 0 ? pa : pb;
                H.ioffs[q] = F.ioff[((p * 2 + side) * Lp + lact) * Lp + lcol];
            } else {
                c0 += F.sc[F.spoff[key]];
            }
        }
        nact += __popc(actm);
        nind += __popc(indm);
    }
    c0 = warp_sum(c0);
    __syncwarp();
    if (lane != 0) return;
    H.c0 = c0 + F.c0const;
    H.coef = P.coefs[t];
    H.m = m; H.R = R;
    H.npair = nact; H.nind = nind;
    H.grid = nact > 0;
    H.bad = 0;
    int mat = 0, NB = 1, NBIn = 1;
    for (int j = 0; j < m; j++) {
        H.oB[j] = mat;  mat += H.nq[j] * H.nb[j];
        H.oBW[j] = mat; mat += H.nb[j] * H.nq[j];
        H.oH[j] = mat;  mat += H.nb[j] * H.nb[j];
        H.bmag[j] = rmag(H.nb[j]);
        H.qmag[j] = rmag(H.nq[j]);
        NB *= H.nb[j];
        if (j < R) NBIn *= H.nb[j];
    }
    if (mat > P.matcap || NB > P.maxnb) { H.bad = 1; return; }
    H.NB = NB; H.NBIn = NBIn; H.NBo = NB / NBIn;
    int st = 1;
    for (int j = R - 1; j >= 0; j--) { H.ostride[j] = st; H.smag[j] = rmag(st); st *= H.nb[j]; }
    st = 1;
    for (int j = m - 1; j >= R; j--) { H.ostride[j] = st; H.smag[j] = rmag(st); st *= H.nb[j]; }
    // vector chunk and slicing: X, Y (NB*vb each) + two grid buffers (stage*vb each)
    auto stage_of = [&](int s) {
        int64_t sz = NBIn;
        for (int j = R + s; j < m; j++) sz *= H.nq[j];
        return sz;
    };
    // slicing depth: the smallest that leaves room for a chunk of 4 vectors (2,
    // then 1, for very large terms).  It depends on the term only, so a
    // vector's arithmetic does not depend on how many vectors are applied
    // together.  The chunk is then the largest that fits at that depth.
    int sv = 0;
    if (H.grid) {
        sv = -1;
        for (int vt = 4; vt >= 1 && sv < 0; vt /= 2)
            for (int s = 0; s <= m - R && sv < 0; s++)
                if ((2 * (int64_t)NB + 2 * stage_of(s)) * vt <= work) sv = s;
        if (sv < 0) { H.bad = 2; return; }
    }
    if (2 * (int64_t)NB > work) { H.bad = 2; return; }
    const int64_t per_vec = 2 * (int64_t)NB + (H.grid ? 2 * stage_of(sv) : 0);
    int vb = nvec < kMaxVB ? nvec : kMaxVB;
    while (vb > 1 && per_vec * vb > work) vb--;
    H.vb = vb; H.s = sv;
    H.NBO = 1; H.nslice = 1;
    for (int j = R; j < R + sv; j++) { H.NBO *= H.nb[j]; H.nslice *= H.nq[j]; }
    H.NBrest = 1; H.NGs = 1;
    for (int j = R + sv; j < m; j++) { H.NBrest *= H.nb[j]; H.NGs *= H.nq[j]; }
    int gs = 1;
    for (int j = m - 1; j >= R + sv; j--) { H.gstride[j] = gs; H.gmag[j] = rmag(gs); gs *= H.nq[j]; }
}

// out[a][r][c] = sum_k M[r][k] in[a][k][c], matrix in registers, one fibre (a, c) per thread
template <typename T, int N, int RR>
__device__ __forceinline__ void fcontract_t(const T *__restrict__ in, T *__restrict__ out, int A, int C,
                                            const T *__restrict__ M)
{
    T mr[RR * N];
#pragma unroll
    for (int i = 0; i < RR * N; i++) mr[i] = M[i];
    const int total = A * C;
    const unsigned mag = rmag(C);
    for (int f = threadIdx.x; f < total; f += kFT) {
        const int a = fdiv(f, C, mag), c = f - a * C;
        const T *ip = in + a * N * C + c;
        T *op = out + a * RR * C + c;
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

template <typename T>
__device__ void fcontract_rt(const T *__restrict__ in, T *__restrict__ out, int A, int n, int r, int C,
                             const T *__restrict__ M)
{
    const int total = A * r * C;
    for (int e = threadIdx.x; e < total; e += kFT) {
        const int c = e % C, tq = e / C, rr = tq % r, a = tq / r;
        const T *ip = in + (a * n) * C + c;
        const T *mp = M + rr * n;
        T acc = T(0);
        for (int k = 0; k < n; k++) acc += mp[k] * ip[k * C];
        out[e] = acc;
    }
}

template <typename T>
__device__ void fcontract(const T *in, T *out, int A, int n, int r, int C, const T *M)
{
#define SG_FC(NN, RRR) case (NN) * 64 + (RRR): fcontract_t<T, NN, RRR>(in, out, A, C, M); return;
    switch (n * 64 + r) {
        SG_FC(2, 2) SG_FC(2, 3) SG_FC(3, 2) SG_FC(3, 3) SG_FC(3, 4) SG_FC(4, 3) SG_FC(4, 4) SG_FC(4, 5)
        SG_FC(5, 4) SG_FC(5, 5) SG_FC(5, 6) SG_FC(6, 5) SG_FC(6, 6) SG_FC(6, 7) SG_FC(7, 6)
        default: fcontract_rt(in, out, A, n, r, C, M); return;
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
template <typename T, int R, int NB1, int NQ1, bool UNI>
__device__ void reg_phase(const KParams &P, const FHdr &H, const T *mats, T *Z, const int vb)
{
    constexpr int NBI = cpow(NB1, R), NGI = cpow(NQ1, R), SZ = NGI;
    constexpr int RA = R > 0 ? R : 1;
    constexpr int NM = UNI ? 1 : RA;
    const T *G = FTab<T>::f(P);
    T Bm[NM][NQ1 * NB1], BWm[NM][NB1 * NQ1];
#pragma unroll
    for (int b = 0; b < NM; b++)
#pragma unroll
        for (int e = 0; e < NQ1 * NB1; e++) {
            Bm[b][e] = R > 0 ? mats[H.oB[b] + e] : T(0);
            BWm[b][e] = R > 0 ? mats[H.oBW[b] + e] : T(0);
        }
    const int s0 = R + H.s, NGs = H.NGs;
    for (int g = threadIdx.x; g < NGs; g += kFT) {
        // potential on the inner grid of this outer point, accumulated pair by pair
        T V[SZ];
#pragma unroll
        for (int gi = 0; gi < NGI; gi++) V[gi] = T(0);
        T vO = T(0);
        for (int p = 0; p < H.npair; p++) {
            const int A = H.pa[p], B = H.pb[p];
            auto uo = [&](int j) {
                if (j < s0) return H.uS[j];
                const int q = fdiv(g, H.gstride[j], H.gmag[j]);
                return q - fdiv(q, H.nq[j], H.qmag[j]) * H.nq[j];
            };
            if (A >= R && B >= R) {
                vO += G[H.pg[p] + uo(A) * H.nq[B] + uo(B)];
            } else if (A >= R) {  // B inner: row u_A of G[u_A][u_B]
                const T *row = G + H.pg[p] + uo(A) * NQ1;
                T rv[NQ1];
#pragma unroll
                for (int u = 0; u < NQ1; u++) rv[u] = row[u];
#pragma unroll
                for (int b = 0; b < R; b++)
                    if (b == B)
#pragma unroll
                        for (int gi = 0; gi < NGI; gi++) V[gi] += rv[(gi / cpow(NQ1, R - 1 - b)) % NQ1];
            } else if (B >= R) {  // A inner: column u_B of G[u_A][u_B]
                const int ub = uo(B), nqb = H.nq[B];
                T cv[NQ1];
#pragma unroll
                for (int u = 0; u < NQ1; u++) cv[u] = G[H.pg[p] + u * nqb + ub];
#pragma unroll
                for (int b = 0; b < R; b++)
                    if (b == A)
#pragma unroll
                        for (int gi = 0; gi < NGI; gi++) V[gi] += cv[(gi / cpow(NQ1, R - 1 - b)) % NQ1];
            } else {              // both inner (inner positions follow mode order: A < B)
#pragma unroll
                for (int q0 = 0; q0 < R; q0++)
#pragma unroll
                    for (int q1 = q0 + 1; q1 < R; q1++)
                        if (q0 == A && q1 == B)
#pragma unroll
                            for (int gi = 0; gi < NGI; gi++)
                                V[gi] += G[H.pg[p] + ((gi / cpow(NQ1, R - 1 - q0)) % NQ1) * NQ1 +
                                           (gi / cpow(NQ1, R - 1 - q1)) % NQ1];
            }
        }
#pragma unroll
        for (int gi = 0; gi < NGI; gi++) V[gi] += vO;
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

template <typename T, int NB1, int NQ1, int RMAX, bool UNI>
__global__ void __launch_bounds__(kFT, sizeof(T) == 4 ? 3 : 2)
    k_apply_fast(const KParams P, const double *__restrict__ x, const long long *__restrict__ maxbits, int nvec)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ FHdr H;
    const int tid = threadIdx.x;
    T *mats = reinterpret_cast<T *>(smraw);
    T *WoF = mats + P.matcap;
    T *WoB = WoF + P.maxnb;
    int *rk = reinterpret_cast<int *>(WoB + P.maxnb);
    T *work = reinterpret_cast<T *>(rk + P.maxnb + (P.maxnb & 1));

    const int t = P.order[blockIdx.x];
    if (tid < 32) fast_decode<NB1, NQ1, RMAX>(P, t, nvec, P.cap, H);
    __syncthreads();
    if (H.bad) {
        if (tid == 0 && P.err) atomicCAS(P.err, 0, 110 + H.bad);
        return;
    }
    const T *tab = FTab<T>::t(P);
    const T *ftab = FTab<T>::f(P);
    const int m = H.m, R = H.R, NB = H.NB, NBo = H.NBo;
    const int Lp = P.L + 1;

    // per-position matrices: B, B^T W (grid part) and H1 = base + induced
    for (int j = 0; j < m; j++) {
        const LevelInfo li = P.lvl[H.mode[j] * Lp + H.lev[j]];
        if (H.grid)
            for (int e = tid; e < li.nb * li.nq; e += kFT) {
                mats[H.oB[j] + e] = tab[li.offB + e];
                mats[H.oBW[j] + e] = tab[li.offBW + e];
            }
        const int h1 = P.fast.h1off[H.mode[j] * Lp + H.lev[j]];
        for (int e = tid; e < li.nb * li.nb; e += kFT) {
            T hv = ftab[h1 + e];
            for (int q = 0; q < H.nind; q++)
                if (H.ipos[q] == j) hv += ftab[H.ioffs[q] + e];
            mats[H.oH[j] + e] = hv;
        }
    }
    // compact index of element e = (i, o), rank accumulated over positions in mode order
    for (int e = tid; e < NB; e += kFT) {
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
        rk[e] = r;
    }
    __syncthreads();

    for (int v0 = 0; v0 < nvec; v0 += H.vb) {
        const int vb = min(H.vb, nvec - v0);
        T *X = work, *Y = work + NB * vb, *bufA = Y + NB * vb;
        // gather: X[i][v][o]
        for (int e = tid; e < NB; e += kFT) {
            const int i = e / NBo, o = e - i * NBo;
            for (int v = 0; v < vb; v++)
                X[(i * vb + v) * NBo + o] = (T)__ldg(x + (size_t)(v0 + v) * P.n_cs + rk[e]);
        }
        __syncthreads();
        // basis part: Y = c0 X + sum_j H1_j x_j X, all vectors of the chunk per element
        for (int e = tid; e < NB; e += kFT) {
            const int i = e / NBo, o = e - i * NBo;
            const int base = i * vb * NBo + o;
            T acc[kMaxVB];
#pragma unroll
            for (int v = 0; v < kMaxVB; v++) acc[v] = v < vb ? (T)H.c0 * X[base + v * NBo] : T(0);
            for (int j = 0; j < m; j++) {
                const int src = j < R ? i : o;
                const int q = fdiv(src, H.ostride[j], H.smag[j]);
                const int nbj = H.nb[j], kj = q - fdiv(q, nbj, H.bmag[j]) * nbj;
                const int st = j < R ? H.ostride[j] * vb * NBo : H.ostride[j];
                const T *xp = X + base - kj * st;
                const T *Hr = mats + H.oH[j] + kj * nbj;
                for (int kp = 0; kp < nbj; kp++) {
                    const T hv = Hr[kp];
#pragma unroll
                    for (int v = 0; v < kMaxVB; v++)
                        if (v < vb) acc[v] = fma_t(hv, xp[kp * st + v * NBo], acc[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < kMaxVB; v++)
                if (v < vb) Y[base + v * NBo] = acc[v];
        }
        __syncthreads();
        if (H.grid) {
            const int p0 = R + H.s;
            const int NBIv = H.NBIn * vb;
            T *bufB = bufA + (size_t)H.NBIn * H.NGs * vb;
            for (int sl = 0; sl < H.nslice; sl++) {
                T *cur, *oth, *spare;
                if (H.s > 0) {
                    if (tid == 0) {
                        int rem = sl;
                        for (int j = p0 - 1; j >= R; j--) { H.uS[j] = rem % H.nq[j]; rem /= H.nq[j]; }
                    }
                    __syncthreads();
                    for (int ko = tid; ko < H.NBO; ko += kFT) {
                        int rem = ko;
                        T wf = T(1), wb = T(1);
                        for (int j = p0 - 1; j >= R; j--) {
                            const int kj = rem % H.nb[j];
                            rem /= H.nb[j];
                            wf *= mats[H.oB[j] + H.uS[j] * H.nb[j] + kj];
                            wb *= mats[H.oBW[j] + kj * H.nq[j] + H.uS[j]];
                        }
                        WoF[ko] = wf; WoB[ko] = wb;
                    }
                    __syncthreads();
                    // Xs[iv][rest] = sum_ko WoF[ko] X[iv][ko][rest]
                    for (int e = tid; e < NBIv * H.NBrest; e += kFT) {
                        const int iv = e / H.NBrest, rr = e - iv * H.NBrest;
                        const T *xp = X + (size_t)iv * NBo + rr;
                        T acc = T(0);
                        for (int ko = 0; ko < H.NBO; ko++) acc += WoF[ko] * xp[ko * H.NBrest];
                        bufA[e] = acc;
                    }
                    __syncthreads();
                    cur = bufA; oth = bufB; spare = bufA;
                } else {
                    cur = X; oth = bufA; spare = bufB;  // X is not needed after the basis part
                }
                // outer basis -> grid (ping-pong between the two grid buffers)
                int A = NBIv;
                for (int j = p0; j < m; j++) {
                    int C = 1;
                    for (int i2 = j + 1; i2 < m; i2++) C *= H.nb[i2];
                    fcontract(cur, oth, A, H.nb[j], H.nq[j], C, mats + H.oB[j]);
                    A *= H.nq[j];
                    T *freed = (cur == X) ? spare : cur;
                    cur = oth; oth = freed;
                    __syncthreads();
                }
                if (cur == X) oth = bufA;
                // inner slots and potential, in registers
                switch (R) {
                    case 0: reg_phase<T, 0, NB1, NQ1, UNI>(P, H, mats, cur, vb); break;
                    case 1: if constexpr (RMAX >= 1) reg_phase<T, 1, NB1, NQ1, UNI>(P, H, mats, cur, vb); break;
                    case 2: if constexpr (RMAX >= 2) reg_phase<T, 2, NB1, NQ1, UNI>(P, H, mats, cur, vb); break;
                    case 3: if constexpr (RMAX >= 3) reg_phase<T, 3, NB1, NQ1, UNI>(P, H, mats, cur, vb); break;
                    default: break;
                }
                __syncthreads();
                // outer grid -> basis, reverse order
                for (int j = m - 1; j >= p0; j--) {
                    int Aj = NBIv, C = 1;
                    for (int i2 = p0; i2 < j; i2++) Aj *= H.nq[i2];
                    for (int i2 = j + 1; i2 < m; i2++) C *= H.nb[i2];
                    fcontract(cur, oth, Aj, H.nq[j], H.nb[j], C, mats + H.oBW[j]);
                    T *tp = cur; cur = oth; oth = tp;
                    __syncthreads();
                }
                // Y[iv][ko][rest] += WoB[ko] cur[iv][rest]
                if (H.s > 0) {
                    for (int e = tid; e < NB * vb; e += kFT) {
                        const int rr = e % H.NBrest, t2 = e / H.NBrest, ko = t2 % H.NBO, iv = t2 / H.NBO;
                        Y[e] += WoB[ko] * cur[iv * H.NBrest + rr];
                    }
                } else {
                    for (int e = tid; e < NB * vb; e += kFT) Y[e] += cur[e];
                }
                __syncthreads();
            }
        }
        // exact compress-add of D_l * y_l
        for (int e = tid; e < NB; e += kFT) {
            const int i = e / NBo, o = e - i * NBo;
            const int r = rk[e];
            for (int v = 0; v < vb; v++) {
                unsigned long long *acc = P.acc + ((size_t)(v0 + v) * P.n_cs + r) * kAccDigits;
                fx::fx_add_real(acc, Y[(i * vb + v) * NBo + o], H.coef, fx::lsb_exponent(maxbits[v0 + v]),
                                P.err);
            }
        }
        __syncthreads();
    }
}

template <typename T, int NB1, int NQ1, int RMAX, bool UNI>
cudaError_t launch_t(const KParams &kp, const double *x, int nvec, const long long *maxbits,
                     size_t smem, cudaStream_t stream, bool configure)
{
    if (configure)
        return cudaFuncSetAttribute(k_apply_fast<T, NB1, NQ1, RMAX, UNI>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_apply_fast<T, NB1, NQ1, RMAX, UNI><<<(unsigned)kp.n_terms, kFT, smem, stream>>>(kp, x, maxbits, nvec);
    return cudaGetLastError();
}

template <typename T, bool UNI>
cudaError_t dispatch_u(const KParams &kp, const double *x, int nvec, const long long *maxbits, size_t smem,
                       cudaStream_t stream, bool configure)
{
    constexpr int RM = sizeof(T) == 4 ? 3 : 1;
    const int nb1 = kp.fast.nb1, nq1 = kp.fast.nq1;
    if (nb1 == 2 && nq1 == 3) return launch_t<T, 2, 3, RM, UNI>(kp, x, nvec, maxbits, smem, stream, configure);
    if (nb1 == 2 && nq1 == 2) return launch_t<T, 2, 2, RM, UNI>(kp, x, nvec, maxbits, smem, stream, configure);
    if (nb1 == 3 && nq1 == 3)
        return launch_t<T, 3, 3, (RM > 2 ? 2 : RM), UNI>(kp, x, nvec, maxbits, smem, stream, configure);
    return launch_t<T, 1, 1, 0, UNI>(kp, x, nvec, maxbits, smem, stream, configure);
}

template <typename T>
cudaError_t dispatch(const KParams &kp, const double *x, int nvec, const long long *maxbits, size_t smem,
                     cudaStream_t stream, bool configure)
{
    return kp.fast.uni1 ? dispatch_u<T, true>(kp, x, nvec, maxbits, smem, stream, configure)
                        : dispatch_u<T, false>(kp, x, nvec, maxbits, smem, stream, configure);
}

}  // namespace

size_t fast_smem_bytes(const KParams &kp, bool fp32)
{
    const size_t rb = fp32 ? 4 : 8;
    return rb * ((size_t)kp.matcap + 2 * (size_t)kp.maxnb + (size_t)kp.cap) +
           4 * (size_t)(kp.maxnb + (kp.maxnb & 1));
}

cudaError_t configure_fast_kernels(const KParams &kp, bool fp32)
{
    const size_t smem = fast_smem_bytes(kp, fp32);
    return fp32 ? dispatch<float>(kp, nullptr, 0, nullptr, smem, 0, true)
                : dispatch<double>(kp, nullptr, 0, nullptr, smem, 0, true);
}

cudaError_t launch_apply_fast(const KParams &kp, bool fp32, const double *x, int nvec,
                              const long long *maxbits, cudaStream_t stream)
{
    if (kp.n_terms == 0) return cudaSuccess;
    const size_t smem = fast_smem_bytes(kp, fp32);
    return fp32 ? dispatch<float>(kp, x, nvec, maxbits, smem, stream, false)
                : dispatch<double>(kp, x, nvec, maxbits, smem, stream, false);
}

}  // namespace sg
