// Smolyak operator action, fast path (sm_103a): potentials whose monomials
// touch at most two modes (the Henon-Heiles family of Sec. 4, Eq. (18)).
//
// One thread block per Smolyak term, terms ordered most-expensive first.  The
// term operator (Alg. 1 of arXiv 2111.13655 with the grid operator split as
// described in build_fast_tables) is
//     y_l = c0 x_l + sum_j H1_j x_l + (x B^T W) diag(V_l) (x B) x_l,
// V_l(u) = sum over the term's active coupled pairs of G_p(u_a, u_b).
// The basis->grid (Eq. (15)) and grid->basis (Eq. (14)) transfers run mode by
// mode.  Layout of a term tensor: up to R "inner" slots of level 1 are the
// slowest positions, the other ("outer") slots follow in mode order.  Outer
// slots are contracted breadth-first in shared memory with the 1D matrix held
// in registers; the inner slots, the potential and their back transfer run in
// registers, one outer grid point per thread.  The compress-add of D_l * y_l
// into the compact result is the exact fixed-point sum of sg_apply.cu.
#include <algorithm>
#include <cstdint>

#include "sg_fixed.cuh"
#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kFT = 128;  // threads per term block

struct FHdr {
    int m, R, nO, NB, grid, bad, coef;
    int s, NBO, NBrest, NBIn, nslice, NGs;
    double c0;
    int mode[kMaxD], lev[kMaxD], nb[kMaxD], nq[kMaxD];  // by layout position
    int stride[kMaxD];                                   // basis strides (last position fastest)
    unsigned smag[kMaxD], bmag[kMaxD];                   // reciprocals of stride and nb
    int oB[kMaxD], oBW[kMaxD], oH[kMaxD];                // shared-memory offsets of B, B^T W, H1
    int gstride[kMaxD];                                  // outer grid strides inside a slice
    unsigned gmag[kMaxD], qmag[kMaxD];                   // reciprocals of gstride and nq
    int bymode[kMaxD];                                   // positions sorted by mode
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

template <typename T> struct FTab;
template <> struct FTab<double> {
    static __device__ const double *f(const KParams &P) { return P.fast.tabd; }
    static __device__ const double *t(const KParams &P) { return P.tabd; }
};
template <> struct FTab<float> {
    static __device__ const float *f(const KParams &P) { return P.fast.tabf; }
    static __device__ const float *t(const KParams &P) { return P.tabf; }
};

// Serial per-term set-up (thread 0).
template <int NB1, int NQ1, int RMAX>
__device__ void fast_decode(const KParams &P, int t, FHdr &H)
{
    const FastParams &F = P.fast;
    const int Lp = P.L + 1;
    const uint8_t *lt = P.levels + (size_t)t * P.Dpad;
    H.bad = 0;
    H.coef = P.coefs[t];
    // active modes in mode order; the last <= RMAX level-1 ones become inner
    int act[kMaxD], na = 0, pos_of_mode[kMaxD];
    double c0 = F.c0const;
    for (int i = 0; i < P.D; i++) {
        const LevelInfo li = P.lvl[i * Lp + lt[i]];
        pos_of_mode[i] = -1;
        if (li.nb > 1) act[na++] = i;
        else c0 += F.sc[F.soff[i * Lp + lt[i]]];
    }
    int R = 0;
    bool inner[kMaxD];
    for (int a = 0; a < na; a++) inner[a] = false;
    if (RMAX > 0)
        for (int a = na - 1; a >= 0 && R < RMAX; a--) {
            const LevelInfo li = P.lvl[act[a] * Lp + lt[act[a]]];
            if (li.nb == NB1 && li.nq == NQ1) { inner[a] = true; R++; }
        }
    H.m = na; H.R = R; H.nO = na - R;
    int pos = 0;
    for (int a = 0; a < na; a++) if (inner[a]) pos_of_mode[act[a]] = pos++;
    for (int a = 0; a < na; a++) if (!inner[a]) pos_of_mode[act[a]] = pos++;
    int mat = 0;
    H.NB = 1;
    for (int a = 0; a < na; a++) {
        const int i = act[a], j = pos_of_mode[i];
        const LevelInfo li = P.lvl[i * Lp + lt[i]];
        H.mode[j] = i; H.lev[j] = lt[i]; H.nb[j] = li.nb; H.nq[j] = li.nq;
        H.bymode[a] = j;
        H.NB *= li.nb;
    }
    for (int j = 0; j < na; j++) {
        H.oB[j] = mat;  mat += H.nq[j] * H.nb[j];
        H.oBW[j] = mat; mat += H.nb[j] * H.nq[j];
        H.oH[j] = mat;  mat += H.nb[j] * H.nb[j];
        H.bmag[j] = rmag(H.nb[j]);
        H.qmag[j] = rmag(H.nq[j]);
    }
    if (mat > P.matcap || H.NB > P.maxnb) { H.bad = 1; return; }
    int st = 1;
    for (int j = na - 1; j >= 0; j--) { H.stride[j] = st; H.smag[j] = rmag(st); st *= H.nb[j]; }
    // pairs: active (both modes transformed), induced (one side collapsed), scalar
    H.npair = 0; H.nind = 0;
    for (int p = 0; p < F.npairs; p++) {
        const int a = F.pair_modes[2 * p], b = F.pair_modes[2 * p + 1];
        const int pa = pos_of_mode[a], pb = pos_of_mode[b];
        const int key = (p * Lp + lt[a]) * Lp + lt[b];
        if (lt[a] + lt[b] > P.L) { H.bad = 4; return; }
        if (pa >= 0 && pb >= 0) {
            H.pa[H.npair] = pa; H.pb[H.npair] = pb; H.pg[H.npair] = F.goff[key]; H.npair++;
        } else if (pa >= 0 || pb >= 0) {
            const int side = pa >= 0 ? 0 : 1;
            const int la = side == 0 ? lt[a] : lt[b], lc = side == 0 ? lt[b] : lt[a];
            H.ipos[H.nind] = side == 0 ? pa : pb;
            H.ioffs[H.nind] = F.ioff[((p * 2 + side) * Lp + la) * Lp + lc];
            H.nind++;
        } else {
            c0 += F.sc[F.spoff[key]];
        }
    }
    H.c0 = c0;
    H.grid = H.npair > 0;
    // slicing over the leading outer positions R .. R+s-1
    int pitch_in = 1;
    for (int j = 0; j < R; j++) pitch_in *= H.nb[j];
    H.NBIn = pitch_in;
    H.s = 0;
    if (H.grid) {
        for (int s = 0; s <= H.nO; s++) {
            int64_t stage = pitch_in;
            for (int j = R + s; j < na; j++) stage *= H.nq[j];
            H.s = s;
            if (stage <= P.cap) break;
        }
        int64_t stage = pitch_in;
        for (int j = R + H.s; j < na; j++) stage *= H.nq[j];
        if (stage > P.cap) { H.bad = 2; return; }
    }
    H.NBO = 1; H.nslice = 1;
    for (int j = R; j < R + H.s; j++) { H.NBO *= H.nb[j]; H.nslice *= H.nq[j]; }
    H.NBrest = 1; H.NGs = 1;
    for (int j = R + H.s; j < na; j++) { H.NBrest *= H.nb[j]; H.NGs *= H.nq[j]; }
    int gs = 1;
    for (int j = na - 1; j >= R + H.s; j--) { H.gstride[j] = gs; H.gmag[j] = rmag(gs); gs *= H.nq[j]; }
}

// out[a][r][c] = sum_k M[r][k] in[a][k][c], matrix in registers, one fibre (a, c) per thread
template <typename T, int N, int RR>
__device__ __forceinline__ void fcontract_t(const T *__restrict__ in, T *__restrict__ out, int A, int C,
                                            const T *__restrict__ M)
{
    T m[RR * N];
#pragma unroll
    for (int i = 0; i < RR * N; i++) m[i] = M[i];
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
            for (int k = 0; k < N; k++) acc += m[r * N + k] * xv[k];
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
        SG_FC(5, 4) SG_FC(5, 5) SG_FC(5, 6) SG_FC(6, 5) SG_FC(6, 6) SG_FC(6, 7) SG_FC(7, 6) SG_FC(7, 7)
        SG_FC(7, 8) SG_FC(8, 7) SG_FC(8, 8)
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
                for (int k = 0; k < N; k++) acc += M[u * N + k] * in[(p * N + k) * Q + q];
                out[(p * RR + u) * Q + q] = acc;
            }
}

// Register phase: for every outer grid point of the slice, the inner slots
// basis -> grid, times the potential, grid -> basis.  Z[i][g] in place.
template <typename T, int R, int NB1, int NQ1>
__device__ void reg_phase(const KParams &P, const FHdr &H, const T *mats, T *Z)
{
    constexpr int NBI = cpow(NB1, R), NGI = cpow(NQ1, R), SZ = NGI;
    constexpr int RA = R > 0 ? R : 1;
    constexpr int NIP = R * (R - 1) / 2 > 0 ? R * (R - 1) / 2 : 1;
    const T *G = FTab<T>::f(P);
    T Bm[RA][NQ1 * NB1], BWm[RA][NB1 * NQ1];
#pragma unroll
    for (int b = 0; b < R; b++)
#pragma unroll
        for (int e = 0; e < NQ1 * NB1; e++) { Bm[b][e] = mats[H.oB[b] + e]; BWm[b][e] = mats[H.oBW[b] + e]; }
    // inner-inner coupling tables (pair (b0,b1) with b0 < b1, mode order = position order)
    T Gin[NIP][NQ1 * NQ1];
    bool hasin[NIP];
#pragma unroll
    for (int q = 0; q < NIP; q++) hasin[q] = false;
    for (int p = 0; p < H.npair; p++) {
        if (H.pa[p] < R && H.pb[p] < R) {
            const int b0 = min(H.pa[p], H.pb[p]), b1 = max(H.pa[p], H.pb[p]);
            const bool tr = H.pa[p] > H.pb[p];
#pragma unroll
            for (int q0 = 0, q = 0; q0 < R; q0++)
#pragma unroll
                for (int q1 = q0 + 1; q1 < R; q1++, q++)
                    if (q0 == b0 && q1 == b1) {
                        if (!hasin[q])
#pragma unroll
                            for (int e = 0; e < NQ1 * NQ1; e++) Gin[q][e] = T(0);
                        hasin[q] = true;
#pragma unroll
                        for (int u0 = 0; u0 < NQ1; u0++)
#pragma unroll
                            for (int u1 = 0; u1 < NQ1; u1++)
                                Gin[q][u0 * NQ1 + u1] += tr ? G[H.pg[p] + u1 * NQ1 + u0] : G[H.pg[p] + u0 * NQ1 + u1];
                    }
        }
    }
    const int s0 = R + H.s;
    for (int g = threadIdx.x; g < H.NGs; g += kFT) {
        // potential parts that depend on the outer grid point
        T vO = T(0);
        T h[RA][NQ1];
#pragma unroll
        for (int b = 0; b < RA; b++)
#pragma unroll
            for (int u = 0; u < NQ1; u++) h[b][u] = T(0);
        for (int p = 0; p < H.npair; p++) {
            const int A = H.pa[p], B = H.pb[p];
            if (A < R && B < R) continue;
            auto uo = [&](int j) {
                if (j < s0) return H.uS[j];
                const int q = fdiv(g, H.gstride[j], H.gmag[j]);
                return q - fdiv(q, H.nq[j], H.qmag[j]) * H.nq[j];
            };
            if (A >= R && B >= R) {
                vO += G[H.pg[p] + uo(A) * H.nq[B] + uo(B)];
            } else if (A >= R) {            // B inner: row u_A of G[u_A][u_B]
                const T *row = G + H.pg[p] + uo(A) * NQ1;
#pragma unroll
                for (int b = 0; b < R; b++)
                    if (b == B)
#pragma unroll
                        for (int u = 0; u < NQ1; u++) h[b][u] += row[u];
            } else {                         // A inner: column u_B of G[u_A][u_B]
                const int ub = uo(B), nqb = H.nq[B];
#pragma unroll
                for (int b = 0; b < R; b++)
                    if (b == A)
#pragma unroll
                        for (int u = 0; u < NQ1; u++) h[b][u] += G[H.pg[p] + u * nqb + ub];
            }
        }
        T va[SZ], vb[SZ];
#pragma unroll
        for (int i = 0; i < NBI; i++) va[i] = Z[i * H.NGs + g];
        // inner basis -> grid (inner position 0 slowest)
        if constexpr (R == 1) {
            rstage<T, SZ, 1, NB1, NQ1, 1>(va, vb, Bm[0]);
        } else if constexpr (R == 2) {
            rstage<T, SZ, 1, NB1, NQ1, NB1>(va, vb, Bm[0]);
            rstage<T, SZ, NQ1, NB1, NQ1, 1>(vb, va, Bm[1]);
        } else if constexpr (R == 3) {
            rstage<T, SZ, 1, NB1, NQ1, NB1 * NB1>(va, vb, Bm[0]);
            rstage<T, SZ, NQ1, NB1, NQ1, NB1>(vb, va, Bm[1]);
            rstage<T, SZ, NQ1 * NQ1, NB1, NQ1, 1>(va, vb, Bm[2]);
        }
        // potential on the inner grid
        if constexpr (R > 0) {
            T (&gv)[SZ] = (R == 2) ? va : vb;
#pragma unroll
            for (int gi = 0; gi < NGI; gi++) {
                T V = vO;
#pragma unroll
                for (int b = 0; b < R; b++) V += h[b][(gi / cpow(NQ1, R - 1 - b)) % NQ1];
#pragma unroll
                for (int q0 = 0, q = 0; q0 < R; q0++)
#pragma unroll
                    for (int q1 = q0 + 1; q1 < R; q1++, q++)
                        if (hasin[q])
                            V += Gin[q][((gi / cpow(NQ1, R - 1 - q0)) % NQ1) * NQ1 +
                                        (gi / cpow(NQ1, R - 1 - q1)) % NQ1];
                gv[gi] *= V;
            }
        }
        // inner grid -> basis
        if constexpr (R == 0) {
            va[0] *= vO;
        } else if constexpr (R == 1) {
            rstage<T, SZ, 1, NQ1, NB1, 1>(vb, va, BWm[0]);
        } else if constexpr (R == 2) {
            rstage<T, SZ, NQ1, NQ1, NB1, 1>(va, vb, BWm[1]);
            rstage<T, SZ, 1, NQ1, NB1, NB1>(vb, va, BWm[0]);
        } else if constexpr (R == 3) {
            rstage<T, SZ, NQ1 * NQ1, NQ1, NB1, 1>(vb, va, BWm[2]);
            rstage<T, SZ, NQ1, NQ1, NB1, NB1>(va, vb, BWm[1]);
            rstage<T, SZ, 1, NQ1, NB1, NB1 * NB1>(vb, va, BWm[0]);
        }
#pragma unroll
        for (int i = 0; i < NBI; i++) Z[i * H.NGs + g] = va[i];
    }
}

template <typename T>
__device__ __forceinline__ void fx_add_T(unsigned long long *acc, T r, int coef, int E, int *err)
{
    fx::fx_add_real(acc, r, coef, E, err);
}

template <typename T, int NB1, int NQ1, int RMAX>
__global__ void __launch_bounds__(kFT) k_apply_fast(const KParams P, const double *__restrict__ x,
                                                    const long long *__restrict__ maxbits, int nvec)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ FHdr H;
    const int tid = threadIdx.x;
    T *mats = reinterpret_cast<T *>(smraw);
    T *X = mats + P.matcap;
    T *Y = X + P.maxnb;
    T *WoF = Y + P.maxnb;
    T *WoB = WoF + P.maxnb;
    T *bufA = WoB + P.maxnb;
    T *bufB = bufA + P.cap;
    int *rk = reinterpret_cast<int *>(bufB + P.cap);

    const int t = P.order[blockIdx.x];
    if (tid == 0) fast_decode<NB1, NQ1, RMAX>(P, t, H);
    __syncthreads();
    if (H.bad) {
        if (tid == 0 && P.err) atomicCAS(P.err, 0, 110 + H.bad);
        return;
    }
    const T *tab = FTab<T>::t(P);
    const T *ftab = FTab<T>::f(P);
    const int m = H.m, R = H.R;
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
            T h = ftab[h1 + e];
            for (int q = 0; q < H.nind; q++)
                if (H.ipos[q] == j) h += ftab[H.ioffs[q] + e];
            mats[H.oH[j] + e] = h;
        }
    }
    // compact indices (rank accumulates over positions in mode order)
    for (int e = tid; e < H.NB; e += kFT) {
        int r = 0, s = 0;
        for (int a = 0; a < m; a++) {
            const int j = H.bymode[a];
            const int q = fdiv(e, H.stride[j], H.smag[j]);
            const int kj = q - fdiv(q, H.nb[j], H.bmag[j]) * H.nb[j];
            const int i = H.mode[j];
            r += P.rank_tab[(i * Lp + s) * P.kw + kj];
            s += P.lmin_tab[i * P.kw + kj];
        }
        rk[e] = r;
    }
    __syncthreads();

    for (int v = 0; v < nvec; v++) {
        const double *xv = x + (size_t)v * P.n_cs;
        unsigned long long *accv = P.acc + (size_t)v * P.n_cs * kAccDigits;
        const int E = fx::lsb_exponent(maxbits[v]);
        for (int e = tid; e < H.NB; e += kFT) X[e] = (T)__ldg(xv + rk[e]);
        __syncthreads();
        // basis part: c0 x + sum_j H1_j x_j
        for (int e = tid; e < H.NB; e += kFT) {
            T acc = (T)H.c0 * X[e];
            for (int j = 0; j < m; j++) {
                const int q = fdiv(e, H.stride[j], H.smag[j]);
                const int nbj = H.nb[j];
                const int kj = q - fdiv(q, nbj, H.bmag[j]) * nbj;
                const int base = e - kj * H.stride[j];
                const T *Hr = mats + H.oH[j] + kj * nbj;
                for (int kp = 0; kp < nbj; kp++) acc += Hr[kp] * X[base + kp * H.stride[j]];
            }
            Y[e] = acc;
        }
        __syncthreads();
        if (H.grid) {
            const int s = H.s, p0 = R + s;
            for (int sl = 0; sl < H.nslice; sl++) {
                if (tid == 0) {
                    int rem = sl;
                    for (int j = p0 - 1; j >= R; j--) { H.uS[j] = rem % H.nq[j]; rem /= H.nq[j]; }
                }
                __syncthreads();
                // slice weights over the sliced positions R..p0-1
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
                // Xs[i][rest] = sum_ko WoF[ko] X[i][ko][rest]
                const int nXs = H.NBIn * H.NBrest;
                for (int e = tid; e < nXs; e += kFT) {
                    const int i = e / H.NBrest, rr = e - i * H.NBrest;
                    const T *xp = X + (size_t)i * H.NBO * H.NBrest + rr;
                    T acc = T(0);
                    for (int ko = 0; ko < H.NBO; ko++) acc += WoF[ko] * xp[ko * H.NBrest];
                    bufA[e] = acc;
                }
                __syncthreads();
                T *cur = bufA, *oth = bufB;
                // outer basis -> grid
                int A = H.NBIn;
                for (int j = p0; j < m; j++) {
                    int C = 1;
                    for (int i = j + 1; i < m; i++) C *= H.nb[i];
                    fcontract(cur, oth, A, H.nb[j], H.nq[j], C, mats + H.oB[j]);
                    A *= H.nq[j];
                    T *tp = cur; cur = oth; oth = tp;
                    __syncthreads();
                }
                // inner slots and potential, in registers
                switch (R) {
                    case 0: reg_phase<T, 0, NB1, NQ1>(P, H, mats, cur); break;
                    case 1: if constexpr (RMAX >= 1) reg_phase<T, 1, NB1, NQ1>(P, H, mats, cur); break;
                    case 2: if constexpr (RMAX >= 2) reg_phase<T, 2, NB1, NQ1>(P, H, mats, cur); break;
                    case 3: if constexpr (RMAX >= 3) reg_phase<T, 3, NB1, NQ1>(P, H, mats, cur); break;
                    default: break;
                }
                __syncthreads();
                // outer grid -> basis, reverse order
                for (int j = m - 1; j >= p0; j--) {
                    int Aj = H.NBIn, C = 1;
                    for (int i = p0; i < j; i++) Aj *= H.nq[i];
                    for (int i = j + 1; i < m; i++) C *= H.nb[i];
                    fcontract(cur, oth, Aj, H.nq[j], H.nb[j], C, mats + H.oBW[j]);
                    T *tp = cur; cur = oth; oth = tp;
                    __syncthreads();
                }
                // Y[i][ko][rest] += WoB[ko] * cur[i][rest]
                for (int e = tid; e < H.NB; e += kFT) {
                    const int rr = e % H.NBrest, t2 = e / H.NBrest, ko = t2 % H.NBO, i = t2 / H.NBO;
                    Y[e] += WoB[ko] * cur[i * H.NBrest + rr];
                }
                __syncthreads();
            }
        }
        for (int e = tid; e < H.NB; e += kFT)
            fx_add_T<T>(accv + (size_t)rk[e] * kAccDigits, Y[e], H.coef, E, P.err);
        __syncthreads();
    }
}

template <typename T, int NB1, int NQ1, int RMAX>
cudaError_t launch_t(const KParams &kp, const double *x, int nvec, const long long *maxbits,
                     size_t smem, cudaStream_t stream, bool configure)
{
    if (configure)
        return cudaFuncSetAttribute(k_apply_fast<T, NB1, NQ1, RMAX>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_apply_fast<T, NB1, NQ1, RMAX><<<(unsigned)kp.n_terms, kFT, smem, stream>>>(kp, x, maxbits, nvec);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const KParams &kp, const double *x, int nvec, const long long *maxbits, size_t smem,
                     cudaStream_t stream, bool configure)
{
    constexpr int RM = sizeof(T) == 4 ? 3 : 1;
    const int nb1 = kp.fast.nb1, nq1 = kp.fast.nq1;
    if (nb1 == 2 && nq1 == 3) return launch_t<T, 2, 3, RM>(kp, x, nvec, maxbits, smem, stream, configure);
    if (nb1 == 2 && nq1 == 2) return launch_t<T, 2, 2, RM>(kp, x, nvec, maxbits, smem, stream, configure);
    if (nb1 == 3 && nq1 == 3) return launch_t<T, 3, 3, (RM > 2 ? 2 : RM)>(kp, x, nvec, maxbits, smem, stream, configure);
    return launch_t<T, 1, 1, 0>(kp, x, nvec, maxbits, smem, stream, configure);
}

}  // namespace

size_t fast_smem_bytes(const KParams &kp, bool fp32)
{
    const size_t rb = fp32 ? 4 : 8;
    return rb * ((size_t)kp.matcap + 4 * (size_t)kp.maxnb + 2 * (size_t)kp.cap) + 4 * (size_t)kp.maxnb;
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
