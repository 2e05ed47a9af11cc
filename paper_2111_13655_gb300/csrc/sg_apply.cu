// Smolyak operator action on the GPU (sm_103a).
//
// One thread block per Smolyak term (terms ordered most-expensive first).  For
// term l the block performs Alg. 1 of arXiv 2111.13655:
//   1. extract the term from the compact vector (mapping table M^B, Table 2),
//      the compact index computed combinatorially;
//   2. basis -> grid, one mode at a time (Eq. (15));
//   3. the operator on the grid: the potential multiplied point-wise;
//   4. grid -> basis (Eq. (14));
//   5. compress-add D_l * result into the compact output (Eq. (16)).
// Operators that act on a single mode -- the kinetic part and every monomial
// of the potential that involves one transformed mode -- are applied as
// nb x nb matrices H1_j = K_j + sum_m c_m B_j^T W_j diag(Q^p) B_j in the basis:
// because B_i^T W_i B_i = I for every other mode (nq >= nb), this equals
// taking them through the grid.  The grid carries the monomials that couple
// two or more transformed modes.  The harmonic part of a mode (when the
// potential holds the quadratic that matches its basis) is diagonal in every
// term and is added once in the compact basis by the finalize kernel.
// The compress-add is exact: each D_l * y_l[k] is converted to an integer
// multiple of 2^E and summed in four 32-bit digits held in int64 words, so the
// result does not depend on the order in which terms finish.
// Modes whose level holds a single basis function (nb = 1) are not expanded:
// their quadrature sum is folded exactly into the potential through the
// moments mu_p = sum_u w_u b_0(Q_u)^2 Q_u^p (the term tensor is rank one along
// such a mode), so only the modes with nb > 1 ("slots") are transformed.
// Terms whose grid does not fit in shared memory are processed in slices over
// their first `s` slots (depth-first over the slice index, breadth-first
// inside), which leaves the arithmetic of every slot unchanged.
#include <algorithm>
#include <cstdint>

#include "sg_fixed.cuh"
#include "sg_internal.h"

namespace sg {

using fx::fx_add_real;
using fx::lsb_exponent;

namespace {

struct Mono1 { int slot, pow; double cf; };
struct Mono2 { int pair, pa, pb, pad; double cf; };
struct PairT { int a, b, off, pad; };
struct MonoG { int m, pad; double cf; };

struct TermHdr {
    int m, NB, s, NBO, NBI, nslice, nfib, bad;
    int n1, npair, n2, ng, grid;
    int mode[kMaxD], lev[kMaxD], nb[kMaxD], nq[kMaxD];
    int oB[kMaxD], oBW[kMaxD], oK[kMaxD];              // shared-memory offsets per slot
    int gM[kMaxD], gK[kMaxD];                          // global offsets of M_p and K per slot
    int gQ[kMaxD];                                     // global offset of Q_u per slot
    int stride[kMaxD];                                 // basis-tensor strides (last slot fastest)
    int slot_of_mode[kMaxD];
    int uS[kMaxD];                                     // grid indices of the current slice
    double c0;                                         // constant of the term (collapsed modes)
    int coef;                                          // D_l
};

__device__ __forceinline__ void set_err(const KParams &P, int code)
{
    if (P.err) atomicCAS(P.err, 0, code);
}

// Serial per-term set-up (thread 0): slots, split, shared-memory offsets, and
// the potential folded over the nb = 1 modes and grouped by the slots it touches.
__device__ void decode_term(const KParams &P, int t, TermHdr &H, Mono1 *m1, Mono2 *m2, PairT *pr,
                            MonoG *mg)
{
    const uint8_t *lt = P.levels + (size_t)t * P.Dpad;
    H.m = 0; H.NB = 1; H.bad = 0; H.c0 = 0.0;
    int mat = 0;
    for (int i = 0; i < P.D; i++) {
        const LevelInfo li = P.lvl[i * (P.L + 1) + lt[i]];
        if (li.nb > 1) {
            int j = H.m++;
            H.mode[j] = i; H.lev[j] = lt[i]; H.nb[j] = li.nb; H.nq[j] = li.nq;
            H.slot_of_mode[i] = j;
            H.oB[j] = mat;  mat += li.nq * li.nb;
            H.oBW[j] = mat; mat += li.nb * li.nq;
            H.oK[j] = mat;  mat += li.nb * li.nb;
            H.gQ[j] = li.offQ; H.gM[j] = li.offM; H.gK[j] = P.harm_mono[i] >= 0 ? -1 : li.offK;
            H.NB *= li.nb;
        } else {
            H.slot_of_mode[i] = -1;
            if (P.harm_mono[i] < 0) H.c0 += P.tabd[li.offK];  // 1x1 kinetic of a collapsed mode
        }
    }
    if (mat > P.matcap || H.NB > P.maxnb) { H.bad = 1; return; }
    int st = 1;
    for (int j = H.m - 1; j >= 0; j--) { H.stride[j] = st; st *= H.nb[j]; }
    // potential: fold collapsed modes through their moments, group by slots
    H.n1 = H.npair = H.n2 = H.ng = 0;
    int voff = 0;
    for (int mm = 0; mm < P.nmono; mm++) {
        bool split = false;
        for (int i = 0; i < P.D && !split; i++) split = (P.harm_mono[i] == mm);
        if (split) continue;  // harmonic part: added in the compact basis
        int fmode[kMaxFac], fpow[kMaxFac], nf = 0;
        for (int q = P.mfoff[mm]; q < P.mfoff[mm + 1]; q++) {
            int md = P.mfmode[q], pw = P.mfpow[q], k = 0;
            while (k < nf && fmode[k] != md) k++;
            if (k == nf) { fmode[nf] = md; fpow[nf] = pw; nf++; } else fpow[k] += pw;
        }
        double cf = P.mcoef[mm];
        int zs[kMaxFac], zp[kMaxFac], nz = 0;
        for (int k = 0; k < nf; k++) {
            int sl = H.slot_of_mode[fmode[k]];
            if (sl < 0) {
                const LevelInfo li = P.lvl[fmode[k] * (P.L + 1) + lt[fmode[k]]];
                cf *= P.tabd[li.offMu + fpow[k]];
            } else { zs[nz] = sl; zp[nz] = fpow[k]; nz++; }
        }
        if (nz == 0) {
            H.c0 += cf;
        } else if (nz == 1) {
            m1[H.n1++] = Mono1{zs[0], zp[0], cf};
        } else if (nz == 2) {
            int a = zs[0], b = zs[1], pa = zp[0], pb = zp[1];
            if (a > b) { int tt = a; a = b; b = tt; tt = pa; pa = pb; pb = tt; }
            int p = 0;
            while (p < H.npair && !(pr[p].a == a && pr[p].b == b)) p++;
            if (p == H.npair) {
                if (voff + H.nq[a] * H.nq[b] > P.vtabcap) { H.bad = 3; return; }
                pr[p] = PairT{a, b, voff, 0};
                voff += H.nq[a] * H.nq[b];
                H.npair++;
            }
            m2[H.n2++] = Mono2{p, pa, pb, 0, cf};
        } else {
            mg[H.ng++] = MonoG{mm, 0, cf};
        }
    }
    H.grid = (H.m > 0) && (H.npair + H.ng > 0);
    // split: smallest s whose inner working set fits a grid buffer
    H.s = 0;
    if (H.grid) {
        for (int s = 0; s < H.m; s++) {
            int64_t stage = H.nb[H.m - 1];
            for (int j = s; j <= H.m - 2; j++) stage *= H.nq[j];
            H.s = s;
            if (stage <= P.cap) break;
        }
        int64_t stage = H.nb[H.m - 1];
        for (int j = H.s; j <= H.m - 2; j++) stage *= H.nq[j];
        if (stage > P.cap) { H.bad = 2; return; }
    }
    H.NBO = 1; H.nslice = 1;
    for (int j = 0; j < H.s; j++) { H.NBO *= H.nb[j]; H.nslice *= H.nq[j]; }
    H.NBI = H.NB / H.NBO;
    H.nfib = 1;
    for (int j = H.s; j <= H.m - 2; j++) H.nfib *= H.nq[j];
    H.coef = P.coefs[t];
}

// compact index of the basis function with per-slot indices k[0..m-1]
__device__ __forceinline__ int rank_of(const KParams &P, const TermHdr &H, const int *k)
{
    int r = 0, s = 0;
    for (int j = 0; j < H.m; j++) {
        const int i = H.mode[j];
        r += P.rank_tab[(i * (P.L + 1) + s) * P.kw + k[j]];
        s += P.lmin_tab[i * P.kw + k[j]];
    }
    return r;
}

template <typename T>
__device__ __forceinline__ T ipow(T q, int p)
{
    T r = T(1);
    for (int e = 0; e < p; e++) r *= q;
    return r;
}

// out[a][r][c] = sum_k M[r*n + k] * in[a][k][c]
template <typename T>
__device__ void contract(const T *in, T *out, int A, int n, int r, int C, const T *M)
{
    const int total = A * r * C;
    for (int e = threadIdx.x; e < total; e += kThreads) {
        const int c = e % C;
        const int tq = e / C;
        const int rr = tq % r;
        const int a = tq / r;
        const T *ip = in + (a * n) * C + c;
        const T *mp = M + rr * n;
        T acc = T(0);
        for (int k = 0; k < n; k++) acc += mp[k] * ip[k * C];
        out[e] = acc;
    }
}

template <typename T> struct Tab;
template <> struct Tab<double> { static __device__ const double *get(const KParams &P) { return P.tabd; } };
template <> struct Tab<float> { static __device__ const float *get(const KParams &P) { return P.tabf; } };

template <typename T>
__global__ void __launch_bounds__(kThreads) k_apply(const KParams P, const double *__restrict__ x,
                                                    const long long *__restrict__ maxbits, int nvec)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ TermHdr H;
    const int tid = threadIdx.x;
    const int nm = P.nmono > 0 ? P.nmono : 1;
    Mono1 *m1 = reinterpret_cast<Mono1 *>(smraw);
    Mono2 *m2 = reinterpret_cast<Mono2 *>(m1 + nm);
    PairT *pr = reinterpret_cast<PairT *>(m2 + nm);
    MonoG *mg = reinterpret_cast<MonoG *>(pr + nm);
    T *mats = reinterpret_cast<T *>(mg + nm);
    T *vtab = mats + P.matcap;
    T *X = vtab + P.vtabcap;
    T *Y = X + P.maxnb;
    T *WoF = Y + P.maxnb;
    T *WoB = WoF + P.maxnb;
    T *bufA = WoB + P.maxnb;
    T *bufB = bufA + P.cap;
    int *rk = reinterpret_cast<int *>(bufB + P.cap);

    const int64_t q = (int64_t)blockIdx.x * P.nparts + P.part;  // this part's processing positions
    if (q >= P.n_terms) return;
    const int t = P.order[q];
    if (tid == 0) decode_term(P, t, H, m1, m2, pr, mg);
    __syncthreads();
    if (H.bad) {
        if (tid == 0) set_err(P, 100 + H.bad);
        return;
    }
    const T *tab = Tab<T>::get(P);
    const int m = H.m;

    // per-slot 1D matrices: B and B^T W (grid part), H1 = K + sum_m c_m M_p (basis part)
    for (int j = 0; j < m; j++) {
        const LevelInfo li = P.lvl[H.mode[j] * (P.L + 1) + H.lev[j]];
        const int nbq = li.nb * li.nq, nb2 = li.nb * li.nb;
        if (H.grid)
            for (int e = tid; e < nbq; e += kThreads) {
                mats[H.oB[j] + e] = tab[li.offB + e];
                mats[H.oBW[j] + e] = tab[li.offBW + e];
            }
        for (int e = tid; e < nb2; e += kThreads) {
            double h = H.gK[j] >= 0 ? P.tabd[H.gK[j] + e] : 0.0;
            for (int a = 0; a < H.n1; a++)
                if (m1[a].slot == j) h += m1[a].cf * P.tabd[H.gM[j] + (m1[a].pow - 1) * nb2 + e];
            mats[H.oK[j] + e] = (T)h;
        }
    }
    // potential tables g_p[ua][ub] of the monomials coupling two slots
    for (int p = 0; p < H.npair; p++) {
        const int a = pr[p].a, b = pr[p].b, nqb = H.nq[b];
        for (int e = tid; e < H.nq[a] * nqb; e += kThreads) {
            const int ua = e / nqb, ub = e % nqb;
            const double qa = P.tabd[H.gQ[a] + ua], qb = P.tabd[H.gQ[b] + ub];
            double v = 0.0;
            for (int c = 0; c < H.n2; c++)
                if (m2[c].pair == p) v += m2[c].cf * ipow(qa, m2[c].pa) * ipow(qb, m2[c].pb);
            vtab[pr[p].off + e] = (T)v;
        }
    }
    // compact indices of the term's basis functions
    for (int e = tid; e < H.NB; e += kThreads) {
        int k[kMaxD], rem = e;
        for (int j = m - 1; j >= 0; j--) { k[j] = rem % H.nb[j]; rem /= H.nb[j]; }
        rk[e] = rank_of(P, H, k);
    }
    __syncthreads();

    for (int v = 0; v < nvec; v++) {
        const double *xv = x + (size_t)v * P.n_cs;
        unsigned long long *accv = P.acc + (size_t)v * fx::Acc<T>::words;  // entry r at r * nvec
        const long long mbv = maxbits[v];
        for (int e = tid; e < H.NB; e += kThreads) { X[e] = (T)__ldg(xv + rk[e]); Y[e] = T(0); }
        __syncthreads();
        if (H.grid) {
            const int s = H.s, mL = m - 1, nbL = H.nb[mL], nqL = H.nq[mL];
            for (int sl = 0; sl < H.nslice; sl++) {
                if (tid == 0) {
                    int rem = sl;
                    for (int j = s - 1; j >= 0; j--) { H.uS[j] = rem % H.nq[j]; rem /= H.nq[j]; }
                }
                __syncthreads();
                // slice weights over the outer slots
                for (int ko = tid; ko < H.NBO; ko += kThreads) {
                    int rem = ko;
                    T wf = T(1), wb = T(1);
                    for (int j = s - 1; j >= 0; j--) {
                        const int kj = rem % H.nb[j];
                        rem /= H.nb[j];
                        wf *= mats[H.oB[j] + H.uS[j] * H.nb[j] + kj];
                        wb *= mats[H.oBW[j] + kj * H.nq[j] + H.uS[j]];
                    }
                    WoF[ko] = wf; WoB[ko] = wb;
                }
                __syncthreads();
                for (int ki = tid; ki < H.NBI; ki += kThreads) {
                    T acc = T(0);
                    for (int ko = 0; ko < H.NBO; ko++) acc += WoF[ko] * X[ko * H.NBI + ki];
                    bufA[ki] = acc;
                }
                __syncthreads();
                T *cur = bufA, *oth = bufB;
                // basis -> grid over the inner slots but the last
                int A = 1;
                for (int j = s; j < mL; j++) {
                    int C = 1;
                    for (int i = j + 1; i < m; i++) C *= H.nb[i];
                    contract(cur, oth, A, H.nb[j], H.nq[j], C, mats + H.oB[j]);
                    A *= H.nq[j];
                    T *tp = cur; cur = oth; oth = tp;
                    __syncthreads();
                }
                // last slot: basis -> grid, coupling potential, grid -> basis, one fibre per thread
                const T *BL = mats + H.oB[mL];
                const T *BWL = mats + H.oBW[mL];
                for (int fb = tid; fb < H.nfib; fb += kThreads) {
                    int u[kMaxD];
                    for (int j = 0; j < s; j++) u[j] = H.uS[j];
                    int rem = fb;
                    for (int j = mL - 1; j >= s; j--) { u[j] = rem % H.nq[j]; rem /= H.nq[j]; }
                    T vpre = T(0);
                    for (int p = 0; p < H.npair; p++)
                        if (pr[p].b != mL) vpre += vtab[pr[p].off + u[pr[p].a] * H.nq[pr[p].b] + u[pr[p].b]];
                    T gin[kMaxLevelSize], acc[kMaxLevelSize];
                    for (int k = 0; k < nbL; k++) { gin[k] = cur[fb * nbL + k]; acc[k] = T(0); }
                    for (int uL = 0; uL < nqL; uL++) {
                        T g = T(0);
                        for (int k = 0; k < nbL; k++) g += BL[uL * nbL + k] * gin[k];
                        T V = vpre;
                        for (int p = 0; p < H.npair; p++)
                            if (pr[p].b == mL) V += vtab[pr[p].off + u[pr[p].a] * nqL + uL];
                        if (H.ng) {
                            u[mL] = uL;
                            for (int c = 0; c < H.ng; c++) {
                                T term = (T)mg[c].cf;
                                const int mm = mg[c].m;
                                for (int q = P.mfoff[mm]; q < P.mfoff[mm + 1]; q++) {
                                    const int sl2 = H.slot_of_mode[P.mfmode[q]];
                                    if (sl2 >= 0)
                                        term *= ipow((T)P.tabd[H.gQ[sl2] + u[sl2]], P.mfpow[q]);
                                }
                                V += term;
                            }
                        }
                        const T w = V * g;
                        for (int k = 0; k < nbL; k++) acc[k] += BWL[k * nqL + uL] * w;
                    }
                    for (int k = 0; k < nbL; k++) cur[fb * nbL + k] = acc[k];
                }
                __syncthreads();
                // grid -> basis over the inner slots but the last, in reverse order
                for (int j = mL - 1; j >= s; j--) {
                    int Aj = 1, C = 1;
                    for (int i = s; i < j; i++) Aj *= H.nq[i];
                    for (int i = j + 1; i < m; i++) C *= H.nb[i];
                    contract(cur, oth, Aj, H.nq[j], H.nb[j], C, mats + H.oBW[j]);
                    T *tp = cur; cur = oth; oth = tp;
                    __syncthreads();
                }
                // accumulate the slice into the term result
                for (int e = tid; e < H.NB; e += kThreads) {
                    const int ko = e / H.NBI, ki = e - ko * H.NBI;
                    Y[e] += WoB[ko] * cur[ki];
                }
                __syncthreads();
            }
        }
        // single-mode matrices in the basis, then the exact compress-add with D_l
        for (int e = tid; e < H.NB; e += kThreads) {
            T acc = (T)H.c0 * X[e];
            int rem = e;
            for (int j = m - 1; j >= 0; j--) {
                const int nbj = H.nb[j], kj = rem % nbj;
                rem /= nbj;
                const int base = e - kj * H.stride[j];
                const T *Kr = mats + H.oK[j] + kj * nbj;
                for (int kp = 0; kp < nbj; kp++) acc += Kr[kp] * X[base + kp * H.stride[j]];
            }
            fx::Acc<T>::add(accv + (size_t)rk[e] * nvec * fx::Acc<T>::words, Y[e] + acc, H.coef, mbv, P.err);
        }
        __syncthreads();
    }
}

// max |x| of each vector (as the bit pattern of a non-negative double)
__global__ void k_maxabs(const double *__restrict__ x, int n, long long *__restrict__ maxbits)
{
    const int v = blockIdx.y;
    long long mb = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long b = __double_as_longlong(x[(size_t)v * n + i]) & 0x7FFFFFFFFFFFFFFFll;
        mb = b > mb ? b : mb;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = other > mb ? other : mb;
    }
    if ((threadIdx.x & 31) == 0 && mb) atomicMax(maxbits + v, mb);
}

// Entry-major copy of the input vectors in the contraction type (rows of
// `stride` elements, a multiple of 4): thread r reads x_v[r] for every vector
// (coalesced across threads per vector) and writes the first xs_stride(nvec)
// values of its row (zero beyond nvec) as 16-byte stores.
template <typename T>
__device__ __forceinline__ void stage_rows(const double *__restrict__ x, long long n, int nvec, int stride,
                                           T *__restrict__ xs, long long r0, long long rstep)
{
    constexpr int U = 16 / (int)sizeof(T);
    struct alignas(16) Unit { T v[U]; };
    const int w = xs_stride(nvec);
    for (long long r = r0; r < n; r += rstep) {
        T *row = xs + (size_t)r * stride;
        for (int v0 = 0; v0 < w; v0 += U) {
            Unit t;
#pragma unroll
            for (int e = 0; e < U; e++) t.v[e] = v0 + e < nvec ? (T)x[(size_t)(v0 + e) * n + r] : T(0);
            *reinterpret_cast<Unit *>(row + v0) = t;
        }
    }
}

template <typename T>
__global__ void k_stage_x(const double *__restrict__ x, int n, int nvec, int stride, T *__restrict__ xs)
{
    stage_rows<T>(x, n, nvec, stride, xs, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                  (long long)gridDim.x * blockDim.x);
}

// Many problems (blockIdx.z = problem j, its vectors from nvec * cs_prefix[j],
// its rows from cs_prefix[j]).
template <typename T>
__global__ void k_stage_x_batch(const double *__restrict__ x, const long long *__restrict__ cs_prefix, int nvec,
                                int stride, T *__restrict__ xs)
{
    const int j = blockIdx.z;
    const long long c0 = cs_prefix[j], n = cs_prefix[j + 1] - c0;
    stage_rows<T>(x + (size_t)nvec * c0, n, nvec, stride, xs + (size_t)c0 * stride,
                  blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// The accumulated integer of one entry times 2^E (E from the vector's max|x|
// bits; NaN when x held a non-finite value); clears the accumulator words.
// FP32 contexts: one signed word; FP64: four signed 32-bit digits.
__device__ __forceinline__ double finalize_value(unsigned long long *a, long long mb, int fp32)
{
    if (fp32) {
        const double v1 = (double)(long long)a[0];
        a[0] = 0ull;
        return ((mb >> 52) & 0x7FF) == 0x7FF ? __longlong_as_double(0x7FF8000000000000ll)
                                              : scalbn(v1, lsb_exponent(mb, kAcc32LsbBelowMax));
    }
    unsigned __int128 tot = 0;
#pragma unroll
    for (int d = 0; d < kAccDigits; d++) {
        const __int128 dv = (__int128)(long long)a[d];
        tot += (unsigned __int128)dv << (32 * d);
        a[d] = 0ull;
    }
    const __int128 st = (__int128)tot;
    const long long hi = (long long)(st >> 64);
    const unsigned long long lo = (unsigned long long)tot;
    const double val = scalbn((double)hi, 64) + (double)lo;
    return ((mb >> 52) & 0x7FF) == 0x7FF ? __longlong_as_double(0x7FF8000000000000ll) : scalbn(val, lsb_exponent(mb));
}

// y = (accumulated integer) * 2^E + esplit * x; clears the accumulators
// (accumulators entry-major: entry r, vector v at r * nvec + v)
__global__ void k_finalize(const KParams P, const double *__restrict__ x, double *__restrict__ y,
                           const long long *__restrict__ maxbits, int nvec, int fp32)
{
    const size_t total = (size_t)nvec * P.n_cs;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / P.n_cs);
        const size_t r = i - (size_t)v * P.n_cs;
        y[i] = finalize_value(P.acc + (r * nvec + v) * acc_words(fp32), maxbits[v], fp32) + P.esplit[r] * x[i];
    }
}

// Many problems (vectors problem after problem, problem j from nvec * cs_prefix[j]):
// per-vector max|x| bits into maxbits[j * nvec + v]; blockIdx.z = problem.
__global__ void k_maxabs_batch(const double *__restrict__ x, const long long *__restrict__ cs_prefix, int nvec,
                               long long *__restrict__ maxbits)
{
    const int j = blockIdx.z, v = blockIdx.y;
    const long long c0 = cs_prefix[j];
    const long long n = cs_prefix[j + 1] - c0;
    const double *xv = x + (size_t)nvec * c0 + (size_t)v * n;
    long long mb = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = __double_as_longlong(xv[i]) & 0x7FFFFFFFFFFFFFFFll;
        mb = b > mb ? b : mb;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long other = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = other > mb ? other : mb;
    }
    if ((threadIdx.x & 31) == 0 && mb) atomicMax(maxbits + (size_t)j * nvec + v, mb);
}

// Many problems: y = (accumulated integer) * 2^E + esplit_j * x, entry by entry;
// blockIdx.y = problem (its entries start at nvec * cs_prefix[j]); clears the
// accumulators.
__global__ void k_finalize_batch(const KParams *__restrict__ kps, const long long *__restrict__ cs_prefix,
                                 const double *__restrict__ x, double *__restrict__ y,
                                 unsigned long long *acc, const long long *__restrict__ maxbits, int nvec,
                                 int fp32)
{
    const int j = blockIdx.y;
    const size_t base = (size_t)nvec * (size_t)cs_prefix[j];
    const size_t n = (size_t)(cs_prefix[j + 1] - cs_prefix[j]);
    const size_t total = (size_t)nvec * n;
    const double *esplit = kps[j].esplit;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / n);
        const size_t r = i - (size_t)v * n;
        const size_t a = base + r * nvec + v;  // entry-major in its problem
        y[base + i] = finalize_value(acc + a * acc_words(fp32), maxbits[(size_t)j * nvec + v], fp32) +
                      esplit[r] * x[base + i];
    }
}

// Mapping table M^B (Table 2) for terms [t0, t0+nt): k_0 fastest inside a term.
__global__ void __launch_bounds__(kThreads) k_index_map(const KParams P, int64_t t0,
                                                        const int64_t *__restrict__ offs,
                                                        int64_t *__restrict__ out)
{
    __shared__ TermHdr H;
    const int64_t t = t0 + blockIdx.x;
    if (threadIdx.x == 0) {
        const uint8_t *lt = P.levels + (size_t)t * P.Dpad;
        H.m = 0; H.NB = 1;
        for (int i = 0; i < P.D; i++) {
            const LevelInfo li = P.lvl[i * (P.L + 1) + lt[i]];
            if (li.nb > 1) { int j = H.m++; H.mode[j] = i; H.nb[j] = li.nb; H.NB *= li.nb; }
        }
    }
    __syncthreads();
    const int64_t base = offs[blockIdx.x];
    for (int e = threadIdx.x; e < H.NB; e += kThreads) {
        int k[kMaxD], rem = e;
        for (int j = 0; j < H.m; j++) { k[j] = rem % H.nb[j]; rem /= H.nb[j]; }
        out[base + e] = rank_of(P, H, k);
    }
}

}  // namespace

size_t apply_smem_bytes(const KParams &kp, bool fp32)
{
    const size_t rb = fp32 ? 4 : 8;
    const size_t nm = kp.nmono > 0 ? kp.nmono : 1;
    return nm * (sizeof(Mono1) + sizeof(Mono2) + sizeof(PairT) + sizeof(MonoG)) +
           rb * ((size_t)kp.matcap + kp.vtabcap + 4 * (size_t)kp.maxnb + 2 * (size_t)kp.cap) +
           4 * (size_t)kp.maxnb;
}

// The limit is a property of the kernel, shared by every context: it is set to
// the most the device allows beside the kernel's static shared memory (not to
// one context's need, which could lower it under another context's launches).
template <typename K>
static cudaError_t set_smem_limit(K kernel, size_t need)
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

cudaError_t configure_kernels(size_t smem, bool fp32)
{
    return fp32 ? set_smem_limit(k_apply<float>, smem) : set_smem_limit(k_apply<double>, smem);
}

cudaError_t launch_apply(const KParams &kp, bool fp32, const double *x, double *y, int nvec,
                         long long *maxbits, int *lsb_exp, cudaStream_t stream)
{
    (void)lsb_exp;
    cudaError_t e = launch_maxabs(kp, x, nvec, maxbits, stream);
    if (e == cudaSuccess) e = launch_apply_terms(kp, fp32, x, maxbits, nvec, stream);
    if (e == cudaSuccess) e = launch_finalize(kp, fp32, x, y, nvec, maxbits, stream);
    return e;
}

cudaError_t launch_maxabs(const KParams &kp, const double *x, int nvec, long long *maxbits, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(long long) * nvec, stream);
    if (e != cudaSuccess) return e;
    k_maxabs<<<dim3(64, nvec), 256, 0, stream>>>(x, kp.n_cs, maxbits);
    return cudaGetLastError();
}

cudaError_t launch_stage_x(const KParams &kp, bool fp32, const double *x, int nvec, cudaStream_t stream)
{
    if (!kp.xs || nvec > kp.xs_nvec) return cudaErrorInvalidValue;
    const int stride = xs_stride(kp.xs_nvec);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((kp.n_cs + 255) / 256, 152 * 16));
    void *xs = const_cast<void *>(kp.xs);
    if (fp32) k_stage_x<float><<<blocks, 256, 0, stream>>>(x, kp.n_cs, nvec, stride, static_cast<float *>(xs));
    else if (kp.fast.df) k_stage_x<df2><<<blocks, 256, 0, stream>>>(x, kp.n_cs, nvec, stride, static_cast<df2 *>(xs));
    else k_stage_x<double><<<blocks, 256, 0, stream>>>(x, kp.n_cs, nvec, stride, static_cast<double *>(xs));
    return cudaGetLastError();
}

cudaError_t launch_stage_x_batch(bool fp32, const double *x, const long long *cs_prefix, int nprob, int64_t max_ncs,
                                 int nvec, int xs_nvec, void *xs, cudaStream_t stream)
{
    if (!xs || nvec > xs_nvec) return cudaErrorInvalidValue;
    const int stride = xs_stride(xs_nvec);
    const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (max_ncs + 255) / 256));
    if (fp32)
        k_stage_x_batch<float><<<dim3(bx, 1, nprob), 256, 0, stream>>>(x, cs_prefix, nvec, stride,
                                                                       static_cast<float *>(xs));
    else
        k_stage_x_batch<double><<<dim3(bx, 1, nprob), 256, 0, stream>>>(x, cs_prefix, nvec, stride,
                                                                        static_cast<double *>(xs));
    return cudaGetLastError();
}

cudaError_t launch_finalize(const KParams &kp, bool fp32, const double *x, double *y, int nvec,
                            const long long *maxbits, cudaStream_t stream)
{
    const size_t total = (size_t)nvec * kp.n_cs;
    const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, 152 * 16));
    k_finalize<<<blocks, 256, 0, stream>>>(kp, x, y, maxbits, nvec, fp32 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_apply_terms(const KParams &kp, bool fp32, const double *x, const long long *maxbits, int nvec,
                               cudaStream_t stream)
{
    if (kp.fast.enabled) {
        if (kp.xs && nvec <= kp.xs_nvec) {
            cudaError_t e = launch_stage_x(kp, fp32, x, nvec, stream);
            return e == cudaSuccess ? launch_apply_fast(kp, fp32, x, nvec, maxbits, stream) : e;
        }
        KParams k2 = kp;  // no staged copy of this size: the term kernels read x
        k2.xs = nullptr;
        return launch_apply_fast(k2, fp32, x, nvec, maxbits, stream);
    }
    if (kp.n_terms <= kp.part) return cudaSuccess;
    const size_t smem = apply_smem_bytes(kp, fp32);
    dim3 grid((unsigned)((kp.n_terms - kp.part + kp.nparts - 1) / kp.nparts));
    if (fp32)
        k_apply<float><<<grid, kThreads, smem, stream>>>(kp, x, maxbits, nvec);
    else
        k_apply<double><<<grid, kThreads, smem, stream>>>(kp, x, maxbits, nvec);
    return cudaGetLastError();
}

cudaError_t launch_maxabs_batch(const double *x, const long long *cs_prefix, int nprob, int64_t max_ncs, int nvec,
                                long long *maxbits, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(long long) * (size_t)nprob * nvec, stream);
    if (e != cudaSuccess) return e;
    const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (max_ncs + 255) / 256));
    k_maxabs_batch<<<dim3(bx, nvec, nprob), 256, 0, stream>>>(x, cs_prefix, nvec, maxbits);
    return cudaGetLastError();
}

cudaError_t launch_finalize_batch(const KParams *kps, const long long *cs_prefix, int nprob, int64_t max_ncs,
                                  const double *x, double *y, unsigned long long *acc, const long long *maxbits,
                                  int nvec, bool fp32, cudaStream_t stream)
{
    // blocks per problem: enough for the largest problem, within about 16 blocks per SM in all
    // (at least 64 per problem)
    const size_t per = (size_t)nvec * (size_t)max_ncs;
    const size_t cap = std::max<size_t>(64, (152 * 16 + (size_t)nprob - 1) / (size_t)std::max(1, nprob));
    const unsigned bx = (unsigned)std::max<size_t>(1, std::min<size_t>((per + 255) / 256, cap));
    k_finalize_batch<<<dim3(bx, (unsigned)nprob), 256, 0, stream>>>(kps, cs_prefix, x, y, acc, maxbits, nvec,
                                                                    fp32 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_index_map(const KParams &kp, int64_t t0, int64_t nt, const int64_t *offs,
                             int64_t *out, cudaStream_t stream)
{
    if (nt <= 0) return cudaSuccess;
    k_index_map<<<(unsigned)nt, kThreads, 0, stream>>>(kp, t0, offs, out);
    return cudaGetLastError();
}

}  // namespace sg
