// Device side of the propagation server (sg_server_api.cpp): one fused update of
// every active request's Chebyshev recurrence after a batched application of
// H_S, and the per-request norm / energy sums logged at the start of each step.
// The recurrence state (term index, step) lives on the device, so one
// iteration's launches are the same every time and can be replayed as a graph.
//
// Chebyshev propagator (Sec. 3, Sec. 5; Tal-Ezer-Kosloff form):
//   psi(t + dt) = e^{-i Ebar dt} sum_{k=0}^{K} c_k (-i)^k T_k,   c_k = (2 - delta_k0) J_k(dE dt),
//   T_0 = psi,  T_1 = (H - Ebar) psi / dE,  T_{k+1} = 2 (H - Ebar) T_k / dE - T_{k-1}.
// Vectors are complex, held as two real vectors (real part, then imaginary
// part) per request, requests one after another (the batch layout, nvec = 2).
#include <algorithm>

#include "sg_internal.h"

namespace sg {

namespace {

// Which request owns complex entry g: the last j with prefix[j] <= g.
__device__ __forceinline__ int owner(const long long *__restrict__ prefix, int n, long long g)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// (-i)^q (tr + i ti)
__device__ __forceinline__ void rot(int q, double tr, double ti, double &outr, double &outi)
{
    switch (q & 3) {
        case 0: outr = tr; outi = ti; break;
        case 1: outr = ti; outi = -tr; break;
        case 2: outr = -tr; outi = -ti; break;
        default: outr = -ti; outi = tr; break;
    }
}

// X = T_k, Y = H T_k, P = T_{k-1} (unused when forming T_1), A = partial sum;
// k, K and the weights come from the request's device state.  Writes T_{k+1}
// (or, on the step's last term, the new psi) into P's slot; the roles of X
// and P are then swapped for every request.  A request past its last step
// keeps psi: it is copied to P's slot.
__global__ void k_cheb_update(const ChebState *__restrict__ st, const long long *__restrict__ prefix, int nitems,
                              const double *__restrict__ X, const double *__restrict__ Y, double *P, double *A)
{
    const long long total = prefix[nitems];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int j = owner(prefix, nitems, g);
        const ChebState &it = st[j];
        const long long n = prefix[j + 1] - prefix[j];
        const long long i = g - prefix[j];
        const long long re = 2 * prefix[j] + i, im = re + n;
        const double xr = X[re], xi = X[im];
        if (it.step >= it.nsteps) {
            P[re] = xr;
            P[im] = xi;
            continue;
        }
        const int kn = it.k + 1;
        const double hr = (Y[re] - it.ebar * xr) * it.inv_de, hi = (Y[im] - it.ebar * xi) * it.inv_de;
        double tr, ti, ar, ai;
        if (it.k == 0) {
            tr = hr;
            ti = hi;
            ar = it.c[0] * xr;
            ai = it.c[0] * xi;
        } else {
            tr = 2.0 * hr - P[re];
            ti = 2.0 * hi - P[im];
            ar = A[re];
            ai = A[im];
        }
        double qr, qi;
        rot(kn, tr, ti, qr, qi);
        const double cn = it.c[kn];
        ar = fma(cn, qr, ar);
        ai = fma(cn, qi, ai);
        if (kn == it.K) {
            P[re] = it.cph * ar - it.sph * ai;
            P[im] = it.sph * ar + it.cph * ai;
        } else {
            P[re] = tr;
            P[im] = ti;
            A[re] = ar;
            A[im] = ai;
        }
    }
}

// Moves every request to its next recurrence term (after k_cheb_update).
__global__ void k_cheb_advance(ChebState *st, int nitems)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nitems) return;
    ChebState &s = st[j];
    if (s.step >= s.nsteps) return;
    if (s.k + 1 == s.K) { s.k = 0; s.step++; }
    else s.k++;
}

// One block per request; requests at the start of a step (k = 0) log
// <psi|psi> and <psi|H psi>/<psi|psi> over their own entries, summed in an
// order that depends on their size only.
constexpr int kLogThreads = 256;
__global__ void __launch_bounds__(kLogThreads) k_cheb_log(const ChebState *__restrict__ st,
                                                          const long long *__restrict__ prefix,
                                                          const double *__restrict__ X,
                                                          const double *__restrict__ Y)
{
    const ChebState &S = st[blockIdx.x];
    if (S.k != 0 || S.step >= S.nsteps) return;
    const long long off = prefix[blockIdx.x], n = prefix[blockIdx.x + 1] - off;
    const double *xr = X + 2 * off, *xi = xr + n, *yr = Y + 2 * off, *yi = yr + n;
    double nn = 0.0, ee = 0.0;
    for (long long i = threadIdx.x; i < n; i += kLogThreads) {
        nn = fma(xr[i], xr[i], fma(xi[i], xi[i], nn));
        ee = fma(xr[i], yr[i], fma(xi[i], yi[i], ee));
    }
    __shared__ double sn[kLogThreads], se[kLogThreads];
    sn[threadIdx.x] = nn;
    se[threadIdx.x] = ee;
    __syncthreads();
    for (int h = kLogThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sn[threadIdx.x] += sn[threadIdx.x + h];
            se[threadIdx.x] += se[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        S.log[2 * S.step] = sn[0];
        S.log[2 * S.step + 1] = se[0] / sn[0];
    }
}

}  // namespace

cudaError_t launch_cheb_iteration(ChebState *st, const long long *prefix, int nitems, int64_t total,
                                  const double *X, const double *Y, double *P, double *A, cudaStream_t s)
{
    if (nitems <= 0 || total <= 0) return cudaSuccess;
    k_cheb_log<<<(unsigned)nitems, kLogThreads, 0, s>>>(st, prefix, X, Y);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
    k_cheb_update<<<blocks, 256, 0, s>>>(st, prefix, nitems, X, Y, P, A);
    k_cheb_advance<<<(unsigned)((nitems + 127) / 128), 128, 0, s>>>(st, nitems);
    return cudaGetLastError();
}

}  // namespace sg
