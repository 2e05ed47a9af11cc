// Device side of the propagation server (sg_server_api.cpp): one fused update of
// every active request's Chebyshev recurrence after a batched application of
// H_S, and the per-request norm / energy sums logged at the start of each step.
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

// X = T_k, Y = H T_k, P = T_{k-1} (unused when forming T_1), A = partial sum.
// Writes T_{k+1} (or, when the step ends, the new psi) into P's slot; the host
// then swaps the roles of X and P for every request.
__global__ void k_cheb_update(const ChebItem *__restrict__ items, const long long *__restrict__ prefix, int nitems,
                              const double *__restrict__ X, const double *__restrict__ Y, double *P, double *A)
{
    const long long total = prefix[nitems];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int j = owner(prefix, nitems, g);
        const ChebItem &it = items[j];
        const long long n = prefix[j + 1] - prefix[j];
        const long long i = g - prefix[j];
        const long long re = 2 * prefix[j] + i, im = re + n;
        const double xr = X[re], xi = X[im];
        const double hr = (Y[re] - it.ebar * xr) * it.inv_de, hi = (Y[im] - it.ebar * xi) * it.inv_de;
        double tr, ti, ar, ai;
        if (it.first) {
            tr = hr;
            ti = hi;
            ar = it.c0 * xr;
            ai = it.c0 * xi;
        } else {
            tr = 2.0 * hr - P[re];
            ti = 2.0 * hi - P[im];
            ar = A[re];
            ai = A[im];
        }
        double qr, qi;
        rot(it.q, tr, ti, qr, qi);
        ar = fma(it.c_new, qr, ar);
        ai = fma(it.c_new, qi, ai);
        if (it.finish) {
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

// One block per logged request: <psi|psi> and <psi|H psi>/<psi|psi> over its
// own entries, summed in an order that depends on its size only.
constexpr int kLogThreads = 256;
__global__ void __launch_bounds__(kLogThreads) k_cheb_log(const ChebLog *__restrict__ logs,
                                                          const double *__restrict__ X,
                                                          const double *__restrict__ Y)
{
    const ChebLog L = logs[blockIdx.x];
    const double *xr = X + 2 * L.off, *xi = xr + L.n, *yr = Y + 2 * L.off, *yi = yr + L.n;
    double nn = 0.0, ee = 0.0;
    for (long long i = threadIdx.x; i < L.n; i += kLogThreads) {
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
        L.out[0] = sn[0];
        L.out[1] = se[0] / sn[0];
    }
}

}  // namespace

cudaError_t launch_cheb_update(const ChebItem *items, const long long *prefix, int nitems, int64_t total,
                               const double *X, const double *Y, double *P, double *A, cudaStream_t s)
{
    if (nitems <= 0 || total <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
    k_cheb_update<<<blocks, 256, 0, s>>>(items, prefix, nitems, X, Y, P, A);
    return cudaGetLastError();
}

cudaError_t launch_cheb_log(const ChebLog *logs, int nlogs, const double *X, const double *Y, cudaStream_t s)
{
    if (nlogs <= 0) return cudaSuccess;
    k_cheb_log<<<(unsigned)nlogs, kLogThreads, 0, s>>>(logs, X, Y);
    return cudaGetLastError();
}

}  // namespace sg
