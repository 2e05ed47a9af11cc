// Solvers around the Smolyak action (Sec. 3, last paragraph: the Davidson
// method for stationary states, the Chebyshev method for wave-packet
// propagation): block Lanczos and block Davidson eigensolvers, Chebyshev
// propagation.  Recurrence vectors, inner products and orthogonalisation are
// FP64 on the device; the small projected problems are solved on the host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kGramRows = 8;   // rows of A per block in the Gram kernel
constexpr int kMaxCols = 8;    // columns of B (block size) per call
constexpr int kGramChunks = 304;

// partial[c][i][j] = sum over chunk c of A[i][e] * B[j][e]  (A: ka x n, B: kb x n, column vectors)
__global__ void __launch_bounds__(256) k_gram_partial(const double *__restrict__ A, int ka,
                                                      const double *__restrict__ B, int kb, int64_t n,
                                                      double *__restrict__ partial)
{
    __shared__ double red[kGramRows * kMaxCols][8];
    const int c = blockIdx.x, i0 = blockIdx.y * kGramRows;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t e0 = c * chunk, e1 = min(n, e0 + chunk);
    double acc[kGramRows][kMaxCols];
#pragma unroll
    for (int r = 0; r < kGramRows; r++)
#pragma unroll
        for (int j = 0; j < kMaxCols; j++) acc[r][j] = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        double b[kMaxCols];
#pragma unroll
        for (int j = 0; j < kMaxCols; j++) b[j] = j < kb ? B[(size_t)j * n + e] : 0.0;
#pragma unroll
        for (int r = 0; r < kGramRows; r++) {
            if (i0 + r >= ka) break;
            const double a = A[(size_t)(i0 + r) * n + e];
#pragma unroll
            for (int j = 0; j < kMaxCols; j++) acc[r][j] = fma(a, b[j], acc[r][j]);
        }
    }
    // block reduction: warp shuffles, then the 8 warps in fixed order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < kGramRows; r++)
#pragma unroll
        for (int j = 0; j < kMaxCols; j++) {
            double v = acc[r][j];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[r * kMaxCols + j][warp] = v;
        }
    __syncthreads();
    for (int q = threadIdx.x; q < kGramRows * kMaxCols; q += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[q][w];
        const int r = q / kMaxCols, j = q % kMaxCols;
        if (i0 + r < ka && j < kb) partial[((size_t)c * ka + i0 + r) * kb + j] = v;
    }
}

// C[i][j] = sum_c partial[c][i][j], in chunk order (deterministic)
__global__ void k_gram_final(const double *__restrict__ partial, int nchunk, int ka, int kb, double *__restrict__ C)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ka * kb) return;
    double v = 0.0;
    for (int c = 0; c < nchunk; c++) v += partial[(size_t)c * ka * kb + q];
    C[q] = v;
}

// out[j][e] = beta * out[j][e] + alpha * sum_i V[i][e] S[i][j]   (S: k x r, row-major, device)
__global__ void __launch_bounds__(256) k_combine(const double *__restrict__ V, int k, const double *__restrict__ S,
                                                 int r, double alpha, double beta, double *__restrict__ out,
                                                 int64_t n)
{
    extern __shared__ double Ss[];
    for (int q = threadIdx.x; q < k * r; q += blockDim.x) Ss[q] = S[q];
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double acc[kMaxCols];
#pragma unroll
        for (int j = 0; j < kMaxCols; j++) acc[j] = 0.0;
        for (int i = 0; i < k; i++) {
            const double v = V[(size_t)i * n + e];
#pragma unroll
            for (int j = 0; j < kMaxCols; j++)
                if (j < r) acc[j] = fma(v, Ss[i * r + j], acc[j]);
        }
        for (int j = 0; j < r; j++) {
            double *o = out + (size_t)j * n + e;
            *o = (beta == 0.0 ? 0.0 : beta * *o) + alpha * acc[j];
        }
    }
}

// y[j] = a * x[j] + b * y[j] over several vectors laid out contiguously
__global__ void k_axpby(int64_t len, double a, const double *__restrict__ x, double b, double *__restrict__ y)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = a * x[e] + (b == 0.0 ? 0.0 : b * y[e]);
}

// element-wise preconditioner: r[j][e] /= (d[e] - theta[j]) (guarded)
__global__ void k_precond(const double *__restrict__ d, const double *__restrict__ theta, int r, int64_t n,
                          double *__restrict__ x)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n);
        const double den = d[e - (int64_t)j * n] - theta[j];
        x[e] /= (fabs(den) < 1e-3 ? (den < 0 ? -1e-3 : 1e-3) : den);
    }
}

}  // namespace

// ---------------------------------------------------------------- device helpers
// C (ka x kb, row-major, device) = A^T B for column vectors A (ka x n), B (kb x n), kb <= kMaxCols.
// partial: gram_partial_doubles(ka) doubles of device scratch.  Deterministic.
cudaError_t dev_gram(const double *A, int ka, const double *B, int kb, int64_t n, double *C_dev,
                     double *partial, cudaStream_t s)
{
    if (kb > kMaxCols || kb < 1 || ka < 1) return cudaErrorInvalidValue;
    dim3 grid(kGramChunks, (ka + kGramRows - 1) / kGramRows);
    k_gram_partial<<<grid, 256, 0, s>>>(A, ka, B, kb, n, partial);
    k_gram_final<<<(ka * kb + 255) / 256, 256, 0, s>>>(partial, kGramChunks, ka, kb, C_dev);
    return cudaGetLastError();
}

size_t gram_partial_doubles(int ka) { return (size_t)kGramChunks * ka * kMaxCols; }

cudaError_t dev_combine(const double *V, int k, const double *S_dev, int r, double alpha, double beta, double *out,
                        int64_t n, cudaStream_t s)
{
    if (r > kMaxCols || r < 1 || k < 1) return cudaErrorInvalidValue;
    k_combine<<<608, 256, sizeof(double) * k * r, s>>>(V, k, S_dev, r, alpha, beta, out, n);
    return cudaGetLastError();
}

cudaError_t dev_axpby(int64_t len, double a, const double *x, double b, double *y, cudaStream_t s)
{
    k_axpby<<<608, 256, 0, s>>>(len, a, x, b, y);
    return cudaGetLastError();
}

cudaError_t dev_precond(const double *d, const double *theta_dev, int r, int64_t n, double *x, cudaStream_t s)
{
    k_precond<<<608, 256, 0, s>>>(d, theta_dev, r, n, x);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- host dense algebra
// Symmetric eigenproblem (cyclic Jacobi): A (n x n, row-major) destroyed;
// eigenvalues ascending in w, eigenvectors as columns of Z (row-major n x n).
void sym_eig(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &Z)
{
    Z.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) Z[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                const double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                const double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; k++) {  // A <- A G (columns p, q)
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {  // A <- G^T A (rows p, q)
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    const double zkp = Z[(size_t)k * n + p], zkq = Z[(size_t)k * n + q];
                    Z[(size_t)k * n + p] = c * zkp - s * zkq;
                    Z[(size_t)k * n + q] = s * zkp + c * zkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; i++) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
    std::vector<double> Zs((size_t)n * n);
    w.assign(n, 0.0);
    for (int c2 = 0; c2 < n; c2++) {
        w[c2] = A[(size_t)idx[c2] * n + idx[c2]];
        for (int k = 0; k < n; k++) Zs[(size_t)k * n + c2] = Z[(size_t)k * n + idx[c2]];
    }
    Z.swap(Zs);
}

// Cholesky G = R^T R (G: b x b row-major, overwritten by R^{-1}, upper triangular).
// Returns the number of leading columns that were numerically independent.
int chol_inverse(int b, std::vector<double> &G)
{
    std::vector<double> R((size_t)b * b, 0.0);
    int rank = b;
    for (int j = 0; j < b; j++) {
        double d = G[(size_t)j * b + j];
        for (int k = 0; k < j; k++) d -= R[(size_t)k * b + j] * R[(size_t)k * b + j];
        if (!(d > 1e-24 * std::max(1.0, std::fabs(G[(size_t)j * b + j])))) { rank = j; break; }
        R[(size_t)j * b + j] = std::sqrt(d);
        for (int i = j + 1; i < b; i++) {
            double v = G[(size_t)j * b + i];
            for (int k = 0; k < j; k++) v -= R[(size_t)k * b + j] * R[(size_t)k * b + i];
            R[(size_t)j * b + i] = v / R[(size_t)j * b + j];
        }
    }
    // inverse of the leading rank x rank block of R (upper triangular), zero elsewhere
    std::vector<double> Ri((size_t)b * b, 0.0);
    for (int j = 0; j < rank; j++) {
        Ri[(size_t)j * b + j] = 1.0 / R[(size_t)j * b + j];
        for (int i = j - 1; i >= 0; i--) {
            double v = 0.0;
            for (int k = i + 1; k <= j; k++) v += R[(size_t)i * b + k] * Ri[(size_t)k * b + j];
            Ri[(size_t)i * b + j] = -v / R[(size_t)i * b + i];
        }
    }
    G.swap(Ri);
    return rank;
}

// Bessel functions J_0..J_{kmax}(x), x > 0, by Miller's backward recurrence
// J_{k-1} = (2k/x) J_k - J_{k+1}, normalised with J_0 + 2 sum_{m>=1} J_{2m} = 1.
std::vector<double> bessel_j(int kmax, double x)
{
    std::vector<double> J(kmax + 1, 0.0);
    if (x == 0.0) { J[0] = 1.0; return J; }
    const int start = 2 * ((std::max(kmax, (int)x) + 30 + (int)(std::sqrt(40.0 * std::max(kmax, (int)x)))) / 2);
    std::vector<double> t(start + 2, 0.0);
    t[start + 1] = 0.0;
    t[start] = 1e-300;
    double norm = 0.0;
    for (int k = start; k >= 1; k--) {
        t[k - 1] = (2.0 * k / x) * t[k] - t[k + 1];
        if (std::fabs(t[k - 1]) > 1e250) {  // rescale to avoid overflow
            for (int q = k - 1; q <= start; q++) t[q] *= 1e-250;
        }
    }
    norm = t[0];
    for (int m = 2; m <= start; m += 2) norm += 2.0 * t[m];
    for (int k = 0; k <= kmax; k++) J[k] = t[k] / norm;
    return J;
}

}  // namespace sg
