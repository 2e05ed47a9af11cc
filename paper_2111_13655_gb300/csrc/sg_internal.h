// Internal declarations of libsmolyak (host setup <-> CUDA kernels <-> C ABI).
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/smolyak.h"

namespace sg {

constexpr int kMaxD = 32;          // modes per problem
constexpr int kMaxLevelSize = 32;  // nb(l), nq(l) at any level
constexpr int kMaxMono = 256;      // monomials in V
constexpr int kMaxFac = 8;         // factors per monomial
constexpr int kMaxPow = 16;        // power of one factor
constexpr int kThreads = 128;      // threads per term-CTA

// Per (mode, level) entry: sizes and element offsets into the flat tables.
struct LevelInfo {
    int nb, nq;
    int offB;   // B[u*nb+k]   = b_k(Q_u)                 (nq x nb)
    int offBW;  // BW[k*nq+u]  = w_u b_k(Q_u)             (nb x nq)
    int offK;   // K[k*nb+k']  = -omega/2 <b_k|d2/dQ2|b_k'> on the grid (nb x nb)
    int offQ;   // Q[u]        = Q_u                      (nq)
    int offMu;  // mu[p]       = sum_u w_u b_0(Q_u)^2 Q_u^p, p = 0..pmax (pmax+1)
    int offM;   // M_p[k*nb+k'] = sum_u w_u b_k(Q_u) Q_u^p b_k'(Q_u), p = 1..pmax (pmax blocks nb x nb)
};

// Fixed-point accumulation of the compact result: every contribution D_l * y_l[k]
// is added exactly as an integer multiple of 2^E (E chosen per vector from
// max|x|), split into four signed 32-bit digits held in int64 words.
constexpr int kAccDigits = 4;
constexpr int kAccLsbBelowMax = 80;  // E = exponent(max|x|) - 80
// FP32 contexts: one signed 64-bit word per entry, unit 2^(exponent(max|x|) - 40)
constexpr int kAcc32LsbBelowMax = 40;
// 64-bit words per accumulated entry of a context's precision
__host__ __device__ constexpr int acc_words(bool fp32) { return fp32 ? 1 : kAccDigits; }

constexpr int kMaxPairs = 64;  // coupled mode pairs handled by the fast path

// Tuning of the fast kernels (FP32 / FP64): the shared-memory budget per
// block that the host plans terms with, the resident blocks per SM the kernels
// are compiled for, and the vectors per chunk below which a term is sliced.
#ifndef SG_F32_SMEM_KB
#define SG_F32_SMEM_KB 52
#endif
#ifndef SG_F32_MINBLOCKS
#define SG_F32_MINBLOCKS 4
#endif
// (defaults: the plan sg_tune picks at D=12 L=10 in both precisions; FP64
// 165.6 -> 149.2 ms per 8-vector apply against a target of 4 vectors)
#ifndef SG_F32_SLICE_VT
#define SG_F32_SLICE_VT 1
#endif
#ifndef SG_F64_SLICE_VT
#define SG_F64_SLICE_VT 1
#endif
// Warp form: terms that fit a quarter of the block's shared memory with a
// chunk of SG_WARP_VT vectors (sliced when SG_WARP_SLICE is 1) run one per warp.
// Measured at D=12 L=10 (mixed): 1 vector 31.29 ms per 8-vector apply, 4
// vectors 31.85, 2 vectors 30.9 (sg_tune's pick there); slicing in the warp
// form 43-60 ms.  1 is kept: the 256-wavepacket batch (nb = nq = l+1) is 12%
// slower with 2.
#ifndef SG_WARP_VT
#define SG_WARP_VT 1
#endif
#ifndef SG_WARP_SLICE
#define SG_WARP_SLICE 0
#endif
#ifndef SG_F64_SMEM_KB
#define SG_F64_SMEM_KB 70
#endif
#ifndef SG_F64_MINBLOCKS
#define SG_F64_MINBLOCKS 3
#endif

// Inner positions of the fast kernel: up to fast_rmax level-1 modes whose
// action at each outer grid point is tabulated per term (inner-block table,
// NBI = nb1^R <= 9 values per inner block).  Level 1 must have the same basis
// size nb1 in every mode (2 or 3); otherwise no position is inner.
inline int fast_inner_nb(int nb1) { return nb1 == 2 || nb1 == 3 ? nb1 : 1; }
inline int fast_rmax(int nb1) { return nb1 == 2 ? 3 : nb1 == 3 ? 2 : 0; }

// Sizes shared by the host planner and the fast kernels.
// Padding of a buffer of n elements to a multiple of u elements (16 bytes).
__host__ __device__ inline int64_t pad_elems(int64_t n, int u) { return (n + u - 1) / u * u; }
#ifndef SG_STAGE_X
#define SG_STAGE_X 1  // the fast path gathers from an entry-major copy of x
#endif
// Row length (elements) of the entry-major input copy for nvec vectors.
__host__ __device__ inline int xs_stride(int nvec) { return (nvec + 3) & ~3; }
// Elements (of a type with u per 16 bytes) that hold a term's NB int32
// compact indices, padded to 16 bytes.
__host__ __device__ inline int64_t ranks_elems(int64_t NB, int u) { return pad_elems((NB * u + 3) / 4, u); }
// Work-area elements a chunk of vb vectors of one term needs: the term's
// compact indices, the gathered basis tensor X (and the slice accumulator Y
// when the term is sliced), and two buffers of the largest grid stage when the
// term has a grid (a term without a grid has a second basis-sized buffer
// instead, for the staged compress-add); every buffer padded to 16 bytes (u
// elements).
__host__ __device__ inline int64_t chunk_need(int64_t NB, int64_t stage, bool sliced, bool grid, int vb, int u)
{
    return ranks_elems(NB, u) + (sliced || !grid ? 2 : 1) * pad_elems(NB * vb, u) +
           (grid ? 2 * pad_elems(stage * vb, u) : 0);
}
// Byte offset, inside a work area of `work_bytes`, of the scratch copy of a
// term record (at most desccap 16-byte units) taken during the prologue: the
// end of the area, 16-byte aligned.  The term's compact indices, copied at the
// same time, occupy the start; the planner keeps the two apart.
__host__ __device__ inline int64_t record_scratch_offset(int64_t work_bytes, int desccap)
{
    return ((work_bytes - 16 * (int64_t)desccap) / 16) * 16;
}
// Inner-block table per outer grid point: the upper triangle of the NBI x NBI
// symmetric block (NBI (NBI+1)/2 values, row by row) in units of mt_unit
// elements (16 bytes, or one element when NBI = 1).
__host__ __device__ inline int mt_unit(int NBI, int u) { return NBI == 1 ? 1 : u; }
__host__ __device__ inline int mt_units(int NBI, int u)
{
    const int ue = mt_unit(NBI, u);
    return (NBI * (NBI + 1) / 2 + ue - 1) / ue;
}

// Per-term record of the fast kernel, in processing order, 16-byte units:
// header | positions[m] | active pairs[npair] | induced matrices[nind] (padded).
// Positions: the inner slots (mode order) first, then the outer slots in the
// order of fewest multiply-adds (ascending 1/nb - 1/nq, ties in mode order).
// Induced matrices: the two-mode monomials whose partner mode is collapsed,
// per position (summed into the term image's H1; listed for the inner-block
// tables).
struct alignas(16) FDescHdr {
    int m, R, NB, coef;          // positions, inner positions, basis size, D_l
    int s, npair, nind, gsize;   // slicing depth, active pairs, induced matrices, G-table words
    double c0;                   // constant of the term (collapsed modes)
    long long rank_off;          // start of the term's compact indices (layout order)
};
struct FDescPos { unsigned char mode, lev, nb, nq; int offB, offBW, offH1; };
struct FDescPair { unsigned char pa, pb, r0, r1; int goff, gsm, r2; };  // gsm: shared-memory offset of G
struct FDescInd { unsigned char pos, r0, r1, r2; int ioff; };
static_assert(sizeof(FDescHdr) == 48 && sizeof(FDescPos) == 16 && sizeof(FDescPair) == 16 &&
              sizeof(FDescInd) == 8, "descriptor layout");

// Fast-path tables (potentials whose monomials touch at most two modes).
// All offsets are element offsets into FastParams::tab (T precision) or
// ::sc (FP64 scalars); -1 marks an absent entry.
struct FastParams {
    int enabled;
    int nb1, nq1;          // uniform sizes of level 1 (0 if modes differ)
    int npairs;            // coupled mode pairs (i < i')
    const int *pair_modes; // [npairs][2]
    const int *h1off;      // [D][L+1]: single-mode matrix (nb x nb) of an active level
    const int *goff;       // [npairs][L+1][L+1]: coupling table G[u_i][u_i'] (active levels)
    const int *ioff;       // [npairs][2][L+1][L+1]: induced matrix on side s's mode at
                           //   level l_s when the partner is collapsed at level l_o
    const int *soff;       // [D][L+1]: scalar of a collapsed mode (into sc)
    const int *spoff;      // [npairs][L+1][L+1]: scalar of a pair with both modes collapsed
    const double *sc;      // scalars
    const double *tabd;    // FP64 fast tables
    const float *tabf;     // FP32 copies
    double c0const;        // constant monomials
    const int4 *desc;      // term records (processing order)
    const unsigned *desc_off;  // [n_terms+1] record starts, in 16-byte units
    const int *ranks;      // compact index of every basis function of every term (layout order)
    const long long *rank_start;  // [n_terms + 1] start of each term's indices in ranks (processing order)
    int desccap;           // largest record, in 16-byte units
    int gcap;              // largest set of a term's G tables, in words
    int nbocap;            // largest sliced outer block (slice weights)
    int n_big;             // terms [0, n_big) run one per block, the rest one per warp
    int work_cta, work_warp;   // work-area capacities (elements) of the two kernels
    // per-term shared-memory images (processing order): the term's B, B^T W and
    // H1 (base + induced, summed on the host) per position, then its G tables
    const double *imgd;        // FP64 contexts
    const float *imgf;         // FP32 contexts
    const long long *img_off;  // [n_terms + 1] image starts, in elements
    // inner-block tables: per term with coupled pairs, the action of its inner
    // positions at every outer grid point (symmetric NBI x NBI, upper triangle),
    // formed once per context; layout [slice][unit][outer grid point][unit elements]
    const double *mtabd;       // FP64 contexts
    const float *mtabf;        // FP32 contexts
    const long long *mt_off;   // [n_terms + 1] starts, in elements (16-byte aligned; 0-size without a grid)
    // double-float contexts (SG_DF64): contractions in pairs of FP32 numbers
    // (hi, lo), FP64 accumulation; images and inner-block tables as (hi, lo)
    int df;
    const float2 *imgx;
    const float2 *mtabx;
};

// Everything a kernel needs, passed by value (a multiple of 16 bytes, so
// that a kernel can copy it in 16-byte units).
struct alignas(16) KParams {
    int D, L, Dpad;
    int nmono, pmax, kw;
    int n_cs;
    int64_t n_terms;
    const uint8_t *levels;   // [n_terms][Dpad], Table-2 order
    const int *coefs;        // [n_terms] combination coefficient D_l
    const int *order;        // [n_terms] Table-2 index of the p-th processed term
    const int *rank_tab;     // [D][L+1][kw]: partial ranks T_i[s][k]
    const uint8_t *lmin_tab; // [D][kw]: smallest level holding function k
    const LevelInfo *lvl;    // [D][L+1]
    const double *tabd;      // flat FP64 tables
    const float *tabf;       // FP32 copies (same offsets)
    const double *mcoef;     // [nmono]
    const int *mnfac;        // [nmono]
    const int *mfoff;        // [nmono+1]
    const int *mfmode;       // [sum nfac]
    const int *mfpow;        // [sum nfac]
    const int *harm_mono;    // [D] monomial holding the harmonic part of mode i (-1: not split)
    const double *esplit;    // [n_cs] sum over split modes of omega_i s_i^2 (k_i + 1/2)
    unsigned long long *acc; // [n_cs][nvec][acc_words] fixed-point accumulators (entry-major)
    // Entry-major copy of the input vectors in the contraction type, made at
    // the start of each apply: xs[r * xs_stride(xs_nvec) + v] = x_v[r] (the
    // vectors of one compact entry adjacent).  Holds up to xs_nvec vectors;
    // nullptr: the term kernels read x itself.
    const void *xs;
    int xs_nvec;
    FastParams fast;
    // capacities of the per-CTA shared-memory areas (elements)
    int cap;       // each of the two grid ping-pong buffers
    int maxnb;     // term basis tensor
    int matcap;    // per-term 1D matrices
    int vtabcap;   // per-term potential tables
    int *err;      // device error word (0 = fine)
    // term-sharded applies: only processing positions p with p % nparts == part
    int part, nparts;
};

// Host-side description of a problem (after validation).
struct Problem {
    int D = 0, L = 0;
    std::vector<sg_basis> basis;
    std::vector<sg_grid> grids;
    std::vector<double> omega;
    std::vector<double> mcoef;
    std::vector<int> mnfac, mfoff, mfmode, mfpow;
    sg_precision prec = SG_FP64;
};

// Result of the host setup: everything that is uploaded.
struct HostTables {
    int Dpad = 0, pmax = 0, kw = 0;
    int64_t n_terms = 0, n_cs = 0, n_s = 0, n_grid = 0;
    std::vector<uint8_t> levels;     // [n_terms][Dpad]
    std::vector<int> coefs;          // [n_terms]
    std::vector<int> order;          // processing order (Table-2 indices)
    std::vector<int64_t> pcost;      // estimated cost of the p-th processed term
    std::vector<int> rank_tab;       // [D][L+1][kw]
    std::vector<uint8_t> lmin_tab;   // [D][kw]
    std::vector<LevelInfo> lvl;      // [D][L+1]
    std::vector<double> tabd;
    std::vector<int> harm_mono;      // [D]
    std::vector<double> esplit;      // [n_cs]
    // fast path
    bool fast = false;
    int nb1 = 0, nq1 = 0;
    std::vector<int> pair_modes, h1off, goff, ioff, soff, spoff;
    std::vector<double> ftab, fsc;
    double c0const = 0.0;
    int fast_cap = 0, fast_maxnb = 0, fast_matcap = 0;
    std::vector<double> fimg;         // per-term shared-memory images (see FastParams)
    std::vector<long long> fimg_off;  // [n_terms + 1]
    std::vector<long long> fvt_off;   // [n_terms + 1] inner-block table starts (see FastParams::mt_off)
    std::vector<int4> fdesc;          // term records
    std::vector<unsigned> fdesc_off;  // [n_terms+1]
    int64_t franks = 0;               // total compact indices (N_s)
    std::vector<long long> frank_start;  // [n_terms + 1] start of each term's indices
    int fdesccap = 0, fgcap = 0, fnbocap = 1, fn_big = 0, fwork_cta = 0, fwork_warp = 0;
    int slice_vt = 0;                 // slicing target the records were planned with (0: default)
    int warp_vt = 0;                  // warp-form threshold the records were planned with (0: default)
    int fbudget = 0;                  // shared-memory budget the records were planned with
    int cap = 0, maxnb = 0, matcap = 0, vtabcap = 0;
    int64_t flops_per_vec = 0;       // FMA-counted work of one real apply (2 flops per FMA)
};

// Host setup (sg_setup.cpp).  Returns an empty string on success, else the error text.
std::string build_tables(const Problem &p, int smem_budget_bytes, int real_bytes, HostTables *out);

// One-mode Gauss-Hermite rule with Hermite-function-normalised weights.
std::string gauss_hermite(int n, std::vector<double> *x, std::vector<double> *wf);

// Kernel launchers (sg_apply.cu).  Return cudaSuccess or the launch error.
cudaError_t launch_apply(const KParams &kp, bool fp32, const double *x, double *y, int nvec,
                         long long *maxbits, int *lsb_exp, cudaStream_t stream);
cudaError_t launch_index_map(const KParams &kp, int64_t t0, int64_t nt, const int64_t *offsets_dev,
                             int64_t *cs_index, cudaStream_t stream);
size_t apply_smem_bytes(const KParams &kp, bool fp32);
cudaError_t configure_kernels(size_t smem_bytes, bool fp32);

// Fast path (sg_apply_fast.cu, sg_setup.cpp)
std::string build_fast_tables(const Problem &p, HostTables *T);
std::string build_fast_descs(const Problem &p, bool fp32, HostTables *T, int fbudget, int rb);
cudaError_t launch_build_ranks(const KParams &kp, int *ranks, cudaStream_t stream);
// Fills the inner-block tables (FastParams::mtab*) from the records and the FP64 tables.
cudaError_t launch_build_mtab(const KParams &kp, bool fp32, cudaStream_t stream);
size_t fast_smem_bytes(const KParams &kp, bool fp32);
cudaError_t configure_fast_kernels(const KParams &kp, bool fp32);
cudaError_t launch_apply_fast(const KParams &kp, bool fp32, const double *x, int nvec,
                              const long long *maxbits, cudaStream_t stream);

// Many problems per apply (sg_batch.cpp): the term kernels of one problem
// without the max|x| and finalisation passes; those two over all problems.
cudaError_t launch_apply_terms(const KParams &kp, bool fp32, const double *x, const long long *maxbits, int nvec,
                               cudaStream_t stream);
// The passes around the term kernels of one problem: per-vector max|x| bits
// (zeroed first), and y = (accumulated integer) * 2^E + esplit * x, which also
// clears kp.acc.
cudaError_t launch_maxabs(const KParams &kp, const double *x, int nvec, long long *maxbits, cudaStream_t stream);
// kp.xs = the input vectors entry-major in the contraction type (kp.xs set, nvec <= kp.xs_nvec; rows of
// xs_stride(kp.xs_nvec) elements); for a batch, every problem's rows from cs_prefix[j].
cudaError_t launch_stage_x(const KParams &kp, bool fp32, const double *x, int nvec, cudaStream_t stream);
cudaError_t launch_stage_x_batch(bool fp32, const double *x, const long long *cs_prefix, int nprob, int64_t max_ncs,
                                 int nvec, int xs_nvec, void *xs, cudaStream_t stream);
cudaError_t launch_finalize(const KParams &kp, bool fp32, const double *x, double *y, int nvec,
                            const long long *maxbits, cudaStream_t stream);
cudaError_t launch_maxabs_batch(const double *x, const long long *cs_prefix, int nprob, int64_t max_ncs, int nvec,
                                long long *maxbits, cudaStream_t stream);
cudaError_t launch_finalize_batch(const KParams *kps, const long long *cs_prefix, int nprob, int64_t max_ncs,
                                  const double *x, double *y, unsigned long long *acc, const long long *maxbits,
                                  int nvec, bool fp32, cudaStream_t stream);
// Propagation server (sg_server_api.cpp, sg_server.cu): device state of one
// active request's Chebyshev recurrence.  One iteration after Y = H X logs
// norm and energy for requests at k = 0, forms T_{k+1} (T_1 from T_0 when
// k = 0), adds c_{k+1} (-i)^{k+1} T_{k+1} to the partial sum and, on the
// step's last term (k + 1 = K), writes e^{-i Ebar dt} * sum; then k, step advance.
struct ChebState {
    int k, K, step, nsteps;
    double ebar, inv_de;   // (H - ebar) * inv_de maps the spectrum into [-1, 1]
    double cph, sph;       // e^{-i Ebar dt} = cph + i sph
    const double *c;       // device: (2 - delta_k0) J_k(dE dt), k = 0..K
    double *log;           // device: [nsteps][norm, energy]
};
cudaError_t launch_cheb_iteration(ChebState *st, const long long *prefix, int nitems, int64_t total,
                                  const double *X, const double *Y, double *P, double *A, cudaStream_t s);
// Chebyshev spectral interval of a context's H_S (Krylov, as sg_propagate); synchronous.
sg_status chebyshev_bounds(sg_ctx *ctx, cudaStream_t stream, double *emin, double *emax);
// Block Davidson of sg_eigs (method SG_DAVIDSON, same start block and
// iteration) with every application of H_S done by `apply` (x, y device, r
// vectors; x is ready when it is called, y must be complete when it returns).
// Vector algebra runs on `stream`.  nconv receives the converged pairs.
using ApplyFn = std::function<sg_status(const double *x, double *y, int r)>;
sg_status davidson_routed(sg_ctx *ctx, cudaStream_t stream, const ApplyFn &apply, int nev, int block, double tol,
                          int max_it, double *evals, double *resid, double *evecs, int *nconv, std::string *err);
// J_0..J_kmax at x (Miller's backward recurrence).
std::vector<double> bessel_j(int kmax, double x);
// Device bytes sg_create would allocate for a planned context (tables, records, M^B).
int64_t planned_device_bytes(const sg_ctx *ctx);

// Shared-memory partition of one term group of the fast kernels (block form or warp form).
size_t fast_part_bytes(const KParams &kp, bool fp32, bool warp_form);
// Fast-path kernels over many problems of one kernel variant; items are
// (problem, processing position) pairs in cost order.
struct FastBatchGroup {
    const KParams *kps;       // device, one per problem of the batch
    const int2 *items[2];     // device: [0] block form, [1] warp form
    int count[2];
    int part[2];              // bytes per term group
};
cudaError_t configure_fast_batch(const KParams &kp_any, bool fp32, const FastBatchGroup &g);
cudaError_t launch_fast_batch(const KParams &kp_any, bool fp32, const FastBatchGroup &g, const double *x,
                              unsigned long long *acc, const long long *maxbits, const long long *cs_prefix,
                              int nvec, cudaStream_t stream);

}  // namespace sg

struct sg_ctx {
    sg::Problem prob;
    sg::HostTables host;
    sg::KParams kp{};
    int device = 0;
    bool fp32 = false;
    bool has_device = false;  // false for contexts made by sg_plan
    size_t smem_bytes = 0;
    int64_t bytes_device = 0;
    std::vector<void *> allocations;
    double *stage_x = nullptr, *stage_y = nullptr;  // host-API staging (device)
    int64_t stage_elems = 0;
    // apply workspace: fixed-point accumulators and per-vector scale exponents
    unsigned long long *acc = nullptr;
    long long *maxbits = nullptr;
    void *xs = nullptr;       // entry-major input copy (fast path), acc_nvec vectors
    int acc_nvec = 0;
    int plan_version = 0;     // incremented whenever sg_tune installs a plan
    std::string last_error;
};

// Calls with device work run on the device the context was made on: from any
// other current device its kernels would be handed another GPU's pointers.
inline bool sg_on_ctx_device(const sg_ctx *ctx)
{
    int cur = -1;
    return cudaGetDevice(&cur) == cudaSuccess && cur == ctx->device;
}
