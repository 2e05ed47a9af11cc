/*
 * smolyak.h -- C ABI of the GB300 Smolyak operator-action library (libsmolyak.so).
 *
 * The library applies the Smolyak-represented Hamiltonian of arXiv 2111.13655
 * to wavefunctions held in the compact Smolyak basis:
 *
 *     y = H_S x,   H_S = sum_{l in R(l)} D_l  P_l^T  A_l  P_l          (Sec. 2, Eq. (16))
 *
 * with R(l): L-n+1 <= |l| <= L and D_l = (-1)^{L-|l|} C(n-1, L-|l|) (Eq. (8)),
 * P_l the restriction of the compact basis to term l (the mapping table M^B of
 * Sec. 3, Table 2), and A_l the term action of Alg. 1: basis->grid (Eq. (15)),
 * the operator on the term's direct-product grid, grid->basis (Eq. (14)).
 *
 * Conventions shared by every call
 *   - Indices are 0-based.  Modes are numbered 0..D-1.
 *   - Compact vectors have N_cs entries in lexicographic order of the
 *     multi-index k = (k_0..k_{D-1}) with k_0 slowest and k_{D-1} fastest
 *     (the compact ordering of Table 2).  A block of nvec vectors is stored
 *     column after column: x[v*N_cs + i].
 *   - Terms are numbered in the order of Table 2: l_0 varies fastest.
 *   - Basis of every mode: orthonormal Hermite functions
 *       b_k(Q) = sqrt(s) h_k(s (Q - q0))   (the "Hm" basis of Sec. 4),
 *     grid: Gauss-Hermite nodes Q_u = q0 + x_u / s with weights chosen so that
 *     sum_u w_u b_k(Q_u) b_k'(Q_u) = delta_kk' whenever nq >= nb.
 *   - Hamiltonian: H = sum_i omega_i/2 (-d^2/dQ_i^2) + V(Q), V a sparse
 *     polynomial (the Henon-Heiles form of Eq. (18) is one instance).
 *   - A context lives on the CUDA device that was current at sg_create; its
 *     calls with device work return SG_EINVAL when another device is current.
 *   - Every call that takes a `stream` is enqueued on that CUDA stream
 *     (cudaStream_t passed as void*, NULL = legacy default stream) and
 *     returns before the GPU work ends, unless stated otherwise.
 *   - Errors are returned as sg_status; nothing is thrown across the ABI, the
 *     process is never terminated and no device trap is raised.  The text of
 *     the last error of a context is available from sg_last_error(ctx); errors
 *     of sg_create are reported by sg_last_error(NULL) (per calling thread).
 *   - A context may be used by one host thread at a time.
 */
#ifndef SMOLYAK_GB300_H
#define SMOLYAK_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_ctx sg_ctx;

typedef enum {
    SG_OK = 0,
    SG_EINVAL = 1,       /* invalid argument (sizes, rules, pointers, precision)      */
    SG_ENOMEM = 2,       /* host or device allocation failed                         */
    SG_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed               */
    SG_ENOCONV = 4,      /* an iterative solver did not converge in max_it            */
    SG_ETIMEOUT = 5,     /* a bounded device wait ran out                             */
    SG_EBUDGET = 6,      /* request exceeds the device-memory budget                  */
    SG_EUNSUPPORTED = 7  /* valid request outside this build's limits (see below)     */
} sg_status;

typedef enum { SG_FP64 = 0, SG_MIXED = 1, SG_DF64 = 2 } sg_precision;

typedef enum { SG_LANCZOS = 0, SG_DAVIDSON = 1 } sg_eig_method;

/* Primitive basis of one mode: nb(l) = nb_A + nb_B * l functions at level l
 * (the level->size rule N_l = A + B l of Sec. 2), Hermite functions centred at
 * q0 with scale factor `scale` (> 0).  Requires nb_A >= 1, nb_B >= 0. */
typedef struct { int nb_A, nb_B; double q0, scale; } sg_basis;

/* Grid of one mode: nq(l) = nq_A + nq_B * l Gauss-Hermite points at level l.
 * Requires nq(l) >= nb(l) for every level (nq_A >= nb_A, nq_B >= nb_B). */
typedef struct { int nq_A, nq_B; } sg_grid;

/* Sparse polynomial potential.  Monomial m contributes
 *     coef[m] * prod_{f = off_m}^{off_m + nfac[m] - 1} Q_{mode[f]}^{power[f]},
 * off_m = nfac[0] + ... + nfac[m-1]: the factors of all monomials are stored
 * back to back in mode/power.  nfac[m] = 0 is a constant.  power >= 1. */
typedef struct {
    int nterms;
    const double *coef;
    const int *nfac;
    const int *mode;
    const int *power;
} sg_poly;

/* H = sum_i omega[i]/2 (-d^2/dQ_i^2) + V(Q).  omega: D host doubles. */
typedef struct {
    const double *omega;
    sg_poly V;
} sg_hamiltonian;

/*
 * sg_create -- build a context for one Smolyak problem (Sec. 3: the three
 * objects -- terms, compact basis, grid -- and the mapping table M^B).
 *   D      number of modes, 1 <= D <= 32.
 *   L      Smolyak level (L^B = L^G = L, Sec. 2), 0 <= L.
 *   basis  D host structs; grids: D host structs.
 *   H      Hamiltonian; all arrays are host memory, copied (caller keeps ownership).
 *   prec   SG_FP64: every step in FP64.  SG_MIXED: per-term contractions and
 *          the grid multiply in FP32, accumulation of the compact result in
 *          FP64 (exact fixed point).  SG_DF64: the contractions in double-float
 *          arithmetic (each value an unevaluated sum of two FP32 numbers,
 *          about 48 significant bits, on the FP32 pipes), accumulation as for
 *          SG_FP64; FP64-class results (relative error about 1e-14 against
 *          1e-16), for problems on the fast path only (V with monomials of one
 *          mode or of two neighbouring modes of a chain; else
 *          SG_EUNSUPPORTED); not accepted by sg_batch_create or the server.
 *   out    receives the context (owned by the caller, release with sg_destroy).
 * Setup runs on the host plus synchronous uploads on the current device.
 * The context keeps on the device M^B (4 bytes per term basis function), the
 * per-term records, images and 1D tables, and, on the fast path, the
 * inner-block tables of every term with a grid (4 bytes per value for
 * SG_MIXED, 8 for SG_FP64 and SG_DF64; 6.65 / 13.1 GB at D=12 L=10,
 * nq = l+2).  sg_size reports the total.
 * Limits of this build (SG_EUNSUPPORTED): nb(L), nq(L) <= 32, N_cs < 2^31,
 * at most 256 monomials with at most 8 factors each, powers <= 16.
 */
sg_status sg_create(int D, int L, const sg_basis *basis, const sg_grid *grids,
                    const sg_hamiltonian *H, sg_precision prec, sg_ctx **out);

/*
 * sg_plan -- the host half of sg_create: validates the problem and builds the
 * terms, the compact ranking and the 1D tables (Sec. 3's three objects) without
 * touching any GPU.  The context answers sg_size, sg_term_levels,
 * sg_compact_rank and sg_mode_tables (e.g. to size a problem before admitting
 * it); calls that need device state return SG_EINVAL.  Release with sg_destroy.
 */
sg_status sg_plan(int D, int L, const sg_basis *basis, const sg_grid *grids,
                  const sg_hamiltonian *H, sg_precision prec, sg_ctx **out);

/* Sizes: n_cs = N_cs (compact basis), n_terms = N_st, n_s = N_s (sum of term
 * basis sizes, Sec. 2, Eq. (11)), n_grid = sum of term grid sizes, bytes_device =
 * device memory held by the context (for a context made by sg_plan: the tables
 * sg_create would allocate for the same problem, without the apply workspace,
 * which grows with the block size).  Any pointer may be NULL. */
sg_status sg_size(const sg_ctx *ctx, int64_t *n_cs, int64_t *n_terms, int64_t *n_s,
                  int64_t *n_grid, int64_t *bytes_device);

/*
 * sg_apply_H -- y = H_S x for nvec real vectors (Eq. (16), every term by Alg. 1).
 *   x, y   DEVICE pointers, N_cs * nvec doubles each, column after column.
 *          y is overwritten; x and y must not overlap.
 *   nvec   >= 1.  A complex vector is passed as two real vectors.
 * Enqueued on `stream`; the result is ready when the stream reaches it.
 * The first call with a larger nvec than before synchronises `stream` and
 * allocates the context's workspace for that many vectors: the fixed-point
 * accumulators (1 word per element for SG_MIXED, 4 otherwise) and, on the
 * fast path, an entry-major copy of x in the contraction type (rows of nvec
 * rounded up to 4 values), which every apply rewrites before its terms
 * gather from it.  Calls on one context must be ordered (one stream, or
 * synchronised streams): they share that workspace.
 */
sg_status sg_apply_H(sg_ctx *ctx, const double *x, double *y, int nvec, void *stream);

/*
 * sg_apply_H_host -- the same operation on HOST buffers: copies x to the
 * device, applies H_S, copies y back, and returns when y is written.
 *   x_host, y_host: N_cs * nvec doubles each (pinned memory gives the fastest copies).
 * Device staging buffers are owned by the context and reused across calls.
 */
sg_status sg_apply_H_host(sg_ctx *ctx, const double *x_host, double *y_host, int nvec,
                          void *stream);

/*
 * Term-sharded apply: the terms of Eq. (16) are independent (the term loop of
 * Alg. 1; the paper's parallel scheme 1, Alg. 2, splits them over MPI ranks
 * and sums the partial results).  Part `part` of `nparts` takes the terms at
 * processing positions p = part (mod nparts) -- the processing order is by
 * decreasing cost, so the parts are balanced -- and adds their contributions
 * exactly into fixed-point accumulators; summing the accumulators of all parts
 * as 64-bit integers (wrapping) and finishing gives bitwise the result of
 * sg_apply_H, whatever nparts.  A multi-GPU apply runs one part per GPU (each
 * with its own context of the same problem and the same x), one integer
 * all-reduce (sum) of acc, and sg_apply_H_finish.
 *
 * sg_apply_H_part -- adds the part's contributions for nvec vectors into acc.
 *   x    DEVICE, as for sg_apply_H.
 *   acc  DEVICE, N_cs * nvec * w int64 words (w = 1 for SG_MIXED, 4 for SG_FP64),
 *        entry-major (entry r, vector v at (r * nvec + v) * w); zero before the
 *        first part is added (cudaMemset), accumulated into by each part.
 * sg_apply_H_finish -- y = H_S x from the summed accumulators of all parts
 *   (and the harmonic part applied in the compact basis); clears acc to zero.
 *   x, y as for sg_apply_H (x the same vectors the parts were given).
 * sg_part_size -- the terms of a part and their summed cost estimate (host;
 *   also on contexts made by sg_plan).  Any output may be NULL.
 * Both device calls are enqueued on `stream`.
 */
sg_status sg_apply_H_part(sg_ctx *ctx, const double *x, int nvec, int part, int nparts, int64_t *acc,
                          void *stream);
sg_status sg_apply_H_finish(sg_ctx *ctx, const double *x, int64_t *acc, double *y, int nvec, void *stream);
sg_status sg_part_size(const sg_ctx *ctx, int part, int nparts, int64_t *n_terms, int64_t *cost);

/*
 * sg_apply_H_noalloc -- the operation of sg_apply_H, with the same arguments
 * and results, for callers that may not allocate device memory when they
 * apply H (e.g. a process whose device memory is all held by another
 * allocator, or a loop that cannot take the synchronisation a cudaMalloc may
 * bring).  It is not part of the method of the paper, which has no counterpart.
 *   The fixed-point accumulators and per-vector exponents that sg_apply_H
 *   keeps in context-owned device memory come here from one array of
 *   SG_NOALLOC_SCRATCH_BYTES compiled into the library; every GPU that loads
 *   the library holds it until the process exits.  The call allocates nothing.
 *   Limits: nvec <= SG_NOALLOC_MAX_NVEC and nvec * N_cs <= SG_NOALLOC_MAX_ELEMS
 *   for SG_FP64 contexts (four accumulator words per element), or
 *   SG_NOALLOC_MAX_ELEMS_MIXED for SG_MIXED contexts (one word per element);
 *   larger requests return SG_EUNSUPPORTED with the limits in sg_last_error.
 *   The context's device must be the current device (else SG_EINVAL).  The
 *   first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) and remembers it; make that first call before any
 *   stream capture.  Each call clears the part of the array it uses on
 *   `stream` first.  All calls on one device share the array: calls whose GPU
 *   work overlaps (other streams, threads or contexts) race and give wrong
 *   results; order them.  x, y: DEVICE, as for sg_apply_H.  Enqueued on `stream`.
 */
#define SG_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)
#define SG_NOALLOC_MAX_NVEC 64
#define SG_NOALLOC_MAX_ELEMS 524272
#define SG_NOALLOC_MAX_ELEMS_MIXED 2097088
sg_status sg_apply_H_noalloc(sg_ctx *ctx, const double *x, double *y, int nvec, void *stream);

/*
 * Batches: y_j = H_S^(j) x_j for many independent problems j in one apply
 * (Eq. (16) per problem).  The terms of every problem are independent work
 * (Sec. 3: the term loop of Alg. 1 and its parallel schemes), so the terms of
 * all problems that share a kernel variant run in one launch per form (block /
 * warp), ordered by estimated cost over all problems; small problems fill the
 * gaps that large ones leave.  Problems outside the fast path (potentials with
 * monomials over three or more modes) get one launch each.
 *
 * sg_batch_create -- n (1..65535) contexts made by sg_create on the current
 *   device, all of one precision (else SG_EINVAL; SG_DF64 contexts:
 *   SG_EUNSUPPORTED).  The batch borrows their
 *   device tables: destroy it before any of them.  The contexts' own
 *   workspaces are not used, so sg_apply_H on a member stays valid.
 * sg_batch_size -- total N_cs and terms over the problems; kernel launches
 *   of one sg_apply_H_batch.
 * sg_apply_H_batch -- x, y: DEVICE, problem after problem, problem j's nvec
 *   vectors (each N_cs^(j) doubles, column after column) starting at
 *   nvec * (N_cs^(0) + ... + N_cs^(j-1)).  y is overwritten; x and y must not
 *   overlap.  1 <= nvec <= 65535.  Results are bitwise those of sg_apply_H
 *   on each context.  The batch owns its workspace (fixed-point accumulators,
 *   32 bytes per vector entry), grown on the first call with a larger nvec.
 *   Enqueued on `stream`.
 */
typedef struct sg_batch sg_batch;
sg_status sg_batch_create(sg_ctx *const *ctxs, int n, sg_batch **out);

sg_status sg_batch_size(const sg_batch *b, int64_t *n_cs_total, int64_t *n_terms_total, int *launches_per_apply);
sg_status sg_apply_H_batch(sg_batch *b, const double *x, double *y, int nvec, void *stream);
const char *sg_batch_last_error(const sg_batch *b);
void sg_batch_destroy(sg_batch *b);

/*
 * sg_tune -- measured choice of the term schedule of a context's fast path
 * (no counterpart in the paper, whose scheme balances MPI ranks by timing).
 * Three knobs of the plan are searched one after another, each candidate
 * timed on nvec-vector applies (median of three after one warm-up) on
 * `stream`, the fastest kept:
 *   - the slicing target (1, 2, 4): a term whose grid leaves room for fewer
 *     than that many vectors per chunk is sliced over its leading outer
 *     positions, else it runs unsliced in more, smaller chunks;
 *   - the block/warp split (1, 2, 4): terms that fit a quarter of a block's
 *     shared memory with that many vectors per chunk run one per warp;
 *   - the shared-memory budget of a block, in KB (52, 70, 104 for SG_MIXED;
 *     70, 104 for SG_FP64 and SG_DF64): more vectors per chunk, fewer
 *     resident blocks.
 * Only the term records, the split and the work-area capacities change;
 * results change by rounding only.  Synchronous; allocates and frees
 * 2 * nvec * N_cs doubles of scratch.  No other work may use the context
 * meanwhile.  A batch made from the context before sg_tune refuses to apply
 * (SG_EINVAL) until it is recreated.
 *   nvec 1..64; slice_vt (out, may be NULL): the slicing target kept (0 when
 *   the context uses the generic kernel, which has no schedule to choose);
 *   ms (out, may be NULL): its time per apply.
 * sg_tune_plan -- the plan a context uses now (tuned or default): slicing
 *   target, block/warp split, shared-memory budget in KB (zeros for the
 *   generic kernel).  Any pointer may be NULL.
 */
sg_status sg_tune(sg_ctx *ctx, int nvec, int *slice_vt, double *ms, void *stream);
sg_status sg_tune_plan(const sg_ctx *ctx, int *slice_vt, int *warp_vt, int *smem_kb);

/*
 * Request server: continuous batching of Chebyshev propagation requests
 * (the propagator of sg_propagate: Sec. 3, Sec. 5) and eigen requests (the
 * block Davidson of sg_eigs: Sec. 3, Sec. 4) of different D, L and basis
 * sizes on one device.  The caller submits requests and drives the engine
 * with sg_server_progress; all calls on one server from one host thread at a
 * time, with the server's device current.  Each eigen request runs its
 * solver on a host thread of its own (vector algebra on its own stream); its
 * block applications of H_S are handed to the engine, whose iterations then
 * apply every waiting block and every propagation request's Chebyshev vector
 * in one sg_apply_H_batch (an eigen block occupies (block + 1) / 2 two-vector
 * slots of the batch).  With eigen requests active an iteration waits (at
 * most 600 s, else SG_ETIMEOUT) until each has handed over its next block or
 * finished.
 *
 * Each engine iteration retires finished requests, admits queued requests
 * first come first served while their planned device memory fits the budget,
 * then applies H_S to every active request's current Chebyshev vector in one
 * sg_apply_H_batch and advances every recurrence by one term in one fused
 * kernel.  Requests that arrive while others run join at the next iteration.
 * A request's results are bitwise the same alone and in any mix (its applies,
 * updates and logged sums do not depend on the other requests).
 *
 * sg_server_create -- precision of every request's contexts (SG_FP64 or
 *   SG_MIXED; else SG_EINVAL); hbm_budget_bytes:
 *   the planned device memory of the active requests never exceeds it
 *   (context tables, M^B, batch items, four state vectors, batch and context
 *   workspaces, logs).  Transient set-up buffers of an admission (the
 *   spectral-bound Krylov run, about 80 vectors) are not counted.
 * sg_server_submit -- copies the request (the caller's arrays may be freed on
 *   return), plans it on the host, and queues it; *id identifies it.
 *   SG_EBUDGET if the request alone needs more than the budget.
 *   Initial state: psi0 (host, 2 * N_cs doubles: real part, imaginary part;
 *   N_cs from sg_plan + sg_size, compact order) or, if psi0 is NULL, the real
 *   product state of `factors` (as sg_product_state, leading dimension ld).
 *   Logs: <psi|psi> and <psi|H psi>/<psi|psi> at the start of each step.
 * sg_server_submit_eigs -- copies and plans an eigen request and queues it;
 *   SG_EBUDGET if it alone needs more than the budget (context tables, M^B,
 *   its batch slots, the Davidson basis of max(3 nev, nev + 6 block) vectors
 *   and its images, Ritz vectors, eigenvectors).
 * sg_server_progress -- runs up to max_iters engine iterations (fewer if
 *   nothing is active); returns the numbers of active and queued requests.
 *   Synchronous.
 * sg_server_query -- state (sg_request_state), N_cs and steps done of a
 *   request (for an eigen request: block applications so far).
 * sg_server_result -- a finished request's psi (host, 2 * N_cs), logs (host,
 *   nsteps each), times[0] = admission - submission, times[1] = completion -
 *   submission (seconds, steady clock); any output may be NULL.
 * sg_server_eig_result -- a finished eigen request's eigenvalues (host, nev,
 *   ascending), residual norms (host, nev), eigenvectors (host, nev * N_cs,
 *   only if the request asked for them), times as sg_server_result, and the
 *   number of converged pairs; any output may be NULL.  Returns SG_ENOCONV
 *   (outputs written) when fewer than nev pairs converged in max_it.
 * sg_server_stats -- engine iterations, real-vector applications of H_S so far
 *   (2 per propagation request per iteration, the vectors of each eigen block),
 *   planned bytes of the active requests.
 */
typedef struct sg_server sg_server;
typedef enum { SG_REQ_QUEUED = 0, SG_REQ_ACTIVE = 1, SG_REQ_DONE = 2, SG_REQ_FAILED = 3 } sg_request_state;
typedef struct {
    int D, L;
    const sg_basis *basis;     /* D entries */
    const sg_grid *grids;      /* D entries */
    const sg_hamiltonian *H;
    const double *psi0;        /* host, 2 * N_cs, or NULL */
    const double *factors;     /* host, D * ld, used when psi0 is NULL */
    int ld;
    double dt;
    int nsteps, order;         /* steps of length dt; Chebyshev order (reduced as in sg_propagate) */
} sg_prop_request;
/* Eigen request: the nev lowest eigenpairs of H_S by the block Davidson of
 * sg_eigs (method SG_DAVIDSON; Sec. 3's time-independent solver), block 1..8
 * (<= 0: min(nev, 8)), convergence ||H x - theta x|| <= tol max(1, |theta|),
 * at most max_it iterations; want_vectors != 0 keeps the eigenvectors for
 * sg_server_eig_result. */
typedef struct {
    int D, L;
    const sg_basis *basis;     /* D entries */
    const sg_grid *grids;      /* D entries */
    const sg_hamiltonian *H;
    int nev, block;
    double tol;
    int max_it;
    int want_vectors;
} sg_eig_request;
sg_status sg_server_create(sg_precision prec, int64_t hbm_budget_bytes, sg_server **out);
sg_status sg_server_submit(sg_server *s, const sg_prop_request *req, int64_t *id);
sg_status sg_server_submit_eigs(sg_server *s, const sg_eig_request *req, int64_t *id);
sg_status sg_server_progress(sg_server *s, int max_iters, int *n_active, int *n_queued);
sg_status sg_server_query(const sg_server *s, int64_t id, int *state, int64_t *n_cs, int *steps_done);
sg_status sg_server_result(sg_server *s, int64_t id, double *psi_host, double *norm_log, double *energy_log,
                           double *times);
sg_status sg_server_eig_result(sg_server *s, int64_t id, double *evals, double *resid, double *evecs_host,
                               double *times, int *converged);
sg_status sg_server_stats(const sg_server *s, int64_t *iterations, int64_t *applications, int64_t *bytes_in_use);
const char *sg_server_last_error(const sg_server *s);
void sg_server_destroy(sg_server *s);

/*
 * sg_term_levels -- levels l of terms [t0, t0+nt) in Table-2 order, D ints per
 * term, into levels_host (nt*D ints), and their combination coefficients D_l
 * (Eq. (8)) into coef_host (nt ints, may be NULL).
 */
sg_status sg_term_levels(const sg_ctx *ctx, int64_t t0, int64_t nt, int *levels_host,
                         int *coef_host);

/*
 * sg_index_map -- the mapping table M^B (Sec. 3, Table 2) for terms
 * [t0, t0+nt) in Table-2 order, computed on the device by the same index
 * arithmetic the operator action uses.
 *   offsets_host  nt+1 int64 (host, out): start of each term's list, relative
 *                 to the first listed term (offsets_host[0] = 0).
 *   cs_index_dev  DEVICE int64 array of offsets_host[nt] entries (out): compact
 *                 index of each basis function of the term, k_0 fastest inside
 *                 the term (Table 2's i^s order).  Call once with
 *                 cs_index_dev = NULL to obtain the offsets (and the size).
 * Synchronises `stream` before returning.
 */
sg_status sg_index_map(sg_ctx *ctx, int64_t t0, int64_t nt, int64_t *offsets_host,
                       int64_t *cs_index_dev, void *stream);

/*
 * sg_compact_rank -- position of multi-indices in the compact basis (Table 2's
 * compact ordering), computed on the host with the same partial-rank tables the
 * GPU uses.  k: n*D host ints; rank: n host int64 (out), -1 for a k outside the
 * compact basis.
 */
sg_status sg_compact_rank(const sg_ctx *ctx, const int *k, int64_t n, int64_t *rank);

/*
 * sg_mode_tables -- host copies of the 1D tables of one mode at one level:
 *   B[u*nb+k]  = b_k(Q_u)                 (basis -> grid, Eq. (15))
 *   BW[k*nq+u] = w_u b_k(Q_u)             (grid -> basis, Eq. (14))
 *   K[k*nb+k'] = -omega/2 sum_u w_u b_k(Q_u) b_k''(Q_u)   (kinetic in the basis)
 *   Q[u]       = Q_u                      (grid coordinates)
 * nb, nq receive the sizes; any output pointer may be NULL.
 */
sg_status sg_mode_tables(const sg_ctx *ctx, int mode, int level, int *nb, int *nq,
                         double *B, double *BW, double *K, double *Q);

/*
 * sg_device_error -- read and clear the context's device error word (0 when
 * every kernel found its term within the capacities fixed at sg_create; a
 * non-zero code names the capacity a kernel refused to exceed -- the kernel
 * then skipped that term instead of touching memory out of bounds).
 * Synchronous: waits for all work on the current device.
 */
sg_status sg_device_error(sg_ctx *ctx, int *code);

/*
 * sg_eigs -- lowest nev eigenpairs of H_S (the time-independent solvers of Sec. 3:
 * the Davidson method; a Lanczos-type method).  Every operator application is
 * sg_apply_H on a block of vectors; the basis, its orthogonalisation (block
 * Gram-Schmidt twice + Cholesky QR), Ritz vectors and residuals are FP64 on
 * the device; the projected matrix is diagonalised on the host.
 *   method  SG_DAVIDSON: block Davidson, diagonal preconditioner
 *           (E_k - theta)^-1 with E_k the harmonic energies of the split modes
 *           (none when no mode is split), restart at max(3 nev, nev + 6 block)
 *           vectors.  SG_LANCZOS: block Krylov with full reorthogonalisation and
 *           Rayleigh-Ritz, at most 320 basis vectors; a block of size >= the
 *           largest multiplicity resolves degenerate eigenvalues.
 *   block   1..8 vectors per operator application (<= 0: min(nev, 8)).
 *   tol     convergence when ||H x - theta x|| <= tol * max(1, |theta|) for the
 *           nev lowest Ritz pairs.  max_it: iterations (blocks added).
 *   evals   host, nev (out, ascending); resid: host, nev residual norms (may be NULL);
 *   evecs   DEVICE, nev * N_cs (out; may be NULL).
 * Synchronous.  SG_ENOCONV when fewer than nev pairs converged (evals, resid and
 * evecs then hold the current approximations).  Allocates its workspace
 * (device memory of about 2 * max(3 nev, nev + 6 block) vectors for Davidson).
 * With a SG_MIXED context the applications are FP32-accurate; use
 * sg_eigs_refine with a SG_FP64 context of the same problem to refine.
 */
sg_status sg_eigs(sg_ctx *ctx, int nev, int method, int block, double tol, int max_it, double *evals,
                  double *evecs, double *resid, void *stream);

/*
 * sg_eigs_refine -- block Davidson started from the nev given vectors (DEVICE,
 * nev * N_cs, in/out), on ctx's precision; used with a SG_FP64 context to bring
 * eigenpairs converged with mixed-precision applications to FP64 accuracy.
 * evals, resid: host (out).  Synchronous.
 */
sg_status sg_eigs_refine(sg_ctx *ctx, int nev, double *evecs, double *evals, double *resid, double tol,
                         int max_it, void *stream);

/*
 * sg_propagate -- nsteps Chebyshev steps of length dt of i d/dt psi = H_S psi
 * (the Chebyshev propagator of Sec. 3 and Sec. 5).  Per step:
 *   psi(t+dt) = e^{-i Ebar dt} sum_{k=0}^{K} (2 - delta_k0) (-i)^k J_k(dE dt) T_k((H - Ebar)/dE) psi(t),
 * Ebar, dE the centre and half-width of the spectral interval, estimated once
 * from a 40-vector Krylov run and widened by the extreme Ritz residuals and 5%
 * of the range.  K = order, reduced to the last k whose Bessel weight J_k is
 * above 1e-17.  J_k by Miller's backward recurrence.
 *   psi     DEVICE, 2 * N_cs doubles: real part, then imaginary part (in/out).
 *   norm_log, energy_log: host, nsteps (may be NULL): <psi|psi> and
 *           <psi|H|psi>/<psi|psi> at the start of each step.
 * Synchronous.
 */
sg_status sg_propagate(sg_ctx *ctx, double *psi, double dt, int nsteps, int order, double *norm_log,
                       double *energy_log, void *stream);

/*
 * sg_product_state -- psi_k = prod_i factors[i * ld + k_i] over the compact basis
 * (compact order), on the host (out_host: N_cs doubles).  ld >= nb(L) of every
 * mode.  Builds e.g. the displaced Gaussian (coherent state) of the propagation
 * examples from its 1D Hermite-function coefficients.
 */
sg_status sg_product_state(const sg_ctx *ctx, const double *factors, int ld, double *out_host);

/*
 * sg_measure_peak -- measured arithmetic throughput of the current device (no
 * counterpart in the paper; it supplies the denominators of the roofline
 * fractions of the operator action, which is bound by CUDA-core arithmetic).
 * Every SM runs 32 warps of register-resident multiply-add chains for about
 * `seconds` (0 < seconds <= 60); the result counts 2 flops per multiply-add.
 *   kind        SG_PEAK_FP32: scalar FP32 fma; SG_PEAK_FP32X2: the packed
 *               two-lane FP32 fma (fma.rn.f32x2, two multiply-adds per
 *               instruction); SG_PEAK_FP64: FP64 fma.
 *   flops_per_s host (out): achieved flop/s of the timed launch.
 *   sms         host (out, may be NULL): the device's multiprocessor count.
 * Synchronous (CUDA events on `stream`).  Allocates and frees 8 bytes per
 * launched thread (about 1.2 MB on a 152-SM device).
 */
typedef enum { SG_PEAK_FP32 = 0, SG_PEAK_FP32X2 = 1, SG_PEAK_FP64 = 2 } sg_peak_kind;
sg_status sg_measure_peak(int kind, double seconds, double *flops_per_s, int *sms, void *stream);

/* Text of the last error of ctx (or of the calling thread's last sg_create
 * when ctx is NULL).  Never NULL; valid until the next call on ctx. */
const char *sg_last_error(const sg_ctx *ctx);

/* Release the context and every device buffer it owns.  NULL is a no-op.
 * The caller must ensure no work using ctx is still running on the GPU. */
void sg_destroy(sg_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SMOLYAK_GB300_H */
