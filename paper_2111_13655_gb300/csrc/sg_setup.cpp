// Host setup of libsmolyak: 1D tables, terms, compact ranking, capacities.
//
// Everything here runs once per sg_create.  The formulas follow the paper
// (arXiv 2111.13655):
//   - terms l in R(l): L-n+1 <= |l| <= L, coefficient D_l = (-1)^{L-|l|} C(n-1, L-|l|)
//     (Sec. 2, Eq. (8)), numbered in Table-2 order (l_0 varies fastest);
//   - level -> size rules nb(l) = A + B l, nq(l) = A' + B' l (Sec. 2);
//   - compact basis = union of the term boxes, lexicographic with mode 0
//     slowest (Table 2), ranked combinatorially instead of through a stored
//     mapping table M^B (Sec. 3);
//   - 1D transfer matrices of Eqs. (14)/(15) on Gauss-Hermite grids.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "sg_internal.h"

namespace sg {

namespace {

// Orthonormal Hermite functions h_0..h_{n-1} at x (stable normalised recurrence).
void hermite_fns(int n, double x, double *h)
{
    const double pi_m14 = 0.75112554446494248286;  // pi^(-1/4)
    h[0] = pi_m14 * std::exp(-0.5 * x * x);
    if (n > 1) h[1] = std::sqrt(2.0) * x * h[0];
    for (int k = 2; k < n; k++)
        h[k] = std::sqrt(2.0 / k) * x * h[k - 1] - std::sqrt((k - 1.0) / k) * h[k - 2];
}

int64_t binom(int n, int k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

int nsz(int A, int B, int l) { return A + B * l; }

}  // namespace

// Gauss-Hermite rule: nodes are the n zeros of h_n, bracketed by a sign scan of
// h_n over (-sqrt(2n+1)-1/2, sqrt(2n+1)+1/2), bisected and Newton-polished with
// h_n' = sqrt(2n) h_{n-1} - x h_n; weights in the Hermite-function
// normalisation from the Christoffel function, wf_u = 1 / sum_{k<n} h_k(x_u)^2
// (so that sum_u wf_u h_k(x_u) h_k'(x_u) = delta_kk' for k, k' < n).
std::string gauss_hermite(int n, std::vector<double> *x, std::vector<double> *wf)
{
    x->assign(n, 0.0);
    wf->assign(n, 0.0);
    if (n < 1 || n > 64) return "gauss_hermite: n out of range";
    std::vector<double> h(n + 1);
    auto hn = [&](double t) { hermite_fns(n + 1, t, h.data()); return h[n]; };
    const double a = std::sqrt(2.0 * n + 1.0) + 0.5;
    const int scan = 400 * n;
    auto polish = [&](double r) {
        for (int it = 0; it < 3; it++) {
            hermite_fns(n + 1, r, h.data());
            double d = std::sqrt(2.0 * n) * h[n - 1] - r * h[n];
            if (d != 0.0 && h[n] != 0.0) r -= h[n] / d;
        }
        return r;
    };
    int found = 0;
    double t0 = -a, f0 = hn(t0);
    for (int i = 1; i <= scan && found < n; i++) {
        double t1 = -a + 2.0 * a * i / scan, f1 = hn(t1);
        if (f1 == 0.0) {                 // the scan landed on a zero
            (*x)[found++] = polish(t1);
        } else if (f0 != 0.0 && (f0 < 0) != (f1 < 0)) {
            double lo = t0, hi = t1, flo = f0;
            for (int it = 0; it < 200 && hi - lo > 1e-15 * (1 + std::fabs(lo)); it++) {
                double mid = 0.5 * (lo + hi), fm = hn(mid);
                if (fm == 0.0) { lo = hi = mid; break; }
                if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
            }
            (*x)[found++] = polish(0.5 * (lo + hi));
        }
        t0 = t1; f0 = f1;
    }
    if (found != n) return "gauss_hermite: root bracketing failed";
    if (n % 2 == 1) (*x)[n / 2] = 0.0;
    for (int u = 0; u < n; u++) {  // enforce the exact symmetry of the rule
        double s = 0.5 * ((*x)[n - 1 - u] - (*x)[u]);
        if (u < n / 2) { (*x)[u] = -s; (*x)[n - 1 - u] = s; }
    }
    for (int u = 0; u < n; u++) {
        hermite_fns(n, (*x)[u], h.data());
        double s = 0.0;
        for (int k = 0; k < n; k++) s += h[k] * h[k];
        (*wf)[u] = 1.0 / s;
    }
    return "";
}

std::string build_tables(const Problem &p, int smem_budget, int rb, HostTables *out)
{
    HostTables &T = *out;
    const int D = p.D, L = p.L;
    char buf[256];

    // ---------------- per (mode, level) 1D tables ----------------
    T.pmax = 0;
    for (int m = 0; m < (int)p.mnfac.size(); m++) {
        // largest total power of one mode inside one monomial
        int pw[kMaxD] = {0};
        for (int f = p.mfoff[m]; f < p.mfoff[m + 1]; f++) pw[p.mfmode[f]] += p.mfpow[f];
        for (int i = 0; i < D; i++) T.pmax = std::max(T.pmax, pw[i]);
    }
    T.lvl.assign((size_t)D * (L + 1), LevelInfo{});
    T.tabd.clear();
    for (int i = 0; i < D; i++) {
        const double q0 = p.basis[i].q0, s = p.basis[i].scale;
        for (int l = 0; l <= L; l++) {
            LevelInfo &li = T.lvl[(size_t)i * (L + 1) + l];
            li.nb = nsz(p.basis[i].nb_A, p.basis[i].nb_B, l);
            li.nq = nsz(p.grids[i].nq_A, p.grids[i].nq_B, l);
            const int nb = li.nb, nq = li.nq;
            std::vector<double> xg, wf;
            std::string e = gauss_hermite(nq, &xg, &wf);
            if (!e.empty()) return e;
            std::vector<double> h(nb + 2), B(nq * nb), BW(nb * nq), D2(nq * nb), Q(nq), W(nq);
            for (int u = 0; u < nq; u++) {
                hermite_fns(nb + 2, xg[u], h.data());
                W[u] = wf[u] / s;
                Q[u] = q0 + xg[u] / s;
                for (int k = 0; k < nb; k++) {
                    B[u * nb + k] = std::sqrt(s) * h[k];
                    // b_k'' from the ladder form of d/dx applied twice:
                    //   h_k'' = 1/2 sqrt(k(k-1)) h_{k-2} - (k+1/2) h_k + 1/2 sqrt((k+1)(k+2)) h_{k+2}
                    double d2 = -(k + 0.5) * h[k] + 0.5 * std::sqrt((k + 1.0) * (k + 2.0)) * h[k + 2];
                    if (k >= 2) d2 += 0.5 * std::sqrt(k * (k - 1.0)) * h[k - 2];
                    D2[u * nb + k] = std::sqrt(s) * s * s * d2;
                }
            }
            for (int k = 0; k < nb; k++)
                for (int u = 0; u < nq; u++) BW[k * nq + u] = W[u] * B[u * nb + k];
            li.offB = (int)T.tabd.size();
            T.tabd.insert(T.tabd.end(), B.begin(), B.end());
            li.offBW = (int)T.tabd.size();
            T.tabd.insert(T.tabd.end(), BW.begin(), BW.end());
            li.offK = (int)T.tabd.size();
            for (int k = 0; k < nb; k++)
                for (int kp = 0; kp < nb; kp++) {
                    double acc = 0.0;
                    for (int u = 0; u < nq; u++) acc += BW[k * nq + u] * D2[u * nb + kp];
                    T.tabd.push_back(-0.5 * p.omega[i] * acc);
                }
            li.offQ = (int)T.tabd.size();
            T.tabd.insert(T.tabd.end(), Q.begin(), Q.end());
            li.offMu = (int)T.tabd.size();
            for (int pw = 0; pw <= T.pmax; pw++) {
                double acc = 0.0;
                for (int u = 0; u < nq; u++) acc += W[u] * B[u * nb] * B[u * nb] * std::pow(Q[u], pw);
                T.tabd.push_back(acc);
            }
            // single-mode potential factors in the basis: M_p = B^T W diag(Q^p) B
            li.offM = (int)T.tabd.size();
            for (int pw = 1; pw <= std::max(T.pmax, 1); pw++)
                for (int k = 0; k < nb; k++)
                    for (int kp = 0; kp < nb; kp++) {
                        double acc = 0.0;
                        for (int u = 0; u < nq; u++) acc += BW[k * nq + u] * std::pow(Q[u], pw) * B[u * nb + kp];
                        T.tabd.push_back(acc);
                    }
        }
    }
    // Harmonic split.  For a mode centred at q0 = 0 with scale s, the basis
    // functions are eigenfunctions of -omega/2 d^2/dQ^2 + omega s^4/2 Q^2 with
    // eigenvalue omega s^2 (k+1/2), at every level and on every grid with
    // nq >= nb.  When the potential holds exactly that quadratic monomial, the
    // pair is diagonal in every term, and the combination identity
    // sum_{l in R(l), l >= k} D_l = 1 adds it once: it is taken out of the
    // term actions and applied in the compact basis.
    T.harm_mono.assign(D, -1);
    for (int i = 0; i < D; i++) {
        if (p.basis[i].q0 != 0.0 || !(p.omega[i] > 0.0)) continue;
        const double s = p.basis[i].scale;
        const double want = 0.5 * p.omega[i] * s * s * s * s;
        for (int m = 0; m < (int)p.mnfac.size(); m++)
            if (p.mnfac[m] == 1 && p.mfmode[p.mfoff[m]] == i && p.mfpow[p.mfoff[m]] == 2 &&
                std::fabs(p.mcoef[m] - want) <= 4e-16 * std::fabs(want)) {
                T.harm_mono[i] = m;
                break;
            }
    }
    if (T.tabd.size() >= (size_t)1 << 30) return "tables too large";

    // ---------------- compact ranking ----------------
    // lmin_i(k) = smallest level whose basis holds function k of mode i.
    T.kw = 0;
    for (int i = 0; i < D; i++) T.kw = std::max(T.kw, nsz(p.basis[i].nb_A, p.basis[i].nb_B, L));
    const int kw = T.kw;
    T.lmin_tab.assign((size_t)D * kw, 255);
    for (int i = 0; i < D; i++)
        for (int k = 0; k < kw; k++) {
            int l = 0;
            while (l <= L && nsz(p.basis[i].nb_A, p.basis[i].nb_B, l) <= k) l++;
            if (l <= L) T.lmin_tab[(size_t)i * kw + k] = (uint8_t)l;
        }
    // cnt[i][R] = number of tails (k_i..k_{D-1}) with sum of lmin <= R (R = 0..L)
    std::vector<int64_t> cnt((size_t)(D + 1) * (L + 1), 0);
    for (int R = 0; R <= L; R++) cnt[(size_t)D * (L + 1) + R] = 1;
    for (int i = D - 1; i >= 0; i--)
        for (int R = 0; R <= L; R++) {
            int64_t c = 0;
            for (int k = 0; k < kw; k++) {
                int lm = T.lmin_tab[(size_t)i * kw + k];
                if (lm <= R) c += cnt[(size_t)(i + 1) * (L + 1) + (R - lm)];
            }
            cnt[(size_t)i * (L + 1) + R] = c;
        }
    T.n_cs = cnt[L];
    if (T.n_cs >= ((int64_t)1 << 31) - 1) return "N_cs >= 2^31 is outside this build's limits";
    // rank(k) = sum_i T_i[s_i][k_i], s_i = sum_{j<i} lmin_j(k_j),
    // T_i[s][k] = sum_{v<k} cnt[i+1][L - s - lmin_i(v)]  (tails that precede k_i = k)
    T.rank_tab.assign((size_t)D * (L + 1) * kw, 0);
    for (int i = 0; i < D; i++)
        for (int s = 0; s <= L; s++) {
            int64_t acc = 0;
            for (int k = 0; k < kw; k++) {
                T.rank_tab[((size_t)i * (L + 1) + s) * kw + k] = (int)acc;
                int lm = T.lmin_tab[(size_t)i * kw + k];
                int R = L - s - lm;
                if (lm <= L && R >= 0) acc += cnt[(size_t)(i + 1) * (L + 1) + R];
            }
        }

    // harmonic energies of the split modes over the compact basis, enumerated
    // in compact order (lexicographic, mode 0 slowest) under sum lmin <= L
    {
        T.esplit.assign(T.n_cs, 0.0);
        std::vector<int> k(D, 0), c(D, 0);
        int sum = 0;
        int64_t r = 0;
        for (;;) {
            double e = 0.0;
            for (int i = 0; i < D; i++)
                if (T.harm_mono[i] >= 0)
                    e += p.omega[i] * p.basis[i].scale * p.basis[i].scale * (k[i] + 0.5);
            if (r >= T.n_cs) return "compact enumeration overran N_cs";
            T.esplit[r++] = e;
            int i = D - 1;
            while (i >= 0) {
                k[i]++;
                int lm = k[i] < kw ? T.lmin_tab[(size_t)i * kw + k[i]] : 255;
                if (lm <= L && sum - c[i] + lm <= L) { sum += lm - c[i]; c[i] = lm; break; }
                sum -= c[i]; c[i] = 0; k[i] = 0; i--;
            }
            if (i < 0) break;
        }
        if (r != T.n_cs) return "compact enumeration does not match N_cs";
    }

    // ---------------- terms in Table-2 order (l_0 fastest) ----------------
    T.Dpad = (D + 3) / 4 * 4;
    T.levels.clear();
    T.coefs.clear();
    std::vector<int> l(D, 0);
    // depth-first over modes D-1 (slowest) .. 0 (fastest), remaining budget `rem`
    struct Rec {
        static void run(int i, int rem, int sum, int D, int L, std::vector<int> &l, HostTables &T)
        {
            if (i < 0) {
                if (sum >= L - D + 1) {
                    for (int j = 0; j < T.Dpad; j++) T.levels.push_back(j < D ? (uint8_t)l[j] : 0);
                    int r = L - sum;
                    int64_t c = binom(D - 1, r);
                    T.coefs.push_back((int)((r % 2) ? -c : c));
                }
                return;
            }
            for (int v = 0; v <= rem; v++) {
                l[i] = v;
                run(i - 1, rem - v, sum + v, D, L, l, T);
            }
            l[i] = 0;
        }
    };
    Rec::run(D - 1, L, 0, D, L, l, T);
    T.n_terms = (int64_t)T.coefs.size();
    if (T.n_terms >= ((int64_t)1 << 31)) return "too many terms";

    // ---------------- per-term sizes, capacities, work ----------------
    // Pair-table bound: distinct mode pairs that share a monomial.
    std::vector<char> pair_seen((size_t)D * D, 0);
    int64_t pair_entries = 0;
    for (int m = 0; m < (int)p.mnfac.size(); m++)
        for (int f = p.mfoff[m]; f < p.mfoff[m + 1]; f++)
            for (int g = f + 1; g < p.mfoff[m + 1]; g++) {
                int a = std::min(p.mfmode[f], p.mfmode[g]), b = std::max(p.mfmode[f], p.mfmode[g]);
                if (a == b || pair_seen[(size_t)a * D + b]) continue;
                pair_seen[(size_t)a * D + b] = 1;
                int nqa = 0, nqb = 0;
                for (int lv = 0; lv <= L; lv++) {
                    nqa = std::max(nqa, T.lvl[(size_t)a * (L + 1) + lv].nq);
                    nqb = std::max(nqb, T.lvl[(size_t)b * (L + 1) + lv].nq);
                }
                pair_entries += (int64_t)nqa * nqb;
            }

    std::vector<int64_t> cost(T.n_terms);
    T.maxnb = 1;
    T.matcap = 1;
    int fsum_max = 1, stage_min_max = 1;
    T.n_s = 0;
    T.n_grid = 0;
    T.flops_per_vec = 0;
    for (int64_t t = 0; t < T.n_terms; t++) {
        const uint8_t *lt = &T.levels[(size_t)t * T.Dpad];
        int nb[kMaxD], nq[kMaxD], m = 0;
        int64_t NB = 1, NG = 1, NGfull = 1;
        int mats = 0, fsum = 0;
        for (int i = 0; i < D; i++) {
            const LevelInfo &li = T.lvl[(size_t)i * (L + 1) + lt[i]];
            NGfull *= li.nq;
            if (li.nb > 1) {
                nb[m] = li.nb; nq[m] = li.nq; m++;
                NB *= li.nb; NG *= li.nq;
                mats += 2 * li.nb * li.nq + li.nb * li.nb;
                fsum += li.nq;
            }
        }
        T.n_s += NB;
        T.n_grid += NGfull;
        T.maxnb = (int)std::max<int64_t>(T.maxnb, NB);
        T.matcap = std::max(T.matcap, mats);
        fsum_max = std::max(fsum_max, fsum);
        if (m > 0) stage_min_max = std::max(stage_min_max, nb[m - 1]);
        // FMA count of the collapsed route: forward and backward chains + kinetic
        int64_t fma = 0;
        for (int tt = 0; tt < m; tt++) {
            int64_t sz = (int64_t)nb[tt] * nq[tt];
            for (int j = 0; j < tt; j++) sz *= nq[j];
            for (int j = tt + 1; j < m; j++) sz *= nb[j];
            fma += 2 * sz;
        }
        for (int j = 0; j < m; j++) fma += NB * nb[j];
        T.flops_per_vec += 2 * fma + NG + 2 * NB;
        cost[t] = 2 * fma + 8 * NG + 16 * NB + 256;
    }
    T.vtabcap = fsum_max + (int)std::min<int64_t>(pair_entries, 1 << 24);

    // Shared memory: fixed part + two grid buffers of `cap` elements.
    const int nm = std::max(1, (int)p.mnfac.size());
    size_t fixed = (size_t)rb * (T.matcap + T.vtabcap + 4 * (size_t)T.maxnb) + 4 * (size_t)T.maxnb +
                   (size_t)nm * (16 + 24 + 16 + 16) + 1024;
    if (fixed + 2 * (size_t)rb * stage_min_max > (size_t)smem_budget) {
        snprintf(buf, sizeof buf, "a term needs %zu bytes of shared memory (budget %d)",
                 fixed + 2 * (size_t)rb * stage_min_max, smem_budget);
        return buf;
    }
    T.cap = (int)(((size_t)smem_budget - fixed) / (2 * (size_t)rb));
    T.cap = std::max(T.cap, stage_min_max);

    // fast path (potentials with at most two-mode monomials)
    std::string fe = build_fast_tables(p, &T);
    if (!fe.empty()) return fe;

    // processing order: most expensive terms first (longest-processing-time first)
    T.order.resize(T.n_terms);
    std::iota(T.order.begin(), T.order.end(), 0);
    std::stable_sort(T.order.begin(), T.order.end(),
                     [&](int a, int b) { return cost[a] > cost[b]; });
    T.pcost.resize(T.n_terms);
    for (int64_t q = 0; q < T.n_terms; q++) T.pcost[q] = cost[T.order[q]];

    if (T.fast) {
        // fast kernel: matrices, G tables, slice weights and ranks, then a work
        // area for X, Y and two grid buffers (sized per term and vector chunk)
        const int fbudget = std::min(smem_budget, rb == 4 ? SG_F32_SMEM_KB * 1024 : SG_F64_SMEM_KB * 1024);
        T.fbudget = fbudget;
        std::string de = build_fast_descs(p, rb == 4, &T, fbudget, rb);
        if (!de.empty()) return de;
    }
    return "";
}

}  // namespace sg

namespace sg {

// Fast-path tables.  Valid when every monomial of V touches at most two
// distinct modes.  A term's operator then splits exactly into
//   c0 I + sum_{slots j} H1_j + (x_j B_j^T W_j) diag(sum_{active pairs p} G_p) (x_j B_j),
// where the single-mode matrices H1_j and the scalar c0 collect, for the
// term's levels, the kinetic part, the one-mode monomials and the two-mode
// monomials whose partner mode holds one basis function (folded through
// that mode's quadrature moments), and G_p tabulates the two-mode monomials
// on the grids of the pair's levels.  Everything here depends only on
// (mode, level) combinations, so it is computed once.
std::string build_fast_tables(const Problem &p, HostTables *Tp)
{
    HostTables &T = *Tp;
    const int D = p.D, L = p.L, Lp = L + 1;
    T.fast = false;
    const int nmono = (int)p.mcoef.size();
    // distinct modes (and summed powers) of every monomial
    std::vector<std::vector<std::pair<int, int>>> facs(nmono);
    for (int m = 0; m < nmono; m++) {
        for (int f = p.mfoff[m]; f < p.mfoff[m + 1]; f++) {
            bool found = false;
            for (auto &pr : facs[m])
                if (pr.first == p.mfmode[f]) { pr.second += p.mfpow[f]; found = true; }
            if (!found) facs[m].push_back({p.mfmode[f], p.mfpow[f]});
        }
        if (facs[m].size() > 2) return "";  // not eligible: the generic kernel handles it
        if (facs[m].size() == 2 && facs[m][0].first > facs[m][1].first) std::swap(facs[m][0], facs[m][1]);
    }
    auto split = [&](int m) {
        for (int i = 0; i < D; i++) if (T.harm_mono[i] == m) return true;
        return false;
    };
    auto LI = [&](int i, int l) -> const LevelInfo & { return T.lvl[(size_t)i * Lp + l]; };
    const double *td = T.tabd.data();
    auto mu = [&](int i, int l, int pw) { return td[LI(i, l).offMu + pw]; };
    auto Mp = [&](int i, int l, int pw) { return td + LI(i, l).offM + (size_t)(pw - 1) * LI(i, l).nb * LI(i, l).nb; };

    // uniform level-1 sizes (for the register block)
    T.nb1 = T.nq1 = 0;
    if (L >= 1) {
        T.nb1 = LI(0, 1).nb; T.nq1 = LI(0, 1).nq;
        for (int i = 1; i < D; i++)
            if (LI(i, 1).nb != T.nb1 || LI(i, 1).nq != T.nq1) { T.nb1 = T.nq1 = 0; break; }
    }
    // coupled pairs
    std::vector<int> pidx((size_t)D * D, -1);
    T.pair_modes.clear();
    for (int m = 0; m < nmono; m++)
        if (facs[m].size() == 2) {
            int a = facs[m][0].first, b = facs[m][1].first;
            if (pidx[(size_t)a * D + b] < 0) {
                pidx[(size_t)a * D + b] = (int)T.pair_modes.size() / 2;
                T.pair_modes.push_back(a);
                T.pair_modes.push_back(b);
            }
        }
    const int np = (int)T.pair_modes.size() / 2;
    if (np > kMaxPairs) return "";
    T.ftab.clear();
    T.fsc.clear();
    T.c0const = 0.0;
    for (int m = 0; m < nmono; m++)
        if (facs[m].empty()) T.c0const += p.mcoef[m];
    // single-mode matrices (active levels) and scalars (collapsed levels)
    T.h1off.assign((size_t)D * Lp, -1);
    T.soff.assign((size_t)D * Lp, -1);
    for (int i = 0; i < D; i++)
        for (int l = 0; l <= L; l++) {
            const LevelInfo &li = LI(i, l);
            const int nb = li.nb;
            const bool sp = T.harm_mono[i] >= 0;
            if (nb > 1) {
                T.h1off[(size_t)i * Lp + l] = (int)T.ftab.size();
                for (int e = 0; e < nb * nb; e++) {
                    double h = sp ? 0.0 : td[li.offK + e];
                    for (int m = 0; m < nmono; m++)
                        if (facs[m].size() == 1 && facs[m][0].first == i && !split(m))
                            h += p.mcoef[m] * Mp(i, l, facs[m][0].second)[e];
                    T.ftab.push_back(h);
                }
            } else {
                T.soff[(size_t)i * Lp + l] = (int)T.fsc.size();
                double sc = sp ? 0.0 : td[li.offK];
                for (int m = 0; m < nmono; m++)
                    if (facs[m].size() == 1 && facs[m][0].first == i && !split(m))
                        sc += p.mcoef[m] * mu(i, l, facs[m][0].second);
                T.fsc.push_back(sc);
            }
        }
    // pair tables, induced matrices, pair scalars
    T.goff.assign((size_t)np * Lp * Lp, -1);
    T.ioff.assign((size_t)np * 2 * Lp * Lp, -1);
    T.spoff.assign((size_t)np * Lp * Lp, -1);
    for (int P = 0; P < np; P++) {
        const int a = T.pair_modes[2 * P], b = T.pair_modes[2 * P + 1];
        for (int la = 0; la <= L; la++)
            for (int lb = 0; la + lb <= L; lb++) {
                const LevelInfo &A = LI(a, la), &B = LI(b, lb);
                const size_t key = ((size_t)P * Lp + la) * Lp + lb;
                if (A.nb > 1 && B.nb > 1) {
                    T.goff[key] = (int)T.ftab.size();
                    for (int ua = 0; ua < A.nq; ua++)
                        for (int ub = 0; ub < B.nq; ub++) {
                            double g = 0.0;
                            for (int m = 0; m < nmono; m++)
                                if (facs[m].size() == 2 && facs[m][0].first == a && facs[m][1].first == b)
                                    g += p.mcoef[m] * std::pow(td[A.offQ + ua], facs[m][0].second) *
                                         std::pow(td[B.offQ + ub], facs[m][1].second);
                            T.ftab.push_back(g);
                        }
                } else if (A.nb > 1 || B.nb > 1) {
                    // one side active: induced single-mode matrix on that side
                    const int side = A.nb > 1 ? 0 : 1;
                    const int act = side == 0 ? a : b, lact = side == 0 ? la : lb;
                    const int col = side == 0 ? b : a, lcol = side == 0 ? lb : la;
                    const int nb = LI(act, lact).nb;
                    T.ioff[(((size_t)P * 2 + side) * Lp + lact) * Lp + lcol] = (int)T.ftab.size();
                    for (int e = 0; e < nb * nb; e++) {
                        double h = 0.0;
                        for (int m = 0; m < nmono; m++)
                            if (facs[m].size() == 2 && facs[m][0].first == a && facs[m][1].first == b) {
                                const int pact = side == 0 ? facs[m][0].second : facs[m][1].second;
                                const int pcol = side == 0 ? facs[m][1].second : facs[m][0].second;
                                h += p.mcoef[m] * mu(col, lcol, pcol) * Mp(act, lact, pact)[e];
                            }
                        T.ftab.push_back(h);
                    }
                } else {
                    T.spoff[key] = (int)T.fsc.size();
                    double sc = 0.0;
                    for (int m = 0; m < nmono; m++)
                        if (facs[m].size() == 2 && facs[m][0].first == a && facs[m][1].first == b)
                            sc += p.mcoef[m] * mu(a, la, facs[m][0].second) * mu(b, lb, facs[m][1].second);
                    T.fsc.push_back(sc);
                }
            }
    }
    if (T.ftab.size() >= ((size_t)1 << 30)) return "fast tables too large";
    if (T.fsc.empty()) T.fsc.push_back(0.0);
    if (T.ftab.empty()) T.ftab.push_back(0.0);
    T.fast = true;
    return "";
}

}  // namespace sg

namespace sg {

namespace {

template <typename S>
void put(std::vector<int4> &v, size_t unit, size_t byte, const S &x)
{
    std::memcpy(reinterpret_cast<char *>(v.data() + unit) + byte, &x, sizeof(S));
}

}  // namespace

// Per-term records of the fast kernel (processing order).  For every term:
// the transformed modes ("positions": for a term with coupled pairs, the last
// fast_rmax level-1 modes first as inner positions, whose action is tabulated
// per outer grid point; then the outer positions in the order of fewest
// multiply-adds) with the offsets of their tables, the term constant c0, the
// active coupled pairs with the offsets of their G tables, the induced
// single-mode matrices, and the slicing depth for its kernel.  The most expensive terms (a prefix of the
// processing order) run one per thread block; the small ones at its tail run
// one per warp, four per block, in a quarter of the block's shared memory
// each (a term goes to the warp form when a chunk of 4 vectors fits that
// quarter without slicing).
std::string build_fast_descs(const Problem &p, bool fp32, HostTables *Tp, int fbudget, int rb)
{
    HostTables &T = *Tp;
    const int D = p.D, L = p.L, Lp = L + 1;
    const int RMAX = fast_rmax(T.nb1);
    const int U = 16 / rb;  // elements per 16 bytes
    const int np = (int)T.pair_modes.size() / 2;
    auto LI = [&](int i, int l) -> const LevelInfo & { return T.lvl[(size_t)i * Lp + l]; };

    struct TermPlan {
        int na, R, posmode[kMaxD];
        int64_t NB, NBIn;
        bool grid;
        int gsize;
        double c0;
        std::vector<FDescPair> prs;
        std::vector<FDescInd> inds;
    };
    auto plan_term = [&](int t, TermPlan &tp) {
        const uint8_t *lt = &T.levels[(size_t)t * T.Dpad];
        int act[kMaxD], na = 0, pos_of_mode[kMaxD];
        bool l1[kMaxD], inner[kMaxD];
        double c0 = T.c0const;
        for (int i = 0; i < D; i++) {
            pos_of_mode[i] = -1;
            const LevelInfo &li = LI(i, lt[i]);
            if (li.nb > 1) { act[na] = i; l1[na] = li.nb == T.nb1 && li.nq == T.nq1; inner[na] = false; na++; }
            else c0 += T.fsc[T.soff[(size_t)i * Lp + lt[i]]];
        }
        // the term has a grid when some coupled pair has both modes transformed;
        // only then are level-1 modes made inner positions
        bool has_grid = false;
        for (int P = 0; P < np && !has_grid; P++)
            has_grid = LI(T.pair_modes[2 * P], lt[T.pair_modes[2 * P]]).nb > 1 &&
                       LI(T.pair_modes[2 * P + 1], lt[T.pair_modes[2 * P + 1]]).nb > 1;
        int R = 0;
        for (int a = na - 1; a >= 0 && R < (has_grid ? RMAX : 0); a--)
            if (l1[a]) { inner[a] = true; R++; }
        int pos = 0;
        for (int a = 0; a < na; a++) if (inner[a]) { pos_of_mode[act[a]] = pos; tp.posmode[pos++] = act[a]; }
        // Outer slots in the order of the forward (basis -> grid) chain that needs
        // the fewest multiply-adds.  A contraction costs (current size) x nq and
        // multiplies the size by nq/nb, so swapping neighbours j, k shows that j
        // goes first iff 1/nb_j - 1/nq_j < 1/nb_k - 1/nq_k (for nb = l+1,
        // nq = l+2: higher levels first).  Compared exactly in integers; ties
        // keep mode order.  The backward chain runs in reverse.
        int outer[kMaxD], no = 0;
        for (int a = 0; a < na; a++) if (!inner[a]) outer[no++] = a;
        std::stable_sort(outer, outer + no, [&](int x, int y) {
            const LevelInfo &u = LI(act[x], lt[act[x]]), &w = LI(act[y], lt[act[y]]);
            return (int64_t)(u.nq - u.nb) * w.nb * w.nq < (int64_t)(w.nq - w.nb) * u.nb * u.nq;
        });
        for (int k = 0; k < no; k++) { pos_of_mode[act[outer[k]]] = pos; tp.posmode[pos++] = act[outer[k]]; }
        tp.na = na; tp.R = R; tp.NB = 1; tp.NBIn = 1;
        for (int j = 0; j < na; j++) {
            tp.NB *= LI(tp.posmode[j], lt[tp.posmode[j]]).nb;
            if (j < R) tp.NBIn *= LI(tp.posmode[j], lt[tp.posmode[j]]).nb;
        }
        tp.prs.clear(); tp.inds.clear();
        tp.gsize = 0;
        for (int P = 0; P < np; P++) {
            const int a = T.pair_modes[2 * P], b = T.pair_modes[2 * P + 1];
            const int pa = pos_of_mode[a], pb = pos_of_mode[b];
            const size_t key = ((size_t)P * Lp + lt[a]) * Lp + lt[b];
            if (pa >= 0 && pb >= 0) {
                tp.prs.push_back(FDescPair{(unsigned char)pa, (unsigned char)pb, 0, 0, T.goff[key], tp.gsize, 0});
                tp.gsize += LI(a, lt[a]).nq * LI(b, lt[b]).nq;
            } else if (pa >= 0 || pb >= 0) {
                const int side = pa >= 0 ? 0 : 1;
                const int lact = side == 0 ? lt[a] : lt[b], lcol = side == 0 ? lt[b] : lt[a];
                tp.inds.push_back(FDescInd{(unsigned char)(side == 0 ? pa : pb), 0, 0, 0,
                                           T.ioff[(((size_t)P * 2 + side) * Lp + lact) * Lp + lcol]});
            } else {
                c0 += T.fsc[T.spoff[key]];
            }
        }
        tp.grid = !tp.prs.empty();
        tp.c0 = c0;
    };
    auto stage_of = [&](int t, const TermPlan &tp, int s) {
        const uint8_t *lt = &T.levels[(size_t)t * T.Dpad];
        int64_t sz = tp.NBIn;
        for (int j = tp.R + s; j < tp.na; j++) sz *= LI(tp.posmode[j], lt[tp.posmode[j]]).nq;
        return sz;
    };
    // slicing depth for a work area: the smallest leaving room for the slicing
    // target's vectors per chunk (else half as many, ...)
    const int vt0 = T.slice_vt > 0 ? T.slice_vt : fp32 ? SG_F32_SLICE_VT : SG_F64_SLICE_VT;
    // (sliced blocks larger than nbocap functions are not used: their slice
    // weights would not fit the group's head)
    const int nbocap = 64;
    // the term's compact indices (start of the work area) and the record's
    // scratch copy (its end) are written at the same time in the prologue
    int rec_units = 1;  // largest record, in 16-byte units (pass 1)
    auto ranks_fit = [&](const TermPlan &tp, int64_t work) {
        return 4 * tp.NB <= record_scratch_offset(work * rb, rec_units);
    };
    auto depth_for = [&](int t, const TermPlan &tp, int64_t work, int smax) {
        if (!ranks_fit(tp, work)) return -1;
        if (!tp.grid) return chunk_need(tp.NB, 0, false, false, 1, U) <= work ? 0 : -1;
        const uint8_t *lt = &T.levels[(size_t)t * T.Dpad];
        for (int vt = vt0; vt >= 1; vt /= 2) {
            int64_t nbo = 1;
            for (int s = 0; s <= std::min(smax, tp.na - tp.R); s++) {
                if (s > 0) nbo *= LI(tp.posmode[tp.R + s - 1], lt[tp.posmode[tp.R + s - 1]]).nb;
                if (nbo > nbocap) break;
                if (chunk_need(tp.NB, stage_of(t, tp, s), s > 0, true, vt, U) <= work) return s;
            }
        }
        return -1;
    };

    // pass 1: capacities
    int gcap = 1, mcap = 1;
    size_t img_total = 0;
    TermPlan tp;
    for (int64_t q = 0; q < T.n_terms; q++) {
        plan_term(T.order[q], tp);
        gcap = std::max(gcap, tp.gsize);
        rec_units = std::max(rec_units, 3 + tp.na + (int)tp.prs.size() + ((int)tp.inds.size() + 1) / 2);
        const uint8_t *lt = &T.levels[(size_t)T.order[q] * T.Dpad];
        int mat = 0;
        for (int j = 0; j < tp.na; j++) {
            const LevelInfo &li = LI(tp.posmode[j], lt[tp.posmode[j]]);
            mat += 2 * li.nb * li.nq + li.nb * li.nb;
        }
        mcap = std::max(mcap, mat);
        img_total += (size_t)mat + tp.gsize;
    }
    const size_t head = ((size_t)rb * (mcap + gcap + 2 * nbocap) + 15) & ~(size_t)15;
    const size_t hdr_static = 4 * 1024;  // per-group header in static shared memory (kHdrBytes)
    const int64_t work_cta = ((int64_t)fbudget - (int64_t)head - 1024) / rb;
    const int64_t work_warp = (((int64_t)fbudget - 4 * (int64_t)hdr_static) / 4 - (int64_t)head - 16) / rb;
    if (work_cta < 2 * T.maxnb + 64 || (size_t)work_cta * rb < 16 * (3 + (size_t)kMaxD + 2 * (size_t)np)) {
        T.fast = false;
        return "";
    }
    T.matcap = std::max(T.matcap, mcap);
    T.fgcap = gcap;
    T.fnbocap = nbocap;
    T.fwork_cta = (int)work_cta;
    T.fwork_warp = (int)std::max<int64_t>(work_warp, 0);
    T.fast_cap = T.fwork_cta;
    // split: terms that fit a warp's quarter with a chunk of warp_vt vectors
    // (unsliced, or sliced when warp-form slicing is on) run one per warp; the
    // last term that does not ends the block-form prefix
    const int warp_vt = T.warp_vt > 0 ? T.warp_vt : SG_WARP_VT;
    const int warp_smax = SG_WARP_SLICE ? kMaxD : 0;
    auto fits_warp = [&](int t, const TermPlan &tp) {
        if (work_warp <= 0 || !ranks_fit(tp, work_warp)) return false;
        if (!tp.grid) return chunk_need(tp.NB, 0, false, false, warp_vt, U) <= work_warp;
        for (int s = 0; s <= std::min(warp_smax, tp.na - tp.R); s++)
            if (chunk_need(tp.NB, stage_of(t, tp, s), s > 0, true, warp_vt, U) <= work_warp) return true;
        return false;
    };
    int64_t n_big = 0;
    for (int64_t q = 0; q < T.n_terms; q++) {
        plan_term(T.order[q], tp);
        if (!fits_warp(T.order[q], tp)) n_big = q + 1;
    }
    T.fn_big = (int)n_big;
    // pass 2: records
    T.fdesc.clear();
    T.fdesc_off.assign(T.n_terms + 1, 0);
    T.fdesccap = 0;
    T.fimg.clear();
    T.fimg.reserve(img_total);
    T.fimg_off.assign(T.n_terms + 1, 0);
    T.fvt_off.assign(T.n_terms + 1, 0);
    T.frank_start.assign(T.n_terms + 1, 0);
    int64_t rank_off = 0;
    for (int64_t q = 0; q < T.n_terms; q++) {
        const int t = T.order[q];
        const uint8_t *lt = &T.levels[(size_t)t * T.Dpad];
        plan_term(t, tp);
        const bool big = q < n_big;
        int sv = depth_for(t, tp, big ? work_cta : work_warp, big ? kMaxD : warp_smax);
        if (sv < 0) { T.fast = false; T.fdesc.clear(); return ""; }  // generic kernel instead
        int64_t nbo = 1;
        for (int j = tp.R; j < tp.R + sv; j++) nbo *= LI(tp.posmode[j], lt[tp.posmode[j]]).nb;
        if (nbo > nbocap) { T.fast = false; T.fdesc.clear(); return ""; }
        const int na = tp.na;
        // the term's shared-memory image: per position B, B^T W, H1 (+ induced), then G tables
        for (int j = 0; j < na; j++) {
            const int i = tp.posmode[j];
            const LevelInfo &li = LI(i, lt[i]);
            const size_t nbq = (size_t)li.nb * li.nq, nbb = (size_t)li.nb * li.nb;
            T.fimg.insert(T.fimg.end(), T.tabd.begin() + li.offB, T.tabd.begin() + li.offB + nbq);
            T.fimg.insert(T.fimg.end(), T.tabd.begin() + li.offBW, T.tabd.begin() + li.offBW + nbq);
            const size_t h0 = T.fimg.size();
            const int hb = T.h1off[(size_t)i * Lp + lt[i]];
            T.fimg.insert(T.fimg.end(), T.ftab.begin() + hb, T.ftab.begin() + hb + nbb);
            for (const FDescInd &d : tp.inds)
                if (d.pos == j)
                    for (size_t e = 0; e < nbb; e++) T.fimg[h0 + e] += T.ftab[d.ioff + e];
        }
        for (const FDescPair &pr : tp.prs) {
            const size_t sz = (size_t)LI(tp.posmode[pr.pa], lt[tp.posmode[pr.pa]]).nq *
                              LI(tp.posmode[pr.pb], lt[tp.posmode[pr.pb]]).nq;
            T.fimg.insert(T.fimg.end(), T.ftab.begin() + pr.goff, T.ftab.begin() + pr.goff + sz);
        }
        T.fimg_off[q + 1] = (long long)T.fimg.size();
        {
            // inner-block table: its units per outer grid point, over every
            // outer grid point (all slices), padded to 16 bytes
            long long sz = 0;
            if (tp.grid) {
                long long ngo = 1;
                for (int j = tp.R; j < na; j++) ngo *= LI(tp.posmode[j], lt[tp.posmode[j]]).nq;
                const int nbi = (int)tp.NBIn;
                sz = pad_elems((int64_t)mt_units(nbi, U) * mt_unit(nbi, U) * ngo, U);
            }
            T.fvt_off[q + 1] = T.fvt_off[q] + sz;
        }
        const int units = 3 + na + (int)tp.prs.size() + ((int)tp.inds.size() + 1) / 2;
        const size_t u0 = T.fdesc.size();
        T.fdesc.resize(u0 + units, int4{0, 0, 0, 0});
        FDescHdr h{};
        h.m = na; h.R = tp.R; h.NB = (int)tp.NB; h.coef = T.coefs[t];
        h.s = sv; h.npair = (int)tp.prs.size(); h.nind = (int)tp.inds.size(); h.gsize = tp.gsize;
        h.c0 = tp.c0; h.rank_off = rank_off;
        put(T.fdesc, u0, 0, h);
        for (int j = 0; j < na; j++) {
            const int i = tp.posmode[j];
            const LevelInfo &li = LI(i, lt[i]);
            FDescPos e{(unsigned char)i, (unsigned char)lt[i], (unsigned char)li.nb, (unsigned char)li.nq,
                       li.offB, li.offBW, T.h1off[(size_t)i * Lp + lt[i]]};
            put(T.fdesc, u0 + 3 + j, 0, e);
        }
        for (size_t q2 = 0; q2 < tp.prs.size(); q2++) put(T.fdesc, u0 + 3 + na + q2, 0, tp.prs[q2]);
        for (size_t q2 = 0; q2 < tp.inds.size(); q2++)
            put(T.fdesc, u0 + 3 + na + tp.prs.size() + q2 / 2, 8 * (q2 % 2), tp.inds[q2]);
        T.fdesc_off[q + 1] = (unsigned)(u0 + units);
        T.fdesccap = std::max(T.fdesccap, units);
        rank_off += tp.NB;
        T.frank_start[q + 1] = rank_off;
    }
    if (T.fdesc.size() >= ((size_t)1 << 32)) return "fast-path records too large";
    T.franks = rank_off;
    return "";
}

}  // namespace sg
