// Host side of the controlled-reduction library: everything before and after
// the recurrence.  arXiv 2602.24155:
//   Sec. 2.3  monomial basis of H^n_dR(U) (cokernel of the Jacobian map)
//   Sec. 2.4  Frobenius expansion (Prop. 2.1) -> start terms
//   Sec. 2.5  precision r, N_m, M
//   Sec. 3.1  Tweak (Algorithm 1); section of the map of J_S used by R_{u,v}
//             (Prop. 3.3, for S = {0..n} or a smaller S with f S-smooth)
//   Sec. 3.3  final Griffiths-Dwork reduction (step (2)) as a linear map
//   Sec. 2.1  normalisation, P(T) = det(1 - T F), functional equation
// All arithmetic mod p^M, M such that p^M < 2^63, in Montgomery form where it
// is hot.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <functional>
#include <new>
#include <thread>
#include <unordered_map>

#include "zeta_internal.h"

namespace zeta {

// ---------------------------------------------------------------------------
// Modular arithmetic
// ---------------------------------------------------------------------------
static inline uint64_t mulmod_slow(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)((u128)a * b % q);
}

static uint64_t invmod(uint64_t a, uint64_t q) {
    i128 t = 0, nt = 1, r = q, nr = a % q;
    while (nr != 0) {
        i128 qq = r / nr;
        i128 tmp = t - qq * nt; t = nt; nt = tmp;
        tmp = r - qq * nr; r = nr; nr = tmp;
    }
    if (r != 1) return 0;
    if (t < 0) t += q;
    return (uint64_t)t;
}

// Montgomery arithmetic mod an odd q < 2^63 with R = 2^64 (Montgomery 1985).
struct Mont {
    uint64_t q = 0, qneg_inv = 0, r2 = 0, one = 0;
    explicit Mont(uint64_t q_) : q(q_) {
        uint64_t inv = 1;                       // q^{-1} mod 2^64 by Newton iteration
        for (int i = 0; i < 7; i++) inv *= 2 - q * inv;
        qneg_inv = (uint64_t)0 - inv;
        uint64_t r1 = (uint64_t)(((u128)1 << 64) % q);
        r2 = (uint64_t)((u128)r1 * r1 % q);
        one = r1;
    }
    inline uint64_t redc(u128 T) const {
        uint64_t m = (uint64_t)T * qneg_inv;
        u128 t = (T + (u128)m * q) >> 64;
        uint64_t r = (uint64_t)t;
        return r >= q ? r - q : r;
    }
    inline uint64_t mul(uint64_t a, uint64_t b) const { return redc((u128)a * b); }
    inline uint64_t to(uint64_t a) const { return mul(a % q, r2); }
    inline uint64_t from(uint64_t a) const { return redc(a); }
    inline uint64_t add(uint64_t a, uint64_t b) const { uint64_t s = a + b; return s >= q ? s - q : s; }
    inline uint64_t sub(uint64_t a, uint64_t b) const { return a >= b ? a - b : a + q - b; }
    uint64_t inv(uint64_t a) const { return to(invmod(from(a), q)); }
};

static bool pow_fits(uint64_t p, uint32_t e, uint64_t limit, uint64_t *out) {
    u128 v = 1;
    for (uint32_t i = 0; i < e; i++) {
        v *= p;
        if (v >= limit) return false;
    }
    *out = (uint64_t)v;
    return true;
}

// ---------------------------------------------------------------------------
// Monomials of one degree in descending lexicographic order (x_0 first)
// ---------------------------------------------------------------------------
static int64_t binom(int64_t a, int64_t b) {
    if (b < 0 || a < b) return 0;
    int64_t r = 1;
    for (int64_t i = 1; i <= b; i++) r = r * (a - b + i) / i;
    return r;
}

struct Monos {
    int nv = 0, deg = 0, count = 0;
    std::vector<int> e;
    const int *at(int i) const { return &e[(size_t)i * nv]; }
};

static void gen_monos(int nv, int deg, int pos, int rem, std::vector<int> &cur, Monos &M) {
    if (pos == nv - 1) {
        cur[pos] = rem;
        M.e.insert(M.e.end(), cur.begin(), cur.end());
        M.count++;
        return;
    }
    for (int t = rem; t >= 0; t--) {
        cur[pos] = t;
        gen_monos(nv, deg, pos + 1, rem - t, cur, M);
    }
}

static Monos monomials(int nv, int deg) {
    Monos M;
    M.nv = nv;
    M.deg = deg;
    if (deg < 0) return M;
    std::vector<int> cur(nv, 0);
    gen_monos(nv, deg, 0, deg, cur, M);
    return M;
}

// Rank of an exponent vector of total degree `deg` in descending lex order:
// the monomials before it are those with a larger entry at the first
// position where they differ; counted by the hockey-stick identity.
static int mono_rank(const int *ex, int nv, int deg) {
    int64_t idx = 0;
    int rem = deg;
    for (int i = 0; i < nv - 1; i++) {
        int k = nv - i - 1;
        int top = rem - ex[i] - 1;
        if (top >= 0) idx += binom(top + k, k);
        rem -= ex[i];
    }
    return (int)idx;
}

// ---------------------------------------------------------------------------
// Linear algebra
// ---------------------------------------------------------------------------
// Pivot columns of the row echelon form over F_p of a rows x cols matrix
// (entries already reduced mod p).  The set depends only on the row space.
static std::vector<int> pivot_columns_mod_p(int rows, int cols, std::vector<uint32_t> A, uint32_t p) {
    std::vector<int> piv;
    int rank = 0;
    for (int c = 0; c < cols && rank < rows; c++) {
        int pr = -1;
        for (int i = rank; i < rows; i++)
            if (A[(size_t)i * cols + c] % p) { pr = i; break; }
        if (pr < 0) continue;
        if (pr != rank)
            for (int j = 0; j < cols; j++) std::swap(A[(size_t)pr * cols + j], A[(size_t)rank * cols + j]);
        uint32_t inv = (uint32_t)invmod(A[(size_t)rank * cols + c], p);
        for (int j = c; j < cols; j++) A[(size_t)rank * cols + j] = A[(size_t)rank * cols + j] * inv % p;
        for (int i = rank + 1; i < rows; i++) {
            uint32_t f = A[(size_t)i * cols + c];
            if (!f) continue;
            for (int j = c; j < cols; j++)
                A[(size_t)i * cols + j] = (A[(size_t)i * cols + j] + (p - f) * A[(size_t)rank * cols + j]) % p;
        }
        piv.push_back(c);
        rank++;
    }
    return piv;
}

// Right inverse X (cols x rows) of a rows x cols matrix of full row rank mod p,
// over Z/q: Gauss-Jordan with unit pivots, columns in order, first unit row as
// pivot, free variables zero.  Input and output in Montgomery form.
static bool right_inverse(int rows, int cols, const std::vector<uint64_t> &A, const Mont &mq,
                          uint64_t p, std::vector<uint64_t> &X) {
    int W = cols + rows;
    std::vector<uint64_t> aug((size_t)rows * W, 0);
    for (int i = 0; i < rows; i++) {
        std::memcpy(&aug[(size_t)i * W], &A[(size_t)i * cols], sizeof(uint64_t) * cols);
        aug[(size_t)i * W + cols + i] = mq.one;
    }
    std::vector<int> pivcols;
    int rank = 0;
    for (int c = 0; c < cols && rank < rows; c++) {
        int pr = -1;
        for (int i = rank; i < rows; i++)
            if (mq.from(aug[(size_t)i * W + c]) % p) { pr = i; break; }
        if (pr < 0) continue;
        if (pr != rank)
            for (int j = 0; j < W; j++) std::swap(aug[(size_t)pr * W + j], aug[(size_t)rank * W + j]);
        uint64_t *prow = &aug[(size_t)rank * W];
        uint64_t inv = mq.inv(prow[c]);
        for (int j = 0; j < W; j++) prow[j] = mq.mul(prow[j], inv);
        for (int i = 0; i < rows; i++) {
            if (i == rank) continue;
            uint64_t *row = &aug[(size_t)i * W];
            uint64_t f = row[c];
            if (!f) continue;
            for (int j = 0; j < W; j++)
                if (prow[j]) row[j] = mq.sub(row[j], mq.mul(f, prow[j]));
        }
        pivcols.push_back(c);
        rank++;
    }
    if (rank < rows) return false;
    X.assign((size_t)cols * rows, 0);
    for (int k = 0; k < rows; k++)
        std::memcpy(&X[(size_t)pivcols[k] * rows], &aug[(size_t)k * W + cols], sizeof(uint64_t) * rows);
    return true;
}

// ---------------------------------------------------------------------------
// Hypersurface data
// ---------------------------------------------------------------------------
struct Poly {
    const Monos *mon;
    std::vector<uint64_t> c;  // coefficients over mon
};

struct Setup {
    int n, d, nv;
    uint32_t p;
    std::vector<uint32_t> f;                // over Homog_d
    std::vector<std::vector<uint32_t>> df;  // d_i f over Homog_{d-1}, exact (< d*p)
    Monos md, md1;
};

// Matrix of M_k: columns (i, nu), nu in Homog_{k-d+1}, i major; rows Homog_k.
// Entries are exact nonnegative integers (< d p).
static void jacobian_columns(const Setup &S, int k, Monos &rows, Monos &src,
                             std::vector<std::vector<std::pair<int, uint32_t>>> &cols) {
    rows = monomials(S.nv, k);
    src = monomials(S.nv, k - S.d + 1);
    cols.clear();
    std::vector<int> e(S.nv);
    for (int i = 0; i < S.nv; i++) {
        for (int a = 0; a < src.count; a++) {
            std::vector<std::pair<int, uint32_t>> col;
            for (int t = 0; t < S.md1.count; t++) {
                uint32_t v = S.df[i][t];
                if (!v) continue;
                for (int z = 0; z < S.nv; z++) e[z] = S.md1.at(t)[z] + src.at(a)[z];
                col.push_back({mono_rank(e.data(), S.nv, k), v});
            }
            cols.push_back(std::move(col));
        }
    }
}

static void setup_poly(Setup &S, const zeta_hypersurface *hs) {
    S.n = hs->n; S.d = hs->d; S.nv = hs->n + 1; S.p = hs->p;
    S.md = monomials(S.nv, S.d);
    S.md1 = monomials(S.nv, S.d - 1);
    S.f.assign(hs->coeffs, hs->coeffs + S.md.count);
    S.df.assign(S.nv, std::vector<uint32_t>(S.md1.count, 0));
    std::vector<int> e(S.nv);
    for (int t = 0; t < S.md.count; t++) {
        if (!S.f[t]) continue;
        for (int i = 0; i < S.nv; i++) {
            int ei = S.md.at(t)[i];
            if (!ei) continue;
            for (int z = 0; z < S.nv; z++) e[z] = S.md.at(t)[z];
            e[i]--;
            S.df[i][mono_rank(e.data(), S.nv, S.d - 1)] += (uint32_t)ei * S.f[t];
        }
    }
}

// Smooth iff the image of M_kappa is all of Homog_kappa mod p (Jacobian criterion; p does not divide d).
static bool smooth(const Setup &S) {
    int kappa = S.nv * (S.d - 2) + 1;
    Monos rows, src;
    std::vector<std::vector<std::pair<int, uint32_t>>> cols;
    jacobian_columns(S, kappa, rows, src, cols);
    std::vector<uint32_t> A((size_t)cols.size() * rows.count, 0);
    for (size_t c = 0; c < cols.size(); c++)
        for (auto &pr : cols[c]) A[c * rows.count + pr.first] = (A[c * rows.count + pr.first] + pr.second) % S.p;
    return (int)pivot_columns_mod_p((int)cols.size(), rows.count, A, S.p).size() == rows.count;
}

// Columns (i, nu) of the map of J_S (Definition 3.1) among those of jacobian_columns:
// for i not in S only the multiples of x_i d_i f, i.e. nu_i >= 1.
static bool in_JS(uint32_t Smask, int i, const int *nu) { return ((Smask >> i) & 1u) || nu[i] >= 1; }

// n' forms of degree e in n' variables (coefficients mod p over Homog_e of those variables) have no common zero
// over the algebraic closure iff they span every form of degree n'(e-1)+1: with no common zero they are a regular
// sequence, whose quotient vanishes above its socle degree n'(e-1) (Macaulay); with one it vanishes in no degree.
static bool no_common_zero(int nv, int e, const std::vector<std::vector<uint32_t>> &forms, uint32_t p) {
    const int D = nv * (e - 1) + 1;
    const Monos rows = monomials(nv, D), src = monomials(nv, D - e), me = monomials(nv, e);
    const int ncols = nv * src.count;
    std::vector<uint32_t> A((size_t)ncols * rows.count, 0);
    std::vector<int> g(nv);
    for (int i = 0; i < nv; i++)
        for (int a = 0; a < src.count; a++) {
            const size_t c = (size_t)i * src.count + a;
            for (int t = 0; t < me.count; t++) {
                const uint32_t v = forms[i][t] % p;
                if (!v) continue;
                for (int z = 0; z < nv; z++) g[z] = me.at(t)[z] + src.at(a)[z];
                uint32_t &x = A[c * rows.count + mono_rank(g.data(), nv, D)];
                x = (x + v) % p;
            }
        }
    return (int)pivot_columns_mod_p(ncols, rows.count, A, p).size() == rows.count;
}

// S-smooth (Definition 3.1): d_i f for i in S and x_i d_i f for i not in S have no common zero.  A common zero x
// with Z = {i not in S : x_i = 0} is a common zero of the n+1-|Z| forms d_i f, i not in Z, restricted to the
// coordinate subspace {x_i = 0, i in Z}; conversely every such zero is one of J_S.  So f is S-smooth iff, for every
// Z within the complement of S, those restricted forms (a square system) have no common zero; Z = {} is the
// Jacobian criterion, tested before.  The largest of these eliminations has |Homog_{(n+1)(d-2)+1}| rows, where the
// map of J_S in degree kappa has |Homog_kappa| (a cubic fourfold: 792 against 6188).
static bool s_smooth(const Setup &S, uint32_t Smask) {
    const uint32_t full = (1u << S.nv) - 1, out = full & ~Smask;
    for (uint32_t Z = out; Z; Z = (Z - 1) & out) {
        std::vector<int> keep;
        for (int z = 0; z < S.nv; z++)
            if (!((Z >> z) & 1u)) keep.push_back(z);
        const int nk = (int)keep.size();
        const Monos me = monomials(nk, S.d - 1);
        std::vector<std::vector<uint32_t>> forms(nk, std::vector<uint32_t>(me.count, 0));
        std::vector<int> ex(S.nv);
        for (int a = 0; a < nk; a++) {
            const int i = keep[a];
            for (int t = 0; t < S.md1.count; t++) {
                const int *e = S.md1.at(t);
                bool on = true;
                for (int z = 0; z < S.nv; z++)
                    if (((Z >> z) & 1u) && e[z]) on = false;
                if (!on || !(S.df[i][t] % S.p)) continue;
                for (int b = 0; b < nk; b++) ex[b] = e[keep[b]];
                forms[a][mono_rank(ex.data(), nk, S.d - 1)] = S.df[i][t] % S.p;
            }
        }
        if (!no_common_zero(nk, S.d - 1, forms, S.p)) return false;
    }
    return true;
}

// Basis of Sec. 2.3: non-pivot monomials of the image of M_k, k = dm - n - 1.
static void cohomology_basis(const Setup &S, std::vector<uint32_t> &pole, std::vector<std::vector<int>> &exps) {
    for (int m = 1; m <= S.n; m++) {
        int k = S.d * m - S.n - 1;
        if (k < 0) continue;
        Monos rows = monomials(S.nv, k);
        std::vector<char> is_piv(rows.count, 0);
        if (k > S.nv * (S.d - 2)) {
            // above the socle degree (n+1)(d-2) of the Jacobian ring of a smooth f (a complete intersection
            // of n+1 forms of degree d-1) the image of M_k is all of Homog_k: every monomial is a pivot
            std::fill(is_piv.begin(), is_piv.end(), 1);
        } else if (k - S.d + 1 >= 0) {
            Monos r2, src;
            std::vector<std::vector<std::pair<int, uint32_t>>> cols;
            jacobian_columns(S, k, r2, src, cols);
            std::vector<uint32_t> A((size_t)cols.size() * rows.count, 0);
            for (size_t c = 0; c < cols.size(); c++)
                for (auto &pr : cols[c]) A[c * rows.count + pr.first] = (A[c * rows.count + pr.first] + pr.second) % S.p;
            for (int c : pivot_columns_mod_p((int)cols.size(), rows.count, A, S.p)) is_piv[c] = 1;
        }
        for (int t = 0; t < rows.count; t++)
            if (!is_piv[t]) {
                pole.push_back(m);
                exps.push_back(std::vector<int>(rows.at(t), rows.at(t) + S.nv));
            }
    }
}

// ---------------------------------------------------------------------------
// Precision (Sec. 2.5).  r: Weil bound on a_i against the Hodge polygon;
// N_m: least N with m - 1 + i - (n-1) floor(log_p(p(m+i))) >= r for i >= N;
// M = max_m r + v_p((p s_m - 1)!) - m + 1.
// ---------------------------------------------------------------------------
static int vp_factorial(uint64_t x, uint64_t p) {
    int e = 0;
    for (u128 t = p; t <= x; t *= p) e += (int)(x / t);
    return e;
}

static int ilog(uint64_t K, uint64_t p) {
    int e = 0;
    for (u128 t = p; t <= K; t *= p) e++;
    return e;
}

// e_i: least e with p^{2e} > 4 C(b,i)^2 p^{(n-1)i}, i = 0..b/2 (a_i is fixed by a_i mod p^{e_i}).
static std::vector<int> coefficient_digits(int n, uint64_t p, int b) {
    std::vector<int> e;
    for (int i = 0; i <= b / 2; i++) {
        // t = 2e - (n-1)i must be the least t with p^t > 4 C^2
        u128 bound = (u128)binom(b, i) * binom(b, i) * 4;
        int t = 0;
        u128 pt = 1;
        while (pt <= bound) { pt *= p; t++; }
        e.push_back((t + (n - 1) * i + 1) / 2);
    }
    return e;
}

// r_m = max(1, max_i e_i - G_m(i)), G_m(i) = (n - m) + the i-1 smallest slopes of
// the other columns: a minor of F on a column set I is known mod
// p^{sum sigma_j + min r_{m_j}} when the pole-order-m columns of C are known mod p^{r_m}.
static int relative_precision_m(int n, uint64_t p, const std::vector<uint32_t> &pole, uint32_t m) {
    int b = (int)pole.size();
    std::vector<int> e = coefficient_digits(n, p, b);
    std::vector<int> others;
    bool skipped = false;
    for (uint32_t mm : pole) {
        if (!skipped && mm == m) { skipped = true; continue; }
        others.push_back(n - (int)mm);
    }
    std::sort(others.begin(), others.end());
    int best = 1, acc = 0;
    for (int i = 1; i <= b / 2; i++) {
        int G = (n - (int)m) + acc;
        best = std::max(best, e[i] - G);
        if (i - 1 < (int)others.size()) acc += others[i - 1];
    }
    return best;
}

static int series_order(int m, int r, int n, uint64_t p) {
    for (int N = 1;; N++) {
        bool ok = true;
        for (int i = N; i <= N + 200; i++)
            if (m - 1 + i - (n - 1) * ilog(p * (uint64_t)(m + i), p) < r) { ok = false; break; }
        if (ok) return N;
    }
}

// ---------------------------------------------------------------------------
// Instance preparation
// ---------------------------------------------------------------------------
static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static inline uint64_t pack_u(const int *U, int nv) {
    uint64_t key = 0;
    for (int i = 0; i < nv; i++) key = (key << 10) | (uint64_t)U[i];
    return key;
}

static void build_solves(const Setup &S, Instance &X);
static zeta_status complete_reduction(const Setup &S, Instance &X, double t0);

zeta_status prepare_instance(const zeta_hypersurface *hs, const zeta_options *opt, bool build_reduction,
                             Instance &X, bool defer_solves) {
    double t0 = now_ms();
    if (!hs || !hs->coeffs) { X.error = "null hypersurface"; return X.status = ZETA_ERR_ARG; }
    uint32_t n = hs->n, d = hs->d, p = hs->p;
    if (n < 1 || n + 1 > (uint32_t)kMaxVars || d < 2 || d > 12) { X.error = "n or d out of range"; return X.status = ZETA_ERR_UNSUPPORTED; }
    bool prime = p >= 2;
    for (uint32_t t = 2; t * t <= p && prime; t++) if (p % t == 0) prime = false;
    if (!prime || p < 7 || p >= 50 || d % p == 0 || p <= n) { X.error = "p must be a prime in [7, 50), p > n, p not dividing d"; return X.status = ZETA_ERR_UNSUPPORTED; }
    // the index set S of Prop. 3.3: {0..n} when d >= n + 1, else {n}, unless the caller names one
    const uint32_t full = (1u << (n + 1)) - 1;
    const uint32_t Smask = (opt && opt->S_mask) ? opt->S_mask : (d >= n + 1 ? full : (1u << n));
    if (Smask & ~full) { X.error = "S_mask names a variable beyond x_n"; return X.status = ZETA_ERR_ARG; }
    const uint32_t Ssize = (uint32_t)__builtin_popcount(Smask);
    if (Ssize > d) { X.error = "controlled reduction needs d >= |S| (Prop. 3.3)"; return X.status = ZETA_ERR_UNSUPPORTED; }
    // step matrices of side s = C(dn, n): up to 512 on the persistent executors, up to 4096 on the
    // whole-GPU one (cubic fourfolds: s = 3003), whose setup's right inverses (the section is 6188 x
    // 18018 for a cubic fourfold) are solved on the device only; refused before the smoothness tests,
    // whose eliminations grow with s
    if (binom(d * n, n) > 4096) { X.error = "step matrices larger than 4096 x 4096 (C(dn, n) > 4096)"; return X.status = ZETA_ERR_UNSUPPORTED; }
    if (binom(d * n, n) > 512 && build_reduction && !defer_solves) {
        X.error = "C(dn, n) > 512: the setup's right inverses are solved on the device (batch calls)";
        return X.status = ZETA_ERR_UNSUPPORTED;
    }
    X.n = n; X.d = d; X.p = p; X.nv = n + 1;
    X.Smask = Smask;
    X.base = Ssize - 1;
    Setup S;
    int ncoef = (int)binom(n + d, n);
    for (int t = 0; t < ncoef; t++)
        if (hs->coeffs[t] >= p) { X.error = "coefficient not reduced mod p"; return X.status = ZETA_ERR_ARG; }
    X.coeffs.assign(hs->coeffs, hs->coeffs + ncoef);
    setup_poly(S, hs);
    if (!smooth(S)) { X.error = "f is not smooth (Jacobian criterion)"; return X.status = ZETA_ERR_NOT_SMOOTH; }
    X.kappa = (n + 1) * (d - 1) + 1 - Ssize;
    if (Smask != full && !s_smooth(S, Smask)) {
        X.error = "f is not S-smooth (Definition 3.1)";
        return X.status = ZETA_ERR_NOT_SMOOTH;
    }
    cohomology_basis(S, X.pole, X.basis_exp);
    X.b = (uint32_t)X.pole.size();
    int64_t bexp = (binom(1, 0) * 0);
    {
        int64_t dm1 = d - 1, pw = 1;
        for (uint32_t i = 0; i < n + 1; i++) pw *= dm1;
        bexp = (pw + ((n + 1) % 2 ? -dm1 : dm1)) / d;
    }
    if ((int64_t)X.b != bexp) { X.error = "basis size disagrees with the Hodge count"; return X.status = ZETA_ERR_INTERNAL; }
    X.s = (uint32_t)binom(d * n - n + n, n);
    X.h_rows = (uint32_t)binom(d * n - n - 1 + n, n);

    // precision (Sec. 2.5): r_m, N_m, M
    int Mp = 0;
    X.r = 0;
    for (uint32_t m = 1; m <= n; m++) {
        bool used = std::find(X.pole.begin(), X.pole.end(), m) != X.pole.end();
        if (!used) { X.N[m - 1] = 0; X.rm[m - 1] = 0; continue; }
        X.rm[m - 1] = (opt && opt->r_override) ? opt->r_override : (uint32_t)relative_precision_m(n, p, X.pole, m);
        X.r = std::max(X.r, X.rm[m - 1]);
        X.N[m - 1] = (opt && opt->N_override[m - 1]) ? opt->N_override[m - 1]
                                                     : (uint32_t)series_order(m, (int)X.rm[m - 1], n, p);
        uint32_t sm = X.N[m - 1] + m - 1;
        Mp = std::max(Mp, (int)X.rm[m - 1] + vp_factorial((uint64_t)p * sm - 1, p) - (int)m + 1);
    }
    X.M = (uint32_t)Mp;
    // the device keeps residues mod q as two 30-bit limbs (vector path) or at most
    // eight balanced base-256 digits (tensor-core path): q < 2^60
    if (!pow_fits(p, X.M, (uint64_t)1 << 60, &X.q)) { X.error = "p^M exceeds 2^60"; return X.status = ZETA_ERR_PRECISION; }
    for (uint32_t m = 1; m <= n; m++) {
        uint64_t tmp;
        if (X.N[m - 1] && !pow_fits(p, X.N[m - 1] + m - 1, (uint64_t)1 << 63, &tmp)) { X.error = "p^s exceeds 2^63"; return X.status = ZETA_ERR_PRECISION; }
    }
    if (!build_reduction) { X.ms_setup = now_ms() - t0; return ZETA_OK; }

    build_solves(S, X);
    if (defer_solves) {
        X.solves_pending = true;
        X.ms_setup = now_ms() - t0;
        return ZETA_OK;
    }
    return complete_reduction(S, X, t0);
}

// The right inverses' matrices (Montgomery form): [0] the section of the map of J_S in degree
// kappa (Prop. 3.3 proof), Sec[(i,nu), gamma] = coefficient of x^nu in G_i, sum_i G_i d_i f =
// x^gamma; columns (i, nu) outside J_S stay zero, so Gauss-Jordan never pivots there and their
// rows of Sec are zero (for S = {0..n} every column is in).  [m], m = 1..n: the final reduction
// at pole order m (Sec. 3.3 step (2)), rows Homog_k, k = dm - n - 1, columns the basis elements
// of pole order m and then the map (i, nu) -> x^nu d_i f from Homog_{k-d+1}; empty when k < 0.
static void build_solves(const Setup &S, Instance &X) {
    const Mont mq(X.q);
    const int n = (int)X.n, d = (int)X.d;
    const uint32_t Smask = X.Smask;
    X.solves.assign(n + 1, SolveJob());
    {
        Monos rows, src;
        std::vector<std::vector<std::pair<int, uint32_t>>> cols;
        jacobian_columns(S, X.kappa, rows, src, cols);
        SolveJob &J = X.solves[0];
        J.R = rows.count;
        J.C = (int)cols.size();
        J.A.assign((size_t)J.R * J.C, 0);
        for (int c = 0; c < J.C; c++) {
            if (!in_JS(Smask, c / src.count, src.at(c % src.count))) continue;
            for (auto &pr : cols[c])
                J.A[(size_t)pr.first * J.C + c] = mq.add(J.A[(size_t)pr.first * J.C + c], mq.to(pr.second));
        }
    }
    for (int m = 1; m <= n; m++) {
        const int k = d * m - n - 1;
        Monos rows = monomials(S.nv, k);
        if (rows.count == 0) continue;
        std::vector<int> bset;
        for (uint32_t t = 0; t < X.b; t++)
            if (X.pole[t] == (uint32_t)m) bset.push_back((int)t);
        std::vector<std::vector<std::pair<int, uint32_t>>> jcols;
        Monos r2, src;
        if (k - d + 1 >= 0) jacobian_columns(S, k, r2, src, jcols);
        SolveJob &J = X.solves[m];
        J.R = rows.count;
        J.C = (int)bset.size() + (int)jcols.size();
        J.A.assign((size_t)J.R * J.C, 0);
        for (size_t c = 0; c < bset.size(); c++)
            J.A[(size_t)mono_rank(X.basis_exp[bset[c]].data(), S.nv, k) * J.C + c] = mq.one;
        const size_t nb = bset.size();
        for (size_t c = 0; c < jcols.size(); c++)
            for (auto &pr : jcols[c])
                J.A[(size_t)pr.first * J.C + nb + c] = mq.add(J.A[(size_t)pr.first * J.C + nb + c], mq.to(pr.second));
    }
}

zeta_status prepare_complete(Instance &X) {
    if (!X.solves_pending) { X.error = "prepare_complete without a deferred prepare_instance"; return X.status = ZETA_ERR_INTERNAL; }
    const double t0 = now_ms() - X.ms_setup;
    zeta_hypersurface hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.n = X.n;
    hs.d = X.d;
    hs.p = X.p;
    hs.coeffs = X.coeffs.data();
    Setup S;
    setup_poly(S, &hs);
    X.solves_pending = false;
    return complete_reduction(S, X, t0);
}

// Everything after the right inverses: the section and the step-matrix tables, the final
// reduction map, the Frobenius expansion.  Solves the jobs still open on the host.
static zeta_status complete_reduction(const Setup &S, Instance &X, double t0) {
    const uint32_t n = X.n, d = X.d, p = X.p;
    const uint32_t Smask = X.Smask;
    const uint64_t q = X.q;
    Mont mq(q);
    const int nv = X.nv;
    for (SolveJob &J : X.solves)
        if (J.R && !J.done) {
            J.ok = right_inverse(J.R, J.C, J.A, mq, p, J.X);
            J.done = true;
        }
    {
        SolveJob &J = X.solves[0];
        if (!J.ok) { X.error = "section: Jacobian map not onto"; return X.status = ZETA_ERR_INTERNAL; }
        const int R = J.R, C = J.C;
        const Monos src = monomials(nv, (int)X.kappa - (int)d + 1);
        X.sec_rows = C;
        X.sec_cols = R;
        X.sec.resize((size_t)C * R);
        for (size_t t = 0; t < X.sec.size(); t++) X.sec[t] = mq.from(J.X[t]);

        // index tables of the device's step-matrix generation: with e = mu + 1 - 1_S the
        // S = {0..n} formulas R[omega, mu] = sum_i (u_i + e_omega,i) Sec[(i, e_omega - 1 + e_i),
        // v + e_mu - 1] and the numerator exponent U + e_mu - 1 are those of any S
        Monos mS = monomials(nv, d * n - n);
        X.tab_monoS.assign((size_t)mS.count * nv, 0);
        X.tab_secrow.assign((size_t)nv * mS.count, -1);
        std::vector<int> g(nv);
        for (int r = 0; r < mS.count; r++) {
            for (int z = 0; z < nv; z++) X.tab_monoS[(size_t)r * nv + z] = mS.at(r)[z] + 1 - (int)((Smask >> z) & 1u);
            for (int i = 0; i < nv; i++) {
                bool ok = true;
                for (int z = 0; z < nv; z++) {
                    g[z] = mS.at(r)[z] - (int)((Smask >> z) & 1u) + (z == i ? 1 : 0);
                    if (g[z] < 0) ok = false;
                }
                if (ok) X.tab_secrow[(size_t)i * mS.count + r] = i * src.count + mono_rank(g.data(), nv, src.deg);
            }
        }
    }

    // Final reduction map (Sec. 3.3 step (2)): Fin[beta, h], h in Homog_{dn-n-1}.
    {
        struct Level { Monos rows; int nb; std::vector<int> bcols; Monos src; std::vector<uint64_t> Xinv; int ncols; };
        std::vector<Level> lev(n + 1);
        for (uint32_t m = 1; m <= n; m++) {
            int k = d * m - n - 1;
            Level &L = lev[m];
            L.rows = monomials(nv, k);
            if (L.rows.count == 0) continue;
            std::vector<int> bset;
            for (uint32_t t = 0; t < X.b; t++)
                if (X.pole[t] == m) bset.push_back((int)t);
            L.nb = (int)bset.size();
            L.bcols = bset;
            if (k - (int)d + 1 >= 0) L.src = monomials(nv, k - (int)d + 1);
            L.ncols = L.nb + nv * L.src.count;
            SolveJob &J = X.solves[m];
            if (!J.ok || J.R != L.rows.count || J.C != L.ncols) { X.error = "final reduction: not onto"; return X.status = ZETA_ERR_INTERNAL; }
            L.Xinv.swap(J.X);
        }
        X.fin.assign((size_t)X.b * X.h_rows, 0);
        std::vector<uint64_t> inv_m(n + 1, 0);
        for (uint32_t m = 2; m <= n; m++) inv_m[m] = mq.inv(mq.to(m - 1));
        std::vector<int> e(nv);
        for (uint32_t h = 0; h < X.h_rows; h++) {
            // start: e_h at pole order n (Montgomery form)
            std::vector<uint64_t> vec(lev[n].rows.count, 0);
            vec[h] = mq.one;
            for (int m = (int)n; m >= 1; m--) {
                Level &L = lev[m];
                if (L.rows.count == 0) break;
                int R = L.rows.count, C = L.ncols;
                std::vector<int> nzr;
                for (int r2 = 0; r2 < R; r2++)
                    if (vec[r2]) nzr.push_back(r2);
                std::vector<uint64_t> sol(C, 0);
                for (int c = 0; c < C; c++) {
                    uint64_t acc = 0;
                    for (int r2 : nzr) acc = mq.add(acc, mq.mul(L.Xinv[(size_t)c * R + r2], vec[r2]));
                    sol[c] = acc;
                }
                for (int c = 0; c < L.nb; c++) X.fin[(size_t)L.bcols[c] * X.h_rows + h] = mq.from(sol[c]);
                if (m == 1) break;
                // next numerator: (1/(m-1)) sum_i d_i h_i, h_i over Homog_{k-d+1}
                Level &Ln = lev[m - 1];
                std::vector<uint64_t> nvec(Ln.rows.count, 0);
                int ns = L.src.count;
                for (int i = 0; i < nv; i++)
                    for (int a = 0; a < ns; a++) {
                        uint64_t val = sol[L.nb + i * ns + a];
                        if (!val) continue;
                        const int *ex = L.src.at(a);
                        if (ex[i] == 0) continue;
                        for (int z = 0; z < nv; z++) e[z] = ex[z];
                        e[i]--;
                        int pos = mono_rank(e.data(), nv, Ln.rows.deg);
                        nvec[pos] = mq.add(nvec[pos], mq.mul(mq.mul(val, mq.to((uint64_t)ex[i])), inv_m[m]));
                    }
                vec.swap(nvec);
            }
        }
    }

    // Frobenius expansion (Prop. 2.1) and Tweak (Alg. 1): start terms grouped by U.
    {
        Monos mS = monomials(nv, d * n - n);
        std::unordered_map<uint64_t, uint32_t> chain_of;
        std::vector<std::vector<Term>> chain_terms;
        std::vector<std::vector<int>> chain_U;
        uint32_t jmax = 0;
        for (uint32_t m = 1; m <= n; m++) jmax = std::max(jmax, X.N[m - 1]);
        std::vector<int> gamma(nv), U(nv), J(nv), e(nv);
        for (uint32_t m = 1; m <= n; m++) {
            uint32_t Nm = X.N[m - 1];
            if (!Nm) continue;
            uint32_t sm = Nm + m - 1;
            uint64_t ps;
            pow_fits(p, sm, (uint64_t)1 << 63, &ps);
            Mont mps(ps);
            // f^j mod p^s, j < N_m
            std::vector<Monos> mj(Nm);
            std::vector<std::vector<uint64_t>> fj(Nm);
            mj[0] = monomials(nv, 0);
            fj[0].assign(1, 1);
            for (uint32_t j = 1; j < Nm; j++) {
                mj[j] = monomials(nv, d * j);
                fj[j].assign(mj[j].count, 0);
                for (int a = 0; a < mj[j - 1].count; a++) {
                    uint64_t ca = fj[j - 1][a];
                    if (!ca) continue;
                    uint64_t cam = mps.to(ca);
                    for (int t = 0; t < S.md.count; t++) {
                        if (!S.f[t]) continue;
                        for (int z = 0; z < nv; z++) e[z] = mj[j - 1].at(a)[z] + S.md.at(t)[z];
                        int pos = mono_rank(e.data(), nv, d * j);
                        fj[j][pos] = (fj[j][pos] + mps.from(mps.mul(cam, mps.to(S.f[t])))) % ps;
                    }
                }
            }
            for (uint32_t col = 0; col < X.b; col++) {
                if (X.pole[col] != m) continue;
                const std::vector<int> &beta = X.basis_exp[col];
                for (uint32_t j = 0; j < Nm; j++) {
                    // D_{j,m} = (-1)^j sum_{i=j}^{N-1} C(m+i-1, i) C(i, j)
                    u128 T = 0;
                    for (uint32_t i = j; i < Nm; i++) T += (u128)binom(m + i - 1, i) * binom(i, j);
                    uint64_t Dm = (uint64_t)(T % ps);
                    if (j % 2 && Dm) Dm = ps - Dm;
                    // (p s - 1)! / (p(m+j) - 1)! mod q
                    uint64_t scale = mq.one;
                    for (uint64_t t = (uint64_t)p * (m + j); t <= (uint64_t)p * sm - 1; t++) scale = mq.mul(scale, mq.to(t));
                    scale = mq.from(scale);
                    for (int a = 0; a < mj[j].count; a++) {
                        uint64_t C = fj[j][a];
                        if (!C) continue;
                        uint64_t c = mulmod_slow(Dm, C, ps);
                        if (!c) continue;
                        uint64_t coeff = mulmod_slow(c, scale, q);
                        if (!coeff) continue;
                        // x^{p(beta+alpha+1)-1} over x^S: gamma = p(beta+alpha+1) - 1 + 1_S
                        for (int z = 0; z < nv; z++)
                            gamma[z] = (int)p * (beta[z] + mj[j].at(a)[z] + 1) - 1 + (int)((Smask >> z) & 1u);
                        // Tweak(gamma, dn - n): remove units from the front
                        int left = (int)(d * n - n);
                        for (int z = 0; z < nv; z++) {
                            int take = std::min(gamma[z], left);
                            U[z] = gamma[z] - take;
                            J[z] = take;
                            left -= take;
                        }
                        uint64_t key = pack_u(U.data(), nv);
                        auto it = chain_of.find(key);
                        uint32_t ci;
                        if (it == chain_of.end()) {
                            ci = (uint32_t)chain_terms.size();
                            chain_of.emplace(key, ci);
                            chain_terms.emplace_back();
                            chain_U.push_back(U);
                        } else {
                            ci = it->second;
                        }
                        chain_terms[ci].push_back(Term{(uint32_t)mono_rank(J.data(), nv, mS.deg), col, coeff});
                        X.nterms++;
                    }
                }
            }
        }
        // chains in decreasing length (the device takes the longest first)
        std::vector<uint32_t> order(chain_terms.size());
        for (size_t i = 0; i < order.size(); i++) order[i] = (uint32_t)i;
        auto normU = [&](uint32_t i) { int s = 0; for (int z = 0; z < nv; z++) s += chain_U[i][z]; return s; };
        std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b2) { return normU(a) > normU(b2); });
        X.chains.clear();
        X.terms.clear();
        for (uint32_t ci : order) {
            Chain ch;
            std::memset(&ch, 0, sizeof(ch));
            for (int z = 0; z < nv; z++) ch.U[z] = chain_U[ci][z];
            ch.term_begin = (uint32_t)X.terms.size();
            X.terms.insert(X.terms.end(), chain_terms[ci].begin(), chain_terms[ci].end());
            ch.term_end = (uint32_t)X.terms.size();
            uint64_t steps = (uint64_t)(normU(ci) - (int)X.base) / d;
            ch.work = steps * X.b * (uint64_t)X.s * X.s;
            X.chains.push_back(ch);
        }
    }
    std::vector<SolveJob>().swap(X.solves);
    X.ms_setup = now_ms() - t0;
    return ZETA_OK;
}

// ---------------------------------------------------------------------------
// Finish: Y = Fin * H, normalisation, det(1 - T F), lift (Sec. 2.1, 2.5)
// ---------------------------------------------------------------------------
// det(T I - F) mod m by Berkowitz's division-free recurrence; returns c_0..c_b.
static std::vector<uint64_t> berkowitz_mod(const std::vector<uint64_t> &F, int b, uint64_t m) {
    std::vector<uint64_t> poly = {1 % m, (m - F[0] % m) % m};
    if (b == 0) return {1 % m};
    for (int r = 1; r < b; r++) {
        uint64_t a = F[(size_t)r * b + r] % m;
        std::vector<uint64_t> t = {1 % m, (m - a) % m};
        std::vector<uint64_t> vec(r), nvec(r);
        for (int i = 0; i < r; i++) vec[i] = F[(size_t)i * b + r] % m;
        for (int it = 0; it < r; it++) {
            u128 acc = 0;
            for (int j = 0; j < r; j++) acc = (acc + (u128)F[(size_t)r * b + j] * vec[j]) % m;
            t.push_back((m - (uint64_t)acc) % m);
            for (int i = 0; i < r; i++) {
                u128 s2 = 0;
                for (int j = 0; j < r; j++) s2 = (s2 + (u128)F[(size_t)i * b + j] * vec[j]) % m;
                nvec[i] = (uint64_t)s2;
            }
            vec.swap(nvec);
        }
        std::vector<uint64_t> np(r + 2, 0);
        for (int i = 0; i < r + 2; i++) {
            u128 s2 = 0;
            for (int j = std::max(0, i - (int)t.size() + 1); j <= std::min(i, r); j++)
                s2 = (s2 + (u128)t[i - j] * poly[j]) % m;
            np[i] = (uint64_t)s2;
        }
        poly.swap(np);
    }
    return poly;
}

zeta_status finish_y_only(Instance &X) {
    const uint32_t b = X.b;
    const uint64_t q = X.q;
    // Y = Fin * H (b x h_rows times h_rows x b)
    X.Y.assign((size_t)b * b, 0);
    for (uint32_t i = 0; i < b; i++)
        for (uint32_t j = 0; j < b; j++) {
            u128 acc = 0;
            for (uint32_t h = 0; h < X.h_rows; h++)
                acc = (acc + (u128)X.fin[(size_t)i * X.h_rows + h] * X.H[(size_t)h * b + j]) % q;
            X.Y[(size_t)i * b + j] = (uint64_t)acc;
        }
    return ZETA_OK;
}

zeta_status finish_instance(Instance &X) {
    double t0 = now_ms();
    const uint32_t b = X.b, n = X.n, p = X.p;
    const uint64_t q = X.q;
    finish_y_only(X);
    // columns c = (n-1)! unit^{-1} Y / p^{v-m+1} mod p^{r_m}, F = c p^{n-m}
    std::vector<uint64_t> Cm((size_t)b * b);
    uint32_t rmin = 0;
    for (uint32_t m = 1; m <= n; m++)
        if (X.rm[m - 1] && (!rmin || X.rm[m - 1] < rmin)) rmin = X.rm[m - 1];
    X.F.assign((size_t)b * b, 0);
    uint64_t fact_n1 = 1;
    for (uint32_t t = 2; t < n; t++) fact_n1 = fact_n1 * t;
    for (uint32_t col = 0; col < b; col++) {
        uint32_t m = X.pole[col];
        uint64_t pr;
        pow_fits(p, X.rm[m - 1], (uint64_t)1 << 63, &pr);
        uint64_t sm = X.N[m - 1] + m - 1;
        uint64_t top = (uint64_t)p * sm - 1;
        int v = vp_factorial(top, p);
        int e = v - (int)m + 1;
        uint64_t unit = 1;
        for (uint64_t t = 1; t <= top; t++) {
            uint64_t u = t;
            while (u % p == 0) u /= p;
            unit = mulmod_slow(unit, u % q, q);
        }
        uint64_t uinv = invmod(unit, q);
        uint64_t pe = 1;
        if (e > 0) pow_fits(p, (uint32_t)e, (uint64_t)1 << 63, &pe);
        uint64_t scale_up = 1;
        if (e < 0) pow_fits(p, (uint32_t)(-e), (uint64_t)1 << 63, &scale_up);
        uint64_t pnm;
        pow_fits(p, n - m, (uint64_t)1 << 63, &pnm);
        for (uint32_t row = 0; row < b; row++) {
            uint64_t y = X.Y[(size_t)row * b + col];
            uint64_t z;
            if (e > 0) {
                if (y % pe) { X.error = "unnormalised column not divisible by p^(v-m+1)"; return X.status = ZETA_ERR_INTERNAL; }
                z = y / pe;
            } else {
                z = mulmod_slow(y, scale_up, q);
            }
            uint64_t c = mulmod_slow(mulmod_slow(z % pr, fact_n1 % pr, pr), uinv % pr, pr);
            Cm[(size_t)row * b + col] = c;  // reduced again mod p^{rmin} for the sign below
            X.F[(size_t)row * b + col] = c * pnm;  // < p^{r+n-m} < 2^63
        }
    }
    // a_i is known mod p^{e_i} (i <= b/2)
    std::vector<int> e = coefficient_digits((int)n, p, (int)b);
    int K = 0;
    for (uint32_t i = 0; i <= b / 2; i++) K = std::max(K, e[i]);
    // a run below the precision rule (relative precision rmin) knows some a_i only mod p^(rmin + H(i)) with
    // rmin + H(i) < e_i, H the Hodge polygon of the slopes n - m of the basis elements in increasing order
    bool truncated_run = false;
    {
        std::vector<int> slope;
        for (uint32_t col = 0; col < b; col++) slope.push_back((int)n - (int)X.pole[col]);
        std::sort(slope.begin(), slope.end());
        for (uint32_t i = 1, H = 0; i <= b / 2; i++) {
            H += (uint32_t)slope[i - 1];
            if ((int)(rmin + H) < e[i]) truncated_run = true;
        }
    }
    uint64_t pK;
    if (!pow_fits(p, (uint32_t)K, (uint64_t)1 << 63, &pK)) {
        // a truncated run takes the charpoly mod the largest power p^K below 2^63: a_i is then known mod
        // p^min(rmin + H(i), K); a run at the rule's precision needs every digit
        if (!truncated_run) { X.error = "charpoly precision exceeds 2^63"; return X.status = ZETA_ERR_PRECISION; }
        K = 0;
        while (pow_fits(p, (uint32_t)K + 1, (uint64_t)1 << 63, &pK)) K++;
        for (auto &x : e) x = std::min(x, K);
        pow_fits(p, (uint32_t)K, (uint64_t)1 << 63, &pK);
    }
    std::vector<uint64_t> cp = berkowitz_mod(X.F, (int)b, pK);
    // eps = (-1)^b det(C) mod p^{min r_m}
    uint64_t pr;
    pow_fits(p, rmin, (uint64_t)1 << 63, &pr);
    for (auto &x : Cm) x %= pr;
    std::vector<uint64_t> cpC = berkowitz_mod(Cm, (int)b, pr);
    uint64_t sgn = cpC[b];  // det(T I - C) at T = 0 is (-1)^b det C; so sgn = (-1)^b det(C)
    if (sgn == 1 % pr) X.eps = 1;
    else if (sgn == pr - 1) X.eps = -1;
    else { X.error = "det of the Frobenius columns is not a unit sign"; return X.status = ZETA_ERR_INTERNAL; }
    X.P.assign(b + 1, 0);
    X.P[0] = 1;
    for (uint32_t i = 1; i <= b / 2; i++) {
        uint64_t mod;
        pow_fits(p, (uint32_t)e[i], (uint64_t)1 << 63, &mod);
        uint64_t x = cp[i] % mod;
        X.P[i] = (x > mod / 2) ? (i128)x - (i128)mod : (i128)x;
    }
    // a_{b-i} = eps p^(w(b-2i)/2) a_i (functional equation, weight w = n - 1): exact while it fits 125 bits; a
    // truncated run whose exact value would not (quintic surfaces: 11^52) gets it mod p^K like its other digits
    int w = (int)n - 1;
    const u128 limit = (u128)1 << 125;
    for (uint32_t i = 0; i < (b + 1) / 2; i++) {
        uint32_t j = b - i;
        if (j <= b / 2) continue;
        const int ex = w * ((int)b - 2 * (int)i) / 2;
        const u128 mag = (u128)(X.P[i] < 0 ? -X.P[i] : X.P[i]);
        u128 pw = 1;
        bool fits = true;
        for (int t = 0; t < ex && fits; t++) {
            pw *= p;
            if (pw > limit / (mag ? mag : 1)) fits = false;
        }
        if (fits) {
            X.P[j] = (i128)X.eps * (i128)pw * X.P[i];
            continue;
        }
        if (!truncated_run) { X.error = "P(T) coefficient exceeds 125 bits"; return X.status = ZETA_ERR_PRECISION; }
        uint64_t pe = 1 % pK;
        for (int t = 0; t < ex; t++) pe = (uint64_t)((u128)pe * p % pK);
        const uint64_t ai = (uint64_t)(((X.P[i] % (i128)pK) + (i128)pK) % (i128)pK);
        uint64_t x = (uint64_t)((u128)pe * ai % pK);
        if (X.eps < 0 && x) x = pK - x;
        X.P[j] = (x > pK / 2) ? (i128)x - (i128)pK : (i128)x;
    }
    X.ms_finish = now_ms() - t0;
    return ZETA_OK;
}

}  // namespace zeta
