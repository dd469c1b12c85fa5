/*
 * ccg_oracle.c -- plain, slow, FP64 CPU reference of the cooperative
 * conjugate gradient method (cCG) of Bhaya, Bliman, Niedu and Pazos,
 * "A cooperative conjugate gradient method for linear systems permitting
 * multithread implementation of low complexity" (arXiv:1204.0069).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA solver is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or helper with
 * the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (notation of the paper, Sec. 3.2):
 *   A (n x n, SPD), b (n), X_0 (n x p; column j is agent j's initial guess).
 *   Residues are gradients, r = A x - b (Eq. "eqbasica", Sec. 2).
 *   Algorithm 2 (cCG):
 *       R_0 = A X_0 - b 1_p^T ;  D_0 = R_0
 *       alpha_k = -R_k^T D_k (D_k^T A D_k)^{-1}
 *       X_{k+1} = X_k + D_k alpha_k^T
 *       R_{k+1} = A X_{k+1} - b 1^T, computed by the recurrence
 *                 R_{k+1} = R_k + A D_k alpha_k^T (proof of Theorem 2)
 *       beta_k  = -R_{k+1}^T A D_k (D_k^T A D_k)^{-1}
 *       D_{k+1} = R_{k+1} + D_k beta_k^T
 *   Algorithm 3 (mcCG): when D_k loses rank, keep a full-rank subset J of
 *   the agents and continue with p_k = |J| agents.
 *   Stopping rule of Algorithm 4: stop once min_j ||R_k e_j|| is below the
 *   tolerance (read as relative to ||b||).
 *
 * Readings where the paper is silent or garbled (all shared with the CUDA
 * solver by specification only, never by code):
 *   - "1_p^T b" is read as b 1_p^T (b in every column).
 *   - The residual is carried by the recurrence (Table 1 counts one n^2
 *     product per iteration); the true residual b - A x is computed at exit.
 *     With explicit_residual set, R_{k+1} = A X_{k+1} - b 1^T is formed
 *     explicitly each iteration, as Algorithm 2 prints it (a second product
 *     with A per iteration, as in Algorithm 4).
 *     If it is above tol, the residual is replaced (R = A X - b 1^T, D = R)
 *     and the iteration continues (optional).
 *   - Rank test: Cholesky of the unit-diagonal scaled Gram
 *     Mt = S M S, S = diag(M)^{-1/2}, taken greedily in agent order; agent j
 *     is dropped when its pivot is below rank_tol.  A pivot below
 *     -sqrt(rank_tol) means A is not positive definite.  The test runs on M_k at
 *     the start of iteration k (before alpha_k); J restricts X, R, D, A D.
 *     The scaled diagonal is taken as exactly one; a zero diagonal of M
 *     (a zero direction) counts as dependent; a negative one means A is not
 *     positive definite.
 *   - The stop test is min_j ||R e_j|| <= tol ||b||; the returned agent is
 *     the argmin (lowest index on ties).
 *   - Iterations = number of alpha computations (A D products in the loop).
 *   - The p x p Gram products D'AD, R'D, R'AD (Table 1, rows 2, 3 and 7),
 *     the residue norms ||R e_j|| and ||b|| are inner products that the
 *     method's analysis takes as exact (Sec. 4 works in exact arithmetic);
 *     they decide the matrix stepsizes and the stop test, and the iteration
 *     count of an ill-conditioned solve is sensitive to their rounding.  They
 *     are evaluated with the compensated dot product Dot2 of Ogita, Rump and
 *     Oishi (SIAM J. Sci. Comput. 26, 2005), which is as accurate as a dot
 *     product computed in twice the working precision and then rounded, so
 *     their value does not depend on n or on the order of summation.  The
 *     block product W = A D is a plain FP64 sum of the n products of each
 *     entry.  The method fixes no summation order; product_order picks one:
 *     0 = l ascending (the default), 1 = l descending, 2 = blocks of 64
 *     consecutive terms, each block summed first, 3 = 64 interleaved partial
 *     sums (term l into sum l mod 64), added in order at the end, 4 = the
 *     compensated sum Dot2 (nearly the exact sum rounded once).  All five
 *     are the same definition up to rounding; the tests use them to measure
 *     how far the iteration count of an ill-conditioned solve moves under
 *     rounding alone.
 *
 * Storage: every n x p block is row-major with leading dimension p
 * (element (i, j) at [i*p + j]); A is row-major with leading dimension lda.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
    ORC_OK = 0,
    ORC_NOT_CONVERGED = 1,
    ORC_ERR_INVALID = -1,
    ORC_ERR_NOT_SPD = -2,
    ORC_ERR_NUMERICAL = -3,
    ORC_ERR_OOM = -4
};

typedef struct {
    int status;
    int iterations;
    int agent;          /* original index of the returned agent */
    int p_final;        /* agents still active at exit */
    int replacements;   /* residual replacements performed */
    int drops;          /* agents removed by the rank test */
    double relres_true; /* ||b - A x|| / ||b|| of the returned x */
    double relres_recur;/* min_j ||R e_j|| / ||b|| from the recurrence */
} oracle_stats;

/* Called with the state after initialisation (k = 0, W/alpha/beta NULL) and
 * after every iteration k -> k+1 (X_{k+1}, R_{k+1}, D_{k+1}, W = A D_k,
 * alpha_k, beta_k), all with pk columns; agent[j] = original index of
 * column j.  alpha and beta are pk x pk row-major (alpha[a*pk+b] = alpha_ab). */
typedef void (*oracle_trace_fn)(void* ctx, int k, int pk, const int* agent,
                                const double* X, const double* R,
                                const double* D, const double* W,
                                const double* alpha, const double* beta);

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014; constants as in Vigna's     */
/* public-domain reference).  The value at counter c is the (c+1)-th output  */
/* of the generator seeded with `seed`.                                      */
/* ------------------------------------------------------------------------ */
uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t counter)
{
    uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Initial block when the caller gives a single x0: column 0 is x0, column
 * j >= 1 is x0 + spread * u_j with u_j(i) uniform in [-1, 1) drawn from the
 * counter c = j*n + i (top 53 bits of the SplitMix64 output). */
void oracle_initial_block(int64_t n, int p, const double* x0, double spread,
                          uint64_t seed, double* X0)
{
    for (int64_t i = 0; i < n; ++i) {
        double base = x0 ? x0[i] : 0.0;
        X0[i * p + 0] = base;
        for (int j = 1; j < p; ++j) {
            uint64_t c = (uint64_t)j * (uint64_t)n + (uint64_t)i;
            double u = (double)(oracle_splitmix64_at(seed, c) >> 11) * 0x1.0p-53;
            X0[i * p + j] = base + spread * (2.0 * u - 1.0);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Plain dense kernels.                                                      */
/* ------------------------------------------------------------------------ */

/* Error-free transformations, exact in binary64 without FMA contraction:
 * Knuth's TwoSum and Dekker's TwoProduct with Veltkamp's splitting. */
static void two_sum(double a, double b, double* s, double* e)
{
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static void split27(double a, double* hi, double* lo)
{
    double c = 134217729.0 * a; /* 2^27 + 1 */
    double h = c - (c - a);
    *hi = h;
    *lo = a - h;
}

static void two_prod(double a, double b, double* p, double* e)
{
    double x = a * b, ah, al, bh, bl;
    split27(a, &ah, &al);
    split27(b, &bh, &bl);
    *e = al * bl - (((x - ah * bh) - al * bh) - ah * bl);
    *p = x;
}

/* Dot2 accumulator: running sum s and the accumulated rounding errors c. */
typedef struct { double s, c; } dot2_t;

static void dot2_add(dot2_t* t, double x, double y)
{
    double p, e, s, f;
    two_prod(x, y, &p, &e);
    two_sum(t->s, p, &s, &f);
    t->s = s;
    t->c += e + f;
}

static double dot2_value(dot2_t t) { return t.s + t.c; }

/* W = A V (n x n times n x q).  Each entry is the FP64 sum over l of
 * A_il V_lc, in the order picked by `order` (see the header); order 4 is the
 * compensated sum Dot2 (as accurate as the plain sum in twice the working
 * precision, rounded once). */
#define ORC_BLOCK 64
static void mat_block(int64_t n, const double* A, int64_t lda, const double* V,
                      int q, double* W, int nthreads, int order)
{
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t i = 0; i < n; ++i) {
        double acc[32];
        const double* Ai = A + i * lda;
        for (int c = 0; c < q; ++c) acc[c] = 0.0;
        if (order == 1) {
            for (int64_t l = n - 1; l >= 0; --l)
                for (int c = 0; c < q; ++c) acc[c] += Ai[l] * V[l * q + c];
        } else if (order == 2) {
            for (int64_t l0 = 0; l0 < n; l0 += ORC_BLOCK) {
                double part[32];
                int64_t l1 = l0 + ORC_BLOCK < n ? l0 + ORC_BLOCK : n;
                for (int c = 0; c < q; ++c) part[c] = 0.0;
                for (int64_t l = l0; l < l1; ++l)
                    for (int c = 0; c < q; ++c) part[c] += Ai[l] * V[l * q + c];
                for (int c = 0; c < q; ++c) acc[c] += part[c];
            }
        } else if (order == 4) {
            for (int c = 0; c < q; ++c) {
                dot2_t t = {0.0, 0.0};
                for (int64_t l = 0; l < n; ++l) dot2_add(&t, Ai[l], V[l * q + c]);
                acc[c] = dot2_value(t);
            }
        } else if (order == 3) {
            for (int c = 0; c < q; ++c) {
                double part[ORC_BLOCK];
                for (int t = 0; t < ORC_BLOCK; ++t) part[t] = 0.0;
                for (int64_t l = 0; l < n; ++l) part[l % ORC_BLOCK] += Ai[l] * V[l * q + c];
                for (int t = 0; t < ORC_BLOCK; ++t) acc[c] += part[t];
            }
        } else {
            for (int64_t l = 0; l < n; ++l)
                for (int c = 0; c < q; ++c) acc[c] += Ai[l] * V[l * q + c];
        }
        for (int c = 0; c < q; ++c) W[i * q + c] = acc[c];
    }
}

/* W = A V alone, in the given order (for the tests that pin mat_block). */
void oracle_block_product(int64_t n, const double* A, int64_t lda, const double* V,
                          int q, double* W, int order)
{
    mat_block(n, A, lda, V, q, W, 1, order);
}


/* G = U^T V (q x q), G[a][b] = sum_i U[i][a] V[i][b] (Dot2, i = 0..n-1). */
static void gram(int64_t n, int q, const double* U, const double* V, double* G)
{
    dot2_t acc[32 * 32];
    for (int e = 0; e < q * q; ++e) { acc[e].s = 0.0; acc[e].c = 0.0; }
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < q; ++a)
            for (int c = 0; c < q; ++c)
                dot2_add(&acc[a * q + c], U[i * q + a], V[i * q + c]);
    for (int e = 0; e < q * q; ++e) G[e] = dot2_value(acc[e]);
}

/* Y += Z T  with Z n x q and T q x q row-major. */
static void add_block_times(int64_t n, int q, double* Y, const double* Z,
                            const double* T)
{
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < q; ++a) {
            double acc = 0.0;
            for (int c = 0; c < q; ++c) acc += Z[i * q + c] * T[c * q + a];
            Y[i * q + a] += acc;
        }
}

/* Column norms s_j = ||R e_j|| (Dot2). */
static void col_norms(int64_t n, int q, const double* R, double* s)
{
    dot2_t acc[32];
    for (int j = 0; j < q; ++j) { acc[j].s = 0.0; acc[j].c = 0.0; }
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < q; ++j) dot2_add(&acc[j], R[i * q + j], R[i * q + j]);
    for (int j = 0; j < q; ++j) s[j] = sqrt(dot2_value(acc[j]));
}

/* Keep columns listed in keep[0..m) of an n x q block, in place -> n x m. */
static void restrict_cols(int64_t n, int q, double* Y, const int* keep, int m)
{
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < m; ++c) Y[i * m + c] = Y[i * q + keep[c]];
}

static void restrict_square(int q, double* Mq, const int* keep, int m)
{
    double tmp[32 * 32];
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c) tmp[a * m + c] = Mq[keep[a] * q + keep[c]];
    memcpy(Mq, tmp, sizeof(double) * (size_t)m * (size_t)m);
}

/* ------------------------------------------------------------------------ */
/* Rank test + factor of the scaled Gram (reading of "D_k full rank",       */
/* Algorithm 2, and of the choice of J in Algorithm 3).                      */
/* On return keep[0..*m) lists the kept columns in order, sc[] holds         */
/* diag(M)^{-1/2} for them and L (m x m, row-major, lower) the Cholesky      */
/* factor of S M S restricted to the kept set.                               */
/* ------------------------------------------------------------------------ */
static int rank_factor(int q, const double* M, double rank_tol, int* keep,
                       int* m, double* sc, double* L)
{
    double s_all[32];
    double Lfull[32 * 32];
    int kept = 0;
    for (int j = 0; j < q; ++j) {
        double mjj = M[j * q + j];
        if (!(mjj == mjj)) return ORC_ERR_NUMERICAL;
        if (mjj < 0.0) return ORC_ERR_NOT_SPD;
        s_all[j] = mjj > 0.0 ? 1.0 / sqrt(mjj) : 0.0;
    }
    for (int j = 0; j < q; ++j) {
        if (M[j * q + j] == 0.0) continue; /* zero direction: dependent */
        /* row j of the factor against the kept columns so far */
        for (int t = 0; t < kept; ++t) {
            int i = keep[t];
            double v = s_all[j] * M[j * q + i] * s_all[i];
            for (int u = 0; u < t; ++u) v -= Lfull[j * 32 + u] * Lfull[i * 32 + u];
            Lfull[j * 32 + t] = v / Lfull[i * 32 + t];
        }
        double d = 1.0; /* scaled diagonal is exactly one */
        for (int u = 0; u < kept; ++u) d -= Lfull[j * 32 + u] * Lfull[j * 32 + u];
        if (!(d == d)) return ORC_ERR_NUMERICAL;
        if (d < -sqrt(rank_tol)) return ORC_ERR_NOT_SPD;
        if (d < rank_tol) continue; /* agent j depends on the kept ones */
        Lfull[j * 32 + kept] = sqrt(d);
        keep[kept++] = j;
    }
    *m = kept;
    for (int a = 0; a < kept; ++a) {
        sc[a] = s_all[keep[a]];
        for (int c = 0; c < kept; ++c)
            L[a * kept + c] = (c <= a) ? Lfull[keep[a] * 32 + c] : 0.0;
    }
    return ORC_OK;
}

/* Solve T^T = -M^{-1} Q^T for a q x q right-hand side, with
 * M = S^{-1} L L^T S^{-1}.  Q is given row-major (Q[a][c]); the result is
 * returned as T[a][c] (so T^T is the matrix applied in the block updates). */
static void neg_solve(int q, const double* sc, const double* L, const double* Q,
                      double* T)
{
    double Y[32 * 32];
    /* Y = S Q^T : Y[a][c] = sc[a] * Q[c][a] */
    for (int a = 0; a < q; ++a)
        for (int c = 0; c < q; ++c) Y[a * q + c] = sc[a] * Q[c * q + a];
    /* forward: L Z = Y (in place) */
    for (int c = 0; c < q; ++c)
        for (int a = 0; a < q; ++a) {
            double v = Y[a * q + c];
            for (int u = 0; u < a; ++u) v -= L[a * q + u] * Y[u * q + c];
            Y[a * q + c] = v / L[a * q + a];
        }
    /* backward: L^T V = Z (in place) */
    for (int c = 0; c < q; ++c)
        for (int a = q - 1; a >= 0; --a) {
            double v = Y[a * q + c];
            for (int u = a + 1; u < q; ++u) v -= L[u * q + a] * Y[u * q + c];
            Y[a * q + c] = v / L[a * q + a];
        }
    /* T^T = -S V  ->  T[c][a] = -sc[a] * V[a][c] */
    for (int a = 0; a < q; ++a)
        for (int c = 0; c < q; ++c) T[c * q + a] = -sc[a] * Y[a * q + c];
}

static int has_nan(int64_t cnt, const double* v)
{
    for (int64_t i = 0; i < cnt; ++i)
        if (!(v[i] == v[i]) || isinf(v[i])) return 1;
    return 0;
}

static double true_relres(int64_t n, const double* A, int64_t lda,
                          const double* b, const double* X, int q, int j,
                          double bnorm, int nthreads)
{
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    if (!r) return NAN;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t i = 0; i < n; ++i) {
        double ax = 0.0;
        const double* Ai = A + i * lda;
        for (int64_t l = 0; l < n; ++l) ax += Ai[l] * X[l * q + j];
        r[i] = b[i] - ax;
    }
    dot2_t acc = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) dot2_add(&acc, r[i], r[i]);
    free(r);
    return sqrt(dot2_value(acc)) / bnorm;
}

/* The p x p Gram G = U^T V of two n x q row-major blocks (q <= 32), each
 * entry a Dot2 sum (Ogita, Rump and Oishi 2005) as in every iteration of the
 * solver below; exported so that the tests can hold it against exact sums. */
void oracle_gram(int64_t n, int q, const double* U, const double* V, double* G)
{
    gram(n, q, U, V, G);
}

double oracle_true_relres(int64_t n, const double* A, int64_t lda,
                          const double* b, const double* x, int nthreads)
{
    dot2_t bacc = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) dot2_add(&bacc, b[i], b[i]);
    double bn = sqrt(dot2_value(bacc));
    if (bn == 0.0) bn = 1.0;
    return true_relres(n, A, lda, b, x, 1, 0, bn, nthreads < 1 ? 1 : nthreads);
}

/* ------------------------------------------------------------------------ */
/* The solver.                                                               */
/* ------------------------------------------------------------------------ */
int oracle_ccg(int64_t n, const double* A, int64_t lda, const double* b,
               const double* X0, int p, double tol, int maxit,
               double rank_tol, int residual_replacement, int explicit_residual,
               int product_order, int nthreads,
               double* x_out, double* X_out, int* agents_out,
               oracle_stats* st, oracle_trace_fn cb, void* cb_ctx)
{
    oracle_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof(*st));
    st->agent = -1;
    if (n < 1 || p < 1 || p > 32 || p > n || lda < n || !(tol > 0.0) ||
        maxit < 0 || !A || !b || !X0 || !x_out || !(rank_tol > 0.0)) {
        st->status = ORC_ERR_INVALID;
        return st->status;
    }
    if (nthreads < 1) nthreads = 1;

    size_t blk = (size_t)n * (size_t)p;
    double* X = (double*)malloc(sizeof(double) * blk);
    double* R = (double*)malloc(sizeof(double) * blk);
    double* D = (double*)malloc(sizeof(double) * blk);
    double* W = (double*)malloc(sizeof(double) * blk);
    double* Dn = (double*)malloc(sizeof(double) * blk);
    if (!X || !R || !D || !W || !Dn) {
        free(X); free(R); free(D); free(W); free(Dn);
        st->status = ORC_ERR_OOM;
        return st->status;
    }
    double M[32 * 32], G[32 * 32], H[32 * 32], L[32 * 32];
    double alpha[32 * 32], beta[32 * 32], sc[32], s[32];
    int agent[32], keep[32];
    int pk = p, k = 0, status = ORC_NOT_CONVERGED;
    int k_replaced = -1; /* iteration count at the last replacement */

    dot2_t bacc = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) dot2_add(&bacc, b[i], b[i]);
    double bnorm = sqrt(dot2_value(bacc));
    for (int j = 0; j < p; ++j) agent[j] = j;

    if (bnorm == 0.0) { /* x* = 0 */
        for (int64_t i = 0; i < n; ++i) x_out[i] = 0.0;
        if (X_out) memset(X_out, 0, sizeof(double) * blk);
        st->status = ORC_OK;
        st->agent = 0;
        st->p_final = p;
        if (agents_out) for (int j = 0; j < p; ++j) agents_out[j] = j;
        free(X); free(R); free(D); free(W); free(Dn);
        return ORC_OK;
    }
    if (has_nan(blk, X0) || has_nan(n, b)) {
        status = ORC_ERR_NUMERICAL;
        goto done;
    }

    /* R_0 = A X_0 - b 1^T ; D_0 = R_0   (Algorithm 2, first lines) */
    memcpy(X, X0, sizeof(double) * blk);
    mat_block(n, A, lda, X, pk, R, nthreads, product_order);
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < pk; ++j) R[i * pk + j] -= b[i];
    memcpy(D, R, sizeof(double) * blk);
    col_norms(n, pk, R, s);
    if (cb) cb(cb_ctx, 0, pk, agent, X, R, D, NULL, NULL, NULL);

    for (;;) {
        /* stop test: min_j ||R e_j|| <= tol ||b||  (Algorithm 4) */
        int jmin = 0;
        for (int j = 1; j < pk; ++j) if (s[j] < s[jmin]) jmin = j;
        if (!(s[jmin] == s[jmin])) { status = ORC_ERR_NUMERICAL; break; }
        int stop = s[jmin] <= tol * bnorm;
        if (stop || k >= maxit) {
            double tr = true_relres(n, A, lda, b, X, pk, jmin, bnorm, nthreads);
            st->relres_true = tr;
            st->relres_recur = s[jmin] / bnorm;
            st->agent = agent[jmin];
            if (tr <= tol) { status = ORC_OK; break; }
            if (k >= maxit || !residual_replacement || k == k_replaced) {
                status = ORC_NOT_CONVERGED;
                break;
            }
            /* residual replacement: R = A X - b 1^T, D = R (restart) */
            mat_block(n, A, lda, X, pk, R, nthreads, product_order);
            for (int64_t i = 0; i < n; ++i)
                for (int j = 0; j < pk; ++j) R[i * pk + j] -= b[i];
            memcpy(D, R, sizeof(double) * (size_t)n * pk);
            col_norms(n, pk, R, s);
            st->replacements++;
            k_replaced = k;
            continue;
        }

        /* W = A D_k ; M = D^T W (symmetrised) ; G = R^T D   (Table 1) */
        mat_block(n, A, lda, D, pk, W, nthreads, product_order);
        gram(n, pk, D, W, M);
        for (int a = 0; a < pk; ++a)
            for (int c = 0; c < a; ++c) {
                double v = 0.5 * (M[a * pk + c] + M[c * pk + a]);
                M[a * pk + c] = v;
                M[c * pk + a] = v;
            }
        gram(n, pk, R, D, G);

        /* rank test and factor (Algorithm 3) */
        int m = 0;
        int rc = rank_factor(pk, M, rank_tol, keep, &m, sc, L);
        if (rc != ORC_OK) { status = rc; break; }
        if (m == 0) { status = ORC_ERR_NUMERICAL; break; }
        if (m < pk) {
            restrict_cols(n, pk, X, keep, m);
            restrict_cols(n, pk, R, keep, m);
            restrict_cols(n, pk, D, keep, m);
            restrict_cols(n, pk, W, keep, m);
            restrict_square(pk, M, keep, m);
            restrict_square(pk, G, keep, m);
            for (int c = 0; c < m; ++c) agent[c] = agent[keep[c]];
            st->drops += pk - m;
            pk = m;
        }

        /* alpha_k = -G M^{-1} ; X += D alpha^T ; R += W alpha^T */
        neg_solve(pk, sc, L, G, alpha);
        double alphaT[32 * 32], betaT[32 * 32];
        for (int a = 0; a < pk; ++a)
            for (int c = 0; c < pk; ++c) alphaT[c * pk + a] = alpha[a * pk + c];
        add_block_times(n, pk, X, D, alphaT);
        if (explicit_residual) {
            /* Algorithm 2 as printed: R_{k+1} = A X_{k+1} - b 1^T */
            mat_block(n, A, lda, X, pk, R, nthreads, product_order);
            for (int64_t i = 0; i < n; ++i)
                for (int j = 0; j < pk; ++j) R[i * pk + j] -= b[i];
        } else {
            add_block_times(n, pk, R, W, alphaT);
        }

        /* beta_k = -R_{k+1}^T W M^{-1} ; D_{k+1} = R_{k+1} + D beta^T */
        gram(n, pk, R, W, H);
        neg_solve(pk, sc, L, H, beta);
        for (int a = 0; a < pk; ++a)
            for (int c = 0; c < pk; ++c) betaT[c * pk + a] = beta[a * pk + c];
        memcpy(Dn, R, sizeof(double) * (size_t)n * pk);
        add_block_times(n, pk, Dn, D, betaT);
        double* t = D; D = Dn; Dn = t;
        k++;
        col_norms(n, pk, R, s);
        if (has_nan((int64_t)pk * pk, alpha) || has_nan((int64_t)pk * pk, beta)) {
            status = ORC_ERR_NUMERICAL;
            break;
        }
        if (cb) cb(cb_ctx, k, pk, agent, X, R, D, W, alpha, beta);
    }

done:
    st->status = status;
    st->iterations = k;
    st->p_final = pk;
    if (status == ORC_OK || status == ORC_NOT_CONVERGED) {
        int jsel = 0;
        for (int j = 0; j < pk; ++j) if (agent[j] == st->agent) jsel = j;
        for (int64_t i = 0; i < n; ++i) x_out[i] = X[i * pk + jsel];
        if (X_out) {
            for (int64_t i = 0; i < n; ++i)
                for (int j = 0; j < pk; ++j) X_out[i * pk + j] = X[i * pk + j];
        }
        if (agents_out) for (int j = 0; j < pk; ++j) agents_out[j] = agent[j];
    }
    free(X); free(R); free(D); free(W); free(Dn);
    return status;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
