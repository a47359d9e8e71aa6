/*
 * FP64 CPU oracle for POD-augmented conjugate gradient
 * (Carlberg, Forstall & Tuminaro, "Krylov-subspace recycling via the
 * POD-augmented conjugate-gradient method").
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY. This is the plain, slow, obviously
 * correct reference the GPU library is checked against. Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg load it. It shares no
 * source, header, table or helper with the CUDA library, and includes nothing from it.
 *
 * Everything is double precision, single threaded, in the order the paper states the
 * steps. Matrices are CSR with 32-bit indices (row_ptr[n+1], col[nnz], val[nnz],
 * columns sorted within each row); dense n-by-k blocks are column-major (column j
 * starts at j*n); small k-by-k matrices are row-major.
 *
 * Readings where the paper is silent (also listed in the design notes):
 *  - stopping test: ||r||_2 <= tol_abs, tol_abs = tol_rel * ||b||_2, checked on r0 before
 *    the loop and after every update; at exit the true residual b - A x is formed and,
 *    if it is above tol_abs, the iteration restarts from it (residual replacement);
 *  - POD with identity metric and unit weights; numerical rank = #{lambda_i > 1e-13 lambda_1};
 *  - a Cholesky failure of W^T A W drops the basis for that system (plain PCG).
 *
 * Compile-time mistake planting: building with -DORC_MUTANT=k (k >= 1) plants one
 * plausible mistake so the pin tests can show they catch it. The normal build has
 * ORC_MUTANT = 0 and every MUT(k) is false.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif
#define MUT(k) (ORC_MUTANT == (k))

enum { ORC_OK = 0, ORC_NOT_SPD = 2, ORC_BREAKDOWN = 3, ORC_MAXIT = 4, ORC_NONFINITE = 5, ORC_ARG = 1 };

/* Reading (not in the paper; off unless orc_set_dependence_stop(1)): stage two and the
 * inner reduced solves of Section 4.3.1 stop before a direction that was numerically in
 * the span of the directions stored before it: its A-norm squared after the
 * re-A-orthogonalisation pass, gamma = phat^T (Y^T A Y) phat, is at most the A-norm
 * squared that the pass removed, sum_i c_i^2 gamma_i (Pythagoras, were the stored
 * directions exactly A-orthogonal). In exact arithmetic Algorithm 1 ends with a zero
 * residual within the reduced dimension and the pass removes nothing; in floating point,
 * once the reduced residual is rounding noise, the new directions are noise that is not
 * A-orthogonal, one Gram-Schmidt pass against them amplifies instead of removing, and the
 * iterate grows without bound. */
static int orc_dep_stop = 0;

int orc_set_dependence_stop(int on)
{
    const int old = orc_dep_stop;
    orc_dep_stop = on != 0;
    return old;
}

typedef struct {
    int status;          /* ORC_* code */
    int iters;           /* Algorithm 1 loop passes, summed over restarts */
    int refinements;     /* residual-replacement restarts */
    int w;               /* basis dimension actually used (0 after a Cholesky failure) */
    int chol_failed;     /* 1 if W^T A W was not numerically SPD */
    int pad_;
    double stage1_relres;   /* ||b - A x0||/||b|| after stage one */
    double final_relres;    /* ||b - A x||/||b|| at exit (true residual) */
    double cond_gram;       /* lambda_max/lambda_min of W^T A W (Jacobi EVD), 0 if w = 0 */
} orc_info;

/* ---------------------------------------------------------------- basic linear algebra */

/* y = A x (CSR). */
void orc_spmv(int n, const int* rp, const int* ci, const double* va, const double* x, double* y)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = rp[i] + (MUT(10) ? 1 : 0); k < rp[i + 1]; ++k) s += va[k] * x[ci[k]];
        y[i] = s;
    }
}

double orc_dot(int n, const double* a, const double* b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* G = X^T Y for column-major X (n x p) and Y (n x q); G row-major p x q. */
void orc_gram(int n, int p, const double* X, int q, const double* Y, double* G)
{
    for (int a = 0; a < p; ++a)
        for (int c = 0; c < q; ++c) G[a * q + c] = orc_dot(n, X + (size_t)a * n, Y + (size_t)c * n);
}

/* AW = A W, one column at a time (w matrix-vector products). */
void orc_spmm(int n, const int* rp, const int* ci, const double* va, int w, const double* W, double* AW)
{
    for (int j = 0; j < w; ++j) orc_spmv(n, rp, ci, va, W + (size_t)j * n, AW + (size_t)j * n);
}

/* Upper Cholesky G = R^T R of a symmetric w x w matrix (row-major; only the upper
 * triangle of G is read). Returns 0, or ORC_NOT_SPD if a pivot is not positive. */
int orc_cholesky(int w, const double* G, double* R)
{
    memset(R, 0, sizeof(double) * (size_t)w * w);
    for (int i = 0; i < w; ++i) {
        double d = G[i * w + i];
        for (int k = 0; k < i; ++k) d -= R[k * w + i] * R[k * w + i];
        if (!(d > 0.0)) return ORC_NOT_SPD;
        double rii = sqrt(d);
        R[i * w + i] = rii;
        for (int j = i + 1; j < w; ++j) {
            double s = MUT(7) ? G[j * w + i] * 0.5 : G[i * w + j];
            for (int k = 0; k < i; ++k) s -= R[k * w + i] * R[k * w + j];
            R[i * w + j] = s / rii;
        }
    }
    return ORC_OK;
}

/* Solve R^T R y = c (forward then backward substitution). */
void orc_chol_solve(int w, const double* R, const double* c, double* y)
{
    double* t = (double*)malloc(sizeof(double) * (w > 0 ? w : 1));
    for (int i = 0; i < w; ++i) {            /* R^T t = c */
        double s = c[i];
        for (int k = 0; k < i; ++k) s -= R[k * w + i] * t[k];
        t[i] = s / R[i * w + i];
    }
    for (int i = w - 1; i >= 0; --i) {       /* R y = t */
        double s = t[i];
        for (int k = i + 1; k < w; ++k) s -= R[i * w + k] * y[k];
        y[i] = s / R[i * w + i];
    }
    free(t);
}

/* Cyclic-by-row Jacobi eigensolver for a symmetric s x s matrix (Golub & Van Loan,
 * "Matrix Computations", section 8.5: two-sided rotations chosen by the 2x2 symmetric
 * Schur decomposition). G is row-major; on return evals[i] are the eigenvalues sorted in
 * decreasing order and column i of the row-major V is the matching unit eigenvector,
 * signed so that its entry of largest magnitude is positive. Returns the sweep count. */
int orc_jacobi_eig(int s, const double* G, double* evals, double* V, int max_sweeps)
{
    double* A = (double*)malloc(sizeof(double) * (size_t)s * s + 8);
    double* U = (double*)malloc(sizeof(double) * (size_t)s * s + 8);
    memcpy(A, G, sizeof(double) * (size_t)s * s);
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) U[i * s + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int i = 0; i < s * s; ++i) fro += A[i] * A[i];
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j)
                if (i != j) off += A[i * s + j] * A[i * s + j];
        if (off <= 1e-32 * fro || off == 0.0) break;
        for (int p = 0; p < s - 1; ++p) {
            for (int q = p + 1; q < s; ++q) {
                double apq = A[p * s + q];
                if (apq == 0.0) continue;
                double theta = (A[q * s + q] - A[p * s + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < s; ++k) {       /* columns p and q */
                    double akp = A[k * s + p], akq = A[k * s + q];
                    A[k * s + p] = c * akp - sn * akq;
                    A[k * s + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < s; ++k) {       /* rows p and q */
                    double apk = A[p * s + k], aqk = A[q * s + k];
                    A[p * s + k] = c * apk - sn * aqk;
                    A[q * s + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < s; ++k) {       /* V <- V J */
                    double ukp = U[k * s + p], ukq = U[k * s + q];
                    U[k * s + p] = c * ukp - sn * ukq;
                    U[k * s + q] = (MUT(9) ? -sn : sn) * ukp + c * ukq;
                }
            }
        }
    }
    /* sort by decreasing eigenvalue (selection sort keeps it obvious) */
    int* order = (int*)malloc(sizeof(int) * (s > 0 ? s : 1));
    for (int i = 0; i < s; ++i) order[i] = i;
    for (int i = 0; i < s; ++i) {
        int best = i;
        for (int j = i + 1; j < s; ++j)
            if (A[order[j] * s + order[j]] > A[order[best] * s + order[best]]) best = j;
        int tmp = order[i]; order[i] = order[best]; order[best] = tmp;
    }
    for (int i = 0; i < s; ++i) {
        int src = order[i];
        evals[i] = A[src * s + src];
        int arg = 0;
        for (int k = 1; k < s; ++k)
            if (fabs(U[k * s + src]) > fabs(U[arg * s + src])) arg = k;
        double sg = U[arg * s + src] < 0.0 ? -1.0 : 1.0;
        for (int k = 0; k < s; ++k) V[k * s + i] = sg * U[k * s + src];
    }
    free(order); free(U); free(A);
    return sweep;
}

/* ------------------------------------------------------------------ POD (Algorithm 4) */

/* POD by the eigenvalue decomposition (Appendix, Algorithm 4) with identity metric and
 * unit weights, i.e. the basis of the POD definition (Section 3.1, eigenproblem
 * S^T S V = V Sigma^2 and W = S [v_1/sigma_1 ... v_w/sigma_w]):
 *   step 1  Kbar = S^T S
 *   step 2  Kbar = V Sigma^2 V^T (symmetric EVD, decreasing eigenvalues)
 *   step 3  w = min{ i <= rank(Kbar) : sum_{k<=i} sigma_k^2 / sum_l sigma_l^2 >= energy },
 *           then capped at w_max
 *   step 4  W = S [v_1/sigma_1 ... v_w/sigma_w]
 * S is column-major n x s. W_out (column-major, room for w_max columns) receives the
 * basis, sigma2_out (length s) all eigenvalues. Returns w. */
int orc_pod_evd(int n, int s, const double* S, double energy, int w_max, double rank_tol,
                double* W_out, double* sigma2_out)
{
    if (s <= 0) return 0;
    double* K = (double*)malloc(sizeof(double) * (size_t)s * s);
    double* V = (double*)malloc(sizeof(double) * (size_t)s * s);
    orc_gram(n, s, S, s, S, K);                                  /* step 1 */
    orc_jacobi_eig(s, K, sigma2_out, V, 60);                     /* step 2 */
    double lam1 = sigma2_out[0];
    int rank = 0;
    if (lam1 > 0.0)
        for (int i = 0; i < s; ++i)
            if (sigma2_out[i] > rank_tol * lam1) rank = i + 1;
    double total = 0.0;
    for (int i = 0; i < s; ++i) total += (MUT(6) ? sqrt(fmax(sigma2_out[i], 0.0)) : fmax(sigma2_out[i], 0.0));
    int w = rank;                                                /* step 3 */
    double cum = 0.0;
    for (int i = 0; i < rank; ++i) {
        cum += MUT(6) ? sqrt(sigma2_out[i]) : sigma2_out[i];
        if (cum / total >= energy) { w = i + 1; break; }
    }
    if (w > w_max) w = w_max;
    for (int j = 0; j < w; ++j) {                                /* step 4 */
        double inv_sigma = MUT(5) ? 1.0 : 1.0 / sqrt(sigma2_out[j]);
        double* wj = W_out + (size_t)j * n;
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int k = 0; k < s; ++k) acc += S[(size_t)k * n + i] * V[k * s + j];
            wj[i] = acc * inv_sigma;
        }
    }
    free(V); free(K);
    return w;
}

/* POD with the metric Theta = A (Algorithm 4 with a metric; Section 3.3's A-norm metric,
 * under which POD minimises a bound on the A-norm error of the next solution): step 1
 * forms Kbar = S^T (A S) with the matrix-vector products A s_k, steps 2-4 as
 * orc_pod_evd. The basis is A-orthonormal: W^T A W = I. */
int orc_pod_evd_metric(int n, int s, const double* S, const int* rp, const int* ci, const double* va,
                       double energy, int w_max, double rank_tol, double* W_out, double* sigma2_out)
{
    if (s <= 0) return 0;
    double* AS = (double*)malloc(sizeof(double) * (size_t)n * s + 8);
    double* K = (double*)malloc(sizeof(double) * (size_t)s * s);
    double* V = (double*)malloc(sizeof(double) * (size_t)s * s);
    orc_spmm(n, rp, ci, va, s, S, AS);                           /* step 1 */
    orc_gram(n, s, S, s, AS, K);
    for (int a = 0; a < s; ++a)                                   /* symmetric part */
        for (int c = a + 1; c < s; ++c) {
            double m = 0.5 * (K[a * s + c] + K[c * s + a]);
            K[a * s + c] = m;
            K[c * s + a] = MUT(19) ? -m : m;
        }
    orc_jacobi_eig(s, K, sigma2_out, V, 60);                     /* step 2 */
    double lam1 = sigma2_out[0];
    int rank = 0;
    if (lam1 > 0.0)
        for (int i = 0; i < s; ++i)
            if (sigma2_out[i] > rank_tol * lam1) rank = i + 1;
    double total = 0.0;
    for (int i = 0; i < s; ++i) total += fmax(sigma2_out[i], 0.0);
    int w = rank;                                                /* step 3 */
    double cum = 0.0;
    for (int i = 0; i < rank; ++i) {
        cum += sigma2_out[i];
        if (cum / total >= energy) { w = i + 1; break; }
    }
    if (w > w_max) w = w_max;
    for (int j = 0; j < w; ++j) {                                /* step 4 */
        double inv_sigma = 1.0 / sqrt(sigma2_out[j]);
        double* wj = W_out + (size_t)j * n;
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int k = 0; k < s; ++k) acc += S[(size_t)k * n + i] * V[k * s + j];
            wj[i] = acc * inv_sigma;
        }
    }
    free(V); free(K); free(AS);
    return w;
}

/* ------------------------------------------- POD with the output metric (Algorithm 5) */

/* Thin SVD of a q x s matrix B (column-major, column j at j*q) by one-sided Jacobi
 * rotations (Hestenes' method; Golub & Van Loan §8.6): pairs of columns are rotated until
 * every pair is orthogonal; the singular values are then the column norms, and V (s x s,
 * row-major) accumulates the rotations. sigma (length s) decreasing, each column of V
 * signed with its largest-magnitude entry positive. Returns the sweeps used. */
int orc_jacobi_svd(int q, int s, const double* B, double* sigma, double* V, int max_sweeps)
{
    double* X = (double*)malloc(sizeof(double) * (size_t)q * s + 8);
    double* U = (double*)malloc(sizeof(double) * (size_t)s * s + 8);
    memcpy(X, B, sizeof(double) * (size_t)q * s);
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) U[i * s + j] = (i == j) ? 1.0 : 0.0;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < s - 1; ++p) {
            for (int r = p + 1; r < s; ++r) {
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int k = 0; k < q; ++k) {
                    double xp = X[(size_t)p * q + k], xr = X[(size_t)r * q + k];
                    alpha += xp * xp;
                    beta += xr * xr;
                    gamma += xp * xr;
                }
                if (gamma == 0.0 || fabs(gamma) <= 1e-15 * sqrt(alpha * beta)) continue;
                rotated = 1;
                /* the rotation that diagonalises [[alpha, gamma], [gamma, beta]] */
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                for (int k = 0; k < q; ++k) {
                    double xp = X[(size_t)p * q + k], xr = X[(size_t)r * q + k];
                    X[(size_t)p * q + k] = c * xp - sn * xr;
                    X[(size_t)r * q + k] = sn * xp + (MUT(17) ? -c : c) * xr;
                }
                for (int k = 0; k < s; ++k) {
                    double up = U[k * s + p], ur = U[k * s + r];
                    U[k * s + p] = c * up - sn * ur;
                    U[k * s + r] = sn * up + c * ur;
                }
            }
        }
        if (!rotated) break;
    }
    double* nrm = (double*)malloc(sizeof(double) * (size_t)(s > 0 ? s : 1));
    for (int j = 0; j < s; ++j) {
        double a = 0.0;
        for (int k = 0; k < q; ++k) a += X[(size_t)j * q + k] * X[(size_t)j * q + k];
        nrm[j] = sqrt(a);
    }
    int* order = (int*)malloc(sizeof(int) * (s > 0 ? s : 1));
    for (int i = 0; i < s; ++i) order[i] = i;
    for (int i = 0; i < s; ++i) {
        int best = i;
        for (int j = i + 1; j < s; ++j)
            if (nrm[order[j]] > nrm[order[best]]) best = j;
        int tmp = order[i]; order[i] = order[best]; order[best] = tmp;
    }
    for (int i = 0; i < s; ++i) {
        int src = order[i];
        sigma[i] = nrm[src];
        int arg = 0;
        for (int k = 1; k < s; ++k)
            if (fabs(U[k * s + src]) > fabs(U[arg * s + src])) arg = k;
        double sg = U[arg * s + src] < 0.0 ? -1.0 : 1.0;
        for (int k = 0; k < s; ++k) V[k * s + i] = sg * U[k * s + src];
    }
    free(order); free(nrm); free(U); free(X);
    return sweep;
}

/* POD with the pseudometric C^T C (Appendix, Algorithm 5; the output-oriented metric of
 * Section 3.3) and unit weights, for q output functionals (C row-major q x n):
 *   step 1  Sbar = C S                                   (q x s)
 *   step 2  thin SVD Sbar = U Sigma V^T                  (one-sided Jacobi, decreasing)
 *   step 3  w = min{ i <= rank(Sbar) : sum_{k<=i} sigma_k^2 / sum_l sigma_l^2 >= energy },
 *           capped at w_max; rank = #{sigma_i^2 > rank_tol sigma_1^2} (as Algorithm 4's)
 *   step 4  W = S [v_1/sigma_1 ... v_w/sigma_w]          (C^T C-orthonormal: (CW)^T CW = I)
 * S column-major n x s; W_out room for w_max columns; sigma2_out (length s) receives the
 * sigma_i^2. Returns w. */
int orc_pod_svd(int n, int s, const double* S, int q, const double* C, double energy, int w_max,
                double rank_tol, double* W_out, double* sigma2_out)
{
    if (s <= 0) return 0;
    double* Sb = (double*)malloc(sizeof(double) * (size_t)q * s + 8);
    double* V = (double*)malloc(sizeof(double) * (size_t)s * s + 8);
    double* sig = (double*)malloc(sizeof(double) * (size_t)s + 8);
    for (int j = 0; j < s; ++j)                                   /* step 1 */
        for (int k = 0; k < q; ++k) Sb[(size_t)j * q + k] = orc_dot(n, C + (size_t)k * n, S + (size_t)j * n);
    orc_jacobi_svd(q, s, Sb, sig, V, 60);                         /* step 2 */
    for (int i = 0; i < s; ++i) sigma2_out[i] = sig[i] * sig[i];
    double lam1 = sigma2_out[0];
    int rank = 0;
    if (lam1 > 0.0)
        for (int i = 0; i < s; ++i)
            if (sigma2_out[i] > rank_tol * lam1) rank = i + 1;
    double total = 0.0;
    for (int i = 0; i < s; ++i) total += sigma2_out[i];
    int w = rank;                                                 /* step 3 */
    double cum = 0.0;
    for (int i = 0; i < rank; ++i) {
        cum += sigma2_out[i];
        if (cum / total >= energy) { w = i + 1; break; }
    }
    if (w > w_max) w = w_max;
    for (int j = 0; j < w; ++j) {                                 /* step 4 */
        double inv_sigma = MUT(18) ? 1.0 : 1.0 / sig[j];
        double* wj = W_out + (size_t)j * n;
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int k = 0; k < s; ++k) acc += S[(size_t)k * n + i] * V[k * s + j];
            wj[i] = acc * inv_sigma;
        }
    }
    free(sig); free(V); free(Sb);
    return w;
}

/* ------------------------------------------------------------- stage one (Algorithm 2) */

/* Direct reduced solve (Section 4.1, Algorithm 2) with initial guess xbar = 0:
 *   Ahat = W^T A W, bhat = W^T b, Ahat = R^T R (Cholesky), Ahat what = bhat.
 * W column-major n x w. R (w x w row-major upper) and what (w) are outputs.
 * Returns ORC_OK or ORC_NOT_SPD when Ahat is not numerically SPD. */
int orc_stage_one(int n, const int* rp, const int* ci, const double* va, const double* b,
                  int w, const double* W, double* R, double* what)
{
    if (w <= 0) return ORC_OK;
    double* AW = (double*)malloc(sizeof(double) * (size_t)n * w);
    double* Ahat = (double*)malloc(sizeof(double) * (size_t)w * w);
    double* bhat = (double*)malloc(sizeof(double) * (size_t)w);
    orc_spmm(n, rp, ci, va, w, W, AW);
    orc_gram(n, w, W, w, AW, Ahat);
    for (int a = 0; a < w; ++a) bhat[a] = orc_dot(n, MUT(3) ? AW + (size_t)a * n : W + (size_t)a * n, b);
    int st = orc_cholesky(w, Ahat, R);
    if (st == ORC_OK) orc_chol_solve(w, R, bhat, what);
    free(bhat); free(Ahat); free(AW);
    return st;
}

/* ----------------------------------------------------- augmented PCG (Algorithm 1) */

/* mu = (W^T A W)^{-1} W^T A z, with W^T A W = R^T R from stage one (Section 4.3 reuses the
 * stage-one factor). The right-hand side is formed literally as W^T (A z). */
static void orc_aug_component(int n, const int* rp, const int* ci, const double* va, int w,
                              const double* W, const double* R, const double* z, double* Az,
                              double* rhs, double* mu)
{
    if (w <= 0) return;
    orc_spmv(n, rp, ci, va, z, Az);
    for (int a = 0; a < w; ++a) rhs[a] = orc_dot(n, W + (size_t)a * n, Az);
    orc_chol_solve(w, R, rhs, mu);
}

/* Augmented preconditioned CG (Section 2.2, Algorithm 1) with augmenting basis Y = W,
 * preconditioner M = diag(A) (Jacobi) and initial reduced coordinates xhat0:
 *   x0 = W xhat0, r0 = b - A x0, z0 = M^{-1} r0, solve W^T A W mu0 = W^T A z0, p0 = z0 - W mu0
 *   loop: gamma = (A p, p), alpha = (r, z)/gamma, x += alpha p, r -= alpha A p,
 *         z = M^{-1} r, beta = (r_new, z_new)/(r, z), solve W^T A W mu = W^T A z,
 *         p = z + beta p - W mu, exit when ||r|| <= tol_abs.
 * The residual test is also applied to r0 (zero iterations allowed). After the loop the
 * true residual b - A x is formed; if it is above tol_abs the loop restarts from it
 * (at most max_refine times). With w = 0 the W terms vanish and this is plain PCG.
 * P_out (optional, column-major n x p_cap) receives the search directions p_k in the
 * order used; gamma_out (optional, p_cap) the matching (A p_k, p_k).
 * x (length n) is the output. Returns the status; info->iters counts loop passes. */
int orc_aug_pcg(int n, const int* rp, const int* ci, const double* va, const double* b,
                int w, const double* W, const double* R, const double* xhat0,
                double tol_abs, int kmax, int max_refine, double* x, orc_info* info,
                double* P_out, double* gamma_out, int p_cap)
{
    size_t nb = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* r = (double*)malloc(nb);
    double* z = (double*)malloc(nb);
    double* p = (double*)malloc(nb);
    double* Ap = (double*)malloc(nb);
    double* Az = (double*)malloc(nb);
    double* dinv = (double*)malloc(nb);
    double* rhs = (double*)malloc(sizeof(double) * (w > 0 ? w : 1));
    double* mu = (double*)malloc(sizeof(double) * (w > 0 ? w : 1));
    int status = ORC_OK, iters = 0, refinements = 0;

    for (int i = 0; i < n; ++i) {                     /* M = diag(A) */
        double d = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == i) d += va[k];
        if (!(d > 0.0)) { status = ORC_NOT_SPD; goto done; }
        dinv[i] = MUT(4) ? d : 1.0 / d;
    }
    for (int i = 0; i < n; ++i) x[i] = 0.0;           /* x0 = W xhat0 (xbar = 0) */
    for (int a = 0; a < w; ++a)
        for (int i = 0; i < n; ++i) x[i] += W[(size_t)a * n + i] * xhat0[a];
    orc_spmv(n, rp, ci, va, x, Ap);                   /* r0 = b - A x0 */
    for (int i = 0; i < n; ++i) r[i] = b[i] - Ap[i];

    for (;;) {   /* one pass of Algorithm 1 from the current (true) residual r */
        for (int i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        orc_aug_component(n, rp, ci, va, w, W, R, z, Az, rhs, mu);
        for (int i = 0; i < n; ++i) p[i] = z[i];
        for (int a = 0; a < w; ++a)
            for (int i = 0; i < n; ++i) p[i] -= W[(size_t)a * n + i] * mu[a];
        double rz = orc_dot(n, r, z);
        double rnorm = sqrt(orc_dot(n, r, r));
        if (!isfinite(rnorm)) { status = ORC_NONFINITE; break; }
        while (rnorm > tol_abs) {
            if (iters >= kmax) { status = ORC_MAXIT; break; }
            orc_spmv(n, rp, ci, va, p, Ap);
            double gamma = orc_dot(n, Ap, p);
            if (P_out && iters < p_cap) {
                memcpy(P_out + (size_t)iters * n, p, nb);
                if (gamma_out) gamma_out[iters] = gamma;
            }
            if (!isfinite(gamma)) { status = ORC_NONFINITE; break; }
            if (!(gamma > 0.0)) { status = ORC_BREAKDOWN; break; }
            double alpha = rz / gamma;
            for (int i = 0; i < n; ++i) x[i] += alpha * p[i];
            for (int i = 0; i < n; ++i) r[i] -= alpha * (MUT(8) ? p[i] : Ap[i]);
            for (int i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
            double rz_new = orc_dot(n, r, z);
            double beta = rz_new / rz;
            orc_aug_component(n, rp, ci, va, w, W, R, z, Az, rhs, mu);
            for (int i = 0; i < n; ++i) p[i] = z[i] + (MUT(1) ? 0.0 : beta) * p[i];
            for (int a = 0; a < w; ++a)
                for (int i = 0; i < n; ++i)
                    p[i] += (MUT(2) ? 1.0 : -1.0) * W[(size_t)a * n + i] * mu[a];
            rz = rz_new;
            rnorm = sqrt(orc_dot(n, r, r));
            ++iters;
            if (!isfinite(rnorm)) { status = ORC_NONFINITE; break; }
        }
        if (status != ORC_OK) break;
        orc_spmv(n, rp, ci, va, x, Ap);               /* true residual */
        for (int i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
        if (sqrt(orc_dot(n, r, r)) <= tol_abs) break;
        if (refinements >= max_refine) { status = ORC_MAXIT; break; }
        ++refinements;                                /* residual replacement */
    }
done:
    info->status = status;
    info->iters = iters;
    info->refinements = refinements;
    free(mu); free(rhs); free(dinv); free(Az); free(Ap); free(p); free(z); free(r);
    return status;
}

/* Plain Jacobi-preconditioned CG from x0 (Section 2.1, optimality (KrylovSolve)), written
 * on its own so that Algorithm 1 with an empty basis can be checked against it. */
int orc_pcg(int n, const int* rp, const int* ci, const double* va, const double* b,
            const double* x0, double tol_abs, int kmax, double* x, int* iters_out)
{
    size_t nb = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* r = (double*)malloc(nb);
    double* z = (double*)malloc(nb);
    double* p = (double*)malloc(nb);
    double* q = (double*)malloc(nb);
    double* dinv = (double*)malloc(nb);
    int status = ORC_OK, k = 0;
    for (int i = 0; i < n; ++i) x[i] = x0 ? x0[i] : 0.0;
    orc_spmv(n, rp, ci, va, x, q);
    for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
    for (int i = 0; i < n; ++i) {                     /* M = diag(A) */
        double d = 0.0;
        for (int kk = rp[i]; kk < rp[i + 1]; ++kk)
            if (ci[kk] == i) d += va[kk];
        if (!(d > 0.0)) { status = ORC_NOT_SPD; goto out; }
        dinv[i] = 1.0 / d;
    }
    for (int i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
    for (int i = 0; i < n; ++i) p[i] = z[i];
    double rz = orc_dot(n, r, z);
    while (sqrt(orc_dot(n, r, r)) > tol_abs) {
        if (k >= kmax) { status = ORC_MAXIT; break; }
        orc_spmv(n, rp, ci, va, p, q);
        double pq = orc_dot(n, q, p);
        if (!(pq > 0.0)) { status = ORC_BREAKDOWN; break; }
        double alpha = rz / pq;
        for (int i = 0; i < n; ++i) x[i] += alpha * p[i];
        for (int i = 0; i < n; ++i) r[i] -= alpha * q[i];
        for (int i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        double rz_new = orc_dot(n, r, z);
        double beta = rz_new / rz;
        for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rz = rz_new;
        ++k;
    }
out:
    *iters_out = k;
    free(dinv); free(q); free(p); free(z); free(r);
    return status;
}

/* --------------------------------------------------------------- one system, end to end */

/* Solve system j of the sequence (Section 2, (sequenceInexact)) with augmenting basis W:
 * stage one (Algorithm 2) when w > 0, then Algorithm 1 started from the stage-one
 * coordinates, with tol_abs = tol_rel ||b||_2. If W^T A W is not numerically SPD the basis
 * is dropped for this system (info->chol_failed = 1) and plain PCG runs instead.
 * cond_gram is the 2-norm condition number of W^T A W from the Jacobi eigensolver
 * (the diagnostic of Section 5.2's reduced-matrix conditioning). */
int orc_solve_system(int n, const int* rp, const int* ci, const double* va, const double* b,
                     int w, const double* W, double tol_rel, int kmax, int max_refine,
                     double* x, orc_info* info, double* P_out, double* gamma_out, int p_cap)
{
    memset(info, 0, sizeof(*info));
    double bnorm = sqrt(orc_dot(n, b, b));
    double tol_abs = tol_rel * bnorm;
    double* R = (double*)malloc(sizeof(double) * (size_t)(w > 0 ? w * w : 1));
    double* what = (double*)calloc((size_t)(w > 0 ? w : 1), sizeof(double));
    int wu = w;
    if (w > 0) {
        int st = orc_stage_one(n, rp, ci, va, b, w, W, R, what);
        if (st != ORC_OK) { info->chol_failed = 1; wu = 0; }
        else {
            double* AW = (double*)malloc(sizeof(double) * (size_t)n * w);
            double* G = (double*)malloc(sizeof(double) * (size_t)w * w);
            double* ev = (double*)malloc(sizeof(double) * (size_t)w);
            double* V = (double*)malloc(sizeof(double) * (size_t)w * w);
            orc_spmm(n, rp, ci, va, w, W, AW);
            orc_gram(n, w, W, w, AW, G);
            for (int a = 0; a < w; ++a)          /* symmetric part, upper triangle as read */
                for (int c = 0; c < a; ++c) G[a * w + c] = G[c * w + a];
            orc_jacobi_eig(w, G, ev, V, 60);
            info->cond_gram = ev[w - 1] > 0.0 ? ev[0] / ev[w - 1] : INFINITY;
            free(V); free(ev); free(G); free(AW);
        }
    }
    info->w = wu;
    /* stage-one residual */
    {
        double* x0 = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        double* r0 = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        for (int a = 0; a < wu; ++a)
            for (int i = 0; i < n; ++i) x0[i] += W[(size_t)a * n + i] * what[a];
        orc_spmv(n, rp, ci, va, x0, r0);
        for (int i = 0; i < n; ++i) r0[i] = b[i] - r0[i];
        info->stage1_relres = bnorm > 0.0 ? sqrt(orc_dot(n, r0, r0)) / bnorm : 0.0;
        free(r0); free(x0);
    }
    int chol = info->chol_failed;
    double cond = info->cond_gram, s1 = info->stage1_relres;
    int st = orc_aug_pcg(n, rp, ci, va, b, wu, W, R, what, tol_abs, kmax, max_refine, x, info,
                         P_out, gamma_out, p_cap);
    info->chol_failed = chol; info->cond_gram = cond; info->stage1_relres = s1; info->w = wu;
    {
        double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        orc_spmv(n, rp, ci, va, x, q);
        double rr = 0.0;
        for (int i = 0; i < n; ++i) rr += (b[i] - q[i]) * (b[i] - q[i]);
        info->final_relres = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
        free(q);
    }
    free(what); free(R);
    return st;
}

/* ------------------------------------- stage two (Section 4.2) and stage three (Section 4.3) */

/* Reduced product qhat = Y^T (A (Y phat)) (Section 4.2): Y^T A Y is never formed; the
 * product costs one matrix-vector product and two passes over Y. v receives Y phat and
 * Av receives A v (length n each). */
static void orc_reduced_product(int n, const int* rp, const int* ci, const double* va, int y,
                                const double* Y, const double* phat, double* v, double* Av, double* qhat)
{
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    for (int l = 0; l < y; ++l)
        for (int i = 0; i < n; ++i) v[i] += Y[(size_t)l * n + i] * phat[l];
    orc_spmv(n, rp, ci, va, v, Av);
    for (int l = 0; l < y; ++l) qhat[l] = orc_dot(n, Y + (size_t)l * n, Av);
}

/* Stage two (Section 4.2): Algorithm 1 applied to the reduced system
 *     (Y^T A Y) yhat = Y^T b                    (xbar = 0)
 * from yhat0 = Phi what with augmenting basis Phi = [I_w; 0] (the stage-one basis in
 * augmenting-subspace coordinates: W = Y Phi is the first w columns of Y), preconditioner
 * M = I and absolute tolerance tol_abs on ||rhat||, for at most kcap iterations. The
 * augmentation solves Phi^T (Y^T A Y) Phi mu = Phi^T (Y^T A Y) zhat reuse the stage-one
 * factor (Phi^T Y^T A Y Phi = W^T A W = R^T R); their right-hand sides are formed
 * literally, with one more reduced product. rhat0 is tested before the loop.
 * Outputs: *k2 iterations; alpha[k] the step lengths (the coordinates of the increment in
 * the stage-two basis); V2 (n x k2 column-major, may be NULL) the lifted directions
 * Y phat_k, i.e. the stage-two basis V2 = Y Phi2; T2[k] = (Y^T A Y phat_k, phat_k), the
 * diagonal of V2^T A V2; *rhat_norm the final ||rhat||. A non-positive or non-finite
 * (Y^T A Y phat, phat) ends stage two with the directions accepted so far.
 * Reading (not in Algorithm 1): every new direction is re-A-orthogonalised against the
 * directions taken so far, phat -= sum_i (qhat_i^T phat / T2[i]) phat_i with the stored
 * reduced products qhat_i = Y^T A Y phat_i (classical Gram-Schmidt, one pass, in the order
 * i = 0..k). In exact arithmetic the correction is zero; in floating point CG directions
 * lose their mutual A-orthogonality once the reduced residual has fallen far (cond(Y^T A Y)
 * is large for an identity-metric POD basis), and stage three uses V2 as an explicit basis
 * whose factor blockdiag(R, sqrt(T2)) assumes that orthogonality. */
static int orc_stage_two_hist(int n, const int* rp, const int* ci, const double* va, const double* b,
                              int y, const double* Y, int w, const double* R, const double* what,
                              double tol_abs, int kcap, int* k2, double* alpha, double* V2, double* T2,
                              double* rhat_norm, double* Ph_out, double* Qh_out)
{
    size_t nb = sizeof(double) * (size_t)(n > 0 ? n : 1);
    size_t yb = sizeof(double) * (size_t)(y > 0 ? y : 1);
    double* v = (double*)malloc(nb);
    double* Av = (double*)malloc(nb);
    double* xh = (double*)calloc(1, yb);
    double* rh = (double*)malloc(yb);
    double* zh = (double*)malloc(yb);
    double* ph = (double*)malloc(yb);
    double* qh = (double*)malloc(yb);
    double* th = (double*)malloc(yb);
    double* mu = (double*)malloc(sizeof(double) * (size_t)(w > 0 ? w : 1));
    double* Ph = (double*)malloc(yb * (size_t)(kcap > 0 ? kcap : 1));   /* directions taken */
    double* Qh = (double*)malloc(yb * (size_t)(kcap > 0 ? kcap : 1));   /* their reduced products */
    double* cf = (double*)malloc(sizeof(double) * (size_t)(kcap > 0 ? kcap : 1));
    int k = 0, status = ORC_OK;

    for (int l = 0; l < y; ++l) xh[l] = (l < w) ? what[l] : 0.0;          /* step 1 */
    orc_reduced_product(n, rp, ci, va, y, Y, xh, v, Av, qh);             /* step 2 */
    for (int l = 0; l < y; ++l)
        rh[l] = orc_dot(n, Y + (size_t)l * n, b) - (MUT(14) ? 0.0 : qh[l]);
    for (int l = 0; l < y; ++l) zh[l] = rh[l];                            /* step 3, M = I */
    if (w > 0) {                                                          /* step 4 */
        orc_reduced_product(n, rp, ci, va, y, Y, zh, v, Av, th);
        orc_chol_solve(w, R, th, mu);
    }
    for (int l = 0; l < y; ++l) ph[l] = zh[l] - ((l < w) ? mu[l] : 0.0);  /* step 5 */
    double rz = 0.0, rr = 0.0;
    for (int l = 0; l < y; ++l) { rz += rh[l] * zh[l]; rr += rh[l] * rh[l]; }
    double rnorm = sqrt(rr);
    double removed = 0.0;   /* A-norm squared removed from the next direction by the pass */
    while (rnorm > tol_abs && k < kcap) {
        orc_reduced_product(n, rp, ci, va, y, Y, ph, v, Av, qh);
        double gamma = 0.0;
        for (int l = 0; l < y; ++l) gamma += qh[l] * ph[l];
        if (!isfinite(gamma) || !(gamma > 0.0)) { status = ORC_BREAKDOWN; break; }
        if (orc_dep_stop && gamma <= removed) break;   /* numerically dependent direction */
        double a = rz / gamma;
        alpha[k] = a;
        T2[k] = gamma;
        memcpy(Ph + (size_t)k * y, ph, yb);
        memcpy(Qh + (size_t)k * y, qh, yb);
        if (V2) memcpy(V2 + (size_t)k * n, v, nb);
        for (int l = 0; l < y; ++l) xh[l] += a * ph[l];
        for (int l = 0; l < y; ++l) rh[l] -= a * qh[l];
        for (int l = 0; l < y; ++l) zh[l] = rh[l];
        double rz_new = 0.0;
        rr = 0.0;
        for (int l = 0; l < y; ++l) { rz_new += rh[l] * zh[l]; rr += rh[l] * rh[l]; }
        double beta = rz_new / rz;
        if (w > 0) {
            orc_reduced_product(n, rp, ci, va, y, Y, zh, v, Av, th);
            orc_chol_solve(w, R, th, mu);
        }
        for (int l = 0; l < y; ++l)
            ph[l] = zh[l] + beta * ph[l] - ((l < w && !MUT(12)) ? mu[l] : 0.0);
        removed = 0.0;
        for (int i = 0; i <= k && !MUT(15); ++i) {          /* re-A-orthogonalisation */
            double c = 0.0;
            for (int l = 0; l < y; ++l) c += Qh[(size_t)i * y + l] * ph[l];
            cf[i] = c / T2[i];
            removed += MUT(20) ? cf[i] : cf[i] * c;
        }
        for (int l = 0; l < y && !MUT(15); ++l) {
            double t = 0.0;
            for (int i = 0; i <= k; ++i) t += cf[i] * Ph[(size_t)i * y + l];
            ph[l] -= t;
        }
        rz = rz_new;
        rnorm = sqrt(rr);
        ++k;
    }
    *k2 = k;
    *rhat_norm = rnorm;
    if (Ph_out) memcpy(Ph_out, Ph, yb * (size_t)k);
    if (Qh_out) memcpy(Qh_out, Qh, yb * (size_t)k);
    free(cf); free(Qh); free(Ph);
    free(mu); free(th); free(qh); free(ph); free(zh); free(rh); free(xh); free(Av); free(v);
    return status;
}

int orc_stage_two(int n, const int* rp, const int* ci, const double* va, const double* b,
                  int y, const double* Y, int w, const double* R, const double* what,
                  double tol_abs, int kcap, int* k2, double* alpha, double* V2, double* T2,
                  double* rhat_norm)
{
    return orc_stage_two_hist(n, rp, ci, va, b, y, Y, w, R, what, tol_abs, kcap, k2, alpha, V2, T2, rhat_norm,
                              NULL, NULL);
}

/* One system by the three-stage algorithm (Section 4; the overall algorithm with the stage-
 * three option of Section 4.3, whose augmenting basis is [W, V2]):
 *   stage one   Algorithm 2 on W = the first w columns of Y (R, what); if W^T A W is not
 *               numerically SPD the stage-one basis is dropped (w = 0);
 *   stage two   Section 4.2 over range(Y) to tol_abs2 = tol2_rel * tol_rel * ||b||: V2, alpha,
 *               T2, with at most min(y - w, w3_cap - w) iterations (the reduced system's
 *               dimension less the stage-one directions it deflates; w3_cap bounds the
 *               stage-three basis dimension w + k2);
 *   stage three Algorithm 1 on A x = b with augmenting basis [W, V2], initial coordinates
 *               [what; alpha] and the Cholesky factor blockdiag(R, sqrt(T2)) of
 *               [W, V2]^T A [W, V2], known from stages one and two (Section 4.3).
 * info as orc_solve_system (info->w = w + k2, the stage-three basis dimension); *k2_out the
 * stage-two iterations; *s2_relres = ||b - A x_2||/||b|| at x_2 = W what + V2 alpha.
 * P_out/gamma_out/p_cap: stage-three directions as orc_aug_pcg. tol3_rel >= 0 replaces
 * tol_rel in stage three's own test only (stage two keeps tol2_rel * tol_rel * ||b||), so a
 * run can be replayed to a given stage-three iteration count with tol3_rel = 0. */
int orc_solve_system3(int n, const int* rp, const int* ci, const double* va, const double* b,
                      int y, const double* Y, int w, double tol_rel, double tol2_rel, int w3_cap,
                      int kmax, int max_refine, double* x, orc_info* info, int* k2_out,
                      double* s2_relres, double* P_out, double* gamma_out, int p_cap, double tol3_rel)
{
    memset(info, 0, sizeof(*info));
    if (w > y) w = y;
    double bnorm = sqrt(orc_dot(n, b, b));
    double tol_abs = tol_rel * bnorm;
    double tol3_abs = (tol3_rel >= 0.0 ? tol3_rel : tol_rel) * bnorm;
    int cap = (y < w3_cap ? y : w3_cap);   /* room for w + k2 columns */
    if (cap < w) cap = w;
    int wt = cap;
    double* R = (double*)calloc((size_t)(w > 0 ? w * w : 1), sizeof(double));
    double* what = (double*)calloc((size_t)(wt > 0 ? wt : 1), sizeof(double));
    double* B = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(wt > 0 ? wt : 1));
    double* R3 = (double*)calloc((size_t)(wt > 0 ? wt * wt : 1), sizeof(double));
    double* T2 = (double*)malloc(sizeof(double) * (size_t)(wt > 0 ? wt : 1));
    double* vv = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int wu = w;
    if (w > 0 && orc_stage_one(n, rp, ci, va, b, w, Y, R, what) != ORC_OK) {   /* stage one */
        info->chol_failed = 1;
        wu = 0;
        for (int a = 0; a < w; ++a) what[a] = 0.0;
    }
    {   /* stage-one residual */
        for (int i = 0; i < n; ++i) vv[i] = 0.0;
        for (int a = 0; a < wu; ++a)
            for (int i = 0; i < n; ++i) vv[i] += Y[(size_t)a * n + i] * what[a];
        double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        orc_spmv(n, rp, ci, va, vv, q);
        double rr = 0.0;
        for (int i = 0; i < n; ++i) rr += (b[i] - q[i]) * (b[i] - q[i]);
        info->stage1_relres = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
        free(q);
    }
    int k2 = 0;                                                            /* stage two */
    double rhat = 0.0;
    orc_stage_two(n, rp, ci, va, b, y, Y, wu, R, what, tol2_rel * tol_abs, cap - wu, &k2,
                  what + wu, B + (size_t)wu * n, T2, &rhat);
    /* stage-three basis [W, V2] and factor blockdiag(R, sqrt(T2)) */
    memcpy(B, Y, sizeof(double) * (size_t)n * (size_t)wu);
    int w3 = wu + k2;
    for (int a = 0; a < wu; ++a)
        for (int c = 0; c < wu; ++c) R3[a * w3 + c] = R[a * wu + c];
    for (int k = 0; k < k2; ++k) R3[(wu + k) * w3 + wu + k] = MUT(13) ? T2[k] : sqrt(T2[k]);
    {   /* stage-two residual */
        for (int i = 0; i < n; ++i) vv[i] = 0.0;
        for (int a = 0; a < w3; ++a)
            for (int i = 0; i < n; ++i) vv[i] += B[(size_t)a * n + i] * what[a];
        double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        orc_spmv(n, rp, ci, va, vv, q);
        double rr = 0.0;
        for (int i = 0; i < n; ++i) rr += (b[i] - q[i]) * (b[i] - q[i]);
        *s2_relres = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
        free(q);
    }
    int chol = info->chol_failed;
    double s1 = info->stage1_relres;
    int st = orc_aug_pcg(n, rp, ci, va, b, w3, B, R3, what, tol3_abs, kmax, max_refine, x, info,  /* stage three */
                         P_out, gamma_out, p_cap);
    info->chol_failed = chol; info->stage1_relres = s1; info->w = w3;
    {
        double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        orc_spmv(n, rp, ci, va, x, q);
        double rr = 0.0;
        for (int i = 0; i < n; ++i) rr += (b[i] - q[i]) * (b[i] - q[i]);
        info->final_relres = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
        free(q);
    }
    *k2_out = k2;
    free(vv); free(T2); free(R3); free(B); free(what); free(R);
    return st;
}

/* ----------------------------------- stage three over the entire augmenting basis (4.3.1) */

/* Inner reduced solve of the "it" stage three (Section 4.3.1): Algorithm 1 on
 *     (Y^T A Y) mu = chat
 * with augmenting basis Psi = [Phi, psi_0 .. psi_{m-1}] (the stage-one coordinates Phi and
 * the reduced directions stored so far by stage two and by earlier inner solves; their
 * factor is blockdiag(R, sqrt(g_i)) by construction), preconditioner M = I and absolute
 * tolerance tol_abs on ||rhat||. Reading: the solve starts from the Galerkin solution over
 * range(Psi), mu0 = Phi R^{-1} R^{-T} Phi^T chat + sum_i psi_i (psi_i^T chat) / g_i; from
 * mu0 = 0, as printed, Psi^T rhat would keep the value Psi^T chat (every direction is
 * A-orthogonal to Psi) and the residual could not fall below it. The directions it takes are
 * appended to Psi (psi, their reduced products qpsi and g; at most m_cap in total) and each
 * new direction is re-A-orthogonalised against all stored ones, as in stage two. The
 * augmentation right-hand side Phi^T (Y^T A Y) zhat is formed literally, with a reduced
 * product. mu (length y) receives the solution; returns the iterations taken. */
static int orc_inner_solve(int n, const int* rp, const int* ci, const double* va, int y, const double* Y,
                           int w, const double* R, double* psi, double* qpsi, double* g, int* m, int m_cap,
                           const double* chat, double tol_abs, double* mu)
{
    size_t yb = sizeof(double) * (size_t)(y > 0 ? y : 1);
    double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* Av = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* rh = (double*)malloc(yb);
    double* ph = (double*)malloc(yb);
    double* qh = (double*)malloc(yb);
    double* th = (double*)malloc(yb);
    double* nu = (double*)malloc(sizeof(double) * (size_t)(w > 0 ? w : 1));
    double* cf = (double*)malloc(sizeof(double) * (size_t)(m_cap > 0 ? m_cap : 1));
    int k = 0;
    /* Galerkin start over range(Psi) */
    for (int l = 0; l < y; ++l) mu[l] = 0.0;
    if (w > 0 && !MUT(16)) {
        orc_chol_solve(w, R, chat, nu);
        for (int a = 0; a < w; ++a) mu[a] += nu[a];
    }
    for (int i = 0; i < *m && !MUT(16); ++i) {
        double c = 0.0;
        for (int l = 0; l < y; ++l) c += psi[(size_t)i * y + l] * chat[l];
        c /= g[i];
        for (int l = 0; l < y; ++l) mu[l] += c * psi[(size_t)i * y + l];
    }
    orc_reduced_product(n, rp, ci, va, y, Y, mu, v, Av, qh);      /* rhat0 = chat - Ahat mu0 */
    for (int l = 0; l < y; ++l) rh[l] = chat[l] - qh[l];
    if (w > 0) {                                                   /* zhat = rhat (M = I); aug */
        orc_reduced_product(n, rp, ci, va, y, Y, rh, v, Av, th);
        orc_chol_solve(w, R, th, nu);
    }
    for (int l = 0; l < y; ++l) ph[l] = rh[l] - ((l < w) ? nu[l] : 0.0);
    double removed = 0.0;   /* A-norm squared removed from the next direction by the pass */
    for (int i = 0; i < *m; ++i) {
        double c = 0.0;
        for (int l = 0; l < y; ++l) c += qpsi[(size_t)i * y + l] * ph[l];
        cf[i] = c / g[i];
        removed += cf[i] * c;
    }
    for (int l = 0; l < y; ++l) {
        double t = 0.0;
        for (int i = 0; i < *m; ++i) t += cf[i] * psi[(size_t)i * y + l];
        ph[l] -= t;
    }
    double rz = 0.0;
    for (int l = 0; l < y; ++l) rz += rh[l] * rh[l];
    double rnorm = sqrt(rz);
    while (rnorm > tol_abs && *m < m_cap) {
        orc_reduced_product(n, rp, ci, va, y, Y, ph, v, Av, qh);
        double gamma = 0.0;
        for (int l = 0; l < y; ++l) gamma += qh[l] * ph[l];
        if (!isfinite(gamma) || !(gamma > 0.0)) break;
        if (orc_dep_stop && gamma <= removed) break;   /* numerically dependent direction */
        double a = rz / gamma;
        memcpy(psi + (size_t)(*m) * y, ph, yb);
        memcpy(qpsi + (size_t)(*m) * y, qh, yb);
        g[*m] = gamma;
        *m += 1;
        for (int l = 0; l < y; ++l) mu[l] += a * ph[l];
        for (int l = 0; l < y; ++l) rh[l] -= a * qh[l];
        double rz_new = 0.0;
        for (int l = 0; l < y; ++l) rz_new += rh[l] * rh[l];
        double beta = rz_new / rz;
        if (w > 0) {
            orc_reduced_product(n, rp, ci, va, y, Y, rh, v, Av, th);
            orc_chol_solve(w, R, th, nu);
        }
        for (int l = 0; l < y; ++l) ph[l] = rh[l] + beta * ph[l] - ((l < w) ? nu[l] : 0.0);
        removed = 0.0;
        for (int i = 0; i < *m; ++i) {
            double c = 0.0;
            for (int l = 0; l < y; ++l) c += qpsi[(size_t)i * y + l] * ph[l];
            cf[i] = c / g[i];
            removed += cf[i] * c;
        }
        for (int l = 0; l < y; ++l) {
            double t = 0.0;
            for (int i = 0; i < *m; ++i) t += cf[i] * psi[(size_t)i * y + l];
            ph[l] -= t;
        }
        rz = rz_new;
        rnorm = sqrt(rz);
        ++k;
    }
    free(cf); free(nu); free(th); free(qh); free(ph); free(rh); free(Av); free(v);
    return k;
}

/* One system by the three-stage algorithm with the stage-three option of Section 4.3.1
 * (orthogonalisation against the entire augmenting subspace, the "it" variant):
 *   stage one   Algorithm 2 on W = the first w columns of Y (R, what);
 *   stage two   Section 4.2 to tol2_rel * tol_rel * ||b|| (as orc_solve_system3), keeping
 *               its reduced directions, products and T2;
 *   stage three Algorithm 1 on A x = b with augmenting basis Y, initial coordinates the
 *               stage-two solution [what; 0] + Phi2 alpha, Jacobi preconditioner, tol_rel;
 *               each augmentation solve (Y^T A Y) mu = Y^T (A z) is the inner reduced solve
 *               above, to tol_in * ||Y^T A z||, its directions accumulating over the
 *               iterations (at most y - w directions in all, so the inner work of a whole
 *               solve is bounded by y - w reduced products). Reading: tol_in is relative to
 *               the inner right-hand side and must be tight (the callers use 1e-12); the
 *               paper's 1e-2 eps_j (absolute) presumes a well-conditioned Y^T A Y, and with an
 *               identity-metric Y inexact projections made stage three diverge (relative
 *               1e-8 still did on a 20-mode basis; 1e-10 converged).
 *               The augmentation solve is skipped once the exit test is met (its direction
 *               would not be used).
 * info as orc_solve_system (info->w = y); *k2_out the stage-two iterations; *inner_out the
 * inner reduced iterations summed over the solve; P_out/gamma_out/p_cap: the stage-three
 * directions as orc_aug_pcg. */
int orc_solve_system3_it(int n, const int* rp, const int* ci, const double* va, const double* b,
                         int y, const double* Y, int w, double tol_rel, double tol2_rel, double tol_in,
                         int kmax, int max_refine, double* x, orc_info* info, int* k2_out, int* inner_out,
                         double* P_out, double* gamma_out, int p_cap)
{
    memset(info, 0, sizeof(*info));
    if (w > y) w = y;
    size_t nb = sizeof(double) * (size_t)(n > 0 ? n : 1);
    size_t yb = sizeof(double) * (size_t)(y > 0 ? y : 1);
    int cap = y > 0 ? y : 1;
    double bnorm = sqrt(orc_dot(n, b, b));
    double tol_abs = tol_rel * bnorm;
    double* R = (double*)calloc((size_t)(w > 0 ? w * w : 1), sizeof(double));
    double* what = (double*)calloc((size_t)cap, sizeof(double));
    double* psi = (double*)malloc(yb * (size_t)cap);
    double* qpsi = (double*)malloc(yb * (size_t)cap);
    double* g = (double*)malloc(sizeof(double) * (size_t)cap);
    double* alpha2 = (double*)malloc(sizeof(double) * (size_t)cap);
    double* xh = (double*)malloc(yb);
    double* chat = (double*)malloc(yb);
    double* mu = (double*)malloc(yb);
    double* r = (double*)malloc(nb);
    double* z = (double*)malloc(nb);
    double* p = (double*)malloc(nb);
    double* q = (double*)malloc(nb);
    double* u = (double*)malloc(nb);
    double* dinv = (double*)malloc(nb);
    int wu = w, status = ORC_OK, iters = 0, refinements = 0, inner = 0;
    if (w > 0 && orc_stage_one(n, rp, ci, va, b, w, Y, R, what) != ORC_OK) {   /* stage one */
        info->chol_failed = 1;
        wu = 0;
        for (int a = 0; a < w; ++a) what[a] = 0.0;
    }
    int k2 = 0, m = 0, m_cap = y - wu;
    double rhat = 0.0;
    orc_stage_two_hist(n, rp, ci, va, b, y, Y, wu, R, what, tol2_rel * tol_abs, m_cap, &k2, alpha2,   /* stage two */
                       NULL, g, &rhat, psi, qpsi);
    m = k2;
    for (int l = 0; l < y; ++l) xh[l] = (l < wu) ? what[l] : 0.0;   /* stage-two solution, reduced */
    for (int k = 0; k < k2; ++k)
        for (int l = 0; l < y; ++l) xh[l] += alpha2[k] * psi[(size_t)k * y + l];
    for (int i = 0; i < n; ++i) {                                   /* M = diag(A) */
        double d = 0.0;
        for (int kk = rp[i]; kk < rp[i + 1]; ++kk)
            if (ci[kk] == i) d += va[kk];
        if (!(d > 0.0)) { status = ORC_NOT_SPD; goto done; }
        dinv[i] = 1.0 / d;
    }
    for (int i = 0; i < n; ++i) {                                   /* x0 = Y xhat0 */
        double t = 0.0;
        for (int l = 0; l < y; ++l) t += Y[(size_t)l * n + i] * xh[l];
        x[i] = t;
    }
    orc_spmv(n, rp, ci, va, x, q);                                  /* r0 = b - A x0 */
    for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
    {
        double rr = 0.0;
        for (int i = 0; i < n; ++i) rr += r[i] * r[i];
        info->stage1_relres = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;   /* after stages one and two */
    }
    for (;;) {   /* one pass of Algorithm 1 from the current (true) residual */
        for (int i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        orc_spmv(n, rp, ci, va, z, u);                              /* Y^T A z; inner solve */
        for (int l = 0; l < y; ++l) chat[l] = orc_dot(n, Y + (size_t)l * n, u);
        {
            double cn = 0.0;
            for (int l = 0; l < y; ++l) cn += chat[l] * chat[l];
            inner += orc_inner_solve(n, rp, ci, va, y, Y, wu, R, psi, qpsi, g, &m, m_cap, chat, tol_in * sqrt(cn), mu);
        }
        for (int i = 0; i < n; ++i) {                               /* p0 = z0 - Y mu0 */
            double t = 0.0;
            for (int l = 0; l < y; ++l) t += Y[(size_t)l * n + i] * mu[l];
            p[i] = z[i] - t;
        }
        double rz = orc_dot(n, r, z);
        double rnorm = sqrt(orc_dot(n, r, r));
        if (!isfinite(rnorm)) { status = ORC_NONFINITE; break; }
        while (rnorm > tol_abs) {
            if (iters >= kmax) { status = ORC_MAXIT; break; }
            orc_spmv(n, rp, ci, va, p, q);
            double gamma = orc_dot(n, q, p);
            if (P_out && iters < p_cap) {
                memcpy(P_out + (size_t)iters * n, p, nb);
                if (gamma_out) gamma_out[iters] = gamma;
            }
            if (!isfinite(gamma)) { status = ORC_NONFINITE; break; }
            if (!(gamma > 0.0)) { status = ORC_BREAKDOWN; break; }
            double a = rz / gamma;
            for (int i = 0; i < n; ++i) x[i] += a * p[i];
            for (int i = 0; i < n; ++i) r[i] -= a * q[i];
            for (int i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
            double rz_new = orc_dot(n, r, z);
            double beta = rz_new / rz;
            rnorm = sqrt(orc_dot(n, r, r));
            ++iters;
            if (!isfinite(rnorm)) { status = ORC_NONFINITE; break; }
            if (rnorm <= tol_abs) break;   /* the augmentation solve is only needed for a next step */
            orc_spmv(n, rp, ci, va, z, u);
            for (int l = 0; l < y; ++l) chat[l] = orc_dot(n, Y + (size_t)l * n, u);
            {
                double cn = 0.0;
                for (int l = 0; l < y; ++l) cn += chat[l] * chat[l];
                inner += orc_inner_solve(n, rp, ci, va, y, Y, wu, R, psi, qpsi, g, &m, m_cap, chat,
                                         tol_in * sqrt(cn), mu);
            }
            for (int i = 0; i < n; ++i) {
                double t = 0.0;
                for (int l = 0; l < y; ++l) t += Y[(size_t)l * n + i] * mu[l];
                p[i] = z[i] + beta * p[i] - t;
            }
            rz = rz_new;
        }
        if (status != ORC_OK) break;
        orc_spmv(n, rp, ci, va, x, q);                              /* true residual */
        for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
        if (sqrt(orc_dot(n, r, r)) <= tol_abs) break;
        if (refinements >= max_refine) { status = ORC_MAXIT; break; }
        ++refinements;                                              /* residual replacement */
    }
done:
    info->status = status;
    info->iters = iters;
    info->refinements = refinements;
    info->w = y;
    {
        orc_spmv(n, rp, ci, va, x, q);
        double rr = 0.0;
        for (int i = 0; i < n; ++i) rr += (b[i] - q[i]) * (b[i] - q[i]);
        info->final_relres = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
    }
    *k2_out = k2;
    *inner_out = inner;
    free(dinv); free(u); free(q); free(p); free(z); free(r); free(mu); free(chat); free(xh);
    free(alpha2); free(g); free(qpsi); free(psi); free(what); free(R);
    return status;
}

/* Gradient of L(theta) = sum_j c^T x_j through A_j(theta) x_j = b_j (the differentiated
 * sequence): with adjoints lambda_j = A_j^{-1} c (A_j symmetric),
 *   dL/dtheta_c = - sum_j lambda_j^T (dA_j/dtheta_c) x_j.
 * A_j(theta) is the cell-centred diffusion operator on an mx x my x mz grid (x fastest;
 * mz == 1 is the 2D five-point operator with no z faces) with k = exp(theta), interior
 * face conductance k_f = 2 k_a k_b / (k_a + k_b) and Dirichlet boundary faces of
 * conductance 2 k_a, plus a theta-independent diagonal shift. A face between cells a and b
 * adds k_f (v_a - v_b)(u_a - u_b) to v^T A u, a boundary face of cell a adds 2 k_a v_a u_a,
 * so, differentiating each face term by the chain rule (dk/dtheta = k):
 *   interior face:  d k_f / d theta_a = k_f k_b / (k_a + k_b)
 *   boundary face:  d (2 k_a) / d theta_a = 2 k_a.
 * lam and xs hold nsys vectors of length n back to back; grad (length n) is overwritten.
 * Written face by face from that definition, one system at a time. */
void orc_theta_grad(int mx, int my, int mz, const double* theta, int nsys, const double* lam, const double* xs,
                    double* grad)
{
    const int n = mx * my * mz;
    const int dims = mz > 1 ? 3 : 2;
    for (int c = 0; c < n; ++c) grad[c] = 0.0;
    for (int j = 0; j < nsys; ++j) {
        const double* l = lam + (size_t)j * n;
        const double* x = xs + (size_t)j * n;
        for (int iz = 0; iz < mz; ++iz)
            for (int iy = 0; iy < my; ++iy)
                for (int ix = 0; ix < mx; ++ix) {
                    const int a = ix + mx * (iy + my * iz);
                    const double ka = exp(theta[a]);
                    /* the six (or four) faces of cell a: -x, +x, -y, +y, -z, +z */
                    for (int f = 0; f < 2 * dims; ++f) {
                        int jx = ix, jy = iy, jz = iz;
                        if (f == 0) jx = ix - 1;
                        if (f == 1) jx = ix + 1;
                        if (f == 2) jy = iy - 1;
                        if (f == 3) jy = iy + 1;
                        if (f == 4) jz = iz - 1;
                        if (f == 5) jz = iz + 1;
                        const int inside = jx >= 0 && jx < mx && jy >= 0 && jy < my && jz >= 0 && jz < mz;
                        if (inside) {
                            const int b = jx + mx * (jy + my * jz);
                            const double kb = exp(theta[b]);
                            const double kf = 2.0 * ka * kb / (ka + kb);
                            const double dkf = kf * (MUT(11) ? ka : kb) / (ka + kb);
                            grad[a] -= dkf * (l[a] - l[b]) * (x[a] - x[b]);
                        } else {
                            grad[a] -= 2.0 * ka * l[a] * x[a];
                        }
                    }
                }
    }
}
