/*
 * kura_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the
 * Kuramoto model on graphs (Boehle, Kuehn, Thalhammer, arXiv 2102.07167).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or helper
 * with the CUDA library.
 *
 * Every function follows a passage of the paper, cited beside it:
 *   - eq:Kuramoto            (Sec. 2)  classical all-to-all model
 *   - eq:KuramotoReformulation / eq:EulerCost (Sec. 2) precomputed S_M, C_M
 *   - eq:OrderParameter      (Sec. 2)  r e^{i psi} = mean of e^{i theta}
 *   - eq:Potential           (Sec. 2)  classical potential
 *   - eq:Means / eq:5c       (Sec. 2)  mean deviation / conserved quantity
 *   - eq:KuramotoGraph       (Sec. 3)  model on a graph, uniform or degree scaling
 *   - eq:KuramotoGraphApproach (Sec. 3) block rule: sparse sum over non-zeros,
 *                            dense: precomputed block sums minus the zeros
 *   - eq:ExtendedPotentialConservation (Sec. 3) graph potential
 * The time integrator is the classical fixed-step fourth-order Runge-Kutta
 * method (the paper's Euler example, Sec. 2, generalised as the paper says is
 * straightforward; the tableau is the textbook one).
 *
 * Conventions (readings of the paper, stated once here):
 *   - Graphs arrive as CSR: row_ptr[n+1] (int64), col[nnz] (int32); row m
 *     lists the l with A_{m l} = 1.  Diagonal entries are ignored: they add
 *     sin(0) = 0 to the sum (Sec. 2, remark on coinciding indices) and are
 *     not counted in the degree used by the non-uniform scaling.
 *   - scaling 0: uniform, calM_m = n.  scaling 1: calM_m = sum_l A_{m l};
 *     a zero row gives theta'_m = omega_m (eq:KuramotoGraph, zero-row case).
 *   - Sums use Neumaier's compensated summation so that the oracle's own
 *     rounding error stays far below every tolerance it is used for.
 *
 * Return codes: 0 ok, -1 bad argument, -2 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Trig-evaluation counter (sin and cos calls), for the cost counts of
 * Table 1 and eq:EulerCost. */
static int64_t g_trig_count = 0;
int64_t orc_trig_count(void) { return g_trig_count; }
void orc_trig_count_reset(void) { g_trig_count = 0; }
static double counted_sin(double x) { g_trig_count++; return sin(x); }
static double counted_cos(double x) { g_trig_count++; return cos(x); }

/* Neumaier compensated accumulator. */
typedef struct { double s, c; } acc_t;
static void acc_add(acc_t* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}
static double acc_val(const acc_t* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* eq:KuramotoGraph by brute force over a dense 0/1 matrix A (row-major,
 * A[m*n + l] = A_{m l}).  Intended for n <= a few hundred. */
int orc_rhs_dense(int64_t n, const uint8_t* A, const double* omega,
                  const double* theta, double K, int scaling, double* out)
{
    if (n <= 0 || !A || !omega || !theta || !out) return -1;
    for (int64_t m = 0; m < n; m++) {
        acc_t sum = {0, 0};
        int64_t deg = 0;
        for (int64_t l = 0; l < n; l++) {
            if (l == m || !A[m * n + l]) continue;
            acc_add(&sum, counted_sin(theta[l] - theta[m]));
            deg++;
        }
        double calM = scaling ? (double)deg : (double)n;
        out[m] = omega[m];
        if (deg > 0) out[m] += (K / calM) * acc_val(&sum);
    }
    return 0;
}

/* eq:KuramotoGraph over CSR edges, for the rows listed in `rows` (all rows
 * when rows == NULL; then nrows must be n).  out[k] is the value of row
 * rows[k]. */
int orc_rhs_csr_rows(int64_t n, const int64_t* row_ptr, const int32_t* col,
                     const double* omega, const double* theta, double K,
                     int scaling, const int64_t* rows, int64_t nrows,
                     double* out)
{
    if (n <= 0 || !row_ptr || !omega || !theta || !out) return -1;
    if (!rows && nrows != n) return -1;
    for (int64_t k = 0; k < nrows; k++) {
        int64_t m = rows ? rows[k] : k;
        if (m < 0 || m >= n) return -1;
        acc_t sum = {0, 0};
        int64_t deg = 0;
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) {
            int64_t l = col[e];
            if (l < 0 || l >= n) return -1;
            if (l == m) continue;
            acc_add(&sum, counted_sin(theta[l] - theta[m]));
            deg++;
        }
        double calM = scaling ? (double)deg : (double)n;
        out[k] = omega[m];
        if (deg > 0) out[k] += (K / calM) * acc_val(&sum);
    }
    return 0;
}

int orc_rhs_csr(int64_t n, const int64_t* row_ptr, const int32_t* col,
                const double* omega, const double* theta, double K,
                int scaling, double* out)
{
    return orc_rhs_csr_rows(n, row_ptr, col, omega, theta, K, scaling,
                            NULL, n, out);
}

/* Classical model through the order-parameter sums, eq:KuramotoReformulation
 * and eq:EulerCost: S_M = mean sin, C_M = mean cos are computed first (2n
 * evaluations), then F = omega + K (S_M cos theta - C_M sin theta) (another
 * 2n evaluations): 4n in total, as counted in Table 1. */
int orc_rhs_complete_op(int64_t n, const double* omega, const double* theta,
                        double K, double* out)
{
    if (n <= 0 || !omega || !theta || !out) return -1;
    acc_t S = {0, 0}, C = {0, 0};
    for (int64_t m = 0; m < n; m++) {
        acc_add(&S, counted_sin(theta[m]));
        acc_add(&C, counted_cos(theta[m]));
    }
    double SM = acc_val(&S) / (double)n, CM = acc_val(&C) / (double)n;
    for (int64_t m = 0; m < n; m++)
        out[m] = omega[m] + K * (SM * counted_cos(theta[m]) - CM * counted_sin(theta[m]));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Finite-valued adjacency (Sec. 1, "Generalisations": A_{ml} in {0, ..., J}),
 * uniform scaling: f_m = omega_m + (K/n) sum_l A_{ml} sin(theta_l - theta_m).
 * CSR form: val[e] is the value of edge e (values 0 are simply absent);
 * dense form: brute force over an n x n int32 matrix.  Diagonal skipped. */
int orc_rhs_valued_csr(int64_t n, const int64_t* row_ptr, const int32_t* col,
                       const int32_t* val, const double* omega,
                       const double* theta, double K, double* out)
{
    if (n <= 0 || !row_ptr || !val || !omega || !theta || !out) return -1;
    for (int64_t m = 0; m < n; m++) {
        acc_t sum = {0, 0};
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) {
            if (col[e] < 0 || col[e] >= n) return -1;
            if (col[e] == m) continue;
            acc_add(&sum, (double)val[e] * counted_sin(theta[col[e]] - theta[m]));
        }
        out[m] = omega[m] + (K / (double)n) * acc_val(&sum);
    }
    return 0;
}

int orc_rhs_valued_dense(int64_t n, const int32_t* A, const double* omega,
                         const double* theta, double K, double* out)
{
    if (n <= 0 || !A || !omega || !theta || !out) return -1;
    for (int64_t m = 0; m < n; m++) {
        acc_t sum = {0, 0};
        for (int64_t l = 0; l < n; l++) {
            if (l == m || !A[m * n + l]) continue;
            acc_add(&sum, (double)A[m * n + l] * sin(theta[l] - theta[m]));
        }
        out[m] = omega[m] + (K / (double)n) * acc_val(&sum);
    }
    return 0;
}

/* Block rule for finite-valued A ("a single value is prevalent in each
 * block"): per block (I, J) over its n_I n_J entries (n_I (n_I - 1) on the
 * diagonal block, whose diagonal is don't-care) the value v* of largest
 * count among the nonzero values (ties: the smaller value); the block is
 * dense with value v* when the fraction of its entries different from v* is
 * below tau, else sparse (value 0).  Row m of community I then sums, per
 * column block J, v_IJ (S_J, C_J) plus (A_{ml} - v_IJ)(sin, cos) theta_l over
 * the l in J with A_{ml} != v_IJ (l != m), and
 * f_m = omega_m + (K/n)(cos theta_m acc_s - sin theta_m acc_c).  For 0/1
 * values this is eq:KuramotoGraphApproach (v* = 1: missing entries
 * subtracted).  max_val bounds the values (1..max_val). */
int orc_rhs_block_valued(int64_t n, const int64_t* row_ptr, const int32_t* col,
                         const int32_t* val, int32_t max_val, const int32_t* label,
                         int32_t n_comm, const double* omega, const double* theta,
                         double K, double tau, double* out, int32_t* block_val)
{
    if (n <= 0 || n_comm <= 0 || max_val < 1 || !row_ptr || !col || !val ||
        !label || !omega || !theta || !out) return -1;
    int64_t nc = n_comm, nv = (int64_t)max_val + 1;
    int64_t* size = calloc((size_t)nc, sizeof(int64_t));
    int64_t* cnt = calloc((size_t)(nc * nc * nv), sizeof(int64_t));
    int32_t* bval = calloc((size_t)(nc * nc), sizeof(int32_t));
    double* S = calloc((size_t)nc, sizeof(double));
    double* C = calloc((size_t)nc, sizeof(double));
    double* sn = malloc((size_t)n * sizeof(double));
    double* cs = malloc((size_t)n * sizeof(double));
    int32_t* arow = calloc((size_t)n, sizeof(int32_t));
    int rc = 0;
    if (!size || !cnt || !bval || !S || !C || !sn || !cs || !arow) { rc = -2; goto done; }
    for (int64_t m = 0; m < n; m++) {
        if (label[m] < 0 || label[m] >= n_comm) { rc = -1; goto done; }
        size[label[m]]++;
    }
    /* value counts per block (nonzero values), diagonal entries ignored */
    for (int64_t m = 0; m < n; m++)
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) {
            if (col[e] < 0 || col[e] >= n || val[e] < 1 || val[e] > max_val) { rc = -1; goto done; }
            if (col[e] == m) continue;
            cnt[((int64_t)label[m] * nc + label[col[e]]) * nv + val[e]]++;
        }
    for (int64_t I = 0; I < nc; I++)
        for (int64_t J = 0; J < nc; J++) {
            double entries = (I == J) ? (double)size[I] * (double)(size[I] - 1)
                                      : (double)size[I] * (double)size[J];
            if (entries <= 0) continue;
            int32_t best = 0;
            int64_t bestc = 0;
            for (int32_t v = 1; v <= max_val; v++)
                if (cnt[(I * nc + J) * nv + v] > bestc) { bestc = cnt[(I * nc + J) * nv + v]; best = v; }
            if (best > 0 && (1.0 - (double)bestc / entries) < tau) bval[I * nc + J] = best;
        }
    if (block_val) for (int64_t q = 0; q < nc * nc; q++) block_val[q] = bval[q];
    for (int64_t l = 0; l < n; l++) { sn[l] = sin(theta[l]); cs[l] = cos(theta[l]); }
    {
        acc_t* sj = calloc((size_t)nc, sizeof(acc_t));
        acc_t* cj = calloc((size_t)nc, sizeof(acc_t));
        if (!sj || !cj) { free(sj); free(cj); rc = -2; goto done; }
        for (int64_t l = 0; l < n; l++) { acc_add(&sj[label[l]], sn[l]); acc_add(&cj[label[l]], cs[l]); }
        for (int64_t J = 0; J < nc; J++) { S[J] = acc_val(&sj[J]); C[J] = acc_val(&cj[J]); }
        free(sj); free(cj);
    }
    for (int64_t m = 0; m < n; m++) {
        int64_t I = label[m];
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++)
            if (col[e] != m) arow[col[e]] = val[e];
        acc_t as = {0, 0}, ac = {0, 0};
        for (int64_t J = 0; J < nc; J++) {
            int32_t v = bval[I * nc + J];
            if (v) { acc_add(&as, (double)v * S[J]); acc_add(&ac, (double)v * C[J]); }
        }
        /* exceptions: every column l != m whose value differs from its block's value */
        for (int64_t l = 0; l < n; l++) {
            if (l == m) continue;
            int32_t w = arow[l] - bval[I * nc + label[l]];
            if (w) { acc_add(&as, (double)w * sn[l]); acc_add(&ac, (double)w * cs[l]); }
        }
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) arow[col[e]] = 0;
        out[m] = omega[m] + (K / (double)n) * (cs[m] * acc_val(&as) - sn[m] * acc_val(&ac));
    }
done:
    free(size); free(cnt); free(bval); free(S); free(C); free(sn); free(cs); free(arow);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Block rule, eq:KuramotoGraphApproach.  The submatrices are the blocks
 * (I, J) = {rows with label I} x {columns with label J}; relabelling the
 * nodes community by community (P A P^T) only reorders rows and columns and
 * does not change any sum, so blocks are addressed through the labels
 * directly.  A block is evaluated by the "dense" rule (precomputed
 * S_J = sum_{l in J} sin theta_l and C_J, minus the sums over the zeros of
 * the block row) when its zero fraction is below tau, and by the "sparse"
 * rule (sum of sin(theta_l - theta_m) over the non-zeros) otherwise.  The
 * zero set of a diagonal block contains l = m itself, literally as in the
 * paper's formula (A_{m m} = 0).
 *
 * stats (nullable, 6 entries): [0] dense blocks with at least one row and
 * column, [1] sparse blocks, [2] zeros summed over by the dense rule,
 * [3] non-zeros summed over by the sparse rule, [4] blocks considered,
 * [5] sin/cos evaluations of this call.
 */
int orc_rhs_block(int64_t n, const int64_t* row_ptr, const int32_t* col,
                  const int32_t* label, int32_t n_comm, const double* omega,
                  const double* theta, double K, int scaling, double tau,
                  double* out, int64_t* stats)
{
    if (n <= 0 || n_comm <= 0 || !row_ptr || !col || !label || !omega ||
        !theta || !out) return -1;
    for (int64_t m = 0; m < n; m++)
        if (label[m] < 0 || label[m] >= n_comm) return -1;
    int64_t trig0 = g_trig_count;
    int64_t nc = n_comm;
    int64_t* size = calloc((size_t)nc, sizeof(int64_t));
    int64_t* nnzb = calloc((size_t)(nc * nc), sizeof(int64_t));
    uint8_t* dense = calloc((size_t)(nc * nc), 1);
    int64_t* member_ptr = calloc((size_t)nc + 1, sizeof(int64_t));
    int64_t* members = malloc((size_t)n * sizeof(int64_t));
    double* S = calloc((size_t)nc, sizeof(double));
    double* C = calloc((size_t)nc, sizeof(double));
    double* sn = malloc((size_t)n * sizeof(double));
    double* cs = malloc((size_t)n * sizeof(double));
    uint8_t* mark = calloc((size_t)n, 1);
    int rc = 0;
    if (!size || !nnzb || !dense || !member_ptr || !members || !S || !C ||
        !sn || !cs || !mark) { rc = -2; goto done; }

    /* community sizes and member lists */
    for (int64_t m = 0; m < n; m++) size[label[m]]++;
    for (int64_t I = 0; I < nc; I++) member_ptr[I + 1] = member_ptr[I] + size[I];
    {
        int64_t* fill = calloc((size_t)nc, sizeof(int64_t));
        if (!fill) { rc = -2; goto done; }
        for (int64_t m = 0; m < n; m++) {
            int64_t I = label[m];
            members[member_ptr[I] + fill[I]++] = m;
        }
        free(fill);
    }
    /* non-zeros per block, diagonal entries ignored */
    for (int64_t m = 0; m < n; m++)
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) {
            if (col[e] < 0 || col[e] >= n) { rc = -1; goto done; }
            if (col[e] == m) continue;
            nnzb[(int64_t)label[m] * nc + label[col[e]]]++;
        }
    /* classification: zero fraction of the block below tau => dense */
    int64_t n_dense = 0, n_sparse = 0, n_zero_terms = 0, n_nz_terms = 0;
    for (int64_t I = 0; I < nc; I++)
        for (int64_t J = 0; J < nc; J++) {
            double entries = (double)size[I] * (double)size[J];
            if (entries == 0) continue;
            double zeros = entries - (double)nnzb[I * nc + J];
            int d = (zeros / entries) < tau;
            dense[I * nc + J] = (uint8_t)d;
            if (d) n_dense++; else n_sparse++;
        }
    /* sin, cos of every phase (2n evaluations) and the block sums S_J, C_J */
    for (int64_t l = 0; l < n; l++) { sn[l] = counted_sin(theta[l]); cs[l] = counted_cos(theta[l]); }
    for (int64_t J = 0; J < nc; J++) {
        acc_t sj = {0, 0}, cj = {0, 0};
        for (int64_t k = member_ptr[J]; k < member_ptr[J + 1]; k++) {
            acc_add(&sj, sn[members[k]]);
            acc_add(&cj, cs[members[k]]);
        }
        S[J] = acc_val(&sj);
        C[J] = acc_val(&cj);
    }
    /* rows */
    for (int64_t m = 0; m < n; m++) {
        int64_t I = label[m];
        int64_t deg = 0;
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++)
            if (col[e] != m) { mark[col[e]] = 1; deg++; }
        acc_t total = {0, 0};
        for (int64_t J = 0; J < nc; J++) {
            if (size[J] == 0) continue;
            if (dense[I * nc + J]) {
                /* (S_J - sum_{zeros} sin) cos theta_m - (C_J - sum_{zeros} cos) sin theta_m */
                acc_t zs = {0, 0}, zc = {0, 0};
                for (int64_t k = member_ptr[J]; k < member_ptr[J + 1]; k++) {
                    int64_t l = members[k];
                    if (mark[l]) continue;          /* A_{m l} = 1: not a zero */
                    acc_add(&zs, sn[l]);
                    acc_add(&zc, cs[l]);
                    n_zero_terms++;
                }
                acc_add(&total, (S[J] - acc_val(&zs)) * cs[m]);
                acc_add(&total, -(C[J] - acc_val(&zc)) * sn[m]);
            } else {
                /* straightforward sum over the non-zeros of the block row */
                for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) {
                    int64_t l = col[e];
                    if (l == m || label[l] != J) continue;
                    acc_add(&total, counted_sin(theta[l] - theta[m]));
                    n_nz_terms++;
                }
            }
        }
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) mark[col[e]] = 0;
        double calM = scaling ? (double)deg : (double)n;
        out[m] = omega[m];
        if (deg > 0) out[m] += (K / calM) * acc_val(&total);
    }
    if (stats) {
        stats[0] = n_dense; stats[1] = n_sparse; stats[2] = n_zero_terms;
        stats[3] = n_nz_terms; stats[4] = n_dense + n_sparse;
        stats[5] = g_trig_count - trig0;
    }
done:
    free(size); free(nnzb); free(dense); free(member_ptr); free(members);
    free(S); free(C); free(sn); free(cs); free(mark);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Classical fixed-step RK4 on the graph model, right-hand side by the CSR
 * definition (orc_rhs_csr).  theta is advanced in place, n_steps steps of
 * size h:
 *   k1 = f(y), k2 = f(y + h/2 k1), k3 = f(y + h/2 k2), k4 = f(y + h k3),
 *   y <- y + h/6 (k1 + 2 k2 + 2 k3 + k4).
 * The phases are kept unwrapped (the conserved quantity, eq:5c, is stated
 * for unwrapped phases). */
int orc_rk4_csr(int64_t n, const int64_t* row_ptr, const int32_t* col,
                const double* omega, double K, int scaling, double* theta,
                double h, int64_t n_steps)
{
    if (n <= 0 || !theta || n_steps < 0) return -1;
    double* k1 = malloc((size_t)n * sizeof(double));
    double* k2 = malloc((size_t)n * sizeof(double));
    double* k3 = malloc((size_t)n * sizeof(double));
    double* k4 = malloc((size_t)n * sizeof(double));
    double* Y = malloc((size_t)n * sizeof(double));
    int rc = 0;
    if (!k1 || !k2 || !k3 || !k4 || !Y) { rc = -2; goto done; }
    for (int64_t s = 0; s < n_steps; s++) {
        if ((rc = orc_rhs_csr(n, row_ptr, col, omega, theta, K, scaling, k1))) goto done;
        for (int64_t i = 0; i < n; i++) Y[i] = theta[i] + 0.5 * h * k1[i];
        if ((rc = orc_rhs_csr(n, row_ptr, col, omega, Y, K, scaling, k2))) goto done;
        for (int64_t i = 0; i < n; i++) Y[i] = theta[i] + 0.5 * h * k2[i];
        if ((rc = orc_rhs_csr(n, row_ptr, col, omega, Y, K, scaling, k3))) goto done;
        for (int64_t i = 0; i < n; i++) Y[i] = theta[i] + h * k3[i];
        if ((rc = orc_rhs_csr(n, row_ptr, col, omega, Y, K, scaling, k4))) goto done;
        for (int64_t i = 0; i < n; i++)
            theta[i] += (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
done:
    free(k1); free(k2); free(k3); free(k4); free(Y);
    return rc;
}

/* Second-order integrators for the long-horizon comparison the paper makes
 * in its numerical section (an explicit second-order Runge-Kutta method
 * against a second-order implicit, geometric one; conserved quantity of
 * eq:5c), with the CSR definition as right-hand side:
 *   method 0, explicit midpoint:  Y = y + h/2 f(y),  y' = y + h f(Y);
 *   method 1, implicit midpoint:  y' = 2 Z - y with Z = y + h/2 f(Z), the
 *     stage Z found by `iters` fixed-point sweeps Z <- y + h/2 f(Z) from the
 *     predictor Z = y + h/2 f(y) (iters >= 1). */
int orc_rk2_csr(int64_t n, const int64_t* row_ptr, const int32_t* col,
                const double* omega, double K, int scaling, double* theta,
                double h, int64_t n_steps, int method, int iters)
{
    if (n <= 0 || !theta || n_steps < 0 || (method != 0 && method != 1) || iters < 1) return -1;
    double* f = malloc((size_t)n * sizeof(double));
    double* Z = malloc((size_t)n * sizeof(double));
    int rc = 0;
    if (!f || !Z) { rc = -2; goto done; }
    for (int64_t s = 0; s < n_steps; s++) {
        if ((rc = orc_rhs_csr(n, row_ptr, col, omega, theta, K, scaling, f))) goto done;
        for (int64_t i = 0; i < n; i++) Z[i] = theta[i] + 0.5 * h * f[i];
        if (method == 0) {
            if ((rc = orc_rhs_csr(n, row_ptr, col, omega, Z, K, scaling, f))) goto done;
            for (int64_t i = 0; i < n; i++) theta[i] += h * f[i];
        } else {
            for (int it = 0; it < iters; it++) {
                if ((rc = orc_rhs_csr(n, row_ptr, col, omega, Z, K, scaling, f))) goto done;
                for (int64_t i = 0; i < n; i++) Z[i] = theta[i] + 0.5 * h * f[i];
            }
            for (int64_t i = 0; i < n; i++) theta[i] = 2.0 * Z[i] - theta[i];
        }
    }
done:
    free(f); free(Z);
    return rc;
}

/* Classical all-to-all model (eq:Kuramoto) integrated with the same RK4,
 * right-hand side by the order-parameter sums (eq:KuramotoReformulation). */
int orc_rk4_complete(int64_t n, const double* omega, double K, double* theta,
                     double h, int64_t n_steps)
{
    if (n <= 0 || !theta || n_steps < 0) return -1;
    double* k1 = malloc((size_t)n * sizeof(double));
    double* k2 = malloc((size_t)n * sizeof(double));
    double* k3 = malloc((size_t)n * sizeof(double));
    double* k4 = malloc((size_t)n * sizeof(double));
    double* Y = malloc((size_t)n * sizeof(double));
    int rc = 0;
    if (!k1 || !k2 || !k3 || !k4 || !Y) { rc = -2; goto done; }
    for (int64_t s = 0; s < n_steps; s++) {
        orc_rhs_complete_op(n, omega, theta, K, k1);
        for (int64_t i = 0; i < n; i++) Y[i] = theta[i] + 0.5 * h * k1[i];
        orc_rhs_complete_op(n, omega, Y, K, k2);
        for (int64_t i = 0; i < n; i++) Y[i] = theta[i] + 0.5 * h * k2[i];
        orc_rhs_complete_op(n, omega, Y, K, k3);
        for (int64_t i = 0; i < n; i++) Y[i] = theta[i] + h * k3[i];
        orc_rhs_complete_op(n, omega, Y, K, k4);
        for (int64_t i = 0; i < n; i++)
            theta[i] += (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
done:
    free(k1); free(k2); free(k3); free(k4); free(Y);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* eq:OrderParameter: r e^{i psi} = (1/n) sum_m e^{i theta_m} = C + i S;
 * r = sqrt(C^2 + S^2), psi = atan2(S, C) (psi = 0 when r = 0).  When label is
 * given, the same quantity restricted to each community ("localised order
 * parameters") is written to r_comm[n_comm], psi_comm[n_comm] (nullable). */
int orc_order_params(int64_t n, const double* theta, double* r, double* psi,
                     const int32_t* label, int32_t n_comm, double* r_comm,
                     double* psi_comm)
{
    if (n <= 0 || !theta || !r || !psi) return -1;
    acc_t S = {0, 0}, C = {0, 0};
    for (int64_t m = 0; m < n; m++) {
        acc_add(&S, sin(theta[m]));
        acc_add(&C, cos(theta[m]));
    }
    double s = acc_val(&S) / (double)n, c = acc_val(&C) / (double)n;
    *r = sqrt(c * c + s * s);
    *psi = (*r == 0.0) ? 0.0 : atan2(s, c);
    if (label && n_comm > 0 && r_comm) {
        for (int32_t I = 0; I < n_comm; I++) {
            acc_t SI = {0, 0}, CI = {0, 0};
            int64_t cnt = 0;
            for (int64_t m = 0; m < n; m++) {
                if (label[m] != I) continue;
                acc_add(&SI, sin(theta[m]));
                acc_add(&CI, cos(theta[m]));
                cnt++;
            }
            double si = cnt ? acc_val(&SI) / (double)cnt : 0.0;
            double ci = cnt ? acc_val(&CI) / (double)cnt : 0.0;
            r_comm[I] = sqrt(ci * ci + si * si);
            if (psi_comm) psi_comm[I] = (r_comm[I] == 0.0) ? 0.0 : atan2(si, ci);
        }
    }
    return 0;
}

/* Potential on a graph, eq:ExtendedPotentialConservation (with the classical
 * eq:Potential as the complete-graph case):
 *   V = -omega^T theta + (K/2) sum_{m,l} calA_{m l} (1 - cos(theta_l - theta_m)),
 * calA_{m l} = A_{m l} / calM_m. */
int orc_potential_csr(int64_t n, const int64_t* row_ptr, const int32_t* col,
                      const double* omega, const double* theta, double K,
                      int scaling, double* V)
{
    if (n <= 0 || !row_ptr || !col || !omega || !theta || !V) return -1;
    acc_t lin = {0, 0}, quad = {0, 0};
    for (int64_t m = 0; m < n; m++) acc_add(&lin, -omega[m] * theta[m]);
    for (int64_t m = 0; m < n; m++) {
        int64_t deg = 0;
        acc_t row = {0, 0};
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) {
            int64_t l = col[e];
            if (l == m) continue;
            acc_add(&row, 1.0 - cos(theta[l] - theta[m]));
            deg++;
        }
        if (deg == 0) continue;
        double calM = scaling ? (double)deg : (double)n;
        acc_add(&quad, acc_val(&row) / calM);
    }
    *V = acc_val(&lin) + 0.5 * K * acc_val(&quad);
    return 0;
}

/* eq:Means: (1/n) sum_m (theta_m(t) - theta_m(0) - t omega_m). */
int orc_mean_deviation(int64_t n, const double* theta_t, const double* theta_0,
                       const double* omega, double t, double* out)
{
    if (n <= 0 || !theta_t || !theta_0 || !omega || !out) return -1;
    acc_t a = {0, 0};
    for (int64_t m = 0; m < n; m++) acc_add(&a, theta_t[m] - theta_0[m] - t * omega[m]);
    *out = acc_val(&a) / (double)n;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of the classical RK4 integrator orc_rk4_csr for a
 * terminal loss L(theta(T)):
 *   loss_kind 0: L = 1 - r(theta(T)), r of eq:OrderParameter;
 *   loss_kind 1: L = 1/2 sum_m (theta_m(T) - target_m)^2.
 * Returns L and the gradients with respect to omega (g_omega[n]), K (*g_K)
 * and theta(0) (g_theta0[n]).  The adjoint of one step y' = y + h/6 (k1 + 2 k2
 * + 2 k3 + k4) with stages k_s = f(Y_s), given lambda = dL/dy':
 *   w4 = h/6 lambda,              a4 = J(Y4)^T w4
 *   w3 = h/3 lambda + h a4,       a3 = J(Y3)^T w3
 *   w2 = h/3 lambda + h/2 a3,     a2 = J(Y2)^T w2
 *   w1 = h/6 lambda + h/2 a2,     a1 = J(Y1)^T w1
 *   dL/dy = lambda + a1 + a2 + a3 + a4,
 *   dL/domega += w1 + w2 + w3 + w4,   dL/dK += sum_s w_s . u(Y_s),
 * with f = omega + K u and J the Jacobian of f (eq:KuramotoGraph):
 *   df_m/dtheta_l = (K/calM_m) A_{ml} cos(theta_l - theta_m)  (l != m),
 *   df_m/dtheta_m = -sum_l of the above.
 * J^T is applied edge by edge from that definition (any A, symmetric or
 * not).  All states are kept, so memory is (n_steps + 1) n doubles. */
static void unit_coupling(int64_t n, const int64_t* row_ptr, const int32_t* col, int scaling,
                          const double* th, double* u)
{
    for (int64_t m = 0; m < n; m++) {
        acc_t sum = {0, 0};
        int64_t deg = 0;
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) {
            int64_t l = col[e];
            if (l == m) continue;
            acc_add(&sum, sin(th[l] - th[m]));
            deg++;
        }
        double calM = scaling ? (double)deg : (double)n;
        u[m] = deg > 0 ? acc_val(&sum) / calM : 0.0;
    }
}

static void jacobian_t(int64_t n, const int64_t* row_ptr, const int32_t* col, double K, int scaling,
                       const double* th, const double* mu, double* out)
{
    for (int64_t m = 0; m < n; m++) out[m] = 0.0;
    for (int64_t m = 0; m < n; m++) {
        int64_t deg = 0;
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) if (col[e] != m) deg++;
        if (deg == 0) continue;
        double scale = K / (scaling ? (double)deg : (double)n);
        for (int64_t e = row_ptr[m]; e < row_ptr[m + 1]; e++) {
            int64_t l = col[e];
            if (l == m) continue;
            double v = scale * mu[m] * cos(th[l] - th[m]);
            out[l] += v;
            out[m] -= v;
        }
    }
}

int orc_adjoint_rk4_csr(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* omega,
                        double K, int scaling, const double* theta0, double h, int64_t n_steps,
                        int loss_kind, const double* target, double* loss, double* g_omega,
                        double* g_K, double* g_theta0)
{
    if (n <= 0 || !theta0 || n_steps < 0 || !loss || !g_omega || !g_K || !g_theta0) return -1;
    if (loss_kind == 1 && !target) return -1;
    double* ys = malloc(sizeof(double) * (size_t)n * (size_t)(n_steps + 1));
    double *Y[5], *k[5], *w = malloc(sizeof(double) * (size_t)n), *a[5], *lam = malloc(sizeof(double) * (size_t)n);
    double* u = malloc(sizeof(double) * (size_t)n);
    int rc = 0;
    for (int s = 0; s < 5; s++) {
        Y[s] = malloc(sizeof(double) * (size_t)n);
        k[s] = malloc(sizeof(double) * (size_t)n);
        a[s] = malloc(sizeof(double) * (size_t)n);
    }
    if (!ys || !w || !lam || !u) { rc = -2; goto done; }
    for (int s = 0; s < 5; s++) if (!Y[s] || !k[s] || !a[s]) { rc = -2; goto done; }
    /* forward, keeping every state */
    memcpy(ys, theta0, sizeof(double) * (size_t)n);
    for (int64_t t = 0; t < n_steps; t++) {
        memcpy(ys + (t + 1) * n, ys + t * n, sizeof(double) * (size_t)n);
        if ((rc = orc_rk4_csr(n, row_ptr, col, omega, K, scaling, ys + (t + 1) * n, h, 1))) goto done;
    }
    /* terminal loss and lambda = dL/dtheta(T) */
    const double* yT = ys + n_steps * n;
    if (loss_kind == 0) {
        double r, psi;
        orc_order_params(n, yT, &r, &psi, NULL, 0, NULL, NULL);
        *loss = 1.0 - r;
        for (int64_t m = 0; m < n; m++) lam[m] = -sin(psi - yT[m]) / (double)n;
    } else {
        acc_t L = {0, 0};
        for (int64_t m = 0; m < n; m++) {
            double d = yT[m] - target[m];
            acc_add(&L, 0.5 * d * d);
            lam[m] = d;
        }
        *loss = acc_val(&L);
    }
    for (int64_t m = 0; m < n; m++) g_omega[m] = 0.0;
    *g_K = 0.0;
    /* backward */
    for (int64_t t = n_steps - 1; t >= 0; t--) {
        const double* y = ys + t * n;
        /* stages of step t: Y1 = y, Y2 = y + h/2 k1, Y3 = y + h/2 k2, Y4 = y + h k3 */
        memcpy(Y[1], y, sizeof(double) * (size_t)n);
        orc_rhs_csr(n, row_ptr, col, omega, Y[1], K, scaling, k[1]);
        for (int64_t m = 0; m < n; m++) Y[2][m] = y[m] + 0.5 * h * k[1][m];
        orc_rhs_csr(n, row_ptr, col, omega, Y[2], K, scaling, k[2]);
        for (int64_t m = 0; m < n; m++) Y[3][m] = y[m] + 0.5 * h * k[2][m];
        orc_rhs_csr(n, row_ptr, col, omega, Y[3], K, scaling, k[3]);
        for (int64_t m = 0; m < n; m++) Y[4][m] = y[m] + h * k[3][m];
        const double cl[5] = {0, h / 6.0, h / 3.0, h / 3.0, h / 6.0};      /* weight of lambda */
        const double ca[5] = {0, 0.5 * h, 0.5 * h, h, 0};                 /* weight of a_{s+1} */
        for (int s = 4; s >= 1; s--) {
            for (int64_t m = 0; m < n; m++) w[m] = cl[s] * lam[m] + (s < 4 ? ca[s] * a[s + 1][m] : 0.0);
            jacobian_t(n, row_ptr, col, K, scaling, Y[s], w, a[s]);
            unit_coupling(n, row_ptr, col, scaling, Y[s], u);
            acc_t gk = {0, 0};
            for (int64_t m = 0; m < n; m++) {
                g_omega[m] += w[m];
                acc_add(&gk, w[m] * u[m]);
            }
            *g_K += acc_val(&gk);
        }
        for (int64_t m = 0; m < n; m++) lam[m] += a[1][m] + a[2][m] + a[3][m] + a[4][m];
    }
    memcpy(g_theta0, lam, sizeof(double) * (size_t)n);
done:
    free(ys); free(w); free(lam); free(u);
    for (int s = 0; s < 5; s++) { free(Y[s]); free(k[s]); free(a[s]); }
    return rc;
}
