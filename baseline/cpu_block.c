/*
 * cpu_block.c -- the block (localised-order-parameter) method on the host
 * CPU, parallelised with OpenMP over all cores: the CPU baseline the GPU
 * path is compared with.  It is neither the oracle (which is the plain,
 * single-threaded definition) nor part of the library: bench.py builds and
 * times it.
 *
 * Method (Boehle, Kuehn, Thalhammer, arXiv 2102.07167, Sec. 3,
 * eq:KuramotoGraphApproach): permute the nodes so that communities are
 * contiguous; a block (I, J) is dense iff its zero fraction is below tau
 * (diagonal blocks over n_I (n_I - 1) entries, the diagonal counted as
 * present); per RK4 stage
 *   s_l, c_l = sin, cos of every phase (FP64),
 *   S_J, C_J = block sums,  T_I = sum over dense J of (S_J, C_J),
 *   acc_m = T_I - sum over the zeros of m's dense blocks + sum over m's
 *           non-zeros in sparse blocks of (s_l, c_l),
 *   f_m = omega_m + (K / n)(c_m acc_s - s_m acc_c),
 * followed by the classical RK4 update; phases stay unwrapped.
 *
 * API (all host arrays; the caller keeps ownership):
 *   cpb_create(n, row_ptr, col, label, n_comm, omega, K, tau) -> handle
 *   cpb_rk4(handle, theta[n], h, steps)   in place, user order
 *   cpb_rhs(handle, theta[n], f[n])       user order
 *   cpb_threads()                         OpenMP threads used
 *   cpb_destroy(handle)
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t n;
    int32_t nc;
    double K;
    int32_t* perm;       /* perm[new] = old */
    int32_t* comm;       /* community of each permuted node */
    int64_t* coff;       /* community offsets in the permuted order */
    int64_t* dptr;       /* dense column blocks of each row block */
    int32_t* dcol;
    int64_t* rptr;       /* per permuted row: [missing | present] permuted columns */
    int32_t* rnm;
    int32_t* ent;
    double* omega;       /* permuted */
    double *y, *Y, *k, *f, *s, *c, *S, *C, *T;
} cpb_t;

int cpb_threads(void) { return omp_get_max_threads(); }

void cpb_destroy(cpb_t* h)
{
    if (!h) return;
    free(h->perm); free(h->comm); free(h->coff); free(h->dptr); free(h->dcol); free(h->rptr); free(h->rnm);
    free(h->ent); free(h->omega); free(h->y); free(h->Y); free(h->k); free(h->f); free(h->s); free(h->c);
    free(h->S); free(h->C); free(h->T);
    free(h);
}

cpb_t* cpb_create(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* label, int32_t n_comm,
                  const double* omega, double K, double tau)
{
    cpb_t* h = calloc(1, sizeof(cpb_t));
    if (!h || n < 1 || n_comm < 1) { free(h); return NULL; }
    const int64_t nc = n_comm;
    h->n = n; h->nc = n_comm; h->K = K;
    h->perm = malloc(sizeof(int32_t) * n); h->comm = malloc(sizeof(int32_t) * n);
    h->coff = calloc(nc + 1, sizeof(int64_t)); h->omega = malloc(sizeof(double) * n);
    int32_t* inv = malloc(sizeof(int32_t) * n);
    int64_t* cnt = calloc(nc * nc, sizeof(int64_t));
    int64_t* fill = calloc(nc, sizeof(int64_t));
    for (int64_t v = 0; v < n; v++) h->coff[label[v] + 1]++;
    for (int64_t I = 0; I < nc; I++) h->coff[I + 1] += h->coff[I];
    for (int64_t v = 0; v < n; v++) {                       /* stable sort by label */
        const int64_t p = h->coff[label[v]] + fill[label[v]]++;
        h->perm[p] = (int32_t)v; inv[v] = (int32_t)p; h->comm[p] = label[v]; h->omega[p] = omega[v];
    }
    for (int64_t v = 0; v < n; v++)
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++)
            if (col[e] != v) cnt[(int64_t)label[v] * nc + label[col[e]]]++;
    h->dptr = calloc(nc + 1, sizeof(int64_t));
    uint8_t* dense = calloc(nc * nc, 1);
    for (int64_t I = 0; I < nc; I++)
        for (int64_t J = 0; J < nc; J++) {
            const double nI = (double)(h->coff[I + 1] - h->coff[I]), nJ = (double)(h->coff[J + 1] - h->coff[J]);
            const double entries = I == J ? nI * (nI - 1.0) : nI * nJ;
            if (entries <= 0) continue;
            if (1.0 - (double)cnt[I * nc + J] / entries < tau) { dense[I * nc + J] = 1; h->dptr[I + 1]++; }
        }
    for (int64_t I = 0; I < nc; I++) h->dptr[I + 1] += h->dptr[I];
    h->dcol = malloc(sizeof(int32_t) * (h->dptr[nc] + 1));
    for (int64_t I = 0, q = 0; I < nc; I++)
        for (int64_t J = 0; J < nc; J++) if (dense[I * nc + J]) h->dcol[q++] = (int32_t)J;
    /* per-row lists: missing entries of dense blocks (diagonal excluded), present entries of sparse blocks;
     * counted, then filled, in parallel over rows (a mark array per thread) */
    h->rptr = calloc(n + 1, sizeof(int64_t));
    h->rnm = calloc(n, sizeof(int32_t));
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            for (int64_t p = 0; p < n; p++) h->rptr[p + 1] += h->rptr[p];
            h->ent = malloc(sizeof(int32_t) * (h->rptr[n] + 1));
        }
#pragma omp parallel
        {
            uint8_t* mark = calloc(n, 1);
#pragma omp for schedule(dynamic, 64)
            for (int64_t p = 0; p < n; p++) {
                const int64_t v = h->perm[p], I = h->comm[p];
                for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) mark[inv[col[e]]] = 1;
                int64_t pos = pass == 1 ? h->rptr[p] : 0;
                int32_t nm = 0;
                for (int64_t k = h->dptr[I]; k < h->dptr[I + 1]; k++) {
                    const int64_t J = h->dcol[k];
                    for (int64_t q = h->coff[J]; q < h->coff[J + 1]; q++)
                        if (!mark[q] && q != p) { if (pass == 1) h->ent[pos] = (int32_t)q; pos++; nm++; }
                }
                for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
                    const int64_t q = inv[col[e]];
                    if (q == p || dense[I * nc + h->comm[q]]) continue;
                    if (pass == 1) h->ent[pos] = (int32_t)q;
                    pos++;
                }
                if (pass == 0) h->rptr[p + 1] = pos;
                else h->rnm[p] = nm;
                for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) mark[inv[col[e]]] = 0;
            }
            free(mark);
        }
    }
    free(dense); free(cnt); free(fill); free(inv);
    h->y = malloc(sizeof(double) * n); h->Y = malloc(sizeof(double) * n); h->k = malloc(sizeof(double) * n);
    h->f = malloc(sizeof(double) * n); h->s = malloc(sizeof(double) * n); h->c = malloc(sizeof(double) * n);
    h->S = malloc(sizeof(double) * nc); h->C = malloc(sizeof(double) * nc); h->T = malloc(sizeof(double) * 2 * nc);
    return h;
}

/* f = F(x), permuted order */
static void rhs_perm(cpb_t* h, const double* x, double* f)
{
    const int64_t n = h->n, nc = h->nc;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; p++) { h->s[p] = sin(x[p]); h->c[p] = cos(x[p]); }
#pragma omp parallel for schedule(static)
    for (int64_t J = 0; J < nc; J++) {
        double a = 0.0, b = 0.0;
        for (int64_t q = h->coff[J]; q < h->coff[J + 1]; q++) { a += h->s[q]; b += h->c[q]; }
        h->S[J] = a; h->C[J] = b;
    }
#pragma omp parallel for schedule(static)
    for (int64_t I = 0; I < nc; I++) {
        double a = 0.0, b = 0.0;
        for (int64_t k = h->dptr[I]; k < h->dptr[I + 1]; k++) { a += h->S[h->dcol[k]]; b += h->C[h->dcol[k]]; }
        h->T[2 * I] = a; h->T[2 * I + 1] = b;
    }
    const double sc = h->K / (double)n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < n; p++) {
        const int64_t I = h->comm[p];
        double as = h->T[2 * I], ac = h->T[2 * I + 1];
        const int64_t b = h->rptr[p], m = b + h->rnm[p], e = h->rptr[p + 1];
        for (int64_t q = b; q < m; q++) { as -= h->s[h->ent[q]]; ac -= h->c[h->ent[q]]; }
        for (int64_t q = m; q < e; q++) { as += h->s[h->ent[q]]; ac += h->c[h->ent[q]]; }
        f[p] = h->omega[p] + sc * (h->c[p] * as - h->s[p] * ac);
    }
}

void cpb_rhs(cpb_t* h, const double* theta, double* f)
{
    const int64_t n = h->n;
    for (int64_t p = 0; p < n; p++) h->Y[p] = theta[h->perm[p]];
    rhs_perm(h, h->Y, h->f);
    for (int64_t p = 0; p < n; p++) f[h->perm[p]] = h->f[p];
}

void cpb_rk4(cpb_t* h, double* theta, double step, int64_t steps)
{
    const int64_t n = h->n;
    for (int64_t p = 0; p < n; p++) h->y[p] = theta[h->perm[p]];
    for (int64_t t = 0; t < steps; t++) {
        rhs_perm(h, h->y, h->f);
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < n; p++) { h->k[p] = h->f[p]; h->Y[p] = h->y[p] + 0.5 * step * h->f[p]; }
        rhs_perm(h, h->Y, h->f);
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < n; p++) { h->k[p] += 2.0 * h->f[p]; h->Y[p] = h->y[p] + 0.5 * step * h->f[p]; }
        rhs_perm(h, h->Y, h->f);
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < n; p++) { h->k[p] += 2.0 * h->f[p]; h->Y[p] = h->y[p] + step * h->f[p]; }
        rhs_perm(h, h->Y, h->f);
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < n; p++) h->y[p] += (step / 6.0) * (h->k[p] + h->f[p]);
    }
    for (int64_t p = 0; p < n; p++) theta[h->perm[p]] = h->y[p];
}
