/*
 * synth.c -- seeded synthetic inputs for the Kuramoto-on-graphs workloads:
 * community sizes, stochastic-block-model (SBM) graphs in CSR, natural
 * frequencies and initial phases.
 *
 * This module holds none of the model's arithmetic; it only draws inputs.
 * Both the CUDA library's tests and the CPU oracle's tests take their inputs
 * from here.  Every draw is a pure function of (seed, stream tag, index):
 * splitmix64 finalisers of the counter, so results do not depend on the
 * thread count or the order in which rows are generated.
 *
 * Graph recipe (the paper's block-matrix experiments, Sec. 3, with the SBM
 * parameters of the workloads): communities are contiguous in the "planted"
 * numbering; an intra-community pair {a, b} is an edge iff a uniform draw
 * keyed by (seed, min, max) is below p_in of that community (so A is
 * symmetric by construction); inter-community edges a < b are drawn by
 * geometric skipping with probability p_out along row a and mirrored.  No
 * self-loops.  The planted numbering is then hidden by a random relabelling
 * sigma (user index = sigma[planted index]), and the CSR is written in user
 * order with sorted rows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLD 0x9E3779B97F4A7C15ull

static inline uint64_t mix64(uint64_t z)
{
    z += GOLD;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* uniform in [0, 1) with 53 random bits, exact and platform independent */
static inline double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }
static inline uint64_t key3(uint64_t seed, uint64_t tag, uint64_t a)
{
    return mix64(mix64(seed * 0xD1B54A32D192ED03ull + tag) ^ a);
}
static inline double draw(uint64_t seed, uint64_t tag, uint64_t a, uint64_t k)
{
    return u01(mix64(key3(seed, tag, a) + k * GOLD));
}

enum { TAG_SIZE = 1, TAG_PERM = 2, TAG_INTRA = 3, TAG_INTER = 4, TAG_PIN = 5,
       TAG_NORMAL = 6, TAG_UNIFORM = 7, TAG_CAUCHY = 8 };

/* ------------------------------------------------------------------------ */
/* Community sizes: min_size + a Dirichlet(alpha) split of the remaining
 * nodes (alpha a positive integer: a Gamma(alpha, 1) draw is the sum of alpha
 * unit exponentials), optionally clipped at max_size with the excess spread
 * over the unclipped communities in proportion to their share, then rounded
 * by largest remainder so the sizes sum to n exactly.  Returns 0, or -1 when
 * the bounds make it impossible. */
int syn_dirichlet_sizes(uint64_t seed, int64_t n, int32_t n_comm, int32_t alpha,
                        int64_t min_size, int64_t max_size, int64_t* sizes)
{
    if (n_comm <= 0 || alpha <= 0 || min_size < 0) return -1;
    int64_t extra = n - (int64_t)n_comm * min_size;
    if (extra < 0) return -1;
    if (max_size > 0 && (max_size < min_size || (int64_t)n_comm * max_size < n)) return -1;
    double cap = (max_size > 0) ? (double)(max_size - min_size) : INFINITY;
    double* raw = malloc(sizeof(double) * (size_t)n_comm);
    uint8_t* fixed = calloc((size_t)n_comm, 1);
    if (!raw || !fixed) { free(raw); free(fixed); return -1; }
    double tot = 0;
    for (int32_t c = 0; c < n_comm; c++) {
        double g = 0;
        for (int32_t k = 0; k < alpha; k++) g -= log1p(-draw(seed, TAG_SIZE, (uint64_t)c, (uint64_t)k));
        raw[c] = g;
        tot += g;
    }
    for (int32_t c = 0; c < n_comm; c++) raw[c] = raw[c] / tot * (double)extra;
    for (int it = 0; it < 4 * n_comm + 4; it++) {
        double over = 0, free_mass = 0;
        for (int32_t c = 0; c < n_comm; c++)
            if (!fixed[c] && raw[c] > cap) { over += raw[c] - cap; raw[c] = cap; fixed[c] = 1; }
        if (over <= 0) break;
        for (int32_t c = 0; c < n_comm; c++) if (!fixed[c]) free_mass += raw[c];
        if (free_mass <= 0) break;
        for (int32_t c = 0; c < n_comm; c++) if (!fixed[c]) raw[c] += over * raw[c] / free_mass;
    }
    int64_t given = 0;
    for (int32_t c = 0; c < n_comm; c++) { sizes[c] = (int64_t)floor(raw[c]); given += sizes[c]; }
    int64_t rem = extra - given;
    while (rem > 0) {                       /* largest remainder, ties by index */
        int32_t best = -1; double bf = -1;
        for (int32_t c = 0; c < n_comm; c++) {
            if (max_size > 0 && sizes[c] >= max_size - min_size) continue;
            double f = raw[c] - (double)sizes[c];
            if (f > bf) { bf = f; best = c; }
        }
        if (best < 0) break;
        sizes[best]++; raw[best] = (double)sizes[best];  /* remainder used */
        rem--;
    }
    for (int32_t c = 0; c < n_comm; c++) sizes[c] += min_size;
    free(raw); free(fixed);
    return rem == 0 ? 0 : -1;
}

/* Uniform random permutation of 0..n-1 (Fisher-Yates driven by one stream). */
void syn_permutation(uint64_t seed, int64_t n, int32_t* perm)
{
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; i--) {
        uint64_t r = mix64(key3(seed, TAG_PERM, 0) + (uint64_t)i * GOLD);
        int64_t j = (int64_t)(r % (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* Per-community intra probabilities drawn uniformly in [lo, hi). */
void syn_pin_uniform(uint64_t seed, int32_t n_comm, double lo, double hi, double* p_in)
{
    for (int32_t c = 0; c < n_comm; c++) p_in[c] = lo + (hi - lo) * draw(seed, TAG_PIN, (uint64_t)c, 0);
}

/* ------------------------------------------------------------------------ */
/* SBM, planted numbering.  comm_off[n_comm+1] are the community boundaries. */
typedef struct {
    int64_t n; int32_t n_comm; const int64_t* off; const double* p_in; double p_out; uint64_t seed;
    const int32_t* comm_of;
} sbm_t;

static inline int intra_edge(const sbm_t* g, int64_t a, int64_t b, int32_t c)
{
    int64_t lo = a < b ? a : b, hi = a < b ? b : a;
    return draw(g->seed, TAG_INTRA, (uint64_t)lo, (uint64_t)hi) < g->p_in[c];
}

/* Upper inter-community neighbours of planted row a: columns b >= off[c+1]
 * (c = community of a) by geometric skipping.  Writes up to cap entries to
 * out (may be NULL) and returns the count. */
static int64_t upper_inter(const sbm_t* g, int64_t a, int32_t* out)
{
    double p = g->p_out;
    if (p <= 0) return 0;
    int64_t b = g->off[g->comm_of[a] + 1], cnt = 0;
    if (p >= 1) { for (; b < g->n; b++) { if (out) out[cnt] = (int32_t)b; cnt++; } return cnt; }
    double lq = log1p(-p);
    uint64_t k = 0;
    while (b < g->n) {
        double u = draw(g->seed, TAG_INTER, (uint64_t)a, k++);
        double skip = floor(log1p(-u) / lq);
        if (skip >= (double)(g->n - b)) break;
        b += (int64_t)skip;
        if (out) out[cnt] = (int32_t)b;
        cnt++;
        b++;
    }
    return cnt;
}

static int cmp_i32(const void* x, const void* y)
{
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    return (a > b) - (a < b);
}

/* Generates the SBM and writes it in user order (user = sigma[planted]).
 * Two calls: with col == NULL it fills row_ptr[n+1] and returns nnz; with
 * col != NULL (size nnz) it fills the sorted rows.  Returns nnz or -1. */
int64_t syn_sbm_csr(uint64_t seed, int64_t n, int32_t n_comm, const int64_t* comm_off,
                    const double* p_in, double p_out, const int32_t* sigma,
                    int64_t* row_ptr, int32_t* col)
{
    if (n <= 0 || n_comm <= 0 || comm_off[0] != 0 || comm_off[n_comm] != n) return -1;
    int32_t* comm_of = malloc(sizeof(int32_t) * (size_t)n);
    int64_t* ucnt = calloc((size_t)n, sizeof(int64_t));
    int64_t* lcnt = calloc((size_t)n + 1, sizeof(int64_t));
    if (!comm_of || !ucnt || !lcnt) { free(comm_of); free(ucnt); free(lcnt); return -1; }
    for (int32_t c = 0; c < n_comm; c++)
        for (int64_t a = comm_off[c]; a < comm_off[c + 1]; a++) comm_of[a] = c;
    sbm_t g = { n, n_comm, comm_off, p_in, p_out, seed, comm_of };

    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t a = 0; a < n; a++) ucnt[a] = upper_inter(&g, a, NULL);
    int64_t* uptr = malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!uptr) { free(comm_of); free(ucnt); free(lcnt); return -1; }
    uptr[0] = 0;
    for (int64_t a = 0; a < n; a++) uptr[a + 1] = uptr[a] + ucnt[a];
    int32_t* up = malloc(sizeof(int32_t) * (size_t)(uptr[n] > 0 ? uptr[n] : 1));
    int64_t* lptr = malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t* low = malloc(sizeof(int32_t) * (size_t)(uptr[n] > 0 ? uptr[n] : 1));
    if (!up || !lptr || !low) { free(comm_of); free(ucnt); free(lcnt); free(uptr); free(up); free(lptr); free(low); return -1; }
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t a = 0; a < n; a++) upper_inter(&g, a, up + uptr[a]);
    /* transpose: lower[b] = {a < b : b in upper[a]}, in increasing a */
    for (int64_t e = 0; e < uptr[n]; e++) lcnt[up[e]]++;
    lptr[0] = 0;
    for (int64_t b = 0; b < n; b++) lptr[b + 1] = lptr[b] + lcnt[b];
    memset(lcnt, 0, sizeof(int64_t) * (size_t)n);
    for (int64_t a = 0; a < n; a++)
        for (int64_t e = uptr[a]; e < uptr[a + 1]; e++) {
            int64_t b = up[e];
            low[lptr[b] + lcnt[b]++] = (int32_t)a;
        }

    int64_t ret = 0;
    if (!col) {
        int64_t* deg = malloc(sizeof(int64_t) * (size_t)n);
        if (!deg) { ret = -1; goto done; }
        #pragma omp parallel for schedule(dynamic, 64)
        for (int64_t a = 0; a < n; a++) {
            int32_t c = comm_of[a];
            int64_t d = 0;
            for (int64_t b = comm_off[c]; b < comm_off[c + 1]; b++)
                if (b != a && intra_edge(&g, a, b, c)) d++;
            deg[a] = d + (uptr[a + 1] - uptr[a]) + (lptr[a + 1] - lptr[a]);
        }
        for (int64_t a = 0; a < n; a++) row_ptr[sigma[a] + 1] = deg[a];
        row_ptr[0] = 0;
        for (int64_t u = 0; u < n; u++) row_ptr[u + 1] += row_ptr[u];
        ret = row_ptr[n];
        free(deg);
    } else {
        #pragma omp parallel for schedule(dynamic, 64)
        for (int64_t a = 0; a < n; a++) {
            int32_t c = comm_of[a];
            int64_t pos = row_ptr[sigma[a]];
            for (int64_t e = lptr[a]; e < lptr[a + 1]; e++) col[pos++] = sigma[low[e]];
            for (int64_t b = comm_off[c]; b < comm_off[c + 1]; b++)
                if (b != a && intra_edge(&g, a, b, c)) col[pos++] = sigma[b];
            for (int64_t e = uptr[a]; e < uptr[a + 1]; e++) col[pos++] = sigma[up[e]];
            int64_t beg = row_ptr[sigma[a]];
            qsort(col + beg, (size_t)(pos - beg), sizeof(int32_t), cmp_i32);
        }
        ret = row_ptr[n];
    }
done:
    free(comm_of); free(ucnt); free(lcnt); free(uptr); free(up); free(lptr); free(low);
    return ret;
}

/* ------------------------------------------------------------------------ */
/* Per-node draws.  Index i is the user (original) node index. */
void syn_uniform(uint64_t seed, uint64_t tag, int64_t n, double lo, double hi, double* out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) out[i] = lo + (hi - lo) * draw(seed, TAG_UNIFORM + 16 * tag, (uint64_t)i, 0);
}

/* standard normal by the Box-Muller transform, one pair of uniforms per node */
void syn_normal(uint64_t seed, uint64_t tag, int64_t n, double mu, double sigma_, double* out)
{
    const double two_pi = 6.283185307179586476925286766559;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double u1 = 1.0 - draw(seed, TAG_NORMAL + 16 * tag, (uint64_t)i, 0);   /* (0, 1] */
        double u2 = draw(seed, TAG_NORMAL + 16 * tag, (uint64_t)i, 1);
        out[i] = mu + sigma_ * sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
    }
}

/* Cauchy(loc, scale) by inversion, clipped to [loc - clip, loc + clip] */
void syn_cauchy(uint64_t seed, uint64_t tag, int64_t n, double loc, double scale, double clip, double* out)
{
    const double pi = 3.14159265358979323846264338328;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double u = draw(seed, TAG_CAUCHY + 16 * tag, (uint64_t)i, 0);
        double x = loc + scale * tan(pi * (u - 0.5));
        if (clip > 0) { if (x > loc + clip) x = loc + clip; if (x < loc - clip) x = loc - clip; }
        out[i] = x;
    }
}
