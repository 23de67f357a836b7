/*
 * gift_oracle.c -- plain, slow, FP64 CPU oracle of the GiFt filter path.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path, and nothing here is tuned.
 * Built twice: single-threaded, and with OpenMP (the row loops spread over the
 * host's cores; the same bits, since every output element is still summed by
 * one thread in the same order).
 *
 * What it computes, step by step in the paper's order:
 *   1. clique net model (Sec. 3.2.3 with Algorithm 1; weight rule after Eq. 4):
 *      every net of M >= 2 pins has weight w = 2/M; every ordered pair of its
 *      pin slots (p, q), p != q, whose cells i != j differ adds w to A[i][j];
 *      the same cell pair in several nets sums (a single w_ij, Sec. 2.1).
 *      The sum for one (i, j) runs in increasing net order.
 *   2. degrees d_i = sum_j A_ij (Sec. 2.1), in FP64, over the stored values.
 *   3. augmented normalised adjacency (Eq. 16):
 *         A~_sigma = (D + sigma I)^-1/2 (A + sigma I) (D + sigma I)^-1/2
 *      and, as a test-only variant, the random-walk form (D+sigma I)^-1 (A+sigma I).
 *   4. GiFt filter (Eq. 15, Algorithm 1 line 2, coefficients of Sec. 4.1):
 *         g' = a0 A~_2^2 g + a1 A~_4^2 g + a2 A~_4^4 g,   (a0,a1,a2) = (0.1,0.7,0.2)
 *      every term computed by fresh repeated application from g.
 *   5. fixed cells keep their given locations (Sec. 3.2.2, Sec. 4.1).
 *   6. HPWL: sum over nets of (max x - min x) + (max y - min y), pins at cell
 *      locations (the paper reports HPWL, Sec. 4.1, without defining it; this is
 *      the standard half-perimeter bounding box).
 *
 * Layout: a signal is row-major [N][K] doubles (K = 2 x number of signals).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t i, j; /* row, column */
    int32_t e;    /* net index: fixes the order of the FP64 sum */
    double w;     /* 2/M of that net */
} oracle_pair;

typedef struct {
    int32_t n;
    int64_t nnz;
    int64_t *row_ptr; /* [n+1] */
    int32_t *col;     /* [nnz] */
    double *val;      /* [nnz] */
} oracle_graph;

static int cmp_pair(const void *pa, const void *pb) {
    const oracle_pair *a = (const oracle_pair *)pa, *b = (const oracle_pair *)pb;
    if (a->i != b->i) return a->i < b->i ? -1 : 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    if (a->e != b->e) return a->e < b->e ? -1 : 1;
    return 0;
}

/* Step 1: clique expansion into CSR with summed duplicates.  Returns NULL on
 * bad input (cell id out of range, decreasing net_ptr) or allocation failure.
 * cut > 0 leaves out the nets of at least `cut` pins (their cliques are then
 * applied implicitly; see oracle_implicit_degrees). */
static oracle_graph *build_cut(int32_t num_cells, int32_t num_nets, const int64_t *net_ptr,
                               const int32_t *pin_cell, int64_t cut) {
    if (num_cells <= 0 || num_nets < 0 || net_ptr[0] != 0) return NULL;
    int64_t npairs = 0;
    for (int32_t e = 0; e < num_nets; ++e) {
        int64_t m = net_ptr[e + 1] - net_ptr[e];
        if (m < 0) return NULL;
        if (m >= 2 && (cut <= 0 || m < cut)) npairs += m * (m - 1);
    }
    for (int64_t p = 0; p < net_ptr[num_nets]; ++p)
        if (pin_cell[p] < 0 || pin_cell[p] >= num_cells) return NULL;

    oracle_pair *pairs = (oracle_pair *)malloc((size_t)(npairs > 0 ? npairs : 1) * sizeof(oracle_pair));
    if (!pairs) return NULL;
    int64_t k = 0;
    for (int32_t e = 0; e < num_nets; ++e) {
        int64_t b = net_ptr[e], m = net_ptr[e + 1] - net_ptr[e];
        if (m < 2) continue;
        if (cut > 0 && m >= cut) continue;
        double w = 2.0 / (double)m;
        for (int64_t p = 0; p < m; ++p)
            for (int64_t q = 0; q < m; ++q) {
                if (p == q) continue;
                int32_t i = pin_cell[b + p], j = pin_cell[b + q];
                if (i == j) continue; /* two pins of one net on one cell: no self edge */
                pairs[k].i = i;
                pairs[k].j = j;
                pairs[k].e = e;
                pairs[k].w = w;
                ++k;
            }
    }
    /* sort by (row, column, net): pairs bucketed by row in generation order,
     * then each row's bucket sorted by (column, net) */
    int64_t *bstart = (int64_t *)calloc((size_t)num_cells + 1, sizeof(int64_t));
    oracle_pair *sorted = (oracle_pair *)malloc((size_t)(k > 0 ? k : 1) * sizeof(oracle_pair));
    if (!bstart || !sorted) {
        free(pairs);
        free(bstart);
        free(sorted);
        return NULL;
    }
    for (int64_t t = 0; t < k; ++t) bstart[pairs[t].i + 1] += 1;
    for (int32_t i = 0; i < num_cells; ++i) bstart[i + 1] += bstart[i];
    {
        int64_t *fill = (int64_t *)malloc(((size_t)num_cells + 1) * sizeof(int64_t));
        if (!fill) {
            free(pairs);
            free(bstart);
            free(sorted);
            return NULL;
        }
        memcpy(fill, bstart, ((size_t)num_cells + 1) * sizeof(int64_t));
        for (int64_t t = 0; t < k; ++t) sorted[fill[pairs[t].i]++] = pairs[t];
        free(fill);
    }
    free(pairs);
    pairs = sorted;
#pragma omp parallel for schedule(dynamic, 256)
    for (int32_t i = 0; i < num_cells; ++i)
        qsort(pairs + bstart[i], (size_t)(bstart[i + 1] - bstart[i]), sizeof(oracle_pair), cmp_pair);
    free(bstart);

    oracle_graph *g = (oracle_graph *)calloc(1, sizeof(oracle_graph));
    g->n = num_cells;
    g->row_ptr = (int64_t *)calloc((size_t)num_cells + 1, sizeof(int64_t));
    g->col = (int32_t *)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
    g->val = (double *)malloc((size_t)(k > 0 ? k : 1) * sizeof(double));
    int64_t nnz = 0;
    for (int64_t t = 0; t < k; ++t) {
        if (nnz > 0 && t > 0 && pairs[t].i == pairs[t - 1].i && pairs[t].j == pairs[t - 1].j) {
            g->val[nnz - 1] += pairs[t].w; /* increasing net order */
        } else {
            g->col[nnz] = pairs[t].j;
            g->val[nnz] = pairs[t].w;
            g->row_ptr[pairs[t].i + 1] += 1;
            ++nnz;
        }
    }
    for (int32_t i = 0; i < num_cells; ++i) g->row_ptr[i + 1] += g->row_ptr[i];
    g->nnz = nnz;
    free(pairs);
    return g;
}

oracle_graph *oracle_build(int32_t num_cells, int32_t num_nets, const int64_t *net_ptr,
                           const int32_t *pin_cell) {
    return build_cut(num_cells, num_nets, net_ptr, pin_cell, 0);
}

oracle_graph *oracle_build_cut(int32_t num_cells, int32_t num_nets, const int64_t *net_ptr,
                               const int32_t *pin_cell, int64_t cut) {
    return build_cut(num_cells, num_nets, net_ptr, pin_cell, cut);
}

static int cmp_i32(const void *pa, const void *pb) {
    const int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Degrees of the cliques left out by oracle_build_cut: a net of M >= cut pins
 * with k of its pins on cell i adds, for each of those k pins, w = 2/M to the
 * pairs with its M - k pins on other cells: d_i += (k * w) * (M - k).  Nets in
 * increasing order, after the expanded part (d holds it on entry).  Returns 0,
 * or -1 on allocation failure. */
int oracle_implicit_degrees(int32_t num_cells, int32_t num_nets, const int64_t *net_ptr, const int32_t *pin_cell,
                            int64_t cut, double *d) {
    (void)num_cells;
    if (cut <= 0) return 0;
    for (int32_t e = 0; e < num_nets; ++e) {
        int64_t b = net_ptr[e], m = net_ptr[e + 1] - net_ptr[e];
        if (m < 2 || m < cut) continue;
        int32_t *cells = (int32_t *)malloc((size_t)m * sizeof(int32_t));
        if (!cells) return -1;
        memcpy(cells, pin_cell + b, (size_t)m * sizeof(int32_t));
        qsort(cells, (size_t)m, sizeof(int32_t), cmp_i32);
        double w = 2.0 / (double)m;
        for (int64_t r = 0; r < m;) {
            int64_t k = 1;
            while (r + k < m && cells[r + k] == cells[r]) ++k;
            d[cells[r]] += ((double)k * w) * (double)(m - k);
            r += k;
        }
        free(cells);
    }
    return 0;
}

int64_t oracle_graph_nnz(const oracle_graph *g) { return g->nnz; }

void oracle_graph_copy(const oracle_graph *g, int64_t *row_ptr, int32_t *col, double *val) {
    memcpy(row_ptr, g->row_ptr, sizeof(int64_t) * ((size_t)g->n + 1));
    if (g->nnz) {
        memcpy(col, g->col, sizeof(int32_t) * (size_t)g->nnz);
        memcpy(val, g->val, sizeof(double) * (size_t)g->nnz);
    }
}

void oracle_graph_free(oracle_graph *g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col);
    free(g->val);
    free(g);
}

/* Round-to-nearest-even of v to a binary format with `prec` significand bits
 * (implicit bit included) and minimum normal exponent `emin`.
 *   fmt 0: keep FP64; 1: binary32 (24, -126); 2: bfloat16 (8, -126); 3: binary16 (11, -14).
 * v / ulp is an exact power-of-two scaling, and nearbyint() rounds to nearest
 * even under the default rounding mode. */
static double round_to(double v, int prec, int emin) {
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    frexp(v, &e);  /* |v| in [2^(e-1), 2^e) */
    int lead = e - 1;
    if (lead < emin) lead = emin; /* subnormal range: fixed quantum */
    double ulp = ldexp(1.0, lead - (prec - 1));
    return nearbyint(v / ulp) * ulp;
}

void oracle_round(int64_t n, const double *in, double *out, int32_t fmt) {
    for (int64_t t = 0; t < n; ++t) {
        switch (fmt) {
        case 1: out[t] = round_to(in[t], 24, -126); break;
        case 2: out[t] = round_to(in[t], 8, -126); break;
        case 3: out[t] = round_to(in[t], 11, -14); break;
        default: out[t] = in[t];
        }
    }
}

/* Step 2: d_i = sum_j A_ij (Sec. 2.1), summed in column order. */
void oracle_degrees(int32_t n, const int64_t *row_ptr, const double *val, double *d) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s += val[k];
        d[i] = s;
    }
}

/* Step 3: y = A~_sigma x for every one of the K columns.
 *   norm 0 (Eq. 16): y_i = s_i * ( sum_j A_ij s_j x_j + sigma s_i x_i ),  s = (d + sigma)^-1/2
 *   norm 1 (random walk): y_i = ( sum_j A_ij x_j + sigma x_i ) / (d_i + sigma)          */
void oracle_apply(int32_t n, int32_t K, const int64_t *row_ptr, const int32_t *col, const double *val,
                  const double *d, double sigma, int32_t norm, const double *x, double *y) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t c = 0; c < K; ++c) {
            double acc = 0.0;
            if (norm == 0) {
                double si = 1.0 / sqrt(d[i] + sigma);
                for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                    int32_t j = col[k];
                    double sj = 1.0 / sqrt(d[j] + sigma);
                    acc += val[k] * sj * x[(int64_t)j * K + c];
                }
                acc += sigma * si * x[(int64_t)i * K + c];
                y[(int64_t)i * K + c] = si * acc;
            } else {
                for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                    acc += val[k] * x[(int64_t)col[k] * K + c];
                acc += sigma * x[(int64_t)i * K + c];
                y[(int64_t)i * K + c] = acc / (d[i] + sigma);
            }
        }
    }
}

/* Step 3 with the cliques of the nets of at least `cut` pins applied from the
 * netlist instead of the CSR (which holds the other nets, oracle_build_cut):
 * same operator as oracle_apply on the full expansion.  In the clique model
 * each pin slot p of such a net e (M pins, weight w = 2/M) on cell i pairs
 * with every slot q on another cell and adds w * xh_cell(q) to row i, where xh
 * is the scaled signal (s x, or x in the random-walk form).  Summed over the
 * slots q first, a slot of cell i adds w * (S_e - k xh_i), with S_e the sum of
 * xh over all M slots and k the slots of e on cell i; cell i's k slots add k
 * times that.  Rows take the CSR part (column order), then the nets in
 * increasing order, then the self-loop.  Returns 0, or -1 on allocation
 * failure. */
int oracle_apply_cut(int32_t n, int32_t K, const int64_t *row_ptr, const int32_t *col, const double *val,
                     const double *d, double sigma, int32_t norm, int32_t num_nets, const int64_t *net_ptr,
                     const int32_t *pin_cell, int64_t cut, const double *x, double *y) {
    size_t len = (size_t)n * (size_t)K;
    double *xh = (double *)malloc((len > 0 ? len : 1) * sizeof(double));
    double *acc = (double *)calloc(len > 0 ? len : 1, sizeof(double));
    double *S = (double *)malloc((size_t)(K > 0 ? K : 1) * sizeof(double));
    if (!xh || !acc || !S) {
        free(xh);
        free(acc);
        free(S);
        return -1;
    }
#pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < n; ++j) {
        double sj = norm == 0 ? 1.0 / sqrt(d[j] + sigma) : 1.0;
        for (int32_t c = 0; c < K; ++c) xh[(int64_t)j * K + c] = sj * x[(int64_t)j * K + c];
    }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t i = 0; i < n; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            for (int32_t c = 0; c < K; ++c) acc[(int64_t)i * K + c] += val[k] * xh[(int64_t)col[k] * K + c];
    for (int32_t e = 0; cut > 0 && e < num_nets; ++e) {
        int64_t b = net_ptr[e], m = net_ptr[e + 1] - net_ptr[e];
        if (m < 2 || m < cut) continue;
        double w = 2.0 / (double)m;
        for (int32_t c = 0; c < K; ++c) {
            double t = 0.0;
            for (int64_t p = 0; p < m; ++p) t += xh[(int64_t)pin_cell[b + p] * K + c];
            S[c] = t;
        }
        int32_t *cells = (int32_t *)malloc((size_t)m * sizeof(int32_t));
        if (!cells) {
            free(xh);
            free(acc);
            free(S);
            return -1;
        }
        memcpy(cells, pin_cell + b, (size_t)m * sizeof(int32_t));
        qsort(cells, (size_t)m, sizeof(int32_t), cmp_i32);
        for (int64_t r = 0; r < m;) {
            int64_t k = 1;
            while (r + k < m && cells[r + k] == cells[r]) ++k;
            int64_t i = cells[r];
            for (int32_t c = 0; c < K; ++c)
                acc[i * K + c] += (double)k * w * (S[c] - (double)k * xh[i * K + c]);
            r += k;
        }
        free(cells);
    }
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double si = norm == 0 ? 1.0 / sqrt(d[i] + sigma) : 1.0;
        for (int32_t c = 0; c < K; ++c) {
            double a = acc[(int64_t)i * K + c] + sigma * xh[(int64_t)i * K + c];
            y[(int64_t)i * K + c] = norm == 0 ? si * a : a / (d[i] + sigma);
        }
    }
    free(xh);
    free(acc);
    free(S);
    return 0;
}

/* Steps 4-5: out = sum_t alpha_t A~_{sigma_t}^{power_t} g, then fixed rows := g.
 * Each term starts again from g (no sharing between terms).  cut > 0: the
 * cliques of the nets of at least cut pins come from the netlist
 * (oracle_apply_cut), the rest from the CSR. */
static int filter_terms(int32_t n, int32_t K, const int64_t *row_ptr, const int32_t *col, const double *val,
                        const double *d, int32_t num_terms, const double *sigma, const int32_t *power,
                        const double *alpha, int32_t norm, int32_t reimpose, const uint8_t *is_fixed,
                        int32_t num_nets, const int64_t *net_ptr, const int32_t *pin_cell, int64_t cut,
                        const double *g, double *out) {
    size_t len = (size_t)n * (size_t)K;
    double *v = (double *)malloc(len * sizeof(double));
    double *t = (double *)malloc(len * sizeof(double));
    if (!v || !t) {
        free(v);
        free(t);
        return -1;
    }
    for (size_t q = 0; q < len; ++q) out[q] = 0.0;
    for (int32_t term = 0; term < num_terms; ++term) {
        memcpy(v, g, len * sizeof(double));
        for (int32_t p = 0; p < power[term]; ++p) {
            if (cut > 0) {
                if (oracle_apply_cut(n, K, row_ptr, col, val, d, sigma[term], norm, num_nets, net_ptr, pin_cell, cut,
                                     v, t) != 0) {
                    free(v);
                    free(t);
                    return -1;
                }
            } else {
                oracle_apply(n, K, row_ptr, col, val, d, sigma[term], norm, v, t);
            }
            double *sw = v;
            v = t;
            t = sw;
        }
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < len; ++q) out[q] += alpha[term] * v[q];
    }
    if (reimpose && is_fixed) {
        for (int32_t i = 0; i < n; ++i)
            if (is_fixed[i])
                for (int32_t c = 0; c < K; ++c) out[(int64_t)i * K + c] = g[(int64_t)i * K + c];
    }
    free(v);
    free(t);
    return 0;
}

int oracle_filter(int32_t n, int32_t K, const int64_t *row_ptr, const int32_t *col, const double *val,
                  const double *d, int32_t num_terms, const double *sigma, const int32_t *power,
                  const double *alpha, int32_t norm, int32_t reimpose, const uint8_t *is_fixed,
                  const double *g, double *out) {
    return filter_terms(n, K, row_ptr, col, val, d, num_terms, sigma, power, alpha, norm, reimpose, is_fixed, 0, NULL,
                        NULL, 0, g, out);
}

int oracle_filter_cut(int32_t n, int32_t K, const int64_t *row_ptr, const int32_t *col, const double *val,
                      const double *d, int32_t num_terms, const double *sigma, const int32_t *power,
                      const double *alpha, int32_t norm, int32_t reimpose, const uint8_t *is_fixed,
                      int32_t num_nets, const int64_t *net_ptr, const int32_t *pin_cell, int64_t cut,
                      const double *g, double *out) {
    return filter_terms(n, K, row_ptr, col, val, d, num_terms, sigma, power, alpha, norm, reimpose, is_fixed,
                        num_nets, net_ptr, pin_cell, cut, g, out);
}

/* Threads the library runs its parallel loops on (1 when built without OpenMP).
 * Every parallel loop writes each output element from one thread, in the
 * serial build's order, so both builds give the same bits. */
#ifdef _OPENMP
#include <omp.h>
int oracle_threads(void) { return omp_get_max_threads(); }
#else
int oracle_threads(void) { return 1; }
#endif

/* Step 6: HPWL of each of S signals; xy is [N][S][2]. */
void oracle_hpwl(int32_t num_nets, const int64_t *net_ptr, const int32_t *pin_cell, int32_t S,
                 const double *xy, double *out) {
    for (int32_t s = 0; s < S; ++s) {
        double total = 0.0;
        for (int32_t e = 0; e < num_nets; ++e) {
            int64_t b = net_ptr[e], m = net_ptr[e + 1] - net_ptr[e];
            if (m < 1) continue;
            double xlo = INFINITY, xhi = -INFINITY, ylo = INFINITY, yhi = -INFINITY;
            for (int64_t p = 0; p < m; ++p) {
                int64_t c = pin_cell[b + p];
                double x = xy[(c * S + s) * 2 + 0], y = xy[(c * S + s) * 2 + 1];
                if (x < xlo) xlo = x;
                if (x > xhi) xhi = x;
                if (y < ylo) ylo = y;
                if (y > yhi) yhi = y;
            }
            total += (xhi - xlo) + (yhi - ylo);
        }
        out[s] = total;
    }
}
