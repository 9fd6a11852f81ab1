/* direct.c -- O1/O2 by direct FP64 summation, compiled (test infrastructure).
 *
 * This file is test infrastructure, like the rest of oracle/: only the test
 * suite, the smoke check and the CPU legs of the benchmark load it.  It shares
 * nothing with the CUDA library.
 *
 * It evaluates the same plain definitions as oracle/expansion.py, in C so that
 * full-size grids finish in seconds on a many-core host:
 *
 *   forward (Eq. 1.4, discrete convolution of Section 3.5, 0-based, periodic)
 *     y[i] = sum_k sum_d h_k[d] w_k[i - d] u[i - d]
 *   adjoint (transpose of the forward map; for real h_k, w_k)
 *     x[j] = sum_k w_k[j] sum_d h_k[d] v[j + d]
 *
 * with indices taken per axis modulo the grid (ny = 1 for 1D).  The sums run
 * over the nonzero taps d of h_k and over the rows and columns where w_k is
 * not zero: every skipped product is exactly zero, so the result is the sum
 * of the definition.  All arithmetic is double precision; float32 inputs are
 * promoted on load.  The order of the sums is fixed (terms, then tap rows,
 * then taps, then columns), so results do not depend on the thread count:
 * each thread owns whole output rows.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* element i of a float32 (f64 == 0) or float64 array */
static double ld(const void* p, int f64, int64_t i) {
    return f64 ? ((const double*)p)[i] : (double)((const float*)p)[i];
}

static int wrap(int64_t i, int n) {
    int64_t r = i % n;
    return (int)(r < 0 ? r + n : r);
}

/* The nonzero taps of one impulse response, grouped by row offset. */
typedef struct {
    int ngroups;
    int* gdr;     /* [ngroups] row offset of the group */
    int* gstart;  /* [ngroups + 1] first tap of each group */
    int* dc;      /* [ntaps] column offset */
    double* val;  /* [ntaps] value */
} Taps;

static int taps_make(Taps* t, const void* h, int f64, int ny, int nx) {
    int64_t n = 0, P = (int64_t)ny * nx;
    for (int64_t i = 0; i < P; ++i)
        if (ld(h, f64, i) != 0.0) ++n;
    t->ngroups = 0;
    t->gdr = (int*)malloc(sizeof(int) * (size_t)(ny + 1));
    t->gstart = (int*)malloc(sizeof(int) * (size_t)(ny + 1));
    t->dc = (int*)malloc(sizeof(int) * (size_t)(n + 1));
    t->val = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    if (!t->gdr || !t->gstart || !t->dc || !t->val) return -1;
    int64_t k = 0;
    for (int r = 0; r < ny; ++r) {
        int64_t first = k;
        for (int c = 0; c < nx; ++c) {
            double v = ld(h, f64, (int64_t)r * nx + c);
            if (v != 0.0) {
                t->dc[k] = c;
                t->val[k] = v;
                ++k;
            }
        }
        if (k > first) {
            t->gdr[t->ngroups] = r;
            t->gstart[t->ngroups] = (int)first;
            ++t->ngroups;
        }
    }
    t->gstart[t->ngroups] = (int)k;
    return 0;
}

static void taps_free(Taps* t) {
    free(t->gdr);
    free(t->gstart);
    free(t->dc);
    free(t->val);
}

/* Where w_k is not zero: a flag per row and the maximal runs of columns in
 * which some row is not zero. */
typedef struct {
    unsigned char* row;
    int nruns;
    int* a;     /* first column of each run */
    int* len;
} Support;

static int support_make(Support* s, const void* w, int f64, int ny, int nx) {
    unsigned char* col = (unsigned char*)calloc((size_t)nx, 1);
    s->row = (unsigned char*)calloc((size_t)ny, 1);
    s->a = (int*)malloc(sizeof(int) * (size_t)(nx + 1));
    s->len = (int*)malloc(sizeof(int) * (size_t)(nx + 1));
    if (!col || !s->row || !s->a || !s->len) {
        free(col);
        return -1;
    }
    for (int r = 0; r < ny; ++r)
        for (int c = 0; c < nx; ++c)
            if (ld(w, f64, (int64_t)r * nx + c) != 0.0) {
                s->row[r] = 1;
                col[c] = 1;
            }
    s->nruns = 0;
    for (int c = 0; c < nx;) {
        if (!col[c]) {
            ++c;
            continue;
        }
        int a = c;
        while (c < nx && col[c]) ++c;
        s->a[s->nruns] = a;
        s->len[s->nruns] = c - a;
        ++s->nruns;
    }
    free(col);
    return 0;
}

static void support_free(Support* s) {
    free(s->row);
    free(s->a);
    free(s->len);
}

/* Number of threads the parallel loops use. */
int pce_oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* y[b] (or x[b] when adjoint) for b < batch, all outputs.
 * u: [batch][ny][nx], w, h: [m][ny][nx] (float32 or float64 by the flags),
 * out: [batch][ny][nx] float64.  Returns 0, or -1 when memory runs out. */
int pce_oracle_apply(int adjoint, int batch, int ny, int nx, int m, const void* u, int u64, const void* w,
                     int w64, const void* h, int h64, double* out) {
    const int64_t P = (int64_t)ny * nx;
    Taps* taps = (Taps*)calloc((size_t)(m > 0 ? m : 1), sizeof(Taps));
    Support* sup = (Support*)calloc((size_t)(m > 0 ? m : 1), sizeof(Support));
    double* v = (double*)malloc(sizeof(double) * (size_t)P);
    int err = (!taps || !sup || !v) ? -1 : 0;
    for (int k = 0; k < m && !err; ++k) {
        err = taps_make(&taps[k], (const char*)h + (size_t)k * P * (h64 ? 8 : 4), h64, ny, nx);
        if (!err) err = support_make(&sup[k], (const char*)w + (size_t)k * P * (w64 ? 8 : 4), w64, ny, nx);
    }
    for (int b = 0; b < batch && !err; ++b) {
        double* o = out + (int64_t)b * P;
        memset(o, 0, sizeof(double) * (size_t)P);
        const int64_t ub = (int64_t)b * P;
        if (adjoint) {
            /* v = the right-hand side, promoted once */
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < P; ++i) v[i] = ld(u, u64, ub + i);
        }
        for (int k = 0; k < m; ++k) {
            const Taps* t = &taps[k];
            const Support* s = &sup[k];
            const int64_t wk = (int64_t)k * P;
            if (t->ngroups == 0 || s->nruns == 0) continue;
            if (!adjoint) {
                /* v = w_k . u_b */
#pragma omp parallel for schedule(static)
                for (int64_t i = 0; i < P; ++i) v[i] = ld(w, w64, wk + i) * ld(u, u64, ub + i);
                /* output row r gathers source rows r - dr */
#pragma omp parallel for schedule(dynamic, 4)
                for (int r = 0; r < ny; ++r) {
                    double* yr = o + (int64_t)r * nx;
                    for (int g = 0; g < t->ngroups; ++g) {
                        const int sr = wrap((int64_t)r - t->gdr[g], ny);
                        if (!s->row[sr]) continue;
                        const double* vs = v + (int64_t)sr * nx;
                        for (int q = t->gstart[g]; q < t->gstart[g + 1]; ++q) {
                            const double hv = t->val[q];
                            const int dc = t->dc[q];
                            for (int run = 0; run < s->nruns; ++run) {
                                const int a = s->a[run], len = s->len[run];
                                const int d0 = wrap((int64_t)a + dc, nx);
                                const int n1 = len < nx - d0 ? len : nx - d0;
                                for (int i = 0; i < n1; ++i) yr[d0 + i] += hv * vs[a + i];
                                for (int i = n1; i < len; ++i) yr[d0 + i - nx] += hv * vs[a + i];
                            }
                        }
                    }
                }
            } else {
                /* rows where w_k is not zero: t = sum_d h_k[d] v[j + d] on the
                 * support columns, then x[j] += w_k[j] t */
#pragma omp parallel
                {
                    double* tr = (double*)malloc(sizeof(double) * (size_t)nx);
#pragma omp for schedule(dynamic, 4)
                    for (int j = 0; j < ny; ++j) {
                        if (!tr || !s->row[j]) continue;
                        for (int run = 0; run < s->nruns; ++run)
                            memset(tr + s->a[run], 0, sizeof(double) * (size_t)s->len[run]);
                        for (int g = 0; g < t->ngroups; ++g) {
                            const double* vs = v + (int64_t)wrap((int64_t)j + t->gdr[g], ny) * nx;
                            for (int q = t->gstart[g]; q < t->gstart[g + 1]; ++q) {
                                const double hv = t->val[q];
                                const int dc = t->dc[q];
                                for (int run = 0; run < s->nruns; ++run) {
                                    const int a = s->a[run], len = s->len[run];
                                    const int d0 = wrap((int64_t)a + dc, nx);
                                    const int n1 = len < nx - d0 ? len : nx - d0;
                                    for (int i = 0; i < n1; ++i) tr[a + i] += hv * vs[d0 + i];
                                    for (int i = n1; i < len; ++i) tr[a + i] += hv * vs[d0 + i - nx];
                                }
                            }
                        }
                        double* xr = o + (int64_t)j * nx;
                        for (int run = 0; run < s->nruns; ++run)
                            for (int i = s->a[run]; i < s->a[run] + s->len[run]; ++i)
                                xr[i] += ld(w, w64, wk + (int64_t)j * nx + i) * tr[i];
                    }
                    if (!tr) {
#pragma omp atomic write
                        err = -1;
                    }
                    free(tr);
                }
            }
        }
    }
    for (int k = 0; k < m && taps && sup; ++k) {
        taps_free(&taps[k]);
        support_free(&sup[k]);
    }
    free(taps);
    free(sup);
    free(v);
    return err;
}

/* The same sums at npts selected outputs (row, column pairs in pts, [npts][2];
 * row 0 for 1D), every right-hand side: out [batch][npts] float64. */
int pce_oracle_apply_at(int adjoint, int batch, int ny, int nx, int m, const void* u, int u64, const void* w,
                        int w64, const void* h, int h64, const int64_t* pts, int64_t npts, double* out) {
    const int64_t P = (int64_t)ny * nx;
    Taps* taps = (Taps*)calloc((size_t)(m > 0 ? m : 1), sizeof(Taps));
    int err = taps ? 0 : -1;
    for (int k = 0; k < m && !err; ++k)
        err = taps_make(&taps[k], (const char*)h + (size_t)k * P * (h64 ? 8 : 4), h64, ny, nx);
    if (!err) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t p = 0; p < npts; ++p) {
            const int r = (int)pts[2 * p], c = (int)pts[2 * p + 1];
            for (int b = 0; b < batch; ++b) {
                const int64_t ub = (int64_t)b * P;
                double acc = 0.0;
                for (int k = 0; k < m; ++k) {
                    const Taps* t = &taps[k];
                    const int64_t wk = (int64_t)k * P;
                    if (!adjoint) {
                        for (int g = 0; g < t->ngroups; ++g) {
                            const int64_t sr = (int64_t)wrap((int64_t)r - t->gdr[g], ny) * nx;
                            for (int q = t->gstart[g]; q < t->gstart[g + 1]; ++q) {
                                const int64_t j = sr + wrap((int64_t)c - t->dc[q], nx);
                                const double wv = ld(w, w64, wk + j);
                                if (wv != 0.0) acc += t->val[q] * (wv * ld(u, u64, ub + j));
                            }
                        }
                    } else {
                        const double wv = ld(w, w64, wk + (int64_t)r * nx + c);
                        if (wv == 0.0) continue;
                        double s = 0.0;
                        for (int g = 0; g < t->ngroups; ++g) {
                            const int64_t sr = (int64_t)wrap((int64_t)r + t->gdr[g], ny) * nx;
                            for (int q = t->gstart[g]; q < t->gstart[g + 1]; ++q)
                                s += t->val[q] * ld(u, u64, ub + sr + wrap((int64_t)c + t->dc[q], nx));
                        }
                        acc += wv * s;
                    }
                }
                out[(int64_t)b * npts + p] = acc;
            }
        }
    }
    for (int k = 0; k < m && taps; ++k) taps_free(&taps[k]);
    free(taps);
    return err;
}
