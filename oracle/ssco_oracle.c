/*
 * ssco_oracle.c -- plain, slow, FP64 reference for the fixed-pattern
 * assemble / Cholesky-refactor / solve / adjoint path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and
 * the bench's CPU-baseline leg load this file's library.  It shares no code,
 * header, table or helper with the CUDA path and includes none of it.
 *
 * What it follows:
 *  - The computation repeated for every new value set on a fixed pattern is
 *    the paper's setting (Sec. 3.3 "Requirements for input code": control flow
 *    independent of the values, cost amortised over many evaluations).  The
 *    paper never factorizes with its own method (Sec. 2 cites sparse Cholesky
 *    code generation as related work; Sec. 5.5/5.6 quote an external solver),
 *    so each function below is the textbook definition of its result:
 *      assembly      K = A^T diag(w) A + shift*I, or K = sum_e E_e K_e^0
 *                    (the element-block form of Sec. 4.2.4), sums taken in
 *                    ascending (e, local index) order;
 *      permutation   K~ = P K P^T with perm[new] = old;
 *      symbolic      column-merge elimination: struct(L_j) = struct(K~_{j:,j})
 *                    united with struct(L_c) \ {c} over the etree children c;
 *                    parent(j) = smallest row > j; fundamental supernodes;
 *                    levels = longest path from the leaves (the "level" of
 *                    Sec. 4.3, read as a height so that a level never holds a
 *                    node together with one that depends on it);
 *      numeric       left-looking Cholesky with a dense accumulator,
 *                    updates subtracted in ascending k, correctly rounded sqrt;
 *      solves        forward substitution by columns of L, backward by
 *                    columns of L^T, then un-permute;
 *      adjoint       wbar_e = -(A mu)_e (A x)_e, Ebar_e = -mu_e^T K_e^0 x_e,
 *                    shiftbar = -mu^T x over shifted diagonals, with K mu = xbar;
 *                    per-call element blocks: -(mu_u x_v + mu_v x_u) per entry;
 *      values        cotangent edge weights (Sec. 5.3) and linear-tet
 *                    stiffness blocks V B^T D B from vertex positions.
 *  - Parity pins (tests): dense numpy Cholesky / solve, tridiag(-1,2,-1)
 *    closed form, reconstruction, brute-force boolean elimination, central
 *    differences; tet blocks: the Lame-constant index formula, rigid-body
 *    null space, the constant-strain energy, scaling and rotation laws.  Built with -O2 -ffp-contract=off, no fast-math.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* triplets sorted by (col, row, seq): duplicates summed in seq order   */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t col, row;
    int64_t seq;
    double v;
} trip;

static int trip_cmp(const void* a, const void* b) {
    const trip* x = (const trip*)a;
    const trip* y = (const trip*)b;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    if (x->row != y->row) return x->row < y->row ? -1 : 1;
    if (x->seq != y->seq) return x->seq < y->seq ? -1 : 1;
    return 0;
}

/* Sum sorted triplets into CSC (colptr[n+1], rowind, val).  Returns nnz. */
static int64_t trips_to_csc(int32_t n, trip* t, int64_t nt, int64_t* colptr,
                            int32_t* rowind, double* val) {
    qsort(t, (size_t)nt, sizeof(trip), trip_cmp);
    int64_t nz = 0;
    for (int32_t j = 0; j <= n; ++j) colptr[j] = 0;
    for (int64_t k = 0; k < nt; ++k) {
        if (nz > 0 && rowind[nz - 1] == t[k].row && k > 0 && t[k - 1].col == t[k].col) {
            val[nz - 1] += t[k].v;
        } else {
            rowind[nz] = t[k].row;
            val[nz] = t[k].v;
            colptr[t[k].col + 1]++;
            nz++;
        }
    }
    for (int32_t j = 0; j < n; ++j) colptr[j + 1] += colptr[j];
    return nz;
}

/* Upper bound on the lower-triangle nonzeros of A^T W A (+ diagonal). */
int64_t or_atwa_cap(int32_t n, int32_t m, const int64_t* rowptr) {
    int64_t cap = n;
    for (int32_t e = 0; e < m; ++e) {
        int64_t d = rowptr[e + 1] - rowptr[e];
        cap += d * (d + 1) / 2;
    }
    return cap;
}

/* K = A^T diag(w) A + shift*I, lower triangle, CSC in the original order.
 * For each row e (ascending) and each pair of its nonzeros (a <= b in
 * storage order): K[max(u,v), min(u,v)] += A_eu * w_e * A_ev; afterwards
 * K_uu += shift for every u.  Returns nnz. */
int64_t or_assemble_atwa(int32_t n, int32_t m, const int64_t* rowptr, const int32_t* colind,
                         const double* aval, const double* w, double shift,
                         int64_t* colptr, int32_t* rowind, double* val) {
    int64_t cap = or_atwa_cap(n, m, rowptr);
    trip* t = (trip*)malloc((size_t)cap * sizeof(trip));
    int64_t nt = 0;
    for (int32_t e = 0; e < m; ++e) {
        for (int64_t a = rowptr[e]; a < rowptr[e + 1]; ++a) {
            for (int64_t b = a; b < rowptr[e + 1]; ++b) {
                int32_t u = colind[a], v = colind[b];
                t[nt].row = u > v ? u : v;
                t[nt].col = u > v ? v : u;
                t[nt].seq = nt;
                t[nt].v = aval[a] * w[e] * aval[b];
                nt++;
            }
        }
    }
    for (int32_t u = 0; u < n; ++u) { /* make every diagonal present */
        t[nt].row = u;
        t[nt].col = u;
        t[nt].seq = nt;
        t[nt].v = 0.0;
        nt++;
    }
    int64_t nz = trips_to_csc(n, t, nt, colptr, rowind, val);
    free(t);
    for (int32_t u = 0; u < n; ++u) val[colptr[u]] += shift; /* diagonal first in column */
    return nz;
}

int64_t or_elem_cap(int32_t n, int32_t m, int32_t dim) {
    return (int64_t)m * dim * (dim + 1) / 2 + n;
}

/* K = sum_e E_e K_e^0 over free DOFs (dofs < 0 are fixed), lower CSC.
 * K0 is [m][dim*(dim+1)/2], row-major lower (i >= j).  A DOF that no
 * element references gets K_ii = 1; every referenced DOF gets + shift. */
int64_t or_assemble_elem(int32_t n, int32_t m, int32_t dim, const int32_t* dofs,
                         const double* K0, const double* E, double shift,
                         int64_t* colptr, int32_t* rowind, double* val) {
    int64_t cap = or_elem_cap(n, m, dim);
    int32_t npk = dim * (dim + 1) / 2;
    trip* t = (trip*)malloc((size_t)cap * sizeof(trip));
    char* touched = (char*)calloc((size_t)n, 1);
    int64_t nt = 0;
    for (int32_t e = 0; e < m; ++e) {
        int32_t p = 0;
        for (int32_t i = 0; i < dim; ++i) {
            for (int32_t j = 0; j <= i; ++j, ++p) {
                int32_t u = dofs[(int64_t)e * dim + i], v = dofs[(int64_t)e * dim + j];
                if (u < 0 || v < 0) continue;
                t[nt].row = u > v ? u : v;
                t[nt].col = u > v ? v : u;
                t[nt].seq = nt;
                t[nt].v = E[e] * K0[(int64_t)e * npk + p];
                nt++;
                touched[u] = 1;
                touched[v] = 1;
            }
        }
    }
    for (int32_t u = 0; u < n; ++u) {
        t[nt].row = u;
        t[nt].col = u;
        t[nt].seq = nt;
        t[nt].v = touched[u] ? 0.0 : 1.0;
        nt++;
    }
    int64_t nz = trips_to_csc(n, t, nt, colptr, rowind, val);
    free(t);
    for (int32_t u = 0; u < n; ++u)
        if (touched[u]) val[colptr[u]] += shift;
    free(touched);
    return nz;
}

/* K~ = P K P^T (lower CSC in, lower CSC out), perm[new] = old. */
void or_permute(int32_t n, const int64_t* colptr, const int32_t* rowind, const double* val,
                const int32_t* perm, int64_t* pcolptr, int32_t* prowind, double* pval) {
    int32_t* iperm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) iperm[perm[i]] = i;
    int64_t nz = colptr[n];
    trip* t = (trip*)malloc((size_t)(nz > 0 ? nz : 1) * sizeof(trip));
    for (int32_t j = 0; j < n; ++j) {
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            int32_t a = iperm[rowind[p]], b = iperm[j];
            t[p].row = a > b ? a : b;
            t[p].col = a > b ? b : a;
            t[p].seq = p;
            t[p].v = val[p];
        }
    }
    trips_to_csc(n, t, nz, pcolptr, prowind, pval);
    free(t);
    free(iperm);
}

/* ------------------------------------------------------------------ */
/* symbolic factorization                                               */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t n;
    int64_t* Kcolptr; /* pattern of K~ (lower) */
    int32_t* Krowind;
    int32_t* parent;
    int32_t* colcount;
    int64_t* Lcolptr;
    int32_t* Lrowind; /* rows ascending, diagonal first */
    int32_t* col_level;
    int32_t n_snodes;
    int32_t* snode_first; /* [n_snodes+1] */
    int32_t* sn_parent;
    int32_t* sn_level;
} or_symb;

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return x < y ? -1 : (x > y);
}

or_symb* or_symbolic(int32_t n, const int64_t* Kcolptr, const int32_t* Krowind) {
    or_symb* s = (or_symb*)calloc(1, sizeof(or_symb));
    s->n = n;
    s->Kcolptr = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    memcpy(s->Kcolptr, Kcolptr, (size_t)(n + 1) * sizeof(int64_t));
    s->Krowind = (int32_t*)malloc((size_t)(Kcolptr[n] > 0 ? Kcolptr[n] : 1) * sizeof(int32_t));
    memcpy(s->Krowind, Krowind, (size_t)Kcolptr[n] * sizeof(int32_t));
    s->parent = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    s->colcount = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    s->col_level = (int32_t*)malloc((size_t)n * sizeof(int32_t));

    /* per-column patterns, grown as we go */
    int32_t** pat = (int32_t**)malloc((size_t)n * sizeof(int32_t*));
    int32_t* plen = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    /* children lists */
    int32_t* head = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* next = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* nchild = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    int32_t* mark = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* buf = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) {
        head[i] = -1;
        mark[i] = -1;
    }
    for (int32_t j = 0; j < n; ++j) {
        int32_t len = 0;
        mark[j] = j;
        buf[len++] = j;
        for (int64_t p = Kcolptr[j]; p < Kcolptr[j + 1]; ++p) {
            int32_t i = Krowind[p];
            if (i > j && mark[i] != j) {
                mark[i] = j;
                buf[len++] = i;
            }
        }
        for (int32_t c = head[j]; c >= 0; c = next[c]) {
            for (int32_t q = 0; q < plen[c]; ++q) {
                int32_t i = pat[c][q];
                if (i > c && mark[i] != j) { /* struct(L_c) \ {c}; all such i >= j */
                    mark[i] = j;
                    buf[len++] = i;
                }
            }
        }
        qsort(buf, (size_t)len, sizeof(int32_t), cmp_i32);
        pat[j] = (int32_t*)malloc((size_t)len * sizeof(int32_t));
        memcpy(pat[j], buf, (size_t)len * sizeof(int32_t));
        plen[j] = len;
        s->colcount[j] = len;
        s->parent[j] = len > 1 ? buf[1] : -1;
        if (s->parent[j] >= 0) {
            int32_t pj = s->parent[j];
            next[j] = head[pj];
            head[pj] = j;
            nchild[pj]++;
        }
        /* level: longest path from a leaf */
        int32_t lv = 0;
        for (int32_t c = head[j]; c >= 0; c = next[c])
            if (s->col_level[c] + 1 > lv) lv = s->col_level[c] + 1;
        s->col_level[j] = lv;
    }
    s->Lcolptr = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    s->Lcolptr[0] = 0;
    for (int32_t j = 0; j < n; ++j) s->Lcolptr[j + 1] = s->Lcolptr[j] + plen[j];
    s->Lrowind = (int32_t*)malloc((size_t)(s->Lcolptr[n] > 0 ? s->Lcolptr[n] : 1) * sizeof(int32_t));
    for (int32_t j = 0; j < n; ++j) {
        memcpy(s->Lrowind + s->Lcolptr[j], pat[j], (size_t)plen[j] * sizeof(int32_t));
        free(pat[j]);
    }
    free(pat);
    free(plen);

    /* fundamental supernodes: j+1 joins j's supernode iff parent(j) = j+1,
     * j+1 has exactly one child, and cnt(j+1) = cnt(j) - 1. */
    s->snode_first = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t ns = 0;
    for (int32_t j = 0; j < n; ++j) {
        int joins = j > 0 && s->parent[j - 1] == j && nchild[j] == 1 &&
                    s->colcount[j] == s->colcount[j - 1] - 1;
        if (!joins) s->snode_first[ns++] = j;
    }
    s->snode_first[ns] = n;
    s->n_snodes = ns;
    int32_t* col2sn = buf; /* reuse */
    for (int32_t k = 0; k < ns; ++k)
        for (int32_t j = s->snode_first[k]; j < s->snode_first[k + 1]; ++j) col2sn[j] = k;
    s->sn_parent = (int32_t*)malloc((size_t)(ns > 0 ? ns : 1) * sizeof(int32_t));
    s->sn_level = (int32_t*)malloc((size_t)(ns > 0 ? ns : 1) * sizeof(int32_t));
    for (int32_t k = 0; k < ns; ++k) {
        int32_t last = s->snode_first[k + 1] - 1;
        s->sn_parent[k] = s->parent[last] >= 0 ? col2sn[s->parent[last]] : -1;
        s->sn_level[k] = 0;
    }
    for (int32_t k = 0; k < ns; ++k) /* parents have larger index */
        if (s->sn_parent[k] >= 0 && s->sn_level[k] + 1 > s->sn_level[s->sn_parent[k]])
            s->sn_level[s->sn_parent[k]] = s->sn_level[k] + 1;
    free(head);
    free(next);
    free(nchild);
    free(mark);
    free(buf);
    return s;
}

int64_t or_symb_nnzL(const or_symb* s) { return s->Lcolptr[s->n]; }
int32_t or_symb_nsnodes(const or_symb* s) { return s->n_snodes; }

void or_symb_get(const or_symb* s, int32_t* parent, int32_t* colcount, int64_t* Lcolptr,
                 int32_t* Lrowind, int32_t* col_level, int32_t* snode_first,
                 int32_t* sn_parent, int32_t* sn_level) {
    int32_t n = s->n;
    if (parent) memcpy(parent, s->parent, (size_t)n * sizeof(int32_t));
    if (colcount) memcpy(colcount, s->colcount, (size_t)n * sizeof(int32_t));
    if (Lcolptr) memcpy(Lcolptr, s->Lcolptr, (size_t)(n + 1) * sizeof(int64_t));
    if (Lrowind) memcpy(Lrowind, s->Lrowind, (size_t)s->Lcolptr[n] * sizeof(int32_t));
    if (col_level) memcpy(col_level, s->col_level, (size_t)n * sizeof(int32_t));
    if (snode_first) memcpy(snode_first, s->snode_first, (size_t)(s->n_snodes + 1) * sizeof(int32_t));
    if (sn_parent) memcpy(sn_parent, s->sn_parent, (size_t)s->n_snodes * sizeof(int32_t));
    if (sn_level) memcpy(sn_level, s->sn_level, (size_t)s->n_snodes * sizeof(int32_t));
}

void or_symb_free(or_symb* s) {
    if (!s) return;
    free(s->Kcolptr);
    free(s->Krowind);
    free(s->parent);
    free(s->colcount);
    free(s->Lcolptr);
    free(s->Lrowind);
    free(s->col_level);
    free(s->snode_first);
    free(s->sn_parent);
    free(s->sn_level);
    free(s);
}

/* ------------------------------------------------------------------ */
/* numeric factorization: left-looking, dense accumulator               */
/* Returns -1 on success, else the first column whose pivot is not > 0. */
/* ------------------------------------------------------------------ */
int32_t or_numeric(const or_symb* s, const double* Kval, double* Lval) {
    int32_t n = s->n;
    const int64_t* Lp = s->Lcolptr;
    const int32_t* Li = s->Lrowind;
    int64_t nzL = Lp[n];
    /* row lists of L (k < j with L_jk != 0), ascending k, with the position
     * of L_jk inside column k */
    int64_t* rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t p = 0; p < nzL; ++p) rp[Li[p] + 1]++;
    for (int32_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
    int32_t* rk = (int32_t*)malloc((size_t)(nzL > 0 ? nzL : 1) * sizeof(int32_t));
    int64_t* rpos = (int64_t*)malloc((size_t)(nzL > 0 ? nzL : 1) * sizeof(int64_t));
    int64_t* fill = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    memcpy(fill, rp, (size_t)n * sizeof(int64_t));
    for (int32_t k = 0; k < n; ++k)
        for (int64_t p = Lp[k]; p < Lp[k + 1]; ++p) {
            rk[fill[Li[p]]] = k;
            rpos[fill[Li[p]]] = p;
            fill[Li[p]]++;
        }
    free(fill);
    double* acc = (double*)calloc((size_t)n, sizeof(double));
    int32_t bad = -1;
    for (int32_t j = 0; j < n && bad < 0; ++j) {
        for (int64_t p = Lp[j]; p < Lp[j + 1]; ++p) acc[Li[p]] = 0.0;
        for (int64_t p = s->Kcolptr[j]; p < s->Kcolptr[j + 1]; ++p)
            if (s->Krowind[p] >= j) acc[s->Krowind[p]] += Kval[p];
        for (int64_t q = rp[j]; q < rp[j + 1]; ++q) {
            int32_t k = rk[q];
            if (k >= j) continue; /* the diagonal entry itself */
            double ljk = Lval[rpos[q]];
            for (int64_t p = rpos[q]; p < Lp[k + 1]; ++p) acc[Li[p]] -= ljk * Lval[p];
        }
        double d = acc[j];
        if (!(d > 0.0)) {
            bad = j;
            break;
        }
        double ljj = sqrt(d);
        Lval[Lp[j]] = ljj;
        for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) Lval[p] = acc[Li[p]] / ljj;
    }
    free(acc);
    free(rp);
    free(rk);
    free(rpos);
    return bad;
}

/* x = P^T L^-T L^-1 P b: forward by columns of L, backward by columns of L^T. */
void or_solve(const or_symb* s, const double* Lval, const int32_t* perm, const double* b,
              double* x) {
    int32_t n = s->n;
    const int64_t* Lp = s->Lcolptr;
    const int32_t* Li = s->Lrowind;
    double* y = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    for (int32_t i = 0; i < n; ++i) y[i] = b[perm[i]];
    for (int32_t j = 0; j < n; ++j) {
        y[j] /= Lval[Lp[j]];
        for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) y[Li[p]] -= Lval[p] * y[j];
    }
    for (int32_t j = n - 1; j >= 0; --j) {
        double t = y[j];
        for (int64_t p = Lp[j] + 1; p < Lp[j + 1]; ++p) t -= Lval[p] * y[Li[p]];
        y[j] = t / Lval[Lp[j]];
    }
    for (int32_t i = 0; i < n; ++i) x[perm[i]] = y[i];
    free(y);
}

/* y = K x with K given by its lower triangle (CSC, any ordering). */
void or_symv(int32_t n, const int64_t* colptr, const int32_t* rowind, const double* val,
             const double* x, double* y) {
    for (int32_t i = 0; i < n; ++i) y[i] = 0.0;
    for (int32_t j = 0; j < n; ++j)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            int32_t i = rowind[p];
            y[i] += val[p] * x[j];
            if (i != j) y[j] += val[p] * x[i];
        }
}

/* ------------------------------------------------------------------ */
/* adjoint: given K mu = xbar (mu computed by or_solve)                 */
/* ------------------------------------------------------------------ */
void or_grad_atwa(int32_t m, const int64_t* rowptr, const int32_t* colind, const double* aval,
                  const double* mu, const double* x, double* wbar) {
    for (int32_t e = 0; e < m; ++e) {
        double am = 0.0, ax = 0.0;
        for (int64_t p = rowptr[e]; p < rowptr[e + 1]; ++p) {
            am += aval[p] * mu[colind[p]];
            ax += aval[p] * x[colind[p]];
        }
        wbar[e] = -am * ax;
    }
}

void or_grad_elem(int32_t m, int32_t dim, const int32_t* dofs, const double* K0, const double* mu,
                  const double* x, double* Ebar) {
    int32_t npk = dim * (dim + 1) / 2;
    for (int32_t e = 0; e < m; ++e) {
        double g = 0.0;
        int32_t p = 0;
        for (int32_t i = 0; i < dim; ++i) {
            for (int32_t j = 0; j <= i; ++j, ++p) {
                int32_t u = dofs[(int64_t)e * dim + i], v = dofs[(int64_t)e * dim + j];
                if (u < 0 || v < 0) continue;
                double k = K0[(int64_t)e * npk + p];
                g += k * mu[u] * x[v];
                if (i != j) g += k * mu[v] * x[u];
            }
        }
        Ebar[e] = -g;
    }
}

/* Cotangent edge weights of a planar triangle mesh (the cotangent Laplacian
 * of the mesh experiments, Sec. 5.3): for every triangle and each of its
 * corners k with the other two corners i, j (in the triangle's cyclic
 * order), cot(angle at k) = (u . v) / |u x v| with u = p_i - p_k,
 * v = p_j - p_k, and half of it is added to the edge opposite k.  One value
 * set; xy is [n_vert][2]. */
void or_cotan_weights(int64_t n_tri, const int32_t* tri, const int32_t* tri_edge, const double* xy, int64_t n_edge,
                      double* w) {
    for (int64_t e = 0; e < n_edge; ++e) w[e] = 0.0;
    for (int64_t t = 0; t < n_tri; ++t) {
        for (int c = 0; c < 3; ++c) {
            int32_t k = tri[3 * t + c], i = tri[3 * t + (c + 1) % 3], j = tri[3 * t + (c + 2) % 3];
            double ux = xy[2 * i] - xy[2 * k], uy = xy[2 * i + 1] - xy[2 * k + 1];
            double vx = xy[2 * j] - xy[2 * k], vy = xy[2 * j + 1] - xy[2 * k + 1];
            double dot = ux * vx + uy * vy;
            double cross = fabs(ux * vy - uy * vx);
            w[tri_edge[3 * t + c]] += 0.5 * dot / cross;
        }
    }
}

/* Adjoint of per-call element blocks (K = sum_e K_e, K_e packed row-major
 * lower, entry p = (i, j), i >= j): with K mu = xbar and x the solution,
 * dloss/dK_e[p] = -mu_u x_u for i == j and -(mu_u x_v + mu_v x_u) for
 * i > j (the entry sits at (u, v) and (v, u)); 0 when u or v is fixed.
 * One value set; out is [m][dim(dim+1)/2]. */
void or_grad_blocks(int32_t m, int32_t dim, const int32_t* dofs, const double* mu, const double* x, double* out) {
    int32_t npk = dim * (dim + 1) / 2;
    for (int32_t e = 0; e < m; ++e) {
        int32_t p = 0;
        for (int32_t i = 0; i < dim; ++i) {
            for (int32_t j = 0; j <= i; ++j, ++p) {
                int32_t u = dofs[(int64_t)e * dim + i], v = dofs[(int64_t)e * dim + j];
                double g = 0.0;
                if (u >= 0 && v >= 0) g = (i == j) ? -(mu[u] * x[u]) : -(mu[u] * x[v] + mu[v] * x[u]);
                out[(int64_t)e * npk + p] = g;
            }
        }
    }
}

/* Stiffness block of a linear (4-node) tetrahedron in isotropic linear
 * elasticity, built the textbook way: shape functions N_a = barycentric
 * coordinates, their gradients from the 4x4 system [1 x_a^T] (the
 * coefficients of N_a = alpha_a + beta_a . x), the 6x12 strain-displacement
 * matrix B (Voigt order xx, yy, zz, yz, xz, xy with engineering shear), the
 * 6x6 isotropic D(E, nu), and K = V B^T D B with V = |det| / 6.  Local DOF
 * 3a+c is component c of vertex a.  One value set; xyz is [n_node][3], E
 * per tet; out is [n_tet][78], the lower triangle packed row-major.
 * Returns the number of tets with a singular vertex matrix (those blocks
 * are zero). */
static int solve4(double M[4][4], double rhs[4], double sol[4]) {
    /* Gaussian elimination with partial pivoting on a copy */
    double A[4][5];
    for (int r = 0; r < 4; ++r) {
        for (int c = 0; c < 4; ++c) A[r][c] = M[r][c];
        A[r][4] = rhs[r];
    }
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return 0;
        if (piv != c)
            for (int k = 0; k < 5; ++k) {
                double t = A[c][k];
                A[c][k] = A[piv][k];
                A[piv][k] = t;
            }
        for (int r = c + 1; r < 4; ++r) {
            double f = A[r][c] / A[c][c];
            for (int k = c; k < 5; ++k) A[r][k] -= f * A[c][k];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double s = A[r][4];
        for (int k = r + 1; k < 4; ++k) s -= A[r][k] * sol[k];
        sol[r] = s / A[r][r];
    }
    return 1;
}

int32_t or_tet_stiffness(int64_t n_tet, const int32_t* tets, const double* xyz, const double* E, double nu,
                         double* out) {
    int32_t bad = 0;
    for (int64_t t = 0; t < n_tet; ++t) {
        double* Kp = out + t * 78;
        double M[4][4];
        for (int a = 0; a < 4; ++a) {
            M[a][0] = 1.0;
            for (int c = 0; c < 3; ++c) M[a][c + 1] = xyz[3 * (int64_t)tets[4 * t + a] + c];
        }
        /* N_a(x) = coefficients solving M coef = e_a: coef = (alpha, beta) */
        double grad[4][3];
        int ok = 1;
        for (int a = 0; a < 4 && ok; ++a) {
            double rhs[4] = {0, 0, 0, 0}, sol[4];
            rhs[a] = 1.0;
            /* N_a(x_b) = delta_ab: rows of M times the coefficient vector */
            ok = solve4(M, rhs, sol);
            for (int c = 0; c < 3; ++c) grad[a][c] = sol[c + 1];
        }
        /* det M by cofactor expansion of the edge vectors (= det J) */
        double e1[3], e2[3], e3[3];
        for (int c = 0; c < 3; ++c) {
            e1[c] = M[1][c + 1] - M[0][c + 1];
            e2[c] = M[2][c + 1] - M[0][c + 1];
            e3[c] = M[3][c + 1] - M[0][c + 1];
        }
        double det = e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                     e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
        if (!ok || det == 0.0 || !isfinite(det)) {
            for (int p = 0; p < 78; ++p) Kp[p] = 0.0;
            bad++;
            continue;
        }
        double V = fabs(det) / 6.0;
        double Bm[6][12];
        memset(Bm, 0, sizeof(Bm));
        for (int a = 0; a < 4; ++a) {
            double gx = grad[a][0], gy = grad[a][1], gz = grad[a][2];
            Bm[0][3 * a + 0] = gx;
            Bm[1][3 * a + 1] = gy;
            Bm[2][3 * a + 2] = gz;
            Bm[3][3 * a + 1] = gz; /* yz */
            Bm[3][3 * a + 2] = gy;
            Bm[4][3 * a + 0] = gz; /* xz */
            Bm[4][3 * a + 2] = gx;
            Bm[5][3 * a + 0] = gy; /* xy */
            Bm[5][3 * a + 1] = gx;
        }
        double Ee = E ? E[t] : 1.0;
        double lam = Ee * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        double mu = Ee / (2.0 * (1.0 + nu));
        double D[6][6];
        memset(D, 0, sizeof(D));
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) D[r][c] = lam;
            D[r][r] += 2.0 * mu;
            D[r + 3][r + 3] = mu;
        }
        double DB[6][12];
        for (int r = 0; r < 6; ++r)
            for (int c = 0; c < 12; ++c) {
                double s = 0.0;
                for (int k = 0; k < 6; ++k) s += D[r][k] * Bm[k][c];
                DB[r][c] = s;
            }
        int p = 0;
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j <= i; ++j, ++p) {
                double s = 0.0;
                for (int k = 0; k < 6; ++k) s += Bm[k][i] * DB[k][j];
                Kp[p] = V * s;
            }
    }
    return bad;
}
