/*
 * ORACLE -- test infrastructure only.  Plain, slow, obviously-correct FP64
 * smoothed-aggregation AMG + preconditioned CG on SCALAR CSR matrices.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may call this code.  It shares no code with the CUDA path: every
 * step below is written here, once, from the paper and from the readings of
 * its silent points that the design notes list.
 *
 * Paper: Demidov, "Efficient solution of 3D elasticity problems with smoothed
 * aggregation algebraic multigrid and block arithmetics" (2022).
 *   Alg. 1 (Sec. 2)  -- setup loop: P_i, B_{i+1} from (A_i, B_i); R_i = P_i^T;
 *                       smoother S_i from A_i; A_{i+1} = R_i A_i P_i; direct
 *                       solver for the coarsest A_L.
 *   Alg. 2 (Sec. 2)  -- V-cycle, used once per preconditioner application.
 *   Sec. 2           -- B is the n x 6 matrix of rigid-body modes; the
 *                       tentative prolongation is built from B in scalar
 *                       arithmetic ("point-wise aggregation with block size 3",
 *                       Sec. 4).
 *   Sec. 4           -- CG outer solver, relative residual 1e-8.
 *
 * Readings of points the paper leaves open (implemented identically, but
 * independently, on the CUDA side):
 *   strength:   node blocks b x b (b = 3 on level 1, 6 below); J != I is
 *               strong iff ||A_IJ||_F^2 > (eps^2 ||A_II||_F) ||A_JJ||_F, with
 *               squares summed in row-major block order; eps_1 = 0.08,
 *               eps_{l+1} = eps_l / 2.  A node without strong neighbours is
 *               isolated: never aggregated, zero prolongation row.
 *   aggregation: three greedy passes in ascending node order (see
 *               orc_aggregate()), or the distance-2 maximal independent set
 *               of orc_aggregate_mis2() (the parallel variant).
 *   P_tent:     per aggregate, stacked B rows, modified Gram-Schmidt with one
 *               re-orthogonalisation pass; a column whose norm after
 *               orthogonalisation is <= 1e-10 x its norm before is dropped
 *               (zero Q column, zero R row).  B_{i+1} = R.
 *   P smoother: damped Jacobi on the unfiltered matrix, P = P_tent -
 *               omega D^{-1} A P_tent with D = diag(A), rho = max_i
 *               sum_j |a_ij| / |a_ii| (Gershgorin), omega = relax (4/3) / rho
 *               with relax = 2 by default (Gershgorin over-estimates
 *               lambda_max(D^{-1} A) by a factor 1.4-2.2 on these matrices,
 *               so relax = 1 leaves P under-smoothed), and the symbolic
 *               pattern.  The strength graph drives only the
 *               aggregation: lumping weak entries into the diagonal (the
 *               classical filtered matrix) leaves near-zero and negative
 *               diagonals on elasticity matrices, which collapses omega.  With
 *               A B = 0, P B_{i+1} = B holds for any threshold.
 *   coarsening stops when n <= coarse_enough, at max_levels levels, when
 *               the aggregates are not fewer than 0.9 x the nodes, or when a
 *               level below the finest has at most 2 coarse_enough rows and
 *               its aggregates would make a level of fewer than
 *               coarse_enough / 4 rows (a tiny last level, aggregated from a
 *               dense operator, doubles the CG iterations or worse).
 *   smoother:   damped SPAI0, M = w_s diag(a_ii / sum_j a_ij^2) (0 for an
 *               empty row), w_s = 0.8 by default: undamped SPAI0 has
 *               lambda_max(M A) of about 2.1-2.25 on Q1 elasticity, which
 *               makes the symmetric V-cycle indefinite and stalls CG.
 *               V(1,1): pre-smoothing from zero is u = M f, post-smoothing is
 *               u += M (f - A u).
 *               Block damped Jacobi (option; the paper names damped Jacobi
 *               among the smoothers of Sec. 2 without a block form or a
 *               damping): M_I = (2 w_s / lambda) A_II^{-1} per node block,
 *               lambda the Rayleigh-quotient estimate of lambda_max(D_b^{-1}
 *               A) after 20 power iterations (orc_block_jacobi_lambda), so the
 *               damped M A peaks near 2 w_s = 1.6: the undamped block Jacobi
 *               of Q1 elasticity has lambda_max 2.6-3.9 (nu 0.2-0.45), and a
 *               fixed damping of 2/3 makes the V-cycle indefinite.
 *   coarsest:   dense Cholesky; a zero row gets a unit pivot and a zero
 *               solution component.
 *   CG:         stop when the recurrence residual ||r||/||f|| <= tol and the
 *               true residual confirms it; otherwise r is replaced by the true
 *               residual and the iteration continues.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off (no FMA contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t nrows, ncols, nnz;
    int64_t *ptr; /* nrows + 1 */
    int32_t *col; /* nnz, ascending within a row */
    double *val;  /* nnz */
} orc_csr;

static orc_csr *csr_new(int64_t nrows, int64_t ncols, int64_t nnz)
{
    orc_csr *A = (orc_csr *)calloc(1, sizeof(orc_csr));
    A->nrows = nrows;
    A->ncols = ncols;
    A->nnz = nnz;
    A->ptr = (int64_t *)calloc((size_t)nrows + 1, sizeof(int64_t));
    A->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    A->val = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    return A;
}

void orc_csr_free(orc_csr *A)
{
    if (!A) return;
    free(A->ptr);
    free(A->col);
    free(A->val);
    free(A);
}

void orc_csr_shape(const orc_csr *A, int64_t *out3)
{
    out3[0] = A->nrows;
    out3[1] = A->ncols;
    out3[2] = A->nnz;
}

void orc_csr_copy(const orc_csr *A, int64_t *ptr, int32_t *col, double *val)
{
    memcpy(ptr, A->ptr, sizeof(int64_t) * (size_t)(A->nrows + 1));
    memcpy(col, A->col, sizeof(int32_t) * (size_t)A->nnz);
    memcpy(val, A->val, sizeof(double) * (size_t)A->nnz);
}

orc_csr *orc_csr_from(int64_t nrows, int64_t ncols, const int64_t *ptr, const int32_t *col,
                      const double *val)
{
    orc_csr *A = csr_new(nrows, ncols, ptr[nrows]);
    memcpy(A->ptr, ptr, sizeof(int64_t) * (size_t)(nrows + 1));
    memcpy(A->col, col, sizeof(int32_t) * (size_t)A->nnz);
    memcpy(A->val, val, sizeof(double) * (size_t)A->nnz);
    return A;
}

/* Block-valued CSR -> scalar CSR (Sec. 2's worked example; the scalar
 * "unblock" view).  Every scalar of a present block is kept, zeros included. */
orc_csr *orc_unblock(int64_t nbrows, int64_t nbcols, int br, int bc, const int32_t *row_ptr,
                     const int32_t *bcol, const double *bval)
{
    int64_t nnzb = row_ptr[nbrows];
    orc_csr *A = csr_new(nbrows * br, nbcols * bc, nnzb * br * bc);
    int64_t q = 0;
    for (int64_t I = 0; I < nbrows; ++I)
        for (int r = 0; r < br; ++r) {
            for (int64_t p = row_ptr[I]; p < row_ptr[I + 1]; ++p)
                for (int c = 0; c < bc; ++c) {
                    A->col[q] = (int32_t)((int64_t)bcol[p] * bc + c);
                    A->val[q] = bval[p * br * bc + r * bc + c];
                    ++q;
                }
            A->ptr[I * br + r + 1] = q;
        }
    return A;
}

/* y = A x, each row summed in ascending column order. */
void orc_spmv(const orc_csr *A, const double *x, double *y)
{
    for (int64_t i = 0; i < A->nrows; ++i) {
        double s = 0.0;
        for (int64_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) s += A->val[p] * x[A->col[p]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ---------------------------------------------------------------------- */
/* Strength of connection on the node graph (Sec. 4: point-wise aggregation
 * with block size b).                                                     */

typedef struct {
    int64_t nnodes, nnz;
    int64_t *ptr;
    int32_t *col;      /* node columns, ascending, diagonal included if present */
    double *norm2;     /* ||A_IJ||_F^2, squares summed in row-major order */
    uint8_t *strong;   /* 1 if J != I and the pair is strong */
} orc_graph;

void orc_graph_free(orc_graph *G)
{
    if (!G) return;
    free(G->ptr);
    free(G->col);
    free(G->norm2);
    free(G->strong);
    free(G);
}

void orc_graph_shape(const orc_graph *G, int64_t *out2)
{
    out2[0] = G->nnodes;
    out2[1] = G->nnz;
}

void orc_graph_copy(const orc_graph *G, int64_t *ptr, int32_t *col, double *norm2,
                    uint8_t *strong)
{
    memcpy(ptr, G->ptr, sizeof(int64_t) * (size_t)(G->nnodes + 1));
    memcpy(col, G->col, sizeof(int32_t) * (size_t)G->nnz);
    memcpy(norm2, G->norm2, sizeof(double) * (size_t)G->nnz);
    memcpy(strong, G->strong, (size_t)G->nnz);
}

/* Node graph of a scalar matrix with node size b: block (I,J) is present if
 * any scalar of it is.  Squared Frobenius norms are accumulated scalar row by
 * scalar row (ascending columns), i.e. in row-major block order. */
orc_graph *orc_strength(const orc_csr *A, int b, double eps)
{
    int64_t nn = A->nrows / b;
    orc_graph *G = (orc_graph *)calloc(1, sizeof(orc_graph));
    G->nnodes = nn;
    G->ptr = (int64_t *)calloc((size_t)nn + 1, sizeof(int64_t));
    double *acc = (double *)calloc((size_t)nn, sizeof(double));
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)nn);
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
    for (int64_t J = 0; J < nn; ++J) mark[J] = -1;
    /* pass 1: pattern size */
    int64_t cap = 0;
    for (int64_t I = 0; I < nn; ++I) {
        int64_t cnt = 0;
        for (int r = 0; r < b; ++r)
            for (int64_t p = A->ptr[I * b + r]; p < A->ptr[I * b + r + 1]; ++p) {
                int64_t J = A->col[p] / b;
                if (mark[J] != I) {
                    mark[J] = I;
                    ++cnt;
                }
            }
        cap += cnt;
        G->ptr[I + 1] = cap;
    }
    G->nnz = cap;
    G->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    G->norm2 = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    G->strong = (uint8_t *)calloc((size_t)(cap > 0 ? cap : 1), 1);
    for (int64_t J = 0; J < nn; ++J) mark[J] = -1;
    /* pass 2: squared norms per block, row-major order */
    for (int64_t I = 0; I < nn; ++I) {
        int64_t nt = 0;
        for (int r = 0; r < b; ++r)
            for (int64_t p = A->ptr[I * b + r]; p < A->ptr[I * b + r + 1]; ++p) {
                int64_t J = A->col[p] / b;
                if (mark[J] != I) {
                    mark[J] = I;
                    acc[J] = 0.0;
                    touched[nt++] = (int32_t)J;
                }
                double a = A->val[p];
                acc[J] = acc[J] + a * a;
            }
        qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
        for (int64_t t = 0; t < nt; ++t) {
            G->col[G->ptr[I] + t] = touched[t];
            G->norm2[G->ptr[I] + t] = acc[touched[t]];
        }
    }
    /* diagonal norms */
    double *dn = (double *)calloc((size_t)nn, sizeof(double));
    for (int64_t I = 0; I < nn; ++I)
        for (int64_t p = G->ptr[I]; p < G->ptr[I + 1]; ++p)
            if (G->col[p] == I) dn[I] = sqrt(G->norm2[p]);
    const double e2 = eps * eps;
    for (int64_t I = 0; I < nn; ++I)
        for (int64_t p = G->ptr[I]; p < G->ptr[I + 1]; ++p) {
            int64_t J = G->col[p];
            if (J == I) continue;
            double thr = e2 * dn[I];
            thr = thr * dn[J];
            G->strong[p] = G->norm2[p] > thr ? 1 : 0;
        }
    free(dn);
    free(acc);
    free(mark);
    free(touched);
    return G;
}

/* Greedy aggregation in three passes, nodes in ascending order.
 *  agg[I] = aggregate id (creation order), or -1 for an isolated node.
 *  pass 1: a node that is free and whose strong neighbours are all free
 *          starts a new aggregate with all of them;
 *  pass 2: a still-free node joins the aggregate of its lowest-index strong
 *          neighbour that was aggregated in pass 1;
 *  pass 3: a still-free node starts a new aggregate with its free strong
 *          neighbours.
 * Returns the number of aggregates. */
int64_t orc_aggregate(const orc_graph *G, int32_t *agg)
{
    const int32_t FREE = -1, ISOLATED = -2;
    int64_t nn = G->nnodes, nagg = 0;
    uint8_t *p1 = (uint8_t *)calloc((size_t)nn + 1, 1);
    for (int64_t I = 0; I < nn; ++I) {
        int has = 0;
        for (int64_t p = G->ptr[I]; p < G->ptr[I + 1]; ++p)
            if (G->strong[p]) has = 1;
        agg[I] = has ? FREE : ISOLATED;
    }
    for (int64_t I = 0; I < nn; ++I) {
        if (agg[I] != FREE) continue;
        int ok = 1;
        for (int64_t p = G->ptr[I]; p < G->ptr[I + 1]; ++p)
            if (G->strong[p] && agg[G->col[p]] != FREE) ok = 0;
        if (!ok) continue;
        agg[I] = (int32_t)nagg;
        p1[I] = 1;
        for (int64_t p = G->ptr[I]; p < G->ptr[I + 1]; ++p)
            if (G->strong[p]) {
                agg[G->col[p]] = (int32_t)nagg;
                p1[G->col[p]] = 1;
            }
        ++nagg;
    }
    for (int64_t I = 0; I < nn; ++I) {
        if (agg[I] != FREE) continue;
        for (int64_t p = G->ptr[I]; p < G->ptr[I + 1]; ++p)
            if (G->strong[p] && p1[G->col[p]]) {
                agg[I] = agg[G->col[p]];
                break;
            }
    }
    for (int64_t I = 0; I < nn; ++I) {
        if (agg[I] != FREE) continue;
        agg[I] = (int32_t)nagg;
        for (int64_t p = G->ptr[I]; p < G->ptr[I + 1]; ++p)
            if (G->strong[p] && agg[G->col[p]] == FREE) agg[G->col[p]] = (int32_t)nagg;
        ++nagg;
    }
    for (int64_t I = 0; I < nn; ++I)
        if (agg[I] == ISOLATED) agg[I] = -1;
    free(p1);
    return nagg;
}

/* MurmurHash3's 32-bit finaliser (Appleby, public domain): two xor-shift /
 * odd-multiply rounds and a last xor-shift, each a bijection of the 32-bit
 * integers, so distinct nodes get distinct priorities. */
uint32_t orc_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* The strong connections made undirected: J is a neighbour of I when either
 * direction is strong (I != J).  Sorted, duplicate-free lists. */
typedef struct {
    int64_t n;
    int64_t *ptr;
    int32_t *adj;
} orc_undirected;

static orc_undirected undirected_strong(const orc_graph *G)
{
    orc_undirected U;
    int64_t nn = G->nnodes, m = 0;
    U.n = nn;
    for (int64_t p = 0; p < G->nnz; ++p) m += G->strong[p] ? 2 : 0;
    int32_t *pi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *pj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int64_t k = 0;
    for (int64_t I = 0; I < nn; ++I)
        for (int64_t p = G->ptr[I]; p < G->ptr[I + 1]; ++p)
            if (G->strong[p]) {
                pi[k] = (int32_t)I; pj[k] = G->col[p]; ++k;
                pi[k] = G->col[p]; pj[k] = (int32_t)I; ++k;
            }
    /* bucket by the first node, then sort and deduplicate each bucket */
    int64_t *cnt = (int64_t *)calloc((size_t)nn + 1, sizeof(int64_t));
    for (int64_t t = 0; t < m; ++t) cnt[pi[t] + 1]++;
    for (int64_t I = 0; I < nn; ++I) cnt[I + 1] += cnt[I];
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn > 0 ? nn : 1));
    for (int64_t I = 0; I < nn; ++I) fill[I] = cnt[I];
    for (int64_t t = 0; t < m; ++t) tmp[fill[pi[t]]++] = pj[t];
    U.ptr = (int64_t *)calloc((size_t)nn + 1, sizeof(int64_t));
    U.adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int64_t w = 0;
    for (int64_t I = 0; I < nn; ++I) {
        int64_t a = cnt[I], b = cnt[I + 1];
        qsort(tmp + a, (size_t)(b - a), sizeof(int32_t), cmp_i32);
        for (int64_t t = a; t < b; ++t)
            if (t == a || tmp[t] != tmp[t - 1]) U.adj[w++] = tmp[t];
        U.ptr[I + 1] = w;
    }
    free(pi);
    free(pj);
    free(cnt);
    free(tmp);
    free(fill);
    return U;
}

static const uint32_t *g_prio_sort;
static int cmp_prio_desc(const void *a, const void *b)
{
    uint32_t x = g_prio_sort[*(const int32_t *)a], y = g_prio_sort[*(const int32_t *)b];
    return (x < y) - (x > y);
}

/* Aggregation by a distance-2 maximal independent set (MIS-2), the
 * parallel alternative to the greedy passes above; the rest of Alg. 1 is
 * unchanged.  On the undirected strong graph:
 *  roots:  visit the nodes that have a neighbour in descending priority
 *          orc_fmix32(I); a node that no earlier root reaches in at most
 *          two edges becomes a root (the greedy MIS of the squared graph);
 *  step 1: a root and its neighbours form an aggregate (roots are at least
 *          three edges apart, so no node neighbours two roots); aggregates
 *          are numbered in ascending root index;
 *  step 2: every other node with a neighbour joins the step-1 aggregate of
 *          its lowest-index neighbour that has one (one exists: the set is
 *          maximal, so some root is two edges away).
 * A node without neighbours stays unaggregated (-1).  Returns the number of
 * aggregates, or -1 if a step-1 conflict or an unplaced node shows the
 * roots are not a maximal distance-2 independent set. */
int64_t orc_aggregate_mis2(const orc_graph *G, int32_t *agg)
{
    int64_t nn = G->nnodes, nagg = 0, bad = 0;
    orc_undirected U = undirected_strong(G);
    uint32_t *prio = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nn > 0 ? nn : 1));
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nn > 0 ? nn : 1));
    uint8_t *reached = (uint8_t *)calloc((size_t)nn + 1, 1);
    uint8_t *root = (uint8_t *)calloc((size_t)nn + 1, 1);
    int32_t *id = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nn > 0 ? nn : 1));
    int32_t *step1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nn > 0 ? nn : 1));
    for (int64_t I = 0; I < nn; ++I) {
        prio[I] = orc_fmix32((uint32_t)I);
        order[I] = (int32_t)I;
    }
    g_prio_sort = prio;
    qsort(order, (size_t)nn, sizeof(int32_t), cmp_prio_desc);
    for (int64_t t = 0; t < nn; ++t) {
        int32_t v = order[t];
        if (U.ptr[v] == U.ptr[v + 1] || reached[v]) continue;
        root[v] = 1;
        reached[v] = 1;
        for (int64_t p = U.ptr[v]; p < U.ptr[v + 1]; ++p) {
            int32_t u = U.adj[p];
            reached[u] = 1;
            for (int64_t q = U.ptr[u]; q < U.ptr[u + 1]; ++q) reached[U.adj[q]] = 1;
        }
    }
    for (int64_t I = 0; I < nn; ++I) id[I] = root[I] ? (int32_t)nagg++ : -1;
    for (int64_t I = 0; I < nn; ++I) {
        step1[I] = id[I];
        if (root[I]) continue;
        for (int64_t p = U.ptr[I]; p < U.ptr[I + 1]; ++p)
            if (root[U.adj[p]]) {
                if (step1[I] >= 0) bad = 1;
                step1[I] = id[U.adj[p]];
            }
    }
    for (int64_t I = 0; I < nn; ++I) {
        agg[I] = step1[I];
        if (agg[I] >= 0 || U.ptr[I] == U.ptr[I + 1]) continue;
        for (int64_t p = U.ptr[I]; p < U.ptr[I + 1]; ++p)
            if (step1[U.adj[p]] >= 0) {
                agg[I] = step1[U.adj[p]];
                break;
            }
        if (agg[I] < 0) bad = 1;
    }
    free(U.ptr);
    free(U.adj);
    free(prio);
    free(order);
    free(reached);
    free(root);
    free(id);
    free(step1);
    return bad ? -1 : nagg;
}

/* Tentative prolongation from the near-nullspace (Sec. 2; Sec. 3 notes this
 * step is scalar).  B is n x ns (n = nnodes * b, ns <= 6), row-major: the six
 * rigid-body modes, or the three translations (the block solver of Sec. 4
 * without a near-nullspace, whose tentative prolongation is the block
 * identity per aggregate).  For aggregate a the member rows of B are stacked
 * in ascending node order and factored by modified Gram-Schmidt with
 * re-orthogonalisation.  P_tent row (b I + r) holds the matching Q row in
 * columns ns a .. ns a + ns - 1 (all stored, zeros included); Bc rows
 * ns a .. ns a + ns - 1 are R.  Isolated nodes get empty rows. */
orc_csr *orc_tentative(int64_t nnodes, int b, const int32_t *agg, int64_t nagg, const double *B,
                       int ns, double *Bc)
{
    int64_t n = nnodes * b;
    int64_t *cnt = (int64_t *)calloc((size_t)nagg + 1, sizeof(int64_t));
    for (int64_t I = 0; I < nnodes; ++I)
        if (agg[I] >= 0) cnt[agg[I] + 1]++;
    for (int64_t a = 0; a < nagg; ++a) cnt[a + 1] += cnt[a];
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt[nagg] + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nagg + 1));
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)(nagg + 1));
    for (int64_t I = 0; I < nnodes; ++I)
        if (agg[I] >= 0) members[fill[agg[I]]++] = I;
    free(fill);

    int64_t naggrows = 0;
    for (int64_t I = 0; I < nnodes; ++I)
        if (agg[I] >= 0) naggrows += b;
    orc_csr *P = csr_new(n, nagg * ns, naggrows * ns);
    for (int64_t I = 0; I < nnodes; ++I)
        for (int r = 0; r < b; ++r)
            P->ptr[I * b + r + 1] = (agg[I] >= 0) ? ns : 0;
    for (int64_t i = 0; i < n; ++i) P->ptr[i + 1] += P->ptr[i];
    memset(Bc, 0, sizeof(double) * (size_t)(nagg * ns * ns));

    for (int64_t a = 0; a < nagg; ++a) {
        int64_t na = cnt[a + 1] - cnt[a], m = na * b;
        double *Q = (double *)calloc((size_t)(m * ns), sizeof(double)); /* column-major m x ns */
        double R[6][6];
        memset(R, 0, sizeof R);
        for (int64_t t = 0; t < na; ++t)
            for (int r = 0; r < b; ++r)
                for (int k = 0; k < ns; ++k)
                    Q[k * m + t * b + r] = B[(members[cnt[a] + t] * b + r) * ns + k];
        int dropped[6] = {0, 0, 0, 0, 0, 0};
        for (int k = 0; k < ns; ++k) {
            double *v = Q + k * m;
            double pre = sqrt(dot(m, v, v));
            for (int pass = 0; pass < 2; ++pass)
                for (int j = 0; j < k; ++j) {
                    if (dropped[j]) continue;
                    double *qj = Q + j * m;
                    double d = dot(m, qj, v);
                    R[j][k] += d;
                    for (int64_t i = 0; i < m; ++i) v[i] -= d * qj[i];
                }
            double post = sqrt(dot(m, v, v));
            if (post <= 1e-10 * pre) {
                dropped[k] = 1;
                for (int64_t i = 0; i < m; ++i) v[i] = 0.0;
                for (int j = 0; j < ns; ++j) R[k][j] = 0.0;
            } else {
                for (int64_t i = 0; i < m; ++i) v[i] /= post;
                R[k][k] = post;
            }
        }
        for (int k = 0; k < ns; ++k)
            for (int j = 0; j < ns; ++j) Bc[(a * ns + k) * ns + j] = R[k][j];
        for (int64_t t = 0; t < na; ++t)
            for (int r = 0; r < b; ++r) {
                int64_t row = members[cnt[a] + t] * b + r, p = P->ptr[row];
                for (int k = 0; k < ns; ++k) {
                    P->col[p + k] = (int32_t)(a * ns + k);
                    P->val[p + k] = Q[k * m + t * b + r];
                }
            }
        free(Q);
    }
    free(cnt);
    free(members);
    return P;
}

/* Data of the damped-Jacobi prolongation smoother (Alg. 1, "construct P_i
 * from A_i"): the scalar diagonal d = diag(A) and the Gershgorin estimate
 * rho = max_i sum_j |a_ij| / |a_ii| of rho(D^{-1} A) over rows with
 * a_ii != 0 (entries summed in ascending column order). */
void orc_jacobi_rho(const orc_csr *A, double *d, double *rho_out)
{
    double rho = 0.0;
    for (int64_t i = 0; i < A->nrows; ++i) {
        double dia = 0.0, s = 0.0;
        for (int64_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
            if (A->col[p] == i) dia = A->val[p];
            s += fabs(A->val[p]);
        }
        d[i] = dia;
        if (dia != 0.0) {
            double g = s / fabs(dia);
            if (g > rho) rho = g;
        }
    }
    *rho_out = rho;
}

/* C = A B (Gustavson), symbolic pattern: every structurally present product
 * term creates an entry, numerically zero or not; columns sorted. */
orc_csr *orc_spgemm(const orc_csr *A, const orc_csr *B)
{
    int64_t n = A->nrows, m = B->ncols;
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; ++j) mark[j] = -1;
    int64_t *ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
            int64_t k = A->col[p];
            for (int64_t s = B->ptr[k]; s < B->ptr[k + 1]; ++s)
                if (mark[B->col[s]] != i) {
                    mark[B->col[s]] = i;
                    ++c;
                }
        }
        ptr[i + 1] = ptr[i] + c;
    }
    orc_csr *C = csr_new(n, m, ptr[n]);
    memcpy(C->ptr, ptr, sizeof(int64_t) * (size_t)(n + 1));
    free(ptr);
    double *acc = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    for (int64_t j = 0; j < m; ++j) mark[j] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t q = C->ptr[i];
        for (int64_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
            int64_t k = A->col[p];
            double a = A->val[p];
            for (int64_t s = B->ptr[k]; s < B->ptr[k + 1]; ++s) {
                int32_t j = B->col[s];
                if (mark[j] != i) {
                    mark[j] = i;
                    acc[j] = 0.0;
                    C->col[q++] = j;
                }
                acc[j] += a * B->val[s];
            }
        }
        qsort(C->col + C->ptr[i], (size_t)(C->ptr[i + 1] - C->ptr[i]), sizeof(int32_t), cmp_i32);
        for (int64_t t = C->ptr[i]; t < C->ptr[i + 1]; ++t) C->val[t] = acc[C->col[t]];
    }
    free(acc);
    free(mark);
    return C;
}

orc_csr *orc_transpose(const orc_csr *A)
{
    orc_csr *T = csr_new(A->ncols, A->nrows, A->nnz);
    for (int64_t p = 0; p < A->nnz; ++p) T->ptr[A->col[p] + 1]++;
    for (int64_t j = 0; j < A->ncols; ++j) T->ptr[j + 1] += T->ptr[j];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(A->ncols + 1));
    memcpy(fill, T->ptr, sizeof(int64_t) * (size_t)(A->ncols + 1));
    for (int64_t i = 0; i < A->nrows; ++i)
        for (int64_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
            int64_t q = fill[A->col[p]]++;
            T->col[q] = (int32_t)i;
            T->val[q] = A->val[p];
        }
    free(fill);
    return T;
}

/* Smoothed prolongation P = P_tent - omega D^{-1} (A P_tent); a row with
 * d_i = 0 keeps its tentative values.  Pattern = union of both patterns. */
orc_csr *orc_smooth_prolongation(const orc_csr *A, const double *d, double omega,
                                 const orc_csr *Pt)
{
    orc_csr *AP = orc_spgemm(A, Pt);
    int64_t n = AP->nrows;
    int64_t *ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) { /* merge count */
        int64_t a = AP->ptr[i], ae = AP->ptr[i + 1], t = Pt->ptr[i], te = Pt->ptr[i + 1], c = 0;
        while (a < ae || t < te) {
            if (t >= te || (a < ae && AP->col[a] < Pt->col[t])) ++a;
            else if (a >= ae || Pt->col[t] < AP->col[a]) ++t;
            else { ++a; ++t; }
            ++c;
        }
        ptr[i + 1] = ptr[i] + c;
    }
    orc_csr *P = csr_new(n, Pt->ncols, ptr[n]);
    memcpy(P->ptr, ptr, sizeof(int64_t) * (size_t)(n + 1));
    free(ptr);
    for (int64_t i = 0; i < n; ++i) {
        double s = (d[i] != 0.0) ? omega / d[i] : 0.0;
        int64_t a = AP->ptr[i], ae = AP->ptr[i + 1], t = Pt->ptr[i], te = Pt->ptr[i + 1],
                q = P->ptr[i];
        while (a < ae || t < te) {
            if (t >= te || (a < ae && AP->col[a] < Pt->col[t])) {
                P->col[q] = AP->col[a];
                P->val[q] = -(s * AP->val[a]);
                ++a;
            } else if (a >= ae || Pt->col[t] < AP->col[a]) {
                P->col[q] = Pt->col[t];
                P->val[q] = Pt->val[t];
                ++t;
            } else {
                P->col[q] = Pt->col[t];
                P->val[q] = Pt->val[t] - s * AP->val[a];
                ++a;
                ++t;
            }
            ++q;
        }
    }
    orc_csr_free(AP);
    return P;
}

/* SPAI0: m_i = a_ii / sum_j a_ij^2, the minimiser of ||I - M A||_F over
 * diagonal M for a symmetric A (0 for an empty row). */
void orc_spai0(const orc_csr *A, double *m)
{
    for (int64_t i = 0; i < A->nrows; ++i) {
        double dia = 0.0, s = 0.0;
        for (int64_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
            if (A->col[p] == i) dia = A->val[p];
            s += A->val[p] * A->val[p];
        }
        m[i] = (s != 0.0) ? dia / s : 0.0;
    }
}

/* Block damped Jacobi: M_I = w A_II^{-1} for every node block I (b x b,
 * row-major in Mb[I * b * b]).  A_II is taken as a dense block (absent
 * entries zero).  A row of A_II that is entirely zero -- a near-nullspace
 * column dropped on the level above gives a zero row and column -- is left
 * out: the inverse is taken of the block on the other rows and columns, and
 * M_I is zero in that row and column.  The inverse is formed in place by
 * Gauss-Jordan elimination without pivoting (A_II is SPD on the kept rows):
 * for each pivot j in turn, row j is multiplied by 1 / a_jj (with a_jj
 * replaced by 1 first), then every other row i loses a_ij times row j (with
 * a_ij replaced by 0 first).  The result is symmetrised exactly, M_ab = M_ba =
 * w (X_ab + X_ba) / 2.  Returns 0, or -(I + 1) for a non-positive pivot in
 * node block I. */
int orc_block_jacobi(const orc_csr *A, int b, double w, double *Mb)
{
    int64_t nn = A->nrows / b;
    for (int64_t I = 0; I < nn; ++I) {
        double blk[6][6] = {{0.0}}, X[6][6] = {{0.0}};
        int keep[6], k = 0;
        for (int r = 0; r < b; ++r) {
            int64_t i = I * b + r;
            for (int64_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
                int64_t j = A->col[p];
                if (j >= I * b && j < I * b + b) blk[r][j - I * b] += A->val[p];
            }
        }
        for (int r = 0; r < b; ++r) {
            int z = 1;
            for (int c = 0; c < b; ++c)
                if (blk[r][c] != 0.0) z = 0;
            if (!z) keep[k++] = r;
        }
        for (int x = 0; x < k; ++x)
            for (int y = 0; y < k; ++y) X[x][y] = blk[keep[x]][keep[y]];
        for (int j = 0; j < k; ++j) {
            double piv = X[j][j];
            if (!(piv > 0.0)) return (int)-(I + 1);
            double inv = 1.0 / piv;
            X[j][j] = 1.0;
            for (int c = 0; c < k; ++c) X[j][c] = X[j][c] * inv;
            for (int i = 0; i < k; ++i) {
                if (i == j) continue;
                double f = X[i][j];
                X[i][j] = 0.0;
                for (int c = 0; c < k; ++c) X[i][c] = X[i][c] - f * X[j][c];
            }
        }
        double *M = Mb + I * b * b;
        for (int e = 0; e < b * b; ++e) M[e] = 0.0;
        for (int x = 0; x < k; ++x)
            for (int y = 0; y < k; ++y)
                M[keep[x] * b + keep[y]] = w * ((X[x][y] + X[y][x]) * 0.5);
    }
    return 0;
}

/* Power-iteration estimate of lambda_max(D_b^{-1} A) for the block diagonal
 * D_b of A (b x b node blocks) whose inverse blocks are W (from
 * orc_block_jacobi with w = 1): x_0 from the integer hash h(i) = (i + 1) *
 * 2654435761 mod 2^32 as x_0[i] = h(i) / 2^32 - 1/2, then `iters` times x
 * = D_b^{-1} A x scaled to unit 2-norm, and last the Rayleigh quotient (x, A
 * x) / (x, D_b x), which never exceeds lambda_max (the generalised
 * eigenvalues of (A, D_b) are those of D_b^{-1} A).  Returns the estimate (0
 * for a zero operator). */
double orc_block_jacobi_lambda(const orc_csr *A, int b, const double *W, int iters)
{
    int64_t n = A->nrows, nn = n / b;
    double *x = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *t = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        uint32_t h = (uint32_t)((uint64_t)(i + 1) * 2654435761u);
        x[i] = (double)h / 4294967296.0 - 0.5;
    }
    for (int k = 0; k < iters; ++k) {
        orc_spmv(A, x, t);
        double nrm = 0.0;
        for (int64_t I = 0; I < nn; ++I)
            for (int a = 0; a < b; ++a) {
                double v = 0.0;
                for (int c = 0; c < b; ++c) v += W[I * b * b + a * b + c] * t[I * b + c];
                x[I * b + a] = v;
                nrm += v * v;
            }
        nrm = sqrt(nrm);
        if (nrm == 0.0) break;
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] / nrm;
    }
    /* Rayleigh quotient: D_b x from A's diagonal blocks */
    orc_spmv(A, x, t);
    double xax = 0.0, xdx = 0.0;
    for (int64_t i = 0; i < n; ++i) xax += x[i] * t[i];
    for (int64_t I = 0; I < nn; ++I)
        for (int r = 0; r < b; ++r) {
            int64_t i = I * b + r;
            double v = 0.0;
            for (int64_t p = A->ptr[i]; p < A->ptr[i + 1]; ++p) {
                int64_t j = A->col[p];
                if (j >= I * b && j < I * b + b) v += A->val[p] * x[j];
            }
            xdx += x[i] * v;
        }
    free(x);
    free(t);
    return xdx > 0.0 ? xax / xdx : 0.0;
}

/* Dense Cholesky A = L L^T in place (lower triangle, row-major n x n).  A row
 * of the original matrix that is entirely zero gets a unit pivot and is
 * flagged in zero_row[] (its solution component is set to 0).  Returns 0, or
 * -(i+1) for a non-positive pivot in row i. */
int orc_cholesky(int64_t n, double *L, uint8_t *zero_row)
{
    for (int64_t i = 0; i < n; ++i) {
        int z = 1;
        for (int64_t j = 0; j < n; ++j)
            if (L[i * n + j] != 0.0) z = 0;
        zero_row[i] = (uint8_t)z;
    }
    for (int64_t j = 0; j < n; ++j) {
        double s = L[j * n + j];
        for (int64_t k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (zero_row[j]) s = 1.0;
        if (!(s > 0.0)) return (int)-(j + 1);
        double ljj = sqrt(s);
        L[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = L[i * n + j];
            for (int64_t k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / ljj;
        }
        for (int64_t i = 0; i < j; ++i) L[i * n + j] = 0.0;
    }
    return 0;
}

void orc_cholesky_solve(int64_t n, const double *L, const uint8_t *zero_row, const double *f,
                        double *u)
{
    for (int64_t i = 0; i < n; ++i) { /* L y = f */
        double s = zero_row[i] ? 0.0 : f[i];
        for (int64_t k = 0; k < i; ++k) s -= L[i * n + k] * u[k];
        u[i] = s / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) { /* L^T u = y */
        double s = u[i];
        for (int64_t k = i + 1; k < n; ++k) s -= L[k * n + i] * u[k];
        u[i] = s / L[i * n + i];
    }
    for (int64_t i = 0; i < n; ++i)
        if (zero_row[i]) u[i] = 0.0;
}

/* ---------------------------------------------------------------------- */
/* Hierarchy (Alg. 1) and its use (Alg. 2, CG).                            */

typedef struct {
    orc_csr *A, *P, *R;
    orc_graph *G;
    int32_t *agg;
    int64_t nagg;
    int b;
    double eps, omega, rho;
    double *M;  /* SPAI0 diagonal */
    double *Mb; /* optional block smoother (b x b per node, row-major), replaces M */
    double bj_lambda; /* block damped Jacobi: the lambda_max(D_b^{-1} A) estimate */
    double *B;  /* near-nullspace of this level, n x ns */
    double *d;  /* filtered diagonal */
    struct orc_ilu *ilu; /* block ILU(0) smoother, when selected */
} orc_level;

struct orc_ilu;
static void ilu_free(struct orc_ilu *F);

typedef struct {
    int nlev;
    orc_level lv[32];
    double *L;        /* coarsest Cholesky factor */
    uint8_t *zrow;
    int64_t nc;
    int npre, npost;
    int ns;           /* near-nullspace columns (6 or 3) = DOFs of a coarse node */
    int ilu_sweeps;   /* Jacobi sweeps per triangular solve of the ILU(0) smoother */
    double *work;     /* scratch, 3 vectors per level */
    double *iwork;    /* scratch of the ILU(0) smoother, 3 vectors of the finest size */
} orc_hier;

typedef struct {
    double eps_strong;   /* 0.08 */
    int coarse_enough;   /* 3000 */
    int max_levels;      /* 15 */
    int npre, npost;     /* 1, 1 */
    double relax;        /* omega multiplier, 2.0 */
    double smooth_relax; /* smoother damping w_s, 0.8 */
    int ns;              /* near-nullspace columns of B: 6 (rigid-body modes) or 3 */
    int smoother;        /* 0: damped SPAI0; 1: block ILU(0); 2: block damped Jacobi */
    int ilu_sweeps;      /* Jacobi sweeps per triangular solve of ILU(0) (2) */
    int aggregation;     /* 0: three greedy passes; 1: MIS-2 (orc_aggregate_mis2) */
} orc_params;

void orc_params_default(orc_params *p)
{
    p->eps_strong = 0.08;
    p->coarse_enough = 3000;
    p->max_levels = 15;
    p->npre = 1;
    p->npost = 1;
    p->relax = 2.0;
    p->smooth_relax = 0.8;
    p->ns = 6;
    p->smoother = 0;
    p->ilu_sweeps = 2;
    p->aggregation = 0;
}

void orc_free(orc_hier *H)
{
    if (!H) return;
    for (int l = 0; l < H->nlev; ++l) {
        orc_level *L = &H->lv[l];
        orc_csr_free(L->A);
        orc_csr_free(L->P);
        orc_csr_free(L->R);
        orc_graph_free(L->G);
        free(L->agg);
        free(L->M);
        free(L->Mb);
        free(L->B);
        free(L->d);
        ilu_free(L->ilu);
    }
    free(H->L);
    free(H->zrow);
    free(H->work);
    free(H->iwork);
    free(H);
}

/* ---------------------------------------------------------------------- */
/* Block ILU(0) smoother (Sec. 4 uses ILU(0) smoothing).                   */
/* The level matrix in b x b blocks (dense blocks, explicit zeros kept) is  */
/* factored as L U on its own block pattern: for every block row I and its  */
/* blocks K < I in ascending order, L_IK = A_IK U_KK^-1, then A_IJ -=       */
/* L_IK A_KJ for the blocks J > K of row I that row K also holds; what is   */
/* left on and above the diagonal is U, and U_II is inverted.  A block      */
/* triangular solve is approximated by a fixed number of Jacobi sweeps, as  */
/* a data-parallel machine does it: L y = r by y <- r - (L - I) y from      */
/* y = r, U x = y by x <- U_D^-1 (y - (U - U_D) x) from x = U_D^-1 y.       */

typedef struct orc_ilu {
    int64_t nb;
    int b;
    int64_t *ptr;    /* block rows */
    int32_t *col;    /* block columns, ascending */
    int64_t *diag;   /* position of the diagonal block of each row */
    double *val;     /* L below, U on and above the diagonal, b x b row-major */
    double *dinv;    /* U_II^-1 */
} orc_ilu;

static void ilu_free(orc_ilu *F)
{
    if (!F) return;
    free(F->ptr);
    free(F->col);
    free(F->diag);
    free(F->val);
    free(F->dinv);
    free(F);
}

/* Gauss-Jordan inverse of a b x b block without pivoting; -1 on a zero or
 * non-finite pivot.  A row of the block that is exactly zero (a DOF whose
 * near-nullspace column was dropped: its whole matrix row and column are
 * zero) gets a unit pivot and a zero row and column in the inverse, so that
 * DOF stays zero, as in the coarse solve. */
static int block_inverse(int b, const double *a, double *inv)
{
    double m[6][12];
    int zero[6];
    for (int r = 0; r < b; ++r) {
        zero[r] = 1;
        for (int c = 0; c < b; ++c) zero[r] &= a[r * b + c] == 0.0;
    }
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < 2 * b; ++c)
            m[r][c] = c < b ? (zero[r] ? (c == r ? 1.0 : 0.0) : a[r * b + c]) : (c - b == r ? 1.0 : 0.0);
    for (int p = 0; p < b; ++p) {
        const double piv = m[p][p];
        if (!(fabs(piv) > 0.0) || !isfinite(piv)) return -1;
        for (int c = 0; c < 2 * b; ++c) m[p][c] /= piv;
        for (int r = 0; r < b; ++r) {
            if (r == p) continue;
            const double f = m[r][p];
            for (int c = 0; c < 2 * b; ++c) m[r][c] -= f * m[p][c];
        }
    }
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) inv[r * b + c] = (zero[r] || zero[c]) ? 0.0 : m[r][b + c];
    return 0;
}

/* C (b x b) = X Y, both b x b row-major */
static void block_mul(int b, const double *X, const double *Y, double *C)
{
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) {
            double v = 0.0;
            for (int k = 0; k < b; ++k) v += X[r * b + k] * Y[k * b + c];
            C[r * b + c] = v;
        }
}

/* Block ILU(0) of A (scalar CSR whose pattern is a union of dense b x b
 * blocks).  Returns NULL if a diagonal block cannot be inverted. */
orc_ilu *orc_ilu0(const orc_csr *A, int b)
{
    const int64_t nb = A->nrows / b, bb = b * b;
    orc_ilu *F = (orc_ilu *)calloc(1, sizeof(orc_ilu));
    F->nb = nb;
    F->b = b;
    F->ptr = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
    /* block pattern from the first scalar row of each block row */
    for (int64_t I = 0; I < nb; ++I) {
        int64_t cnt = 0, last = -1;
        for (int64_t p = A->ptr[I * b]; p < A->ptr[I * b + 1]; ++p)
            if (A->col[p] / b != last) {
                last = A->col[p] / b;
                ++cnt;
            }
        F->ptr[I + 1] = F->ptr[I] + cnt;
    }
    const int64_t nnzb = F->ptr[nb];
    F->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnzb > 0 ? nnzb : 1));
    F->val = (double *)calloc((size_t)(nnzb > 0 ? nnzb : 1) * bb, sizeof(double));
    F->diag = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
    F->dinv = (double *)calloc((size_t)(nb > 0 ? nb : 1) * bb, sizeof(double));
    for (int64_t I = 0; I < nb; ++I) {
        int64_t q = F->ptr[I] - 1, last = -1;
        for (int64_t p = A->ptr[I * b]; p < A->ptr[I * b + 1]; ++p)
            if (A->col[p] / b != last) {
                last = A->col[p] / b;
                F->col[++q] = (int32_t)last;
            }
        F->diag[I] = -1;
        for (int64_t q2 = F->ptr[I]; q2 < F->ptr[I + 1]; ++q2)
            if (F->col[q2] == I) F->diag[I] = q2;
        for (int r = 0; r < b; ++r) {
            int64_t q2 = F->ptr[I];
            for (int64_t p = A->ptr[I * b + r]; p < A->ptr[I * b + r + 1]; ++p) {
                const int32_t J = A->col[p] / b, c = A->col[p] % b;
                while (F->col[q2] != J) ++q2;
                F->val[q2 * bb + r * b + c] = A->val[p];
            }
        }
    }
    double T[36];
    for (int64_t I = 0; I < nb; ++I) {
        for (int64_t pk = F->ptr[I]; pk < F->ptr[I + 1] && F->col[pk] < I; ++pk) {
            const int32_t K = F->col[pk];
            block_mul(b, F->val + pk * bb, F->dinv + K * bb, T); /* L_IK = A_IK U_KK^-1 */
            memcpy(F->val + pk * bb, T, sizeof(double) * (size_t)bb);
            int64_t pkj = F->diag[K] + 1;
            for (int64_t pj = pk + 1; pj < F->ptr[I + 1]; ++pj) {
                const int32_t J = F->col[pj];
                while (pkj < F->ptr[K + 1] && F->col[pkj] < J) ++pkj;
                if (pkj >= F->ptr[K + 1] || F->col[pkj] != J) continue;
                block_mul(b, F->val + pk * bb, F->val + pkj * bb, T); /* A_IJ -= L_IK A_KJ */
                for (int e = 0; e < bb; ++e) F->val[pj * bb + e] -= T[e];
            }
        }
        if (F->diag[I] < 0 || block_inverse(b, F->val + F->diag[I] * bb, F->dinv + I * bb) != 0) {
            ilu_free(F);
            return NULL;
        }
    }
    return F;
}

/* out = ILU^-1 r, approximately: `sweeps` Jacobi sweeps per triangular
 * solve (work: 2 vectors of the level's size). */
void orc_ilu_apply(const orc_ilu *F, int sweeps, const double *r, double *out, double *work)
{
    const int b = F->b, bb = b * b;
    const int64_t nb = F->nb, n = nb * b;
    double *y = work, *t = work + n;
    memcpy(y, r, sizeof(double) * (size_t)n);
    for (int s = 0; s < sweeps; ++s) {
        for (int64_t I = 0; I < nb; ++I)
            for (int rr = 0; rr < b; ++rr) {
                double v = 0.0;
                for (int64_t p = F->ptr[I]; p < F->diag[I]; ++p)
                    for (int c = 0; c < b; ++c) v += F->val[p * bb + rr * b + c] * y[F->col[p] * b + c];
                t[I * b + rr] = r[I * b + rr] - v;
            }
        memcpy(y, t, sizeof(double) * (size_t)n);
    }
    for (int64_t I = 0; I < nb; ++I)
        for (int rr = 0; rr < b; ++rr) {
            double v = 0.0;
            for (int c = 0; c < b; ++c) v += F->dinv[I * bb + rr * b + c] * y[I * b + c];
            out[I * b + rr] = v;
        }
    for (int s = 0; s < sweeps; ++s) {
        for (int64_t I = 0; I < nb; ++I) {
            double res[6];
            for (int rr = 0; rr < b; ++rr) {
                double v = 0.0;
                for (int64_t p = F->diag[I] + 1; p < F->ptr[I + 1]; ++p)
                    for (int c = 0; c < b; ++c) v += F->val[p * bb + rr * b + c] * out[F->col[p] * b + c];
                res[rr] = y[I * b + rr] - v;
            }
            for (int rr = 0; rr < b; ++rr) {
                double v = 0.0;
                for (int c = 0; c < b; ++c) v += F->dinv[I * bb + rr * b + c] * res[c];
                t[I * b + rr] = v;
            }
        }
        memcpy(out, t, sizeof(double) * (size_t)n);
    }
}

/* Factor copies for tests: the blocks (nnzb x b x b) and the diagonal
 * inverses (nb x b x b); NULL pointers skip. */
void orc_ilu_shape(const orc_ilu *F, int64_t *out3)
{
    out3[0] = F->nb;
    out3[1] = F->b;
    out3[2] = F->ptr[F->nb];
}

void orc_ilu_copy(const orc_ilu *F, int64_t *ptr, int32_t *col, double *val, double *dinv)
{
    const int64_t bb = (int64_t)F->b * F->b;
    if (ptr) memcpy(ptr, F->ptr, sizeof(int64_t) * (size_t)(F->nb + 1));
    if (col) memcpy(col, F->col, sizeof(int32_t) * (size_t)F->ptr[F->nb]);
    if (val) memcpy(val, F->val, sizeof(double) * (size_t)(F->ptr[F->nb] * bb));
    if (dinv) memcpy(dinv, F->dinv, sizeof(double) * (size_t)(F->nb * bb));
}

void orc_ilu_free(orc_ilu *F) { ilu_free(F); }

/* Alg. 1.  A is scalar CSR (n = nnodes * bs rows), B is n x prm->ns; coarse
 * nodes carry ns DOFs.  The hierarchy takes a copy of A.  Returns NULL on
 * failure, with *status < 0. */
orc_hier *orc_setup(const orc_csr *A0, int bs, const double *B0, const orc_params *prm,
                    int *status)
{
    orc_hier *H = (orc_hier *)calloc(1, sizeof(orc_hier));
    H->npre = prm->npre;
    H->npost = prm->npost;
    const int ns = prm->ns;
    if (ns != 3 && ns != 6) {
        *status = -1;
        free(H);
        return NULL;
    }
    H->ns = ns;
    H->ilu_sweeps = prm->ilu_sweeps;
    orc_level *L0 = &H->lv[0];
    L0->A = orc_csr_from(A0->nrows, A0->ncols, A0->ptr, A0->col, A0->val);
    L0->b = bs;
    L0->B = (double *)malloc(sizeof(double) * (size_t)(A0->nrows * ns));
    memcpy(L0->B, B0, sizeof(double) * (size_t)(A0->nrows * ns));
    L0->eps = prm->eps_strong;
    H->nlev = 1;
    *status = 0;
    for (;;) {
        orc_level *C = &H->lv[H->nlev - 1];
        int64_t n = C->A->nrows;
        if (n <= prm->coarse_enough || H->nlev >= prm->max_levels || H->nlev >= 31) break;
        C->G = orc_strength(C->A, C->b, C->eps);
        int64_t nn = n / C->b;
        C->agg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nn > 0 ? nn : 1));
        C->nagg = prm->aggregation == 1 ? orc_aggregate_mis2(C->G, C->agg)
                                        : orc_aggregate(C->G, C->agg);
        if (C->nagg < 0) {
            *status = -5;
            orc_free(H);
            return NULL;
        }
        /* Stop rule (Alg. 1 leaves it open): no aggregates, or too few nodes
         * merged; and a level below the finest that is already small (at most
         * 2 coarse_enough rows) becomes the coarsest instead of being
         * coarsened into a tiny level (fewer than coarse_enough / 4 rows). */
        if (C->nagg == 0 || (double)C->nagg >= 0.9 * (double)nn ||
            (H->nlev > 1 && n <= 2 * (int64_t)prm->coarse_enough &&
             4 * C->nagg * (int64_t)ns < (int64_t)prm->coarse_enough)) {
            orc_graph_free(C->G);
            C->G = NULL;
            free(C->agg);
            C->agg = NULL;
            C->nagg = 0;
            break;
        }
        orc_level *N = &H->lv[H->nlev];
        N->B = (double *)malloc(sizeof(double) * (size_t)(C->nagg * ns * ns));
        orc_csr *Pt = orc_tentative(nn, C->b, C->agg, C->nagg, C->B, ns, N->B);
        C->d = (double *)malloc(sizeof(double) * (size_t)n);
        orc_jacobi_rho(C->A, C->d, &C->rho);
        C->omega = (C->rho > 0.0) ? prm->relax * (4.0 / 3.0) / C->rho : 0.0;
        C->P = orc_smooth_prolongation(C->A, C->d, C->omega, Pt);
        orc_csr_free(Pt);
        C->R = orc_transpose(C->P);
        orc_csr *AP = orc_spgemm(C->A, C->P);
        N->A = orc_spgemm(C->R, AP);
        orc_csr_free(AP);
        C->M = (double *)malloc(sizeof(double) * (size_t)n);
        orc_spai0(C->A, C->M);
        for (int64_t i = 0; i < n; ++i) C->M[i] = prm->smooth_relax * C->M[i];
        if (prm->smoother == 2) {
            C->Mb = (double *)malloc(sizeof(double) * (size_t)(n * C->b));
            if (orc_block_jacobi(C->A, C->b, 1.0, C->Mb) != 0) {
                *status = -4;
                orc_free(H);
                return NULL;
            }
            double lam = orc_block_jacobi_lambda(C->A, C->b, C->Mb, 20);
            double w = lam > 0.0 ? 2.0 * prm->smooth_relax / lam : 0.0;
            for (int64_t e = 0; e < n * C->b; ++e) C->Mb[e] = w * C->Mb[e];
            C->bj_lambda = lam;
        }
        if (prm->smoother == 1) {
            C->ilu = orc_ilu0(C->A, C->b);
            if (!C->ilu) {
                *status = -4;
                orc_free(H);
                return NULL;
            }
        }
        N->b = ns;
        N->eps = C->eps * 0.5;
        H->nlev++;
    }
    orc_level *Lc = &H->lv[H->nlev - 1];
    int64_t nc = Lc->A->nrows;
    if (nc > 40000) {
        *status = -2;
        orc_free(H);
        return NULL;
    }
    H->nc = nc;
    H->L = (double *)calloc((size_t)(nc * nc > 0 ? nc * nc : 1), sizeof(double));
    H->zrow = (uint8_t *)calloc((size_t)(nc > 0 ? nc : 1), 1);
    for (int64_t i = 0; i < nc; ++i)
        for (int64_t p = Lc->A->ptr[i]; p < Lc->A->ptr[i + 1]; ++p)
            H->L[i * nc + Lc->A->col[p]] += Lc->A->val[p];
    int rc = orc_cholesky(nc, H->L, H->zrow);
    if (rc != 0) {
        *status = -3;
        orc_free(H);
        return NULL;
    }
    int64_t tot = 0;
    for (int l = 0; l < H->nlev; ++l) tot += 3 * H->lv[l].A->nrows;
    H->work = (double *)calloc((size_t)tot, sizeof(double));
    H->iwork = (double *)calloc((size_t)(3 * H->lv[0].A->nrows + 1), sizeof(double));
    return H;
}

/* out = M x (diagonal SPAI0), the b x b block smoother when one is set
 * (block damped Jacobi, or learned 3x3 blocks), or the block ILU(0)
 * smoother; with add != 0, out += M x. */
static void apply_smoother(const orc_hier *H, const orc_level *L, int64_t n, const double *x,
                           double *out, int add)
{
    if (L->ilu) {
        double *z = H->iwork + 2 * n;
        orc_ilu_apply(L->ilu, H->ilu_sweeps, x, z, H->iwork);
        for (int64_t i = 0; i < n; ++i) out[i] = add ? out[i] + z[i] : z[i];
    } else if (L->Mb) {
        const int bs = L->b;
        for (int64_t I = 0; I < n / bs; ++I)
            for (int a = 0; a < bs; ++a) {
                double v = 0.0;
                for (int c = 0; c < bs; ++c)
                    v += L->Mb[I * bs * bs + a * bs + c] * x[I * bs + c];
                out[I * bs + a] = add ? out[I * bs + a] + v : v;
            }
    } else {
        for (int64_t i = 0; i < n; ++i) out[i] = add ? out[i] + L->M[i] * x[i] : L->M[i] * x[i];
    }
}

/* Replace the smoother of level l by symmetric 3x3 blocks (node block size
 * 3 only).  Returns 0, or -1 if the level has no smoother or other blocks. */
int orc_set_block_smoother(orc_hier *H, int l, const double *Mb)
{
    if (l < 0 || l >= H->nlev - 1 || H->lv[l].b != 3) return -1;
    orc_level *L = &H->lv[l];
    int64_t n = L->A->nrows;
    free(L->Mb);
    L->Mb = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    memcpy(L->Mb, Mb, sizeof(double) * (size_t)(3 * n));
    return 0;
}

/* Alg. 2, one cycle from a zero initial guess on every level. */
static void vcycle_level(orc_hier *H, int l, const double *f, double *u, double *work)
{
    orc_level *L = &H->lv[l];
    int64_t n = L->A->nrows;
    if (l == H->nlev - 1) {
        orc_cholesky_solve(n, H->L, H->zrow, f, u);
        return;
    }
    double *e = work, *fc = work + n, *uc = fc + L->R->nrows, *next = uc + L->R->nrows;
    /* pre-smoothing from u = 0: the first sweep gives u = M f */
    if (H->npre > 0) apply_smoother(H, L, n, f, u, 0);
    else
        for (int64_t i = 0; i < n; ++i) u[i] = 0.0;
    for (int s = 1; s < H->npre; ++s) {
        orc_spmv(L->A, u, e);
        for (int64_t i = 0; i < n; ++i) e[i] = f[i] - e[i];
        apply_smoother(H, L, n, e, u, 1);
    }
    /* residual and restriction: f_{l+1} = R (f - A u) */
    orc_spmv(L->A, u, e);
    for (int64_t i = 0; i < n; ++i) e[i] = f[i] - e[i];
    orc_spmv(L->R, e, fc);
    vcycle_level(H, l + 1, fc, uc, next);
    /* prolongation and correction: u += P u_{l+1} */
    orc_spmv(L->P, uc, e);
    for (int64_t i = 0; i < n; ++i) u[i] += e[i];
    /* post-smoothing */
    for (int s = 0; s < H->npost; ++s) {
        orc_spmv(L->A, u, e);
        for (int64_t i = 0; i < n; ++i) e[i] = f[i] - e[i];
        apply_smoother(H, L, n, e, u, 1);
    }
}

void orc_vcycle(orc_hier *H, const double *f, double *u)
{
    vcycle_level(H, 0, f, u, H->work);
}

/* Preconditioned CG (Sec. 4: CG with one V-cycle as the preconditioner,
 * relative residual 1e-8).  u holds the initial guess on entry.  Returns the
 * number of iterations (A p products), or -1 on breakdown; *rel_out is the
 * final true relative residual ||f - A u|| / ||f||. */
int orc_pcg(orc_hier *H, const double *f, double *u, double tol, int maxiter, double *rel_out)
{
    const orc_csr *A = H->lv[0].A;
    int64_t n = A->nrows;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    int it = 0, status = 0;
    double nf = sqrt(dot(n, f, f));
    if (nf == 0.0) {
        for (int64_t i = 0; i < n; ++i) u[i] = 0.0;
        *rel_out = 0.0;
        goto done;
    }
    orc_spmv(A, u, q);
    for (int64_t i = 0; i < n; ++i) r[i] = f[i] - q[i];
    if (sqrt(dot(n, r, r)) / nf <= tol) {
        *rel_out = sqrt(dot(n, r, r)) / nf;
        goto done;
    }
    orc_vcycle(H, r, z);
    memcpy(p, z, sizeof(double) * (size_t)n);
    double rz = dot(n, r, z);
    *rel_out = sqrt(dot(n, r, r)) / nf;
    while (it < maxiter) {
        orc_spmv(A, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0) || !(rz > 0.0)) {
            status = -1;
            break;
        }
        double alpha = rz / pq;
        for (int64_t i = 0; i < n; ++i) u[i] += alpha * p[i];
        for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
        ++it;
        double res = sqrt(dot(n, r, r)) / nf;
        *rel_out = res;
        if (res <= tol) {
            orc_spmv(A, u, q);
            for (int64_t i = 0; i < n; ++i) r[i] = f[i] - q[i];
            double tr = sqrt(dot(n, r, r)) / nf;
            *rel_out = tr;
            if (tr <= tol) break;
        }
        if (it >= maxiter) break;
        orc_vcycle(H, r, z);
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
done:
    free(r);
    free(z);
    free(p);
    free(q);
    return status < 0 ? status : it;
}

/* ---- accessors for the test harness ---------------------------------- */
int orc_nlevels(const orc_hier *H) { return H->nlev; }

/* info: [nrows, b, nagg, has_P, nnz_A] ; scalars: [eps, omega, rho] */
void orc_level_info(const orc_hier *H, int l, int64_t *info, double *scal)
{
    const orc_level *L = &H->lv[l];
    info[0] = L->A->nrows;
    info[1] = L->b;
    info[2] = L->nagg;
    info[3] = L->P != NULL;
    info[4] = L->A->nnz;
    scal[0] = L->eps;
    scal[1] = L->omega;
    scal[2] = L->rho;
    scal[3] = L->bj_lambda;
}

const orc_csr *orc_level_matrix(const orc_hier *H, int l, int which) /* 0 A, 1 P, 2 R */
{
    const orc_level *L = &H->lv[l];
    return which == 0 ? L->A : which == 1 ? L->P : L->R;
}

const orc_graph *orc_level_graph(const orc_hier *H, int l) { return H->lv[l].G; }

void orc_level_vectors(const orc_hier *H, int l, int32_t *agg, double *M, double *B, double *d)
{
    const orc_level *L = &H->lv[l];
    int64_t n = L->A->nrows;
    if (agg && L->agg) memcpy(agg, L->agg, sizeof(int32_t) * (size_t)(n / L->b));
    if (M && L->M) memcpy(M, L->M, sizeof(double) * (size_t)n);
    if (B && L->B) memcpy(B, L->B, sizeof(double) * (size_t)(n * H->ns));
    if (d && L->d) memcpy(d, L->d, sizeof(double) * (size_t)n);
}

/* The block smoother of level l (n / b blocks of b x b, row-major); returns
 * 0, or -1 when the level has none. */
int orc_level_blocks(const orc_hier *H, int l, double *Mb)
{
    const orc_level *L = &H->lv[l];
    if (!L->Mb) return -1;
    memcpy(Mb, L->Mb, sizeof(double) * (size_t)(L->A->nrows * L->b));
    return 0;
}

void orc_coarse_factor(const orc_hier *H, double *L, uint8_t *zrow)
{
    memcpy(L, H->L, sizeof(double) * (size_t)(H->nc * H->nc));
    memcpy(zrow, H->zrow, (size_t)H->nc);
}
