/*
 * fe_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the
 * batched finite-element cell kernels and global assembly of
 * "Mixed-precision finite element kernels and assembly: rounding error
 * analysis and hardware acceleration" (Croci & Wells).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library may include, link or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code with the CUDA path.
 *
 * Every routine is the textbook definition written out with loops in double
 * precision, no blocking, no tensor decomposition, no reuse of intermediate
 * products beyond what the definition names:
 *
 *   geometry            Sec. 4.2, Eqs. for J, det J, J^{-1}, G (affine map);
 *                       det and inverse by LU with partial pivoting, the
 *                       algorithm the paper's analysis assumes (Sec. 2, LU
 *                       determinant / inverse bounds).
 *   element matrices    Sec. 3.1: mass a(w,v)=int z w v, Poisson
 *                       a(w,v)=int z grad w . grad v, mapped to the reference
 *                       cell and integrated by the quadrature rule; the
 *                       coefficient z is given at the quadrature points.
 *   global assembly     Sec. 3.3, Eq. (global assembly) A^g = L D L^T: each
 *                       element entry is added to its global entry, cells in
 *                       increasing order.
 *   dof map / pattern   continuous Lagrange local-to-global map L (Sec. 3.3)
 *                       under a canonical numbering (vertex dofs take the
 *                       vertex id; other nodes are numbered by their sorted
 *                       key); the paper does not fix a numbering.
 *   condition number    kappa_q^A of Corollary 4.10 (Sec. 4.4).
 *   adjoint             gradient of L = v^T A^g u with respect to kappa at the
 *                       quadrature points and to the vertex coordinates
 *                       (calculus; not in the paper).
 *
 * Parity status: every function here is pinned by the tests in
 * tests/test_oracle_*.py (closed forms, invariants, brute force).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FO_OK 0
#define FO_ERR_DEGENERATE -3
#define FO_ERR_ARG -1
#define FO_ERR_OOM -5

/* ------------------------------------------------------------------------ */
/* Small dense linear algebra: LU with partial pivoting (row interchanges).  */
/* ------------------------------------------------------------------------ */

/* Factor the d x d row-major matrix M in place: P M = L U.  perm receives the
 * row permutation, *sign the permutation parity.  Returns 0 or -1 if a zero
 * pivot is met (singular matrix). */
static int lu_factor(int d, double *M, int *perm, int *sign) {
    *sign = 1;
    for (int i = 0; i < d; ++i) perm[i] = i;
    for (int k = 0; k < d; ++k) {
        int piv = k;
        double best = fabs(M[k * d + k]);
        for (int i = k + 1; i < d; ++i) {
            if (fabs(M[i * d + k]) > best) { best = fabs(M[i * d + k]); piv = i; }
        }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < d; ++j) {
                double t = M[k * d + j]; M[k * d + j] = M[piv * d + j]; M[piv * d + j] = t;
            }
            int t = perm[k]; perm[k] = perm[piv]; perm[piv] = t;
            *sign = -*sign;
        }
        for (int i = k + 1; i < d; ++i) {
            double l = M[i * d + k] / M[k * d + k];
            M[i * d + k] = l;
            for (int j = k + 1; j < d; ++j) M[i * d + j] -= l * M[k * d + j];
        }
    }
    return 0;
}

/* Solve (P M) x = P b with the LU factors: forward then back substitution. */
static void lu_solve(int d, const double *LU, const int *perm, const double *b, double *x) {
    double y[3];
    for (int i = 0; i < d; ++i) {
        double s = b[perm[i]];
        for (int j = 0; j < i; ++j) s -= LU[i * d + j] * y[j];
        y[i] = s;
    }
    for (int i = d - 1; i >= 0; --i) {
        double s = y[i];
        for (int j = i + 1; j < d; ++j) s -= LU[i * d + j] * x[j];
        x[i] = s / LU[i * d + i];
    }
}

/* Affine simplex geometry.  xv: the d+1 vertex coordinates, [(d+1)][d].
 * J_ij = sum_k x_i^k d_j psi_k with the P1 reference basis psi, i.e. column
 * j of J is x^(j+1) - x^(0) (Sec. 4.2, Jacobian definition).  Outputs J,
 * det J (LU product of pivots times permutation sign) and J^{-1} (column by
 * column from LU solves).  Returns FO_ERR_DEGENERATE if J is singular. */
int fo_geometry(int d, const double *xv, double *J, double *detJ, double *Jinv) {
    if (d != 2 && d != 3) return FO_ERR_ARG;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j)
            J[i * d + j] = xv[(j + 1) * d + i] - xv[0 * d + i];
    double LU[9];
    int perm[3], sign;
    memcpy(LU, J, sizeof(double) * d * d);
    if (lu_factor(d, LU, perm, &sign) != 0) { *detJ = 0.0; return FO_ERR_DEGENERATE; }
    double det = (double)sign;
    for (int i = 0; i < d; ++i) det *= LU[i * d + i];
    *detJ = det;
    for (int j = 0; j < d; ++j) {
        double e[3] = {0, 0, 0}, col[3];
        e[j] = 1.0;
        lu_solve(d, LU, perm, e, col);
        for (int i = 0; i < d; ++i) Jinv[i * d + j] = col[i];
    }
    return FO_OK;
}

/* Poisson geometry tensor G = |det J| J^{-1} J^{-T} (Sec. 3.1).  Row-major d x d. */
static void geometry_tensor(int d, const double *Jinv, double absdet, double *G) {
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += Jinv[i * d + k] * Jinv[j * d + k];
            G[i * d + j] = absdet * s;
        }
}

static void gather_cell(int d, const int32_t *cells, const double *vertices, int64_t c, double *xv) {
    for (int k = 0; k <= d; ++k) {
        int64_t v = cells[c * (d + 1) + k];
        for (int i = 0; i < d; ++i) xv[k * d + i] = vertices[v * d + i];
    }
}

/* Per-cell geometry for a whole mesh: detJ[c], G[c][d][d]. */
int fo_mesh_geometry(int d, int64_t n_cells, const int32_t *cells, const double *vertices,
                     double *detJ, double *G) {
    for (int64_t c = 0; c < n_cells; ++c) {
        double xv[12], J[9], Jinv[9], det;
        gather_cell(d, cells, vertices, c, xv);
        int st = fo_geometry(d, xv, J, &det, Jinv);
        if (st != FO_OK) return st;
        detJ[c] = det;
        if (G) geometry_tensor(d, Jinv, fabs(det), G + c * d * d);
    }
    return FO_OK;
}

/* ------------------------------------------------------------------------ */
/* Element matrices (Sec. 3.1).                                              */
/* ------------------------------------------------------------------------ */
/* Tabulation inputs (computed by the oracle's Python side in FP64):
 *   phi  [n_phi][n_q]      phi_k(X_q)
 *   dphi [d][n_phi][n_q]   d phi_k / d X_s at X_q
 * form 1 = mass:      A[k][l] = sum_q w_q kappa_cq |det J| phi_k phi_l
 * form 2 = stiffness: A[k][l] = sum_q w_q kappa_cq |det J| (J^{-T} grad phi_k).(J^{-T} grad phi_l)
 * The physical gradient is formed explicitly, (J^{-T} g)_i = sum_s Jinv[s][i] g_s,
 * which is the definition before the paper's rearrangement into G.
 * Cells [c0, c1) are computed; A is indexed by the absolute cell id.       */
int fo_element_matrices(int d, int64_t c0, int64_t c1, const int32_t *cells, const double *vertices,
                        int n_phi, int n_q, const double *w, const double *phi, const double *dphi,
                        const double *kappa, int form, double *A) {
    if (form != 1 && form != 2) return FO_ERR_ARG;
    double *grad = NULL;
    if (form == 2) {
        grad = (double *)malloc(sizeof(double) * (size_t)n_phi * n_q * d);
        if (!grad) return FO_ERR_OOM;
    }
    for (int64_t c = c0; c < c1; ++c) {
        double xv[12], J[9], Jinv[9], det;
        gather_cell(d, cells, vertices, c, xv);
        int st = fo_geometry(d, xv, J, &det, Jinv);
        if (st != FO_OK) { free(grad); return st; }
        double absdet = fabs(det);
        double *Ac = A + c * (int64_t)n_phi * n_phi;
        if (form == 2) {
            for (int k = 0; k < n_phi; ++k)
                for (int q = 0; q < n_q; ++q)
                    for (int i = 0; i < d; ++i) {
                        double s = 0.0;
                        for (int r = 0; r < d; ++r) s += Jinv[r * d + i] * dphi[((int64_t)r * n_phi + k) * n_q + q];
                        grad[((int64_t)k * n_q + q) * d + i] = s;
                    }
        }
        for (int k = 0; k < n_phi; ++k)
            for (int l = 0; l < n_phi; ++l) {
                double s = 0.0;
                for (int q = 0; q < n_q; ++q) {
                    double f = w[q] * kappa[c * n_q + q] * absdet;
                    double integrand;
                    if (form == 1) {
                        integrand = phi[(int64_t)k * n_q + q] * phi[(int64_t)l * n_q + q];
                    } else {
                        integrand = 0.0;
                        for (int i = 0; i < d; ++i)
                            integrand += grad[((int64_t)k * n_q + q) * d + i] * grad[((int64_t)l * n_q + q) * d + i];
                    }
                    s += f * integrand;
                }
                Ac[(int64_t)k * n_phi + l] = s;
            }
    }
    free(grad);
    return FO_OK;
}

/* kappa_q^A of Corollary 4.10 for cells [c0, c1):
 *   || sum_{s,t} |B_s| |C_st| |B_t|^T ||_max / || A ||_max
 * with C_st = diag_q(w_q kappa_cq G_st) (Poisson) or diag_q(w_q kappa_cq |det J|)
 * (mass) and B_s = dphi[s] (Poisson) or phi (mass).  A is the exact element
 * matrix of the same cell (computed above), passed in. */
int fo_kappa_q(int d, int64_t c0, int64_t c1, const int32_t *cells, const double *vertices,
               int n_phi, int n_q, const double *w, const double *phi, const double *dphi,
               const double *kappa, int form, const double *A, double *kq) {
    for (int64_t c = c0; c < c1; ++c) {
        double xv[12], J[9], Jinv[9], det, G[9];
        gather_cell(d, cells, vertices, c, xv);
        int st = fo_geometry(d, xv, J, &det, Jinv);
        if (st != FO_OK) return st;
        double absdet = fabs(det);
        geometry_tensor(d, Jinv, absdet, G);
        int nd = (form == 2) ? d : 1;
        double num = 0.0, den = 0.0;
        const double *Ac = A + c * (int64_t)n_phi * n_phi;
        for (int k = 0; k < n_phi; ++k)
            for (int l = 0; l < n_phi; ++l) {
                double s = 0.0;
                for (int a = 0; a < nd; ++a)
                    for (int b = 0; b < nd; ++b)
                        for (int q = 0; q < n_q; ++q) {
                            double g = (form == 2) ? G[a * d + b] : absdet;
                            double cq = fabs(w[q] * kappa[c * n_q + q] * g);
                            double bk = (form == 2) ? dphi[((int64_t)a * n_phi + k) * n_q + q] : phi[(int64_t)k * n_q + q];
                            double bl = (form == 2) ? dphi[((int64_t)b * n_phi + l) * n_q + q] : phi[(int64_t)l * n_q + q];
                            s += fabs(bk) * cq * fabs(bl);
                        }
                if (s > num) num = s;
                if (fabs(Ac[(int64_t)k * n_phi + l]) > den) den = fabs(Ac[(int64_t)k * n_phi + l]);
            }
        kq[c] = (den > 0.0) ? num / den : INFINITY;
    }
    return FO_OK;
}

/* ------------------------------------------------------------------------ */
/* Canonical continuous-Lagrange dof map.                                    */
/* ------------------------------------------------------------------------ */
/* nodes: [n_phi][d+1] barycentric multi-indices a (|a| = p) of the local
 * nodes in local order.  A node a of cell c with vertex ids g_i has the key
 * {(g_i, a_i) : a_i > 0} sorted by g.  Vertex nodes (one nonzero a_i) take
 * the global vertex id.  The other keys are sorted by (support size, sorted
 * vertex ids, multiplicities in that order) and numbered from n_vertices. */
typedef struct {
    int32_t size;
    int32_t g[4];
    int32_t a[4];
    int64_t slot; /* c * n_phi + k */
} node_key;

static int key_cmp(const void *pa, const void *pb) {
    const node_key *x = (const node_key *)pa, *y = (const node_key *)pb;
    if (x->size != y->size) return x->size < y->size ? -1 : 1;
    for (int i = 0; i < x->size; ++i)
        if (x->g[i] != y->g[i]) return x->g[i] < y->g[i] ? -1 : 1;
    for (int i = 0; i < x->size; ++i)
        if (x->a[i] != y->a[i]) return x->a[i] < y->a[i] ? -1 : 1;
    if (x->slot != y->slot) return x->slot < y->slot ? -1 : 1;
    return 0;
}

static int key_same(const node_key *x, const node_key *y) {
    if (x->size != y->size) return 0;
    for (int i = 0; i < x->size; ++i)
        if (x->g[i] != y->g[i] || x->a[i] != y->a[i]) return 0;
    return 1;
}

int fo_dofmap(int d, int n_phi, const int32_t *nodes, int64_t n_vertices, int64_t n_cells,
              const int32_t *cells, int32_t *cell_dofs, int64_t *n_dofs) {
    int64_t n_other = 0;
    for (int k = 0; k < n_phi; ++k) {
        int nz = 0;
        for (int i = 0; i <= d; ++i) nz += nodes[k * (d + 1) + i] > 0;
        if (nz > 1) n_other++;
    }
    node_key *keys = NULL;
    if (n_other > 0) {
        keys = (node_key *)malloc(sizeof(node_key) * (size_t)(n_other * n_cells));
        if (!keys) return FO_ERR_OOM;
    }
    int64_t m = 0;
    for (int64_t c = 0; c < n_cells; ++c) {
        for (int k = 0; k < n_phi; ++k) {
            const int32_t *a = nodes + k * (d + 1);
            int nz = 0, which = -1;
            for (int i = 0; i <= d; ++i)
                if (a[i] > 0) { nz++; which = i; }
            if (nz == 1) {
                cell_dofs[c * n_phi + k] = cells[c * (d + 1) + which];
                continue;
            }
            node_key key;
            key.size = 0;
            for (int i = 0; i <= d; ++i)
                if (a[i] > 0) {
                    key.g[key.size] = cells[c * (d + 1) + i];
                    key.a[key.size] = a[i];
                    key.size++;
                }
            /* sort the (g, a) pairs by g: insertion sort on <= 4 entries */
            for (int i = 1; i < key.size; ++i)
                for (int j = i; j > 0 && key.g[j - 1] > key.g[j]; --j) {
                    int32_t tg = key.g[j]; key.g[j] = key.g[j - 1]; key.g[j - 1] = tg;
                    int32_t ta = key.a[j]; key.a[j] = key.a[j - 1]; key.a[j - 1] = ta;
                }
            for (int i = key.size; i < 4; ++i) { key.g[i] = -1; key.a[i] = 0; }
            key.slot = c * n_phi + k;
            keys[m++] = key;
        }
    }
    qsort(keys, (size_t)m, sizeof(node_key), key_cmp);
    int64_t next = n_vertices;
    for (int64_t i = 0; i < m; ++i) {
        if (i > 0 && !key_same(&keys[i], &keys[i - 1])) next++;
        cell_dofs[keys[i].slot] = (int32_t)next;
    }
    *n_dofs = (m > 0) ? next + 1 : n_vertices;
    free(keys);
    return FO_OK;
}

/* ------------------------------------------------------------------------ */
/* CSR sparsity pattern and assembly (Sec. 3.3, A^g = L D L^T).              */
/* ------------------------------------------------------------------------ */
static int int_cmp(const void *pa, const void *pb) {
    int32_t x = *(const int32_t *)pa, y = *(const int32_t *)pb;
    return (x > y) - (x < y);
}

/* Build, for every global dof, the list of cells that contain it. */
static int build_incidence(int64_t n_dofs, int64_t n_cells, int n_phi, const int32_t *cell_dofs,
                           int64_t **ptr_out, int64_t **cell_out) {
    int64_t *ptr = (int64_t *)calloc((size_t)n_dofs + 1, sizeof(int64_t));
    int64_t *lst = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cells * n_phi + 1));
    if (!ptr || !lst) { free(ptr); free(lst); return FO_ERR_OOM; }
    for (int64_t i = 0; i < n_cells * n_phi; ++i) ptr[cell_dofs[i] + 1]++;
    for (int64_t i = 0; i < n_dofs; ++i) ptr[i + 1] += ptr[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_dofs + 1));
    if (!fill) { free(ptr); free(lst); return FO_ERR_OOM; }
    memcpy(fill, ptr, sizeof(int64_t) * (size_t)(n_dofs + 1));
    for (int64_t c = 0; c < n_cells; ++c)
        for (int k = 0; k < n_phi; ++k) lst[fill[cell_dofs[c * n_phi + k]]++] = c;
    free(fill);
    *ptr_out = ptr;
    *cell_out = lst;
    return FO_OK;
}

/* Row i of the pattern = sorted set of dofs of all cells containing dof i.
 * If col_idx is NULL only row_ptr (n_dofs+1 entries) is filled. */
int fo_csr_pattern(int64_t n_dofs, int64_t n_cells, int n_phi, const int32_t *cell_dofs,
                   int64_t *row_ptr, int32_t *col_idx) {
    int64_t *iptr, *icell;
    int st = build_incidence(n_dofs, n_cells, n_phi, cell_dofs, &iptr, &icell);
    if (st != FO_OK) return st;
    int64_t maxc = 0;
    for (int64_t i = 0; i < n_dofs; ++i)
        if (iptr[i + 1] - iptr[i] > maxc) maxc = iptr[i + 1] - iptr[i];
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxc * n_phi + 1));
    if (!buf) { free(iptr); free(icell); return FO_ERR_OOM; }
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n_dofs; ++i) {
        int64_t m = 0;
        for (int64_t e = iptr[i]; e < iptr[i + 1]; ++e) {
            int64_t c = icell[e];
            for (int l = 0; l < n_phi; ++l) buf[m++] = cell_dofs[c * n_phi + l];
        }
        qsort(buf, (size_t)m, sizeof(int32_t), int_cmp);
        int64_t u = 0;
        for (int64_t j = 0; j < m; ++j)
            if (j == 0 || buf[j] != buf[j - 1]) buf[u++] = buf[j];
        if (col_idx) memcpy(col_idx + row_ptr[i], buf, sizeof(int32_t) * (size_t)u);
        row_ptr[i + 1] = row_ptr[i] + u;
    }
    free(buf);
    free(iptr);
    free(icell);
    return FO_OK;
}

static int64_t find_col(const int64_t *row_ptr, const int32_t *col_idx, int64_t row, int32_t col) {
    int64_t lo = row_ptr[row], hi = row_ptr[row + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col_idx[mid] == col) return mid;
        if (col_idx[mid] < col) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* values[nnz] = sum over cells (increasing c) of A[c][k][l] into
 * (cell_dofs[c][k], cell_dofs[c][l]).  If absval != 0 the absolute values
 * |A| are assembled instead (used for the bound L |D| L^T). */
int fo_assemble(int64_t n_cells, int n_phi, const int32_t *cell_dofs, const double *A,
                const int64_t *row_ptr, const int32_t *col_idx, int64_t nnz, int absval, double *values) {
    for (int64_t j = 0; j < nnz; ++j) values[j] = 0.0;
    for (int64_t c = 0; c < n_cells; ++c)
        for (int k = 0; k < n_phi; ++k)
            for (int l = 0; l < n_phi; ++l) {
                int64_t pos = find_col(row_ptr, col_idx, cell_dofs[c * n_phi + k], cell_dofs[c * n_phi + l]);
                if (pos < 0) return FO_ERR_ARG;
                double a = A[(c * n_phi + k) * (int64_t)n_phi + l];
                values[pos] += absval ? fabs(a) : a;
            }
    return FO_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of L = v^T A^g u for the Poisson form (calculus, not in the paper) */
/* ------------------------------------------------------------------------ */
/* With the reference gradients gu_q = sum_l dphi[:, l, q] u_{dof(c,l)} and
 * gv_q likewise, and K = J^{-1}:
 *   L_c = sum_q w_q kappa_cq |det J| (K^T gv_q) . (K^T gu_q)
 *   dL/dkappa_cq = w_q |det J| (K^T gv_q) . (K^T gu_q)
 *   with S = sum_q w_q kappa_cq gu_q gv_q^T:
 *   dL_c/dJ = |det J| [ tr(K K^T S) K^T - K^T S^T K K^T - K^T S K K^T ]
 *   dL/dx^(j) = column j-1 of dL_c/dJ for j >= 1, and minus their sum for j = 0,
 *   summed into the global vertices.  kappa at the quadrature points is held
 *   fixed when the vertices move.
 * g_kappa [n_cells][n_q] and g_vertices [n_vertices][d] may be NULL. L_out
 * receives L. */
int fo_adjoint_stiffness(int d, int64_t n_cells, const int32_t *cells, const double *vertices, int64_t n_vertices,
                         int n_phi, int n_q, const double *w, const double *dphi, const double *kappa,
                         const int32_t *cell_dofs, const double *u, const double *v,
                         double *g_kappa, double *g_vertices, double *L_out) {
    if (g_vertices)
        for (int64_t i = 0; i < n_vertices * d; ++i) g_vertices[i] = 0.0;
    double L = 0.0;
    for (int64_t c = 0; c < n_cells; ++c) {
        double xv[12], J[9], K[9], det;
        gather_cell(d, cells, vertices, c, xv);
        int st = fo_geometry(d, xv, J, &det, K);
        if (st != FO_OK) return st;
        double absdet = fabs(det);
        double S[9] = {0};
        for (int q = 0; q < n_q; ++q) {
            double gu[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
            for (int s = 0; s < d; ++s)
                for (int l = 0; l < n_phi; ++l) {
                    double b = dphi[((int64_t)s * n_phi + l) * n_q + q];
                    gu[s] += b * u[cell_dofs[c * n_phi + l]];
                    gv[s] += b * v[cell_dofs[c * n_phi + l]];
                }
            /* physical gradients K^T g */
            double pu[3] = {0, 0, 0}, pv[3] = {0, 0, 0};
            for (int i = 0; i < d; ++i)
                for (int r = 0; r < d; ++r) {
                    pu[i] += K[r * d + i] * gu[r];
                    pv[i] += K[r * d + i] * gv[r];
                }
            double dot = 0.0;
            for (int i = 0; i < d; ++i) dot += pu[i] * pv[i];
            double wk = w[q] * kappa[c * n_q + q];
            if (g_kappa) g_kappa[c * n_q + q] = w[q] * absdet * dot;
            L += wk * absdet * dot;
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) S[i * d + j] += wk * gu[i] * gv[j];
        }
        if (!g_vertices) continue;
        double KKt[9], tr = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double s = 0.0;
                for (int k = 0; k < d; ++k) s += K[i * d + k] * K[j * d + k];
                KKt[i * d + j] = s;
            }
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) tr += KKt[i * d + j] * S[j * d + i];
        /* T1 = K^T S^T K K^T, T2 = K^T S K K^T */
        double dJ[9];
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double t1 = 0.0, t2 = 0.0;
                for (int a = 0; a < d; ++a)
                    for (int b = 0; b < d; ++b) {
                        t1 += K[a * d + i] * S[b * d + a] * KKt[b * d + j];
                        t2 += K[a * d + i] * S[a * d + b] * KKt[b * d + j];
                    }
                dJ[i * d + j] = absdet * (tr * K[j * d + i] - t1 - t2);
            }
        for (int j = 1; j <= d; ++j) {
            int64_t vj = cells[c * (d + 1) + j];
            int64_t v0 = cells[c * (d + 1) + 0];
            for (int i = 0; i < d; ++i) {
                g_vertices[vj * d + i] += dJ[i * d + (j - 1)];
                g_vertices[v0 * d + i] -= dJ[i * d + (j - 1)];
            }
        }
    }
    if (L_out) *L_out = L;
    return FO_OK;
}

/* ------------------------------------------------------------------------ */
/* Boxed cells (quadrilaterals, hexahedra; Sec. 3.1 and the lemma on the     */
/* Jacobian in Sec. 4.2): the reference cell is [0,1]^d, the map is the      */
/* multilinear Q1 map x(X) = sum_v x_v psi_v(X) over the 2^d vertices, so    */
/* J(X) = sum_v x_v grad psi_v(X)^T varies with X and the geometry is        */
/* formed at every quadrature point.                                         */
/* ------------------------------------------------------------------------ */

/* J at quadrature point q of cell c: J_ij = sum_v x_{v,i} dpsi[j][v][q]. */
static void box_jacobian(int d, int nv, const int32_t *cells, const double *vertices, int64_t c,
                         const double *dpsi, int n_q, int q, double *J) {
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int v = 0; v < nv; ++v)
                s += vertices[(int64_t)cells[c * nv + v] * d + i] * dpsi[((int64_t)j * nv + v) * n_q + q];
            J[i * d + j] = s;
        }
}

/* J^{-1} and det J of the d x d matrix J by LU with partial pivoting. */
static int lu_geometry(int d, const double *J, double *det, double *Jinv) {
    double M[9];
    int perm[3], sign;
    memcpy(M, J, sizeof(double) * d * d);
    if (lu_factor(d, M, perm, &sign) != 0) return FO_ERR_DEGENERATE;
    double dt = sign;
    for (int i = 0; i < d; ++i) dt *= M[i * d + i];
    *det = dt;
    for (int col = 0; col < d; ++col) {
        double e[3] = {0, 0, 0}, x[3];
        e[col] = 1.0;
        lu_solve(d, M, perm, e, x);
        for (int i = 0; i < d; ++i) Jinv[i * d + col] = x[i];
    }
    return FO_OK;
}

/* Element matrices of boxed cells [c0, c1): the literal quadrature sum of
 * Sec. 3.1 with the geometry of every point:
 *   mass       A_kl = sum_q w_q kappa_cq |det J_q| phi_k phi_l
 *   stiffness  A_kl = sum_q w_q kappa_cq |det J_q| (J_q^-T grad phi_k).(J_q^-T grad phi_l). */
int fo_element_matrices_box(int d, int64_t c0, int64_t c1, const int32_t *cells, const double *vertices,
                            int n_phi, int n_q, const double *w, const double *phi, const double *dphi,
                            const double *dpsi, const double *kappa, int form, double *A) {
    const int nv = 1 << d;
    double *grad = (double *)malloc(sizeof(double) * (size_t)n_phi * d);
    if (!grad) return FO_ERR_OOM;
    for (int64_t c = c0; c < c1; ++c) {
        double *Ac = A + c * (int64_t)n_phi * n_phi;
        for (int64_t i = 0; i < (int64_t)n_phi * n_phi; ++i) Ac[i] = 0.0;
        for (int q = 0; q < n_q; ++q) {
            double J[9], Jinv[9], det;
            box_jacobian(d, nv, cells, vertices, c, dpsi, n_q, q, J);
            if (lu_geometry(d, J, &det, Jinv) != FO_OK) { free(grad); return FO_ERR_DEGENERATE; }
            const double f = w[q] * kappa[c * n_q + q] * fabs(det);
            if (form == 2)
                for (int k = 0; k < n_phi; ++k)
                    for (int i = 0; i < d; ++i) {
                        double s = 0.0;
                        for (int r = 0; r < d; ++r) s += Jinv[r * d + i] * dphi[((int64_t)r * n_phi + k) * n_q + q];
                        grad[k * d + i] = s;
                    }
            for (int k = 0; k < n_phi; ++k)
                for (int l = 0; l < n_phi; ++l) {
                    double integrand;
                    if (form == 1) {
                        integrand = phi[(int64_t)k * n_q + q] * phi[(int64_t)l * n_q + q];
                    } else {
                        integrand = 0.0;
                        for (int i = 0; i < d; ++i) integrand += grad[k * d + i] * grad[l * d + i];
                    }
                    Ac[(int64_t)k * n_phi + l] += f * integrand;
                }
        }
    }
    free(grad);
    return FO_OK;
}

/* kappa_q^A of Corollary 4.10 for boxed cells [c0, c1): C_st = diag_q(w_q
 * kappa_cq G_st(X_q)) with G(X_q) = |det J_q| J_q^-1 J_q^-T (mass: w_q
 * kappa_cq |det J_q|); A: the exact element matrices of the same cells. */
int fo_kappa_q_box(int d, int64_t c0, int64_t c1, const int32_t *cells, const double *vertices, int n_phi,
                   int n_q, const double *w, const double *phi, const double *dphi, const double *dpsi,
                   const double *kappa, int form, const double *A, double *kq) {
    const int nv = 1 << d;
    const int nd = (form == 2) ? d : 1;
    double *Cq = (double *)malloc(sizeof(double) * (size_t)n_q * 9);
    if (!Cq) return FO_ERR_OOM;
    for (int64_t c = c0; c < c1; ++c) {
        for (int q = 0; q < n_q; ++q) {
            double J[9], Jinv[9], det, G[9];
            box_jacobian(d, nv, cells, vertices, c, dpsi, n_q, q, J);
            if (lu_geometry(d, J, &det, Jinv) != FO_OK) { free(Cq); return FO_ERR_DEGENERATE; }
            geometry_tensor(d, Jinv, fabs(det), G);
            for (int a = 0; a < nd; ++a)
                for (int b = 0; b < nd; ++b)
                    Cq[(int64_t)q * 9 + a * nd + b] = fabs(w[q] * kappa[c * n_q + q] * ((form == 2) ? G[a * d + b] : fabs(det)));
        }
        double num = 0.0, den = 0.0;
        const double *Ac = A + c * (int64_t)n_phi * n_phi;
        for (int k = 0; k < n_phi; ++k)
            for (int l = 0; l < n_phi; ++l) {
                double s = 0.0;
                for (int a = 0; a < nd; ++a)
                    for (int b = 0; b < nd; ++b)
                        for (int q = 0; q < n_q; ++q) {
                            double bk = (form == 2) ? dphi[((int64_t)a * n_phi + k) * n_q + q] : phi[(int64_t)k * n_q + q];
                            double bl = (form == 2) ? dphi[((int64_t)b * n_phi + l) * n_q + q] : phi[(int64_t)l * n_q + q];
                            s += fabs(bk) * Cq[(int64_t)q * 9 + a * nd + b] * fabs(bl);
                        }
                if (s > num) num = s;
                if (fabs(Ac[(int64_t)k * n_phi + l]) > den) den = fabs(Ac[(int64_t)k * n_phi + l]);
            }
        kq[c] = (den > 0.0) ? num / den : INFINITY;
    }
    free(Cq);
    return FO_OK;
}

/* Canonical dof map from node weights: node k of a cell carries the integer
 * weights node_w[k][v] >= 0 over the cell's nv vertices (the multilinear, or
 * barycentric, coordinates of the node times p^d, resp. p).  Its key is the
 * multiset {(g_v, node_w[k][v]) : node_w[k][v] > 0} sorted by global vertex
 * id g_v; a node with one nonzero weight is that vertex's dof; all other keys
 * are sorted by (support size, vertex ids, weights in that order) and numbered
 * from n_vertices.  For simplices with the barycentric multiplicities this is
 * the numbering of fo_dofmap. */
typedef struct {
    int32_t size;
    int32_t g[8];
    int32_t a[8];
    int64_t slot;
} node_key8;

static int key8_cmp(const void *pa, const void *pb) {
    const node_key8 *x = (const node_key8 *)pa, *y = (const node_key8 *)pb;
    if (x->size != y->size) return x->size < y->size ? -1 : 1;
    for (int i = 0; i < x->size; ++i)
        if (x->g[i] != y->g[i]) return x->g[i] < y->g[i] ? -1 : 1;
    for (int i = 0; i < x->size; ++i)
        if (x->a[i] != y->a[i]) return x->a[i] < y->a[i] ? -1 : 1;
    if (x->slot != y->slot) return x->slot < y->slot ? -1 : 1;
    return 0;
}

int fo_dofmap_weights(int nv, int n_phi, const int32_t *node_w, int64_t n_vertices, int64_t n_cells,
                      const int32_t *cells, int32_t *cell_dofs, int64_t *n_dofs) {
    if (nv > 8) return FO_ERR_ARG;
    node_key8 *keys = (node_key8 *)malloc(sizeof(node_key8) * (size_t)(n_phi * n_cells + 1));
    if (!keys) return FO_ERR_OOM;
    int64_t m = 0;
    for (int64_t c = 0; c < n_cells; ++c)
        for (int k = 0; k < n_phi; ++k) {
            const int32_t *a = node_w + k * nv;
            node_key8 key;
            key.size = 0;
            for (int v = 0; v < nv; ++v)
                if (a[v] > 0) {
                    key.g[key.size] = cells[c * nv + v];
                    key.a[key.size] = a[v];
                    key.size++;
                }
            if (key.size == 1) {
                cell_dofs[c * n_phi + k] = key.g[0];
                continue;
            }
            for (int i = 1; i < key.size; ++i)
                for (int j = i; j > 0 && key.g[j - 1] > key.g[j]; --j) {
                    int32_t tg = key.g[j]; key.g[j] = key.g[j - 1]; key.g[j - 1] = tg;
                    int32_t ta = key.a[j]; key.a[j] = key.a[j - 1]; key.a[j - 1] = ta;
                }
            for (int i = key.size; i < 8; ++i) { key.g[i] = -1; key.a[i] = 0; }
            key.slot = c * n_phi + k;
            keys[m++] = key;
        }
    qsort(keys, (size_t)m, sizeof(node_key8), key8_cmp);
    int64_t next = n_vertices;
    for (int64_t i = 0; i < m; ++i) {
        if (i > 0) {
            const node_key8 *x = &keys[i], *y = &keys[i - 1];
            int same = x->size == y->size;
            for (int j = 0; same && j < x->size; ++j) same = x->g[j] == y->g[j] && x->a[j] == y->a[j];
            if (!same) next++;
        }
        cell_dofs[keys[i].slot] = (int32_t)next;
    }
    *n_dofs = (m > 0) ? next + 1 : n_vertices;
    free(keys);
    return FO_OK;
}
