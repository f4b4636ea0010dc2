/*
 * fe_gb300.h -- C ABI of the GB300 (sm_103a) library for batched
 * finite-element cell kernels and global assembly, after Croci & Wells,
 * "Mixed-precision finite element kernels and assembly: rounding error
 * analysis and hardware acceleration".
 *
 * The library computes, for a mesh of affine simplices (triangles or
 * tetrahedra) and continuous degree-p Lagrange elements:
 *   - per-cell geometry J, det J, J^{-1} and G = |det J| J^{-1} J^{-T}
 *     (Sec. 4.2) in FP64,
 *   - the factors C_st = diag_q(w_q kappa_cq G_st) (Sec. 3.1, Eq. for C_st)
 *     with the coefficient kappa given at the quadrature points,
 *   - element matrices A^c = sum_{s,t} B_s C_st B_t^T (Sec. 3.1, triple
 *     products; Algorithm 1) for the mass and Poisson (stiffness) forms, as
 *     one dense contraction per tile of cells on the tensor cores (BF16,
 *     FP16, TF32, split TF32 or FP8 e4m3 operands, FP32 accumulation) or on
 *     the FP64 units,
 *   - global assembly A^g = L D L^T (Sec. 3.3, Eq. global assembly) into a
 *     CSR matrix by a deterministic segmented reduction,
 *   - the adjoint of L = v^T A^g u with respect to kappa at the quadrature
 *     points and to the vertex coordinates (not in the paper).
 *
 * Conventions
 *   - Every function returns an fe_status.  On failure a thread-local
 *     message is available from fe_last_error().
 *   - Pointers marked "device" must be CUDA device (or managed) memory on the
 *     current device; pointers marked "host" are ordinary host memory.  The
 *     caller owns every buffer it passes; the library never frees them and
 *     never keeps them after the call returns.
 *   - Compute calls are asynchronous on the plan's CUDA stream.  Errors that
 *     kernels detect (degenerate or non-finite cells, exhausted bounded
 *     waits) are recorded in a device status word and reported by
 *     fe_sync_status() or by the next synchronous call.
 *   - Element matrices are stored row-major per cell, [n_cells][n_phi][n_phi],
 *     A[c][k][l] = a(phi_l, phi_k) on cell c (Sec. 3.1, A_ji = a(phi_i, phi_j)),
 *     in double for FE_PREC_FP64 and in float otherwise.
 *   - Local node order: barycentric lattice multi-indices a (|a| = p) sorted
 *     by support size, then by the support's vertex tuple, then by a in
 *     descending lexicographic order (vertices, edges 01,02,03,12,13,23,
 *     faces, interior).  Reference cells: (0,0),(1,0),(0,1) and the
 *     tetrahedron (0,0,0),(1,0,0),(0,1,0),(0,0,1) (Sec. 5.1).
 *   - Global numbering (the paper fixes none): vertex dofs take the vertex
 *     id; every other node has the key {(g_i, a_i) : a_i > 0} sorted by the
 *     global vertex id g_i, and these keys are numbered from n_vertices in
 *     increasing (support size, vertex ids, multiplicities) order.
 */
#ifndef FE_GB300_H
#define FE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FE_OK = 0,
    FE_ERR_INVALID_ARG = -1,     /* null pointer, size or enum out of range  */
    FE_ERR_UNSUPPORTED = -2,     /* degree, cell type or size not supported  */
    FE_ERR_DEGENERATE_CELL = -3, /* det J == 0 on some cell                   */
    FE_ERR_NONFINITE = -4,       /* non-finite coordinate, coefficient or J   */
    FE_ERR_OOM = -5,             /* device or host allocation failed          */
    FE_ERR_CUDA = -6,            /* a CUDA runtime call failed                */
    FE_ERR_TIMEOUT = -7,         /* a bounded wait inside a kernel gave up    */
    FE_ERR_NO_DEVICE = -8        /* no CUDA device is visible                 */
} fe_status;

/* Cell types.  Simplices (Sec. 3.1, affine: J constant per cell) and boxed
 * cells (Sec. 3.1 boxed cells on the reference [0,1]^d, Sec. 5.1: the
 * multilinear Q1 map, so J, det J and G are formed at every quadrature
 * point).  A boxed cell lists its 2^d vertices in tensor order: vertex v is
 * the corner (bit_0(v), bit_1(v), bit_2(v)) of the reference cell.  Boxed
 * cells carry the Q_p Lagrange space on the equispaced lattice a/p,
 * a in {0..p}^d, node k = a_0 + (p+1)(a_1 + (p+1) a_2), n_phi = (p+1)^d. */
typedef enum { FE_TRIANGLE = 2, FE_TETRAHEDRON = 3, FE_QUADRILATERAL = 4, FE_HEXAHEDRON = 5 } fe_cell_type;

/* Forms (bitmask).  Sec. 3.1: mass a(w,v) = int z w v and Poisson
 * a(w,v) = int z grad w . grad v with coefficient z = kappa.
 * FE_PLAN_ELEMENTS_ONLY, or-ed into fe_plan_create's form mask, builds a plan
 * for element matrices only (the paper's kernel experiments, Sec. 5): no dof
 * map, CSR pattern or assembly streams, so plan creation stays cheap on large
 * high-degree meshes; calls that need them (assembly, actions, adjoints,
 * fe_csr_pattern, fe_cell_dofs) return FE_ERR_INVALID_ARG. */
enum { FE_FORM_MASS = 1, FE_FORM_STIFFNESS = 2, FE_PLAN_ELEMENTS_ONLY = 0x100 };

/* Contraction precisions (List 1: the storage precision u_s of C and of the
 * tabulated operand; products and accumulation are FP32 on the tensor cores,
 * geometry and tabulation FP64).  FE_PREC_FP64 runs the whole kernel in
 * FP64 on the CUDA cores.  FE_PREC_TF32X3 splits each operand into a TF32
 * head and tail and sums three TF32 products (u_s ~ 2^-21). */
typedef enum {
    FE_PREC_FP64 = 0,
    FE_PREC_TF32X3 = 1,
    FE_PREC_TF32 = 2,
    FE_PREC_BF16 = 3,
    FE_PREC_FP16 = 4,
    FE_PREC_E4M3 = 5
} fe_precision;
#define FE_PREC_MASK(p) (1u << (unsigned)(p))

/* Quadrature families for fe_quadrature_rule. */
enum {
    FE_QUAD_COLLAPSED_GAUSS_JACOBI = 0, /* simplices: m points per direction, exact to 2m-1 */
    FE_QUAD_TRIANGLE_3POINT = 1,        /* (1/6,1/6),(2/3,1/6),(1/6,2/3), w = 1/6 */
    FE_QUAD_GAUSS_LEGENDRE_TENSOR = 2   /* boxed cells: m^d Gauss-Legendre points on [0,1]^d,
                                           exact to degree 2m-1 in each variable, x fastest */
};

typedef struct fe_plan fe_plan;
typedef struct fe_pattern fe_pattern;

typedef struct {
    fe_cell_type type;
    int64_t n_vertices;
    const double *vertices; /* host, [n_vertices][d] */
    int64_t n_cells;
    const int32_t *cells;   /* host, [n_cells][d+1] (simplices) or [n_cells][2^d] (boxed cells), vertex ids */
} fe_mesh;

typedef struct {
    int32_t n_q;
    const double *points;   /* host, [n_q][d], reference-cell coordinates */
    const double *weights;  /* host, [n_q] */
} fe_quadrature;

/* ---------------------------------------------------------------------- */
/* Host helpers (no GPU needed)                                           */
/* ---------------------------------------------------------------------- */

/* Reference-cell quadrature rule (Sec. 3.1 assumes exact rules).
 * FE_QUAD_COLLAPSED_GAUSS_JACOBI: collapsed (Duffy) product of m-point
 * Gauss-Jacobi rules with weights (1-t)^0, (1-t)^1 (and (1-t)^2 on
 * tetrahedra), exact to degree 2m-1, n_q = m^d, point q = ia + m (ib + m ic)
 * with the 1-D nodes ascending; x = a(1-b)(1-c), y = b(1-c), z = c.
 * FE_QUAD_TRIANGLE_3POINT: the degree-2 interior rule (m ignored).
 * FE_QUAD_GAUSS_LEGENDRE_TENSOR (quadrilaterals, hexahedra): the tensor
 * product of m-point Gauss-Legendre rules on [0,1], point q = ia + m (ib +
 * m ic).  points/weights (host) may be NULL to query n_q only.  m in 1..32. */
fe_status fe_quadrature_rule(fe_cell_type type, int family, int m, int32_t *n_q, double *points,
                             double *weights);

/* Continuous Lagrange dof map and CSR pattern (Sec. 3.3, assembly matrix L).
 * cells: host [n_cells][vertices per cell].  degree 1..8 (tetrahedra), 1..10
 * (triangles), 1..5 (hexahedra), 1..8 (quadrilaterals).  The pattern of row i
 * is the sorted set of global dofs that share a cell with dof i; the diagonal
 * is always present.  Boxed cells: a node's key is its Q1 weights over the
 * cell's vertices, w_v = prod_i (bit_i(v) ? a_i : p - a_i), on the vertices
 * with w_v > 0 sorted by global id (simplices: the barycentric multiplicities);
 * vertex nodes take the vertex id, the other keys are numbered from
 * n_vertices in (support size, vertex ids, weights) order. */
fe_status fe_pattern_create(fe_pattern **out, fe_cell_type type, int64_t n_vertices, int64_t n_cells,
                            const int32_t *cells, int degree);
/* n_dofs, nnz, n_phi, and the longest row; any output pointer may be NULL. */
fe_status fe_pattern_sizes(const fe_pattern *pat, int64_t *n_dofs, int64_t *nnz, int32_t *n_phi,
                           int32_t *max_row);
/* Copies into host buffers: cell_dofs [n_cells][n_phi], row_ptr [n_dofs+1],
 * col_idx [nnz].  Any output pointer may be NULL. */
fe_status fe_pattern_copy(const fe_pattern *pat, int32_t *cell_dofs, int64_t *row_ptr, int32_t *col_idx);
fe_status fe_pattern_destroy(fe_pattern *pat);

/* Thread-local description of the last error ("" if none). */
const char *fe_last_error(void);

/* ---------------------------------------------------------------------- */
/* Plans                                                                   */
/* ---------------------------------------------------------------------- */

/* Build a plan for one mesh, degree and quadrature rule (Algorithm 1, step 1
 * and the setup of Sec. 3.3): FP64 tabulation of phi and grad phi at the
 * rule's points (Appendix A product form), the per-precision contraction
 * operands rounded once to the storage format (List 1, u_s), the dof map,
 * the CSR pattern and the assembly index streams.  The plan copies the mesh
 * and the rule to the device; the caller's host arrays are not retained.
 * form_mask: FE_FORM_* bits the plan must serve.  prec_mask: FE_PREC_MASK()
 * bits of the precisions the plan must serve.  cuda_stream: a cudaStream_t
 * (NULL = legacy default stream) on which all later calls run.
 * Synchronous.  Returns FE_ERR_UNSUPPORTED for degrees outside 1..8 on
 * tetrahedra or 1..10 on triangles, FE_ERR_NO_DEVICE without a GPU. */
fe_status fe_plan_create(fe_plan **out, const fe_mesh *mesh, int degree, const fe_quadrature *rule,
                         unsigned form_mask, unsigned prec_mask, void *cuda_stream);
fe_status fe_plan_destroy(fe_plan *plan);
fe_status fe_plan_set_stream(fe_plan *plan, void *cuda_stream);
/* Limit on how long one bounded wait inside this plan's kernels (the
 * pipeline barriers of the persistent tensor-core kernel) may see no
 * progress before the kernel gives up: it then stops issuing work, lets its
 * copies and MMAs in flight finish, releases its tensor memory and returns,
 * and the call reports FE_ERR_TIMEOUT through fe_sync_status (outputs are
 * then incomplete; the plan stays usable and the next call starts afresh).
 * The limit applies to each wait from its own start, not to a whole launch,
 * so a long launch whose waits all complete never trips it.  limit_ns = 0
 * restores the default of 2 s.  A batch uses the largest limit of its plans
 * at creation.  Not an error path a healthy GPU takes: it exists so that a
 * stalled pipeline ends with an error instead of hanging the device. */
fe_status fe_plan_set_wait_limit(fe_plan *plan, uint64_t limit_ns);
/* Fused assembly of fe_assemble (see there): mode 1 on, 0 off (the default).
 * active (may be NULL) receives 1 when fe_assemble without element-matrix
 * outputs will take the fused path on this plan. */
fe_status fe_plan_set_fusion(fe_plan *plan, int mode, int *active);
/* Assembly algorithm of this plan's fe_assemble / fe_assemble_elements (and
 * of batches, from their first plan): 0 (default) the chunked segmented
 * reduction (element entries staged in segment order, one thread per CSR
 * value); 1 one warp per CSR row walking the row's element rows in cell order
 * into shared-memory accumulators at their column slots (also the kernel of
 * the fused path; measured about 2x slower than 0 on the P3 24^3 x 6
 * workload, where rows are short).  Both sum every CSR value's entries in
 * increasing cell order from zero: bitwise the same values. */
fe_status fe_plan_set_assembly(fe_plan *plan, int algo);
/* Window prefetch of the tensor-core element kernel, where a job reads more
 * than one coefficient window (more quadrature points than one 128-byte K
 * chunk holds, or boxed cells, whose geometry gives each pair its own window):
 * the builder threads copy their next window asynchronously into shared
 * memory while the current one is used, at the price of a shared-memory slot
 * per thread that would otherwise hold an operand stage.  mode -1 (default):
 * as the plan's autotuner measured fastest per precision and form; 0 off;
 * 1 on wherever it fits.  The element matrices are bitwise the same in every
 * mode. */
fe_status fe_plan_set_window_prefetch(fe_plan *plan, int mode);
/* N layout of the tensor-core contraction for these forms in this (reduced)
 * precision: whole-row passes of `rows` rows of every element matrix each
 * (rows * n_phi columns, at most 512; above 256 a pass is wide: both halves of
 * the tensor memory form one accumulator and each coefficient chunk feeds two
 * MMAs), replacing the layout the plan's autotuner chose.  The element
 * matrices agree with every other layout to FP32 accumulation order. */
fe_status fe_plan_set_rows_per_pass(fe_plan *plan, fe_precision prec, unsigned forms, int rows);
/* Launch shape the tensor-core element kernel takes for these forms and this
 * (reduced) precision on this plan, as fe_element_matrices would launch it
 * now: stages of the built-operand ring (ring_a) and of the shared-operand
 * ring (ring_b), whether the builders prefetch windows (win_buf, 0/1),
 * whether the epilogue stages through shared memory (staged, 0/1), and the
 * number of tensor-memory accumulators (n_acc: 2 of 256 columns, or 1 of 512
 * when a pass is wide).  Any output pointer may be NULL.  No device work. */
fe_status fe_plan_tc_config(fe_plan *plan, unsigned forms, fe_precision prec, int32_t *ring_a, int32_t *ring_b,
                            int32_t *win_buf, int32_t *staged, int32_t *n_acc);
/* Device memory the plan holds, in bytes: plan_bytes for what plan creation
 * allocated (mesh, tabulations, operand images, dof map, pattern, assembly
 * streams, action tables built so far), workspace_bytes for the workspaces
 * that compute calls allocate on first use and keep (element matrices,
 * coefficient windows, copies of host buffers, adjoint scratch).  Host only;
 * any output pointer may be NULL. */
fe_status fe_plan_memory(const fe_plan *plan, int64_t *plan_bytes, int64_t *workspace_bytes);
/* Any output pointer may be NULL. */
fe_status fe_plan_sizes(const fe_plan *plan, int64_t *n_cells, int64_t *n_vertices, int64_t *n_dofs,
                        int64_t *nnz, int32_t *n_phi, int32_t *n_q);
/* Device copies of the pattern: row_ptr int64 [n_dofs+1], col_idx int32 [nnz]. */
fe_status fe_csr_pattern(const fe_plan *plan, int64_t *row_ptr, int32_t *col_idx);
/* Device copy of the dof map, int32 [n_cells][n_phi]. */
fe_status fe_cell_dofs(const fe_plan *plan, int32_t *cell_dofs);

/* Element matrices (Algorithm 1 for every cell; Sec. 3.1).
 * forms: FE_FORM_* bits (subset of the plan's form_mask).
 * vertices: device [n_vertices][d] FP64, or NULL for the plan's copy.
 * kappa: device [n_cells][n_q] FP64, the coefficient at the quadrature points.
 * A_stiffness / A_mass: device [n_cells][n_phi][n_phi], double for
 * FE_PREC_FP64 else float; the pointer of a form not in `forms` is ignored.
 * The reduced-precision paths run two kernels: a factor kernel (geometry,
 * the coefficient window w_q kappa_cq in FP32 and the per-cell scales, into
 * a plan workspace of 4 * (n_q rounded up to 4) + 64 bytes per cell, allocated
 * on first use) and the tensor-core kernel.  Asynchronous on the plan's
 * stream; device status (degenerate or non-finite cells, timeouts) is read
 * by fe_sync_status. */
fe_status fe_element_matrices(fe_plan *plan, unsigned forms, fe_precision prec, const double *vertices,
                              const double *kappa, void *A_stiffness, void *A_mass);

/* Element matrices followed by global assembly A^g = L D L^T (Sec. 3.3).
 * A_stiffness / A_mass may be NULL: the element matrices then live in a plan
 * workspace.  csr_stiffness / csr_mass: device [nnz] values in the plan's
 * pattern (double for FE_PREC_FP64 else float).  Each CSR value is the sum
 * of its element entries in increasing (cell, k, l) order starting from 0,
 * so results are bitwise reproducible.
 * Fused assembly (opt-in, fe_plan_set_fusion): with both element-matrix
 * pointers NULL (reduced precision), the plan processes the cells in slices
 * of one wave of tiles (SMs * 128 cells): each slice's element matrices go to
 * a ring of a few slices that stays in L2, and the rows whose cells are all
 * done are assembled from it at once (row-wise kernel), so the element
 * matrices make no round trip through HBM.  The results are bitwise those of
 * the unfused path.  Eligible where the mesh spans several slices, each
 * row's cells span at most three slices, and the ring (both forms) fits in a
 * third of the L2 cache.  Off by default: on this part the per-slice launches
 * cost the persistent kernel its overlap across tiles, which outweighs the
 * saved traffic (measured slower on P2 32^3 x 6 tetrahedra). */
fe_status fe_assemble(fe_plan *plan, unsigned forms, fe_precision prec, const double *vertices,
                      const double *kappa, void *A_stiffness, void *A_mass, void *csr_stiffness,
                      void *csr_mass);

/* Same as fe_assemble with HOST buffers: copies kappa (host [n_cells][n_q])
 * to the device, computes, and copies the CSR values back to the host
 * buffers (host [nnz]; NULL skips a form's copy).  Synchronous.  Pinned host
 * memory gives the fastest copies. */
fe_status fe_assemble_host(fe_plan *plan, unsigned forms, fe_precision prec, const double *kappa_host,
                           void *csr_stiffness_host, void *csr_mass_host);

/* fe_assemble_host for a sequence of n coefficient sets (a parameter sweep,
 * samples of a random coefficient): item i takes kappa_host[i] (host
 * [n_cells][n_q]) and leaves its CSR values in csr_stiffness_host[i] /
 * csr_mass_host[i] (host [nnz] each; either array, or an entry, may be NULL
 * to skip that form's copy).  The upload of item i+1, the computation of item
 * i and the download of item i-1 overlap: two slots of device buffers (kept
 * by the plan), an upload and a download stream, ordered by events, so that
 * the host link in both directions and the GPU work at once.  Results are
 * bitwise those of fe_assemble_host.  A host output buffer may be reused by
 * item i+2 and later (their downloads are ordered).  Synchronous: returns
 * after the last download; pinned host memory gives the fastest copies. */
fe_status fe_assemble_host_many(fe_plan *plan, unsigned forms, fe_precision prec, int n,
                                const double *const *kappa_host, void *const *csr_stiffness_host,
                                void *const *csr_mass_host);

/* Assembly only, from caller element matrices (device, layout as above). */
fe_status fe_assemble_elements(fe_plan *plan, unsigned forms, fe_precision prec, const void *A_stiffness,
                               const void *A_mass, void *csr_stiffness, void *csr_mass);

/* Linear forms (Algorithm 2; Sec. 3.1 v_j = a_K(w, phi_j)): the action of
 * the mass and/or Poisson form on the FE function with global coefficients w,
 *   b^c = sum_s B_s r_s,  r_s = vstack_q(w_q z(X_q) (G grad w(X_q))_s)
 * (mass: r = vstack_q(w_q z(X_q) |det J| w(X_q))), and the vector assembly
 * v^g = L b (Sec. 3.3), each entry summed over its cells in increasing cell
 * order (bitwise reproducible).
 * prec: FE_PREC_FP64 (FP64 throughout), or FE_PREC_TF32 / BF16 / FP16: the
 * tabulated B and each cell's coefficients rounded once to the storage format
 * (the casting remark of Sec. 4.5), r_s computed in FP32 and rounded once to
 * the storage format (the theorem on r_s, Sec. 4.5), both contractions
 * accumulated in FP32.  Others: FE_ERR_UNSUPPORTED.  Both forms requested
 * together are computed in one pass over kappa and the geometry.
 * kappa: device [n_cells][n_q] FP64.  w: device [n_dofs] FP64.
 * b_stiffness / b_mass: device [n_cells][n_phi] cell vectors (double for FP64
 * else float) or NULL; v_stiffness / v_mass: device [n_dofs] (same type) or
 * NULL; a requested form needs at least one of its two outputs (cell vectors
 * then live in a plan workspace).  Asynchronous on the plan's stream. */
fe_status fe_action(fe_plan *plan, unsigned forms, fe_precision prec, const double *vertices, const double *kappa,
                    const double *w, void *b_stiffness, void *b_mass, void *v_stiffness, void *v_mass);

/* Adjoint of L = v^T A^g u for the stiffness form (not in the paper):
 *   g_kappa[c][q] = dL/dkappa_cq = w_q |det J| (J^{-T} grad u_h(X_q)).(J^{-T} grad v_h(X_q))
 *   g_vertices[v][i] = dL/dx_{v,i}, kappa at the quadrature points held fixed,
 * with the geometry recomputed from the vertices (nothing stored from the
 * forward pass).  u, v: device float [n_dofs]; vertices: device or NULL;
 * kappa: device; g_kappa: device double [n_cells][n_q] or NULL; g_vertices:
 * device double [n_vertices][d] or NULL (overwritten, not accumulated);
 * L_out: device double [1] or NULL.  Computed in FP64 on the CUDA cores. */
fe_status fe_adjoint(fe_plan *plan, const double *vertices, const double *kappa, const float *u,
                     const float *v, double *g_kappa, double *g_vertices, double *L_out);

/* Adjoint of L = sum_e g_e A^g_e for the stiffness form and a given gradient
 * g on the CSR values (the backward pass of the assembly; not in the paper):
 * with G^c_kl = g at the CSR slot of (dof(c,k), dof(c,l)) -- the transpose of
 * A^g = L D L^T, Sec. 3.3 --
 *   g_kappa[c][q] = dL/dkappa_cq = w_q sum_kl G^c_kl grad phi_l^T G grad phi_k (X_q),
 *   g_vertices    = dL/dx (kappa at the quadrature points held fixed),
 * G = |det J| J^-1 J^-T recomputed from the vertices.  grad_values: device
 * double [nnz] in the plan's CSR order; vertices, kappa, outputs as for
 * fe_adjoint (g_kappa / g_vertices / L_out may be NULL).  FP64 on the CUDA
 * cores, one warp per cell with G^c in shared memory (n_phi^2 doubles: larger
 * elements than 160 local dofs return FE_ERR_UNSUPPORTED).  Deterministic. */
fe_status fe_adjoint_values(fe_plan *plan, const double *vertices, const double *kappa, const double *grad_values,
                            double *g_kappa, double *g_vertices, double *L_out);

/* Allocation-free variant of fe_adjoint; the paper has no counterpart.
 *
 * Some callers may not allocate device memory while they run: applications
 * whose device memory belongs to their own allocator or to a fixed budget,
 * and latency-critical loops that cannot afford the implicit device
 * synchronisation of cudaMalloc / cudaFree.  fe_adjoint allocates its
 * per-cell scratch (the vertex-gradient contributions of every cell and the
 * per-cell L) in a plan workspace on first use; this entry point computes
 * the same results with the same kernels but takes that scratch from one
 * fixed device array of 32 MiB (4,194,304 doubles) declared statically in
 * the library, which every GPU that loads the library holds until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine; the caller still passes every input and output.
 *
 * Limit: n_cells * ((d+1)*d + 1) doubles of scratch with g_vertices, n_cells
 * without (at most 322,638 tetrahedra or 599,186 triangles with vertex
 * gradients); a larger plan returns FE_ERR_UNSUPPORTED and fe_last_error()
 * states the sizes.  The array is shared by every call in the process,
 * whatever the plan or stream, and keeps the last call's contents: calls
 * whose kernels overlap on the GPU race on it, so serialise them.  Every
 * scratch entry a call reads is written earlier in the same call, so nothing
 * needs clearing.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, once per device); make that first call
 * before any stream capture begins.  Arguments as for fe_adjoint. */
fe_status fe_adjoint_noalloc(fe_plan *plan, const double *vertices, const double *kappa, const float *u,
                             const float *v, double *g_kappa, double *g_vertices, double *L_out);

/* ---------------------------------------------------------------------- */
/* Diagnostics: the paper's error studies (Sec. 5.2, 5.3)                  */
/* ---------------------------------------------------------------------- */

/* Geometry tensor G = |det J| J^-1 J^-T and |det J| of cells [c0, c1)
 * (Sec. 4.2, the Poisson geometry; Sec. 5.2 studies its rounding error
 * against the condition number of J).  mode:
 *   FE_GEOMETRY_FP64   J, cofactors, det J and G in FP64;
 *   FE_GEOMETRY_FP32   the same formulas exclusively in FP32 from the vertex
 *                      coordinates rounded to FP32, each operation an IEEE
 *                      FP32 operation in a fixed order (reproducible bits):
 *                      J_ij = x_{j+1,i} - x_{0,i}; cofactors C as 2x2 minors
 *                      fl(fl(a b) - fl(c e)); det = fl(fl(J00 C0 + J01 C1) +
 *                      J02 C2); G_st = fl(fl(sum_r C_rs C_rt, r increasing) *
 *                      fl(1 / |det|));
 *   FE_GEOMETRY_MIXED  the reduced-precision kernels' own path: FP64
 *                      cofactors and det J, G in FP32, and G in FP64 rounded
 *                      once on cells whose off-diagonal sums cancel (the
 *                      per-cell geometry precision of the remark in Sec. 5.2);
 *                      used_fp64[i] = 1 for those cells.
 * vertices: device [n_vertices][d] or NULL (the plan's).  G: device double
 * [c1-c0][d(d+1)/2], pairs (0,0),(0,1),(0,2),(1,1),(1,2),(2,2) (d = 2:
 * (0,0),(0,1),(1,1)); absdet: device double [c1-c0] or NULL; used_fp64:
 * device int32 [c1-c0] or NULL (MIXED only).  Asynchronous. */
enum { FE_GEOMETRY_FP64 = 0, FE_GEOMETRY_FP32 = 1, FE_GEOMETRY_MIXED = 2 };
fe_status fe_geometry(fe_plan *plan, int mode, const double *vertices, int64_t c0, int64_t c1, double *G,
                      double *absdet, int32_t *used_fp64);

/* The mass bilinear form and the mass action of cells [c0, c1) with the
 * matrix-matrix (matrix-vector) products in FP16 and everything else in FP32
 * (Sec. 5.3: u_s = u_g = u_p = 2^-24, u_q = 2^-11), the experiment that
 * measures how the accumulation error grows with n_q:
 *   C_q  = fl32(fl32(w_q kappa_cq) |det J|) 2^e      (|det J| in FP32 from FP32 coordinates)
 *   H_kq = fl32(C_q phi_kq),   A_kl = 2^-e sum16_q fl16(phi_lq H_kq)
 *   w_q  = sum32_l fl32(phi_lq w_l 2^f),  r_q = fl32(C_q w_q),
 *   b_k  = 2^-e 2^-f sum16_q fl16(phi_kq r_q)
 * with sums over q increasing from 0, sum16 one FP16 rounding per addition,
 * fl16 one rounding of the exact product, and powers of two per cell (2^e:
 * sum_q |C_q| 2^e in [2^9, 2^10); 2^f: max|w^c| 2^f in [1, 2)) that keep the
 * FP16 values in range.  kappa: device [n_cells][n_q]; w: device double
 * [n_dofs] (needed for b); A: device float [c1-c0][n_phi][n_phi] or NULL; b:
 * device float [c1-c0][n_phi] or NULL.  One CUDA thread per (cell, k): a
 * diagnostic, not a fast path.  Asynchronous. */
fe_status fe_mass_fp16_products(fe_plan *plan, const double *kappa, const double *w, int64_t c0, int64_t c1, float *A,
                                float *b);

/* ---------------------------------------------------------------------- */
/* Batches                                                                 */
/* ---------------------------------------------------------------------- */

/* A batch of plans run as one factor launch and one persistent tensor-core
 * launch (the cell batching of Sec. 3.1, generalised to meshes of uneven
 * size, cell type and degree) followed by one assembly launch over the rows
 * of every plan, captured once in a CUDA graph and replayed by fe_batch_run.
 * Each plan's tile shape (N-pass width) is the one its autotuner chose.
 * plans: n_plans plans on the current device, each serving `forms` and
 * `prec` (FE_PREC_FP64 runs the FP64 kernels, one per plan and form, inside
 * the same graph).  kappa[i]: device coefficients of plan i.  A_stiffness /
 * A_mass: arrays of n_plans device outputs (element matrices), or NULL (the
 * batch owns workspaces); an entry may be NULL likewise.  csr_stiffness /
 * csr_mass: arrays of n_plans device CSR value outputs, both NULL to skip
 * assembly.  Every buffer must stay valid, at the same address, for the
 * batch's lifetime: the graph reads and writes them at each run.
 * cuda_stream must be a non-default stream.  Creation runs the batch once
 * eagerly (errors surface there) and synchronises. */
typedef struct fe_batch fe_batch;
fe_status fe_batch_create(fe_batch **out, fe_plan *const *plans, int n_plans, unsigned forms, fe_precision prec,
                          const double *const *kappa, void *const *A_stiffness, void *const *A_mass,
                          void *const *csr_stiffness, void *const *csr_mass, void *cuda_stream);
/* Replay the batch's graph on its stream (asynchronous). */
fe_status fe_batch_run(fe_batch *batch);
/* Wait for the batch's stream and report (and clear) its device status word. */
fe_status fe_batch_sync(fe_batch *batch);
/* Total cells and nnz over the plans, and kernel launches per run. */
fe_status fe_batch_sizes(const fe_batch *batch, int64_t *n_cells, int64_t *nnz, int32_t *launches);
fe_status fe_batch_destroy(fe_batch *batch);

/* Wait for the plan's stream and report the device status word (and clear it). */
fe_status fe_sync_status(fe_plan *plan);

/* Per-stage GPU times (milliseconds) of the most recent call made while
 * timing was enabled: [0] element-matrix kernel(s), [1] assembly kernel,
 * [2] adjoint kernel(s), [3] factor kernel (geometry, coefficient window and
 * per-cell scales of the tensor-core paths).  n <= 4 values are written.
 * Timing uses CUDA events on the plan's stream. */
fe_status fe_plan_enable_timing(fe_plan *plan, int enable);
fe_status fe_plan_stage_times(fe_plan *plan, float *ms, int n);

/* Number of kernel launches made by the most recent compute call. */
fe_status fe_plan_last_launches(const fe_plan *plan, int32_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* FE_GB300_H */
