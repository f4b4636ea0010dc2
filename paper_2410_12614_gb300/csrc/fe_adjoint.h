// Adjoint of the assembly for a general gradient on the CSR values (the
// backward pass of values = assemble(kappa, x) for the stiffness form).
#pragma once

#include "fe_internal.h"

namespace fe {

// base: geometry, kappa, weights, tables, dofs and outputs as for the
// quadratic-form adjoint (u, v unused).
struct AdjValArgs {
    AdjArgs base;
    const double *gvals;       // [nnz] dL/d(CSR value)
    const int64_t *row_ptr;    // [n_dofs + 1]
    const int32_t *col_idx;    // [nnz], sorted within each row
};

// Per-cell kernel, then the vertex gather and the ordered sum of L as for the
// quadratic form.  Returns the launches made or a negative cudaError_t.
int launch_adjoint_values(const AdjValArgs &a, const int64_t *vinc_ptr, const int32_t *vinc, double *g_vertices,
                          double *L_out, cudaStream_t s);

}  // namespace fe
