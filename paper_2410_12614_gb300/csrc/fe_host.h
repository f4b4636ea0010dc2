// Host-side plan construction: quadrature, reference basis, dof map, CSR
// pattern, assembly index streams and the packed contraction operands.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace fe {
namespace host {

// Collapsed Gauss-Jacobi rule (see fe_quadrature_rule in the public header).
bool gauss_jacobi(int m, int alpha, std::vector<double> &t, std::vector<double> &w);
bool collapsed_rule(int d, int m, std::vector<double> &pts, std::vector<double> &wts);

int n_phi(int d, int p);
// Barycentric multi-indices of the local nodes, [n_phi][d+1], local order.
std::vector<int> lattice_nodes(int d, int p);
// phi [n_phi][n_q] and dphi [d][n_phi][n_q] at the points [n_q][d], FP64.
void tabulate(int d, int p, const double *pts, int n_q, std::vector<double> &phi, std::vector<double> &dphi);

// Boxed cells (quadrilaterals d = 2, hexahedra d = 3) on the reference
// [0,1]^d: tensor Gauss-Legendre rule (m points per direction, x fastest),
// n_phi = (p+1)^d, lattice nodes a in {0..p}^d with node k = a_0 + (p+1)(a_1 +
// (p+1) a_2), cell vertex v at the corner (bit_0(v), bit_1(v), bit_2(v)).
bool tensor_rule(int d, int m, std::vector<double> &pts, std::vector<double> &wts);
int n_phi_box(int d, int p);
void tabulate_box(int d, int p, const double *pts, int n_q, std::vector<double> &phi, std::vector<double> &dphi);

// Row chunks of the block-wide assembly: consecutive CSR rows holding at most
// kAsmChunkEntries element entries and kAsmChunkIncidences incidences (a row
// above the entry limit forms a chunk of its own).
constexpr int kAsmChunkEntries = 4096;
constexpr int kAsmChunkIncidences = 256;

struct Pattern {
    int d = 0, p = 0, n_phi = 0;
    int64_t n_vertices = 0, n_cells = 0, n_dofs = 0, nnz = 0;
    int max_row = 0;
    std::vector<int32_t> cell_dofs;   // [n_cells][n_phi]
    std::vector<int64_t> row_ptr;     // [n_dofs+1]
    std::vector<int32_t> col_idx;     // [nnz]
    // assembly index streams (built on demand)
    std::vector<int64_t> inc_ptr;     // [n_dofs+1]
    std::vector<int32_t> inc_elem;    // c * n_phi + k, sorted by (dof, c)
    std::vector<uint16_t> inc_slot;   // [n_inc][n_phi]
    // per CSR entry, its element-entry contributions in increasing cell order:
    // code t | l << 8 (t = incidence index counted from the first incidence of
    // the row's chunk, l = local column)
    std::vector<uint8_t> contrib_cnt;   // [nnz]
    std::vector<int64_t> contrib_base;  // [n_dofs + 1] first code of each row
    std::vector<uint16_t> contrib_code; // [n_cells * n_phi * n_phi]
    std::vector<int32_t> chunk_row;     // [n_chunks + 1] first row of each assembly chunk
    // [n_chunks + 1][4]: first row, first code, first incidence, first CSR value
    std::vector<int64_t> chunk_desc;
    // per chunk, its element entries in incidence order (incidence t of the
    // chunk, local column l at t * n_phi + l) mapped to their position in the
    // chunk's code order (the concatenated CSR-value segments)
    std::vector<uint16_t> contrib_dest; // [n_cells * n_phi * n_phi]
    // fused assembly (cells in slices of slice_cells): the slice after which
    // every row of a chunk is complete (the largest slice of its rows' cells),
    // and the widest range of slices one row's cells span (+1); empty / 0
    // without slicing
    std::vector<int32_t> chunk_slice;   // [n_chunks]
    int slice_span = 0;
    // vertex -> (cell, local vertex) incidence for the adjoint scatter
    std::vector<int64_t> vinc_ptr;    // [n_vertices+1]
    std::vector<int32_t> vinc;        // c * (d+1) + j, sorted by (vertex, c)
};

// Returns "" on success, else an error message.  boxed: cells are
// quadrilaterals / hexahedra with 2^d vertices in tensor order.
// slice_cells > 0: assembly chunks also end where the rows' completion slice
// (the slice of their last incident cell, cells in slices of slice_cells)
// changes, and chunk_slice / slice_span are filled.
std::string build_pattern(int d, int p, int64_t n_vertices, int64_t n_cells, const int32_t *cells, Pattern &out,
                          bool with_streams, bool boxed = false, int64_t slice_cells = 0);

// Round x to a binary format with `mbits` explicit mantissa bits, minimum
// normal exponent `emin` and largest finite value `maxfinite`
// (round-to-nearest-even, gradual underflow, saturating at +-maxfinite).
double round_to_format(double x, int mbits, int emin, double maxfinite);

// Storage formats of the contraction operands.
struct Format {
    int elem_bytes;
    int mbits;
    int emin;
    double maxfinite;
    int target_exp;   // scale the largest magnitude into [2^(t-1), 2^t)
};
Format format_of(int prec);
// Bit pattern of an exactly representable value (as produced by round_to_format).
uint32_t encode(int prec, double r);

// Build the swizzled operand image of one form (see fe_plan.cpp).
struct OperandImage {
    std::vector<uint8_t> bytes;
    int n_kchunks = 0, n_qw = 0, n_pairs = 1, n_pass = 0, NP = 0, n_cols = 0, n_blk = 1;
    int rows_per_pass = 0;   // 0: symmetric-pair columns; R > 0: each pass holds R full rows (k, every l)
    double p_inv_scale = 1.0;
};
// np_pass: N columns per pass (multiple of 16 in 16..256) of the symmetric-
// pair layout, 0 for the default layout (pairs in one pass if n_sym <= 256;
// else full-row passes when row_block_default says so, pair passes of 256
// otherwise), or -R for the full-row layout with R rows per pass.
// col_of_sym: the operand column of each symmetric pair (k <= l) in the pair
// layout, or empty for column = pair index.
void build_operand(int prec, int form, int d, int n_phi, int n_q, const std::vector<double> &phi,
                   const std::vector<double> &dphi, OperandImage &img, int np_pass = 0,
                   const std::vector<int> &col_of_sym = {});

// Operand columns of the symmetric pairs (k <= l, in row order) for the staged
// epilogue: a column's staged value sits in shared-memory bank (column mod 32),
// and one gather instruction of the epilogue reads the 32 output positions of a
// group (v4: positions 128 it + 4 j + e, j = 0..31, for fixed it and e; else 32
// consecutive positions).  The pairs of a group get distinct banks where the
// greedy colouring (with restarts) finds it; columns stay below
// 16 * ceil(n_sym / 16).  Identity for n_sym > 256 (multi-pass shapes).
// conflicts (optional): the remaining excess over one per bank, summed over groups.
std::vector<int> stage_columns(int n_phi, bool v4, int *conflicts = nullptr);
// Candidate layouts for the autotuner (np_pass values as above): the pair
// layout's default width and the narrowest widths that keep the minimal number
// of passes, and for n_sym > 256 the full-row layout.
std::vector<int> np_candidates(int n_phi);
// Rows per pass of the full-row layout (R * n_phi <= 240 columns), and whether
// it is the default for shapes whose pairs need several passes (at most twice
// the passes of the pair layout).
int row_block_rows(int n_phi);
bool row_block_default(int n_phi);

unsigned hardware_threads();

}  // namespace host
}  // namespace fe
