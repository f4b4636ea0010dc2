// Internal declarations shared by the host plan builder (fe_plan.cpp,
// fe_abi.cpp) and the CUDA kernels.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fe_gb300.h"

namespace fe {

// Device status word bits (set by kernels with atomicOr, read by fe_sync_status).
enum : int {
    ST_DEGENERATE = 1,
    ST_NONFINITE = 2,
    ST_TIMEOUT = 4,
    ST_SATURATED = 8,
};

// Tile of the tensor-core element kernel: 128 cells on the MMA M dimension.
constexpr int TC_M = 128;
constexpr int TC_THREADS = 256;        // two threads per cell
constexpr int TC_STAGES = 2;
constexpr int TC_CHUNK_BYTES = 128;      // one 128B-swizzled K-major row per chunk
constexpr int TC_MAX_NP = 256;           // N of one MMA pass
constexpr int MAX_FORMS = 2;             // 0 = stiffness, 1 = mass
constexpr int TC_JOB_EPI_COST = 2;       // a job's epilogue, in K chunks, for the work split
constexpr int TC_MAX_RING_A = 4;         // deepest ring of built (per-cell) operand chunks
constexpr int TC_MAX_RING_B = 8;         // deepest ring of shared-operand chunks in flight

// Quadrature points per window (K block) for a storage format: 64 for every
// format of at most 16 bits, 32 for TF32.
__host__ __device__ constexpr int tc_window_points(int prec) {
    return prec == FE_PREC_TF32 || prec == FE_PREC_TF32X3 ? 32 : 64;
}

// Operand description of one form in one precision.
// K is split into blocks h = (qw * n_pairs + j) * n_blk + blk: quadrature
// window qw (KW = tc_window_points consecutive points) of pair j and split
// block blk.  A 128-byte chunk holds KCE / KW consecutive blocks (KCE =
// 128/elem_bytes elements): one for the 16- and 32-bit formats (KW = KCE),
// two 64-point blocks for e4m3.  Each chunk of the shared operand is stored
// as an NP x 128 B swizzled K-major tile.
struct TcOperand {
    const uint8_t *img = nullptr;  // [n_pass][n_kchunks][NP][128 B] swizzled images
    int n_kchunks = 0;             // K chunks of 128 bytes
    int n_qw = 0;                  // quadrature windows
    int n_pairs = 1;               // symmetric (s,t) pairs (stiffness) or 1 (mass)
    int n_pass = 0;                // N passes
    int NP = 0;                    // N per pass (multiple of 16; <= 256, or <= 512 for a wide full-row pass)
    int n_cols = 0;                // operand columns that may carry a pair (sym_kl entries)
    int n_blk = 1;                 // 1, or 3 for split TF32 (head, head, tail)
    int rows_per_pass = 0;         // 0: columns are symmetric pairs; R: pass n holds rows nR..nR+R-1 (all l)
    float p_inv_scale = 1.f;       // 2^-e_P
    int win_pref = 0;              // 1: the builders prefetch the next window (autotuned where a job reads several)
};

// One plan's share of a (possibly batched) tensor-core element launch.
struct TcSeg {
    const double *vertices;
    const int32_t *cells;
    int64_t n_cells;
    int d;
    const double *kappa;
    const double *weights;
    int n_q;
    int n_phi;
    int n_pairs;      // d(d+1)/2
    int form_mask;    // bit 0 stiffness, bit 1 mass (internal order)
    TcOperand op[MAX_FORMS];
    float *out[MAX_FORMS];
    const int32_t *sym_kl;     // [operand column] k | l << 16, -1 for padding columns
    const int16_t *full2sym;   // [n_phi * n_phi] operand column of entry (k, l)
    int staged;                // 1: staged coalesced epilogue (single pass)
    int64_t tile_begin;        // first global tile of this segment
    int64_t tiles;             // tiles of this segment
    // Work split: a job is one (tile, form, N pass) and costs the form's K
    // chunks plus TC_JOB_EPI_COST; every tile of a segment costs tile_cost,
    // and the segment's first job starts at cost_begin of the launch's total.
    int64_t cost_begin;
    int tile_cost;
    // written by the factor kernel, read by the element kernel
    float *win;                // [n_cells][win_slots][ldw] coefficient windows in FP32 (zero past n_q)
    float *cellf;              // [n_cells][CELLF] per-cell factors (CELLF_* slots)
    int ldw;                   // n_q rounded up to a multiple of 4
    // Simplices: win_slots = 1, the window w_q kappa_cq shared by every pair and
    // form (G constant per cell, in cellf).  Boxed cells: win_slots = n_pairs + 1,
    // slot j < n_pairs holding w_q kappa_cq G_j(X_q) and slot n_pairs w_q kappa_cq
    // |det J(X_q)| (the geometry varies with the point); cellf then carries only
    // the power-of-two scales.
    int win_slots;
    int nv;                    // vertices per cell (d + 1, or 2^d for boxed cells)
    const double *dpsi;        // boxed cells: Q1 derivatives at the rule's points [d][nv][n_q]
};

// Per-cell factor record (floats): the scaled geometry of each pair, the
// scaled |det J| for the mass form, and the unscale of each form's accumulator.
constexpr int CELLF = 16;
constexpr int CELLF_G = 0;         // [0, 6): G_st * 2^e_stiffness
constexpr int CELLF_DET = 6;       // |det J| * 2^e_mass
constexpr int CELLF_UNSCALE = 8;   // [8, 10): unscale of form 0 / form 1
inline int win_ld(int n_q) { return (n_q + 3) & ~3; }

struct TcArgs {
    TcSeg seg0;                // the only segment when segs == nullptr
    const TcSeg *segs;         // device array of n_segs segments (batched launch)
    int n_segs;
    int64_t n_tiles;           // total tiles over all segments
    int64_t n_jobs;            // (tile, form, pass) jobs over all segments
    int64_t total_cost;        // summed job costs; CTA i of G takes the jobs starting in [iT/G, (i+1)T/G)
    int prec;                  // fe_precision
    int elem_bytes;            // storage bytes per operand element
    uint32_t idesc;            // instruction descriptor without the N field
    int target_exp;            // per-cell scale target: max|C| * 2^e in [2^(t-1), 2^t)
    int np_max;                // largest N per pass over the segments
    int nq_max;                // largest n_q
    int pitch_max;             // staging pitch (floats) over staged segments, 0 if none
    int ring_a;                // stages of the built-operand ring (2..TC_MAX_RING_A)
    int ring_b;                // stages of the shared-operand ring (2..TC_MAX_RING_B)
    int win_buf;               // 1: a per-builder-thread shared-memory slot for the next window
    int n_acc;                 // TMEM accumulators: 2 of 256 columns, or 1 of 512 when a pass is wide
    int job_rr;                // 1: jobs in pass-major order dealt round-robin (single plan, large operand)
    int *status;
    unsigned long long timeout_ns;
};

struct F64Args {
    const double *vertices;
    const int32_t *cells;
    int64_t n_cells;
    int d;
    const double *kappa;
    const double *weights;
    int n_q;
    int n_phi;
    const double *tab;   // stiffness: dphi [d][n_phi][n_q]; mass: phi [n_phi][n_q]
    int form;            // FE_FORM_MASS or FE_FORM_STIFFNESS
    double *out;
    int tc;              // cells per block
    int qc;              // quadrature points per chunk
    int *status;
    const double *geo_q; // boxed cells: [n_cells][n_q][7] G pairs and |det J| per point (else null)
};

// One plan's share of a (possibly batched) assembly launch.
// Row chunks of the assembly (fe_host.h kAsmChunkEntries / kAsmChunkIncidences).
constexpr int ASM_CHUNK = 4096;
constexpr int ASM_CHUNK_INC = 256;

struct AsmSeg {
    int64_t n_rows;
    const int64_t *row_ptr;
    const int64_t *inc_ptr;    // [n_rows + 1] into inc_elem
    const int32_t *inc_elem;   // element-row ids c * n_phi + k, sorted by (row, c)
    const uint8_t *contrib_cnt;     // [nnz] number of element entries summed into each CSR value
    const int64_t *contrib_base;    // [n_rows + 1] first contribution code of each row
    const uint16_t *contrib_code;   // incidence index in the chunk | local column << 8, per row in slot order
    const uint16_t *contrib_dest;   // per chunk, entry (t, l) at t * n_phi + l -> its position in code order
    const int64_t *chunk_desc;      // [n_chunks + 1][4] first row, code, incidence and CSR value of each chunk
    int64_t n_chunks;
    int n_phi;
    const void *A[MAX_FORMS];
    void *out[MAX_FORMS];
    int64_t row_begin;         // first global row of this segment
    int64_t chunk_begin;       // first global chunk of this segment
    const uint16_t *inc_slot;       // [n_inc][n_phi] column slot of entry (incidence, l) in its row (row kernel)
    // fused assembly: the element matrices of cell c sit in ring slot
    // (c / ring_cells) % ring_slots at cell offset c % ring_cells (0: no ring)
    int64_t ring_cells;
    int ring_slots;
};

struct AsmArgs {
    AsmSeg seg0;               // the only segment when segs == nullptr
    const AsmSeg *segs;        // device array (batched launch)
    int n_segs;
    int64_t n_rows;            // total rows over all segments
    int64_t n_chunks;          // total chunks over all segments
    int n_forms;
    const int32_t *chunk_list; // optional: the chunks to assemble (device), walked from its end
    int64_t list_count;
    int algo;                  // 0: chunked segmented reduction, 1: one warp per row (assemble_rows_kernel)
    const int32_t *row_list;   // row kernel, optional: the rows to assemble (device)
    int64_t row_count;
};
constexpr int ASM_ROW_CAP = 512;   // row kernel: longest row summed in shared memory

struct AdjArgs {
    const double *vertices;
    const int32_t *cells;
    int64_t n_cells;
    int64_t n_vertices;
    int d;
    const double *kappa;
    const double *weights;
    int n_q;
    int n_phi;
    const double *dphi;       // [d][n_phi][n_q]
    const int32_t *cell_dofs; // [n_cells][n_phi]
    const float *u;
    const float *v;
    double *g_kappa;
    double *g_cell_x;         // per-cell vertex gradients [n_cells][d+1][d] (scratch)
    double *L_cell;           // per-cell L contribution [n_cells] (scratch)
    int *status;
};

// One form's action on a FE function (Algorithm 2) over one plan.
struct ActArgs {
    const double *vertices;
    const int32_t *cells;
    const int32_t *cell_dofs;  // [n_cells][n_phi]
    int64_t n_cells;
    int d, n_phi, n_q;
    int form;                  // warp-per-cell kernel: FE_FORM_MASS or FE_FORM_STIFFNESS
    int forms;                 // thread-per-cell kernel: bit 0 Poisson, bit 1 mass
    int prec;                  // FE_PREC_FP64 or a storage format
    const double *kappa;       // [n_cells][n_q]
    const double *weights;     // [n_q]
    const double *w;           // [n_dofs] global coefficients
    // Tables: the thread-per-cell kernel (action_per_cell) reads tab only, packed
    // [n_q][act_row_floats]: per point, the Poisson segments s = 0 .. d-1 (if
    // requested) then the mass segment (if requested), each act_seg_floats long
    // (entries k = 0 .. n_phi-1, zero-padded).  The warp-per-cell kernel reads tab
    // [n_d][n_phi][n_q] and tab_t [n_d][n_q][n_phi].  Double for FP64, else float
    // values rounded to the storage format.
    const void *tab;
    const void *tab_t;
    void *b;                   // [n_cells][n_phi] cell vectors (double or float): the form, or Poisson
    void *b_mass;              // thread-per-cell kernel: the mass form's cell vectors
    int *status;
    int qw;                    // quadrature points per shared-memory window (thread-per-cell kernel)
    // FP16 range scaling (prec == FE_PREC_FP16 only; see fe_action.cu): per form
    // (0 Poisson, 1 mass) max_q w_q * max_{s,q} sum_k |B_skq| * 2^ACT_W_TARGET, the
    // a-priori bound on |r_s| / (kappa * gnorm) (gnorm = max_s sum_t |G_st|, mass: |det J|)
    float r_bound[2];
};
// Target binades of the per-cell scales of the FP16 action: the cell's
// coefficients to max|w^c| 2^e_w in [2^(W-1), 2^W), the a-priori bound of r_s
// to [2^(R-1), 2^R) (so r_s stays finite for kappa below 2^(15-R) 65504/2^15).
constexpr int ACT_W_TARGET = 8;
constexpr int ACT_R_TARGET = 4;

// Packed action table: floats per segment (one derivative direction, or the
// basis values, over the local dofs, padded to a multiple of 4) and per
// quadrature point for the requested forms (bit 0 Poisson: d segments; bit 1
// mass: one segment).
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int act_seg_floats(int n_phi) { return (n_phi + 3) / 4 * 4; }
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int act_row_floats(int d, int n_phi, int forms) {
    return act_seg_floats(n_phi) * (((forms & 1) ? d : 0) + ((forms & 2) ? 1 : 0));
}
constexpr int kActSmemTarget = 48 * 1024;   // shared memory per CTA the quadrature window is sized for

// Kernel launchers (defined in the .cu files).  Return the number of
// kernel launches made, or a negative cudaError_t on launch failure.
int launch_tc_elements(const TcArgs &a, size_t smem_bytes, cudaStream_t s, int grid = 0);
// Geometry, coefficient window and per-cell scales of every tile (the factor
// kernel; run before launch_tc_elements on the same arguments).
int launch_factor(const TcArgs &a, cudaStream_t s);
size_t tc_smem_bytes(const TcArgs &a);
int launch_action(const ActArgs &a, bool fp64, cudaStream_t s);
size_t action_smem_bytes(const ActArgs &a, bool fp64);
// Whether the thread-per-cell action kernel serves (d, n_phi, precision), and
// its quadrature window for the requested forms.
bool action_per_cell(int d, int n_phi, bool fp64);
int action_window(int d, int n_phi, int n_q, int forms);
// v0 = L b0 (and v1 = L b1 when b1 is not NULL) in one launch.
int launch_vector_assemble(int64_t n_dofs, const int64_t *inc_ptr, const int32_t *inc_elem, const void *b0,
                           const void *b1, void *v0, void *v1, bool fp64, cudaStream_t s);
// Whether a segment can use the staged epilogue under the given global shape.
bool tc_can_stage(const TcArgs &a, const TcSeg &seg);
int launch_f64_elements(const F64Args &a, cudaStream_t s);
// Boxed cells: G pairs and |det J| at every quadrature point in FP64 into
// geo_q [n_cells][n_q][7] (the per-point geometry of the FP64 path).
int launch_box_geometry(const double *vertices, const int32_t *cells, int64_t n_cells, int d, int nv,
                        const double *dpsi, int n_q, double *geo_q, int *status, cudaStream_t s);
int launch_assemble(const AsmArgs &a, bool fp64, cudaStream_t s);
// Capacity (in doubles) of the fixed scratch array of the allocation-free
// adjoint, and the lookup of its device address on the current device.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 22;  // 32 MiB
cudaError_t noalloc_scratch(double **ptr);
// Diagnostic kernels (fe_diag.cu): the geometry tensor of cells [c0, c1) in
// FP64 (mode 0), exclusively FP32 (1) or the production mixed path (2); and the
// mass form / action with FP16 products and sums.
int launch_diag_geometry(const double *vertices, const int32_t *cells, int64_t c0, int64_t c1, int d, int mode,
                         double *G, double *absdet, int32_t *used_fp64, int *status, cudaStream_t s);
int launch_diag_mass_fp16(const double *vertices, const int32_t *cells, const int32_t *cell_dofs, int64_t c0,
                          int64_t c1, int d, int n_phi, int n_q, const double *kappa, const double *weights,
                          const double *phi, const double *w, float *A, float *b, int *status, cudaStream_t s);
int launch_adjoint(const AdjArgs &a, const int64_t *vert_inc_ptr, const int32_t *vert_inc, double *g_vertices,
                   double *L_out, cudaStream_t s);

}  // namespace fe
