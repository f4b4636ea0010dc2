// C ABI of the library: plan lifecycle, argument validation, device memory
// owned by plans, kernel launches and the status / error conventions of
// fe_gb300.h.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "fe_adjoint.h"
#include "fe_host.h"
#include "fe_internal.h"

static_assert(fe::host::kAsmChunkEntries == fe::ASM_CHUNK && fe::host::kAsmChunkIncidences == fe::ASM_CHUNK_INC,
              "host and device assembly chunk limits differ");

using namespace fe;

namespace {

thread_local std::string g_err;

fe_status fail(fe_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

fe_status cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) return fail(FE_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(FE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define FE_CUDA(call, what)                          \
    do {                                             \
        cudaError_t _e = (call);                     \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

int form_index(unsigned form) { return form == FE_FORM_STIFFNESS ? 0 : 1; }

bool supported_degree(int d, int p, bool boxed = false) {
    if (boxed) return p >= 1 && ((d == 3 && p <= 5) || (d == 2 && p <= 8));
    return p >= 1 && ((d == 3 && p <= 8) || (d == 2 && p <= 10));
}

// Dimension and kind of a cell type (0 for an unknown type).
int cell_dim(fe_cell_type t, bool &boxed) {
    boxed = (t == FE_QUADRILATERAL || t == FE_HEXAHEDRON);
    switch (t) {
        case FE_TRIANGLE: case FE_QUADRILATERAL: return 2;
        case FE_TETRAHEDRON: case FE_HEXAHEDRON: return 3;
        default: return 0;
    }
}

// Default limit on how long one bounded wait inside a kernel may see no
// progress before the kernel gives up (fe_plan_set_wait_limit).
constexpr unsigned long long kDefaultWaitLimitNs = 2000000000ull;

}  // namespace

struct fe_pattern {
    host::Pattern P;
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t b) {
        if (p && bytes >= b) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, b ? b : 16);
        if (e == cudaSuccess) bytes = b;
        return e;
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

struct fe_plan {
    int d = 0, p = 0, n_phi = 0, n_q = 0, n_pairs = 0, n_sym = 0;
    bool boxed = false;                  // quadrilaterals / hexahedra: geometry per quadrature point
    bool elements_only = false;          // FE_PLAN_ELEMENTS_ONLY: no dof map, pattern or assembly streams
    int nv = 0;                          // vertices per cell
    DevBuf dpsi_box;                     // boxed: Q1 derivatives at the rule's points [d][nv][n_q]
    DevBuf ws_geoq;                      // boxed FP64 path: G pairs and |det J| per point [n_cells][n_q][7]
    // fused assembly: cells in slices of fuse_cells, element matrices in a ring of
    // fuse_slots slices, the chunks of each slice (device list + host offsets)
    int64_t fuse_cells = 0;
    int fuse_slots = 0, fuse_slices = 0;
    bool fuse_ok = false;
    DevBuf fuse_rows, ws_ring[2];
    std::vector<int64_t> fuse_row_off;
    DevBuf inc_slot;                     // [n_inc][n_phi] column slots (row-wise assembly)
    int asm_algo = 0;                    // fe_plan_set_assembly: 0 chunked segments (default), 1 one warp per row
    int wpref_mode = -1;                 // fe_plan_set_window_prefetch: -1 tuned, 0 off, 1 on
    // fe_assemble_host: the assembly in kHostPieces ranges of chunks (consecutive
    // rows), whose CSR values leave for the host while the next range is summed
    std::vector<int64_t> piece_chunk;    // [pieces + 1] first chunk of each range
    std::vector<int64_t> piece_val;      // [pieces + 1] first CSR value of each range
    DevBuf chunk_iota;                   // [n_chunks] 0, 1, 2, ... (chunk lists of the ranges)
    cudaEvent_t piece_done[8] = {};
    bool pieces_ready = false;
    int fuse_mode = 0;                   // fe_plan_set_fusion: 1 on where eligible, 0 off (default)
    unsigned form_mask = 0, prec_mask = 0;
    int64_t n_cells = 0, n_vertices = 0, n_dofs = 0, nnz = 0;
    int max_row = 0;
    cudaStream_t stream = nullptr;
    int sms = 0;
    DevBuf vertices, cells, weights, cell_dofs, row_ptr, col_idx, inc_ptr, inc_elem, vinc_ptr, vinc;
    DevBuf contrib_cnt, contrib_base, contrib_code, contrib_dest, chunk_desc;
    int64_t n_chunks = 0;                // assembly row chunks
    DevBuf phi, dphi, sym_kl, full2sym, status;
    DevBuf img[6][2];
    TcOperand op[6][2];
    DevBuf ws_elem[2], ws_kappa, ws_csr[2], ws_adj_x, ws_adj_L, ws_Lsum;
    DevBuf ws_win, ws_cellf;             // factor kernel outputs (window, per-cell factors)
    DevBuf act_tab[6][2], act_tab_t[6][2];  // warp-per-cell action tables per precision and form (B, transposed B)
    DevBuf act_packed[6][3];                // thread-per-cell action tables per precision and forms mask - 1
    DevBuf ws_act_b[2];                  // action cell vectors when the caller keeps none
    bool timing = false;
    cudaEvent_t ev[8] = {};
    float stage_ms[4] = {0, 0, 0, 0};
    int last_launches = 0;
    int stage_marks = 0;
    std::vector<int> host_status;
    std::vector<double> h_phi, h_dphi;   // FP64 tabulation kept for re-packing operands
    std::vector<int> col_of_sym;         // operand column of each pair (k <= l)
    int tuned_np[6][2] = {};             // autotuned N-pass width per precision and form
    unsigned long long wait_limit_ns = kDefaultWaitLimitNs;   // no-progress limit of every bounded kernel wait
    float act_rbound[2] = {0.f, 0.f};    // FP16 action scaling bounds (ActArgs::r_bound)
    // pipelined host path (fe_assemble_host_many): two slots of device inputs and outputs,
    // an upload and a download stream, and the events that order them
    DevBuf ws_pipe_kappa[2], ws_pipe_csr[2][2];
    bool pipe_ready = false;
    cudaStream_t pipe_h2d = nullptr, pipe_d2h = nullptr;
    cudaEvent_t pipe_in[2] = {}, pipe_used[2] = {}, pipe_out[2] = {};
    ~fe_plan() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        for (int i = 0; i < 2; ++i)
            for (cudaEvent_t e : {pipe_in[i], pipe_used[i], pipe_out[i]})
                if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : piece_done)
            if (e) cudaEventDestroy(e);
        if (pipe_h2d) cudaStreamDestroy(pipe_h2d);
        if (pipe_d2h) cudaStreamDestroy(pipe_d2h);
    }
};

static uint32_t idesc_for(int prec) {
    uint32_t fmt = 0;
    if (prec == FE_PREC_BF16) fmt = 1;
    else if (prec == FE_PREC_TF32 || prec == FE_PREC_TF32X3) fmt = 2;
    else fmt = 0;  // FP16, E4M3
    uint32_t d = (1u << 4);                     // FP32 accumulator
    d |= (fmt << 7) | (fmt << 10);              // A and B formats
    d |= (uint32_t)(TC_M >> 4) << 24;           // M = 128
    return d;
}

template <class T>
static cudaError_t upload(DevBuf &b, const std::vector<T> &v, cudaStream_t s) {
    cudaError_t e = b.alloc(sizeof(T) * v.size());
    if (e != cudaSuccess) return e;
    if (v.empty()) return cudaSuccess;
    return cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s);
}

static fe_status pack_operand(fe_plan &P, int prec, int fi, int np_pass);
// ranges of the assembly in fe_assemble_host, each downloaded as soon as it is summed
constexpr int kHostPieces = 4;
static fe_status autotune_plan(fe_plan &P);
static fe_status need_pattern(const fe_plan *plan);
static fe_status check_call(fe_plan *plan, unsigned forms, fe_precision prec);
static TcSeg make_tc_seg(fe_plan *P, unsigned forms, int prec, const double *vertices, const double *kappa,
                         void *const A[2], float *win, float *cellf);
static void tc_finalize(TcArgs &a, TcSeg *segs, int n, int prec, int *status, unsigned long long wait_limit_ns);

extern "C" {

const char *fe_last_error(void) { return g_err.c_str(); }

fe_status fe_quadrature_rule(fe_cell_type type, int family, int m, int32_t *n_q, double *points, double *weights) {
    g_err.clear();
    if (!n_q) return fail(FE_ERR_INVALID_ARG, "n_q is NULL");
    bool boxed = false;
    const int d = cell_dim(type, boxed);
    if (d == 0) return fail(FE_ERR_INVALID_ARG, "unknown cell type %d", (int)type);
    if (family == FE_QUAD_GAUSS_LEGENDRE_TENSOR) {
        if (!boxed) return fail(FE_ERR_INVALID_ARG, "the tensor Gauss-Legendre rule is for boxed cells");
        if (m < 1 || m > 32) return fail(FE_ERR_UNSUPPORTED, "m must lie in 1..32");
        int nq = 1;
        for (int i = 0; i < d; ++i) nq *= m;
        *n_q = nq;
        if (!points || !weights) return FE_OK;
        std::vector<double> pts, wts;
        if (!host::tensor_rule(d, m, pts, wts)) return fail(FE_ERR_INVALID_ARG, "rule construction failed");
        std::memcpy(points, pts.data(), sizeof(double) * pts.size());
        std::memcpy(weights, wts.data(), sizeof(double) * wts.size());
        return FE_OK;
    }
    if (boxed) return fail(FE_ERR_INVALID_ARG, "boxed cells take FE_QUAD_GAUSS_LEGENDRE_TENSOR");
    if (family == FE_QUAD_TRIANGLE_3POINT) {
        if (d != 2) return fail(FE_ERR_INVALID_ARG, "the 3-point rule is for triangles");
        *n_q = 3;
        if (points && weights) {
            const double P[6] = {1.0 / 6, 1.0 / 6, 2.0 / 3, 1.0 / 6, 1.0 / 6, 2.0 / 3};
            for (int i = 0; i < 6; ++i) points[i] = P[i];
            for (int i = 0; i < 3; ++i) weights[i] = 1.0 / 6;
        }
        return FE_OK;
    }
    if (family != FE_QUAD_COLLAPSED_GAUSS_JACOBI) return fail(FE_ERR_INVALID_ARG, "unknown family %d", family);
    if (m < 1 || m > 32) return fail(FE_ERR_UNSUPPORTED, "m must lie in 1..32");
    int nq = 1;
    for (int i = 0; i < d; ++i) nq *= m;
    *n_q = nq;
    if (!points || !weights) return FE_OK;
    std::vector<double> pts, wts;
    if (!host::collapsed_rule(d, m, pts, wts)) return fail(FE_ERR_INVALID_ARG, "rule construction failed");
    std::memcpy(points, pts.data(), sizeof(double) * pts.size());
    std::memcpy(weights, wts.data(), sizeof(double) * wts.size());
    return FE_OK;
}

fe_status fe_pattern_create(fe_pattern **out, fe_cell_type type, int64_t n_vertices, int64_t n_cells,
                            const int32_t *cells, int degree) {
    g_err.clear();
    if (!out || !cells) return fail(FE_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    bool boxed = false;
    const int d = cell_dim(type, boxed);
    if (d == 0) return fail(FE_ERR_INVALID_ARG, "unknown cell type %d", (int)type);
    if (!supported_degree(d, degree, boxed)) return fail(FE_ERR_UNSUPPORTED, "degree %d not supported", degree);
    if (n_vertices <= 0 || n_cells <= 0) return fail(FE_ERR_INVALID_ARG, "empty mesh");
    auto pat = std::make_unique<fe_pattern>();
    std::string err = host::build_pattern(d, degree, n_vertices, n_cells, cells, pat->P, false, boxed);
    if (!err.empty()) return fail(FE_ERR_INVALID_ARG, "%s", err.c_str());
    *out = pat.release();
    return FE_OK;
}

fe_status fe_pattern_sizes(const fe_pattern *pat, int64_t *n_dofs, int64_t *nnz, int32_t *n_phi, int32_t *max_row) {
    if (!pat) return fail(FE_ERR_INVALID_ARG, "NULL pattern");
    if (n_dofs) *n_dofs = pat->P.n_dofs;
    if (nnz) *nnz = pat->P.nnz;
    if (n_phi) *n_phi = pat->P.n_phi;
    if (max_row) *max_row = pat->P.max_row;
    return FE_OK;
}

fe_status fe_pattern_copy(const fe_pattern *pat, int32_t *cell_dofs, int64_t *row_ptr, int32_t *col_idx) {
    if (!pat) return fail(FE_ERR_INVALID_ARG, "NULL pattern");
    const auto &P = pat->P;
    if (cell_dofs) std::memcpy(cell_dofs, P.cell_dofs.data(), sizeof(int32_t) * P.cell_dofs.size());
    if (row_ptr) std::memcpy(row_ptr, P.row_ptr.data(), sizeof(int64_t) * P.row_ptr.size());
    if (col_idx) std::memcpy(col_idx, P.col_idx.data(), sizeof(int32_t) * P.col_idx.size());
    return FE_OK;
}

fe_status fe_pattern_destroy(fe_pattern *pat) {
    delete pat;
    return FE_OK;
}

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
fe_status fe_plan_create(fe_plan **out, const fe_mesh *mesh, int degree, const fe_quadrature *rule,
                         unsigned form_mask, unsigned prec_mask, void *cuda_stream) {
    g_err.clear();
    if (!out || !mesh || !rule || !mesh->vertices || !mesh->cells || !rule->points || !rule->weights)
        return fail(FE_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    bool boxed = false;
    const int d = cell_dim(mesh->type, boxed);
    if (d == 0) return fail(FE_ERR_INVALID_ARG, "unknown cell type %d", (int)mesh->type);
    if (!supported_degree(d, degree, boxed))
        return fail(FE_ERR_UNSUPPORTED, "degree %d not supported for this cell type", degree);
    if (mesh->n_vertices <= 0 || mesh->n_cells <= 0) return fail(FE_ERR_INVALID_ARG, "empty mesh");
    if (rule->n_q <= 0 || rule->n_q > 4096) return fail(FE_ERR_UNSUPPORTED, "n_q must lie in 1..4096");
    const bool elements_only = (form_mask & FE_PLAN_ELEMENTS_ONLY) != 0;
    form_mask &= ~(unsigned)FE_PLAN_ELEMENTS_ONLY;
    if (form_mask == 0 || (form_mask & ~3u)) return fail(FE_ERR_INVALID_ARG, "bad form mask");
    if (prec_mask == 0 || (prec_mask & ~63u)) return fail(FE_ERR_INVALID_ARG, "bad precision mask");
    for (int64_t i = 0; i < mesh->n_vertices * d; ++i)
        if (!std::isfinite(mesh->vertices[i])) return fail(FE_ERR_NONFINITE, "non-finite vertex coordinate");
    for (int i = 0; i < rule->n_q; ++i)
        if (!std::isfinite(rule->weights[i])) return fail(FE_ERR_NONFINITE, "non-finite quadrature weight");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(FE_ERR_NO_DEVICE, "no CUDA device");
    }
    auto pl = std::make_unique<fe_plan>();
    fe_plan &P = *pl;
    P.d = d;
    P.p = degree;
    P.boxed = boxed;
    P.nv = boxed ? (1 << d) : d + 1;
    P.n_phi = boxed ? host::n_phi_box(d, degree) : host::n_phi(d, degree);
    P.n_q = rule->n_q;
    P.n_pairs = d * (d + 1) / 2;
    P.n_sym = P.n_phi * (P.n_phi + 1) / 2;
    P.form_mask = form_mask;
    P.prec_mask = prec_mask;
    P.n_cells = mesh->n_cells;
    P.n_vertices = mesh->n_vertices;
    P.stream = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&P.sms, cudaDevAttrMultiProcessorCount, dev);

    if ((int64_t)mesh->n_cells * P.n_phi * P.n_phi >= INT32_MAX)
        return fail(FE_ERR_UNSUPPORTED, "n_cells * n_phi^2 must stay below 2^31 (32-bit element offsets)");
    host::Pattern pat;
    // slices of one wave of tiles for the fused assembly
    P.fuse_cells = (int64_t)std::max(1, P.sms) * TC_M;
    P.elements_only = elements_only;
    if (elements_only) {
        // no dof map, pattern or assembly streams: check the connectivity only
        for (int64_t i = 0; i < mesh->n_cells * P.nv; ++i)
            if (mesh->cells[i] < 0 || mesh->cells[i] >= mesh->n_vertices)
                return fail(FE_ERR_INVALID_ARG, "cell vertex index out of range");
        pat.chunk_row.assign(1, 0);
        pat.inc_ptr.assign(1, 0);
    } else {
        std::string err =
            host::build_pattern(d, degree, mesh->n_vertices, mesh->n_cells, mesh->cells, pat, true, boxed);
        if (!err.empty()) return fail(FE_ERR_INVALID_ARG, "%s", err.c_str());
    }
    P.n_dofs = pat.n_dofs;
    P.nnz = pat.nnz;
    P.max_row = pat.max_row;
    P.n_chunks = (int64_t)pat.chunk_row.size() - 1;
    if (!elements_only) {
        const int pieces = (int)std::min<int64_t>(kHostPieces, std::max<int64_t>(1, P.n_chunks));
        for (int k = 0; k <= pieces; ++k) {
            const int64_t c = P.n_chunks * k / pieces;
            P.piece_chunk.push_back(c);
            P.piece_val.push_back(pat.row_ptr[c < P.n_chunks ? pat.chunk_row[c] : pat.n_dofs]);
        }
    }

    std::vector<double> phi, dphi, psi_box, dpsi_box;
    if (boxed) {
        host::tabulate_box(d, degree, rule->points, rule->n_q, phi, dphi);
        host::tabulate_box(d, 1, rule->points, rule->n_q, psi_box, dpsi_box);   // the multilinear map
    } else {
        host::tabulate(d, degree, rule->points, rule->n_q, phi, dphi);
    }

    cudaStream_t s = P.stream;
    std::vector<double> verts(mesh->vertices, mesh->vertices + mesh->n_vertices * d);
    std::vector<int32_t> cl(mesh->cells, mesh->cells + mesh->n_cells * P.nv);
    std::vector<double> wts(rule->weights, rule->weights + rule->n_q);
    FE_CUDA(upload(P.vertices, verts, s), "upload vertices");
    FE_CUDA(upload(P.cells, cl, s), "upload cells");
    FE_CUDA(upload(P.weights, wts, s), "upload weights");
    FE_CUDA(upload(P.cell_dofs, pat.cell_dofs, s), "upload dofs");
    FE_CUDA(upload(P.row_ptr, pat.row_ptr, s), "upload row_ptr");
    FE_CUDA(upload(P.col_idx, pat.col_idx, s), "upload col_idx");
    FE_CUDA(upload(P.inc_ptr, pat.inc_ptr, s), "upload inc_ptr");
    FE_CUDA(upload(P.inc_elem, pat.inc_elem, s), "upload inc_elem");
    FE_CUDA(upload(P.contrib_cnt, pat.contrib_cnt, s), "upload contribution counts");
    FE_CUDA(upload(P.contrib_base, pat.contrib_base, s), "upload contribution bases");
    FE_CUDA(upload(P.contrib_code, pat.contrib_code, s), "upload contribution codes");
    FE_CUDA(upload(P.contrib_dest, pat.contrib_dest, s), "upload contribution destinations");
    FE_CUDA(upload(P.chunk_desc, pat.chunk_desc, s), "upload assembly chunks");
    FE_CUDA(upload(P.inc_slot, pat.inc_slot, s), "upload column slots");
    FE_CUDA(upload(P.vinc_ptr, pat.vinc_ptr, s), "upload vinc_ptr");
    FE_CUDA(upload(P.vinc, pat.vinc, s), "upload vinc");
    FE_CUDA(upload(P.phi, phi, s), "upload phi");
    FE_CUDA(upload(P.dphi, dphi, s), "upload dphi");
    if (boxed) FE_CUDA(upload(P.dpsi_box, dpsi_box, s), "upload Q1 derivatives");
    // operand column of every pair (k <= l): a bank-conflict-free order for the
    // staged epilogue's gathers; sym_kl maps a column back to its pair (-1: padding)
    P.col_of_sym = host::stage_columns(P.n_phi, (P.n_phi * P.n_phi) % 4 == 0);
    std::vector<int32_t> symkl((size_t)(P.n_sym + 15) / 16 * 16, -1);
    std::vector<int16_t> f2s((size_t)P.n_phi * P.n_phi);
    {
        int pr = 0;
        for (int k = 0; k < P.n_phi; ++k)
            for (int l = k; l < P.n_phi; ++l, ++pr) {
                const int col = P.col_of_sym[pr];
                f2s[(size_t)k * P.n_phi + l] = f2s[(size_t)l * P.n_phi + k] = (int16_t)col;
                symkl[col] = k | (l << 16);
            }
    }
    if (P.n_sym > 32767) f2s.assign(f2s.size(), 0);  // only used by single-pass shapes (n_sym <= 256)
    FE_CUDA(upload(P.sym_kl, symkl, s), "upload sym table");
    FE_CUDA(upload(P.full2sym, f2s, s), "upload sym map");
    std::vector<int> zero(4, 0);
    FE_CUDA(upload(P.status, zero, s), "status word");

    // fused assembly (fe_assemble without element-matrix outputs): used when the
    // mesh spans several slices and the ring of element matrices of
    // slice_span slices (both forms) fits in a third of the L2 cache
    {
        P.fuse_slices = (int)((P.n_cells + P.fuse_cells - 1) / P.fuse_cells);
        // the widest range of slices one row's cells span (incidences are in cell order)
        P.fuse_slots = 0;
        for (int64_t i = 0; i < P.n_dofs; ++i)
            if (pat.inc_ptr[i + 1] > pat.inc_ptr[i]) {
                const int64_t lo = (pat.inc_elem[pat.inc_ptr[i]] / P.n_phi) / P.fuse_cells;
                const int64_t hi = (pat.inc_elem[pat.inc_ptr[i + 1] - 1] / P.n_phi) / P.fuse_cells;
                P.fuse_slots = std::max<int>(P.fuse_slots, (int)(hi - lo + 1));
            }
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        int nf = 0;
        for (unsigned f : {(unsigned)FE_FORM_STIFFNESS, (unsigned)FE_FORM_MASS}) nf += (form_mask & f) ? 1 : 0;
        const double ring = (double)P.fuse_slots * P.fuse_cells * P.n_phi * P.n_phi * 4.0 * nf;
        P.fuse_ok = P.fuse_slices >= 2 && P.fuse_slots >= 1 && P.fuse_slots <= 3 && l2 > 0 && ring <= l2 / 3.0;
        if (P.fuse_ok) {
            // rows grouped by the slice of their last cell (the row-wise kernel's lists)
            std::vector<int32_t> rows((size_t)P.n_dofs);
            std::vector<int32_t> rs((size_t)P.n_dofs, 0);
            for (int64_t i = 0; i < P.n_dofs; ++i) {
                rows[i] = (int32_t)i;
                if (pat.inc_ptr[i + 1] > pat.inc_ptr[i])
                    rs[i] = (int32_t)((pat.inc_elem[pat.inc_ptr[i + 1] - 1] / P.n_phi) / P.fuse_cells);
            }
            std::stable_sort(rows.begin(), rows.end(), [&](int32_t x, int32_t y) { return rs[x] < rs[y]; });
            P.fuse_row_off.assign(P.fuse_slices + 1, 0);
            for (int64_t i = 0; i < P.n_dofs; ++i) P.fuse_row_off[rs[i] + 1]++;
            for (int sl = 0; sl < P.fuse_slices; ++sl) P.fuse_row_off[sl + 1] += P.fuse_row_off[sl];
            FE_CUDA(upload(P.fuse_rows, rows, s), "upload fused row lists");
        }
    }
    P.h_phi = phi;
    P.h_dphi = dphi;
    {
        // a-priori bounds of the FP16 action's r_s (ActArgs::r_bound): the largest
        // weight times max_{s,q} sum_k |B_skq| times 2^ACT_W_TARGET
        double wmax = 0.0, bs = 0.0, bm = 0.0;
        for (int q = 0; q < P.n_q; ++q) {
            wmax = std::max(wmax, std::fabs(rule->weights[q]));
            double m = 0.0;
            for (int k = 0; k < P.n_phi; ++k) m += std::fabs(phi[(size_t)k * P.n_q + q]);
            bm = std::max(bm, m);
            for (int sd = 0; sd < d; ++sd) {
                double g = 0.0;
                for (int k = 0; k < P.n_phi; ++k) g += std::fabs(dphi[((size_t)sd * P.n_phi + k) * P.n_q + q]);
                bs = std::max(bs, g);
            }
        }
        P.act_rbound[0] = (float)std::ldexp(wmax * bs, ACT_W_TARGET);
        P.act_rbound[1] = (float)std::ldexp(wmax * bm, ACT_W_TARGET);
    }
    for (int prec = 1; prec <= 5; ++prec) {
        if (!(prec_mask & FE_PREC_MASK(prec))) continue;
        for (unsigned form : {(unsigned)FE_FORM_STIFFNESS, (unsigned)FE_FORM_MASS}) {
            if (!(form_mask & form)) continue;
            fe_status st = pack_operand(P, prec, form_index(form), 0);
            if (st) return st;
        }
    }
    FE_CUDA(cudaStreamSynchronize(s), "plan upload");
    for (auto &e : P.ev) FE_CUDA(cudaEventCreate(&e), "event");
    {
        fe_status st = autotune_plan(P);
        if (st) return st;
    }
    *out = pl.release();
    return FE_OK;
}

fe_status fe_plan_destroy(fe_plan *plan) {
    if (plan) {
        cudaStreamSynchronize(plan->stream);
        delete plan;
    }
    return FE_OK;
}

fe_status fe_plan_set_stream(fe_plan *plan, void *stream) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    plan->stream = static_cast<cudaStream_t>(stream);
    return FE_OK;
}

fe_status fe_plan_memory(const fe_plan *plan, int64_t *plan_bytes, int64_t *workspace_bytes) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    const fe_plan &P = *plan;
    const DevBuf *ws[] = {&P.ws_elem[0], &P.ws_elem[1], &P.ws_kappa, &P.ws_csr[0], &P.ws_csr[1], &P.ws_adj_x,
                          &P.ws_adj_L, &P.ws_Lsum, &P.ws_win, &P.ws_cellf, &P.ws_act_b[0], &P.ws_act_b[1]};
    int64_t w = 0;
    for (const DevBuf *b : ws) w += (int64_t)b->bytes;
    for (int i = 0; i < 2; ++i)
        w += (int64_t)(P.ws_pipe_kappa[i].bytes + P.ws_pipe_csr[i][0].bytes + P.ws_pipe_csr[i][1].bytes);
    w += (int64_t)P.ws_geoq.bytes + (int64_t)P.ws_ring[0].bytes + (int64_t)P.ws_ring[1].bytes;
    int64_t t = 0;
    const DevBuf *own[] = {&P.vertices, &P.cells, &P.weights, &P.cell_dofs, &P.row_ptr, &P.col_idx, &P.inc_ptr,
                           &P.inc_elem, &P.vinc_ptr, &P.vinc, &P.contrib_cnt, &P.contrib_base, &P.contrib_code,
                           &P.contrib_dest, &P.chunk_desc, &P.phi, &P.dphi, &P.sym_kl, &P.full2sym, &P.status,
                           &P.fuse_rows, &P.inc_slot, &P.dpsi_box};
    for (const DevBuf *b : own) t += (int64_t)b->bytes;
    for (int i = 0; i < 6; ++i)
        for (int f = 0; f < 2; ++f) t += (int64_t)(P.img[i][f].bytes + P.act_tab[i][f].bytes + P.act_tab_t[i][f].bytes);
    for (int i = 0; i < 6; ++i)
        for (int f = 0; f < 3; ++f) t += (int64_t)P.act_packed[i][f].bytes;
    if (plan_bytes) *plan_bytes = t;
    if (workspace_bytes) *workspace_bytes = w;
    return FE_OK;
}

fe_status fe_plan_set_assembly(fe_plan *plan, int algo) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    if (algo != 0 && algo != 1) return fail(FE_ERR_INVALID_ARG, "algo must be 0 or 1");
    plan->asm_algo = algo;
    return FE_OK;
}

fe_status fe_plan_set_window_prefetch(fe_plan *plan, int mode) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    if (mode < -1 || mode > 1) return fail(FE_ERR_INVALID_ARG, "mode must be -1 (tuned), 0 (off) or 1 (on)");
    plan->wpref_mode = mode;
    return FE_OK;
}

fe_status fe_plan_set_rows_per_pass(fe_plan *plan, fe_precision prec, unsigned forms, int rows) {
    g_err.clear();
    fe_status st = check_call(plan, forms, prec);
    if (st) return st;
    if (prec == FE_PREC_FP64) return fail(FE_ERR_INVALID_ARG, "the FP64 path has no N layout");
    if (rows < 1 || rows > plan->n_phi || rows * plan->n_phi > 2 * TC_MAX_NP)
        return fail(FE_ERR_INVALID_ARG, "rows must lie in 1..min(n_phi, 512 / n_phi)");
    for (int fi = 0; fi < 2; ++fi)
        if (forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS)) {
            const int wp = plan->op[prec][fi].win_pref;
            st = pack_operand(*plan, prec, fi, -rows);
            if (st) return st;
            plan->op[prec][fi].win_pref = wp;
        }
    FE_CUDA(cudaStreamSynchronize(plan->stream), "operand upload");
    return FE_OK;
}

fe_status fe_plan_tc_config(fe_plan *plan, unsigned forms, fe_precision prec, int32_t *ring_a, int32_t *ring_b,
                            int32_t *win_buf, int32_t *staged, int32_t *n_acc) {
    g_err.clear();
    fe_status st = check_call(plan, forms, prec);
    if (st) return st;
    if (prec == FE_PREC_FP64) return fail(FE_ERR_INVALID_ARG, "the FP64 path does not use the tensor-core kernel");
    TcArgs a{};
    void *A[2] = {nullptr, nullptr};
    a.seg0 = make_tc_seg(plan, forms, prec, nullptr, nullptr, A, nullptr, nullptr);
    a.segs = nullptr;
    a.n_segs = 1;
    tc_finalize(a, &a.seg0, 1, prec, nullptr, plan->wait_limit_ns);
    if (ring_a) *ring_a = a.ring_a;
    if (ring_b) *ring_b = a.ring_b;
    if (win_buf) *win_buf = a.win_buf;
    if (staged) *staged = a.seg0.staged;
    if (n_acc) *n_acc = a.n_acc;
    return FE_OK;
}

fe_status fe_plan_set_fusion(fe_plan *plan, int mode, int *active) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    if (mode != 0 && mode != 1) return fail(FE_ERR_INVALID_ARG, "mode must be 1 (on) or 0 (off)");
    plan->fuse_mode = mode;
    if (active) *active = (plan->fuse_ok && mode == 1) ? 1 : 0;
    return FE_OK;
}

fe_status fe_plan_set_wait_limit(fe_plan *plan, uint64_t limit_ns) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    plan->wait_limit_ns = limit_ns ? (unsigned long long)limit_ns : kDefaultWaitLimitNs;
    return FE_OK;
}

fe_status fe_plan_sizes(const fe_plan *plan, int64_t *n_cells, int64_t *n_vertices, int64_t *n_dofs, int64_t *nnz,
                        int32_t *n_phi, int32_t *n_q) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    if (n_cells) *n_cells = plan->n_cells;
    if (n_vertices) *n_vertices = plan->n_vertices;
    if (n_dofs) *n_dofs = plan->n_dofs;
    if (nnz) *nnz = plan->nnz;
    if (n_phi) *n_phi = plan->n_phi;
    if (n_q) *n_q = plan->n_q;
    return FE_OK;
}

fe_status fe_csr_pattern(const fe_plan *plan, int64_t *row_ptr, int32_t *col_idx) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    if (need_pattern(plan)) return FE_ERR_INVALID_ARG;
    if (row_ptr)
        FE_CUDA(cudaMemcpyAsync(row_ptr, plan->row_ptr.p, sizeof(int64_t) * (plan->n_dofs + 1),
                                cudaMemcpyDeviceToDevice, plan->stream), "copy row_ptr");
    if (col_idx)
        FE_CUDA(cudaMemcpyAsync(col_idx, plan->col_idx.p, sizeof(int32_t) * plan->nnz, cudaMemcpyDeviceToDevice,
                                plan->stream), "copy col_idx");
    return FE_OK;
}

fe_status fe_cell_dofs(const fe_plan *plan, int32_t *cell_dofs) {
    if (!plan || !cell_dofs) return fail(FE_ERR_INVALID_ARG, "NULL argument");
    if (need_pattern(plan)) return FE_ERR_INVALID_ARG;
    FE_CUDA(cudaMemcpyAsync(cell_dofs, plan->cell_dofs.p, sizeof(int32_t) * plan->n_cells * plan->n_phi,
                            cudaMemcpyDeviceToDevice, plan->stream), "copy dofs");
    return FE_OK;
}

fe_status fe_plan_enable_timing(fe_plan *plan, int enable) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    plan->timing = enable != 0;
    return FE_OK;
}

fe_status fe_plan_stage_times(fe_plan *plan, float *ms, int n) {
    if (!plan || !ms) return fail(FE_ERR_INVALID_ARG, "NULL argument");
    if (plan->timing && plan->stage_marks) {
        FE_CUDA(cudaStreamSynchronize(plan->stream), "timing sync");
        for (int i = 0; i < 4; ++i) {
            plan->stage_ms[i] = 0.f;
            if (plan->stage_marks & (1 << i)) cudaEventElapsedTime(&plan->stage_ms[i], plan->ev[2 * i], plan->ev[2 * i + 1]);
        }
        plan->stage_marks = 0;
    }
    for (int i = 0; i < n && i < 4; ++i) ms[i] = plan->stage_ms[i];
    return FE_OK;
}

fe_status fe_plan_last_launches(const fe_plan *plan, int32_t *launches) {
    if (!plan || !launches) return fail(FE_ERR_INVALID_ARG, "NULL argument");
    *launches = plan->last_launches;
    return FE_OK;
}

fe_status fe_sync_status(fe_plan *plan) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    int st = 0;
    FE_CUDA(cudaMemcpyAsync(&st, plan->status.p, sizeof(int), cudaMemcpyDeviceToHost, plan->stream), "read status");
    FE_CUDA(cudaStreamSynchronize(plan->stream), "sync");
    if (st) FE_CUDA(cudaMemsetAsync(plan->status.p, 0, sizeof(int), plan->stream), "clear status");
    if (st & ST_TIMEOUT) return fail(FE_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
    if (st & ST_NONFINITE) return fail(FE_ERR_NONFINITE, "non-finite geometry or coefficient");
    if (st & ST_DEGENERATE) return fail(FE_ERR_DEGENERATE_CELL, "degenerate cell (det J == 0)");
    if (st & ST_SATURATED) return fail(FE_ERR_NONFINITE, "a reduced-precision value overflowed its storage format");
    return FE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// compute
// ---------------------------------------------------------------------------
static void mark(fe_plan *P, int stage, bool begin) {
    if (!P->timing) return;
    cudaEventRecord(P->ev[2 * stage + (begin ? 0 : 1)], P->stream);
    if (!begin) P->stage_marks |= 1 << stage;
}

static fe_status need_pattern(const fe_plan *plan) {
    if (plan && plan->elements_only)
        return fail(FE_ERR_INVALID_ARG, "the plan was built with FE_PLAN_ELEMENTS_ONLY: no dof map or pattern");
    return FE_OK;
}

static fe_status check_call(fe_plan *plan, unsigned forms, fe_precision prec) {
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    if (forms == 0 || (forms & ~plan->form_mask)) return fail(FE_ERR_INVALID_ARG, "forms not served by the plan");
    if ((int)prec < 0 || (int)prec > 5) return fail(FE_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (prec != FE_PREC_FP64 && !(plan->prec_mask & FE_PREC_MASK(prec)))
        return fail(FE_ERR_INVALID_ARG, "precision %d not prepared by the plan", (int)prec);
    return FE_OK;
}

// ---------------------------------------------------------------------------
// segments shared by single-plan calls and batches
// ---------------------------------------------------------------------------
static fe_status ensure_ws(DevBuf &b, size_t bytes, const char *what) {
    cudaError_t e = b.alloc(bytes);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return FE_OK;
}

// Bytes of the factor kernel's outputs for one plan.
static int win_slots(const fe_plan *P) { return P->boxed ? P->n_pairs + 1 : 1; }
static size_t win_bytes(const fe_plan *P) {
    return sizeof(float) * (size_t)P->n_cells * win_ld(P->n_q) * win_slots(P);
}
static size_t cellf_bytes(const fe_plan *P) { return sizeof(float) * (size_t)P->n_cells * CELLF; }

static TcSeg make_tc_seg(fe_plan *P, unsigned forms, int prec, const double *vertices, const double *kappa,
                         void *const A[2], float *win, float *cellf) {
    TcSeg g{};
    g.win = win;
    g.cellf = cellf;
    g.ldw = win_ld(P->n_q);
    g.vertices = vertices ? vertices : P->vertices.as<double>();
    g.cells = P->cells.as<int32_t>();
    g.n_cells = P->n_cells;
    g.d = P->d;
    g.kappa = kappa;
    g.weights = P->weights.as<double>();
    g.n_q = P->n_q;
    g.n_phi = P->n_phi;
    g.n_pairs = P->n_pairs;
    g.form_mask = 0;
    for (unsigned form : {(unsigned)FE_FORM_STIFFNESS, (unsigned)FE_FORM_MASS}) {
        if (!(forms & form)) continue;
        const int fi = form_index(form);
        g.form_mask |= 1 << fi;
        g.op[fi] = P->op[prec][fi];
        if (P->wpref_mode >= 0) g.op[fi].win_pref = P->wpref_mode;
        g.out[fi] = static_cast<float *>(A[fi]);
    }
    g.sym_kl = P->sym_kl.as<int32_t>();
    g.full2sym = P->full2sym.as<int16_t>();
    g.staged = 0;
    g.tile_begin = 0;
    g.win_slots = win_slots(P);
    g.nv = P->nv;
    g.dpsi = P->boxed ? P->dpsi_box.as<double>() : nullptr;
    return g;
}

// Global launch shape over the segments: operand maxima, then the staged
// epilogue for every segment that fits (greedy, in segment order).
// Shared-operand size above which one plan's launch takes the pass-major job
// order: a quarter of GB300's 126 MB L2.
constexpr size_t kJobRrOperandBytes = (size_t)32 << 20;

static void tc_finalize(TcArgs &a, TcSeg *segs, int n, int prec, int *status, unsigned long long wait_limit_ns) {
    a.win_buf = 0;   // (the staging decisions below are taken without it)
    a.n_acc = 2;     // two 256-column accumulators unless a pass is wide
    for (int i = 0; i < n; ++i)
        for (int f = 0; f < MAX_FORMS; ++f)
            if (((segs[i].form_mask >> f) & 1) && segs[i].op[f].NP > TC_MAX_NP) a.n_acc = 1;
    a.prec = prec;
    a.elem_bytes = host::format_of(prec).elem_bytes;
    a.idesc = idesc_for(prec);
    a.target_exp = host::format_of(prec).target_exp;
    a.np_max = 16;
    a.nq_max = 1;
    a.pitch_max = 0;
    int64_t tiles = 0, jobs = 0, cost = 0;
    for (int i = 0; i < n; ++i) {
        int tile_cost = 0, tile_jobs = 0;
        for (int f = 0; f < MAX_FORMS; ++f)
            if ((segs[i].form_mask >> f) & 1) {
                const TcOperand &op = segs[i].op[f];
                a.np_max = std::max(a.np_max, op.NP);
                tile_cost += op.n_pass * (op.n_kchunks + TC_JOB_EPI_COST);
                tile_jobs += op.n_pass;
            }
        a.nq_max = std::max(a.nq_max, segs[i].n_q);
        segs[i].tile_begin = tiles;
        segs[i].tiles = (segs[i].n_cells + TC_M - 1) / TC_M;
        segs[i].cost_begin = cost;
        segs[i].tile_cost = tile_cost;
        tiles += segs[i].tiles;
        jobs += segs[i].tiles * tile_jobs;
        cost += segs[i].tiles * tile_cost;
    }
    a.n_tiles = tiles;
    a.n_jobs = jobs;
    a.total_cost = cost;
    for (int i = 0; i < n; ++i) {
        if (tc_can_stage(a, segs[i])) {
            segs[i].staged = 1;
            int np = 16;
            for (int f = 0; f < MAX_FORMS; ++f)
                if ((segs[i].form_mask >> f) & 1) np = std::max(np, segs[i].op[f].NP);
            a.pitch_max = std::max(a.pitch_max, np + 1);
        }
    }
    a.status = status;
    a.timeout_ns = wait_limit_ns;  // per wait, counted from the wait's start
    // job order: contiguous cost ranges per CTA, or, for one plan whose shared
    // operand (every pass and form) exceeds a quarter of the L2 cache and whose
    // forms have the same number of passes, pass-major round robin so that the
    // CTAs share each operand chunk through L2
    a.job_rr = 0;
    if (n == 1) {
        size_t op_bytes = 0;
        int passes = -1;
        bool same = true;
        for (int f = 0; f < MAX_FORMS; ++f)
            if ((segs[0].form_mask >> f) & 1) {
                const TcOperand &op = segs[0].op[f];
                op_bytes += (size_t)op.n_pass * op.n_kchunks * op.NP * TC_CHUNK_BYTES;
                if (passes >= 0 && passes != op.n_pass) same = false;
                passes = op.n_pass;
            }
        if (same && op_bytes > kJobRrOperandBytes) a.job_rr = 1;
    }
    // a next-window slot per builder thread where a job reads more than one
    // window (more points than one window holds, or one window per pair) and
    // the autotuner measured the prefetch faster for one of the forms
    for (int i = 0; i < n; ++i)
        if (segs[i].n_q > tc_window_points(prec) || segs[i].win_slots > 1)
            for (int f = 0; f < MAX_FORMS; ++f)
                if (((segs[i].form_mask >> f) & 1) && segs[i].op[f].win_pref) a.win_buf = 1;
    a.ring_a = a.ring_b = 2;
    if (a.win_buf && tc_smem_bytes(a) > 227 * 1024) a.win_buf = 0;
    // operand rings beside the staging area: the built-operand ring first, up to
    // four stages (16 KB each: the builders then run further ahead of the MMAs,
    // which hides the handshake latency of each chunk), then shared-operand stages
    // up to the maximum (each one more bulk copy in flight against the L2 latency)
    a.ring_a = a.ring_b = 2;
    const auto grow = [&a](int &r, int to) {
        while (r < to) {
            ++r;
            if (tc_smem_bytes(a) > 227 * 1024) {
                --r;
                return false;
            }
        }
        return true;
    };
    grow(a.ring_a, TC_MAX_RING_A);
    grow(a.ring_b, TC_MAX_RING_B);
}

static AsmSeg make_asm_seg(fe_plan *P, unsigned forms, const void *const A[2], void *const csr[2]) {
    AsmSeg g{};
    g.n_rows = P->n_dofs;
    g.row_ptr = P->row_ptr.as<int64_t>();
    g.inc_ptr = P->inc_ptr.as<int64_t>();
    g.inc_elem = P->inc_elem.as<int32_t>();
    g.contrib_cnt = P->contrib_cnt.as<uint8_t>();
    g.contrib_base = P->contrib_base.as<int64_t>();
    g.contrib_code = P->contrib_code.as<uint16_t>();
    g.contrib_dest = P->contrib_dest.as<uint16_t>();
    g.chunk_desc = P->chunk_desc.as<int64_t>();
    g.n_chunks = P->n_chunks;
    g.n_phi = P->n_phi;
    g.inc_slot = P->inc_slot.as<uint16_t>();
    int nf = 0;
    for (int fi = 0; fi < 2; ++fi) {
        unsigned form = fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS;
        if (!(forms & form)) continue;
        g.A[nf] = A[fi];
        g.out[nf] = csr[fi];
        ++nf;
    }
    g.row_begin = 0;
    g.chunk_begin = 0;
    return g;
}

static int n_forms_of(unsigned forms) { return ((forms & FE_FORM_STIFFNESS) ? 1 : 0) + ((forms & FE_FORM_MASS) ? 1 : 0); }

static fe_status run_elements(fe_plan *P, unsigned forms, fe_precision prec, const double *vertices,
                              const double *kappa, void *A[2], int &launches) {
    const double *verts = vertices ? vertices : P->vertices.as<double>();
    if (prec == FE_PREC_FP64) {
        mark(P, 0, true);
        const double *geo_q = nullptr;
        if (P->boxed) {
            fe_status st = ensure_ws(P->ws_geoq, sizeof(double) * 7 * (size_t)P->n_cells * P->n_q, "geometry workspace");
            if (st) return st;
            const int r = launch_box_geometry(verts, P->cells.as<int32_t>(), P->n_cells, P->d, P->nv,
                                              P->dpsi_box.as<double>(), P->n_q, P->ws_geoq.as<double>(),
                                              P->status.as<int>(), P->stream);
            if (r < 0) return cuda_fail((cudaError_t)(-r), "geometry kernel launch");
            launches += r;
            geo_q = P->ws_geoq.as<double>();
        }
        for (unsigned form : {(unsigned)FE_FORM_STIFFNESS, (unsigned)FE_FORM_MASS}) {
            if (!(forms & form)) continue;
            F64Args a{};
            a.vertices = verts;
            a.cells = P->cells.as<int32_t>();
            a.n_cells = P->n_cells;
            a.d = P->d;
            a.kappa = kappa;
            a.weights = P->weights.as<double>();
            a.n_q = P->n_q;
            a.n_phi = P->n_phi;
            a.tab = (form == FE_FORM_STIFFNESS) ? P->dphi.as<double>() : P->phi.as<double>();
            a.form = (int)form;
            a.out = static_cast<double *>(A[form_index(form)]);
            a.status = P->status.as<int>();
            a.geo_q = geo_q;
            int r = launch_f64_elements(a, P->stream);
            if (r < 0) return cuda_fail((cudaError_t)(-r), "FP64 element kernel launch");
            launches += r;
        }
    } else {
        TcArgs a{};
        fe_status st = ensure_ws(P->ws_win, win_bytes(P), "coefficient window workspace");
        if (!st) st = ensure_ws(P->ws_cellf, cellf_bytes(P), "cell factor workspace");
        if (st) return st;
        a.seg0 = make_tc_seg(P, forms, prec, verts, kappa, A, P->ws_win.as<float>(), P->ws_cellf.as<float>());
        a.segs = nullptr;
        a.n_segs = 1;
        tc_finalize(a, &a.seg0, 1, prec, P->status.as<int>(), P->wait_limit_ns);
        const size_t smem = tc_smem_bytes(a);
        mark(P, 3, true);
        int r = launch_factor(a, P->stream);
        if (r < 0) return cuda_fail((cudaError_t)(-r), "factor kernel launch");
        launches += r;
        mark(P, 3, false);
        mark(P, 0, true);
        r = launch_tc_elements(a, smem, P->stream);
        if (r < 0) return cuda_fail((cudaError_t)(-r), "tensor-core element kernel launch");
        launches += r;
    }
    mark(P, 0, false);
    return FE_OK;
}

static fe_status run_assembly(fe_plan *P, unsigned forms, bool fp64, const void *A[2], void *csr[2], int &launches) {
    for (int fi = 0; fi < 2; ++fi)
        if ((forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS)) && !csr[fi])
            return fail(FE_ERR_INVALID_ARG, "NULL CSR output");
    AsmArgs a{};
    a.seg0 = make_asm_seg(P, forms, A, csr);
    a.segs = nullptr;
    a.n_segs = 1;
    a.n_rows = P->n_dofs;
    a.n_chunks = P->n_chunks;
    a.n_forms = n_forms_of(forms);
    a.algo = P->asm_algo;
    mark(P, 1, true);
    int r = launch_assemble(a, fp64, P->stream);
    if (r < 0) return cuda_fail((cudaError_t)(-r), "assembly kernel launch");
    launches += r;
    mark(P, 1, false);
    return FE_OK;
}

// Fused assembly (no element-matrix outputs): the cells in slices of one wave
// of tiles; per slice the factor and element kernels write the slice's element
// matrices into ring slot (slice mod fuse_slots) -- a few tens of MB that stay
// in L2 -- and the assembly kernel sums the rows whose last incident cell lies
// in that slice, reading the ring.  Every CSR value is still the sum of its
// entries in increasing cell order from zero: bitwise the unfused result.
static fe_status run_fused(fe_plan *P, unsigned forms, fe_precision prec, const double *vertices, const double *kappa,
                           void *csr[2]) {
    for (int fi = 0; fi < 2; ++fi)
        if ((forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS)) && !csr[fi])
            return fail(FE_ERR_INVALID_ARG, "NULL CSR output");
    const int64_t S = P->fuse_cells;
    const size_t slot_elems = (size_t)S * P->n_phi * P->n_phi;
    void *ring[2] = {nullptr, nullptr};
    for (int fi = 0; fi < 2; ++fi)
        if (forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS)) {
            fe_status st = ensure_ws(P->ws_ring[fi], sizeof(float) * slot_elems * P->fuse_slots, "fused ring");
            if (st) return st;
            ring[fi] = P->ws_ring[fi].p;
        }
    fe_status st = ensure_ws(P->ws_win, win_bytes(P), "coefficient window workspace");
    if (!st) st = ensure_ws(P->ws_cellf, cellf_bytes(P), "cell factor workspace");
    if (st) return st;
    const double *verts = vertices ? vertices : P->vertices.as<double>();
    const int ldw = win_ld(P->n_q), slots = win_slots(P);
    int launches = 0;
    mark(P, 0, true);
    for (int sl = 0; sl < P->fuse_slices; ++sl) {
        const int64_t c0 = (int64_t)sl * S;
        const int64_t cnt = std::min<int64_t>(S, P->n_cells - c0);
        void *A[2] = {nullptr, nullptr};
        for (int fi = 0; fi < 2; ++fi)
            if (ring[fi]) A[fi] = static_cast<float *>(ring[fi]) + (size_t)(sl % P->fuse_slots) * slot_elems;
        TcArgs a{};
        a.seg0 = make_tc_seg(P, forms, prec, verts, kappa + c0 * P->n_q, A, P->ws_win.as<float>() + c0 * ldw * slots,
                             P->ws_cellf.as<float>() + c0 * CELLF);
        a.seg0.cells = P->cells.as<int32_t>() + c0 * P->nv;
        a.seg0.n_cells = cnt;
        a.segs = nullptr;
        a.n_segs = 1;
        tc_finalize(a, &a.seg0, 1, prec, P->status.as<int>(), P->wait_limit_ns);
        int r = launch_factor(a, P->stream);
        if (r < 0) return cuda_fail((cudaError_t)(-r), "factor kernel launch");
        launches += r;
        r = launch_tc_elements(a, tc_smem_bytes(a), P->stream);
        if (r < 0) return cuda_fail((cudaError_t)(-r), "tensor-core element kernel launch");
        launches += r;
        const int64_t lc = P->fuse_row_off[sl + 1] - P->fuse_row_off[sl];
        if (lc > 0) {
            AsmArgs as{};
            const void *Ar[2] = {ring[0], ring[1]};
            as.seg0 = make_asm_seg(P, forms, Ar, csr);
            as.seg0.ring_cells = S;
            as.seg0.ring_slots = P->fuse_slots;
            as.segs = nullptr;
            as.n_segs = 1;
            as.n_rows = P->n_dofs;
            as.n_chunks = P->n_chunks;
            as.n_forms = n_forms_of(forms);
            as.algo = 1;   // the row-wise kernel over the slice's completed rows
            as.row_list = P->fuse_rows.as<int32_t>() + P->fuse_row_off[sl];
            as.row_count = lc;
            r = launch_assemble(as, false, P->stream);
            if (r < 0) return cuda_fail((cudaError_t)(-r), "assembly kernel launch");
            launches += r;
        }
    }
    mark(P, 0, false);
    P->last_launches = launches;
    return FE_OK;
}

// ---------------------------------------------------------------------------
// operand packing and the autotuner
// ---------------------------------------------------------------------------
static fe_status pack_operand(fe_plan &P, int prec, int fi, int np_pass) {
    host::OperandImage img;
    const unsigned form = fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS;
    host::build_operand(prec, (int)form, P.d, P.n_phi, P.n_q, P.h_phi, P.h_dphi, img, np_pass, P.col_of_sym);
    FE_CUDA(upload(P.img[prec][fi], img.bytes, P.stream), "upload operand image");
    TcOperand &o = P.op[prec][fi];
    o.img = P.img[prec][fi].as<uint8_t>();
    o.n_kchunks = img.n_kchunks;
    o.n_qw = img.n_qw;
    o.n_pairs = img.n_pairs;
    o.n_pass = img.n_pass;
    o.NP = img.NP;
    o.n_cols = img.n_cols;
    o.n_blk = img.n_blk;
    o.rows_per_pass = img.rows_per_pass;
    o.p_inv_scale = (float)img.p_inv_scale;
    P.tuned_np[prec][fi] = img.rows_per_pass > 0 ? -img.rows_per_pass : img.NP;
    return FE_OK;
}

namespace {
std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, int>> g_tune_cache;  // "(d,p,n_q,prec,forms,boxed)" -> (N layout, window prefetch)
}  // namespace

// Autotuner for the tile shape of every (cell type, degree, quadrature size,
// precision, set of forms): the N layout of the contraction when the symmetric
// pairs need more than one 256-column accumulator (whole rows per pass, wide
// passes of up to 512 columns, or pairs in passes of a given width), and, where
// a job reads several coefficient windows, the builders' window prefetch.
// Candidates come from host::np_candidates; each is applied to all the plan's
// forms and timed with CUDA events as one launch of them, as production runs
// it, on a sample of this plan's own cells (unit coefficient) -- two full waves
// of tiles, so that every SM runs as in a production launch, with the L2
// flushed before each run -- and the fastest is kept.  Results are cached per
// key for the life of the process.  FE_GB300_AUTOTUNE=0 keeps the default
// shapes.
static fe_status autotune_plan(fe_plan &P) {
    const char *env = getenv("FE_GB300_AUTOTUNE");
    if (env && env[0] == '0') return FE_OK;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned forms = P.form_mask & (FE_FORM_STIFFNESS | FE_FORM_MASS);
    const int n_forms = n_forms_of(forms);
    for (int prec = 1; prec <= 5; ++prec) {
        if (!(P.prec_mask & FE_PREC_MASK(prec))) continue;
        std::vector<int> cand = host::np_candidates(P.n_phi);
        // the builders' next-window prefetch is a choice wherever a job reads
        // more than one window: it costs a shared-memory slot per builder
        // thread, which may otherwise hold an operand stage
        const bool multi_win = P.n_q > tc_window_points(prec) || win_slots(&P) > 1;
        const int n_wp = multi_win ? 2 : 1;
        if (cand.size() * n_wp < 2) continue;
        char key[96];
        snprintf(key, sizeof(key), "%d,%d,%d,%d,%u,%d", P.d, P.p, P.n_q, prec, forms, (int)P.boxed);
        int best = INT_MIN, best_wp = 0;
        {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                best = it->second.first;
                best_wp = it->second.second;
            }
        }
        if (best == INT_MIN) {
            // Every candidate is timed as production runs it: one launch of all the
            // plan's forms with the same layout (a wide pass in one form makes the
            // launch single-accumulator for both), on two full waves of tiles
            // (every SM busy; a partial wave would time one tile's latency
            // instead), at most 4 GB of sample output, unit coefficient.
            int64_t n = std::min<int64_t>(P.n_cells, 2ll * sms * TC_M);
            n = std::min<int64_t>(n, std::max<int64_t>(TC_M, (4096ll << 20) / (4ll * n_forms * P.n_phi * P.n_phi)));
            DevBuf kap, out[2], win, cellf, flush;
            FE_CUDA(kap.alloc(sizeof(double) * n * P.n_q), "autotune buffer");
            // written before every timed run so that each candidate starts with
            // the sample's output out of L2, as a production launch does: the
            // layouts differ in how many partially written sectors they leave
            const size_t flush_bytes = (size_t)256 << 20;
            FE_CUDA(flush.alloc(flush_bytes), "autotune buffer");
            // the factor kernel's windows: one per cell (simplices) or one per
            // pair and one for the mass form (boxed cells), as win_bytes
            FE_CUDA(win.alloc(sizeof(float) * n * win_ld(P.n_q) * win_slots(&P)), "autotune buffer");
            FE_CUDA(cellf.alloc(sizeof(float) * n * CELLF), "autotune buffer");
            void *A[2] = {nullptr, nullptr};
            for (int fi = 0; fi < 2; ++fi)
                if (forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS)) {
                    FE_CUDA(out[fi].alloc(sizeof(float) * n * P.n_phi * P.n_phi), "autotune buffer");
                    A[fi] = out[fi].p;
                }
            std::vector<double> ones((size_t)n * P.n_q, 1.0);
            FE_CUDA(cudaMemcpyAsync(kap.p, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice,
                                    P.stream), "autotune upload");
            float best_ms = 1e30f;
            for (size_t ci = 0; ci < cand.size() * n_wp; ++ci) {
                const int np = cand[ci / n_wp], wp = (int)(ci % n_wp);
                for (int fi = 0; fi < 2; ++fi) {
                    if (!(forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS))) continue;
                    if (wp == 0) {
                        fe_status st = pack_operand(P, prec, fi, np);
                        if (st) return st;
                    }
                    P.op[prec][fi].win_pref = wp;
                }
                TcArgs a{};
                a.seg0 = make_tc_seg(&P, forms, prec, nullptr, kap.as<double>(), A, win.as<float>(), cellf.as<float>());
                a.seg0.n_cells = n;
                a.n_segs = 1;
                tc_finalize(a, &a.seg0, 1, prec, P.status.as<int>(), kDefaultWaitLimitNs);
                const size_t smem = tc_smem_bytes(a);
                {
                    const int r = launch_factor(a, P.stream);
                    if (r < 0) return cuda_fail((cudaError_t)(-r), "autotune factor launch");
                }
                float ms_min = 1e30f;
                for (int rep = 0; rep < 5; ++rep) {   // the first run warms up; the best of the other four counts
                    FE_CUDA(cudaMemsetAsync(flush.p, rep, flush_bytes, P.stream), "autotune flush");
                    FE_CUDA(cudaEventRecord(P.ev[4], P.stream), "autotune event");
                    int r = launch_tc_elements(a, smem, P.stream);
                    if (r < 0) return cuda_fail((cudaError_t)(-r), "autotune launch");
                    FE_CUDA(cudaEventRecord(P.ev[5], P.stream), "autotune event");
                    FE_CUDA(cudaEventSynchronize(P.ev[5]), "autotune sync");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, P.ev[4], P.ev[5]);
                    if (rep > 0) ms_min = std::min(ms_min, ms);
                }
                if (ms_min < best_ms) {
                    best_ms = ms_min;
                    best = np;
                    best_wp = wp;
                }
            }
            int stw = 0;
            cudaMemcpy(&stw, P.status.p, sizeof(int), cudaMemcpyDeviceToHost);
            if (stw) {
                cudaMemset(P.status.p, 0, sizeof(int));
                return fail(FE_ERR_CUDA, "autotune run reported status %d", stw);
            }
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            g_tune_cache[key] = {best, best_wp};
        }
        for (int fi = 0; fi < 2; ++fi) {
            if (!(forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS))) continue;
            if (P.tuned_np[prec][fi] != best) {
                fe_status st = pack_operand(P, prec, fi, best);
                if (st) return st;
            }
            P.op[prec][fi].win_pref = best_wp;
        }
    }
    FE_CUDA(cudaStreamSynchronize(P.stream), "autotune");
    return FE_OK;
}

extern "C" {

fe_status fe_element_matrices(fe_plan *plan, unsigned forms, fe_precision prec, const double *vertices,
                              const double *kappa, void *A_stiffness, void *A_mass) {
    g_err.clear();
    fe_status st = check_call(plan, forms, prec);
    if (st) return st;
    if (!kappa) return fail(FE_ERR_INVALID_ARG, "NULL kappa");
    void *A[2] = {A_stiffness, A_mass};
    if ((forms & FE_FORM_STIFFNESS) && !A_stiffness) return fail(FE_ERR_INVALID_ARG, "NULL stiffness output");
    if ((forms & FE_FORM_MASS) && !A_mass) return fail(FE_ERR_INVALID_ARG, "NULL mass output");
    int launches = 0;
    st = run_elements(plan, forms, prec, vertices, kappa, A, launches);
    plan->last_launches = launches;
    return st;
}

fe_status fe_assemble(fe_plan *plan, unsigned forms, fe_precision prec, const double *vertices, const double *kappa,
                      void *A_stiffness, void *A_mass, void *csr_stiffness, void *csr_mass) {
    g_err.clear();
    fe_status st = check_call(plan, forms, prec);
    if (st) return st;
    st = need_pattern(plan);
    if (st) return st;
    if (!kappa) return fail(FE_ERR_INVALID_ARG, "NULL kappa");
    const bool fp64 = prec == FE_PREC_FP64;
    if (!fp64 && !A_stiffness && !A_mass && plan->fuse_ok && plan->fuse_mode == 1) {
        void *csr[2] = {csr_stiffness, csr_mass};
        return run_fused(plan, forms, prec, vertices, kappa, csr);
    }
    const size_t ebytes = (fp64 ? 8 : 4) * (size_t)plan->n_cells * plan->n_phi * plan->n_phi;
    void *A[2] = {A_stiffness, A_mass};
    for (int fi = 0; fi < 2; ++fi) {
        unsigned form = fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS;
        if ((forms & form) && !A[fi]) {
            st = ensure_ws(plan->ws_elem[fi], ebytes, "element workspace");
            if (st) return st;
            A[fi] = plan->ws_elem[fi].p;
        }
    }
    int launches = 0;
    st = run_elements(plan, forms, prec, vertices, kappa, A, launches);
    if (st) return st;
    const void *Ac[2] = {A[0], A[1]};
    void *csr[2] = {csr_stiffness, csr_mass};
    st = run_assembly(plan, forms, fp64, Ac, csr, launches);
    plan->last_launches = launches;
    return st;
}

fe_status fe_assemble_elements(fe_plan *plan, unsigned forms, fe_precision prec, const void *A_stiffness,
                               const void *A_mass, void *csr_stiffness, void *csr_mass) {
    g_err.clear();
    fe_status st = check_call(plan, forms, prec);
    if (st) return st;
    st = need_pattern(plan);
    if (st) return st;
    const void *A[2] = {A_stiffness, A_mass};
    for (int fi = 0; fi < 2; ++fi)
        if ((forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS)) && !A[fi])
            return fail(FE_ERR_INVALID_ARG, "NULL element matrices");
    void *csr[2] = {csr_stiffness, csr_mass};
    int launches = 0;
    st = run_assembly(plan, forms, prec == FE_PREC_FP64, A, csr, launches);
    plan->last_launches = launches;
    return st;
}

fe_status fe_assemble_host(fe_plan *plan, unsigned forms, fe_precision prec, const double *kappa_host,
                           void *csr_stiffness_host, void *csr_mass_host) {
    g_err.clear();
    fe_status st = check_call(plan, forms, prec);
    if (st) return st;
    st = need_pattern(plan);
    if (st) return st;
    if (!kappa_host) return fail(FE_ERR_INVALID_ARG, "NULL kappa");
    const bool fp64 = prec == FE_PREC_FP64;
    const size_t kbytes = sizeof(double) * (size_t)plan->n_cells * plan->n_q;
    const size_t vbytes = (fp64 ? 8 : 4) * (size_t)plan->nnz;
    st = ensure_ws(plan->ws_kappa, kbytes, "kappa workspace");
    if (st) return st;
    void *csr[2] = {nullptr, nullptr};
    for (int fi = 0; fi < 2; ++fi) {
        if (!(forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS))) continue;
        st = ensure_ws(plan->ws_csr[fi], vbytes, "CSR workspace");
        if (st) return st;
        csr[fi] = plan->ws_csr[fi].p;
    }
    FE_CUDA(cudaMemcpyAsync(plan->ws_kappa.p, kappa_host, kbytes, cudaMemcpyHostToDevice, plan->stream), "copy kappa");
    void *hout[2] = {csr_stiffness_host, csr_mass_host};
    const int pieces = (int)plan->piece_chunk.size() - 1;
    if (pieces < 2 || plan->asm_algo != 0 || (plan->fuse_ok && plan->fuse_mode == 1)) {
        st = fe_assemble(plan, forms, prec, nullptr, plan->ws_kappa.as<double>(), nullptr, nullptr, csr[0], csr[1]);
        if (st) return st;
        for (int fi = 0; fi < 2; ++fi)
            if (csr[fi] && hout[fi])
                FE_CUDA(cudaMemcpyAsync(hout[fi], csr[fi], vbytes, cudaMemcpyDeviceToHost, plan->stream), "copy CSR");
        return fe_sync_status(plan);
    }
    // the element matrices, then the assembly in ranges of consecutive rows (the
    // last first, as the whole-range launch walks them); each range's CSR values
    // are downloaded on the copy stream while the next range is summed
    fe_plan &P = *plan;
    if (!P.pieces_ready) {
        std::vector<int32_t> iota((size_t)P.n_chunks);
        for (int64_t c = 0; c < P.n_chunks; ++c) iota[(size_t)c] = (int32_t)c;
        FE_CUDA(upload(P.chunk_iota, iota, P.stream), "upload chunk list");
        if (!P.pipe_ready) {
            FE_CUDA(cudaStreamCreateWithFlags(&P.pipe_h2d, cudaStreamNonBlocking), "pipeline stream");
            FE_CUDA(cudaStreamCreateWithFlags(&P.pipe_d2h, cudaStreamNonBlocking), "pipeline stream");
            for (int slot = 0; slot < 2; ++slot) {
                FE_CUDA(cudaEventCreateWithFlags(&P.pipe_in[slot], cudaEventDisableTiming), "pipeline event");
                FE_CUDA(cudaEventCreateWithFlags(&P.pipe_used[slot], cudaEventDisableTiming), "pipeline event");
                FE_CUDA(cudaEventCreateWithFlags(&P.pipe_out[slot], cudaEventDisableTiming), "pipeline event");
            }
            P.pipe_ready = true;
        }
        for (int k = 0; k < pieces; ++k)
            FE_CUDA(cudaEventCreateWithFlags(&P.piece_done[k], cudaEventDisableTiming), "piece event");
        P.pieces_ready = true;
    }
    const size_t ebytes = (fp64 ? 8 : 4) * (size_t)P.n_cells * P.n_phi * P.n_phi;
    void *A[2] = {nullptr, nullptr};
    for (int fi = 0; fi < 2; ++fi)
        if (forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS)) {
            st = ensure_ws(P.ws_elem[fi], ebytes, "element workspace");
            if (st) return st;
            A[fi] = P.ws_elem[fi].p;
        }
    int launches = 0;
    st = run_elements(plan, forms, prec, nullptr, P.ws_kappa.as<double>(), A, launches);
    if (st) return st;
    const void *Ac[2] = {A[0], A[1]};
    const size_t vsize = fp64 ? 8 : 4;
    mark(plan, 1, true);
    for (int k = pieces - 1; k >= 0; --k) {
        AsmArgs a{};
        a.seg0 = make_asm_seg(plan, forms, Ac, csr);
        a.segs = nullptr;
        a.n_segs = 1;
        a.n_rows = P.n_dofs;
        a.n_chunks = P.n_chunks;
        a.n_forms = n_forms_of(forms);
        a.algo = 0;
        a.chunk_list = P.chunk_iota.as<int32_t>() + P.piece_chunk[k];
        a.list_count = P.piece_chunk[k + 1] - P.piece_chunk[k];
        if (a.list_count > 0) {
            const int r = launch_assemble(a, fp64, P.stream);
            if (r < 0) return cuda_fail((cudaError_t)(-r), "assembly kernel launch");
            launches += r;
        }
        FE_CUDA(cudaEventRecord(P.piece_done[k], P.stream), "piece event");
        FE_CUDA(cudaStreamWaitEvent(P.pipe_d2h, P.piece_done[k], 0), "piece wait");
        const int64_t v0 = P.piece_val[k], nv = P.piece_val[k + 1] - v0;
        for (int fi = 0; fi < 2; ++fi)
            if (csr[fi] && hout[fi] && nv > 0)
                FE_CUDA(cudaMemcpyAsync(static_cast<char *>(hout[fi]) + v0 * vsize,
                                        static_cast<const char *>(csr[fi]) + v0 * vsize, (size_t)nv * vsize,
                                        cudaMemcpyDeviceToHost, P.pipe_d2h), "copy CSR");
    }
    mark(plan, 1, false);
    P.last_launches = launches;
    FE_CUDA(cudaStreamSynchronize(P.pipe_d2h), "copy CSR");
    return fe_sync_status(plan);
}

fe_status fe_assemble_host_many(fe_plan *plan, unsigned forms, fe_precision prec, int n,
                                const double *const *kappa_host, void *const *csr_stiffness_host,
                                void *const *csr_mass_host) {
    g_err.clear();
    fe_status st = check_call(plan, forms, prec);
    if (st) return st;
    st = need_pattern(plan);
    if (st) return st;
    if (n <= 0 || !kappa_host) return fail(FE_ERR_INVALID_ARG, "empty sequence or NULL kappa array");
    for (int i = 0; i < n; ++i)
        if (!kappa_host[i]) return fail(FE_ERR_INVALID_ARG, "NULL kappa for item %d", i);
    fe_plan &P = *plan;
    const bool fp64 = prec == FE_PREC_FP64;
    const size_t kbytes = sizeof(double) * (size_t)P.n_cells * P.n_q;
    const size_t vbytes = (fp64 ? 8 : 4) * (size_t)P.nnz;
    // two slots of device inputs and outputs (allocated once, kept by the plan)
    for (int slot = 0; slot < 2; ++slot) {
        st = ensure_ws(P.ws_pipe_kappa[slot], kbytes, "pipeline kappa workspace");
        if (st) return st;
        for (int fi = 0; fi < 2; ++fi)
            if (forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS)) {
                st = ensure_ws(P.ws_pipe_csr[slot][fi], vbytes, "pipeline CSR workspace");
                if (st) return st;
            }
    }
    if (!P.pipe_ready) {
        FE_CUDA(cudaStreamCreateWithFlags(&P.pipe_h2d, cudaStreamNonBlocking), "pipeline stream");
        FE_CUDA(cudaStreamCreateWithFlags(&P.pipe_d2h, cudaStreamNonBlocking), "pipeline stream");
        for (int slot = 0; slot < 2; ++slot) {
            FE_CUDA(cudaEventCreateWithFlags(&P.pipe_in[slot], cudaEventDisableTiming), "pipeline event");
            FE_CUDA(cudaEventCreateWithFlags(&P.pipe_used[slot], cudaEventDisableTiming), "pipeline event");
            FE_CUDA(cudaEventCreateWithFlags(&P.pipe_out[slot], cudaEventDisableTiming), "pipeline event");
        }
        P.pipe_ready = true;
    }
    // everything issued earlier on the plan's stream comes first
    FE_CUDA(cudaEventRecord(P.pipe_used[0], P.stream), "pipeline event");
    FE_CUDA(cudaStreamWaitEvent(P.pipe_h2d, P.pipe_used[0], 0), "pipeline wait");
    FE_CUDA(cudaStreamWaitEvent(P.pipe_d2h, P.pipe_used[0], 0), "pipeline wait");
    FE_CUDA(cudaEventRecord(P.pipe_used[1], P.stream), "pipeline event");
    FE_CUDA(cudaEventRecord(P.pipe_out[0], P.pipe_d2h), "pipeline event");
    FE_CUDA(cudaEventRecord(P.pipe_out[1], P.pipe_d2h), "pipeline event");
    for (int i = 0; i < n; ++i) {
        const int slot = i & 1;
        // upload item i once the computation of item i - 2 has consumed the slot
        FE_CUDA(cudaStreamWaitEvent(P.pipe_h2d, P.pipe_used[slot], 0), "pipeline wait");
        FE_CUDA(cudaMemcpyAsync(P.ws_pipe_kappa[slot].p, kappa_host[i], kbytes, cudaMemcpyHostToDevice, P.pipe_h2d),
                "copy kappa");
        FE_CUDA(cudaEventRecord(P.pipe_in[slot], P.pipe_h2d), "pipeline event");
        // compute item i once its input has landed and item i - 2's results have left the slot
        FE_CUDA(cudaStreamWaitEvent(P.stream, P.pipe_in[slot], 0), "pipeline wait");
        FE_CUDA(cudaStreamWaitEvent(P.stream, P.pipe_out[slot], 0), "pipeline wait");
        void *csr[2] = {P.ws_pipe_csr[slot][0].p, P.ws_pipe_csr[slot][1].p};
        st = fe_assemble(plan, forms, prec, nullptr, P.ws_pipe_kappa[slot].as<double>(), nullptr, nullptr,
                         (forms & FE_FORM_STIFFNESS) ? csr[0] : nullptr, (forms & FE_FORM_MASS) ? csr[1] : nullptr);
        if (st) return st;
        FE_CUDA(cudaEventRecord(P.pipe_used[slot], P.stream), "pipeline event");
        // download item i's CSR values
        FE_CUDA(cudaStreamWaitEvent(P.pipe_d2h, P.pipe_used[slot], 0), "pipeline wait");
        void *hout[2] = {csr_stiffness_host ? csr_stiffness_host[i] : nullptr, csr_mass_host ? csr_mass_host[i] : nullptr};
        for (int fi = 0; fi < 2; ++fi)
            if ((forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS)) && hout[fi])
                FE_CUDA(cudaMemcpyAsync(hout[fi], csr[fi], vbytes, cudaMemcpyDeviceToHost, P.pipe_d2h), "copy CSR");
        FE_CUDA(cudaEventRecord(P.pipe_out[slot], P.pipe_d2h), "pipeline event");
    }
    FE_CUDA(cudaStreamSynchronize(P.pipe_d2h), "pipeline sync");
    FE_CUDA(cudaStreamSynchronize(P.pipe_h2d), "pipeline sync");
    return fe_sync_status(plan);
}

fe_status fe_adjoint(fe_plan *plan, const double *vertices, const double *kappa, const float *u, const float *v,
                     double *g_kappa, double *g_vertices, double *L_out) {
    g_err.clear();
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    if (need_pattern(plan)) return FE_ERR_INVALID_ARG;
    if (plan->boxed) return fail(FE_ERR_UNSUPPORTED, "fe_adjoint: simplices only");
    if (!(plan->form_mask & FE_FORM_STIFFNESS)) return fail(FE_ERR_INVALID_ARG, "plan does not serve stiffness");
    if (!kappa || !u || !v) return fail(FE_ERR_INVALID_ARG, "NULL argument");
    fe_status st;
    if (g_vertices) {
        st = ensure_ws(plan->ws_adj_x, sizeof(double) * plan->n_cells * (plan->d + 1) * plan->d, "adjoint workspace");
        if (st) return st;
    }
    st = ensure_ws(plan->ws_adj_L, sizeof(double) * plan->n_cells, "adjoint workspace");
    if (st) return st;
    AdjArgs a{};
    a.vertices = vertices ? vertices : plan->vertices.as<double>();
    a.cells = plan->cells.as<int32_t>();
    a.n_cells = plan->n_cells;
    a.n_vertices = plan->n_vertices;
    a.d = plan->d;
    a.kappa = kappa;
    a.weights = plan->weights.as<double>();
    a.n_q = plan->n_q;
    a.n_phi = plan->n_phi;
    a.dphi = plan->dphi.as<double>();
    a.cell_dofs = plan->cell_dofs.as<int32_t>();
    a.u = u;
    a.v = v;
    a.g_kappa = g_kappa;
    a.g_cell_x = g_vertices ? plan->ws_adj_x.as<double>() : nullptr;
    a.L_cell = plan->ws_adj_L.as<double>();
    a.status = plan->status.as<int>();
    mark(plan, 2, true);
    int r = launch_adjoint(a, plan->vinc_ptr.as<int64_t>(), plan->vinc.as<int32_t>(), g_vertices, L_out, plan->stream);
    if (r < 0) return cuda_fail((cudaError_t)(-r), "adjoint kernel launch");
    mark(plan, 2, false);
    plan->last_launches = r;
    return FE_OK;
}

fe_status fe_adjoint_values(fe_plan *plan, const double *vertices, const double *kappa, const double *grad_values,
                            double *g_kappa, double *g_vertices, double *L_out) {
    g_err.clear();
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    if (need_pattern(plan)) return FE_ERR_INVALID_ARG;
    if (plan->boxed) return fail(FE_ERR_UNSUPPORTED, "fe_adjoint_values: simplices only");
    if (!(plan->form_mask & FE_FORM_STIFFNESS)) return fail(FE_ERR_INVALID_ARG, "plan does not serve stiffness");
    if (!kappa || !grad_values) return fail(FE_ERR_INVALID_ARG, "NULL argument");
    if ((size_t)plan->n_phi * plan->n_phi * sizeof(double) > (size_t)200 << 10)
        return fail(FE_ERR_UNSUPPORTED, "n_phi = %d: the cell's gradient block does not fit shared memory", plan->n_phi);
    fe_status st;
    if (g_vertices) {
        st = ensure_ws(plan->ws_adj_x, sizeof(double) * plan->n_cells * (plan->d + 1) * plan->d, "adjoint workspace");
        if (st) return st;
    }
    st = ensure_ws(plan->ws_adj_L, sizeof(double) * plan->n_cells, "adjoint workspace");
    if (st) return st;
    AdjValArgs av{};
    AdjArgs &a = av.base;
    a.vertices = vertices ? vertices : plan->vertices.as<double>();
    a.cells = plan->cells.as<int32_t>();
    a.n_cells = plan->n_cells;
    a.n_vertices = plan->n_vertices;
    a.d = plan->d;
    a.kappa = kappa;
    a.weights = plan->weights.as<double>();
    a.n_q = plan->n_q;
    a.n_phi = plan->n_phi;
    a.dphi = plan->dphi.as<double>();
    a.cell_dofs = plan->cell_dofs.as<int32_t>();
    a.g_kappa = g_kappa;
    a.g_cell_x = g_vertices ? plan->ws_adj_x.as<double>() : nullptr;
    a.L_cell = plan->ws_adj_L.as<double>();
    a.status = plan->status.as<int>();
    av.gvals = grad_values;
    av.row_ptr = plan->row_ptr.as<int64_t>();
    av.col_idx = plan->col_idx.as<int32_t>();
    mark(plan, 2, true);
    const int r = launch_adjoint_values(av, plan->vinc_ptr.as<int64_t>(), plan->vinc.as<int32_t>(), g_vertices, L_out,
                                        plan->stream);
    if (r < 0) return cuda_fail((cudaError_t)(-r), "adjoint kernel launch");
    mark(plan, 2, false);
    plan->last_launches = r;
    return FE_OK;
}

// Tables of the warp-per-cell action kernel for one precision and form: B
// [n_d][n_phi][n_q] and its transpose [n_d][n_q][n_phi], in FP64 or rounded once
// to the storage format (kept as FP32 values).
static fe_status action_tables(fe_plan *P, int prec, int fi) {
    if (P->act_tab[prec][fi].p) return FE_OK;
    const bool stiff = fi == 0;
    const int nd = stiff ? P->d : 1, nph = P->n_phi, nq = P->n_q;
    const std::vector<double> &src = stiff ? P->h_dphi : P->h_phi;
    std::vector<double> t((size_t)nd * nph * nq), tt(t.size());
    const host::Format F = host::format_of(prec);
    for (int s = 0; s < nd; ++s)
        for (int k = 0; k < nph; ++k)
            for (int q = 0; q < nq; ++q) {
                double v = src[((size_t)s * nph + k) * nq + q];
                if (prec != FE_PREC_FP64) v = host::round_to_format(v, F.mbits, F.emin, F.maxfinite);
                t[((size_t)s * nph + k) * nq + q] = v;
                tt[((size_t)s * nq + q) * nph + k] = v;
            }
    if (prec == FE_PREC_FP64) {
        FE_CUDA(upload(P->act_tab[prec][fi], t, P->stream), "upload action table");
        FE_CUDA(upload(P->act_tab_t[prec][fi], tt, P->stream), "upload action table");
    } else {
        std::vector<float> f(t.begin(), t.end()), ft(tt.begin(), tt.end());
        FE_CUDA(upload(P->act_tab[prec][fi], f, P->stream), "upload action table");
        FE_CUDA(upload(P->act_tab_t[prec][fi], ft, P->stream), "upload action table");
    }
    return FE_OK;
}

// Packed table of the thread-per-cell action kernel for one storage format and
// forms mask (bit 0 Poisson, bit 1 mass): per quadrature point the Poisson
// segments B_skq (s = 0 .. d-1) then the mass segment B_kq, each over k and
// zero-padded to act_seg_floats, rounded once to the storage format.
static fe_status action_packed(fe_plan *P, int prec, int forms) {
    DevBuf &dst = P->act_packed[prec][forms - 1];
    if (dst.p) return FE_OK;
    const int nph = P->n_phi, nq = P->n_q, d = P->d;
    const int seg = act_seg_floats(nph), row = act_row_floats(d, nph, forms);
    const host::Format F = host::format_of(prec);
    std::vector<float> packed((size_t)nq * row, 0.f);
    for (int q = 0; q < nq; ++q) {
        int off = 0;
        if (forms & 1)
            for (int s = 0; s < d; ++s, off += seg)
                for (int k = 0; k < nph; ++k)
                    packed[(size_t)q * row + off + k] = (float)host::round_to_format(
                        P->h_dphi[((size_t)s * nph + k) * nq + q], F.mbits, F.emin, F.maxfinite);
        if (forms & 2)
            for (int k = 0; k < nph; ++k)
                packed[(size_t)q * row + off + k] =
                    (float)host::round_to_format(P->h_phi[(size_t)k * nq + q], F.mbits, F.emin, F.maxfinite);
    }
    FE_CUDA(upload(dst, packed, P->stream), "upload action table");
    return FE_OK;
}

fe_status fe_action(fe_plan *plan, unsigned forms, fe_precision prec, const double *vertices, const double *kappa,
                    const double *w, void *b_stiffness, void *b_mass, void *v_stiffness, void *v_mass) {
    g_err.clear();
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    if (need_pattern(plan)) return FE_ERR_INVALID_ARG;
    if (plan->boxed) return fail(FE_ERR_UNSUPPORTED, "fe_action: simplices only");
    if (forms == 0 || (forms & ~plan->form_mask)) return fail(FE_ERR_INVALID_ARG, "forms not served by the plan");
    if (prec != FE_PREC_FP64 && prec != FE_PREC_TF32 && prec != FE_PREC_BF16 && prec != FE_PREC_FP16)
        return fail(FE_ERR_UNSUPPORTED, "fe_action supports FP64, TF32, BF16 and FP16");
    if (!kappa || !w) return fail(FE_ERR_INVALID_ARG, "NULL kappa or w");
    const bool fp64 = prec == FE_PREC_FP64;
    void *bs[2] = {b_stiffness, b_mass}, *vs[2] = {v_stiffness, v_mass};
    const unsigned form_bit[2] = {FE_FORM_STIFFNESS, FE_FORM_MASS};
    int mask = 0;   // bit 0 Poisson, bit 1 mass
    for (int fi = 0; fi < 2; ++fi) {
        if (!(forms & form_bit[fi])) continue;
        if (!bs[fi] && !vs[fi]) return fail(FE_ERR_INVALID_ARG, "no output for a requested form");
        mask |= 1 << fi;
        if (!bs[fi]) {
            fe_status st = ensure_ws(plan->ws_act_b[fi], (fp64 ? 8 : 4) * (size_t)plan->n_cells * plan->n_phi,
                                     "action workspace");
            if (st) return st;
            bs[fi] = plan->ws_act_b[fi].p;
        }
    }
    ActArgs a{};
    a.vertices = vertices ? vertices : plan->vertices.as<double>();
    a.cells = plan->cells.as<int32_t>();
    a.cell_dofs = plan->cell_dofs.as<int32_t>();
    a.n_cells = plan->n_cells;
    a.d = plan->d;
    a.n_phi = plan->n_phi;
    a.n_q = plan->n_q;
    a.prec = (int)prec;
    a.kappa = kappa;
    a.weights = plan->weights.as<double>();
    a.w = w;
    a.status = plan->status.as<int>();
    a.r_bound[0] = plan->act_rbound[0];
    a.r_bound[1] = plan->act_rbound[1];
    int launches = 0;
    if (action_per_cell(plan->d, plan->n_phi, fp64)) {
        // every requested form in one launch
        fe_status st = action_packed(plan, (int)prec, mask);
        if (st) return st;
        a.forms = mask;
        a.tab = plan->act_packed[prec][mask - 1].p;
        a.b = bs[0];
        a.b_mass = bs[1];
        a.qw = action_window(plan->d, plan->n_phi, plan->n_q, mask);
        if (action_smem_bytes(a, fp64) > 200 * 1024) return fail(FE_ERR_UNSUPPORTED, "element too large for fe_action");
        const int r = launch_action(a, fp64, plan->stream);
        if (r < 0) return cuda_fail((cudaError_t)(-r), "action kernel launch");
        launches += r;
    } else {
        for (int fi = 0; fi < 2; ++fi) {
            if (!(mask & (1 << fi))) continue;
            fe_status st = action_tables(plan, (int)prec, fi);
            if (st) return st;
            a.form = (int)form_bit[fi];
            a.tab = plan->act_tab[prec][fi].p;
            a.tab_t = plan->act_tab_t[prec][fi].p;
            a.b = bs[fi];
            if (action_smem_bytes(a, fp64) > 200 * 1024)
                return fail(FE_ERR_UNSUPPORTED, "element too large for fe_action");
            const int r = launch_action(a, fp64, plan->stream);
            if (r < 0) return cuda_fail((cudaError_t)(-r), "action kernel launch");
            launches += r;
        }
    }
    // vector assembly of the forms whose assembled vector was asked for (one launch)
    const void *vb[2] = {nullptr, nullptr};
    void *vv[2] = {nullptr, nullptr};
    int nv = 0;
    for (int fi = 0; fi < 2; ++fi)
        if ((mask & (1 << fi)) && vs[fi]) {
            vb[nv] = bs[fi];
            vv[nv++] = vs[fi];
        }
    if (nv > 0) {
        const int r = launch_vector_assemble(plan->n_dofs, plan->inc_ptr.as<int64_t>(), plan->inc_elem.as<int32_t>(),
                                             vb[0], vb[1], vv[0], vv[1], fp64, plan->stream);
        if (r < 0) return cuda_fail((cudaError_t)(-r), "vector assembly launch");
        launches += r;
    }
    plan->last_launches = launches;
    return FE_OK;
}

fe_status fe_adjoint_noalloc(fe_plan *plan, const double *vertices, const double *kappa, const float *u,
                             const float *v, double *g_kappa, double *g_vertices, double *L_out) {
    g_err.clear();
    if (!plan) return fail(FE_ERR_INVALID_ARG, "NULL plan");
    if (need_pattern(plan)) return FE_ERR_INVALID_ARG;
    if (plan->boxed) return fail(FE_ERR_UNSUPPORTED, "fe_adjoint_noalloc: simplices only");
    if (!(plan->form_mask & FE_FORM_STIFFNESS)) return fail(FE_ERR_INVALID_ARG, "plan does not serve stiffness");
    if (!kappa || !u || !v) return fail(FE_ERR_INVALID_ARG, "NULL argument");
    const size_t per_cell = (g_vertices ? (size_t)(plan->d + 1) * plan->d : 0) + 1;
    const size_t need = (size_t)plan->n_cells * per_cell;
    if (need > kNoAllocScratchDoubles)
        return fail(FE_ERR_UNSUPPORTED,
                    "fe_adjoint_noalloc: %lld cells need %zu doubles of scratch, above the fixed capacity of %zu "
                    "(%zu cells with vertex gradients, %zu without); use fe_adjoint",
                    (long long)plan->n_cells, need, kNoAllocScratchDoubles,
                    kNoAllocScratchDoubles / ((size_t)(plan->d + 1) * plan->d + 1), kNoAllocScratchDoubles);
    double *scratch = nullptr;
    FE_CUDA(noalloc_scratch(&scratch), "fe_adjoint_noalloc scratch lookup");
    AdjArgs a{};
    a.vertices = vertices ? vertices : plan->vertices.as<double>();
    a.cells = plan->cells.as<int32_t>();
    a.n_cells = plan->n_cells;
    a.n_vertices = plan->n_vertices;
    a.d = plan->d;
    a.kappa = kappa;
    a.weights = plan->weights.as<double>();
    a.n_q = plan->n_q;
    a.n_phi = plan->n_phi;
    a.dphi = plan->dphi.as<double>();
    a.cell_dofs = plan->cell_dofs.as<int32_t>();
    a.u = u;
    a.v = v;
    a.g_kappa = g_kappa;
    // every scratch entry read by the kernels is written earlier in the same call
    a.L_cell = scratch;
    a.g_cell_x = g_vertices ? scratch + plan->n_cells : nullptr;
    a.status = plan->status.as<int>();
    mark(plan, 2, true);
    int r = launch_adjoint(a, plan->vinc_ptr.as<int64_t>(), plan->vinc.as<int32_t>(), g_vertices, L_out, plan->stream);
    if (r < 0) return cuda_fail((cudaError_t)(-r), "adjoint kernel launch");
    mark(plan, 2, false);
    plan->last_launches = r;
    return FE_OK;
}

// ---------------------------------------------------------------------------
// diagnostics (Sec. 5.2, 5.3)
// ---------------------------------------------------------------------------
fe_status fe_geometry(fe_plan *plan, int mode, const double *vertices, int64_t c0, int64_t c1, double *G,
                      double *absdet, int32_t *used_fp64) {
    g_err.clear();
    if (!plan || !G) return fail(FE_ERR_INVALID_ARG, "NULL argument");
    if (plan->boxed) return fail(FE_ERR_UNSUPPORTED, "fe_geometry: simplices only");
    if (mode < FE_GEOMETRY_FP64 || mode > FE_GEOMETRY_MIXED) return fail(FE_ERR_INVALID_ARG, "unknown mode %d", mode);
    if (c0 < 0 || c1 > plan->n_cells || c0 > c1) return fail(FE_ERR_INVALID_ARG, "cell range out of bounds");
    const int r = launch_diag_geometry(vertices ? vertices : plan->vertices.as<double>(), plan->cells.as<int32_t>(), c0,
                                       c1, plan->d, mode, G, absdet, used_fp64, plan->status.as<int>(), plan->stream);
    if (r < 0) return cuda_fail((cudaError_t)(-r), "geometry kernel launch");
    plan->last_launches = r;
    return FE_OK;
}

fe_status fe_mass_fp16_products(fe_plan *plan, const double *kappa, const double *w, int64_t c0, int64_t c1, float *A,
                                float *b) {
    g_err.clear();
    if (!plan || !kappa || (!A && !b)) return fail(FE_ERR_INVALID_ARG, "NULL argument");
    if (plan->boxed) return fail(FE_ERR_UNSUPPORTED, "fe_mass_fp16_products: simplices only");
    if (b && !w) return fail(FE_ERR_INVALID_ARG, "the action needs w");
    if (c0 < 0 || c1 > plan->n_cells || c0 > c1) return fail(FE_ERR_INVALID_ARG, "cell range out of bounds");
    const int r = launch_diag_mass_fp16(plan->vertices.as<double>(), plan->cells.as<int32_t>(),
                                        plan->cell_dofs.as<int32_t>(), c0, c1, plan->d, plan->n_phi, plan->n_q, kappa,
                                        plan->weights.as<double>(), plan->phi.as<double>(), w, A, b,
                                        plan->status.as<int>(), plan->stream);
    if (r < 0) return cuda_fail((cudaError_t)(-r), "FP16-product kernel launch");
    plan->last_launches = r;
    return FE_OK;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
}  // extern "C"

struct fe_batch {
    std::vector<fe_plan *> plans;
    unsigned forms = 0;
    int prec = 0;
    cudaStream_t stream = nullptr;
    TcArgs targs{};
    AsmArgs aargs{};
    size_t smem = 0;
    bool assemble = false;
    DevBuf tc_segs, asm_segs, status;
    std::vector<std::unique_ptr<DevBuf>> ws;
    std::vector<F64Args> f64;   // FP64 path: one launch per plan and form
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t n_cells = 0, nnz = 0;
    int launches = 0;
    ~fe_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

static fe_status batch_launch(fe_batch &B, int &launches) {
    launches = 0;
    if (B.prec == FE_PREC_FP64) {
        for (const F64Args &f : B.f64) {
            int r = launch_f64_elements(f, B.stream);
            if (r < 0) return cuda_fail((cudaError_t)(-r), "FP64 element kernel launch");
            launches += r;
        }
    } else {
        int r = launch_factor(B.targs, B.stream);
        if (r < 0) return cuda_fail((cudaError_t)(-r), "factor kernel launch");
        launches += r;
        r = launch_tc_elements(B.targs, B.smem, B.stream);
        if (r < 0) return cuda_fail((cudaError_t)(-r), "tensor-core element kernel launch");
        launches += r;
    }
    if (B.assemble) {
        int r = launch_assemble(B.aargs, B.prec == FE_PREC_FP64, B.stream);
        if (r < 0) return cuda_fail((cudaError_t)(-r), "assembly kernel launch");
        launches += r;
    }
    return FE_OK;
}

extern "C" {

fe_status fe_batch_create(fe_batch **out, fe_plan *const *plans, int n_plans, unsigned forms, fe_precision prec,
                          const double *const *kappa, void *const *A_stiffness, void *const *A_mass,
                          void *const *csr_stiffness, void *const *csr_mass, void *cuda_stream) {
    g_err.clear();
    if (!out || !plans || !kappa || n_plans <= 0) return fail(FE_ERR_INVALID_ARG, "NULL argument or empty batch");
    *out = nullptr;
    if (!cuda_stream) return fail(FE_ERR_INVALID_ARG, "a batch needs a non-default stream (it is captured in a graph)");
    if ((int)prec < 0 || (int)prec > 5) return fail(FE_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (forms == 0 || (forms & ~3u)) return fail(FE_ERR_INVALID_ARG, "bad form mask");
    const bool want_csr = csr_stiffness || csr_mass;
    for (int i = 0; i < n_plans; ++i) {
        fe_status st = check_call(plans[i], forms, prec);
        if (st) return st;
        if (plans[i]->boxed) return fail(FE_ERR_UNSUPPORTED, "batches take simplex plans only (plan %d is boxed)", i);
        if (want_csr && need_pattern(plans[i])) return FE_ERR_INVALID_ARG;
        if (!kappa[i]) return fail(FE_ERR_INVALID_ARG, "NULL kappa for plan %d", i);
        if (want_csr) {
            if ((forms & FE_FORM_STIFFNESS) && (!csr_stiffness || !csr_stiffness[i]))
                return fail(FE_ERR_INVALID_ARG, "NULL stiffness CSR output for plan %d", i);
            if ((forms & FE_FORM_MASS) && (!csr_mass || !csr_mass[i]))
                return fail(FE_ERR_INVALID_ARG, "NULL mass CSR output for plan %d", i);
        }
    }
    auto bt = std::make_unique<fe_batch>();
    fe_batch &B = *bt;
    B.plans.assign(plans, plans + n_plans);
    B.forms = forms;
    B.prec = (int)prec;
    B.stream = static_cast<cudaStream_t>(cuda_stream);
    B.assemble = want_csr;
    std::vector<int> zero(4, 0);
    FE_CUDA(upload(B.status, zero, B.stream), "batch status");
    const bool fp64 = prec == FE_PREC_FP64;
    std::vector<TcSeg> tsegs;
    std::vector<AsmSeg> asegs;
    int64_t rows = 0, chunks = 0;
    for (int i = 0; i < n_plans; ++i) {
        fe_plan *P = plans[i];
        void *A[2] = {A_stiffness ? A_stiffness[i] : nullptr, A_mass ? A_mass[i] : nullptr};
        const size_t ebytes = (fp64 ? 8 : 4) * (size_t)P->n_cells * P->n_phi * P->n_phi;
        for (int fi = 0; fi < 2; ++fi) {
            if (!(forms & (fi == 0 ? FE_FORM_STIFFNESS : FE_FORM_MASS)) || A[fi]) continue;
            B.ws.emplace_back(new DevBuf);
            fe_status st = ensure_ws(*B.ws.back(), ebytes, "batch element workspace");
            if (st) return st;
            A[fi] = B.ws.back()->p;
        }
        B.n_cells += P->n_cells;
        B.nnz += P->nnz;
        if (fp64) {
            for (unsigned form : {(unsigned)FE_FORM_STIFFNESS, (unsigned)FE_FORM_MASS}) {
                if (!(forms & form)) continue;
                F64Args a{};
                a.vertices = P->vertices.as<double>();
                a.cells = P->cells.as<int32_t>();
                a.n_cells = P->n_cells;
                a.d = P->d;
                a.kappa = kappa[i];
                a.weights = P->weights.as<double>();
                a.n_q = P->n_q;
                a.n_phi = P->n_phi;
                a.tab = (form == FE_FORM_STIFFNESS) ? P->dphi.as<double>() : P->phi.as<double>();
                a.form = (int)form;
                a.out = static_cast<double *>(A[form_index(form)]);
                a.status = B.status.as<int>();
                B.f64.push_back(a);
            }
        } else {
            B.ws.emplace_back(new DevBuf);
            DevBuf &w = *B.ws.back();
            B.ws.emplace_back(new DevBuf);
            DevBuf &cf = *B.ws.back();
            fe_status st = ensure_ws(w, win_bytes(P), "batch window workspace");
            if (!st) st = ensure_ws(cf, cellf_bytes(P), "batch cell factor workspace");
            if (st) return st;
            tsegs.push_back(make_tc_seg(P, forms, (int)prec, nullptr, kappa[i], A, w.as<float>(), cf.as<float>()));
        }
        if (want_csr) {
            void *csr[2] = {csr_stiffness ? csr_stiffness[i] : nullptr, csr_mass ? csr_mass[i] : nullptr};
            const void *Ac[2] = {A[0], A[1]};
            asegs.push_back(make_asm_seg(P, forms, Ac, csr));
            asegs.back().row_begin = rows;
            asegs.back().chunk_begin = chunks;
            rows += P->n_dofs;
            chunks += P->n_chunks;
        }
    }
    if (!fp64) {
        TcArgs &a = B.targs;
        unsigned long long limit = 0;
        for (fe_plan *P : B.plans) limit = std::max(limit, P->wait_limit_ns);
        tc_finalize(a, tsegs.data(), (int)tsegs.size(), (int)prec, B.status.as<int>(), limit);
        FE_CUDA(upload(B.tc_segs, tsegs, B.stream), "upload batch segments");
        a.segs = B.tc_segs.as<TcSeg>();
        a.n_segs = (int)tsegs.size();
        B.smem = tc_smem_bytes(a);
        if (B.smem > 227 * 1024) return fail(FE_ERR_UNSUPPORTED, "batch shapes need %zu bytes of shared memory", B.smem);
    }
    if (want_csr) {
        FE_CUDA(upload(B.asm_segs, asegs, B.stream), "upload batch assembly segments");
        B.aargs.segs = B.asm_segs.as<AsmSeg>();
        B.aargs.n_segs = (int)asegs.size();
        B.aargs.n_rows = rows;
        B.aargs.n_chunks = chunks;
        B.aargs.n_forms = n_forms_of(forms);
        B.aargs.algo = plans[0]->asm_algo;
    }
    // one eager run (sets kernel attributes, checks the inputs), then capture
    int launches = 0;
    fe_status st = batch_launch(B, launches);
    if (st) return st;
    FE_CUDA(cudaStreamSynchronize(B.stream), "batch warm-up");
    int stw = 0;
    FE_CUDA(cudaMemcpy(&stw, B.status.p, sizeof(int), cudaMemcpyDeviceToHost), "batch status");
    if (stw) return fail(stw & ST_TIMEOUT ? FE_ERR_TIMEOUT : (stw & ST_NONFINITE ? FE_ERR_NONFINITE : FE_ERR_DEGENERATE_CELL),
                         "batch warm-up reported status %d", stw);
    FE_CUDA(cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    st = batch_launch(B, launches);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(B.stream, &g);
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    B.graph = g;
    FE_CUDA(cudaGraphInstantiate(&B.exec, B.graph, 0), "graph instantiate");
    B.launches = launches;
    *out = bt.release();
    return FE_OK;
}

fe_status fe_batch_run(fe_batch *batch) {
    g_err.clear();
    if (!batch) return fail(FE_ERR_INVALID_ARG, "NULL batch");
    FE_CUDA(cudaGraphLaunch(batch->exec, batch->stream), "graph launch");
    return FE_OK;
}

fe_status fe_batch_sync(fe_batch *batch) {
    if (!batch) return fail(FE_ERR_INVALID_ARG, "NULL batch");
    int st = 0;
    FE_CUDA(cudaStreamSynchronize(batch->stream), "sync");
    FE_CUDA(cudaMemcpy(&st, batch->status.p, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    if (st) FE_CUDA(cudaMemset(batch->status.p, 0, sizeof(int)), "clear status");
    if (st & ST_TIMEOUT) return fail(FE_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
    if (st & ST_NONFINITE) return fail(FE_ERR_NONFINITE, "non-finite geometry or coefficient");
    if (st & ST_DEGENERATE) return fail(FE_ERR_DEGENERATE_CELL, "degenerate cell (det J == 0)");
    if (st & ST_SATURATED) return fail(FE_ERR_NONFINITE, "a reduced-precision value overflowed its storage format");
    return FE_OK;
}

fe_status fe_batch_sizes(const fe_batch *batch, int64_t *n_cells, int64_t *nnz, int32_t *launches) {
    if (!batch) return fail(FE_ERR_INVALID_ARG, "NULL batch");
    if (n_cells) *n_cells = batch->n_cells;
    if (nnz) *nnz = batch->nnz;
    if (launches) *launches = batch->launches;
    return FE_OK;
}

fe_status fe_batch_destroy(fe_batch *batch) {
    if (batch) {
        cudaStreamSynchronize(batch->stream);
        delete batch;
    }
    return FE_OK;
}

}  // extern "C"
