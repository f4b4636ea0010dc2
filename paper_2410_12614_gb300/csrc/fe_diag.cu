// Diagnostic kernels reproducing the paper's error studies (Sec. 5.2, 5.3).
// They are opt-in experiments, not part of the production path.
//
// geometry_kernel (Sec. 5.2, geometry errors): the Poisson geometry tensor
// G = |det J| J^-1 J^-T and |det J| of every cell in one of three modes:
//   FP64   J, cofactors, det J and G in FP64 (the reference);
//   FP32   the same formulas evaluated exclusively in FP32 from the vertex
//          coordinates rounded to FP32 (the paper's experiment), every
//          operation an explicitly rounded IEEE FP32 operation in a fixed
//          order, so that the result is reproducible bit for bit;
//   MIXED  the production path of the reduced-precision kernels: FP64
//          cofactors and det J, G in FP32, and FP64 G on cells whose
//          off-diagonal sums cancel or leave FP32's range (the per-cell
//          geometry precision that the remark after the experiment suggests);
//          a flag per cell tells which cells took FP64.
//
// mass_fp16_kernel (Sec. 5.3, accumulation errors): the mass bilinear form
// and the mass action with the matrix-matrix (matrix-vector) products in FP16
// and everything else in FP32, as in the paper's experiment
// (u_s = u_g = u_p = 2^-24, u_q = 2^-11): one thread per (cell, k),
//   C_q   = fl32(fl32(w_q kappa_cq) |det J|) 2^e       (|det J| from FP32 geometry)
//   H_kq  = fl32(C_q phi_kq)                           (Algorithm 1, H = C B^T)
//   A_kl  = 2^-e sum16_q fl16(phi_lq H_kq)              (q increasing, from 0)
//   w_q   = sum32_l phi_lq w_l                          (l increasing, from 0)
//   r_q   = fl32(C_q w_q)                               (Algorithm 2, r)
//   b_k   = 2^-e sum16_q fl16(phi_kq r_q)
// where sum16 adds in FP16 with one rounding per addition and fl16 rounds the
// exact product once.  2^e (per cell) keeps the FP16 partial sums in range:
// sum_q |C_q| 2^e in [2^9, 2^10).  The FE coefficients are scaled by a power
// of two per cell as well (max |w^c| in [1, 2)) and unscaled at the end.
#include <cuda_fp16.h>

#include "fe_device.cuh"

namespace fe {

namespace {

struct DiagGeoArgs {
    const double *vertices;
    const int32_t *cells;
    int64_t c0, c1;
    int d, mode;
    double *G;        // [c1 - c0][d(d+1)/2]
    double *absdet;   // [c1 - c0] or null
    int32_t *used_fp64;
    int *status;
};

__global__ void geometry_kernel(const DiagGeoArgs a) {
    const int64_t c = a.c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.c1) return;
    const int d = a.d, np = d * (d + 1) / 2;
    const int64_t i = c - a.c0;
    double G[6] = {0, 0, 0, 0, 0, 0}, adet = 0.0;
    int used = 0, st = 0;
    if (a.mode == 0) {
        CellGeom geo;
        st = cell_geometry(a.vertices, a.cells, c, d, geo);
        for (int j = 0; j < np; ++j) G[j] = geo.G[j];
        adet = geo.absdet;
    } else if (a.mode == 1) {
        float x[4][3];
        const int nv = d + 1;
        for (int k = 0; k < nv; ++k) {
            const int64_t v = a.cells[c * nv + k];
            for (int r = 0; r < d; ++r) x[k][r] = __double2float_rn(a.vertices[v * d + r]);
        }
        float J[3][3], C[9], det;
        if (d == 3) {
            for (int r = 0; r < 3; ++r)
                for (int j = 0; j < 3; ++j) J[r][j] = __fsub_rn(x[j + 1][r], x[0][r]);
            auto m2 = [](float p, float q, float s, float t) { return __fsub_rn(__fmul_rn(p, q), __fmul_rn(s, t)); };
            C[0] = m2(J[1][1], J[2][2], J[1][2], J[2][1]);
            C[1] = m2(J[1][2], J[2][0], J[1][0], J[2][2]);
            C[2] = m2(J[1][0], J[2][1], J[1][1], J[2][0]);
            C[3] = m2(J[0][2], J[2][1], J[0][1], J[2][2]);
            C[4] = m2(J[0][0], J[2][2], J[0][2], J[2][0]);
            C[5] = m2(J[0][1], J[2][0], J[0][0], J[2][1]);
            C[6] = m2(J[0][1], J[1][2], J[0][2], J[1][1]);
            C[7] = m2(J[0][2], J[1][0], J[0][0], J[1][2]);
            C[8] = m2(J[0][0], J[1][1], J[0][1], J[1][0]);
            det = __fadd_rn(__fadd_rn(__fmul_rn(J[0][0], C[0]), __fmul_rn(J[0][1], C[1])), __fmul_rn(J[0][2], C[2]));
        } else {
            J[0][0] = __fsub_rn(x[1][0], x[0][0]);
            J[0][1] = __fsub_rn(x[2][0], x[0][0]);
            J[1][0] = __fsub_rn(x[1][1], x[0][1]);
            J[1][1] = __fsub_rn(x[2][1], x[0][1]);
            C[0] = J[1][1];
            C[1] = -J[1][0];
            C[2] = -J[0][1];
            C[3] = J[0][0];
            det = __fsub_rn(__fmul_rn(J[0][0], J[1][1]), __fmul_rn(J[0][1], J[1][0]));
        }
        const float ad = fabsf(det);
        const float inv = __fdiv_rn(1.0f, ad);
        if (!isfinite(det) || det == 0.f) st = isfinite(det) ? ST_DEGENERATE : ST_NONFINITE;
        int j = 0;
        for (int s = 0; s < d; ++s)
            for (int t = s; t < d; ++t) {
                float acc = __fmul_rn(C[s], C[t]);
                for (int r = 1; r < d; ++r) acc = __fadd_rn(acc, __fmul_rn(C[r * d + s], C[r * d + t]));
                G[j++] = (double)__fmul_rn(acc, inv);
            }
        adet = (double)ad;
    } else {
        float g6[6], ad = 0.f;
        st = cell_g32_tagged(a.vertices, a.cells, c, d, g6, ad, used);
        for (int j = 0; j < np; ++j) G[j] = (double)g6[j];
        adet = (double)ad;
    }
    if (st) atomicOr(a.status, st);
    for (int j = 0; j < np; ++j) a.G[i * np + j] = G[j];
    if (a.absdet) a.absdet[i] = adet;
    if (a.used_fp64) a.used_fp64[i] = used;
}

struct DiagMassArgs {
    const double *vertices;
    const int32_t *cells;
    const int32_t *cell_dofs;
    int64_t c0, c1;
    int d, n_phi, n_q;
    const double *kappa;     // [n_cells][n_q]
    const double *weights;   // [n_q]
    const double *phi;       // [n_phi][n_q]
    const double *w;         // [n_dofs] or null
    float *A;                // [c1 - c0][n_phi][n_phi] or null
    float *b;                // [c1 - c0][n_phi] or null
    int *status;
};

// |det J| of cell c from FP32 coordinates in FP32 (fixed order, no contraction).
__device__ float absdet_f32(const double *vertices, const int32_t *cells, int64_t c, int d) {
    float x[4][3];
    const int nv = d + 1;
    for (int k = 0; k < nv; ++k) {
        const int64_t v = cells[c * nv + k];
        for (int r = 0; r < d; ++r) x[k][r] = __double2float_rn(vertices[v * d + r]);
    }
    if (d == 2) {
        const float j00 = __fsub_rn(x[1][0], x[0][0]), j01 = __fsub_rn(x[2][0], x[0][0]);
        const float j10 = __fsub_rn(x[1][1], x[0][1]), j11 = __fsub_rn(x[2][1], x[0][1]);
        return fabsf(__fsub_rn(__fmul_rn(j00, j11), __fmul_rn(j01, j10)));
    }
    float J[3][3];
    for (int r = 0; r < 3; ++r)
        for (int j = 0; j < 3; ++j) J[r][j] = __fsub_rn(x[j + 1][r], x[0][r]);
    const float c0 = __fsub_rn(__fmul_rn(J[1][1], J[2][2]), __fmul_rn(J[1][2], J[2][1]));
    const float c1 = __fsub_rn(__fmul_rn(J[1][2], J[2][0]), __fmul_rn(J[1][0], J[2][2]));
    const float c2 = __fsub_rn(__fmul_rn(J[1][0], J[2][1]), __fmul_rn(J[1][1], J[2][0]));
    return fabsf(__fadd_rn(__fadd_rn(__fmul_rn(J[0][0], c0), __fmul_rn(J[0][1], c1)), __fmul_rn(J[0][2], c2)));
}

// e such that x 2^e lies in [2^(t-1), 2^t) (0 for zero or non-finite x)
__device__ __forceinline__ int diag_scale_exp(float x, int t) {
    if (!(x > 0.f) || !isfinite(x)) return 0;
    int e;
    frexpf(x, &e);
    return t - e;
}

__global__ void mass_fp16_kernel(const DiagMassArgs a) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nph = a.n_phi, nq = a.n_q;
    const int64_t c = a.c0 + gid / nph;
    const int k = (int)(gid % nph);
    if (c >= a.c1) return;
    const int64_t i = c - a.c0;
    const float adet = absdet_f32(a.vertices, a.cells, c, a.d);
    // sum_q |C_q| in FP32 for the cell's scale
    float csum = 0.f;
    for (int q = 0; q < nq; ++q) {
        const float wk = __fmul_rn(__double2float_rn(a.weights[q]), __double2float_rn(a.kappa[c * nq + q]));
        csum = __fadd_rn(csum, fabsf(__fmul_rn(wk, adet)));
    }
    const int e = diag_scale_exp(csum, 10);
    const float sc = ldexpf(1.f, e), us = ldexpf(1.f, -e);
    if (a.A) {
        for (int l = 0; l < nph; ++l) {
            __half acc = __float2half_rn(0.f);
            for (int q = 0; q < nq; ++q) {
                const float wk = __fmul_rn(__double2float_rn(a.weights[q]), __double2float_rn(a.kappa[c * nq + q]));
                const float Cq = __fmul_rn(__fmul_rn(wk, adet), sc);
                const float H = __fmul_rn(Cq, __double2float_rn(a.phi[(size_t)k * nq + q]));
                const float pl = __double2float_rn(a.phi[(size_t)l * nq + q]);
                acc = __hadd(acc, __double2half((double)pl * (double)H));
            }
            a.A[(i * nph + k) * nph + l] = __fmul_rn(__half2float(acc), us);
        }
    }
    if (a.b) {
        // the cell's coefficients scaled to max |w^c| in [1, 2)
        float wmax = 0.f;
        for (int l = 0; l < nph; ++l) wmax = fmaxf(wmax, fabsf(__double2float_rn(a.w[a.cell_dofs[c * nph + l]])));
        const int ew = diag_scale_exp(wmax, 1);
        const float sw = ldexpf(1.f, ew);
        __half acc = __float2half_rn(0.f);
        for (int q = 0; q < nq; ++q) {
            float wq = 0.f;
            for (int l = 0; l < nph; ++l)
                wq = __fadd_rn(wq, __fmul_rn(__double2float_rn(a.phi[(size_t)l * nq + q]),
                                            __fmul_rn(__double2float_rn(a.w[a.cell_dofs[c * nph + l]]), sw)));
            const float wk = __fmul_rn(__double2float_rn(a.weights[q]), __double2float_rn(a.kappa[c * nq + q]));
            const float Cq = __fmul_rn(__fmul_rn(wk, adet), sc);
            const float r = __fmul_rn(Cq, wq);
            const float pk = __double2float_rn(a.phi[(size_t)k * nq + q]);
            acc = __hadd(acc, __double2half((double)pk * (double)r));
        }
        a.b[i * nph + k] = __fmul_rn(__fmul_rn(__half2float(acc), us), ldexpf(1.f, -ew));
    }
}

}  // namespace

int launch_diag_geometry(const double *vertices, const int32_t *cells, int64_t c0, int64_t c1, int d, int mode,
                         double *G, double *absdet, int32_t *used_fp64, int *status, cudaStream_t s) {
    if (c1 <= c0) return 0;
    DiagGeoArgs a{vertices, cells, c0, c1, d, mode, G, absdet, used_fp64, status};
    const unsigned blocks = (unsigned)((c1 - c0 + 127) / 128);
    geometry_kernel<<<blocks, 128, 0, s>>>(a);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

int launch_diag_mass_fp16(const double *vertices, const int32_t *cells, const int32_t *cell_dofs, int64_t c0,
                          int64_t c1, int d, int n_phi, int n_q, const double *kappa, const double *weights,
                          const double *phi, const double *w, float *A, float *b, int *status, cudaStream_t s) {
    if (c1 <= c0) return 0;
    DiagMassArgs a{vertices, cells, cell_dofs, c0, c1, d, n_phi, n_q, kappa, weights, phi, w, A, b, status};
    const int64_t threads = (c1 - c0) * n_phi;
    const unsigned blocks = (unsigned)((threads + 127) / 128);
    mass_fp16_kernel<<<blocks, 128, 0, s>>>(a);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

}  // namespace fe
