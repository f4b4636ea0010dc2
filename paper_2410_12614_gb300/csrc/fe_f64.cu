// FP64 element-matrix kernel on the CUDA cores (the double-precision
// reference path).
//
// Algorithm 1 with the variant of the Remark that follows it: for each cell
//   H~_s[q][l] = sum_t C_stq B_tlq,   C_stq = w_q kappa_cq G_st   (Sec. 3.1)
//   A[k][l]    = sum_s sum_q B_skq H~_s[q][l]                      (k <= l)
// (mass: one "s", C_q = w_q kappa_cq |det J|, B = phi).  Everything is FP64.
// Boxed cells take G_st and |det J| per quadrature point from geo_q, which
// box_geometry_kernel forms from the multilinear map at every point.
// A block owns `tc` cells; the tabulation B and H~ are staged in shared
// memory `qc` quadrature points at a time; every thread accumulates EPT
// upper-triangle entries in registers and writes both mirror positions.
#include <algorithm>

#include "fe_device.cuh"

namespace fe {

namespace {

constexpr int F64_THREADS = 256;

constexpr int F64_EPT = 16;  // upper-triangle entries per thread

__global__ void __launch_bounds__(F64_THREADS) f64_element_kernel(const __grid_constant__ F64Args a, int n_echunks) {
    extern __shared__ double sm64[];
    const int d = a.d;
    const int nd = (a.form == FE_FORM_STIFFNESS) ? d : 1;
    const int nph = a.n_phi;
    const int n_sym = nph * (nph + 1) / 2;
    const int TC = a.tc, QC = a.qc;
    double *tab = sm64;                          // [nd][nph][QC]
    double *W = tab + (size_t)nd * nph * QC;     // [TC][QC]
    double *H = W + (size_t)TC * QC;             // [TC][nd][QC][nph]
    double *Gs = H + (size_t)TC * nd * QC * nph; // [TC][7]: G pairs and |det J|
    const int tid = threadIdx.x;
    const int64_t cell0 = (int64_t)(blockIdx.x / n_echunks) * TC;
    const int e_base = (blockIdx.x % n_echunks) * (F64_THREADS * F64_EPT);

    for (int c = tid; c < TC; c += F64_THREADS) {
        const int64_t cg = cell0 + c;
        double *g = Gs + c * 7;
        for (int j = 0; j < 7; ++j) g[j] = 0.0;
        if (cg < a.n_cells && !a.geo_q) {
            CellGeom geo;
            int st = cell_geometry(a.vertices, a.cells, cg, d, geo);
            if (st) {
                if (e_base == 0) atomicOr(a.status, st);
            } else {
                for (int j = 0; j < 6; ++j) g[j] = geo.G[j];
                g[6] = geo.absdet;
            }
        }
    }
    // entries owned by this thread, packed as c | k << 8 | l << 16 (-1: none)
    int ent[F64_EPT];
    double acc[F64_EPT];
#pragma unroll
    for (int r = 0; r < F64_EPT; ++r) {
        const int e = e_base + tid + r * F64_THREADS;
        ent[r] = -1;
        acc[r] = 0.0;
        if (e < TC * n_sym) {
            const int c = e / n_sym, s = e - c * n_sym;
            int k = 0, rem = s;  // s -> (k, l), k <= l, row-major upper triangle
            while (rem >= nph - k) {
                rem -= nph - k;
                ++k;
            }
            if (cell0 + c < a.n_cells) ent[r] = c | (k << 8) | ((k + rem) << 16);
        }
    }
    __syncthreads();
    for (int q0 = 0; q0 < a.n_q; q0 += QC) {
        for (int i = tid; i < nd * nph * QC; i += F64_THREADS) {
            const int qq = i % QC, k = (i / QC) % nph, s = i / (QC * nph);
            const int q = q0 + qq;
            tab[i] = (q < a.n_q) ? __ldg(a.tab + ((size_t)s * nph + k) * a.n_q + q) : 0.0;
        }
        for (int i = tid; i < TC * QC; i += F64_THREADS) {
            const int c = i / QC, qq = i - c * QC;
            const int64_t cg = cell0 + c;
            const int q = q0 + qq;
            W[i] = (cg < a.n_cells && q < a.n_q) ? __ldg(a.weights + q) * __ldg(a.kappa + cg * a.n_q + q) : 0.0;
        }
        __syncthreads();
        for (int i = tid; i < TC * nd * QC * nph; i += F64_THREADS) {
            const int l = i % nph, qq = (i / nph) % QC, s = (i / (nph * QC)) % nd, c = i / (nph * QC * nd);
            const double w = W[c * QC + qq];
            // simplices: the cell's G; boxed cells: G at this point (zero weight past the ends)
            const double *g = Gs + c * 7;
            if (a.geo_q && w != 0.0) g = a.geo_q + ((cell0 + c) * a.n_q + q0 + qq) * 7;
            double h;
            if (nd == 1) {
                h = w * g[6] * tab[l * QC + qq];
            } else {
                h = 0.0;
                for (int t = 0; t < nd; ++t) {
                    // index of the symmetric pair (min(s,t), max(s,t))
                    const int lo = s < t ? s : t, hi = s < t ? t : s;
                    const int pj = (d == 3) ? (lo == 0 ? hi : (lo == 1 ? 2 + hi : 5)) : (lo + hi);
                    h += w * g[pj] * tab[((size_t)t * nph + l) * QC + qq];
                }
            }
            H[i] = h;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < F64_EPT; ++r) {
            if (ent[r] < 0) continue;
            const int c = ent[r] & 0xFF, k = (ent[r] >> 8) & 0xFF, l = ent[r] >> 16;
            double sum = acc[r];
            for (int s = 0; s < nd; ++s) {
                const double *bk = tab + ((size_t)s * nph + k) * QC;
                const double *hl = H + (((size_t)c * nd + s) * QC) * nph + l;
                for (int qq = 0; qq < QC; ++qq) sum = fma(bk[qq], hl[(size_t)qq * nph], sum);
            }
            acc[r] = sum;
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < F64_EPT; ++r) {
        if (ent[r] < 0) continue;
        const int c = ent[r] & 0xFF, k = (ent[r] >> 8) & 0xFF, l = ent[r] >> 16;
        double *dst = a.out + (cell0 + c) * (int64_t)nph * nph;
        dst[k * nph + l] = acc[r];
        dst[l * nph + k] = acc[r];
    }
}

// One thread per (cell, point): G pairs and |det J| of a boxed cell at a
// quadrature point, FP64 (box_point_geometry).
__global__ void box_geometry_kernel(const double *__restrict__ vertices, const int32_t *__restrict__ cells,
                                    int64_t n_cells, int d, int nv, const double *__restrict__ dpsi, int n_q,
                                    double *__restrict__ geo_q, int *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cells * n_q) return;
    const int64_t c = i / n_q;
    const int q = (int)(i - c * n_q);
    double xv[8 * 3];
    for (int v = 0; v < nv; ++v) {
        const int64_t vid = __ldg(cells + c * nv + v);
        for (int r = 0; r < 3; ++r) xv[v * 3 + r] = (r < d) ? __ldg(vertices + vid * d + r) : 0.0;
    }
    CellGeom g;
    const int st = box_point_geometry(xv, nv, dpsi, n_q, q, d, g);
    if (st) atomicOr(status, st);
    double *o = geo_q + i * 7;
    for (int j = 0; j < 6; ++j) o[j] = st ? 0.0 : g.G[j];
    o[6] = st ? 0.0 : g.absdet;
}

}  // namespace

int launch_box_geometry(const double *vertices, const int32_t *cells, int64_t n_cells, int d, int nv,
                        const double *dpsi, int n_q, double *geo_q, int *status, cudaStream_t s) {
    const int64_t n = n_cells * n_q;
    if (n <= 0) return 0;
    box_geometry_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(vertices, cells, n_cells, d, nv, dpsi, n_q, geo_q,
                                                                     status);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

int launch_f64_elements(const F64Args &a0, cudaStream_t s) {
    if (a0.n_cells <= 0) return 0;
    F64Args a = a0;
    const int nd = (a.form == FE_FORM_STIFFNESS) ? a.d : 1;
    const int n_sym = a.n_phi * (a.n_phi + 1) / 2;
    const int per_block = F64_THREADS * F64_EPT;
    int n_echunks = 1;
    if (n_sym <= per_block) {
        a.tc = std::max(1, std::min(64, per_block / n_sym));
    } else {
        a.tc = 1;
        n_echunks = (n_sym + per_block - 1) / per_block;
    }
    a.qc = 16;
    auto bytes = [&](int tc, int qc) {
        return sizeof(double) * ((size_t)nd * a.n_phi * qc + (size_t)tc * qc + (size_t)tc * nd * qc * a.n_phi + 7 * tc);
    };
    while (bytes(a.tc, a.qc) > 96 * 1024 && a.qc > 4) a.qc /= 2;
    while (bytes(a.tc, a.qc) > 96 * 1024 && a.tc > 1) a.tc = (a.tc + 1) / 2;
    const size_t smem = bytes(a.tc, a.qc);
    const int64_t grid = (a.n_cells + a.tc - 1) / a.tc * n_echunks;
    cudaError_t e = cudaFuncSetAttribute(f64_element_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -(int)e;
    f64_element_kernel<<<(unsigned)grid, F64_THREADS, smem, s>>>(a, n_echunks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return -(int)e;
    return 1;
}

}  // namespace fe
