// Adjoint of L = v^T A^g u for the stiffness form (calculus; the paper has
// no adjoint).  With the reference gradients of the FE functions at the
// quadrature points, gu_q = sum_l B_{.lq} u_dof(c,l) and gv_q likewise, and
// K = J^{-1} = C^T / det J (cofactors, recomputed here from the vertices):
//   L_c            = sum_q w_q kappa_cq |det J| (K^T gu_q).(K^T gv_q)
//   dL/dkappa_cq   = w_q |det J| (K^T gu_q).(K^T gv_q)
//   S              = sum_q w_q kappa_cq gu_q gv_q^T
//   dL_c/dJ        = |det J| [ tr(K K^T S) K^T - K^T S^T K K^T - K^T S K K^T ]
//   dL/dx^(j)      = column j-1 of dL_c/dJ (j >= 1), minus their sum (j = 0).
// Kernel 1 (one thread per cell, FP64) writes g_kappa, the per-cell vertex
// contributions and L_c; kernel 2 sums the contributions of each vertex in
// increasing cell order (vertex incidence stream, no atomics); kernel 3 sums
// L_c in a fixed order.  Everything is deterministic.
//
// General gradient g on the CSR values (L = sum_e g_e A^g_e, the backward pass
// of the assembly): with G^c_kl = g at the CSR slot of (dof(c,k), dof(c,l))
// (the transpose of A^g = L D L^T, Sec. 3.3) the rank-one gu_q gv_q^T above
// becomes
//   T_q[r][b]      = sum_kl G^c_kl B_{r l q} B_{b k q},
//   dL/dkappa_cq   = w_q |det J| sum_rb (K K^T)_rb T_q[r][b],
//   S              = sum_q w_q kappa_cq T_q,   L_c = |det J| sum_rb (K K^T)_rb S_rb,
// and dL_c/dJ is the same function of S.  One warp per cell: the lanes gather
// G^c into shared memory (each slot by binary search in its sorted CSR row),
// then take one quadrature point each; S is summed across the warp in a fixed
// butterfly order.
#include <mutex>

#include "fe_adjoint.h"
#include "fe_device.cuh"

namespace fe {

namespace {

// dL_c/dx for the d + 1 vertices of a cell from K = J^{-1}, |det J| and S.
__device__ void vertex_contributions(const double (&K)[3][3], double absdet, const double (&S)[3][3], int d,
                                     double *gx) {
    double KKt[3][3], tr = 0.0;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += K[i][k] * K[j][k];
            KKt[i][j] = s;
        }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) tr += KKt[i][j] * S[j][i];
    // M1 = S K K^T and M2 = S^T K K^T, then T = K^T (M1 + M2)
    double dJ[3][3];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double t = 0.0;
            for (int r = 0; r < d; ++r) {
                double m = 0.0;
                for (int b = 0; b < d; ++b) m += (S[r][b] + S[b][r]) * KKt[b][j];
                t += K[r][i] * m;
            }
            dJ[i][j] = absdet * (tr * K[j][i] - t);
        }
    for (int i = 0; i < d; ++i) {
        double sum = 0.0;
        for (int j = 0; j < d; ++j) {
            gx[(j + 1) * d + i] = dJ[i][j];
            sum += dJ[i][j];
        }
        gx[0 * d + i] = -sum;
    }
}

__global__ void __launch_bounds__(128) adjoint_cell_kernel(const __grid_constant__ AdjArgs a) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.n_cells) return;
    const int d = a.d, nph = a.n_phi, nq = a.n_q;
    CellGeom geo;
    int st = cell_geometry(a.vertices, a.cells, c, d, geo);
    double *gx = a.g_cell_x ? a.g_cell_x + c * (d + 1) * d : nullptr;
    if (st) {
        atomicOr(a.status, st);
        if (a.g_kappa)
            for (int q = 0; q < nq; ++q) a.g_kappa[c * nq + q] = 0.0;
        if (gx)
            for (int i = 0; i < (d + 1) * d; ++i) gx[i] = 0.0;
        a.L_cell[c] = 0.0;
        return;
    }
    // K = J^{-1} = C^T / det  ->  K[r][i] = C[i][r] / det
    double K[3][3];
    const double idet = 1.0 / geo.det;
    for (int r = 0; r < d; ++r)
        for (int i = 0; i < d; ++i) K[r][i] = geo.C[i * d + r] * idet;
    double S[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double L = 0.0;
    const int32_t *dofs = a.cell_dofs + c * nph;
    for (int q = 0; q < nq; ++q) {
        double gu[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
        for (int l = 0; l < nph; ++l) {
            const int32_t g = __ldg(dofs + l);
            const double ul = (double)__ldg(a.u + g), vl = (double)__ldg(a.v + g);
            for (int s = 0; s < d; ++s) {
                const double b = __ldg(a.dphi + ((size_t)s * nph + l) * nq + q);
                gu[s] = fma(b, ul, gu[s]);
                gv[s] = fma(b, vl, gv[s]);
            }
        }
        double dot = 0.0;
        for (int i = 0; i < d; ++i) {
            double pu = 0.0, pv = 0.0;
            for (int r = 0; r < d; ++r) {
                pu = fma(K[r][i], gu[r], pu);
                pv = fma(K[r][i], gv[r], pv);
            }
            dot = fma(pu, pv, dot);
        }
        const double w = __ldg(a.weights + q);
        const double kap = __ldg(a.kappa + c * nq + q);
        if (a.g_kappa) a.g_kappa[c * nq + q] = w * geo.absdet * dot;
        const double wk = w * kap;
        L = fma(wk * geo.absdet, dot, L);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) S[i][j] = fma(wk * gu[i], gv[j], S[i][j]);
    }
    a.L_cell[c] = L;
    if (!gx) return;
    vertex_contributions(K, geo.absdet, S, d, gx);
}

// Index of col in the sorted CSR row `row` (the entry exists: the pattern
// holds every pair of dofs that share a cell).
__device__ __forceinline__ int64_t csr_slot(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                                            int32_t row, int32_t col) {
    int64_t lo = __ldg(row_ptr + row), hi = __ldg(row_ptr + row + 1) - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(col_idx + mid) < col) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int D>
__global__ void adjoint_values_kernel(const __grid_constant__ AdjValArgs av) {
    const AdjArgs &a = av.base;
    extern __shared__ double adjv_sm[];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    constexpr int d = D;
    const int nph = a.n_phi, nq = a.n_q;
    double *Gs = adjv_sm + (size_t)warp * nph * nph;   // G^c, row-major k, l
    for (int64_t c = (int64_t)blockIdx.x * nwarps + warp; c < a.n_cells; c += (int64_t)gridDim.x * nwarps) {
        const int32_t *dofs = a.cell_dofs + c * nph;
        for (int i = lane; i < nph * nph; i += 32) {
            const int k = i / nph, l = i - k * nph;
            Gs[i] = __ldg(av.gvals + csr_slot(av.row_ptr, av.col_idx, __ldg(dofs + k), __ldg(dofs + l)));
        }
        // geometry on lane 0, broadcast
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, absdet = 0.0;
        int st = 0;
        if (lane == 0) {
            CellGeom geo;
            st = cell_geometry(a.vertices, a.cells, c, d, geo);
            if (!st) {
                const double idet = 1.0 / geo.det;
                for (int r = 0; r < d; ++r)
                    for (int i = 0; i < d; ++i) K[r][i] = geo.C[i * d + r] * idet;
                absdet = geo.absdet;
            }
        }
        st = __shfl_sync(full, st, 0);
        absdet = __shfl_sync(full, absdet, 0);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int i = 0; i < 3; ++i) K[r][i] = __shfl_sync(full, K[r][i], 0);
        __syncwarp();
        double *gx = a.g_cell_x ? a.g_cell_x + c * (d + 1) * d : nullptr;
        if (st) {
            if (lane == 0) {
                atomicOr(a.status, st);
                a.L_cell[c] = 0.0;
                if (gx)
                    for (int i = 0; i < (d + 1) * d; ++i) gx[i] = 0.0;
            }
            if (a.g_kappa)
                for (int q = lane; q < nq; q += 32) a.g_kappa[c * nq + q] = 0.0;
            __syncwarp();
            continue;
        }
        double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int r = 0; r < d; ++r)
            for (int b = 0; b < d; ++b) {
                double m = 0.0;
                for (int i = 0; i < d; ++i) m += K[r][i] * K[b][i];
                M[r][b] = m;
            }
        double S[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int q = lane; q < nq; q += 32) {
            double T[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
            for (int k = 0; k < nph; ++k) {
                double Z[3] = {0, 0, 0};   // Z_r = sum_l G^c_kl B_{r l q}
                for (int l = 0; l < nph; ++l) {
                    const double g = Gs[k * nph + l];
                    for (int r = 0; r < d; ++r) Z[r] = fma(g, __ldg(a.dphi + ((size_t)r * nph + l) * nq + q), Z[r]);
                }
                for (int b = 0; b < d; ++b) {
                    const double bb = __ldg(a.dphi + ((size_t)b * nph + k) * nq + q);
                    for (int r = 0; r < d; ++r) T[r][b] = fma(Z[r], bb, T[r][b]);
                }
            }
            double mt = 0.0;
            for (int r = 0; r < d; ++r)
                for (int b = 0; b < d; ++b) mt = fma(M[r][b], T[r][b], mt);
            const double w = __ldg(a.weights + q);
            if (a.g_kappa) a.g_kappa[c * nq + q] = w * absdet * mt;
            const double wk = w * __ldg(a.kappa + c * nq + q);
            for (int r = 0; r < d; ++r)
                for (int b = 0; b < d; ++b) S[r][b] = fma(wk, T[r][b], S[r][b]);
        }
        // S over the warp: a butterfly, the same sum on every lane
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) S[r][b] += __shfl_xor_sync(full, S[r][b], o);
        if (lane == 0) {
            double L = 0.0;
            for (int r = 0; r < d; ++r)
                for (int b = 0; b < d; ++b) L = fma(M[r][b], S[r][b], L);
            a.L_cell[c] = absdet * L;
            if (gx) vertex_contributions(K, absdet, S, d, gx);
        }
        __syncwarp();   // Gs is rewritten for the next cell
    }
}

// Sum each vertex's per-cell contributions in increasing cell order.
__global__ void vertex_gather_kernel(int64_t n_vertices, int d, const int64_t *__restrict__ vinc_ptr,
                                     const int32_t *__restrict__ vinc, const double *__restrict__ g_cell_x,
                                     double *__restrict__ g_vertices) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_vertices * d) return;
    const int64_t v = t / d;
    const int i = (int)(t - v * d);
    double s = 0.0;
    for (int64_t e = vinc_ptr[v]; e < vinc_ptr[v + 1]; ++e) s += g_cell_x[(int64_t)vinc[e] * d + i];
    g_vertices[t] = s;
}

// Fixed-order sum of n values by one block.
__global__ void ordered_sum_kernel(const double *__restrict__ x, int64_t n, double *__restrict__ out) {
    __shared__ double part[1024];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int64_t i = t; i < n; i += blockDim.x) s += x[i];
    part[t] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w) part[t] += part[t + w];
        __syncthreads();
    }
    if (t == 0) *out = part[0];
}

}  // namespace

// ---------------------------------------------------------------------------
// Fixed scratch for fe_adjoint_noalloc.  Callers that may not allocate device
// memory (their device memory belongs to their own allocator or a fixed
// budget, or they cannot afford the implicit device synchronisation of
// cudaMalloc / cudaFree inside a latency-critical loop) get the adjoint's
// per-cell scratch -- the vertex-gradient contributions of every cell and the
// per-cell L -- from this file-scope array instead of a plan workspace.  It is
// part of the module, so every GPU that loads the library holds it until the
// process exits.  In host code the name g_noalloc_scratch is only a host-side
// stand-in: the device address comes from cudaGetSymbolAddress, looked up
// once per device below with that device current.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {
std::mutex g_noalloc_mutex;
constexpr int kMaxDevices = 64;
double *g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

cudaError_t noalloc_scratch(double **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *ptr = g_noalloc_ptr[dev];
    return cudaSuccess;
}

int launch_adjoint_values(const AdjValArgs &av, const int64_t *vinc_ptr, const int32_t *vinc, double *g_vertices,
                          double *L_out, cudaStream_t s) {
    const AdjArgs &a = av.base;
    if (a.n_cells <= 0) return 0;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t per_warp = sizeof(double) * (size_t)a.n_phi * a.n_phi;
    int warps = (int)((size_t)(96 << 10) / per_warp);
    warps = warps < 1 ? 1 : (warps > 4 ? 4 : warps);
    const size_t smem = per_warp * warps;
    auto kern = a.d == 3 ? adjoint_values_kernel<3> : adjoint_values_kernel<2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -(int)e;
    int64_t blocks = (a.n_cells + warps - 1) / warps;
    if (blocks > (int64_t)sms * 32) blocks = (int64_t)sms * 32;
    kern<<<(unsigned)blocks, 32 * warps, smem, s>>>(av);
    int launches = 1;
    if (g_vertices) {
        const int64_t n = a.n_vertices * a.d;
        vertex_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a.n_vertices, a.d, vinc_ptr, vinc,
                                                                          a.g_cell_x, g_vertices);
        ++launches;
    }
    if (L_out) {
        ordered_sum_kernel<<<1, 1024, 0, s>>>(a.L_cell, a.n_cells, L_out);
        ++launches;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return -(int)e;
    return launches;
}

int launch_adjoint(const AdjArgs &a, const int64_t *vinc_ptr, const int32_t *vinc, double *g_vertices, double *L_out,
                   cudaStream_t s) {
    if (a.n_cells <= 0) return 0;
    int launches = 0;
    adjoint_cell_kernel<<<(unsigned)((a.n_cells + 127) / 128), 128, 0, s>>>(a);
    ++launches;
    if (g_vertices) {
        const int64_t n = a.n_vertices * a.d;
        vertex_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a.n_vertices, a.d, vinc_ptr, vinc,
                                                                          a.g_cell_x, g_vertices);
        ++launches;
    }
    if (L_out) {
        ordered_sum_kernel<<<1, 1024, 0, s>>>(a.L_cell, a.n_cells, L_out);
        ++launches;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return -(int)e;
    return launches;
}

}  // namespace fe
