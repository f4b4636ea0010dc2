// Linear forms (Algorithm 2 of the paper): the action of the mass or Poisson
// form on a known FE function w,
//
//   b^c_j = a_K(w, phi_j) = sum_s sum_q B_sjq r_sq,
//   r_sq  = w_q z(X_q) (G grad w(X_q))_s        (Poisson, Sec. 3.1)
//   r_q   = w_q z(X_q) |det J| w(X_q)           (mass),
//
// with grad w(X_q) = sum_k w^c_k B_skq the reference gradient, followed by the
// vector assembly v^g = L b (Sec. 3.3).  The work is a few flops per byte of
// kappa, so it runs on the CUDA cores: one warp per cell, lanes over the
// quadrature points for grad w and r, lanes over the local dofs for b (the
// transposed table B_t[s][q][k] keeps those loads coalesced).  Precisions:
// FP64 throughout, or the mixed strategy of Sec. 4.5 with the tabulated B and
// the cell's coefficients w^c rounded once to the storage format (TF32, BF16,
// FP16) and everything else in FP32.  The vector assembly sums each dof's cell
// entries in increasing cell order (the incidence lists), so every result is
// bitwise reproducible.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fe_device.cuh"

namespace fe {

namespace {

constexpr int ACT_WARPS = 4;

__device__ __forceinline__ float round_storage(float x, int prec) {
    if (prec == FE_PREC_BF16) return __bfloat162float(__float2bfloat16_rn(x));
    if (prec == FE_PREC_FP16) return __half2float(__float2half_rn(x));
    if (prec == FE_PREC_TF32 || prec == FE_PREC_TF32X3) return __uint_as_float(round_tf32(x));
    return x;
}

template <typename T>
__global__ void __launch_bounds__(ACT_WARPS * 32) action_kernel(const __grid_constant__ ActArgs a) {
    extern __shared__ __align__(16) unsigned char act_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = a.d, nph = a.n_phi, nq = a.n_q;
    const int nd = (a.form == FE_FORM_STIFFNESS) ? d : 1;
    const int nph_pad = (nph + 1) & ~1;
    T *ws = reinterpret_cast<T *>(act_smem) + (size_t)warp * (nph_pad + nd * nq + 10);
    T *rs = ws + nph_pad;                 // [nd][nq]
    T *gs = rs + nd * nq;                 // G (d x d), |det J|
    const T *__restrict__ B = static_cast<const T *>(a.tab);      // [nd][nph][nq]
    const T *__restrict__ Bt = static_cast<const T *>(a.tab_t);   // [nd][nq][nph]
    const int64_t total_warps = (int64_t)gridDim.x * ACT_WARPS;
    for (int64_t c = (int64_t)blockIdx.x * ACT_WARPS + warp; c < a.n_cells; c += total_warps) {
        // the cell's coefficients (rounded to the storage format on the mixed paths)
        for (int k = lane; k < nph; k += 32) {
            const double wv = __ldg(a.w + __ldg(a.cell_dofs + c * nph + k));
            ws[k] = (sizeof(T) == 8) ? (T)wv : (T)round_storage((float)wv, a.prec);
        }
        if (lane == 0) {
            CellGeom geo;
            const int st = cell_geometry(a.vertices, a.cells, c, d, geo);
            if (st) atomicOr(a.status, st);
            int j = 0;
            for (int s = 0; s < d; ++s)
                for (int t = s; t < d; ++t, ++j) {
                    const T g = st ? T(0) : (T)geo.G[j];
                    gs[s * d + t] = g;
                    gs[t * d + s] = g;
                }
            gs[9] = st ? T(0) : (T)geo.absdet;
        }
        __syncwarp();
        // grad w (or w) at the quadrature points, then r
        for (int q = lane; q < nq; q += 32) {
            const T wk = (T)__ldg(a.weights + q) * (T)__ldg(a.kappa + c * nq + q);
            if (nd == 1) {
                T val = T(0);
                for (int k = 0; k < nph; ++k) val = fma(B[(size_t)k * nq + q], ws[k], val);
                rs[q] = wk * gs[9] * val;
            } else {
                T gw[3] = {T(0), T(0), T(0)};
                for (int k = 0; k < nph; ++k) {
                    const T wkv = ws[k];
                    for (int s = 0; s < d; ++s) gw[s] = fma(B[((size_t)s * nph + k) * nq + q], wkv, gw[s]);
                }
                for (int s = 0; s < d; ++s) {
                    T acc = T(0);
                    for (int t = 0; t < d; ++t) acc = fma(gs[s * d + t], gw[t], acc);
                    rs[s * nq + q] = wk * acc;
                }
            }
        }
        __syncwarp();
        // b_k = sum_s sum_q B_skq r_sq
        for (int k = lane; k < nph; k += 32) {
            T acc = T(0);
            for (int s = 0; s < nd; ++s)
                for (int q = 0; q < nq; ++q) acc = fma(Bt[((size_t)s * nq + q) * nph + k], rs[s * nq + q], acc);
            static_cast<T *>(a.b)[c * nph + k] = acc;
        }
        __syncwarp();
    }
}

// v_i = sum of b over the incidences (c, k) of dof i, in increasing cell order.
template <typename T>
__global__ void vector_assemble_kernel(int64_t n_dofs, const int64_t *__restrict__ inc_ptr,
                                       const int32_t *__restrict__ inc_elem, const T *__restrict__ b,
                                       T *__restrict__ v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_dofs) return;
    T s = T(0);
    for (int64_t j = __ldg(inc_ptr + i); j < __ldg(inc_ptr + i + 1); ++j) s += b[__ldg(inc_elem + j)];
    v[i] = s;
}

}  // namespace

size_t action_smem_bytes(const ActArgs &a, bool fp64) {
    const int nd = (a.form == FE_FORM_STIFFNESS) ? a.d : 1;
    return (size_t)ACT_WARPS * (((a.n_phi + 1) & ~1) + nd * a.n_q + 10) * (fp64 ? 8 : 4);
}

int launch_action(const ActArgs &a, bool fp64, cudaStream_t s) {
    if (a.n_cells <= 0) return 0;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    const size_t smem = action_smem_bytes(a, fp64);
    int64_t blocks = (a.n_cells + ACT_WARPS - 1) / ACT_WARPS;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    cudaError_t e;
    if (fp64) {
        e = cudaFuncSetAttribute(action_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) action_kernel<double><<<(unsigned)blocks, ACT_WARPS * 32, smem, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(action_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) action_kernel<float><<<(unsigned)blocks, ACT_WARPS * 32, smem, s>>>(a);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

int launch_vector_assemble(int64_t n_dofs, const int64_t *inc_ptr, const int32_t *inc_elem, const void *b, void *v,
                           bool fp64, cudaStream_t s) {
    if (n_dofs <= 0) return 0;
    const unsigned blocks = (unsigned)((n_dofs + 255) / 256);
    if (fp64)
        vector_assemble_kernel<double><<<blocks, 256, 0, s>>>(n_dofs, inc_ptr, inc_elem, static_cast<const double *>(b),
                                                             static_cast<double *>(v));
    else
        vector_assemble_kernel<float><<<blocks, 256, 0, s>>>(n_dofs, inc_ptr, inc_elem, static_cast<const float *>(b),
                                                            static_cast<float *>(v));
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

}  // namespace fe
