// Linear forms (Algorithm 2 of the paper): the action of the mass or Poisson
// form on a known FE function w,
//
//   b^c_j = a_K(w, phi_j) = sum_s sum_q B_sjq r_sq,
//   r_sq  = w_q z(X_q) (G grad w(X_q))_s        (Poisson, Sec. 3.1)
//   r_q   = w_q z(X_q) |det J| w(X_q)           (mass),
//
// with grad w(X_q) = sum_k w^c_k B_skq the reference gradient, followed by the
// vector assembly v^g = L b (Sec. 3.3).
//
// Precisions.  FP64 throughout, or the mixed strategy of Sec. 4.5: the
// tabulated B and the cell's coefficients w^c rounded once to the storage
// format (TF32, BF16, FP16; the casting remark after the theorem on r_s), G
// and w_q z(X_q) in FP32 as for the bilinear forms, r_s computed in FP32 and
// rounded once to the storage format (the theorem on r_s), and both
// contractions accumulated in FP32 -- each product of two stored values is
// exact in FP32, as on the tensor cores.  FP16's narrow range needs scaling:
// on a fine mesh r_s (about w_q kappa h^d) falls far below FP16's smallest
// normal number.  For FP16 each cell's coefficients are rounded as
// w^c 2^e_w with max|w^c| 2^e_w in [2^7, 2^8), and r_s as r_s 2^(e_w + e_r),
// where e_r brings the a-priori bound of |r_s / kappa| (largest weight *
// max_s sum_t |G_st| (mass: |det J|) * max_{s,q} sum_k |B_skq| * 2^8) to
// [2^3, 2^4); the cell vector is unscaled at the end.  Powers of two are
// exact, so the rounding errors are those of the unscaled values wherever
// both are normal numbers; an r_s that still overflows FP16 (kappa above
// about 4096) sets the saturation status instead of returning infinities.
//
// Kernels.  The work is a few tens of flops per byte of kappa, below what the
// tensor cores need to matter, so it runs on the CUDA cores.  Mixed
// precisions, n_phi <= 56 (P1-P8 triangles, P1-P5 tetrahedra): one thread per
// cell serving every requested form in one pass (kappa, the geometry and the
// conversions shared), its coefficients and cell vectors in registers as
// pairs of local dofs, both contractions as paired FP32 FMAs (two FMAs per
// instruction) against the packed table B[q][s][k] of a window of quadrature
// points in shared memory (every thread reads the same entry: broadcast
// loads), and w_q z(X_q) of the window formed once per (cell, point) from
// coalesced 16-byte kappa loads (several rows in flight per warp) and staged
// transposed at an odd pitch (conflict-free reads).  The paired FMAs keep the
// FP32 rounding of each product-sum exactly as scalar FMAs.  FP64 and larger
// elements: one warp per cell, lanes over the
// quadrature points for grad w and r, lanes over the local dofs for b (the
// transposed table B_t[s][q][k] keeps those loads coalesced).  The vector
// assembly sums each dof's cell entries in increasing cell order (the
// incidence lists), so every result is bitwise reproducible.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fe_device.cuh"

namespace fe {

namespace {

constexpr int ACT_WARPS = 4;
constexpr int ACT_CELLS = 128;   // cells (threads) per CTA of the thread-per-cell kernel

__device__ __forceinline__ float round_storage(float x, int prec) {
    if (prec == FE_PREC_BF16) return __bfloat162float(__float2bfloat16_rn(x));
    if (prec == FE_PREC_FP16) return __half2float(__float2half_rn(x));
    if (prec == FE_PREC_TF32 || prec == FE_PREC_TF32X3) return __uint_as_float(round_tf32(x));
    return x;
}

// Rounding to the storage format without a branch: the FP32 fraction rounded
// to 7 (BF16) or 10 (TF32, FP16) bits, half to even, on the integer units (a
// carry into the exponent gives the correctly rounded power of two); FP16's
// narrower range by selects: below 2^-14 the fixed subnormal quantum 2^-24
// (round to nearest even integer multiple), from 65520 on infinity.
struct StorageRound {
    unsigned shift, mask, bias;
    bool half;
    __device__ explicit StorageRound(int prec)
        : shift(prec == FE_PREC_BF16 ? 16u : 13u), mask(~((1u << shift) - 1u)), bias((1u << (shift - 1u)) - 1u),
          half(prec == FE_PREC_FP16) {}
    __device__ __forceinline__ float operator()(float x) const {
        const unsigned u = __float_as_uint(x);
        float y = __uint_as_float((u + bias + ((u >> shift) & 1u)) & mask);
        const float ax = fabsf(x);
        const float sub = __fmul_rn(rintf(__fmul_rn(x, 0x1p24f)), 0x1p-24f);
        y = (half && ax < 0x1p-14f) ? sub : y;
        y = (half && ax >= 65520.f) ? copysignf(__int_as_float(0x7f800000), x) : y;
        return y;
    }
};

// FP64 -> FP32, round to nearest even: values whose FP32 image is a normal
// number take the exponent rebias and the rounding of the 29 dropped bits as
// one 64-bit add; everything else goes through f64_to_f32_rne.
__device__ __forceinline__ float to_f32(double x, int &nonfinite) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned hi = static_cast<unsigned>(u >> 32);
    if (((hi >> 20) & 0x7FFu) - 897u < 254u) {
        const unsigned long long r = u - (896ull << 52) + 0x0FFFFFFFull + ((u >> 29) & 1ull);
        return __uint_as_float((static_cast<unsigned>(r >> 29) & 0x7FFFFFFFu) | (hi & 0x80000000u));
    }
    return f64_to_f32_rne(x, nonfinite);
}

// e such that x 2^e lies in [2^(target-1), 2^target) (0 for zero or a
// non-finite x), clamped to [-120, 120] so that 2^e and 2^-e are normal FP32.
__device__ __forceinline__ int scale_exp(float x, int target) {
    if (!(x > 0.f) || !isfinite(x)) return 0;
    int e;
    frexpf(x, &e);
    return min(120, max(-120, target - e));
}

// Index of G_st in the packed upper triangle (G00 G01 G02 G11 G12 G22; d = 2:
// G00 G01 G11).
__device__ __forceinline__ constexpr int sym_index(int d, int s, int t) {
    return (s <= t) ? s * d - s * (s - 1) / 2 + (t - s) : t * d - t * (t - 1) / 2 + (s - t);
}

// ---------------------------------------------------------------------------
// One thread per cell (mixed precisions)
// ---------------------------------------------------------------------------
// Shared-memory load the compiler may not merge with an earlier load of the
// same address: the second pass over the table re-reads it instead of keeping
// the first pass's values live (which spills for the larger elements).
__device__ __forceinline__ float4 lds4_fresh(const float *p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(smem_u32(p)));
    return v;
}

template <bool FRESH>
__device__ __forceinline__ float4 lds4(const float *p) {
    if constexpr (FRESH) return lds4_fresh(p);
    return *reinterpret_cast<const float4 *>(p);
}

// acc += sum over the pairs of one table segment (KE floats, pairs of local
// dofs) times the coefficient pairs
template <int NP2, int KE, bool FRESH>
__device__ __forceinline__ float2 seg_dot(const float *seg, const float2 (&wp)[NP2], float2 acc) {
#pragma unroll
    for (int c4 = 0; c4 < KE / 4; ++c4) {
        const float4 L = lds4<FRESH>(seg + 4 * c4);
        if (2 * c4 < NP2) acc = __ffma2_rn(make_float2(L.x, L.y), wp[2 * c4], acc);
        if (2 * c4 + 1 < NP2) acc = __ffma2_rn(make_float2(L.z, L.w), wp[2 * c4 + 1], acc);
    }
    return acc;
}
// bp += table segment * r (pairs)
template <int NP2, int KE, bool FRESH>
__device__ __forceinline__ void seg_axpy(const float *seg, float r, float2 (&bp)[NP2]) {
    const float2 rr = make_float2(r, r);
#pragma unroll
    for (int c4 = 0; c4 < KE / 4; ++c4) {
        const float4 L = lds4<FRESH>(seg + 4 * c4);
        if (2 * c4 < NP2) bp[2 * c4] = __ffma2_rn(make_float2(L.x, L.y), rr, bp[2 * c4]);
        if (2 * c4 + 1 < NP2) bp[2 * c4 + 1] = __ffma2_rn(make_float2(L.z, L.w), rr, bp[2 * c4 + 1]);
    }
}

// CTAs per SM the register budget is sized for: 5 (at most 96 registers) where
// the mass-carrying instances fit it, so that a mesh of up to 5 x 128 cells
// per SM runs in one wave; 3 for the largest elements
constexpr int act_min_ctas(int nphi, int forms) {
    return (nphi > 36 || (forms == 3 && nphi > 21)) ? 3 : (nphi <= 20 && forms != 1) ? 5 : 4;
}

template <int D, int NPHI, int FORMS>
__global__ void __launch_bounds__(ACT_CELLS, act_min_ctas(NPHI, FORMS))
action_cells_kernel(const __grid_constant__ ActArgs a) {
    constexpr bool STIFF = FORMS & 1, MASS = FORMS & 2;
    constexpr int NP2 = (NPHI + 1) / 2;             // pairs of local dofs
    constexpr int KE = act_seg_floats(NPHI);        // floats per table segment
    constexpr int ROW = act_row_floats(D, NPHI, FORMS);
    constexpr int OP = NPHI | 1;                    // odd pitch of the output staging: conflict-free
    // keep the first pass's table entries in registers for the second pass
    // while they fit beside the coefficients and cell vectors; else re-read
    constexpr bool FRESH = KE * ((STIFF ? D : 0) + (MASS ? 1 : 0)) + 2 * NP2 * (1 + STIFF + MASS) > 112;
    extern __shared__ __align__(16) float act_sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c0 = (int64_t)blockIdx.x * ACT_CELLS;
    const int ncl = (int)((a.n_cells - c0) < ACT_CELLS ? (a.n_cells - c0) : ACT_CELLS);
    const bool live = tid < ncl;
    const int64_t c = c0 + tid;
    const int nq = a.n_q, QW = a.qw;
    float *tab_s = act_sm;                            // [QW][ROW] table window
    float *wk_s = act_sm + (size_t)QW * ROW;          // [QW][ACT_CELLS + 1] w_q z(X_q) of the window
    float *wts_s = wk_s + (size_t)QW * (ACT_CELLS + 1);  // [n_q] FP32 weights
    const StorageRound rnd(a.prec);
    float2 wp[NP2], bs[NP2], bm[NP2];
    float g6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, adet = 0.f;
#pragma unroll
    for (int p = 0; p < NP2; ++p) {
        wp[p] = make_float2(0.f, 0.f);
        bs[p] = make_float2(0.f, 0.f);
        bm[p] = make_float2(0.f, 0.f);
    }
    int nonfinite = 0;
    for (int q = tid; q < nq; q += ACT_CELLS) wts_s[q] = f64_to_f32_rne(__ldg(a.weights + q), nonfinite);
    const bool fp16 = a.prec == FE_PREC_FP16;
    float unscale[2] = {1.f, 1.f};   // Poisson, mass
    if (live) {
        const int32_t *dofs = a.cell_dofs + c * NPHI;
        float wl[NPHI];
        float wmax = 0.f;
#pragma unroll
        for (int k = 0; k < NPHI; ++k) {
            wl[k] = to_f32(__ldg(a.w + __ldg(dofs + k)), nonfinite);
            wmax = fmaxf(wmax, fabsf(wl[k]));
        }
        const int st = cell_g32(a.vertices, a.cells, c, D, g6, adet);
        if (st) {
            atomicOr(a.status, st);
#pragma unroll
            for (int j = 0; j < 6; ++j) g6[j] = 0.f;
            adet = 0.f;
        }
        if (fp16) {
            const int e_w = scale_exp(wmax, ACT_W_TARGET);
            const float sw = ldexpf(1.f, e_w);
#pragma unroll
            for (int k = 0; k < NPHI; ++k) wl[k] *= sw;
            float gn = 0.f;
#pragma unroll
            for (int s = 0; s < D; ++s) {
                float row = 0.f;
#pragma unroll
                for (int t = 0; t < D; ++t) row += fabsf(g6[sym_index(D, s, t)]);
                gn = fmaxf(gn, row);
            }
            const int e_s = scale_exp(a.r_bound[0] * gn, ACT_R_TARGET);
            const int e_m = scale_exp(a.r_bound[1] * adet, ACT_R_TARGET);
#pragma unroll
            for (int j = 0; j < 6; ++j) g6[j] = ldexpf(g6[j], e_s);
            adet = ldexpf(adet, e_m);
            unscale[0] = ldexpf(ldexpf(1.f, -e_w), -e_s);
            unscale[1] = ldexpf(ldexpf(1.f, -e_w), -e_m);
        }
#pragma unroll
        for (int k = 0; k < NPHI; ++k) wl[k] = rnd(wl[k]);
#pragma unroll
        for (int p = 0; p < NP2; ++p) wp[p] = make_float2(wl[2 * p], 2 * p + 1 < NPHI ? wl[2 * p + 1] : 0.f);
    }
    // kappa rows as 16-byte pairs when the rows and the window start are even
    const bool pairs = ((nq & 1) == 0) && ((reinterpret_cast<uintptr_t>(a.kappa) & 15) == 0);
    for (int q0 = 0; q0 < nq; q0 += QW) {
        const int qn = (nq - q0) < QW ? (nq - q0) : QW;
        __syncthreads();   // the previous window is consumed
        {
            const float4 *src = reinterpret_cast<const float4 *>(static_cast<const float *>(a.tab) + (size_t)q0 * ROW);
            float4 *dst = reinterpret_cast<float4 *>(tab_s);
            for (int i = tid; i < qn * (ROW / 4); i += ACT_CELLS) dst[i] = __ldg(src + i);
        }
        // w_q z(X_q) = FP32(kappa) * FP32(w_q): a warp per row, its lanes over the
        // window's points, several rows in flight per warp
        constexpr int RU = 4;
        if (pairs && (q0 & 1) == 0) {
            const int npair = (qn + 1) >> 1;
            for (int r0 = warp; r0 < ncl; r0 += 4 * RU) {
                for (int j = lane; j < npair; j += 32) {
                    double2 v[RU];
#pragma unroll
                    for (int u = 0; u < RU; ++u) {
                        const int cl = r0 + 4 * u;
                        v[u] = cl < ncl ? __ldg(reinterpret_cast<const double2 *>(a.kappa + (c0 + cl) * nq + q0) + j)
                                        : make_double2(0.0, 0.0);
                    }
#pragma unroll
                    for (int u = 0; u < RU; ++u) {
                        const int cl = r0 + 4 * u;
                        if (cl >= ncl) continue;
                        const int qq = 2 * j;
                        wk_s[qq * (ACT_CELLS + 1) + cl] = to_f32(v[u].x, nonfinite) * wts_s[q0 + qq];
                        if (qq + 1 < qn) wk_s[(qq + 1) * (ACT_CELLS + 1) + cl] = to_f32(v[u].y, nonfinite) * wts_s[q0 + qq + 1];
                    }
                }
            }
        } else {
            for (int r0 = warp; r0 < ncl; r0 += 4 * RU) {
                for (int qq = lane; qq < qn; qq += 32) {
                    double v[RU];
#pragma unroll
                    for (int u = 0; u < RU; ++u) {
                        const int cl = r0 + 4 * u;
                        v[u] = cl < ncl ? __ldg(a.kappa + (c0 + cl) * nq + q0 + qq) : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < RU; ++u) {
                        const int cl = r0 + 4 * u;
                        if (cl < ncl) wk_s[qq * (ACT_CELLS + 1) + cl] = to_f32(v[u], nonfinite) * wts_s[q0 + qq];
                    }
                }
            }
        }
        __syncthreads();
        if (live) for (int qq = 0; qq < qn; ++qq) {
            const float wq = wk_s[qq * (ACT_CELLS + 1) + tid];
            const float *Bq = tab_s + (size_t)qq * ROW;
            if constexpr (STIFF) {
                // reference gradient of w, two partial sums per component
                float gw[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int s = 0; s < D; ++s) {
                    const float2 acc = seg_dot<NP2, KE, false>(Bq + s * KE, wp, make_float2(0.f, 0.f));
                    gw[s] = acc.x + acc.y;
                }
                float r[3];
                if constexpr (D == 3) {
                    r[0] = rnd(wq * fmaf(g6[0], gw[0], fmaf(g6[1], gw[1], g6[2] * gw[2])));
                    r[1] = rnd(wq * fmaf(g6[1], gw[0], fmaf(g6[3], gw[1], g6[4] * gw[2])));
                    r[2] = rnd(wq * fmaf(g6[2], gw[0], fmaf(g6[4], gw[1], g6[5] * gw[2])));
                } else {
                    r[0] = rnd(wq * fmaf(g6[0], gw[0], g6[1] * gw[1]));
                    r[1] = rnd(wq * fmaf(g6[1], gw[0], g6[2] * gw[1]));
                }
#pragma unroll
                for (int s = 0; s < D; ++s) seg_axpy<NP2, KE, FRESH>(Bq + s * KE, r[s], bs);
            }
            if constexpr (MASS) {
                const float *Bm = Bq + (STIFF ? D * KE : 0);
                const float2 acc = seg_dot<NP2, KE, false>(Bm, wp, make_float2(0.f, 0.f));
                const float rm = rnd(wq * adet * (acc.x + acc.y));
                seg_axpy<NP2, KE, FRESH>(Bm, rm, bm);
            }
        }
    }
    if (nonfinite) atomicOr(a.status, ST_NONFINITE);
    // cell vectors: staged, then one contiguous block per CTA and form
    float *out_s = act_sm;
    bool overflow = false;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        if (!(FORMS & (1 << f))) continue;
        __syncthreads();
        if (live) {
            const float2 *bp = f == 0 ? bs : bm;
            const float us = unscale[f];
#pragma unroll
            for (int p = 0; p < NP2; ++p) {
                overflow = overflow || !isfinite(bp[p].x) || !isfinite(bp[p].y);
                out_s[tid * OP + 2 * p] = bp[p].x * us;
                if (2 * p + 1 < NPHI) out_s[tid * OP + 2 * p + 1] = bp[p].y * us;
            }
        }
        __syncthreads();
        float *dst = static_cast<float *>(f == 0 ? a.b : a.b_mass) + c0 * NPHI;
        for (int i = tid; i < ncl * NPHI; i += ACT_CELLS) {
            const int cl = i / NPHI;
            dst[i] = out_s[cl * OP + (i - cl * NPHI)];
        }
    }
    // an FP16 r_s beyond the format's range (finite inputs, non-finite result)
    if (fp16 && overflow && !nonfinite) atomicOr(a.status, ST_SATURATED);
}

// ---------------------------------------------------------------------------
// One warp per cell (FP64, and elements above the thread-per-cell sizes)
// ---------------------------------------------------------------------------
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
        // the cell's coefficients (rounded to the storage format on the mixed
        // paths; FP16: scaled by 2^e_w first, see the file comment)
        const bool fp16 = sizeof(T) == 4 && a.prec == FE_PREC_FP16;
        float wmax = 0.f;
        for (int k = lane; k < nph; k += 32) {
            const double wv = __ldg(a.w + __ldg(a.cell_dofs + c * nph + k));
            ws[k] = (T)wv;
            wmax = fmaxf(wmax, fabsf((float)wv));
        }
        int e_w = 0;
        if (fp16) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
            e_w = scale_exp(wmax, ACT_W_TARGET);
        }
        if (sizeof(T) == 4)
            for (int k = lane; k < nph; k += 32) ws[k] = (T)round_storage(ldexpf((float)ws[k], e_w), a.prec);
        float unscale = 1.f;
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
            if (fp16) {
                float bound;
                if (nd == 1) {
                    bound = a.r_bound[1] * (float)gs[9];
                } else {
                    float gn = 0.f;
                    for (int s = 0; s < d; ++s) {
                        float row = 0.f;
                        for (int t = 0; t < d; ++t) row += fabsf((float)gs[s * d + t]);
                        gn = fmaxf(gn, row);
                    }
                    bound = a.r_bound[0] * gn;
                }
                const int e_r = scale_exp(bound, ACT_R_TARGET);
                for (int i = 0; i < 10; ++i) gs[i] = (T)ldexpf((float)gs[i], e_r);
                unscale = ldexpf(ldexpf(1.f, -e_w), -e_r);
            }
        }
        unscale = __shfl_sync(0xffffffffu, unscale, 0);
        __syncwarp();
        // grad w (or w) at the quadrature points, then r
        for (int q = lane; q < nq; q += 32) {
            const double kq = __ldg(a.kappa + c * nq + q);
            if (!isfinite(kq)) atomicOr(a.status, ST_NONFINITE);
            const T wk = (T)__ldg(a.weights + q) * (T)kq;
            if (nd == 1) {
                T val = T(0);
                for (int k = 0; k < nph; ++k) val = fma(B[(size_t)k * nq + q], ws[k], val);
                rs[q] = (sizeof(T) == 8) ? wk * gs[9] * val : (T)round_storage((float)(wk * gs[9] * val), a.prec);
            } else {
                T gw[3] = {T(0), T(0), T(0)};
                for (int k = 0; k < nph; ++k) {
                    const T wkv = ws[k];
                    for (int s = 0; s < d; ++s) gw[s] = fma(B[((size_t)s * nph + k) * nq + q], wkv, gw[s]);
                }
                for (int s = 0; s < d; ++s) {
                    T acc = T(0);
                    for (int t = 0; t < d; ++t) acc = fma(gs[s * d + t], gw[t], acc);
                    rs[s * nq + q] = (sizeof(T) == 8) ? wk * acc : (T)round_storage((float)(wk * acc), a.prec);
                }
            }
        }
        __syncwarp();
        // b_k = sum_s sum_q B_skq r_sq
        bool overflow = false;
        for (int k = lane; k < nph; k += 32) {
            T acc = T(0);
            for (int s = 0; s < nd; ++s)
                for (int q = 0; q < nq; ++q) acc = fma(Bt[((size_t)s * nq + q) * nph + k], rs[s * nq + q], acc);
            overflow = overflow || !isfinite((float)acc);
            static_cast<T *>(a.b)[c * nph + k] = acc * (T)unscale;
        }
        if (fp16 && overflow) atomicOr(a.status, ST_SATURATED);
        __syncwarp();
    }
}

// v_i = sum of b over the incidences (c, k) of dof i, in increasing cell order,
// for one or two forms; the loads of four incidences are issued together.
template <typename T, int NF>
__global__ void vector_assemble_kernel(int64_t n_dofs, const int64_t *__restrict__ inc_ptr,
                                       const int32_t *__restrict__ inc_elem, const T *__restrict__ b0,
                                       const T *__restrict__ b1, T *__restrict__ v0, T *__restrict__ v1) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_dofs) return;
    const int64_t j1 = __ldg(inc_ptr + i + 1);
    int64_t j = __ldg(inc_ptr + i);
    T s0 = T(0), s1 = T(0);
    for (; j + 4 <= j1; j += 4) {
        int e[4];
        T x0[4], x1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) e[u] = __ldg(inc_elem + j + u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x0[u] = b0[e[u]];
            if (NF > 1) x1[u] = b1[e[u]];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            s0 += x0[u];
            if (NF > 1) s1 += x1[u];
        }
    }
    for (; j < j1; ++j) {
        const int e = __ldg(inc_elem + j);
        s0 += b0[e];
        if (NF > 1) s1 += b1[e];
    }
    v0[i] = s0;
    if (NF > 1) v1[i] = s1;
}

template <int D, int NPHI, int FORMS>
int launch_cells(const ActArgs &a, size_t smem, cudaStream_t s) {
    auto k = action_cells_kernel<D, NPHI, FORMS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -(int)e;
    const int64_t blocks = (a.n_cells + ACT_CELLS - 1) / ACT_CELLS;
    k<<<(unsigned)blocks, ACT_CELLS, smem, s>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

template <int D, int NPHI>
int launch_forms(const ActArgs &a, size_t smem, cudaStream_t s) {
    switch (a.forms) {
    case 1: return launch_cells<D, NPHI, 1>(a, smem, s);
    case 2: return launch_cells<D, NPHI, 2>(a, smem, s);
    case 3: return launch_cells<D, NPHI, 3>(a, smem, s);
    default: return -(int)cudaErrorInvalidValue;
    }
}

int dispatch_cells(const ActArgs &a, size_t smem, cudaStream_t s) {
    if (a.d == 2) {
        switch (a.n_phi) {
        case 3: return launch_forms<2, 3>(a, smem, s);
        case 6: return launch_forms<2, 6>(a, smem, s);
        case 10: return launch_forms<2, 10>(a, smem, s);
        case 15: return launch_forms<2, 15>(a, smem, s);
        case 21: return launch_forms<2, 21>(a, smem, s);
        case 28: return launch_forms<2, 28>(a, smem, s);
        case 36: return launch_forms<2, 36>(a, smem, s);
        case 45: return launch_forms<2, 45>(a, smem, s);
        default: return -(int)cudaErrorInvalidValue;
        }
    }
    switch (a.n_phi) {
    case 4: return launch_forms<3, 4>(a, smem, s);
    case 10: return launch_forms<3, 10>(a, smem, s);
    case 20: return launch_forms<3, 20>(a, smem, s);
    case 35: return launch_forms<3, 35>(a, smem, s);
    case 56: return launch_forms<3, 56>(a, smem, s);
    default: return -(int)cudaErrorInvalidValue;
    }
}

}  // namespace

bool action_per_cell(int d, int n_phi, bool fp64) {
    if (fp64) return false;
    // P1-P8 triangles (n_phi = (p+1)(p+2)/2 = 3 .. 45) and P1-P5 tetrahedra (4 .. 56)
    if (d == 2) return n_phi == 3 || n_phi == 6 || n_phi == 10 || n_phi == 15 || n_phi == 21 || n_phi == 28 ||
                       n_phi == 36 || n_phi == 45;
    return n_phi == 4 || n_phi == 10 || n_phi == 20 || n_phi == 35 || n_phi == 56;
}

int action_window(int d, int n_phi, int n_q, int forms) {
    const int per_q = act_row_floats(d, n_phi, forms) * 4 + (ACT_CELLS + 1) * 4;
    int qw = (kActSmemTarget - n_q * 4) / per_q;
    if (qw < 1) qw = 1;
    if (qw >= n_q) return n_q;
    const int nwin = (n_q + qw - 1) / qw;
    return (n_q + nwin - 1) / nwin;
}

size_t action_smem_bytes(const ActArgs &a, bool fp64) {
    if (action_per_cell(a.d, a.n_phi, fp64)) {
        // table window, w_q z(X_q) window [QW][ACT_CELLS + 1], FP32 weights; the
        // output staging reuses the same space
        const size_t win = (size_t)a.qw * (act_row_floats(a.d, a.n_phi, a.forms) + ACT_CELLS + 1) * 4 +
                           (size_t)a.n_q * 4;
        const size_t out = (size_t)ACT_CELLS * (a.n_phi | 1) * 4;
        return win > out ? win : out;
    }
    const int nd = (a.form == FE_FORM_STIFFNESS) ? a.d : 1;
    return (size_t)ACT_WARPS * (((a.n_phi + 1) & ~1) + nd * a.n_q + 10) * (fp64 ? 8 : 4);
}

int launch_action(const ActArgs &a, bool fp64, cudaStream_t s) {
    if (a.n_cells <= 0) return 0;
    const size_t smem = action_smem_bytes(a, fp64);
    if (action_per_cell(a.d, a.n_phi, fp64)) return dispatch_cells(a, smem, s);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
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

int launch_vector_assemble(int64_t n_dofs, const int64_t *inc_ptr, const int32_t *inc_elem, const void *b0,
                           const void *b1, void *v0, void *v1, bool fp64, cudaStream_t s) {
    if (n_dofs <= 0) return 0;
    const unsigned blocks = (unsigned)((n_dofs + 255) / 256);
    if (fp64) {
        auto B0 = static_cast<const double *>(b0), B1 = static_cast<const double *>(b1);
        auto V0 = static_cast<double *>(v0), V1 = static_cast<double *>(v1);
        if (b1) vector_assemble_kernel<double, 2><<<blocks, 256, 0, s>>>(n_dofs, inc_ptr, inc_elem, B0, B1, V0, V1);
        else vector_assemble_kernel<double, 1><<<blocks, 256, 0, s>>>(n_dofs, inc_ptr, inc_elem, B0, B0, V0, V0);
    } else {
        auto B0 = static_cast<const float *>(b0), B1 = static_cast<const float *>(b1);
        auto V0 = static_cast<float *>(v0), V1 = static_cast<float *>(v1);
        if (b1) vector_assemble_kernel<float, 2><<<blocks, 256, 0, s>>>(n_dofs, inc_ptr, inc_elem, B0, B1, V0, V1);
        else vector_assemble_kernel<float, 1><<<blocks, 256, 0, s>>>(n_dofs, inc_ptr, inc_elem, B0, B0, V0, V0);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

}  // namespace fe
