// Factor kernel: the per-cell inputs of the tensor-core contraction.
//
// For every tile of 128 cells (the element kernel's tiles, over one plan or a
// batch of segments) it forms
//   * the coefficient window w_q kappa_cq in FP32 (kappa rounded once from
//     FP64 on the integer units, times the FP32 weight), row-major with a
//     row length padded to a multiple of 4 points and zero past n_q;
//   * the geometry of Sec. 4.2 / 3.1: J, its cofactors and det J in FP64;
//     G = |det J| J^-1 J^-T = C^T C / |det J| from the cofactors either in
//     FP64 and rounded once (TF32x3, whose storage precision is close to
//     FP32's) or in FP32 from the cofactors and det J rounded once (the
//     other formats: G then carries a few FP32 roundings, far below their
//     u_s, and the FP64 pipe -- about two FMAs per clock per SM on this part
//     -- does a third of the work);
// C_(st,q) = (w_q kappa_cq) * (G_st 2^e_c) is then one FP32 product per
// operand element in the element kernel, rounded once to the storage format
// (the mixed strategy of Sec. 4.5 with u_s on C).
//
// Boxed cells (quadrilaterals, hexahedra) have a multilinear map whose J varies
// with the point: for them the kernel forms J, det J and G in FP64 at every
// quadrature point and writes one window per symmetric pair (w_q kappa_cq
// G_st(X_q), FP32 from the FP64 G rounded once) and one for the mass form
// (w_q kappa_cq |det J(X_q)|); the per-cell record then holds only the
// power-of-two scales, each form's chosen from the largest magnitude of its
// windows.
//
// Each CTA owns half a tile (64 cells): its four warps stream that part of
// the kappa block (a contiguous range) with coalesced loads, so the factor
// work runs at full occupancy instead of on the element kernel's four
// builder warps.
#include "fe_device.cuh"

namespace fe {

namespace {

constexpr int F_THREADS = 128;
constexpr int F_CELLS = 64;      // cells per CTA (half a tile): enough CTAs to hide the load latency
constexpr int F_WTS = 1024;   // weights table in shared memory (points)

template <bool BATCHED>
__device__ __forceinline__ const TcSeg &fseg_of(const TcArgs &a, int64_t t) {
    if (!BATCHED) return a.seg0;
    int lo = 0, hi = a.n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    return a.segs[lo];
}

template <bool BATCHED, bool G64>
__global__ void __launch_bounds__(F_THREADS, 8) factor_kernel(const __grid_constant__ TcArgs a) {
    __shared__ int rowmax[F_CELLS];       // max_q |w_q kappa_cq| of each row, as non-negative float bits
    __shared__ float wts[F_WTS];          // the segment's weights in FP32 (when they fit)
    __shared__ int flags;
    const int tid = threadIdx.x;
    const int64_t t = blockIdx.x / (TC_M / F_CELLS);
    const TcSeg &S = fseg_of<BATCHED>(a, t);
    const int64_t c0 = (t - S.tile_begin) * TC_M + (blockIdx.x % (TC_M / F_CELLS)) * F_CELLS;
    const int64_t left = S.n_cells - c0;
    const int nvalid = (int)(left < F_CELLS ? (left > 0 ? left : 0) : F_CELLS);
    const int n_q = S.n_q, ldw = S.ldw;
    const double *__restrict__ kb = S.kappa + c0 * n_q;   // the tile's kappa block
    const double *__restrict__ weights = S.weights;
    float *__restrict__ wb = S.win + c0 * ldw;             // the tile's window block
    const bool wts_smem = ldw <= F_WTS;
    if (tid < F_CELLS) rowmax[tid] = 0;
    if (tid == 0) flags = 0;
    if (wts_smem)
        for (int q = tid; q < ldw; q += F_THREADS) wts[q] = q < n_q ? (float)__ldg(weights + q) : 0.f;
    __syncthreads();
    // 1. the window, one item of 4 points per thread and step (consecutive
    //    threads, consecutive items: coalesced loads and 16-byte stores)
    int nonfinite = 0;
    const int ipr = ldw >> 2;
    const int n_items = nvalid * ipr;
    const bool need_max = a.target_exp > 1;
    const bool vec = ((n_q & 1) == 0) && ((reinterpret_cast<uintptr_t>(S.kappa) & 15) == 0);
    constexpr int IU = 4;
    for (int i0 = tid; i0 < n_items; i0 += F_THREADS * IU) {
        double raw[IU][4];
        int rr[IU], qq[IU];
#pragma unroll
        for (int u = 0; u < IU; ++u) {
            const int i = i0 + u * F_THREADS;
            const int r = i / ipr;
            const int q = 4 * (i - r * ipr);
            rr[u] = r;
            qq[u] = q;
            const double *src = kb + (int64_t)r * n_q + q;
            if (i < n_items && vec) {
                const double2 z = make_double2(0.0, 0.0);
                const double2 lo = q < n_q ? __ldg(reinterpret_cast<const double2 *>(src)) : z;
                const double2 hi = q + 2 < n_q ? __ldg(reinterpret_cast<const double2 *>(src + 2)) : z;
                raw[u][0] = lo.x;
                raw[u][1] = lo.y;
                raw[u][2] = hi.x;
                raw[u][3] = hi.y;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) raw[u][e] = (i < n_items && q + e < n_q) ? __ldg(src + e) : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < IU; ++u) {
            const int i = i0 + u * F_THREADS;
            if (i >= n_items) continue;
            const int q = qq[u];
            float v[4];
            float m = 0.f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float w = wts_smem ? wts[q + e] : (q + e < n_q ? (float)__ldg(weights + q + e) : 0.f);
                v[e] = (q + e < n_q) ? f64_to_f32_rne(raw[u][e], nonfinite) * w : 0.f;
                m = fmaxf(m, fabsf(v[e]));
            }
            *reinterpret_cast<float4 *>(wb + (int64_t)rr[u] * ldw + q) = make_float4(v[0], v[1], v[2], v[3]);
            if (need_max) atomicMax(&rowmax[rr[u]], __float_as_int(m));
        }
    }
    if (nonfinite) atomicOr(&flags, ST_NONFINITE);
    __syncthreads();
    // 2. geometry and scales, one thread per cell
    if (tid < nvalid) {
        const int64_t c = c0 + tid;
        float g6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, adet = 0.f;
        int st;
        if (G64) {
            CellGeom geo;
            st = cell_geometry(S.vertices, S.cells, c, S.d, geo);
            if (!st) {
#pragma unroll
                for (int j = 0; j < 6; ++j) g6[j] = (float)geo.G[j];
                adet = (float)geo.absdet;
            }
        } else {
            st = cell_g32(S.vertices, S.cells, c, S.d, g6, adet);
        }
        if (st) {
            atomicOr(&flags, st);
#pragma unroll
            for (int j = 0; j < 6; ++j) g6[j] = 0.f;
            adet = 0.f;
        }
        const float wmax = __int_as_float(rowmax[tid]);
        float rec[CELLF];
#pragma unroll
        for (int i = 0; i < CELLF; ++i) rec[i] = 0.f;
        for (int f = 0; f < MAX_FORMS; ++f) {
            if (!(S.form_mask & (1 << f))) continue;
            float gmax = 0.f;
            if (f == 0) {
#pragma unroll
                for (int j = 0; j < 6; ++j) gmax = fmaxf(gmax, fabsf(g6[j]));
            } else {
                gmax = adet;
            }
            int e_c = 0;
            if (need_max && !st) {
                const float cmax = wmax * gmax;
                if (cmax > 0.f && isfinite(cmax)) {
                    int e;
                    frexpf(cmax, &e);
                    e_c = a.target_exp - e;
                }
            }
            const float scale = ldexpf(1.f, e_c);
            rec[CELLF_UNSCALE + f] = ldexpf(S.op[f].p_inv_scale, -e_c);
            if (f == 0) {
#pragma unroll
                for (int j = 0; j < 6; ++j) rec[CELLF_G + j] = g6[j] * scale;
            } else {
                rec[CELLF_DET] = adet * scale;
            }
        }
        float4 *dst = reinterpret_cast<float4 *>(S.cellf + c * CELLF);
#pragma unroll
        for (int i = 0; i < CELLF / 4; ++i) dst[i] = make_float4(rec[4 * i], rec[4 * i + 1], rec[4 * i + 2], rec[4 * i + 3]);
    }
    __syncthreads();
    if (tid == 0 && flags) atomicOr(a.status, flags);
}

// Boxed cells (single plan): the geometry of every point in FP64, one window
// per symmetric pair and one for the mass form, and the per-cell scales.
__global__ void __launch_bounds__(F_THREADS) factor_box_kernel(const __grid_constant__ TcArgs a) {
    __shared__ int rowmax[F_CELLS];       // max |C| of each cell's pair windows, as non-negative float bits
    __shared__ int rowmax2[F_CELLS];      // max |C| of each cell's mass window
    __shared__ float wts[F_WTS];
    __shared__ int flags;
    const int tid = threadIdx.x;
    const int64_t t = blockIdx.x / (TC_M / F_CELLS);
    const TcSeg &S = a.seg0;
    const int64_t c0 = (t - S.tile_begin) * TC_M + (blockIdx.x % (TC_M / F_CELLS)) * F_CELLS;
    const int64_t left = S.n_cells - c0;
    const int nvalid = (int)(left < F_CELLS ? (left > 0 ? left : 0) : F_CELLS);
    const int n_q = S.n_q, ldw = S.ldw;
    const double *__restrict__ kb = S.kappa + c0 * n_q;
    const double *__restrict__ weights = S.weights;
    float *__restrict__ wb = S.win + c0 * ldw * S.win_slots;
    const bool wts_smem = ldw <= F_WTS;
    if (tid < F_CELLS) {
        rowmax[tid] = 0;
        rowmax2[tid] = 0;
    }
    if (tid == 0) flags = 0;
    if (wts_smem)
        for (int q = tid; q < ldw; q += F_THREADS) wts[q] = q < n_q ? (float)__ldg(weights + q) : 0.f;
    __syncthreads();
    // boxed cells: the geometry of every point (FP64), then the windows
    // C_(j),q = fl32(fl32(kappa) w_q) * fl32(G_j(X_q)) for the pairs and
    // fl32(kappa) w_q * fl32(|det J(X_q)|) for the mass form
    const int d = S.d, nv = S.nv, np = S.n_pairs, slots = S.win_slots;
    const bool need_max = a.target_exp > 1;
    int stat = 0, nonfinite = 0;
    for (int i = tid; i < nvalid * n_q; i += F_THREADS) {
        const int r = i / n_q, q = i - r * n_q;
        const int64_t c = c0 + r;
        double xv[8 * 3];
        for (int v = 0; v < nv; ++v) {
            const int64_t vid = __ldg(S.cells + c * nv + v);
            for (int k = 0; k < 3; ++k) xv[v * 3 + k] = (k < d) ? __ldg(S.vertices + vid * d + k) : 0.0;
        }
        CellGeom g;
        const int st = box_point_geometry(xv, nv, S.dpsi, n_q, q, d, g);
        stat |= st;
        const float w = wts_smem ? wts[q] : (float)__ldg(weights + q);
        const float wk = f64_to_f32_rne(__ldg(kb + (int64_t)r * n_q + q), nonfinite) * w;
        float *row = wb + (int64_t)r * slots * ldw;
        float ms = 0.f;
        for (int j = 0; j < np; ++j) {
            const float v = st ? 0.f : wk * (float)g.G[j];
            row[j * ldw + q] = v;
            ms = fmaxf(ms, fabsf(v));
        }
        const float vm = st ? 0.f : wk * (float)g.absdet;
        row[np * ldw + q] = vm;
        if (need_max) {
            atomicMax(&rowmax[r], __float_as_int(ms));
            atomicMax(&rowmax2[r], __float_as_int(fabsf(vm)));
        }
    }
    // zero padding of every slot past n_q
    for (int i = tid; i < nvalid * slots * (ldw - n_q); i += F_THREADS) {
        const int pad = ldw - n_q;
        const int r = i / (slots * pad), rem = i - r * slots * pad;
        wb[((int64_t)r * slots + rem / pad) * ldw + n_q + rem % pad] = 0.f;
    }
    if (stat) atomicOr(&flags, stat);
    if (nonfinite) atomicOr(&flags, ST_NONFINITE);
    __syncthreads();
    if (tid < nvalid) {
        const int64_t c = c0 + tid;
        float rec[CELLF];
#pragma unroll
        for (int i = 0; i < CELLF; ++i) rec[i] = 0.f;
        for (int f = 0; f < MAX_FORMS; ++f) {
            if (!(S.form_mask & (1 << f))) continue;
            const float cmax = __int_as_float(f == 0 ? rowmax[tid] : rowmax2[tid]);
            int e_c = 0;
            if (need_max && cmax > 0.f && isfinite(cmax)) {
                int e;
                frexpf(cmax, &e);
                e_c = a.target_exp - e;
            }
            const float scale = ldexpf(1.f, e_c);
            rec[CELLF_UNSCALE + f] = ldexpf(S.op[f].p_inv_scale, -e_c);
            if (f == 0) {
#pragma unroll
                for (int j = 0; j < 6; ++j) rec[CELLF_G + j] = scale;
            } else {
                rec[CELLF_DET] = scale;
            }
        }
        float4 *dst = reinterpret_cast<float4 *>(S.cellf + c * CELLF);
#pragma unroll
        for (int i = 0; i < CELLF / 4; ++i)
            dst[i] = make_float4(rec[4 * i], rec[4 * i + 1], rec[4 * i + 2], rec[4 * i + 3]);
    }
    __syncthreads();
    if (tid == 0 && flags) atomicOr(a.status, flags);
}

}  // namespace

int launch_factor(const TcArgs &a, cudaStream_t s) {
    if (a.n_tiles <= 0) return 0;
    const bool g64 = a.prec == FE_PREC_TF32X3;
    const unsigned grid = (unsigned)(a.n_tiles * (TC_M / F_CELLS));
    if (!a.segs && a.seg0.win_slots > 1) {
        factor_box_kernel<<<grid, F_THREADS, 0, s>>>(a);
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? 1 : -(int)e;
    }
    if (a.segs) {
        if (g64) factor_kernel<true, true><<<grid, F_THREADS, 0, s>>>(a);
        else factor_kernel<true, false><<<grid, F_THREADS, 0, s>>>(a);
    } else {
        if (g64) factor_kernel<false, true><<<grid, F_THREADS, 0, s>>>(a);
        else factor_kernel<false, false><<<grid, F_THREADS, 0, s>>>(a);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

}  // namespace fe
