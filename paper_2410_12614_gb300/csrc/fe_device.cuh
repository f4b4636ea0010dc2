// Device helpers: affine simplex geometry in FP64 and thin inline-PTX
// wrappers for mbarriers, bulk copies and the tcgen05 tensor-core
// instructions of sm_103a.
#pragma once

#include <cstdint>

#include "fe_internal.h"
#include "fe_wait.h"

namespace fe {

// --------------------------------------------------------------------------
// Geometry (Sec. 4.2): J = [x1 - x0, ..., xd - x0], det J, and the Poisson
// geometry tensor G = |det J| J^{-1} J^{-T} (Sec. 3.1).  Computed from the
// cofactor matrix C of J: J^{-1} = C^T / det, so G = C^T C / |det J|.
// Returns the status bits (0 if the cell is valid).
// --------------------------------------------------------------------------
struct CellGeom {
    double absdet;
    double det;
    double C[9];   // cofactor matrix, row-major d x d
    double G[6];   // symmetric pairs (0,0),(0,1),(0,2),(1,1),(1,2),(2,2) (d=3) or (0,0),(0,1),(1,1)
};

// The d+1 vertex coordinates of cell c (unused entries zero).
__device__ __forceinline__ void cell_vertices(const double *__restrict__ vertices, const int32_t *__restrict__ cells,
                                              int64_t c, int d, double (&x)[4][3]) {
    const int nv = d + 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t v = (k < nv) ? __ldg(cells + c * nv + k) : 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) x[k][i] = (k < nv && i < d) ? __ldg(vertices + v * d + i) : 0.0;
    }
}

// Cofactor matrix and det J in FP64 from J; returns the status bits.
__device__ __forceinline__ int cofactors_of(const double (&J)[3][3], int d, CellGeom &g) {
    if (d == 3) {
        g.C[0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        g.C[1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        g.C[2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        g.C[3] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        g.C[4] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        g.C[5] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        g.C[6] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        g.C[7] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        g.C[8] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        g.det = J[0][0] * g.C[0] + J[0][1] * g.C[1] + J[0][2] * g.C[2];
    } else {
        g.C[0] = J[1][1];
        g.C[1] = -J[1][0];
        g.C[2] = -J[0][1];
        g.C[3] = J[0][0];
        g.det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    }
    g.absdet = fabs(g.det);
    int st = 0;
    if (!isfinite(g.det)) st |= ST_NONFINITE;
    else if (g.det == 0.0) st |= ST_DEGENERATE;
    return st;
}

// J = [x1 - x0, ..., xd - x0] of an affine simplex, its cofactors and det J.
__device__ __forceinline__ int cell_cofactors_x(const double (&x)[4][3], int d, CellGeom &g) {
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (i < d && j < d) J[i][j] = x[j + 1][i] - x[0][i];
    return cofactors_of(J, d, g);
}

// Boxed cells: J at one quadrature point of the multilinear map,
// J_ij = sum_v x_{v,i} dpsi[j][v][q] (dpsi: the Q1 derivative table
// [d][nv][n_q] at the rule's points), then its cofactors, det J and
// G = C^T C / |det J|, all in FP64.  Returns the status bits.
__device__ __forceinline__ int box_point_geometry(const double *__restrict__ xv, int nv, const double *__restrict__ dpsi,
                                                  int n_q, int q, int d, CellGeom &g) {
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int j = 0; j < d; ++j)
        for (int v = 0; v < nv; ++v) {
            const double dp = __ldg(dpsi + ((size_t)j * nv + v) * n_q + q);
            for (int i = 0; i < d; ++i) J[i][j] = fma(xv[v * 3 + i], dp, J[i][j]);
        }
    const int st = cofactors_of(J, d, g);
    const double inv = (st == 0) ? 1.0 / g.absdet : 0.0;
    int k = 0;
    for (int s2 = 0; s2 < d; ++s2)
        for (int t = s2; t < d; ++t) {
            double acc = 0.0;
            for (int r = 0; r < d; ++r) acc = fma(g.C[r * d + s2], g.C[r * d + t], acc);
            g.G[k++] = acc * inv;
        }
    for (; k < 6; ++k) g.G[k] = 0.0;
    return st;
}

__device__ __forceinline__ int cell_cofactors(const double *__restrict__ vertices, const int32_t *__restrict__ cells,
                                              int64_t c, int d, CellGeom &g) {
    double x[4][3];
    cell_vertices(vertices, cells, c, d, x);
    return cell_cofactors_x(x, d, g);
}

__device__ __forceinline__ int cell_geometry_x(const double (&x)[4][3], int d, CellGeom &g) {
    const int st = cell_cofactors_x(x, d, g);
    const double inv = (st == 0) ? 1.0 / g.absdet : 0.0;
    if (d == 3) {
        int j = 0;
#pragma unroll
        for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int t = s; t < 3; ++t) {
                g.G[j++] = (g.C[0 * 3 + s] * g.C[0 * 3 + t] + g.C[1 * 3 + s] * g.C[1 * 3 + t] +
                            g.C[2 * 3 + s] * g.C[2 * 3 + t]) * inv;
            }
    } else {
        g.G[0] = (g.C[0] * g.C[0] + g.C[2] * g.C[2]) * inv;
        g.G[1] = (g.C[0] * g.C[1] + g.C[2] * g.C[3]) * inv;
        g.G[2] = (g.C[1] * g.C[1] + g.C[3] * g.C[3]) * inv;
        g.G[3] = g.G[4] = g.G[5] = 0.0;
    }
    return st;
}

__device__ __forceinline__ int cell_geometry(const double *__restrict__ vertices, const int32_t *__restrict__ cells,
                                             int64_t c, int d, CellGeom &g) {
    double x[4][3];
    cell_vertices(vertices, cells, c, d, x);
    return cell_geometry_x(x, d, g);
}

// FP64 -> FP32 with round-to-nearest-even (IEEE 754), entirely on the
// integer units so that the per-quadrature-point path never touches the FP64
// pipe: the exponent is rebiased in place and the 29 dropped mantissa bits are
// rounded half to even (a carry into the exponent gives the correctly rounded
// power of two, and infinity past the largest finite value).  Magnitudes below
// FP32's smallest normal number (2^-126) are flushed to a signed zero;
// non-finite inputs set the flag and give infinity or NaN.
__device__ __forceinline__ float f64_to_f32_rne(double x, int &nonfinite) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned e = static_cast<unsigned>(u >> 52) & 0x7FFu;
    const unsigned sign = static_cast<unsigned>(u >> 63) << 31;
    const unsigned long long mag = (u & 0x7FFFFFFFFFFFFFFFull) - (static_cast<unsigned long long>(1023 - 127) << 52);
    const unsigned long long r = mag + 0x0FFFFFFFull + ((mag >> 29) & 1ull);
    unsigned bits = static_cast<unsigned>(r >> 29);
    bits = (e < 1023u - 126u) ? 0u : bits;
    bits = (e > 1023u + 127u) ? 0x7F800000u : bits;
    if (e == 0x7FFu) {
        nonfinite = 1;
        bits = (u & 0xFFFFFFFFFFFFFull) ? 0x7FC00000u : 0x7F800000u;
    }
    return __uint_as_float(bits | sign);
}

// G = |det J| J^-1 J^-T = C^T C / |det J| (upper triangle: G00 G01 G02 G11
// G12 G22; d = 2: G00 G01 G11) and |det J| in FP32, formed from the FP64
// cofactors and determinant rounded once each.  A cell gets G computed in
// FP64 and rounded once instead when its cofactors or determinant leave
// FP32's normal range, or when an off-diagonal entry cancels: sum_r |C_rs C_rt|
// above kG32Cancel |G_st| |det J| (a sheared or needle-shaped cell; an exact
// zero counts).  The FP32 G therefore carries a relative error of at most
// about (4 + 2 kG32Cancel) 2^-24 per entry.  Returns the geometry status; on a
// nonzero status g6 and adet are left as they were.
constexpr float kG32Cancel = 16.f;
__device__ __forceinline__ int cell_g32_tagged(const double *__restrict__ vertices, const int32_t *__restrict__ cells,
                                               int64_t c, int d, float (&g6)[6], float &adet, int &used_fp64) {
    CellGeom geo;
    const int st = cell_cofactors(vertices, cells, c, d, geo);
    if (st) return st;
    int nf = 0;
    float C[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) C[i] = f64_to_f32_rne(geo.C[i], nf);
    adet = f64_to_f32_rne(geo.absdet, nf);
    const float inv = 1.0f / adet;
    bool cancel = false;
    if (d == 3) {
        int j = 0;
#pragma unroll
        for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int u = s; u < 3; ++u) {
                const float sum = fmaf(C[s], C[u], fmaf(C[3 + s], C[3 + u], C[6 + s] * C[6 + u]));
                if (u != s) {
                    const float mag = fmaf(fabsf(C[s]), fabsf(C[u]),
                                           fmaf(fabsf(C[3 + s]), fabsf(C[3 + u]), fabsf(C[6 + s] * C[6 + u])));
                    cancel = cancel || !(mag <= kG32Cancel * fabsf(sum));
                }
                g6[j++] = sum * inv;
            }
    } else {
        g6[0] = fmaf(C[0], C[0], C[2] * C[2]) * inv;
        const float sum = fmaf(C[0], C[1], C[2] * C[3]);
        const float mag = fmaf(fabsf(C[0]), fabsf(C[1]), fabsf(C[2] * C[3]));
        cancel = !(mag <= kG32Cancel * fabsf(sum));
        g6[1] = sum * inv;
        g6[2] = fmaf(C[1], C[1], C[3] * C[3]) * inv;
    }
    bool fin = nf == 0 && adet > 0.f && isfinite(inv) && !cancel;
#pragma unroll
    for (int j = 0; j < 6; ++j) fin = fin && isfinite(g6[j]);
    used_fp64 = fin ? 0 : 1;
    if (!fin) {
        const double inv64 = 1.0 / geo.absdet;
        int j = 0;
        if (d == 3) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int u = s; u < 3; ++u)
                    g6[j++] = (float)((geo.C[s] * geo.C[u] + geo.C[3 + s] * geo.C[3 + u] + geo.C[6 + s] * geo.C[6 + u]) *
                                      inv64);
        } else {
            g6[0] = (float)((geo.C[0] * geo.C[0] + geo.C[2] * geo.C[2]) * inv64);
            g6[1] = (float)((geo.C[0] * geo.C[1] + geo.C[2] * geo.C[3]) * inv64);
            g6[2] = (float)((geo.C[1] * geo.C[1] + geo.C[3] * geo.C[3]) * inv64);
        }
        adet = (float)geo.absdet;
    }
    return 0;
}

__device__ __forceinline__ int cell_g32(const double *__restrict__ vertices, const int32_t *__restrict__ cells,
                                        int64_t c, int d, float (&g6)[6], float &adet) {
    int used;
    return cell_g32_tagged(vertices, cells, c, d, g6, adet, used);
}

// --------------------------------------------------------------------------
// PTX wrappers
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Asynchronous global -> shared copy of 4, 8 or 16 bytes (both addresses
// aligned to the size); cp_async_wait_all waits for the thread's copies.
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// 16-byte asynchronous copy that reads src_bytes (0 or 16) from src and fills
// the rest of the 16 bytes with zeros.
__device__ __forceinline__ void cp_async16_zfill(void *dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
// Groups of asynchronous copies: close the thread's current group; wait until
// at most N of its groups are still in flight.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// A probing thread is suspended until the phase completes or the suspend hint
// passes (fe_wait.h), so that waiting warps leave the issue slots to the
// working ones.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait on an mbarrier phase: false once the phase has made no
// progress for limit_ns nanoseconds since this wait began (wait_expired).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns) {
    const uint32_t hint = wait_suspend_hint(limit_ns);
    if (mbar_try_wait(bar, parity, hint)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity, hint)) {
        if (wait_expired(t0, global_ns(), limit_ns)) return false;
    }
    return true;
}

// The same, with one outcome for the whole warp (every lane waits; a lane that
// timed out makes the warp give up), for waits followed by warp-collective code.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, unsigned long long limit_ns) {
    return __all_sync(0xffffffffu, mbar_wait(bar, parity, limit_ns)) != 0;
}

// 1-D bulk copy global -> shared memory, completion counted on an mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Bulk prefetch of a contiguous global block into L2 (a hint; no completion).
// The address and size must be multiples of 16 bytes.
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// --- tcgen05 -----------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand in 128-byte swizzled
// rows, 8-row atoms of 1024 bytes stacked along M/N (stride 1024 bytes).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t desc = 0;
    desc |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    desc |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
    desc |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset
    desc |= (uint64_t)1 << 46;                      // descriptor version
    desc |= (uint64_t)2 << 61;                      // 128-byte swizzle
    return desc;
}

template <int KIND>  // 0: f16/bf16, 1: tf32, 2: f8f6f4
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else if constexpr (KIND == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive columns without waiting (tmem_wait_ld32 completes them).
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%33];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr), "r"(taddr + 16u));
}
// Wait for every outstanding TMEM load of this thread; r is named so that no
// use of the loaded registers is scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Two 32x32b.x16 loads (32 consecutive columns) followed by one wait.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    tmem_ld32_async(taddr, r);
    tmem_wait_ld32(r);
}

// --- conversions (round to nearest even) -----------------------------------
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ uint32_t pack_e4m3x2(float lo, float hi) {
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
    return r;
}
// FP32 -> TF32 (10 explicit mantissa bits), round to nearest even, kept in FP32 bits.
__device__ __forceinline__ uint32_t round_tf32(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u) return u;
    u += 0xFFFu + ((u >> 13) & 1u);
    return u & 0xFFFFE000u;
}

}  // namespace fe
