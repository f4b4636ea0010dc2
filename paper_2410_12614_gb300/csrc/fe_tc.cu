// Tensor-core element-matrix kernel (sm_103a, tcgen05).
//
// Algorithm 1 of the paper for a tile of 128 cells at once, written as one
// dense contraction per tile with the cells on the MMA M dimension:
//
//   A^c_{kl} = sum_{(s<=t), q} C^c_{(st,q)} P_{(st,q),(kl)}          (k <= l)
//
// where C^c_{(st,q)} = w_q kappa_cq G^c_st (Sec. 3.1, C_st = diag_q(w_q z(X_q)
// G_st)) is formed per cell from the FP64 geometry, and
// P_{(st,q),(kl)} = B_skq B_tlq + [s != t] B_tkq B_slq is the product of the
// tabulated reference derivatives (the triple products B_s C_st B_t^T of
// Sec. 3.1 folded over the symmetric pairs), precomputed in FP64 at plan time
// and rounded once to the storage format.  For the mass form there is one
// pair, G = |det J| and B = phi.  The storage precision u_s applies to C and
// P; products and accumulation are FP32 in tensor memory (u_q): the mixed
// strategy of Sec. 4.5.  Only the upper triangle k <= l is computed; the
// epilogue mirrors it.
//
// CTA: 256 threads, two per cell.  K is streamed in 128-byte chunks through a
// 2-stage ring.  A chunk holds one window of consecutive quadrature points of
// one (s,t) pair, so a thread converts its cell's coefficient window
// w_q = w_q kappa_cq to FP32 once and reuses it for every pair.  The shared
// operand P arrives by a 1-D bulk copy of a pre-swizzled image (no
// multicast); thread 0 issues tcgen05.mma into an FP32 TMEM accumulator of
// N <= 256 columns and commits to mbarriers.  The epilogue mirrors the upper
// triangle into a conflict-free shared-memory staging area and writes whole
// element matrices with coalesced 16-byte stores.  Every wait is bounded
// (globaltimer); a timeout sets the status word and the CTA exits after
// releasing its tensor memory.
#include <cstdio>

#include "fe_device.cuh"

namespace fe {

namespace {

constexpr int TC_CELLS_PER_HALF = 16;  // epilogue staging granularity per lane group

struct TcSmem {
    uint8_t *A;       // [TC_STAGES][128 rows][128 B]
    uint8_t *B;       // [TC_STAGES][NPmax rows][128 B]
    float *stage;     // epilogue staging (aliases A and B)
    float *geo;       // [128][8]: G pairs, |det J|, spare
    float *wmax;      // [2][128]
    float *omega;     // [n_q] quadrature weights in FP32
    int32_t *symkl;   // [n_sym_pad] k | l << 16
    uint64_t *full;   // [TC_STAGES]
    uint64_t *empty;  // [TC_STAGES]
    uint64_t *acc;
    uint32_t *tmem_holder;
    int *flags;       // [0] abort, [1] status bits
};

__host__ __device__ inline int np_max(const TcArgs &a) {
    int m = 16;
    for (int f = 0; f < MAX_FORMS; ++f)
        if (a.form_mask & (1 << f)) m = (a.op[f].NP > m) ? a.op[f].NP : m;
    return m;
}

// the shared-memory copy of the sym table is used by the staged epilogue only
__host__ __device__ inline int sym_pad(const TcArgs &a) {
    if (!a.staged) return 0;
    int n = a.n_phi * (a.n_phi + 1) / 2;
    return (n + 3) & ~3;
}

__host__ __device__ inline uint32_t tmem_cols_for(int np) {
    uint32_t c = 32;
    while (c < (uint32_t)np) c <<= 1;
    return c;
}

__host__ __device__ inline int stage_pitch(const TcArgs &a) { return (a.n_phi * a.n_phi) | 1; }

__host__ __device__ inline size_t union_bytes(const TcArgs &a) {
    size_t ring = (size_t)TC_STAGES * TC_M * TC_CHUNK_BYTES + (size_t)TC_STAGES * np_max(a) * TC_CHUNK_BYTES;
    size_t stg = a.staged ? (size_t)4 * TC_CELLS_PER_HALF * stage_pitch(a) * sizeof(float) : 0;
    size_t u = ring > stg ? ring : stg;
    return (u + 1023) & ~size_t(1023);
}

__device__ inline TcSmem carve(uint8_t *raw, const TcArgs &a) {
    uintptr_t p = (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023);
    TcSmem s;
    s.A = reinterpret_cast<uint8_t *>(p);
    s.B = s.A + TC_STAGES * TC_M * TC_CHUNK_BYTES;
    s.stage = reinterpret_cast<float *>(s.A);
    uint8_t *q = s.A + union_bytes(a);
    s.geo = reinterpret_cast<float *>(q);
    s.wmax = s.geo + TC_M * 8;
    s.omega = s.wmax + 2 * TC_M;
    s.symkl = reinterpret_cast<int32_t *>(s.omega + ((a.n_q + 3) & ~3));
    q = reinterpret_cast<uint8_t *>(s.symkl + sym_pad(a));
    q = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(q) + 7) & ~uintptr_t(7));
    s.full = reinterpret_cast<uint64_t *>(q);
    s.empty = s.full + TC_STAGES;
    s.acc = s.empty + TC_STAGES;
    s.tmem_holder = reinterpret_cast<uint32_t *>(s.acc + 1);
    s.flags = reinterpret_cast<int *>(s.tmem_holder + 2);
    return s;
}

// FP64 -> FP32 with round-to-nearest-even (IEEE 754) done on the integer
// units for results in the normal FP32 range; other inputs (zero,
// subnormal, out of range, non-finite) take the hardware conversion.  The
// exponent is rebiased in place and the 29 dropped mantissa bits are rounded
// half to even.  Keeps the per-quadrature-point path off the FP64 pipe.
__device__ __forceinline__ float f64_to_f32_rne(double x, int &nonfinite) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned e = static_cast<unsigned>(u >> 52) & 0x7FFu;
    if (e >= 1023u - 126u && e <= 1023u + 126u) {
        const unsigned long long mag = (u & 0x7FFFFFFFFFFFFFFFull) - (static_cast<unsigned long long>(1023 - 127) << 52);
        const unsigned long long r = mag + 0x0FFFFFFFull + ((mag >> 29) & 1ull);
        return __uint_as_float(static_cast<unsigned>(r >> 29) | (static_cast<unsigned>(u >> 63) << 31));
    }
    if (e == 0x7FFu) nonfinite = 1;
    return static_cast<float>(x);
}

template <int EB>
struct Conv;
template <>
struct Conv<2> {
    // 8 values -> 16 bytes
    template <int PREC>
    __device__ static uint4 pack(const float *v) {
        uint4 r;
        if constexpr (PREC == FE_PREC_BF16) {
            r.x = pack_bf16x2(v[0], v[1]);
            r.y = pack_bf16x2(v[2], v[3]);
            r.z = pack_bf16x2(v[4], v[5]);
            r.w = pack_bf16x2(v[6], v[7]);
        } else {
            r.x = pack_f16x2(v[0], v[1]);
            r.y = pack_f16x2(v[2], v[3]);
            r.z = pack_f16x2(v[4], v[5]);
            r.w = pack_f16x2(v[6], v[7]);
        }
        return r;
    }
};

template <int PREC>
__global__ void __launch_bounds__(TC_THREADS, 2) tc_element_kernel(const __grid_constant__ TcArgs a) {
    constexpr int EB = (PREC == FE_PREC_E4M3) ? 1 : ((PREC == FE_PREC_TF32 || PREC == FE_PREC_TF32X3) ? 4 : 2);
    constexpr int KIND = (PREC == FE_PREC_E4M3) ? 2 : ((EB == 4) ? 1 : 0);
    constexpr int KCE = TC_CHUNK_BYTES / EB;  // quadrature points per chunk
    constexpr int HW = KCE / 2;               // points per thread (half window)
    constexpr int EP = 16 / EB;               // elements per 16-byte piece

    // a CTA that starts after another one gave up does no work at all
    if (*reinterpret_cast<volatile int *>(a.status) & ST_TIMEOUT) return;

    extern __shared__ uint8_t smem_raw[];
    TcSmem sm = carve(smem_raw, a);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int cl = tid & (TC_M - 1), half = tid >> 7;
    const int64_t cell0 = (int64_t)blockIdx.x * TC_M;
    const int64_t cell = cell0 + cl;
    const bool valid = cell < a.n_cells;
    const int NPm = np_max(a);
    const uint32_t ncols = tmem_cols_for(NPm);
    const int nph = a.n_phi, nph2 = nph * nph;
    const int n_sym = nph * (nph + 1) / 2;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        mbar_init(sm.acc, 1);
        sm.flags[0] = 0;
        sm.flags[1] = 0;
        fence_mbar_init();
    }
    for (int i = tid; i < a.n_q; i += TC_THREADS) sm.omega[i] = (float)__ldg(a.weights + i);
    if (a.staged)
        for (int i = tid; i < n_sym; i += TC_THREADS) sm.symkl[i] = __ldg(a.sym_kl + i);
    if (warp == 0) {
        tmem_alloc(sm.tmem_holder, ncols);
        tmem_relinquish();
    }
    // ---- geometry in FP64, one cell per thread of the first half ----
    if (half == 0) {
        float *g = sm.geo + cl * 8;
        int st = 0;
        if (valid) {
            CellGeom geo;
            st = cell_geometry(a.vertices, a.cells, cell, a.d, geo);
            for (int j = 0; j < 6; ++j) g[j] = st ? 0.f : (float)geo.G[j];
            g[6] = st ? 0.f : (float)geo.absdet;
        } else {
            for (int j = 0; j < 7; ++j) g[j] = 0.f;
        }
        g[7] = __int_as_float(st);
        if (st) atomicOr(&sm.flags[1], st);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_holder;
    const unsigned long long deadline = global_ns() + a.timeout_ns;
    const double *krow = a.kappa + (valid ? cell : 0) * (int64_t)a.n_q;
    const bool ok = valid && (__float_as_int(sm.geo[cl * 8 + 7]) == 0);
    int nonfinite = 0;

    // per-cell scaling (formats with a narrow exponent range): the largest |w_q kappa_cq|
    float wmax = 0.f;
    if (a.target_exp > 1) {
        if (ok)
            for (int q = half; q < a.n_q; q += 2)
                wmax = fmaxf(wmax, fabsf(f64_to_f32_rne(__ldg(krow + q), nonfinite) * sm.omega[q]));
        sm.wmax[half * TC_M + cl] = wmax;
    }
    __syncthreads();
    if (a.target_exp > 1) wmax = fmaxf(sm.wmax[cl], sm.wmax[TC_M + cl]);

    int chunk = 0, pass_count = 0;
    bool aborted = false;
    float win[HW];
#pragma unroll 1
    for (int f = 0; f < MAX_FORMS && !aborted; ++f) {
        if (!(a.form_mask & (1 << f))) continue;
        const TcOperand &op = a.op[f];
        float g[6];
        float gmax = 0.f;
        if (f == 0) {
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                g[j] = sm.geo[cl * 8 + j];
                gmax = fmaxf(gmax, fabsf(g[j]));
            }
        } else {
            g[0] = sm.geo[cl * 8 + 6];
#pragma unroll
            for (int j = 1; j < 6; ++j) g[j] = 0.f;
            gmax = g[0];
        }
        int e_c = 0;
        if (a.target_exp > 1 && ok) {
            const float cmax = wmax * gmax;
            if (cmax > 0.f && isfinite(cmax)) {
                int e;
                frexpf(cmax, &e);
                e_c = a.target_exp - e;
            }
        }
        const float scale = ldexpf(1.f, e_c);
        const float unscale = ldexpf(op.p_inv_scale, -e_c);
        const uint32_t idesc = a.idesc | ((uint32_t)(op.NP >> 3) << 17);
        const uint32_t bbytes = (uint32_t)op.NP * TC_CHUNK_BYTES;
        const int per_qw = op.n_pairs * op.n_blk;

#pragma unroll 1
        for (int n = 0; n < op.n_pass && !aborted; ++n) {
            int qw_loaded = -1;
#pragma unroll 1
            for (int ch = 0; ch < op.n_kchunks; ++ch) {
                const int s = chunk % TC_STAGES;
                const int use = chunk / TC_STAGES;
                if (chunk >= TC_STAGES) {
                    if (!mbar_wait(&sm.empty[s], (use - 1) & 1, deadline)) sm.flags[0] = 1;
                }
                uint8_t *stA = sm.A + s * (TC_M * TC_CHUNK_BYTES);
                uint8_t *stB = sm.B + (size_t)s * NPm * TC_CHUNK_BYTES;
                if (tid == 0 && !sm.flags[0]) {
                    fence_proxy_async();
                    mbar_arrive_expect_tx(&sm.full[s], bbytes);
                    bulk_g2s(stB, op.img + ((size_t)n * op.n_kchunks + ch) * bbytes, bbytes, &sm.full[s]);
                }
                // ---- operand C: this thread's half of the cell's 128-byte row ----
                const int qw = ch / per_qw;
                const int j = (ch / op.n_blk) % op.n_pairs;
                const int blk = ch % op.n_blk;
                if (qw != qw_loaded) {
                    qw_loaded = qw;
#pragma unroll
                    for (int i = 0; i < HW; ++i) {
                        const int q = qw * KCE + half * HW + i;
                        win[i] = (ok && q < a.n_q) ? f64_to_f32_rne(__ldg(krow + q), nonfinite) * sm.omega[q] : 0.f;
                    }
                }
                float gj = 0.f;
#pragma unroll
                for (int jj = 0; jj < 6; ++jj)
                    if (jj == j) gj = g[jj];
                gj *= scale;
                uint8_t *rowp = stA + (cl >> 3) * 1024 + (cl & 7) * 128;
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
                    const int piece = half * 4 + pp;
                    uint4 val;
                    float v[EP];
#pragma unroll
                    for (int i = 0; i < EP; ++i) v[i] = win[pp * EP + i] * gj;
                    if constexpr (EB == 2) {
                        val = Conv<2>::pack<PREC>(v);
                    } else if constexpr (EB == 4) {
                        uint32_t w4[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            uint32_t h = round_tf32(v[i]);
                            if (PREC == FE_PREC_TF32X3 && blk == 2) h = round_tf32(v[i] - __uint_as_float(h));
                            w4[i] = h;
                        }
                        val = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                    } else {
                        uint32_t w4[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            w4[i] = pack_e4m3x2(v[4 * i], v[4 * i + 1]) | (pack_e4m3x2(v[4 * i + 2], v[4 * i + 3]) << 16);
                        val = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                    }
                    *reinterpret_cast<uint4 *>(rowp + ((piece ^ (cl & 7)) << 4)) = val;
                }
                fence_proxy_async();
                __syncthreads();
                if (sm.flags[0]) {
                    aborted = true;
                    break;
                }
                if (tid == 0) {
                    if (!mbar_wait(&sm.full[s], use & 1, deadline)) {
                        sm.flags[0] = 1;
                    } else {
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(stA), b0 = smem_u32(stB);
#pragma unroll
                        for (int ks = 0; ks < TC_CHUNK_BYTES / 32; ++ks) {
                            umma<KIND>(tmem, sdesc_sw128(a0 + 32 * ks), sdesc_sw128(b0 + 32 * ks), idesc,
                                       (ch | ks) != 0 ? 1u : 0u);
                        }
                        umma_commit(&sm.empty[s]);
                        if (ch == op.n_kchunks - 1) umma_commit(sm.acc);
                    }
                }
                ++chunk;
            }
            if (aborted) break;
            // ---- epilogue of pass n ----
            const bool acc_ok = mbar_wait(sm.acc, pass_count & 1, deadline);
            ++pass_count;
            if (!acc_ok) sm.flags[0] = 1;
            __syncthreads();
            if (sm.flags[0]) {
                aborted = true;
                break;
            }
            tc_fence_after();
            float *out = a.out[f];
            const int lg = warp & 3;       // TMEM lane group = 32 cells
            const int cpar = warp >> 2;    // column-chunk parity handled by this warp
            const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16);
            if (a.staged) {
                const int pitch = stage_pitch(a);
                float *stg = sm.stage + lg * TC_CELLS_PER_HALF * pitch;
#pragma unroll 1
                for (int h2 = 0; h2 < 2; ++h2) {
                    const bool active = (lane >> 4) == h2;
                    float *mine = stg + (lane & 15) * pitch;
#pragma unroll 1
                    for (int c0 = 16 * cpar; c0 < op.NP; c0 += 32) {
                        uint32_t r[16];
                        tmem_ld16(tbase + (uint32_t)c0, r);
                        if (active) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const int col = c0 + i;
                                if (col < op.n_cols) {
                                    const int32_t kl = sm.symkl[col];
                                    const int k = kl & 0xFFFF, l = kl >> 16;
                                    const float v = __uint_as_float(r[i]) * unscale;
                                    mine[k * nph + l] = v;
                                    mine[l * nph + k] = v;
                                }
                            }
                        }
                    }
                    named_bar_sync(1 + lg, 64);
                    // coalesced copy of 16 consecutive cells (contiguous in global memory)
                    const int64_t cfirst = cell0 + lg * 32 + h2 * TC_CELLS_PER_HALF;
                    const int64_t rem_cells = a.n_cells - cfirst;
                    const int ncp = rem_cells < TC_CELLS_PER_HALF ? (int)rem_cells : TC_CELLS_PER_HALF;
                    const int t64 = cpar * 32 + lane;
                    if (ncp > 0 && out) {
                        float *dst = out + cfirst * (int64_t)nph2;
                        if ((nph2 & 3) == 0) {
                            const int n4 = nph2 >> 2;
                            for (int i = t64; i < ncp * n4; i += 64) {
                                const int cc = i / n4, kl = (i - cc * n4) * 4;
                                const float *src = stg + cc * pitch + kl;
                                reinterpret_cast<float4 *>(dst)[i] = make_float4(src[0], src[1], src[2], src[3]);
                            }
                        } else {
                            for (int i = t64; i < ncp * nph2; i += 64) {
                                const int cc = i / nph2, kl = i - cc * nph2;
                                dst[i] = stg[cc * pitch + kl];
                            }
                        }
                    }
                    named_bar_sync(1 + lg, 64);
                }
            } else if (out) {
                // direct mirrored stores (multi-pass shapes)
#pragma unroll 1
                for (int c0 = 16 * cpar; c0 < op.NP; c0 += 32) {
                    uint32_t r[16];
                    tmem_ld16(tbase + (uint32_t)c0, r);
                    const int64_t mycell = cell0 + lg * 32 + lane;
                    if (mycell < a.n_cells) {
                        float *dst = out + mycell * (int64_t)nph2;
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int col = n * op.NP + c0 + i;
                            if (col < op.n_cols) {
                                const int32_t kl = __ldg(a.sym_kl + col);
                                const int k = kl & 0xFFFF, l = kl >> 16;
                                const float v = __uint_as_float(r[i]) * unscale;
                                dst[k * nph + l] = v;
                                dst[l * nph + k] = v;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncthreads();
        }
    }
    if (nonfinite) atomicOr(&sm.flags[1], ST_NONFINITE);
    if (aborted || sm.flags[0]) {
        if (tid == 0) atomicOr(&sm.flags[1], ST_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && sm.flags[1]) atomicOr(a.status, sm.flags[1]);
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace

size_t tc_smem_bytes(const TcArgs &a) {
    size_t b = 1024;  // alignment slack
    b += union_bytes(a);
    b += (size_t)TC_M * 8 * sizeof(float) + 2 * TC_M * sizeof(float);
    b += (size_t)((a.n_q + 3) & ~3) * sizeof(float);
    b += (size_t)sym_pad(a) * sizeof(int32_t) + 8;
    b += (2 * TC_STAGES + 1) * sizeof(uint64_t) + 8 + 16;
    return b;
}

template <int PREC>
static int launch_prec(const TcArgs &a, size_t smem, cudaStream_t s, int64_t grid) {
    cudaError_t e = cudaFuncSetAttribute(tc_element_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -(int)e;
    tc_element_kernel<PREC><<<(unsigned)grid, TC_THREADS, smem, s>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

int launch_tc_elements(const TcArgs &a, size_t smem, cudaStream_t s) {
    if (a.n_cells <= 0) return 0;
    const int64_t grid = (a.n_cells + TC_M - 1) / TC_M;
    switch (a.prec) {
        case FE_PREC_BF16: return launch_prec<FE_PREC_BF16>(a, smem, s, grid);
        case FE_PREC_FP16: return launch_prec<FE_PREC_FP16>(a, smem, s, grid);
        case FE_PREC_TF32: return launch_prec<FE_PREC_TF32>(a, smem, s, grid);
        case FE_PREC_TF32X3: return launch_prec<FE_PREC_TF32X3>(a, smem, s, grid);
        case FE_PREC_E4M3: return launch_prec<FE_PREC_E4M3>(a, smem, s, grid);
        default: return -(int)cudaErrorInvalidValue;
    }
}

}  // namespace fe
