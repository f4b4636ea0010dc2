// Tensor-core element-matrix kernel (sm_103a, tcgen05).
//
// Algorithm 1 of the paper for a tile of 128 cells at once, written as one
// dense contraction per tile with the cells on the MMA M dimension:
//
//   A^c_{kl} = sum_{q, (s<=t)} C^c_{(q,st)} P_{(q,st),(kl)}        (k <= l)
//
// where C^c_{(q,st)} = w_q kappa_cq G^c_st (Sec. 3.1, C_st = diag_q(w_q z(X_q)
// G_st)) is formed per cell on the CUDA cores from FP64 geometry, and
// P_{(q,st),(kl)} = B_skq B_tlq + [s != t] B_tkq B_slq is the product of the
// tabulated reference derivatives (the triple products B_s C_st B_t^T of
// Sec. 3.1 folded over the symmetric pairs), precomputed in FP64 at plan time
// and rounded once to the storage format.  For the mass form the pairs
// reduce to one and B = phi.  Storage precision u_s applies to C and P, the
// products and their accumulation are FP32 in tensor memory (u_q), exactly
// the mixed strategy of Sec. 4.5.  Only the upper triangle k <= l is
// computed; the epilogue mirrors it.
//
// Per CTA: 128 threads, one cell per thread for geometry, operand build and
// epilogue.  K is streamed in 128-byte chunks through a 2-stage ring: the
// shared operand P arrives by a bulk copy (pre-swizzled image in global
// memory, one copy per chunk, no multicast), the per-cell operand C is
// written by the threads; thread 0 issues tcgen05.mma into an FP32 TMEM
// accumulator of N <= 256 columns and commits to mbarriers.  Every wait is
// bounded (globaltimer); a timeout sets the status word and the CTA exits
// after releasing its tensor memory.
#include <cstdio>

#include "fe_device.cuh"

namespace fe {

namespace {

struct TcSmem {
    uint8_t *A;       // [TC_STAGES][128 rows][128 B]
    uint8_t *B;       // [TC_STAGES][NPmax rows][128 B]
    uint64_t *full;   // [TC_STAGES]
    uint64_t *empty;  // [TC_STAGES]
    uint64_t *acc;
    uint32_t *tmem_holder;
    int *abort_flag;
    int16_t *f2s;     // [n_phi^2]
};

__host__ __device__ inline int np_max(const TcArgs &a) {
    int m = 16;
    for (int f = 0; f < MAX_FORMS; ++f)
        if (a.form_mask & (1 << f)) m = (a.op[f].NP > m) ? a.op[f].NP : m;
    return m;
}

__host__ __device__ inline uint32_t tmem_cols_for(int np) {
    uint32_t c = 32;
    while (c < (uint32_t)np) c <<= 1;
    return c;
}

__device__ inline TcSmem carve(uint8_t *raw, const TcArgs &a) {
    uintptr_t p = (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023);
    TcSmem s;
    s.A = reinterpret_cast<uint8_t *>(p);
    s.B = s.A + TC_STAGES * TC_M * TC_CHUNK_BYTES;
    uint8_t *q = s.B + (size_t)TC_STAGES * np_max(a) * TC_CHUNK_BYTES;
    s.full = reinterpret_cast<uint64_t *>(q);
    s.empty = s.full + TC_STAGES;
    s.acc = s.empty + TC_STAGES;
    s.tmem_holder = reinterpret_cast<uint32_t *>(s.acc + 1);
    s.abort_flag = reinterpret_cast<int *>(s.tmem_holder + 1);
    s.f2s = reinterpret_cast<int16_t *>(s.abort_flag + 2);
    return s;
}

// Per-cell operand value C at contraction index Kin of one form.
struct CellOperand {
    const double *kappa_row;  // kappa[c][*]
    const double *weights;
    float g[6];               // G pairs (stiffness) or |det J| in g[0] (mass)
    float scale;              // 2^e_c
    int n_pairs;
    int K_true;
};

__device__ __forceinline__ float operand_value(const CellOperand &o, int Kin, int &q_cached, float &w_cached) {
    if (Kin >= o.K_true) return 0.f;
    int q = Kin / o.n_pairs;
    int j = Kin - q * o.n_pairs;
    if (q != q_cached) {
        q_cached = q;
        w_cached = (float)(__ldg(o.weights + q) * __ldg(o.kappa_row + q));
    }
    return w_cached * o.g[j] * o.scale;
}

// Build this thread's row (one cell) of chunk kc of the A operand: 128 bytes,
// written as 8 swizzled 16-byte pieces.
__device__ __forceinline__ void build_row(uint8_t *stageA, int row, const TcArgs &a, const TcOperand &op,
                                          const CellOperand &o, int kc, bool valid) {
    const int eb = a.elem_bytes;
    const int KCE = TC_CHUNK_BYTES / eb;
    const int Kg0 = kc * KCE;
    const int blk = Kg0 / op.K_blk;
    const int Kin0 = Kg0 - blk * op.K_blk;
    const bool tail = (a.prec == FE_PREC_TF32X3) && (blk == 2);
    uint8_t *rowp = stageA + (row >> 3) * 1024 + (row & 7) * 128;
    int q_cached = -1;
    float w_cached = 0.f;
#pragma unroll 1
    for (int piece = 0; piece < 8; ++piece) {
        uint32_t w4[4];
        const int per = 16 / eb;  // elements per 16-byte piece
        const int K0 = Kin0 + piece * per;
        if (!valid) {
            w4[0] = w4[1] = w4[2] = w4[3] = 0u;
        } else if (eb == 2) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float v0 = operand_value(o, K0 + 2 * i, q_cached, w_cached);
                float v1 = operand_value(o, K0 + 2 * i + 1, q_cached, w_cached);
                w4[i] = (a.prec == FE_PREC_BF16) ? pack_bf16x2(v0, v1) : pack_f16x2(v0, v1);
            }
        } else if (eb == 4) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float v = operand_value(o, K0 + i, q_cached, w_cached);
                uint32_t h = round_tf32(v);
                if (tail) h = round_tf32(v - __uint_as_float(h));
                w4[i] = h;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float v0 = operand_value(o, K0 + 4 * i + 0, q_cached, w_cached);
                float v1 = operand_value(o, K0 + 4 * i + 1, q_cached, w_cached);
                float v2 = operand_value(o, K0 + 4 * i + 2, q_cached, w_cached);
                float v3 = operand_value(o, K0 + 4 * i + 3, q_cached, w_cached);
                w4[i] = pack_e4m3x2(v0, v1) | (pack_e4m3x2(v2, v3) << 16);
            }
        }
        uint4 val = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        *reinterpret_cast<uint4 *>(rowp + ((piece ^ (row & 7)) << 4)) = val;
    }
}

template <int KIND>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_element_kernel(const __grid_constant__ TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    TcSmem sm = carve(smem_raw, a);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t cell0 = (int64_t)blockIdx.x * TC_M;
    const int64_t cell = cell0 + tid;
    const bool valid = cell < a.n_cells;
    const int NPm = np_max(a);
    const uint32_t ncols = tmem_cols_for(NPm);
    const int n_phi2 = a.n_phi * a.n_phi;

    // a CTA that starts after another one gave up does no work at all
    if (*reinterpret_cast<volatile int *>(a.status) & ST_TIMEOUT) return;
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        mbar_init(sm.acc, 1);
        *sm.abort_flag = 0;
        fence_mbar_init();
    }
    if (a.staged)
        for (int i = tid; i < n_phi2; i += TC_THREADS) sm.f2s[i] = a.full2sym[i];
    if (warp == 0) {
        tmem_alloc(sm.tmem_holder, ncols);
        tmem_relinquish();
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_holder;
    const unsigned long long deadline = global_ns() + a.timeout_ns;

    // ---- geometry in FP64 (one cell per thread) ----
    CellGeom geo;
    int st = 0;
    if (valid) st = cell_geometry(a.vertices, a.cells, cell, a.d, geo);
    bool ok = valid && (st == 0);
    const double *krow = a.kappa + (valid ? cell : 0) * (int64_t)a.n_q;
    // per-cell scale: the largest |w_q kappa_cq| times the largest factor
    float wmax = 0.f;
    if (ok) {
        for (int q = 0; q < a.n_q; ++q) {
            double w = __ldg(a.weights + q) * __ldg(krow + q);
            if (!isfinite(w)) st |= ST_NONFINITE;
            wmax = fmaxf(wmax, fabsf((float)w));
        }
        ok = (st == 0);
    }
    if (st) atomicOr(a.status, st);

    int chunk = 0, pass_count = 0;
    bool aborted = false;
#pragma unroll 1
    for (int f = 0; f < MAX_FORMS && !aborted; ++f) {
        if (!(a.form_mask & (1 << f))) continue;
        const TcOperand &op = a.op[f];
        CellOperand o;
        o.kappa_row = krow;
        o.weights = a.weights;
        o.n_pairs = (f == 0) ? a.n_pairs : 1;
        o.K_true = a.n_q * o.n_pairs;
        float gmax = 0.f;
        if (f == 0) {
            for (int j = 0; j < 6; ++j) {
                o.g[j] = ok ? (float)geo.G[j] : 0.f;
                gmax = fmaxf(gmax, fabsf(o.g[j]));
            }
        } else {
            o.g[0] = ok ? (float)geo.absdet : 0.f;
            for (int j = 1; j < 6; ++j) o.g[j] = 0.f;
            gmax = o.g[0];
        }
        int e_c = 0;
        if (a.target_exp > 1 && ok) {
            float cmax = wmax * gmax;
            if (cmax > 0.f && isfinite(cmax)) {
                int e;
                frexpf(cmax, &e);
                e_c = a.target_exp - e;
            }
        }
        o.scale = ldexpf(1.f, e_c);
        const float unscale = ldexpf(op.p_inv_scale, -e_c);
        const uint32_t idesc = a.idesc | ((uint32_t)(op.NP >> 3) << 17);
        const uint32_t bbytes = (uint32_t)op.NP * TC_CHUNK_BYTES;

#pragma unroll 1
        for (int n = 0; n < op.n_pass && !aborted; ++n) {
#pragma unroll 1
            for (int kc = 0; kc < op.n_kchunks; ++kc) {
                const int s = chunk % TC_STAGES;
                const int use = chunk / TC_STAGES;
                if (chunk >= TC_STAGES) {
                    if (!mbar_wait(&sm.empty[s], (use - 1) & 1, deadline)) *sm.abort_flag = 1;
                }
                uint8_t *stA = sm.A + s * (TC_M * TC_CHUNK_BYTES);
                uint8_t *stB = sm.B + (size_t)s * NPm * TC_CHUNK_BYTES;
                if (tid == 0 && !*sm.abort_flag) {
                    fence_proxy_async();
                    mbar_arrive_expect_tx(&sm.full[s], bbytes);
                    bulk_g2s(stB, op.img + ((size_t)n * op.n_kchunks + kc) * bbytes, bbytes, &sm.full[s]);
                }
                build_row(stA, tid, a, op, o, kc, ok);
                fence_proxy_async();
                __syncthreads();
                if (*sm.abort_flag) {
                    aborted = true;
                    break;
                }
                if (tid == 0) {
                    if (!mbar_wait(&sm.full[s], use & 1, deadline)) {
                        *sm.abort_flag = 1;
                    } else {
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(stA), b0 = smem_u32(stB);
#pragma unroll
                        for (int ks = 0; ks < TC_CHUNK_BYTES / 32; ++ks) {
                            umma<KIND>(tmem, sdesc_sw128(a0 + 32 * ks), sdesc_sw128(b0 + 32 * ks), idesc,
                                       (kc | ks) != 0 ? 1u : 0u);
                        }
                        umma_commit(&sm.empty[s]);
                        if (kc == op.n_kchunks - 1) umma_commit(sm.acc);
                    }
                }
                ++chunk;
            }
            if (aborted) break;
            // ---- epilogue of pass n ----
            const bool acc_ok = mbar_wait(sm.acc, pass_count & 1, deadline);
            ++pass_count;
            if (!acc_ok) *sm.abort_flag = 1;
            __syncthreads();
            if (*sm.abort_flag) {
                aborted = true;
                break;
            }
            tc_fence_after();
            float *out = a.out[f];
            const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
            if (a.staged) {
                // stage 16 cells of this warp at a time (pitch NP+1 floats: conflict-free)
                const int pitch = op.NP + 1;
                float *stg = reinterpret_cast<float *>(sm.A) + warp * 16 * pitch;
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
#pragma unroll 1
                    for (int c0 = 0; c0 < op.NP; c0 += 16) {
                        uint32_t r[16];
                        tmem_ld16(tbase + (uint32_t)c0, r);
                        if ((lane >> 4) == h) {
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                stg[(lane & 15) * pitch + c0 + i] = __uint_as_float(r[i]) * unscale;
                        }
                    }
                    __syncwarp();
                    if (out) {
#pragma unroll 1
                        for (int cc = 0; cc < 16; ++cc) {
                            const int64_t cg = cell0 + warp * 32 + h * 16 + cc;
                            if (cg >= a.n_cells) break;
                            float *dst = out + cg * (int64_t)n_phi2;
                            const float *src = stg + cc * pitch;
                            for (int kl = lane; kl < n_phi2; kl += 32) dst[kl] = src[sm.f2s[kl]];
                        }
                    }
                    __syncwarp();
                }
            } else if (out) {
                // direct mirrored stores (multi-pass shapes)
#pragma unroll 1
                for (int c0 = 0; c0 < op.NP; c0 += 16) {
                    uint32_t r[16];
                    tmem_ld16(tbase + (uint32_t)c0, r);
                    if (valid) {
                        float *dst = out + cell * (int64_t)n_phi2;
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int col = n * op.NP + c0 + i;
                            if (col < op.n_cols) {
                                const int32_t kl = __ldg(a.sym_kl + col);
                                const int k = kl & 0xFFFF, l = kl >> 16;
                                const float v = __uint_as_float(r[i]) * unscale;
                                dst[k * a.n_phi + l] = v;
                                dst[l * a.n_phi + k] = v;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncthreads();
        }
    }
    if (aborted || *sm.abort_flag) {
        if (tid == 0) atomicOr(a.status, ST_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace

size_t tc_smem_bytes(const TcArgs &a) {
    size_t b = 1024;  // alignment slack
    b += (size_t)TC_STAGES * TC_M * TC_CHUNK_BYTES;
    b += (size_t)TC_STAGES * np_max(a) * TC_CHUNK_BYTES;
    b += (2 * TC_STAGES + 1) * sizeof(uint64_t) + 16;
    b += (size_t)a.n_phi * a.n_phi * sizeof(int16_t) + 16;
    return b;
}

int launch_tc_elements(const TcArgs &a, size_t smem, cudaStream_t s) {
    if (a.n_cells <= 0) return 0;
    const int64_t grid = (a.n_cells + TC_M - 1) / TC_M;
    cudaError_t e;
    if (a.prec == FE_PREC_E4M3) {
        e = cudaFuncSetAttribute(tc_element_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return -(int)e;
        tc_element_kernel<2><<<(unsigned)grid, TC_THREADS, smem, s>>>(a);
    } else if (a.prec == FE_PREC_TF32 || a.prec == FE_PREC_TF32X3) {
        e = cudaFuncSetAttribute(tc_element_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return -(int)e;
        tc_element_kernel<1><<<(unsigned)grid, TC_THREADS, smem, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(tc_element_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return -(int)e;
        tc_element_kernel<0><<<(unsigned)grid, TC_THREADS, smem, s>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return -(int)e;
    return 1;
}

}  // namespace fe
