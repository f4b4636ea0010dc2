// Tensor-core element-matrix kernel (sm_103a, tcgen05), persistent and
// warp-specialised, over one plan or a batch of plans (segments).
//
// Algorithm 1 of the paper for a tile of 128 cells at once, written as one
// dense contraction per tile with the cells on the MMA M dimension:
//
//   A^c_{kl} = sum_{(s<=t), q} C^c_{(st,q)} P_{(st,q),(kl)}          (k <= l)
//
// where C^c_{(st,q)} = w_q kappa_cq G^c_st (Sec. 3.1, C_st = diag_q(w_q z(X_q)
// G_st)) is formed per cell from the factor kernel's outputs (FP32 window
// w_q kappa_cq and the FP64 geometry rounded to FP32, with the per-cell
// scale of the narrow formats), and
// P_{(st,q),(kl)} = B_skq B_tlq + [s != t] B_tkq B_slq is the product of the
// tabulated reference derivatives (the triple products B_s C_st B_t^T of
// Sec. 3.1 folded over the symmetric pairs), precomputed in FP64 at plan time
// and rounded once to the storage format.  For the mass form there is one
// pair, G = |det J| and B = phi.  The storage precision u_s applies to C and
// P; products and accumulation are FP32 in tensor memory (u_q): the mixed
// strategy of Sec. 4.5.  Only the upper triangle k <= l is computed; the
// epilogue mirrors it.
//
// The cell batching of Sec. 3.1 is generalised to uneven meshes: the global
// tile sequence is the concatenation of every segment's (plan's) tiles, each
// tile carrying its segment's shapes (cell type, degree, quadrature size) and
// buffers.  One CTA per SM walks its tiles; a job is one (tile, form, N pass).
// Roles:
//   warps 0-3  builders, one thread per cell: its factors and its window
//              (shared by every (s,t) pair and both forms) in registers, its
//              128-byte swizzled K-major row of C written into a 2-stage ring
//              (one a_full arrival per warp).
//   warps 4-11 epilogue, two warps per TMEM lane group: drain a finished
//              accumulator into a conflict-free staging area, release it, and
//              write row-major element matrices with coalesced stores: whole
//              matrices gathered from the pair columns (mirroring k <= l to
//              k > l; the columns are ordered so that these gathers hit
//              distinct banks), or, for the full-row layout of large
//              elements, each pass's rows as one contiguous run.
//   warp 12    bulk copies of the pre-swizzled P chunks into a 2-stage ring
//              (one 1-D copy per chunk, no multicast) and tcgen05.mma into
//              one of two 256-column FP32 TMEM accumulators (lane 0 issues).
// So the build of tile t+1, the MMAs and the stores of tile t overlap.  Every
// wait is bounded (globaltimer): a wait that sees no progress for the launch's
// limit (timeout_ns, counted from the start of that wait) sets the status word
// and all roles leave after in-flight copies and MMAs have drained.
#include <cstdio>

#include "fe_device.cuh"

namespace fe {

namespace {

constexpr int V_THREADS = 416;   // 13 warps
constexpr int W_EPI0 = 4;        // warps 4-11: epilogue, two per TMEM lane group
constexpr int N_EPI = 8;
constexpr int W_MMA = 12;
constexpr int RING = 2;          // A and B ring stages
constexpr int ACC_COLS = 256;    // columns per TMEM accumulator (2 of them)
constexpr int MAX_F2S_IT = 16;   // n_phi^2 <= 512 for the staged epilogue

struct Smem {
    uint8_t *A;        // [RING][128][128 B]
    uint8_t *B;        // [RING][np_max][128 B]
    float *stage;      // [4][32][pitch_max]
    float *meta;       // [2][128] unscale per cell for the two accumulators
    float *rowc;       // [128][8] per cell: G pairs * scale (stiffness), |det J| * scale (mass)
    uint64_t *a_full, *a_empty, *b_full, *b_empty, *acc_full, *acc_empty, *meta_full, *meta_empty, *drain;
    uint32_t *tmem_holder;
    int *flags;        // [0] abort, [1] status bits
};

__host__ __device__ inline size_t align1k(size_t x) { return (x + 1023) & ~size_t(1023); }
__host__ __device__ inline size_t bytes_A() { return (size_t)RING * TC_M * TC_CHUNK_BYTES; }
__host__ __device__ inline size_t bytes_B(const TcArgs &a) { return (size_t)RING * a.np_max * TC_CHUNK_BYTES; }
__host__ __device__ inline size_t bytes_stage(const TcArgs &a) {
    return a.pitch_max > 0 ? align1k((size_t)4 * 32 * a.pitch_max * sizeof(float)) : 0;
}

__device__ inline Smem carve(uint8_t *raw, const TcArgs &a) {
    uintptr_t p = (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023);
    Smem s;
    s.A = reinterpret_cast<uint8_t *>(p);
    s.B = s.A + bytes_A();
    s.stage = reinterpret_cast<float *>(s.B + bytes_B(a));
    uint8_t *q = reinterpret_cast<uint8_t *>(s.stage) + bytes_stage(a);
    s.meta = reinterpret_cast<float *>(q);
    s.rowc = s.meta + 2 * TC_M;
    q = reinterpret_cast<uint8_t *>(s.rowc + 8 * TC_M);
    q = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(q) + 7) & ~uintptr_t(7));
    uint64_t *b = reinterpret_cast<uint64_t *>(q);
    s.a_full = b;
    s.a_empty = b + RING;
    s.b_full = b + 2 * RING;
    s.b_empty = b + 3 * RING;
    s.acc_full = b + 4 * RING;
    s.acc_empty = s.acc_full + 2;
    s.meta_full = s.acc_empty + 2;
    s.meta_empty = s.meta_full + 2;
    s.drain = s.meta_empty + 2;
    s.tmem_holder = reinterpret_cast<uint32_t *>(s.drain + 1);
    s.flags = reinterpret_cast<int *>(s.tmem_holder + 2);
    return s;
}

// Segment of a global tile (binary search over the segments' first tiles).
// The single-plan instantiation addresses the kernel parameter directly.
template <bool BATCHED>
__device__ __forceinline__ const TcSeg &seg_of(const TcArgs &a, int64_t t) {
    if (!BATCHED) return a.seg0;
    int lo = 0, hi = a.n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    return a.segs[lo];
}

__device__ __forceinline__ int first_form(const TcSeg &S) { return (S.form_mask & 1) ? 0 : 1; }

template <int PREC, bool BATCHED>
__global__ void __launch_bounds__(V_THREADS, 1) tc_element_kernel(const __grid_constant__ TcArgs a) {
    constexpr int EB = (PREC == FE_PREC_E4M3) ? 1 : ((PREC == FE_PREC_TF32 || PREC == FE_PREC_TF32X3) ? 4 : 2);
    constexpr int KIND = (PREC == FE_PREC_E4M3) ? 2 : ((EB == 4) ? 1 : 0);
    constexpr int KCE = TC_CHUNK_BYTES / EB;  // quadrature points per chunk

    // a CTA that starts after another one gave up does no work at all: one
    // thread reads the status word and the whole CTA takes its answer, before
    // any barrier or warp-collective (.sync.aligned) instruction
    __shared__ int s_gave_up;
    if (threadIdx.x == 0) s_gave_up = (*reinterpret_cast<volatile int *>(a.status) & ST_TIMEOUT) != 0;
    __syncthreads();
    if (s_gave_up) return;

    extern __shared__ uint8_t smem_raw[];
    Smem sm = carve(smem_raw, a);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t n_tiles = a.n_tiles;
    const int NPm = a.np_max;

    if (tid == 0) {
        for (int s = 0; s < RING; ++s) {
            mbar_init(&sm.a_full[s], TC_M / 32);         // one arrival per builder warp
            mbar_init(&sm.a_empty[s], 1);
            mbar_init(&sm.b_full[s], 1);
            mbar_init(&sm.b_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sm.acc_full[b], 1);
            mbar_init(&sm.acc_empty[b], N_EPI);          // one per epilogue warp
            mbar_init(&sm.meta_full[b], TC_M / 32);
            mbar_init(&sm.meta_empty[b], N_EPI);
        }
        mbar_init(sm.drain, 1);
        sm.flags[0] = 0;
        sm.flags[1] = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(sm.tmem_holder, 2 * ACC_COLS);
        tmem_relinquish();
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sm.tmem_holder;
    const unsigned long long deadline = a.timeout_ns;   // per wait: the longest a wait may see no progress
    volatile int *abort_flag = sm.flags;

    if (warp < 4) {
        // ======================= builders =======================
        // The factor kernel has left, per cell, the FP32 coefficient window
        // w_q kappa_cq and the scaled geometry factors.  For the 16- and 32-bit
        // formats the operand C is built with one thread per cell: the thread
        // keeps its cell's window (one 128-byte chunk's worth of points) in
        // registers and writes its own 128-byte K-major row as eight swizzled
        // 16-byte stores.  For e4m3 (128 points per chunk) the window is held
        // one lane per 4 points over the warp's 32 cells, with coalesced loads
        // and one 32-bit word per lane and row.
        constexpr bool CELL_ROWS = (PREC != FE_PREC_E4M3);
        constexpr int QL = KCE / 32;            // e4m3: points per lane
        const int cl = tid;
        const int wrow0 = warp * 32;
        int ac = 0, jb = 0;
        float win[CELL_ROWS ? KCE : 1];
        // win[i] = the window row wrow's entry q = qw * KCE + i (wrow = this
        // thread's cell, times the slots per cell, plus the slot)
        auto load_own = [&](const float *__restrict__ W, int ldw, int64_t wrow, bool valid, int qw) {
            const float *row = W + wrow * ldw + qw * KCE;
#pragma unroll
            for (int i = 0; i < KCE; i += 4) {
                const float4 v = (valid && qw * KCE + i < ldw) ? __ldg(reinterpret_cast<const float4 *>(row + i))
                                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                win[i] = v.x;
                win[i + 1] = v.y;
                win[i + 2] = v.z;
                win[i + 3] = v.w;
            }
        };
        // dst[r * QL + i] = entry q = qw * KCE + lane * QL + i of slot `slot` of
        // cell r's window (e4m3)
        auto load_rows = [&](const float *__restrict__ W, int ldw, int slots, int slot, int64_t n_cells,
                             int64_t tile_cell0, int qw, float *dst) {
            const int q = qw * KCE + lane * QL;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int64_t cell_r = tile_cell0 + wrow0 + r;
                const float4 v = (cell_r < n_cells && q < ldw)
                                     ? __ldg(reinterpret_cast<const float4 *>(W + (cell_r * slots + slot) * ldw + q))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                dst[r * QL] = v.x;
                dst[r * QL + 1] = v.y;
                dst[r * QL + 2] = v.z;
                dst[r * QL + 3] = v.w;
            }
        };
        // the window and factor blocks of a tile are contiguous: pull the next
        // tile's into L2 while this one is built
        auto prefetch_tile = [&](int64_t tt) {
            if (tt >= n_tiles || cl != 0) return;
            const TcSeg &S = seg_of<BATCHED>(a, tt);
            const int64_t c0 = (tt - S.tile_begin) * TC_M;
            const int64_t nc = (S.n_cells - c0) < TC_M ? (S.n_cells - c0) : TC_M;
            prefetch_l2(S.win + c0 * S.ldw * S.win_slots, (uint32_t)(nc * S.ldw * S.win_slots * sizeof(float)));
            prefetch_l2(S.cellf + c0 * CELLF, (uint32_t)(nc * CELLF * sizeof(float)));
        };
        prefetch_tile(blockIdx.x);
        for (int64_t t = blockIdx.x; t < n_tiles && !*abort_flag; t += gridDim.x) {
            prefetch_tile(t + gridDim.x);
            const TcSeg &S = seg_of<BATCHED>(a, t);
            const float *__restrict__ s_win = S.win;
            const int s_ldw = S.ldw;
            const int64_t s_ncells = S.n_cells;
            const int s_nq = S.n_q;
            const int64_t tile_cell0 = (t - S.tile_begin) * TC_M;
            const int64_t cell = tile_cell0 + cl;
            const bool valid = cell < s_ncells;
            // this cell's factors: scaled geometry to the shared row table, unscales
            float unscale_f[MAX_FORMS] = {1.f, 1.f};
            {
                float rec[12];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float4 v = valid ? __ldg(reinterpret_cast<const float4 *>(S.cellf + cell * CELLF) + i)
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                    rec[4 * i] = v.x;
                    rec[4 * i + 1] = v.y;
                    rec[4 * i + 2] = v.z;
                    rec[4 * i + 3] = v.w;
                }
#pragma unroll
                for (int j = 0; j < 7; ++j) sm.rowc[cl * 8 + j] = rec[CELLF_G + j];
                if (valid) {
                    unscale_f[0] = rec[CELLF_UNSCALE];
                    unscale_f[1] = rec[CELLF_UNSCALE + 1];
                }
            }
            // a tile whose points fit one window (shared by every pair) loads it
            // once, here; loaded = qw * 16 + slot of the registers' window
            const int s_slots = S.win_slots;
            int qw_loaded = -1;
            if (CELL_ROWS && s_nq <= KCE && s_slots == 1) {
                load_own(s_win, s_ldw, cell, valid, 0);
                qw_loaded = 0;
            }
            __syncwarp();
            for (int f = 0; f < MAX_FORMS; ++f) {
                if (!(S.form_mask & (1 << f))) continue;
                const TcOperand op = S.op[f];
                const int per_qw = op.n_pairs * op.n_blk;
                for (int n = 0; n < op.n_pass; ++n) {
                    const int b = jb & 1, ub = jb >> 1;
                    if (jb >= 2 && !mbar_wait_warp(&sm.meta_empty[b], (ub - 1) & 1, deadline)) {
                        sm.flags[0] = 1;
                        break;
                    }
                    sm.meta[b * TC_M + cl] = unscale_f[f];
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.meta_full[b]);
                    for (int ch = 0; ch < op.n_kchunks; ++ch) {
                        const int s = ac % RING, ua = ac / RING;
                        if (ac >= RING && !mbar_wait_warp(&sm.a_empty[s], (ua - 1) & 1, deadline)) {
                            sm.flags[0] = 1;
                            break;
                        }
                        const int qw = ch / per_qw;
                        const int j = (ch / op.n_blk) % op.n_pairs;
                        const int blk = ch % op.n_blk;
                        const int cidx = (f == 0) ? j : 6;
                        // window slot: simplices share one; boxed cells have one per pair and one for the mass form
                        const int slot = (s_slots == 1) ? 0 : ((f == 0) ? j : s_slots - 1);
                        uint8_t *stA = sm.A + s * (TC_M * TC_CHUNK_BYTES);
                        if constexpr (CELL_ROWS) {
                            if (qw * 16 + slot != qw_loaded) {
                                qw_loaded = qw * 16 + slot;
                                load_own(s_win, s_ldw, cell * s_slots + slot, valid, qw);
                            }
                            const float gj = sm.rowc[cl * 8 + cidx];
                            uint8_t *rowp = stA + (cl >> 3) * 1024 + (cl & 7) * 128;
                            constexpr int GE = 16 / EB;   // elements per 16-byte granule
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const float *w = win + k * GE;
                                uint4 v;
                                if constexpr (PREC == FE_PREC_BF16) {
                                    v.x = pack_bf16x2(w[0] * gj, w[1] * gj);
                                    v.y = pack_bf16x2(w[2] * gj, w[3] * gj);
                                    v.z = pack_bf16x2(w[4] * gj, w[5] * gj);
                                    v.w = pack_bf16x2(w[6] * gj, w[7] * gj);
                                } else if constexpr (PREC == FE_PREC_FP16) {
                                    v.x = pack_f16x2(w[0] * gj, w[1] * gj);
                                    v.y = pack_f16x2(w[2] * gj, w[3] * gj);
                                    v.z = pack_f16x2(w[4] * gj, w[5] * gj);
                                    v.w = pack_f16x2(w[6] * gj, w[7] * gj);
                                } else {
                                    uint32_t u[4];
#pragma unroll
                                    for (int e = 0; e < 4; ++e) {
                                        const float x = w[e] * gj;
                                        u[e] = round_tf32(x);
                                        if (PREC == FE_PREC_TF32X3 && blk == 2) u[e] = round_tf32(x - __uint_as_float(u[e]));
                                    }
                                    v = make_uint4(u[0], u[1], u[2], u[3]);
                                }
                                *reinterpret_cast<uint4 *>(rowp + ((k ^ (cl & 7)) << 4)) = v;
                            }
                        } else {
                            float w[32 * QL];
                            load_rows(s_win, s_ldw, s_slots, slot, s_ncells, tile_cell0, qw, w);
                            const int byte = lane * 4;   // this lane's word inside a 128-byte row
#pragma unroll
                            for (int r = 0; r < 32; ++r) {
                                const int R = wrow0 + r;
                                const float gj = sm.rowc[R * 8 + cidx];
                                const uint32_t word = pack_e4m3x2(w[r * QL] * gj, w[r * QL + 1] * gj) |
                                                      (pack_e4m3x2(w[r * QL + 2] * gj, w[r * QL + 3] * gj) << 16);
                                *reinterpret_cast<uint32_t *>(stA + (R >> 3) * 1024 + (R & 7) * 128 +
                                                              ((((byte >> 4) ^ (R & 7)) & 7) << 4) + (byte & 15)) = word;
                            }
                        }
                        fence_proxy_async();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sm.a_full[s]);
                        ++ac;
                    }
                    ++jb;
                    if (*abort_flag) break;
                }
                if (*abort_flag) break;
            }
        }
    } else if (warp == W_MMA) {
        // ======================= bulk copies + MMA =======================
        // B cursor: (tile, form, pass, chunk) of the next shared-operand copy;
        // bc counts the copies issued (the same in every lane).
        int64_t bt = blockIdx.x, bc = 0;
        int bf = 0, bn = 0, bch = 0;
        if (bt < n_tiles) bf = first_form(seg_of<BATCHED>(a, bt));
        auto issue_b = [&](int64_t upto) -> bool {
            while (bc < upto && bt < n_tiles) {
                const TcSeg &S = seg_of<BATCHED>(a, bt);
                const TcOperand &op = S.op[bf];
                const uint32_t bytes = (uint32_t)op.NP * TC_CHUNK_BYTES;
                const int s = (int)(bc % RING);
                const int64_t ub = bc / RING;
                if (bc >= RING && !mbar_wait_warp(&sm.b_empty[s], (uint32_t)((ub - 1) & 1), deadline)) return false;
                if (lane == 0) {
                    mbar_arrive_expect_tx(&sm.b_full[s], bytes);
                    bulk_g2s(sm.B + (size_t)s * NPm * TC_CHUNK_BYTES, op.img + ((size_t)bn * op.n_kchunks + bch) * bytes,
                             bytes, &sm.b_full[s]);
                }
                __syncwarp();
                ++bc;
                if (++bch == op.n_kchunks) {
                    bch = 0;
                    if (++bn == op.n_pass) {
                        bn = 0;
                        int nf = bf + 1;
                        while (nf < MAX_FORMS && !(S.form_mask & (1 << nf))) ++nf;
                        if (nf < MAX_FORMS) {
                            bf = nf;
                        } else {
                            bt += gridDim.x;
                            if (bt < n_tiles) bf = first_form(seg_of<BATCHED>(a, bt));
                        }
                    }
                }
            }
            return true;
        };
        int64_t mc = 0;
        int jb = 0;
        bool fail = !issue_b(RING);
        for (int64_t t = blockIdx.x; t < n_tiles && !fail; t += gridDim.x) {
            const TcSeg &S = seg_of<BATCHED>(a, t);
            for (int f = 0; f < MAX_FORMS && !fail; ++f) {
                if (!(S.form_mask & (1 << f))) continue;
                const TcOperand op = S.op[f];
                const uint32_t idesc = a.idesc | ((uint32_t)(op.NP >> 3) << 17);
                for (int n = 0; n < op.n_pass && !fail; ++n) {
                    const int b = jb & 1, ub = jb >> 1;
                    if (jb >= 2 && !mbar_wait_warp(&sm.acc_empty[b], (ub - 1) & 1, deadline)) {
                        fail = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dacc = tmem + (uint32_t)(b * ACC_COLS);
                    for (int ch = 0; ch < op.n_kchunks; ++ch) {
                        const int sa = (int)(mc % RING);
                        const uint32_t par = (uint32_t)((mc / RING) & 1);
                        if (!mbar_wait_warp(&sm.a_full[sa], par, deadline) || !mbar_wait_warp(&sm.b_full[sa], par, deadline)) {
                            fail = true;
                            break;
                        }
                        tc_fence_after();
                        if (lane == 0) {
                            const uint32_t a0 = smem_u32(sm.A + sa * (TC_M * TC_CHUNK_BYTES));
                            const uint32_t b0 = smem_u32(sm.B + (size_t)sa * NPm * TC_CHUNK_BYTES);
#pragma unroll
                            for (int ks = 0; ks < TC_CHUNK_BYTES / 32; ++ks)
                                umma<KIND>(dacc, sdesc_sw128(a0 + 32 * ks), sdesc_sw128(b0 + 32 * ks), idesc,
                                           (ch | ks) != 0 ? 1u : 0u);
                            umma_commit(&sm.a_empty[sa]);
                            umma_commit(&sm.b_empty[sa]);
                            if (ch == op.n_kchunks - 1) umma_commit(&sm.acc_full[b]);
                        }
                        __syncwarp();
                        ++mc;
                        // refill the stage of chunk mc-1 once its MMAs are done
                        if (!issue_b(mc + RING)) {
                            fail = true;
                            break;
                        }
                    }
                    ++jb;
                    if (*abort_flag) fail = true;
                }
            }
        }
        if (fail) sm.flags[0] = 1;
        // drain: every issued MMA finished, every issued bulk copy landed
        if (lane == 0) umma_commit(sm.drain);
        __syncwarp();
        const unsigned long long drain_deadline = 200000000ull;   // 0.2 s per wait
        mbar_wait(sm.drain, 0, drain_deadline);
        for (int64_t c = mc; c < bc; ++c) mbar_wait(&sm.b_full[c % RING], (uint32_t)((c / RING) & 1), drain_deadline);
    } else if (warp >= W_EPI0 && warp < W_EPI0 + N_EPI) {
        // ======================= epilogue =======================
        // warps 4-7 and 8-11: lane group g = warp % 4 (TMEM lanes 32g..32g+31),
        // half h: alternate 32-column blocks when draining TMEM, cells
        // 16h..16h+15 of the lane group when writing out.
        const int g = warp & 3;
        const int h = (warp - W_EPI0) >> 2;
        __shared__ volatile int pair_ok[8];   // [lane group][half]: outcome of the current pass's waits
        const int pitch = a.pitch_max;
        float *stg = sm.stage + g * 32 * pitch;
        int f2s_reg[MAX_F2S_IT];
        const TcSeg *cur = nullptr;
        int jb = 0;
        // Every decision to stop is taken per pass, after the pass's waits, and
        // (for staged segments) jointly by the two warps of the lane group.
        bool stop = false;
        for (int64_t t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x) {
            const TcSeg &S = seg_of<BATCHED>(a, t);
            const int nph = S.n_phi, nph2 = nph * nph;
            const int n_it = (nph2 + 31) / 32;
            // 16-byte stores when every matrix starts on a 16-byte boundary
            const bool v4 = (nph2 & 3) == 0;
            if (&S != cur) {
                // sym index of each output position this lane writes: v4 -> positions
                // 128 it + 4 lane + e in register 4 it + e; otherwise lane + 32 it
#pragma unroll
                for (int it = 0; it < MAX_F2S_IT; ++it) {
                    const int pos = v4 ? 128 * (it >> 2) + 4 * lane + (it & 3) : lane + 32 * it;
                    f2s_reg[it] = (S.staged && pos < nph2) ? __ldg(S.full2sym + pos) : 0;
                }
                cur = &S;
            }
            for (int f = 0; f < MAX_FORMS; ++f) {
                if (!(S.form_mask & (1 << f))) continue;
                const TcOperand op = S.op[f];
                float *__restrict__ out = S.out[f];
                const int64_t s_ncells = S.n_cells;
                const int s_staged = S.staged;
                const int32_t *__restrict__ s_symkl = S.sym_kl;
                for (int n = 0; n < op.n_pass; ++n) {
                    const int b = jb & 1, ub = jb >> 1;
                    bool ok = !*abort_flag && mbar_wait_warp(&sm.acc_full[b], ub & 1, deadline) &&
                              mbar_wait_warp(&sm.meta_full[b], ub & 1, deadline);
                    if (s_staged) {
                        // the two warps of this lane group meet at named barriers below:
                        // they take one common outcome here, so that a wait that gave up
                        // in one of them cannot leave the other alone at a barrier
                        if (lane == 0) pair_ok[g * 2 + h] = ok ? 1 : 0;
                        named_bar_sync(1 + g, 64);
                        ok = pair_ok[g * 2] && pair_ok[g * 2 + 1];
                    }
                    if (!ok) {
                        sm.flags[0] = 1;
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const float us = sm.meta[b * TC_M + g * 32 + lane];
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.meta_empty[b]);
                    const uint32_t tbase = tmem + (uint32_t)(b * ACC_COLS) + ((uint32_t)(g * 32) << 16);
                    const int64_t cell0 = (t - S.tile_begin) * TC_M + g * 32;
                    if (s_staged) {
                        float *mine = stg + lane * pitch;
                        for (int c0 = 32 * h; c0 < op.NP; c0 += 64) {
                            uint32_t r[32];
                            tmem_ld32(tbase + (uint32_t)c0, r);
#pragma unroll
                            for (int i = 0; i < 32; ++i)
                                if (c0 + i < op.NP) mine[c0 + i] = __uint_as_float(r[i]) * us;
                        }
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sm.acc_empty[b]);
                        named_bar_sync(1 + g, 64);
                        // whole row-major matrices of 16 consecutive cells (loads first, then stores)
                        if (out && op.rows_per_pass > 0) {
                            // full-row pass: rows [k0, k0 + R) of each cell are one contiguous run
                            const int k0 = n * op.rows_per_pass;
                            const int len = (nph - k0 < op.rows_per_pass ? nph - k0 : op.rows_per_pass) * nph;
                            for (int cc = 16 * h; cc < 16 * h + 16; ++cc) {
                                if (cell0 + cc >= s_ncells) break;
                                float *__restrict__ dst = out + (cell0 + cc) * (int64_t)nph2 + (int64_t)k0 * nph;
                                const float *__restrict__ src = stg + cc * pitch;
                                for (int i0 = 0; i0 < len; i0 += 128) {
                                    float x[4];
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        const int i = i0 + u * 32 + lane;
                                        x[u] = i < len ? src[i] : 0.f;
                                    }
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        const int i = i0 + u * 32 + lane;
                                        if (i < len) __stcs(dst + i, x[u]);
                                    }
                                }
                            }
                        } else if (out && v4) {
                            // two cells per step, 16-byte coalesced stores
                            for (int cc = 16 * h; cc < 16 * h + 16; cc += 2) {
                                float4 vals[2][MAX_F2S_IT / 4];
#pragma unroll
                                for (int u = 0; u < 2; ++u) {
                                    const float *__restrict__ src = stg + (cc + u) * pitch;
#pragma unroll
                                    for (int it = 0; it < MAX_F2S_IT / 4; ++it)
                                        vals[u][it] = make_float4(src[f2s_reg[4 * it]], src[f2s_reg[4 * it + 1]],
                                                                  src[f2s_reg[4 * it + 2]], src[f2s_reg[4 * it + 3]]);
                                }
#pragma unroll
                                for (int u = 0; u < 2; ++u) {
                                    if (cell0 + cc + u >= s_ncells) break;
                                    float *__restrict__ dst = out + (cell0 + cc + u) * (int64_t)nph2;
#pragma unroll
                                    for (int it = 0; it < MAX_F2S_IT / 4; ++it) {
                                        const int pos = 128 * it + 4 * lane;
                                        if (pos < nph2) __stcs(reinterpret_cast<float4 *>(dst + pos), vals[u][it]);
                                    }
                                }
                            }
                        } else if (out) {
                            for (int cc = 16 * h; cc < 16 * h + 16; ++cc) {
                                if (cell0 + cc >= s_ncells) break;
                                float *__restrict__ dst = out + (cell0 + cc) * (int64_t)nph2;
                                const float *__restrict__ src = stg + cc * pitch;
                                float vals[MAX_F2S_IT];
#pragma unroll
                                for (int it = 0; it < MAX_F2S_IT; ++it) vals[it] = (it < n_it) ? src[f2s_reg[it]] : 0.f;
#pragma unroll
                                for (int it = 0; it < MAX_F2S_IT; ++it) {
                                    const int pos = lane + 32 * it;
                                    if (it < n_it && pos < nph2) __stcs(dst + pos, vals[it]);
                                }
                            }
                        }
                        named_bar_sync(1 + g, 64);
                    } else {
                        const int64_t mycell = cell0 + lane;
                        for (int c0 = 32 * h; c0 < op.NP; c0 += 64) {
                            uint32_t r[32];
                            tmem_ld32(tbase + (uint32_t)c0, r);
                            if (mycell < s_ncells && out) {
                                float *dst = out + mycell * (int64_t)nph2;
#pragma unroll
                                for (int i = 0; i < 32; ++i) {
                                    const int col = n * op.NP + c0 + i;
                                    if (op.rows_per_pass > 0) {
                                        // full-row layout: column c of pass n is entry (nR + c / n_phi, c % n_phi)
                                        const int cc = c0 + i;
                                        const int k = n * op.rows_per_pass + cc / nph;
                                        if (cc < op.NP && cc < op.rows_per_pass * nph && k < nph)
                                            __stcs(dst + k * nph + cc % nph, __uint_as_float(r[i]) * us);
                                        continue;
                                    }
                                    const int32_t kl = (c0 + i < op.NP && col < op.n_cols) ? __ldg(s_symkl + col) : -1;
                                    if (kl >= 0) {   // (padding columns carry no pair)
                                        const int k = kl & 0xFFFF, l = kl >> 16;
                                        const float v = __uint_as_float(r[i]) * us;
                                        __stcs(dst + k * nph + l, v);
                                        __stcs(dst + l * nph + k, v);
                                    }
                                }
                            }
                        }
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sm.acc_empty[b]);
                    }
                    ++jb;
                }
                if (stop) break;
            }
        }
    }
    if (sm.flags[0] && tid == 0) atomicOr(&sm.flags[1], ST_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && sm.flags[1]) atomicOr(a.status, sm.flags[1]);
    if (warp == 0) tmem_dealloc(tmem, 2 * ACC_COLS);
}

}  // namespace

size_t tc_smem_bytes(const TcArgs &a) {
    size_t b = 1024;  // alignment slack
    b += bytes_A() + bytes_B(a) + bytes_stage(a);
    b += 2 * TC_M * sizeof(float) + 8 * TC_M * sizeof(float);
    b += 8;
    b += (4 * RING + 9) * sizeof(uint64_t) + 8 + 16;
    return b;
}

bool tc_can_stage(const TcArgs &a, const TcSeg &seg) {
    int np = 16;
    bool pairs = false;
    for (int f = 0; f < MAX_FORMS; ++f)
        if ((seg.form_mask >> f) & 1) {
            // the pair layout is staged in one pass; the full-row layout in any number
            if (seg.op[f].rows_per_pass == 0) {
                if (seg.op[f].n_pass != 1) return false;
                pairs = true;
            }
            np = seg.op[f].NP > np ? seg.op[f].NP : np;
        }
    if (pairs && seg.n_phi * seg.n_phi > 32 * MAX_F2S_IT) return false;
    TcArgs t = a;
    t.pitch_max = (np + 1) > a.pitch_max ? (np + 1) : a.pitch_max;
    return tc_smem_bytes(t) <= 227 * 1024;
}

template <int PREC, bool BATCHED>
static int launch_prec2(const TcArgs &a, size_t smem, cudaStream_t s, int grid) {
    cudaError_t e =
        cudaFuncSetAttribute(tc_element_kernel<PREC, BATCHED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -(int)e;
    tc_element_kernel<PREC, BATCHED><<<(unsigned)grid, V_THREADS, smem, s>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

template <int PREC>
static int launch_prec(const TcArgs &a, size_t smem, cudaStream_t s, int grid) {
    return a.segs ? launch_prec2<PREC, true>(a, smem, s, grid) : launch_prec2<PREC, false>(a, smem, s, grid);
}

int launch_tc_elements(const TcArgs &a, size_t smem, cudaStream_t s, int grid) {
    if (a.n_tiles <= 0) return 0;
    if (grid <= 0) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = sms;
    }
    if (grid > a.n_tiles) grid = (int)a.n_tiles;
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
