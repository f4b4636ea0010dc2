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
// buffers.  A job is one (tile, form, N pass); one CTA per SM takes a
// contiguous run of jobs of equal cost (K chunks plus an epilogue share), so
// the SMs stay evenly loaded when the tiles do not divide over them, or, for
// one plan whose shared operand exceeds a quarter of L2, every G-th job in
// pass-major order, so that all CTAs stream the same operand chunks at once.
// Roles:
//   warps 0-3  builders, one thread per cell: its factors and its window
//              (shared by every (s,t) pair and both forms) in registers, its
//              128-byte swizzled K-major row of C written into a 2- to 4-stage
//              ring (one a_full arrival per warp); where a job reads several
//              windows, optionally the next one copied asynchronously into a
//              per-thread shared-memory slot while the current one is used.
//   warps 4-11 epilogue, two warps per TMEM lane group: drain a finished
//              accumulator into a conflict-free staging area, release it, and
//              write row-major element matrices with coalesced stores: whole
//              matrices gathered from the pair columns (mirroring k <= l to
//              k > l; the columns are ordered so that these gathers hit
//              distinct banks), or, for the full-row layout of large
//              elements, each pass's rows as one contiguous run.  Full-row
//              passes that do not fit the staging area, and wide passes,
//              leave from registers: each lane writes its own cell's run in
//              16-byte stores where it is aligned.
//   warp 12    tcgen05.mma into one of two 256-column FP32 TMEM accumulators,
//              or, for a wide full-row pass (up to 512 columns), into both
//              halves as one accumulator with two MMAs per K step (lane 0
//              issues); it only waits for operands, never for its own MMAs,
//              so the tensor pipe always has the next chunk queued.
//   warp 13    bulk copies of the pre-swizzled P chunks (one 1-D copy per
//              chunk, no multicast) into a ring of 2-8 stages, as deep as shared
//              memory allows beside the staging area: the copies in flight
//              cover the L2 latency of the next chunks.
// So the build of tile t+1, the MMAs and the stores of tile t overlap.  Every
// wait is bounded (globaltimer): a wait that sees no progress for the launch's
// limit (timeout_ns, counted from the start of that wait) sets the status word
// and all roles leave after in-flight copies and MMAs have drained.
#include <cstdio>

#include "fe_device.cuh"

namespace fe {

namespace {

constexpr int V_THREADS = 448;   // 14 warps
constexpr int W_EPI0 = 4;        // warps 4-11: epilogue, two per TMEM lane group
constexpr int N_EPI = 8;
constexpr int W_MMA = 12;
constexpr int W_PROD = 13;       // bulk copies of the shared operand
constexpr int ACC_COLS = 256;    // columns per TMEM accumulator (2 of them)
constexpr int MAX_F2S_IT = 16;   // n_phi^2 <= 512 for the staged epilogue

struct Smem {
    uint8_t *A;        // [ring_a][128][128 B]
    uint8_t *B;        // [ring_b][np_max][128 B]
    float *stage;      // [4][32][pitch_max]
    float *meta;       // [2][128] unscale per cell for the two accumulators
    float *wnext;      // [128][KW + 4] each builder thread's next window (win_buf)
    uint64_t *a_full, *a_empty, *b_full, *b_empty, *acc_full, *acc_empty, *meta_full, *meta_empty, *drain;
    uint32_t *tmem_holder;
    int *flags;        // [0] abort, [1] status bits
};

__host__ __device__ inline size_t align1k(size_t x) { return (x + 1023) & ~size_t(1023); }
__host__ __device__ inline size_t bytes_A(const TcArgs &a) { return (size_t)a.ring_a * TC_M * TC_CHUNK_BYTES; }
__host__ __device__ inline size_t bytes_B(const TcArgs &a) { return (size_t)a.ring_b * a.np_max * TC_CHUNK_BYTES; }
__host__ __device__ inline size_t bytes_stage(const TcArgs &a) {
    return a.pitch_max > 0 ? align1k((size_t)4 * 32 * a.pitch_max * sizeof(float)) : 0;
}
// the next-window slots: a pitch of KW + 4 floats keeps each quarter warp's
// 16-byte accesses on distinct banks
__host__ __device__ inline int wnext_pitch(const TcArgs &a) { return tc_window_points(a.prec) + 4; }
__host__ __device__ inline size_t bytes_wnext(const TcArgs &a) {
    return a.win_buf ? (size_t)TC_M * wnext_pitch(a) * sizeof(float) : 0;
}

__device__ inline Smem carve(uint8_t *raw, const TcArgs &a) {
    uintptr_t p = (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023);
    Smem s;
    s.A = reinterpret_cast<uint8_t *>(p);
    s.B = s.A + bytes_A(a);
    s.stage = reinterpret_cast<float *>(s.B + bytes_B(a));
    uint8_t *q = reinterpret_cast<uint8_t *>(s.stage) + bytes_stage(a);
    s.wnext = reinterpret_cast<float *>(q);
    q += bytes_wnext(a);
    s.meta = reinterpret_cast<float *>(q);
    q = reinterpret_cast<uint8_t *>(s.meta + 2 * TC_M);
    q = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(q) + 7) & ~uintptr_t(7));
    uint64_t *b = reinterpret_cast<uint64_t *>(q);
    s.a_full = b;
    s.a_empty = b + TC_MAX_RING_A;
    s.b_full = b + 2 * TC_MAX_RING_A;
    s.b_empty = s.b_full + TC_MAX_RING_B;
    s.acc_full = s.b_empty + TC_MAX_RING_B;
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

// The launch's jobs, (tile, form, N pass), in order: tiles in global order,
// then the passes, and in each pass the forms (so the short mass passes, whose
// stores outlast their MMAs, alternate with the long stiffness passes).  A job
// costs its form's K chunks
// plus TC_JOB_EPI_COST.  CTA i of G takes the contiguous jobs whose cost
// offset lies in [i T / G, (i + 1) T / G) of the total T, so the CTAs get the
// same work to within one job even when the tiles do not divide evenly over
// the SMs (a few hundred tiles of a high-degree element).  A tile may be
// split between two CTAs at a form or pass boundary.  Every role walks the
// same sequence with its own cursor.
template <bool BATCHED>
//
// Pass-major order (job_rr, one plan whose forms have the same number of
// passes): the jobs ordered (pass, form, tile) and dealt round-robin, CTA i
// taking jobs i, i + G, i + 2G, ...  All CTAs then work on the same pass at
// the same time, so each chunk of the shared operand is read from DRAM once
// and served to the others from L2 -- the order for an operand larger than
// the L2 share it can keep (high degrees).  The load stays balanced to one job.
struct Jobs {
    const TcSeg *S;   // segment of tile t
    int64_t t;        // global tile
    int f, n;         // form, pass
    int64_t c;        // cost offset of this job
    int64_t hi;       // end of this CTA's cost range
    int64_t n_tiles;
    // pass-major round robin
    bool rr;
    int stride, fidx, nf_rr, form_rr0, form_rr1, n_pass_rr;   // (the forms as scalars: no local array)

    __device__ __forceinline__ bool live() const { return rr ? n < n_pass_rr : (c < hi && t < n_tiles); }

    // the first form after g whose layout has pass `pass` (-1: none)
    __device__ __forceinline__ int form_after(int g, int pass) const {
        for (++g; g < MAX_FORMS; ++g)
            if ((S->form_mask & (1 << g)) && pass < S->op[g].n_pass) return g;
        return -1;
    }

    __device__ __forceinline__ void advance() {
        if (rr) {
            t += stride;
            while (t >= n_tiles && n < n_pass_rr) {
                t -= n_tiles;
                if (++fidx == nf_rr) {
                    fidx = 0;
                    ++n;
                }
            }
            f = fidx ? form_rr1 : form_rr0;
            return;
        }
        c += S->op[f].n_kchunks + TC_JOB_EPI_COST;
        int nf = form_after(f, n);
        if (nf < 0) nf = form_after(-1, ++n);
        if (nf >= 0) {
            f = nf;
            return;
        }
        n = 0;
        if (++t >= n_tiles) return;
        if (BATCHED)
            while (t >= S->tile_begin + S->tiles) ++S;   // t < n_tiles: a later segment holds it
        f = first_form(*S);
    }

    __device__ __forceinline__ void start(const TcArgs &a, int i, int G) {
        n_tiles = a.n_tiles;
        rr = !BATCHED && a.job_rr;
        if (rr) {
            S = &a.seg0;
            stride = G;
            form_rr0 = first_form(*S);
            form_rr1 = 1;
            nf_rr = (S->form_mask & 3) == 3 ? 2 : 1;
            n_pass_rr = S->op[form_rr0].n_pass;
            // job i: (pass, form, tile) = i in mixed radix (n_pass, forms, tiles)
            t = i % n_tiles;
            const int64_t q = i / n_tiles;
            fidx = (int)(q % nf_rr);
            n = (int)(q / nf_rr);
            f = fidx ? form_rr1 : form_rr0;
            c = hi = 0;
            return;
        }
        const int64_t T = a.total_cost;
        const int64_t lo = T * i / G;
        hi = T * (i + 1) / G;
        if (BATCHED) {
            int l = 0, h = a.n_segs - 1;   // the last segment starting at or before lo
            while (l < h) {
                const int mid = (l + h + 1) >> 1;
                if (a.segs[mid].cost_begin <= lo) l = mid; else h = mid - 1;
            }
            S = a.segs + l;
        } else {
            S = &a.seg0;
        }
        int64_t tt = S->tile_cost > 0 ? (lo - S->cost_begin) / S->tile_cost : 0;
        if (tt >= S->tiles) tt = S->tiles - 1;
        t = S->tile_begin + tt;
        c = S->cost_begin + tt * S->tile_cost;
        f = first_form(*S);
        n = 0;
        while (c < lo && t < n_tiles) advance();   // at most one tile's jobs
    }
};

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

    const int RA = a.ring_a, RB = a.ring_b;
    // accumulators: two 256-column buffers (pass j in buffer j % 2), or, when a
    // pass is wide, one of 512 columns (pass j a new use of buffer 0)
    const int NACC = a.n_acc, acc_mask = NACC - 1, acc_shift = NACC - 1;
    if (tid == 0) {
        for (int s = 0; s < RA; ++s) {
            mbar_init(&sm.a_full[s], TC_M / 32);         // one arrival per builder warp
            mbar_init(&sm.a_empty[s], 1);
        }
        for (int s = 0; s < RB; ++s) {
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
        // w_q kappa_cq and the scaled geometry factors.  The operand C is built
        // with one thread per cell: the thread keeps its cell's current window
        // (KW consecutive points of one slot) in registers and writes its own
        // 128-byte K-major row of each chunk as eight swizzled 16-byte stores:
        // one K block of KW points per chunk for the 16- and 32-bit formats, two
        // 64-point blocks for e4m3 (128 points per chunk).
        constexpr int KW = tc_window_points(PREC);   // points per window (K block)
        constexpr int WPC = KCE / KW;                // K blocks per chunk
        constexpr int GE = 16 / EB;                  // elements per 16-byte granule
        constexpr int GPB = KW / GE;                 // granules per K block
        static_assert(WPC * GPB == 8, "a chunk row is eight granules");
        const int cl = tid;
        int ac = 0, jb = 0;
        float win[KW];
        // win[i] = the window row wrow's entry q = qw * KW + i (wrow = this
        // thread's cell, times the slots per cell, plus the slot)
        auto load_own = [&](const float *__restrict__ W, int ldw, int64_t wrow, bool valid, int qw) {
            const float *row = W + wrow * ldw + qw * KW;
#pragma unroll
            for (int i = 0; i < KW; i += 4) {
                const float4 v = (valid && qw * KW + i < ldw) ? __ldg(reinterpret_cast<const float4 *>(row + i))
                                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                win[i] = v.x;
                win[i + 1] = v.y;
                win[i + 2] = v.z;
                win[i + 3] = v.w;
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
        Jobs<BATCHED> J;
        J.start(a, blockIdx.x, gridDim.x);
        if (J.live()) prefetch_tile(J.t);
        int64_t cur_t = -1;
        float unscale_f[MAX_FORMS] = {1.f, 1.f};
        float gf[7];          // this cell's scaled G pairs and |det J|
        int qw_loaded = -1;
        // window prefetch (win_buf): the next distinct window this thread will
        // need is copied asynchronously into its own shared-memory slot while
        // the current one is used; key = qw * 16 + slot, -1 for none
        float *const myslot = sm.wnext + cl * wnext_pitch(a);
        int pf_key = -1, want_pf = -1;
        auto issue_pf = [&](const float *__restrict__ W, int ldw, int slots, int64_t c, bool valid, int key) {
            const int pq = key >> 4, ps = key & 15;
            const float *row = W + (c * slots + ps) * ldw + pq * KW;
#pragma unroll
            for (int i = 0; i < KW; i += 4) {
                const bool in = valid && pq * KW + i < ldw;
                cp_async16_zfill(myslot + i, in ? row + i : W, in ? 16u : 0u);
            }
            cp_async_commit();
        };
        int as = 0;           // built-operand stage of chunk ac, and its use parity
        uint32_t aph = 0;
        for (; J.live() && !*abort_flag; J.advance()) {
            const int64_t t = J.t;
            const TcSeg &S = *J.S;
            const float *__restrict__ s_win = S.win;
            const int s_ldw = S.ldw;
            const int64_t s_ncells = S.n_cells;
            const int s_nq = S.n_q;
            const int64_t tile_cell0 = (t - S.tile_begin) * TC_M;
            const int64_t cell = tile_cell0 + cl;
            const bool valid = cell < s_ncells;
            const int s_slots = S.win_slots;
            if (t != cur_t) {
                // a new tile: this cell's factors (scaled geometry, unscales) and,
                // where its points fit one window, the window
                cur_t = t;
                if (pf_key >= 0) cp_async_wait_all();   // (the slot is reused below)
                pf_key = -1;
                prefetch_tile(t + 1);
                unscale_f[0] = unscale_f[1] = 1.f;
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
                    for (int j = 0; j < 7; ++j) gf[j] = rec[CELLF_G + j];
                    if (valid) {
                        unscale_f[0] = rec[CELLF_UNSCALE];
                        unscale_f[1] = rec[CELLF_UNSCALE + 1];
                    }
                }
                // a tile whose points fit one window (shared by every pair) loads it
                // once, here; loaded = qw * 16 + slot of the registers' window
                qw_loaded = -1;
                if (s_nq <= KW && s_slots == 1) {
                    load_own(s_win, s_ldw, cell, valid, 0);
                    qw_loaded = 0;
                }
                __syncwarp();
            }
            const int f = J.f;
            const TcOperand op = S.op[f];
            const int b = jb & 1, ub = jb >> 1;   // (the unscales are double-buffered whatever the accumulators)
            if (jb >= 2 && !mbar_wait_warp(&sm.meta_empty[b], (ub - 1) & 1, deadline)) {
                sm.flags[0] = 1;
                break;
            }
            sm.meta[b * TC_M + cl] = unscale_f[f];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.meta_full[b]);
            // running K block (window qw, pair j, split block blk) of the chunk row
            int qw = 0, j = 0, blk = 0;
            for (int ch = 0; ch < op.n_kchunks; ++ch) {
                const int s = as;
                if (ac >= RA && !mbar_wait_warp(&sm.a_empty[s], aph ^ 1u, deadline)) {
                    sm.flags[0] = 1;
                    break;
                }
                uint8_t *stA = sm.A + s * (TC_M * TC_CHUNK_BYTES);
                uint8_t *rowp = stA + (cl >> 3) * 1024 + (cl & 7) * 128;
#pragma unroll
                for (int sub = 0; sub < WPC; ++sub) {
                    const bool live = qw < op.n_qw;    // (e4m3: the last chunk may end with a zero block)
                    // window slot: simplices share one; boxed cells have one per pair and one for the mass form
                    const int slot = (s_slots == 1) ? 0 : ((f == 0) ? j : s_slots - 1);
                    const int key = qw * 16 + slot;
                    if (live && key != qw_loaded) {
                        if (key == pf_key) {
                            cp_async_wait_all();
#pragma unroll
                            for (int i = 0; i < KW; i += 4) {
                                const float4 v = *reinterpret_cast<const float4 *>(myslot + i);
                                win[i] = v.x;
                                win[i + 1] = v.y;
                                win[i + 2] = v.z;
                                win[i + 3] = v.w;
                            }
                        } else {
                            if (pf_key >= 0) cp_async_wait_all();   // a stale copy lands before the slot is reused
                            load_own(s_win, s_ldw, cell * s_slots + slot, valid, qw);
                        }
                        pf_key = -1;
                        qw_loaded = key;
                        if (a.win_buf) {
                            // the next window of this job that differs from this one ...
                            int nk = -1;
                            if (s_slots > 1 && f == 0) {
                                if (j + 1 < op.n_pairs) nk = qw * 16 + j + 1;
                                else if (qw + 1 < op.n_qw) nk = (qw + 1) * 16;
                            } else if (qw + 1 < op.n_qw) {
                                nk = (qw + 1) * 16 + slot;
                            }
                            // ... or the first window of the next job, when it is this tile's
                            if (nk < 0) {
                                Jobs<BATCHED> Jn = J;
                                Jn.advance();
                                if (Jn.live() && Jn.t == t) nk = (s_slots == 1 || Jn.f == 0) ? 0 : s_slots - 1;
                            }
                            want_pf = (nk == key) ? -1 : nk;
                        }
                    }
                    float gj = gf[6];
                    if (f == 0) {
                        gj = gf[0];
#pragma unroll
                        for (int i = 1; i < 6; ++i) gj = (j == i) ? gf[i] : gj;
                    }
#pragma unroll
                    for (int kk = 0; kk < GPB; ++kk) {
                        const int k = sub * GPB + kk;   // granule of the 128-byte row
                        const float *w = win + kk * GE;
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
                        } else if constexpr (PREC == FE_PREC_E4M3) {
                            uint32_t u[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                u[e] = pack_e4m3x2(w[4 * e] * gj, w[4 * e + 1] * gj) |
                                       (pack_e4m3x2(w[4 * e + 2] * gj, w[4 * e + 3] * gj) << 16);
                            v = make_uint4(u[0], u[1], u[2], u[3]);
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
                        if (!live) v = make_uint4(0u, 0u, 0u, 0u);
                        *reinterpret_cast<uint4 *>(rowp + ((k ^ (cl & 7)) << 4)) = v;
                    }
                    if (want_pf >= 0) {   // issued once this block's window registers are consumed
                        issue_pf(s_win, s_ldw, s_slots, cell, valid, want_pf);
                        pf_key = want_pf;
                        want_pf = -1;
                    }
                    if (++blk == op.n_blk) {
                        blk = 0;
                        if (++j == op.n_pairs) {
                            j = 0;
                            ++qw;
                        }
                    }
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.a_full[s]);
                ++ac;
                if (++as == RA) {
                    as = 0;
                    aph ^= 1u;
                }
            }
            ++jb;
        }
        cp_async_wait_all();   // no prefetch may still be landing when the CTA leaves
    } else if (warp == W_MMA) {
        // ======================= MMA =======================
        // Consumes chunk mc from the two rings (stage mc % RA of the built
        // operand, mc % RB of the shared one) and queues its MMAs at once: the
        // completions free the stages asynchronously, so the tensor pipe always
        // holds the next chunk's MMAs while the producers refill.
        int64_t mc = 0;
        int sa = 0, sb = 0;          // stages of chunk mc in the two rings
        uint32_t pa = 0, pb = 0;     // their use parities
        int jb = 0;
        bool fail = false;
        Jobs<BATCHED> J;
        J.start(a, blockIdx.x, gridDim.x);
        for (; J.live() && !fail; J.advance()) {
            const TcOperand op = J.S->op[J.f];
            // a wide pass (N > 256, both TMEM halves as one accumulator) takes two
            // MMAs per K step: columns [0, 256) and [256, NP), B rows likewise
            const bool wide = op.NP > ACC_COLS;
            const uint32_t idesc = a.idesc | ((uint32_t)((wide ? ACC_COLS : op.NP) >> 3) << 17);
            const uint32_t idesc2 = a.idesc | ((uint32_t)((wide ? op.NP - ACC_COLS : 16) >> 3) << 17);
            const int b = jb & acc_mask, ub = jb >> acc_shift;
            if (jb >= NACC && !mbar_wait_warp(&sm.acc_empty[b], (ub - 1) & 1, deadline)) {
                fail = true;
                break;
            }
            tc_fence_after();
            const uint32_t dacc = tmem + (uint32_t)(b * ACC_COLS);
            for (int ch = 0; ch < op.n_kchunks; ++ch) {
                if (!mbar_wait_warp(&sm.a_full[sa], pa, deadline) || !mbar_wait_warp(&sm.b_full[sb], pb, deadline)) {
                    fail = true;
                    break;
                }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t a0 = smem_u32(sm.A + sa * (TC_M * TC_CHUNK_BYTES));
                    const uint32_t b0 = smem_u32(sm.B + (size_t)sb * NPm * TC_CHUNK_BYTES);
#pragma unroll
                    for (int ks = 0; ks < TC_CHUNK_BYTES / 32; ++ks) {
                        const uint64_t ad = sdesc_sw128(a0 + 32 * ks);
                        umma<KIND>(dacc, ad, sdesc_sw128(b0 + 32 * ks), idesc, (ch | ks) != 0 ? 1u : 0u);
                        if (wide)
                            umma<KIND>(dacc + ACC_COLS, ad, sdesc_sw128(b0 + ACC_COLS * TC_CHUNK_BYTES + 32 * ks), idesc2,
                                       (ch | ks) != 0 ? 1u : 0u);
                    }
                    umma_commit(&sm.a_empty[sa]);
                    umma_commit(&sm.b_empty[sb]);
                    if (ch == op.n_kchunks - 1) umma_commit(&sm.acc_full[b]);
                }
                __syncwarp();
                ++mc;
                if (++sa == RA) {
                    sa = 0;
                    pa ^= 1u;
                }
                if (++sb == RB) {
                    sb = 0;
                    pb ^= 1u;
                }
            }
            ++jb;
            if (*abort_flag) fail = true;
        }
        if (fail) sm.flags[0] = 1;
        // drain: every issued MMA finished (a CTA that issued none has nothing
        // to wait for)
        if (mc > 0) {
            if (lane == 0) umma_commit(sm.drain);
            __syncwarp();
            mbar_wait(sm.drain, 0, 200000000ull);   // 0.2 s
        }
    } else if (warp == W_PROD) {
        // ======================= shared-operand producer =======================
        // One 1-D bulk copy per chunk (NP rows of 128 bytes, pre-swizzled) into
        // stage bc % RB, once the MMAs of the chunk that last used the stage are
        // done: up to RB copies in flight hide the L2 latency.
        Jobs<BATCHED> BJ;
        BJ.start(a, blockIdx.x, gridDim.x);
        int64_t bc = 0;
        int bch = 0;
        int s = 0;             // stage of copy bc, and its use parity
        uint32_t ph = 0;
        bool fail = false;
        while (BJ.live() && !*abort_flag) {
            const TcOperand &op = BJ.S->op[BJ.f];
            const uint32_t bytes = (uint32_t)op.NP * TC_CHUNK_BYTES;
            if (bc >= RB && !mbar_wait_warp(&sm.b_empty[s], ph ^ 1u, deadline)) {
                fail = true;
                break;
            }
            if (lane == 0) {
                mbar_arrive_expect_tx(&sm.b_full[s], bytes);
                bulk_g2s(sm.B + (size_t)s * NPm * TC_CHUNK_BYTES, op.img + ((size_t)BJ.n * op.n_kchunks + bch) * bytes,
                         bytes, &sm.b_full[s]);
            }
            __syncwarp();
            ++bc;
            if (++s == RB) {
                s = 0;
                ph ^= 1u;
            }
            if (++bch == op.n_kchunks) {
                bch = 0;
                BJ.advance();
            }
        }
        if (fail) sm.flags[0] = 1;
        // every issued copy has landed before the CTA leaves (the last copy of
        // each stage is the one its current phase waits for)
        const int64_t first = bc > RB ? bc - RB : 0;
        for (int64_t c = first; c < bc; ++c)
            mbar_wait(&sm.b_full[c % RB], (uint32_t)((c / RB) & 1), 200000000ull);
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
        Jobs<BATCHED> J;
        J.start(a, blockIdx.x, gridDim.x);
        for (; J.live() && !stop; J.advance()) {
            const int64_t t = J.t;
            const TcSeg &S = *J.S;
            const int nph = S.n_phi, nph2 = nph * nph;
            const int n_it = (nph2 + 31) / 32;
            // 16-byte stores when every matrix starts on a 16-byte boundary
            const bool v4 = (nph2 & 3) == 0 &&
                            ((reinterpret_cast<uintptr_t>(S.out[0]) | reinterpret_cast<uintptr_t>(S.out[1])) & 15) == 0;
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
            const int f = J.f, n = J.n;
            const TcOperand op = S.op[f];
            float *__restrict__ out = S.out[f];
            const int64_t s_ncells = S.n_cells;
            const int s_staged = S.staged;
            const int32_t *__restrict__ s_symkl = S.sym_kl;
            const int b = jb & acc_mask, ub = jb >> acc_shift;   // accumulator
            const int mb = jb & 1, mub = jb >> 1;                  // unscale buffer
            bool ok = !*abort_flag && mbar_wait_warp(&sm.acc_full[b], ub & 1, deadline) &&
                      mbar_wait_warp(&sm.meta_full[mb], mub & 1, deadline);
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
            const float us = sm.meta[mb * TC_M + g * 32 + lane];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.meta_empty[mb]);
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
            } else if (op.rows_per_pass > 0) {
                // full-row pass not staged (or wide): this cell's rows [k0, k0 + R) are one
                // contiguous run of len values, column c of the pass at offset c; each lane
                // writes its own cell's 32 columns per block, as 16-byte stores where the
                // run starts on a 16-byte boundary
                const int64_t mycell = cell0 + lane;
                const int k0 = n * op.rows_per_pass;
                const int len = (nph - k0 < op.rows_per_pass ? nph - k0 : op.rows_per_pass) * nph;
                float *__restrict__ run = (out && mycell < s_ncells) ? out + mycell * (int64_t)nph2 + (int64_t)k0 * nph : nullptr;
                const bool v4r = (nph & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
                for (int c0 = 32 * h; c0 < op.NP; c0 += 64) {
                    uint32_t r[32];
                    tmem_ld32(tbase + (uint32_t)c0, r);
                    if (!run) continue;
                    if (v4r && c0 + 32 <= len) {
#pragma unroll
                        for (int i = 0; i < 32; i += 4)
                            __stcs(reinterpret_cast<float4 *>(run + c0 + i),
                                   make_float4(__uint_as_float(r[i]) * us, __uint_as_float(r[i + 1]) * us,
                                               __uint_as_float(r[i + 2]) * us, __uint_as_float(r[i + 3]) * us));
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (c0 + i < len) __stcs(run + c0 + i, __uint_as_float(r[i]) * us);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.acc_empty[b]);
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
    b += bytes_A(a) + bytes_B(a) + bytes_stage(a) + bytes_wnext(a);
    b += 2 * TC_M * sizeof(float);
    b += 8;
    b += (2 * TC_MAX_RING_A + 2 * TC_MAX_RING_B + 9) * sizeof(uint64_t) + 8 + 16;
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
            if (seg.op[f].NP > ACC_COLS) return false;   // a wide pass leaves from registers
            np = seg.op[f].NP > np ? seg.op[f].NP : np;
        }
    if (pairs && seg.n_phi * seg.n_phi > 32 * MAX_F2S_IT) return false;
    TcArgs t = a;
    t.pitch_max = (np + 1) > a.pitch_max ? (np + 1) : a.pitch_max;
    t.ring_a = t.ring_b = 2;   // staging is decided at the shallowest rings; deeper rings take what is left
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
    if (grid > a.n_jobs) grid = (int)a.n_jobs;
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
