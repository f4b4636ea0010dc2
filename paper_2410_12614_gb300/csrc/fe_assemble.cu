// Global assembly A^g = L D L^T (Sec. 3.3) as a deterministic segmented
// reduction.
//
// The element entries (c, k, l) sorted by their CSR slot form one segment per
// CSR value; inside a segment they are in increasing cell order.  The plan
// stores, per CSR row i, its incidences (c, k) with dof(c, k) = i sorted by
// cell (inc_ptr / inc_elem), and per CSR value the length of its segment
// (contrib_cnt, at most m_K of Corollary 4.11) and its entries as
// (incidence index, local column l) codes (contrib_code).  Rows are grouped
// into chunks of consecutive rows with at most ASM_CHUNK entries and
// ASM_CHUNK_INC incidences, whose codes, incidences, counts and CSR values are
// contiguous ranges of those streams.  One CTA owns one chunk:
//   1. it loads the chunk's incidences and counts into shared memory and the
//      stage positions of its entries into registers (one round trip, every
//      load independent);
//   2. each thread gathers its ~16 element entries in incidence order -- so
//      that a warp reads whole element rows, contiguous in memory -- straight
//      into their positions in the shared stage with asynchronous 4- or
//      8-byte copies (no registers held);
//   3. a block-wide scan of the counts gives each CSR value's segment in the
//      stage; one thread per value sums it in order, starting from zero, and
//      the values leave in coalesced stores.
// Chunks are taken from the last one down (the element matrices written last
// by the element kernel are still in L2).  A row with more than ASM_CHUNK
// entries is a chunk of its own and is summed by one warp straight from global
// memory in the same order.  Every value is
// bitwise reproducible and independent of the launch shape.  Accumulation is
// in the element precision (FP32 for the reduced-precision paths, FP64 for
// the FP64 path), as in the u_q of Corollary 4.11.
#include "fe_device.cuh"

namespace fe {

namespace {

constexpr int ASM_THREADS = 256;
constexpr int ASM_PER = ASM_CHUNK / ASM_THREADS;   // element entries per thread

// Segment of a global chunk (binary search over the segments' first chunks).
// The single-plan instantiation addresses the kernel parameter directly.
template <bool BATCHED>
__device__ __forceinline__ const AsmSeg &aseg_of(const AsmArgs &a, int64_t chunk) {
    if (!BATCHED) return a.seg0;
    int lo = 0, hi = a.n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].chunk_begin <= chunk) lo = mid; else hi = mid - 1;
    }
    return a.segs[lo];
}

// Incidence id c * n_phi + k of the element row, moved into the ring of
// element matrices of the fused assembly (identity without a ring).
__device__ __forceinline__ uint32_t ring_inc(const AsmSeg &S, uint32_t inc, uint32_t nph) {
    if (S.ring_slots == 0) return inc;
    const int64_t c = inc / nph;
    const int64_t sl = c / S.ring_cells;
    return (uint32_t)((int64_t)inc + ((sl % S.ring_slots) - sl) * S.ring_cells * (int64_t)nph);
}

// One row with more entries than a chunk holds, summed by one warp from
// global memory: lane j of each 32-value group owns CSR value j and walks its
// segment in order.  e0 is the chunk's first incidence.
template <typename T, int NF>
__device__ void big_row(const AsmSeg &S, const T *__restrict__ A0, const T *__restrict__ A1, T *__restrict__ O0,
                        T *__restrict__ O1, int64_t v0, int len, int64_t e0, int64_t c0, int lane) {
    const uint32_t nph = (uint32_t)S.n_phi;
    int64_t off = c0;
    for (int j0 = 0; j0 < len; j0 += 32) {
        const int j = j0 + lane;
        const int cnt = (j < len) ? (int)__ldg(S.contrib_cnt + v0 + j) : 0;
        int incl = cnt, mx = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        const int64_t start = off + (incl - cnt);
        T s0 = T(0), s1 = T(0);
        for (int k = 0; k < mx; ++k) {
            if (k < cnt) {
                const uint32_t code = __ldg(S.contrib_code + start + k);
                const uint32_t e = ring_inc(S, (uint32_t)__ldg(S.inc_elem + e0 + (code & 0xFFu)), nph) * nph + (code >> 8);
                s0 += __ldg(A0 + e);
                if (NF > 1) s1 += __ldg(A1 + e);
            }
        }
        if (j < len) {
            O0[v0 + j] = s0;
            if (NF > 1) O1[v0 + j] = s1;
        }
        off += __shfl_sync(0xffffffffu, incl, 31);
    }
}

template <typename T, int NF, bool BATCHED>
__global__ void __launch_bounds__(ASM_THREADS) assemble_kernel(const __grid_constant__ AsmArgs a) {
    extern __shared__ __align__(16) unsigned char asm_smem[];
    T *st0 = reinterpret_cast<T *>(asm_smem);                                 // [NF][ASM_CHUNK] gathered entries
    T *st1 = st0 + (NF > 1 ? ASM_CHUNK : 0);
    int32_t *inc_s = reinterpret_cast<int32_t *>(st0 + NF * ASM_CHUNK);     // [ASM_CHUNK_INC]
    uint16_t *start_s = reinterpret_cast<uint16_t *>(inc_s + ASM_CHUNK_INC);  // [ASM_CHUNK] segment starts
    uint8_t *cnt_s = reinterpret_cast<uint8_t *>(start_s + ASM_CHUNK);        // [ASM_CHUNK] segment lengths
    __shared__ int warp_tot[ASM_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // chunks from the last row down: the element kernel that ran just before
    // wrote the highest cells last, so their element matrices are the ones
    // still in L2 and are read first
    const int64_t n_work = a.chunk_list ? a.list_count : a.n_chunks;
    for (int64_t gi = blockIdx.x; gi < n_work; gi += gridDim.x) {
        const int64_t g = a.chunk_list ? (int64_t)__ldg(a.chunk_list + (n_work - 1 - gi)) : a.n_chunks - 1 - gi;
        const AsmSeg &S = aseg_of<BATCHED>(a, g);
        const int64_t ch = g - S.chunk_begin;
        const T *__restrict__ A0 = static_cast<const T *>(S.A[0]);
        const T *__restrict__ A1 = static_cast<const T *>(S.A[NF > 1 ? 1 : 0]);
        T *__restrict__ O0 = static_cast<T *>(S.out[0]);
        T *__restrict__ O1 = static_cast<T *>(S.out[NF > 1 ? 1 : 0]);
        const uint32_t nph = (uint32_t)S.n_phi;
        const int64_t *__restrict__ dsc = S.chunk_desc + ch * 4;
        const int64_t ra = __ldg(dsc + 0), c0 = __ldg(dsc + 1), e0 = __ldg(dsc + 2), v0 = __ldg(dsc + 3);
        const int64_t rb = __ldg(dsc + 4);
        const int64_t nc = __ldg(dsc + 5) - c0;
        const int ne = (int)(__ldg(dsc + 6) - e0);
        const int nv = (int)(__ldg(dsc + 7) - v0);
        if (nc > ASM_CHUNK || nv > ASM_CHUNK || ne > ASM_CHUNK_INC) {
            // (only a single row above the entry limit comes here)
            if (warp == 0)
                for (int64_t r = ra; r < rb; ++r) {
                    const int64_t rv0 = __ldg(S.row_ptr + r);
                    big_row<T, NF>(S, A0, A1, O0, O1, rv0, (int)(__ldg(S.row_ptr + r + 1) - rv0), e0,
                                   __ldg(S.contrib_base + r), lane);
                }
            continue;
        }
        // 1. stage positions to registers; incidences and counts to shared memory
        const uint16_t *__restrict__ dest = S.contrib_dest + c0;
        uint32_t dpos[ASM_PER];
#pragma unroll
        for (int u = 0; u < ASM_PER; ++u) {
            const int q = u * ASM_THREADS + tid;
            dpos[u] = (q < nc) ? (uint32_t)__ldg(dest + q) : 0u;
        }
        for (int i = tid; i < ne; i += ASM_THREADS) inc_s[i] = (int32_t)ring_inc(S, (uint32_t)__ldg(S.inc_elem + e0 + i), nph);
        for (int i = tid; i < nv; i += ASM_THREADS) cnt_s[i] = __ldg(S.contrib_cnt + v0 + i);
        __syncthreads();
        // 2. gather in incidence order (each element row read as one contiguous
        //    run) into the stage at the entries' positions in code order
        {
            uint32_t t = (uint32_t)tid / nph, l = (uint32_t)tid - t * nph;
            const uint32_t dt = ASM_THREADS / nph, dl = ASM_THREADS - dt * nph;
#pragma unroll
            for (int u = 0; u < ASM_PER; ++u) {
                const int q = u * ASM_THREADS + tid;
                if (q < nc) {
                    const uint32_t e = (uint32_t)inc_s[t] * nph + l;
                    cp_async_small<sizeof(T)>(st0 + dpos[u], A0 + e);
                    if (NF > 1) cp_async_small<sizeof(T)>(st1 + dpos[u], A1 + e);
                }
                t += dt;
                l += dl;
                if (l >= nph) {
                    l -= nph;
                    ++t;
                }
            }
        }
        // 3a. exclusive scan of the counts (thread tid owns values [vb, ve))
        const int vpt = (nv + ASM_THREADS - 1) / ASM_THREADS;
        const int vb = min(nv, tid * vpt), ve = min(nv, vb + vpt);
        int loc = 0;
        for (int v = vb; v < ve; ++v) loc += cnt_s[v];
        int incl = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        int run = incl - loc;
        for (int w = 0; w < warp; ++w) run += warp_tot[w];
        for (int v = vb; v < ve; ++v) {
            start_s[v] = (uint16_t)run;
            run += cnt_s[v];
        }
        cp_async_wait_all();
        __syncthreads();
        // 3b. one thread per CSR value sums its segment in order
        for (int v = tid; v < nv; v += ASM_THREADS) {
            const int cnt = cnt_s[v], s = start_s[v];
            T s0 = T(0), s1 = T(0);
            for (int k = 0; k < cnt; ++k) {
                s0 += st0[s + k];
                if (NF > 1) s1 += st1[s + k];
            }
            O0[v0 + v] = s0;
            if (NF > 1) O1[v0 + v] = s1;
        }
        __syncthreads();   // the next chunk reuses the shared arrays
    }
}

// ---------------------------------------------------------------------------
// One warp per CSR row.  Row i's incidences (c, k) -- the element rows whose
// dof is i -- are walked in increasing cell order; each adds its n_phi
// entries A[c][k][l] into the row's accumulators at their column slots
// (distinct within one incidence), so every CSR value is again the sum of its
// entries in increasing cell order from zero: bitwise the chunked kernel's
// result.  The accumulators live in shared memory (rows up to ASM_ROW_CAP
// values) or, for longer rows, in the output itself.  Element rows are read
// coalesced (lanes over l, 32 columns per item, items incidence-major),
// ROW_U items ahead.
// ---------------------------------------------------------------------------
constexpr int ROW_WARPS = 8;
constexpr int ROW_U = 4;

template <bool BATCHED>
__device__ __forceinline__ const AsmSeg &rseg_of(const AsmArgs &a, int64_t row) {
    if (!BATCHED) return a.seg0;
    int lo = 0, hi = a.n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].row_begin <= row) lo = mid; else hi = mid - 1;
    }
    return a.segs[lo];
}

template <typename T, int NF, bool BATCHED>
__global__ void __launch_bounds__(ROW_WARPS * 32) assemble_rows_kernel(const __grid_constant__ AsmArgs a) {
    extern __shared__ __align__(16) unsigned char row_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *accw = reinterpret_cast<T *>(row_smem) + (size_t)warp * NF * ASM_ROW_CAP;
    const int64_t n_work = a.row_list ? a.row_count : a.n_rows;
    for (int64_t gw = (int64_t)blockIdx.x * ROW_WARPS + warp; gw < n_work; gw += (int64_t)gridDim.x * ROW_WARPS) {
        const int64_t g = a.row_list ? (int64_t)__ldg(a.row_list + gw) : gw;
        const AsmSeg &S = rseg_of<BATCHED>(a, g);
        const int64_t r = g - S.row_begin;
        const uint32_t nph = (uint32_t)S.n_phi;
        const T *__restrict__ A0 = static_cast<const T *>(S.A[0]);
        const T *__restrict__ A1 = static_cast<const T *>(S.A[NF > 1 ? 1 : 0]);
        T *__restrict__ O0 = static_cast<T *>(S.out[0]);
        T *__restrict__ O1 = static_cast<T *>(S.out[NF > 1 ? 1 : 0]);
        const int64_t v0 = __ldg(S.row_ptr + r);
        const int len = (int)(__ldg(S.row_ptr + r + 1) - v0);
        const int64_t i0 = __ldg(S.inc_ptr + r);
        const int ninc = (int)(__ldg(S.inc_ptr + r + 1) - i0);
        const bool shared = len <= ASM_ROW_CAP;
        T *acc0 = shared ? accw : O0 + v0;
        T *acc1 = shared ? accw + ASM_ROW_CAP : O1 + v0;
        for (int j = lane; j < len; j += 32) {
            acc0[j] = T(0);
            if (NF > 1) acc1[j] = T(0);
        }
        __syncwarp();
        // items (incidence t, block of 32 local columns), t-major: a slot takes
        // at most one entry per incidence, so adding the items in this order
        // keeps every slot's entries in increasing cell order
        const int nch = (int)((nph + 31) >> 5);
        const int n_items = ninc * nch;
        for (int i0b = 0; i0b < n_items; i0b += ROW_U) {
            T x0[ROW_U], x1[ROW_U];
            int sl[ROW_U];
#pragma unroll
            for (int u = 0; u < ROW_U; ++u) {
                const int item = i0b + u;
                const int t = item / nch;
                const uint32_t l = (uint32_t)(item - t * nch) * 32u + (uint32_t)lane;
                sl[u] = -1;
                if (item < n_items && l < nph) {
                    const uint32_t inc = ring_inc(S, (uint32_t)__ldg(S.inc_elem + i0 + t), nph);
                    const size_t e = (size_t)inc * nph + l;
                    x0[u] = __ldg(A0 + e);
                    if (NF > 1) x1[u] = __ldg(A1 + e);
                    sl[u] = (int)__ldg(S.inc_slot + (size_t)(i0 + t) * nph + l);
                }
            }
#pragma unroll
            for (int u = 0; u < ROW_U; ++u) {
                if (sl[u] >= 0) {
                    acc0[sl[u]] += x0[u];
                    if (NF > 1) acc1[sl[u]] += x1[u];
                }
                __syncwarp();   // item u's additions land before item u+1's
            }
        }
        if (shared) {
            for (int j = lane; j < len; j += 32) {
                O0[v0 + j] = acc0[j];
                if (NF > 1) O1[v0 + j] = acc1[j];
            }
        }
        __syncwarp();   // the accumulators are reused by the warp's next row
    }
}

template <typename T>
int launch_rows_t(const AsmArgs &a, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (size_t)ROW_WARPS * a.n_forms * ASM_ROW_CAP * sizeof(T);
    const int64_t n_work = a.row_list ? a.row_count : a.n_rows;
    int64_t blocks = (n_work + ROW_WARPS - 1) / ROW_WARPS;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const bool batched = a.segs != nullptr;
    auto go = [&](auto kernel) -> cudaError_t {
        const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kernel<<<(unsigned)blocks, ROW_WARPS * 32, smem, s>>>(a);
        return cudaGetLastError();
    };
    cudaError_t e;
    if (a.n_forms == 2)
        e = batched ? go(assemble_rows_kernel<T, 2, true>) : go(assemble_rows_kernel<T, 2, false>);
    else
        e = batched ? go(assemble_rows_kernel<T, 1, true>) : go(assemble_rows_kernel<T, 1, false>);
    return e == cudaSuccess ? 1 : -(int)e;
}

template <typename T>
int launch_t(const AsmArgs &a, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (size_t)a.n_forms * ASM_CHUNK * sizeof(T) + ASM_CHUNK_INC * sizeof(int32_t) +
                        ASM_CHUNK * (sizeof(uint16_t) + sizeof(uint8_t));
    int64_t blocks = a.chunk_list ? a.list_count : a.n_chunks;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const bool batched = a.segs != nullptr;
    auto go = [&](auto kernel) -> cudaError_t {
        const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kernel<<<(unsigned)blocks, ASM_THREADS, smem, s>>>(a);
        return cudaGetLastError();
    };
    cudaError_t e;
    if (a.n_forms == 2)
        e = batched ? go(assemble_kernel<T, 2, true>) : go(assemble_kernel<T, 2, false>);
    else
        e = batched ? go(assemble_kernel<T, 1, true>) : go(assemble_kernel<T, 1, false>);
    if (e != cudaSuccess) return -(int)e;
    return 1;
}

}  // namespace

int launch_assemble(const AsmArgs &a, bool fp64, cudaStream_t s) {
    if (a.algo == 1) {
        if (a.n_rows <= 0 || (a.row_list && a.row_count <= 0)) return 0;
        return fp64 ? launch_rows_t<double>(a, s) : launch_rows_t<float>(a, s);
    }
    if (a.n_chunks <= 0 || (a.chunk_list && a.list_count <= 0)) return 0;
    return fp64 ? launch_t<double>(a, s) : launch_t<float>(a, s);
}

}  // namespace fe
