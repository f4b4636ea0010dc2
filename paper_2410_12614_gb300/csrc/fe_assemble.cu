// Global assembly A^g = L D L^T (Sec. 3.3) as a deterministic segmented
// reduction.
//
// The element entries (c, k, l) sorted by their CSR slot form one segment per
// CSR value; inside a segment they are in increasing cell order.  The plan
// stores, per CSR row i, its incidences (c, k) with dof(c, k) = i sorted by
// cell (inc_ptr / inc_elem), and per CSR value the length of its segment
// (contrib_cnt, at most m_K of Corollary 4.11) and its entries as
// (incidence index, local column l) codes (contrib_code).  One warp owns one
// row; each lane owns one CSR value, sums its segment in order starting from
// zero and writes it: every value is bitwise reproducible.  Accumulation is
// in the element precision (FP32 for the reduced-precision paths, FP64 for
// the FP64 path), as in the u_q of Corollary 4.11.
#include "fe_device.cuh"

namespace fe {

namespace {

// Segment of a global row (binary search over the segments' first rows).
// The single-plan instantiation addresses the kernel parameter directly.
template <bool BATCHED>
__device__ __forceinline__ const AsmSeg &aseg_of(const AsmArgs &a, int64_t row) {
    if (!BATCHED) return a.seg0;
    int lo = 0, hi = a.n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].row_begin <= row) lo = mid; else hi = mid - 1;
    }
    return a.segs[lo];
}

template <typename T, int NF, bool BATCHED>
__global__ void __launch_bounds__(256) assemble_kernel(const __grid_constant__ AsmArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t total_warps = (int64_t)gridDim.x * a.warps_per_block;
    for (int64_t grow = (int64_t)blockIdx.x * a.warps_per_block + warp; grow < a.n_rows; grow += total_warps) {
        const AsmSeg &S = aseg_of<BATCHED>(a, grow);
        const int64_t row = grow - S.row_begin;
        const T *__restrict__ A0 = static_cast<const T *>(S.A[0]);
        const T *__restrict__ A1 = static_cast<const T *>(S.A[NF > 1 ? 1 : 0]);
        T *__restrict__ O0 = static_cast<T *>(S.out[0]);
        T *__restrict__ O1 = static_cast<T *>(S.out[NF > 1 ? 1 : 0]);
        const uint32_t nph = (uint32_t)S.n_phi;
        // the segment's fields, read once per row into registers
        const int32_t *__restrict__ inc_elem = S.inc_elem;
        const uint8_t *__restrict__ contrib_cnt = S.contrib_cnt;
        const uint16_t *__restrict__ contrib_code = S.contrib_code;
        const int64_t r0 = __ldg(S.row_ptr + row);
        const int len = (int)(__ldg(S.row_ptr + row + 1) - r0);
        const int64_t i0 = __ldg(S.inc_ptr + row);
        const int ninc = (int)(__ldg(S.inc_ptr + row + 1) - i0);
        const int myelem = (lane < ninc) ? __ldg(inc_elem + i0 + lane) : 0;
        int64_t off = __ldg(S.contrib_base + row);
        for (int j0 = 0; j0 < len; j0 += 32) {
            const int j = j0 + lane;
            const int cnt = (j < len) ? (int)__ldg(contrib_cnt + r0 + j) : 0;
            // exclusive scan and maximum of the counts over the warp
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
                const bool v = k < cnt;
                const uint32_t code = v ? (uint32_t)__ldg(contrib_code + start + k) : 0u;
                const int t = (int)(code & 0xFFu);
                int el = __shfl_sync(0xffffffffu, myelem, t & 31);
                if (t >= 32) el = __ldg(inc_elem + i0 + t);
                if (v) {
                    const uint32_t e = (uint32_t)el * nph + (code >> 8);
                    s0 += __ldg(A0 + e);
                    if (NF > 1) s1 += __ldg(A1 + e);
                }
            }
            if (j < len) {
                O0[r0 + j] = s0;
                if (NF > 1) O1[r0 + j] = s1;
            }
            off += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

template <typename T>
int launch_t(const AsmArgs &a0, cudaStream_t s, int wpb) {
    AsmArgs a = a0;
    a.warps_per_block = wpb;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (a.n_rows + wpb - 1) / wpb;
    const int64_t cap = (int64_t)sms * (2048 / (32 * wpb)) * 4;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const bool batched = a.segs != nullptr;
    if (a.n_forms == 2) {
        if (batched) assemble_kernel<T, 2, true><<<(unsigned)blocks, wpb * 32, 0, s>>>(a);
        else assemble_kernel<T, 2, false><<<(unsigned)blocks, wpb * 32, 0, s>>>(a);
    } else {
        if (batched) assemble_kernel<T, 1, true><<<(unsigned)blocks, wpb * 32, 0, s>>>(a);
        else assemble_kernel<T, 1, false><<<(unsigned)blocks, wpb * 32, 0, s>>>(a);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return -(int)e;
    return 1;
}

}  // namespace

int launch_assemble(const AsmArgs &a, bool fp64, cudaStream_t s, int warps_per_block) {
    if (a.n_rows <= 0) return 0;
    if (warps_per_block < 1 || warps_per_block > 8) warps_per_block = 8;
    return fp64 ? launch_t<double>(a, s, warps_per_block) : launch_t<float>(a, s, warps_per_block);
}

}  // namespace fe
