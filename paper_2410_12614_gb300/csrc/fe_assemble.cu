// Global assembly A^g = L D L^T (Sec. 3.3) as a deterministic segmented
// reduction.
//
// The element entries (c, k, l) are grouped by their CSR slot: each CSR row
// i is one segment of incidences (c, k) with dof(c, k) = i, sorted by cell
// (the plan's inc_ptr / inc_elem streams), and inside an incidence the
// destination column of entry l is the plan's precomputed slot
// inc_slot[(c,k), l].  One warp owns one row: it clears the row's
// accumulators in shared memory, adds the incidences one after another
// (a whole element row A[c][k][:] per step, coalesced; the slots of one
// incidence are distinct, so lanes never collide), and writes the row out.
// Every CSR value is therefore the sum of its element entries in increasing
// cell order starting from zero: bitwise reproducible.  Accumulation is in
// the element precision (FP32 for the reduced-precision paths, FP64 for the
// FP64 path; Corollary 4.11 charges m_K u_q for it).
#include "fe_device.cuh"

namespace fe {

namespace {

template <typename T, int NF>
__global__ void __launch_bounds__(256) assemble_kernel(const __grid_constant__ AsmArgs a) {
    extern __shared__ __align__(16) uint8_t smraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int stride_row = a.max_row;
    T *acc0 = reinterpret_cast<T *>(smraw) + (size_t)warp * NF * stride_row;
    T *acc1 = acc0 + (NF > 1 ? stride_row : 0);
    const T *__restrict__ A0 = static_cast<const T *>(a.A[0]);
    const T *__restrict__ A1 = static_cast<const T *>(a.A[NF > 1 ? 1 : 0]);
    T *O0 = static_cast<T *>(a.out[0]);
    T *O1 = static_cast<T *>(a.out[NF > 1 ? 1 : 0]);
    const int nph = a.n_phi;
    const int64_t total_warps = (int64_t)gridDim.x * a.warps_per_block;
    for (int64_t row = (int64_t)blockIdx.x * a.warps_per_block + warp; row < a.n_rows; row += total_warps) {
        const int64_t r0 = __ldg(a.row_ptr + row);
        const int len = (int)(__ldg(a.row_ptr + row + 1) - r0);
        const int64_t i0 = __ldg(a.inc_ptr + row);
        const int ninc = (int)(__ldg(a.inc_ptr + row + 1) - i0);
        for (int j = lane; j < len; j += 32) {
            acc0[j] = T(0);
            if (NF > 1) acc1[j] = T(0);
        }
        const uint16_t *__restrict__ slots = a.inc_slot + i0 * nph;
        for (int base = 0; base < ninc; base += 32) {
            // the element-row ids of up to 32 incidences, broadcast one by one below
            const int myelem = (base + lane < ninc) ? __ldg(a.inc_elem + i0 + base + lane) : 0;
            const int cnt = (ninc - base) < 32 ? (ninc - base) : 32;
            __syncwarp();
            if (nph <= 32) {
                // one element-row entry per lane; the next incidence's loads are
                // issued before the current one is accumulated
                const bool act = lane < nph;
                int e = __shfl_sync(0xffffffffu, myelem, 0);
                uint32_t off = (uint32_t)e * (uint32_t)nph + (uint32_t)lane;
                int sl = act ? __ldg(slots + (size_t)base * nph + lane) : 0;
                T v0 = act ? __ldg(A0 + off) : T(0);
                T v1 = (NF > 1 && act) ? __ldg(A1 + off) : T(0);
                for (int t = 0; t < cnt; ++t) {
                    int sl_n = 0;
                    T v0_n = T(0), v1_n = T(0);
                    if (t + 1 < cnt) {
                        const int en = __shfl_sync(0xffffffffu, myelem, t + 1);
                        const uint32_t offn = (uint32_t)en * (uint32_t)nph + (uint32_t)lane;
                        if (act) {
                            sl_n = __ldg(slots + (size_t)(base + t + 1) * nph + lane);
                            v0_n = __ldg(A0 + offn);
                            if (NF > 1) v1_n = __ldg(A1 + offn);
                        }
                    }
                    if (act) {
                        acc0[sl] += v0;
                        if (NF > 1) acc1[sl] += v1;
                    }
                    __syncwarp();
                    sl = sl_n;
                    v0 = v0_n;
                    v1 = v1_n;
                }
            } else {
                for (int t = 0; t < cnt; ++t) {
                    const int e = __shfl_sync(0xffffffffu, myelem, t);
                    const T *r0p = A0 + (size_t)e * nph;
                    const T *r1p = A1 + (size_t)e * nph;
                    const uint16_t *sp = slots + (size_t)(base + t) * nph;
                    for (int l = lane; l < nph; l += 32) {
                        const int sl = __ldg(sp + l);
                        acc0[sl] += __ldg(r0p + l);
                        if (NF > 1) acc1[sl] += __ldg(r1p + l);
                    }
                    __syncwarp();
                }
            }
        }
        __syncwarp();
        for (int j = lane; j < len; j += 32) {
            O0[r0 + j] = acc0[j];
            if (NF > 1) O1[r0 + j] = acc1[j];
        }
        __syncwarp();
    }
}

template <typename T>
int launch_t(const AsmArgs &a0, cudaStream_t s) {
    AsmArgs a = a0;
    const size_t per_warp = sizeof(T) * (size_t)a.n_forms * a.max_row;
    int wpb = 8;
    while (wpb > 1 && per_warp * wpb > 96 * 1024) wpb /= 2;
    if (per_warp * wpb > 200 * 1024) return -(int)cudaErrorInvalidValue;
    a.warps_per_block = wpb;
    const size_t smem = per_warp * wpb;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (a.n_rows + wpb - 1) / wpb;
    const int64_t cap = (int64_t)sms * (64 / wpb) * 4;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    cudaError_t e;
    if (a.n_forms == 2) {
        e = cudaFuncSetAttribute(assemble_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return -(int)e;
        assemble_kernel<T, 2><<<(unsigned)blocks, wpb * 32, smem, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(assemble_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return -(int)e;
        assemble_kernel<T, 1><<<(unsigned)blocks, wpb * 32, smem, s>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return -(int)e;
    return 1;
}

}  // namespace

int launch_assemble(const AsmArgs &a, bool fp64, cudaStream_t s) {
    if (a.n_rows <= 0) return 0;
    return fp64 ? launch_t<double>(a, s) : launch_t<float>(a, s);
}

}  // namespace fe
