// batched.cu -- many independent small systems in one persistent launch.
//
// Each block pulls system indices from a device work counter and reduces
// that system with the paper's column-by-column Gauss-Jordan loop (section
// 3.2): lowest nonzero pivot at or below the current rank, row swap, scaling
// of the pivot row by the inverse of its head, elimination of the pivot
// column from every other row.  Systems are independent, so there is no
// inter-block communication at all.
#include <algorithm>
#include <climits>

#include "linac_host.h"
#include "profile.h"

namespace linac {

constexpr int BATCH_THREADS = 256;

__global__ void __launch_bounds__(BATCH_THREADS)
batched_gj_kernel(uint32_t* __restrict__ data, const int64_t* __restrict__ offsets,
                  const int32_t* __restrict__ dm, const int32_t* __restrict__ dn,
                  const int32_t* __restrict__ dld, const int32_t* __restrict__ dns, int batch, Field f,
                  int32_t* __restrict__ ranks, int32_t* __restrict__ pivots,
                  const int64_t* __restrict__ piv_off, int32_t* __restrict__ sys_status,
                  unsigned int* __restrict__ counter) {
    __shared__ int s_sys, s_q;
    __shared__ int s_red[BATCH_THREADS / 32];
    __shared__ uint32_t s_hinv;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = BATCH_THREADS / 32;
    for (;;) {
        if (tid == 0) s_sys = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int s = s_sys;
        __syncthreads();
        if (s >= batch) return;
        const int m = dm[s], n = dn[s];
        const int64_t ld = dld[s];
        const int ns = dns ? min(dns[s], n) : n;
        uint32_t* A = data + offsets[s];
        int32_t* piv = pivots + piv_off[s];
        const int npiv = min(m, ns);
        for (int i = tid; i < npiv; i += BATCH_THREADS) piv[i] = -1;
        int r = 0;
        for (int c = 0; c < ns && r < m; ++c) {
            int ci = INT_MAX;
            for (int q = r + tid; q < m; q += BATCH_THREADS)
                if (A[(int64_t)q * ld + c] != 0) { ci = q; break; }
            for (int o = 16; o; o >>= 1) ci = min(ci, __shfl_xor_sync(0xffffffffu, ci, o));
            if (lane == 0) s_red[warp] = ci;
            __syncthreads();
            if (warp == 0) {
                int v = lane < nwarps ? s_red[lane] : INT_MAX;
                for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
                if (lane == 0) {
                    s_q = v;
                    if (v != INT_MAX) s_hinv = inverse_mod(A[(int64_t)v * ld + c], f.p);
                }
            }
            __syncthreads();
            const int q = s_q;
            if (q == INT_MAX) continue;
            uint32_t* prow = A + (int64_t)r * ld;
            const uint32_t hinv = s_hinv;
            if (q != r) {
                uint32_t* qrow = A + (int64_t)q * ld;
                for (int j = c + tid; j < n; j += BATCH_THREADS) {
                    const uint32_t t = qrow[j];
                    qrow[j] = prow[j];
                    prow[j] = mulmod(t, hinv, f);
                }
            } else {
                for (int j = c + tid; j < n; j += BATCH_THREADS) prow[j] = mulmod(prow[j], hinv, f);
            }
            __syncthreads();
            for (int i = warp; i < m; i += nwarps) {
                if (i == r) continue;
                uint32_t* row = A + (int64_t)i * ld;
                const uint32_t fi = row[c];
                __syncwarp();
                if (fi == 0) continue;
                const uint64_t nf = f.p - fi;
                for (int j = c + lane; j < n; j += 32) row[j] = reduce64((uint64_t)row[j] + nf * prow[j], f);
            }
            __syncthreads();
            if (tid == 0) piv[r] = c;
            ++r;
        }
        if (tid == 0) {
            ranks[s] = r;
            if (sys_status) sys_status[s] = 0;
        }
        __syncthreads();
    }
}

linac_status batched_rref(uint32_t* d_data, const int64_t* d_offsets, const int32_t* d_m,
                          const int32_t* d_n, const int32_t* d_ld, const int32_t* d_nsearch,
                          int32_t batch, int32_t max_m, int32_t max_n, const Field& f, uint32_t flags,
                          int32_t* d_ranks, int32_t* d_pivots, const int64_t* d_piv_offsets,
                          int32_t* d_status, cudaStream_t stream) {
    (void)max_m;
    (void)max_n;
    (void)flags;
    void* buf = nullptr;
    linac_status s = scratch_get_slot(stream, 2, 256, &buf);
    if (s != LINAC_OK) return s;
    unsigned int* counter = (unsigned int*)buf;
    LINAC_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned int), stream));
    const int grid = std::max(1, std::min(batch, sm_count() * 8));
    ProfScope ps(stream, PROF_BATCHED);
    batched_gj_kernel<<<grid, BATCH_THREADS, 0, stream>>>(d_data, d_offsets, d_m, d_n, d_ld, d_nsearch, batch, f,
                                                          d_ranks, d_pivots, d_piv_offsets, d_status, counter);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

}  // namespace linac
