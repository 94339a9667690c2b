// host_io.cu -- linac_rref_host: the in-place RREF of a matrix that lives in
// page-locked HOST memory, with the transfers inside the call.
//
// The matrix is copied into library scratch on the device, reduced there by
// the dense driver (dense.cu), and copied back, all ordered on the caller's
// stream with no host synchronisation.  The copies are made by the SMs, not
// by the copy engines: a grid-stride kernel reads (or writes) the host rows
// through their device mapping in 16-byte words.  On GB300 the copy engines'
// host-to-device rate was measured to fall from 211 GB/s to 25-60 GB/s after
// any sustained GPU work (a 4.3 GB copy took 75-170 ms instead of 20.5 ms),
// while the SM-driven copy kept 211 GB/s in every state; the device-to-host
// direction was unaffected either way.
#include <algorithm>

#include "linac_host.h"
#include "profile.h"

namespace linac {

namespace {

// dst[i] = src[i] for n16 16-byte words; either side may be mapped host memory.
__global__ void __launch_bounds__(512)
hostio_copy_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n16) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Rank and pivots from device scratch to their (mapped) host outputs.
__global__ void hostio_results_kernel(const int32_t* __restrict__ d_rank, const int32_t* __restrict__ d_piv,
                                      int64_t npiv, int32_t* __restrict__ h_rank, int32_t* __restrict__ h_piv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npiv; i += (int64_t)gridDim.x * blockDim.x)
        h_piv[i] = d_piv[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) *h_rank = *d_rank;
}

// Device address of page-locked host memory (registered or allocated by
// cudaHostAlloc); nullptr for any other pointer.
void* mapped(void* h) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost) return nullptr;
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return d;
}

linac_status copy_words(const void* src, void* dst, size_t bytes, cudaStream_t stream) {
    if (bytes == 0) return LINAC_OK;
    const size_t n16 = bytes / 16;
    const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>((n16 + 511) / 512, (size_t)sm_count() * 8));
    ProfScope ps(stream, PROF_HOST_COPY);
    hostio_copy_kernel<<<blocks, 512, 0, stream>>>((const uint4*)src, (uint4*)dst, n16);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

}  // namespace

}  // namespace linac

using namespace linac;

extern "C" linac_status linac_rref_host(uint32_t* h_A, int64_t m, int64_t n, int64_t ld, uint32_t p,
                                        int32_t* h_rank, int32_t* h_pivots, cudaStream_t stream) {
    if (m < 0 || n < 0 || ld < n || m > INT32_MAX || n > INT32_MAX) return LINAC_ERR_ARG;
    if (!h_rank || (m > 0 && n > 0 && !h_A) || (std::min(m, n) > 0 && !h_pivots)) return LINAC_ERR_ARG;
    if (ld % 4 != 0 || ((uintptr_t)h_A % 16) != 0) return LINAC_ERR_ALIGN;
    if (!prime_ok(p)) return LINAC_ERR_PRIME;
    const int64_t npiv = std::min(m, n);
    uint32_t* dA_h = m > 0 && n > 0 ? (uint32_t*)mapped(h_A) : nullptr;
    int32_t* drank_h = (int32_t*)mapped(h_rank);
    int32_t* dpiv_h = npiv > 0 ? (int32_t*)mapped(h_pivots) : nullptr;
    if ((m > 0 && n > 0 && !dA_h) || !drank_h || (npiv > 0 && !dpiv_h)) return LINAC_ERR_ARG;
    const size_t abytes = (size_t)m * (size_t)ld * 4;
    const size_t rbytes = align_up(((size_t)npiv + 1) * 4, 256);
    void* buf = nullptr;
    linac_status s = scratch_get_slot(stream, 9, std::max<size_t>(abytes, 16) + rbytes, &buf);
    if (s != LINAC_OK) return s;
    uint32_t* dA = (uint32_t*)buf;
    int32_t* d_rank = (int32_t*)((char*)buf + align_up(std::max<size_t>(abytes, 16), 256));
    int32_t* d_piv = d_rank + 1;
    const Field f = make_field(p);
    int* st = status_word(stream);
    if (!st) return LINAC_ERR_NOMEM;
    LINAC_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(int), stream));
    if ((s = copy_words(dA_h, dA, abytes, stream)) != LINAC_OK) return s;
    s = dense_rref(dA, m, n, ld, f, n, d_rank, d_piv, auto_path(m, n), 0, stream);
    if (s != LINAC_OK) return s;
    if ((s = copy_words(dA, dA_h, abytes, stream)) != LINAC_OK) return s;
    {
        ProfScope ps(stream, PROF_HOST_COPY);
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((npiv + 255) / 256, 64));
        hostio_results_kernel<<<blocks, 256, 0, stream>>>(d_rank, d_piv, npiv, drank_h, dpiv_h);
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    return LINAC_OK;
}
