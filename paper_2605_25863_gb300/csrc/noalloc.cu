// noalloc.cu -- linac_rref_noalloc: the in-place RREF of linac_rref for
// callers that cannot allocate device memory.
//
// Who needs it.  linac_rref takes its scratch from a buffer the library
// allocates with cudaMalloc on first use.  Some callers cannot allow that:
// applications whose own pool allocator has reserved the whole device (a
// foreign cudaMalloc then fails or fragments their pool), latency-critical
// loops that cannot afford cudaMalloc's implicit device synchronisation and
// unpredictable cost, and plugins hosted by a process whose policy forbids
// device allocations outside its own allocator.  This entry point allocates
// nothing: its scratch lives in one fixed file-scope device array,
// g_noalloc_scratch, that the CUDA runtime reserves on every device that
// loads the library and keeps until the process exits.
//
// Limits and rules.
//  - m <= 2048 and n <= 2048 (the array is 4 MiB); larger sizes return
//    LINAC_ERR_UNSUPPORTED before anything is launched.  The trailing update
//    always uses the plain CUDA-core path, with the default panel width.
//  - The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make
//    that first call before any stream capture on the device.
//  - Every call, on every stream, shares the one array and leaves its
//    contents behind; each call re-initialises everything it reads before
//    reading it.  Calls whose executions overlap on the GPU (two streams, or
//    two host threads) race on the array and give wrong results: serialise
//    them.
//  - Pivots come from the same places as in linac_rref: the window of the
//    first nb + 16 remaining rows on an 8-block cluster, and the grid-wide
//    search when the window lacks a pivot.
//  - A device-side failure (a bounded wait that gave up, which never happens
//    in correct operation, or a zero pivot head) is recorded in the array's
//    status word, not in linac_last_device_status().  A final one-thread
//    kernel then writes minus that status to *d_rank (-6 for
//    LINAC_ERR_TIMEOUT), so the caller sees the failure in the output it
//    already reads, without another call.
#include <algorithm>
#include <climits>
#include <mutex>

#include "dense_kernels.cuh"
#include "linac_host.h"
#include "update.cuh"

namespace linac {

namespace {

constexpr int64_t kNoallocMaxDim = 2048;
constexpr size_t kNoallocBytes = (size_t)4 << 20;
constexpr int kNoallocMaxGrid = (int)((kNoallocMaxDim + 127) / 128);   // panel blocks for m <= 2048

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

struct NoallocLayout {
    size_t off_status, off_state, off_cand, off_panel, off_e, off_ft, off_w, off_r, total;
    int64_t ldF, ldW;
};

NoallocLayout noalloc_layout(int64_t m, int64_t n) {
    NoallocLayout L;
    size_t o = 0;
    L.off_status = o; o = align_up(o + 256, 256);
    L.off_state = o;  o = align_up(o + sizeof(DenseState), 256);
    L.off_cand = o;   o = align_up(o + (size_t)2 * kNoallocMaxGrid * (NB_MAX + 1) * 4, 256);
    L.off_panel = o;  o = align_up(o + (size_t)NB_MAX * NB_MAX * 4, 256);
    L.off_e = o;      o = align_up(o + (size_t)NB_MAX * NB_MAX * 4, 256);
    L.ldF = (int64_t)align_up((size_t)std::max<int64_t>(m, 1), 4);
    L.off_ft = o;     o = align_up(o + (size_t)NB_MAX * L.ldF * 4, 256);
    L.ldW = (int64_t)align_up((size_t)std::max<int64_t>(n, 1), 4);
    L.off_w = o;      o = align_up(o + (size_t)NB_MAX * L.ldW * 4, 256);
    L.off_r = o;      o = align_up(o + (size_t)NB_MAX * L.ldW * 4, 256);
    L.total = o;
    return L;
}

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};

// Device address of g_noalloc_scratch on the current device (set up once per
// device).  In host code the array's name is only a host-side stand-in, so
// kernels must be given this address instead.
linac_status noalloc_base(void** out) {
    int dev = 0;
    LINAC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return LINAC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return LINAC_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return LINAC_OK;
}

// A failure recorded in the status word replaces the rank by its negation.
__global__ void noalloc_report_kernel(const int* __restrict__ status, int32_t* d_rank) {
    const int v = *status;
    if (v != 0) *d_rank = -v;
}

}  // namespace

}  // namespace linac

using namespace linac;

extern "C" linac_status linac_rref_noalloc(uint32_t* d_A, int64_t m, int64_t n, int64_t ld, uint32_t p,
                                           int32_t* d_rank, int32_t* d_pivots, cudaStream_t stream) {
    if (m < 0 || n < 0 || ld < n) return LINAC_ERR_ARG;
    if (m > kNoallocMaxDim || n > kNoallocMaxDim) return LINAC_ERR_UNSUPPORTED;
    if (m > 0 && n > 0 && !d_A) return LINAC_ERR_ARG;
    if (!d_rank || (std::min(m, n) > 0 && !d_pivots)) return LINAC_ERR_ARG;
    if (ld % 4 != 0 || ((uintptr_t)d_A % 16) != 0) return LINAC_ERR_ALIGN;
    if (!prime_ok(p)) return LINAC_ERR_PRIME;
    const Field f = make_field(p);

    const int nb = dense_default_nb(m, n);
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>((m + 127) / 128, sm_count()));
    const int S_max = (int)((std::max<int64_t>(m, 1) + G - 1) / G);
    const size_t psmem = (size_t)S_max * (nb + 1) * 4 + NB_MAX * 4 + NB_MAX * 4 + (size_t)S_max + 16;
    const NoallocLayout L = noalloc_layout(m, n);
    if (L.total > kNoallocBytes || G > kNoallocMaxGrid) return LINAC_ERR_UNSUPPORTED;

    void* base = nullptr;
    linac_status s = noalloc_base(&base);
    if (s != LINAC_OK) return s;
    char* ws = (char*)base;
    int* status = (int*)(ws + L.off_status);
    DenseState* st = (DenseState*)(ws + L.off_state);
    uint32_t* cand = (uint32_t*)(ws + L.off_cand);
    uint32_t* panelU = (uint32_t*)(ws + L.off_panel);
    int32_t* Ft = (int32_t*)(ws + L.off_ft);
    int32_t* Et = (int32_t*)(ws + L.off_e);
    int32_t* W = (int32_t*)(ws + L.off_w);
    int32_t* R = (int32_t*)(ws + L.off_r);

    if ((s = ensure_dynamic_smem((const void*)panel_kernel, (int)psmem)) != LINAC_OK) return s;
    if ((s = ensure_dynamic_smem((const void*)einv_kernel, (int)EINV_SMEM)) != LINAC_OK) return s;
    int occ = 0;
    LINAC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, panel_kernel, PANEL_THREADS, psmem));
    if (occ < 1 || G > occ * sm_count()) return LINAC_ERR_UNSUPPORTED;

    // the status word and the elimination state start from zero / their
    // initial values on every call (the array keeps the previous call's data)
    LINAC_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), stream));
    const int64_t npiv = std::min(m, n);
    const unsigned iblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((npiv + 255) / 256, 1024));
    init_kernel<<<iblocks, 256, 0, stream>>>(st, d_pivots, npiv, d_rank);
    LINAC_CUDA_TRY(cudaGetLastError());
    if (m == 0 || n == 0) return LINAC_OK;

    const WaitLimit wl0 = wait_limit();
    for (int64_t c0 = 0; c0 < n; c0 += nb) {
        const int w = (int)std::min<int64_t>(nb, n - c0);
        const int64_t ncols = n - c0;
        launch_window(d_A, m, ld, (int)c0, w, f, st, panelU, G, nullptr, stream);
        {
            const uint32_t* Mc = d_A;
            int64_t m_ = m, ld_ = ld;
            int c0_ = (int)c0, w_ = w, S_ = S_max;
            Field f_ = f;
            WaitLimit wl = wl0;
            const int32_t* rowmap = nullptr;
            void* args[] = {(void*)&Mc, &m_, &ld_, &c0_, &w_, &S_, &f_, &st, &cand, &panelU, &status, &wl, &rowmap};
            LINAC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)panel_kernel, dim3(G), dim3(PANEL_THREADS),
                                                       args, psmem, stream));
        }
        gather_f_kernel<<<(unsigned)((m + 63) / 64), 256, 0, stream>>>(d_A, m, ld, (int)c0, w, f, st, Ft, L.ldF,
                                                                       nullptr);
        const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ncols + 1023) / 1024, 64));
        gather_w_kernel<<<dim3(gx, NB_MAX), 256, 0, stream>>>(d_A, ld, ncols, (int)c0, f, st, W, L.ldW);
        heads_inverse_kernel<<<1, NB_MAX, 0, stream>>>(st, panelU, (int)c0, f.p, status);
        einv_kernel<<<NB_MAX / EINV_COLS, 256, EINV_SMEM, stream>>>(st, panelU, (int)c0, f, Et);
        s = launch_gemm_assign(f, st, Et, NB_MAX, W, L.ldW, ncols, R, L.ldW, stream);
        if (s != LINAC_OK) return s;
        move_kernel<<<NB_MAX, 256, 0, stream>>>(d_A, ld, n, (int)c0, st, Ft, L.ldF);
        s = launch_update(LINAC_PATH_PLAIN, d_A, m, n, ld, (int)c0, f, st, Ft, L.ldF, R, L.ldW, nullptr, nullptr,
                         status, nullptr, stream);
        if (s != LINAC_OK) return s;
        finish_kernel<<<1, NB_MAX, 0, stream>>>(st, d_pivots, d_rank);
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    noalloc_report_kernel<<<1, 1, 0, stream>>>(status, d_rank);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}
