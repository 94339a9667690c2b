// int_rates.cu -- throughput probes for the roofline denominators of the
// trailing-update paths: the integer multiply-add pipe (mad.wide.s32, the
// instruction of the plain path) and the integer tensor pipe
// (mma.sync m16n8k32 u8 -> s32 of the limb path, s8 -> s32 of the
// multi-modular path), plus dp4a for comparison.
//
// Measurement tooling only: built into its own library, liblinac_probes.so,
// which the benchmark loads for --measure-peaks; liblinac.so does not
// contain it.  Each probe keeps many independent chains in flight so the
// pipe, not latency, is the limit, and feeds every multiply an operand that
// changes each iteration (a loop-invariant product could be hoisted by the
// compiler, turning the probe into an add-throughput probe).
#include <cstdint>
#include <cuda_runtime.h>

#include "int_rates.h"

namespace linac_probes {

__global__ void probe_imad_wide(unsigned long long* out, uint32_t seed, int iters) {
    long long acc[8];
#pragma unroll
    for (int j = 0; j < 8; j++) acc[j] = (long long)(seed * (j + 1) + threadIdx.x);
    const int b = (int)(seed ^ 0x9e3779b9u) | 1;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int a = (int)(unsigned)acc[j];   // low word of the accumulator: data dependent
            asm volatile("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc[j]) : "r"(a), "r"(b));
        }
    }
    long long s = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) s += acc[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (unsigned long long)s;
}

__global__ void probe_dp4a(int* out, uint32_t seed, int iters) {
    int acc[8];
#pragma unroll
    for (int j = 0; j < 8; j++) acc[j] = (int)(seed * (j + 1) + threadIdx.x);
    const int b = (int)(seed ^ 0x9e3779b9u);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < 8; j++) asm volatile("dp4a.u32.u32 %0, %0, %1, %0;" : "+r"(acc[j]) : "r"(b));
    }
    int s = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) s += acc[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_imma_u8(int* out, uint32_t seed, int iters) {
    const uint32_t a0 = seed ^ threadIdx.x, a1 = a0 * 3, a2 = a0 * 5, a3 = a0 * 7, b0 = a0 * 11, b1 = a0 * 13;
    int d[4][4];
#pragma unroll
    for (int c = 0; c < 4; c++) d[c][0] = d[c][1] = d[c][2] = d[c][3] = 0;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < 4; c++)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    int s = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_imma_s8(int* out, uint32_t seed, int iters) {
    const uint32_t a0 = seed ^ threadIdx.x, a1 = a0 * 3, a2 = a0 * 5, a3 = a0 * 7, b0 = a0 * 11, b1 = a0 * 13;
    int d[4][4];
#pragma unroll
    for (int c = 0; c < 4; c++) d[c][0] = d[c][1] = d[c][2] = d[c][3] = 0;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < 4; c++)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    int s = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Co-issue: warps 0-7 run mad.wide.s32 chains (multiply pipe), warps 8-15
// run mma.sync u8 (tensor pipe).  MODE 0: only the first group works,
// 1: only the second, 2: both at once.
template <int MODE>
__global__ void __launch_bounds__(512, 1) probe_coissue(long long* out, int it_imad, int it_imma) {
    const int warp = threadIdx.x >> 5;
    long long s = 0;
    if (warp < 8) {
        if (MODE == 0 || MODE == 2) {
            long long acc[16];
#pragma unroll
            for (int j = 0; j < 16; j++) acc[j] = threadIdx.x * 31 + j;
            const int b = 0x12345 | 1;
            for (int it = 0; it < it_imad; ++it) {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int a = (int)(unsigned)acc[j];
                    asm volatile("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc[j]) : "r"(a), "r"(b));
                }
            }
#pragma unroll
            for (int j = 0; j < 16; j++) s += acc[j];
        }
    } else if (MODE == 1 || MODE == 2) {
        const uint32_t a0 = threadIdx.x * 3, a1 = a0 * 5, a2 = a0 * 7, a3 = a0 * 11, b0 = a0 * 13, b1 = a0 * 17;
        int d[4][4];
#pragma unroll
        for (int c = 0; c < 4; c++) d[c][0] = d[c][1] = d[c][2] = d[c][3] = 0;
        for (int it = 0; it < it_imma; ++it) {
#pragma unroll
            for (int c = 0; c < 4; c++)
                asm volatile(
                    "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};\n"
                    : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                    : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
#pragma unroll
        for (int c = 0; c < 4; c++) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    }
    out[blockIdx.x * 512 + threadIdx.x] = s;
}

}  // namespace linac_probes

using namespace linac_probes;

extern "C" int linac_probe_int_rates(linac_int_rates* out, cudaStream_t stream) {
    if (!out) return 1;
    int dev = 0, nsm = 0, clk = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 4;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) return 4;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    const int grid = nsm * 8, threads = 256, iters = 4096;
    void* buf = nullptr;
    if (cudaMalloc(&buf, (size_t)grid * threads * 8) != cudaSuccess) return 5;   // >= nsm * 512 * 8 for the co-issue probe
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    auto time_it = [&](auto launch) -> double {
        launch(16);   // warm-up
        cudaEventRecord(e0, stream);
        launch(iters);
        cudaEventRecord(e1, stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        return ms * 1e-3;
    };
    const double lanes = (double)grid * threads;
    double t = time_it([&](int it) { probe_imad_wide<<<grid, threads, 0, stream>>>((unsigned long long*)buf, 1u, it); });
    out->imad_wide_per_s = lanes * iters * 8 / t;
    t = time_it([&](int it) { probe_dp4a<<<grid, threads, 0, stream>>>((int*)buf, 1u, it); });
    out->dp4a_u8_mac_per_s = lanes * iters * 8 * 4 / t;
    t = time_it([&](int it) { probe_imma_u8<<<grid, threads, 0, stream>>>((int*)buf, 1u, it); });
    out->imma_u8_mac_per_s = (double)grid * (threads / 32) * iters * 4 * 4096.0 / t;
    t = time_it([&](int it) { probe_imma_s8<<<grid, threads, 0, stream>>>((int*)buf, 1u, it); });
    out->imma_s8_mac_per_s = (double)grid * (threads / 32) * iters * 4 * 4096.0 / t;
    {
        // co-issue of the two pipes in one block per SM
        const int ii = 2048, im = 1024;
        out->coissue_imad_only_ms =
            1e3 * time_it([&](int) { probe_coissue<0><<<nsm, 512, 0, stream>>>((long long*)buf, ii, im); });
        out->coissue_imma_only_ms =
            1e3 * time_it([&](int) { probe_coissue<1><<<nsm, 512, 0, stream>>>((long long*)buf, ii, im); });
        out->coissue_both_ms =
            1e3 * time_it([&](int) { probe_coissue<2><<<nsm, 512, 0, stream>>>((long long*)buf, ii, im); });
    }
    out->sm_clock_khz = clk;
    out->sm_count = nsm;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaGetLastError();
    cudaFree(buf);
    return e == cudaSuccess ? 0 : 4;
}
