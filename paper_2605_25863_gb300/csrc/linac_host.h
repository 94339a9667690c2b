// linac_host.h -- host-side helpers shared by the library's translation units:
// per-prime constants, scratch memory, launch error checks.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/linac.h"
#include "field64.cuh"
#include "linac_device.cuh"

namespace linac {

// Constants for the prime p (see Field in linac_device.cuh).
Field make_field(uint32_t p);

// Shift parameters of fold_any / reduce_alu for p (linac_device.cuh).
// Returns the number of set bits of 2^32 mod p when it is at most three
// (0 = use the multiply-pipe fold, and reduce_alu does not apply).
int fold_shifts(const Field& f, FoldShifts* fs);

// Deterministic Miller-Rabin for 32-bit n with bases 2, 7, 61 (these three
// bases have no common strong pseudoprime below 4,759,123,141; Jaeschke 1993).
bool is_prime_u32(uint32_t n);

// Odd prime below 2^31?
inline bool prime_ok(uint32_t p) { return p >= 3 && p < (1u << 31) && is_prime_u32(p); }

// Scratch memory: one growing device buffer per (device, stream).  The
// returned pointer stays valid until the next call that grows it on the same
// (device, stream); growing synchronises the stream first.
linac_status scratch_get(cudaStream_t stream, size_t bytes, void** ptr);
// Same, for an independent buffer `slot` (0 = dense elimination, 1 = solve's
// augmented matrix, 2 = batched driver, 3 = limb planes, 4 = null-space
// column positions, 6 = uint64 elimination, 7 = the uint64 solve's
// augmented matrix, 8 = residue planes of the multi-modular update, 9 = the
// device copy of linac_rref_host's matrix, 10 = the LUP factorisation).
linac_status scratch_get_slot(cudaStream_t stream, int slot, size_t bytes, void** ptr);

// Device status word of the most recent call on this (device, stream): lives
// in a small per-(device, stream) allocation that is never freed.
int* status_word(cudaStream_t stream);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

#define LINAC_CUDA_TRY(expr)                                   \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) {                               \
            (void)cudaGetLastError();                          \
            return e_ == cudaErrorMemoryAllocation ? LINAC_ERR_NOMEM : LINAC_ERR_CUDA; \
        }                                                      \
    } while (0)

// Limit of the device-side waits for the next launch: the limit set with
// linac_set_wait_limit (kSpinCycles by default) and the injected failure of
// linac_debug_inject_wait_failure.
WaitLimit wait_limit();

// cudaFuncSetAttribute(fn, MaxDynamicSharedMemorySize, bytes) on the current
// device only when bytes exceeds the value already set there, so repeated
// calls (and calls made while a stream is being captured) issue no runtime
// call after the first of each size.
linac_status ensure_dynamic_smem(const void* fn, int bytes);

// The trailing-update path LINAC_PATH_AUTO selects for an m x n elimination.
int auto_path(int64_t m, int64_t n);

// Number of SMs on the current device (cached per device).
int sm_count();
// Opt-in shared memory per block of the current device in bytes (cached per
// device; 0 if the query failed).
int max_smem_optin();

// Dense elimination driver (dense.cu): in-place RREF of the m x n matrix with
// pivots searched in [0, nsearch).  Scratch comes from scratch_get.
linac_status dense_rref(uint32_t* dA, int64_t m, int64_t n, int64_t ld, const Field& f,
                        int64_t nsearch, int32_t* d_rank, int32_t* d_pivots,
                        int path, int nb, cudaStream_t stream);
size_t dense_workspace_bytes(int64_t m, int64_t n, int nb);
int dense_default_nb(int64_t m, int64_t n);

// LUP factorisation P A = L U (lup.cu): L is m x min(m, n), U is m x n.
linac_status lup_factor(const uint32_t* dA, int64_t m, int64_t n, int64_t ldA, const Field& f, uint32_t* dL,
                        int64_t ldL, uint32_t* dU, int64_t ldU, int32_t* d_perm, int32_t* d_rank,
                        int32_t* d_pivots, cudaStream_t stream);

// Solve helpers (dense.cu).
linac_status solve_pack(const uint32_t* dA, int64_t m, int64_t nA, int64_t ldA,
                        const uint32_t* dB, int64_t k, int64_t ldB,
                        uint32_t* dM, int64_t ldM, cudaStream_t stream);
linac_status solve_extract(const uint32_t* dM, int64_t m, int64_t nA, int64_t k, int64_t ldM,
                           const int32_t* d_rank, const int32_t* d_pivots,
                           uint32_t* dX, int64_t ldX, uint8_t* d_consistent, cudaStream_t stream);

// Range validation (dense.cu): sets *status = LINAC_ERR_RANGE if any entry >= p.
linac_status validate_range(const uint32_t* dA, int64_t m, int64_t n, int64_t ld, uint32_t p,
                            int* d_status, cudaStream_t stream);

// Batched driver (batched.cu).
linac_status batched_rref(uint32_t* d_data, const int64_t* d_offsets, const int32_t* d_m,
                          const int32_t* d_n, const int32_t* d_ld, const int32_t* d_nsearch,
                          int32_t batch, int32_t max_m, int32_t max_n, const Field& f,
                          uint32_t flags, int32_t* d_ranks, int32_t* d_pivots,
                          const int64_t* d_piv_offsets, int32_t* d_status, cudaStream_t stream);

// Batched autotuner (batched.cu): per size bucket (m <= 64, 128, 256, 512,
// 1024) time the feasible panel widths and keep the fastest for this device.
linac_status batched_tune(const Field& f, int32_t* nb_out, cudaStream_t stream);
void batched_get_nb(int32_t* nb_out);
linac_status batched_set_nb(const int32_t* nb);

// uint64 residues, primes below 2^64 (dense64.cu; constants and the prime
// test in api.cu).
Field64 make_field64(uint64_t p);
// Deterministic Miller-Rabin for 64-bit n with the first twelve primes as
// bases (no strong pseudoprime to all of them below 3.3e24; Sorenson and
// Webster 2015).
bool is_prime_u64(uint64_t n);
inline bool prime64_ok(uint64_t p) { return p >= 3 && (p & 1) && is_prime_u64(p); }
linac_status dense64_rref(uint64_t* dA, int64_t m, int64_t n, int64_t ld, const Field64& f, int64_t nsearch,
                          int32_t* d_rank, int32_t* d_pivots, cudaStream_t stream);
size_t dense64_workspace_bytes(int64_t m, int64_t n);
linac_status solve64_pack(const uint64_t* dA, int64_t m, int64_t nA, int64_t ldA, const uint64_t* dB, int64_t k,
                          int64_t ldB, uint64_t* dM, int64_t ldM, cudaStream_t stream);
linac_status solve64_extract(const uint64_t* dM, int64_t m, int64_t nA, int64_t k, int64_t ldM,
                             const int32_t* d_rank, const int32_t* d_pivots, uint64_t* dX, int64_t ldX,
                             uint8_t* d_consistent, cudaStream_t stream);
linac_status validate64_range(const uint64_t* dA, int64_t m, int64_t n, int64_t ld, uint64_t p, int* d_status,
                              cudaStream_t stream);

}  // namespace linac
