// api.cu -- the extern "C" entry points declared in include/linac.h: argument
// checks, the prime test, per-prime constants, scratch memory, dispatch.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "linac_host.h"
#include "update.cuh"

namespace linac {

// ---------------------------------------------------------------------------
// Primes and constants

static uint64_t mulmod64_host(uint64_t a, uint64_t b, uint64_t n) {
    return (uint64_t)(((unsigned __int128)a * b) % n);
}

static uint64_t powmod64_host(uint64_t a, uint64_t e, uint64_t n) {
    uint64_t r = 1 % n;
    a %= n;
    while (e) {
        if (e & 1) r = mulmod64_host(r, a, n);
        a = mulmod64_host(a, a, n);
        e >>= 1;
    }
    return r;
}

bool is_prime_u32(uint32_t n) {
    if (n < 2) return false;
    for (uint32_t q : {2u, 3u, 5u, 7u, 11u, 13u, 17u, 19u, 23u, 29u, 31u, 37u, 61u}) {
        if (n == q) return true;
        if (n % q == 0) return false;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (uint64_t a : {2ull, 7ull, 61ull}) {
        uint64_t x = powmod64_host(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool composite = true;
        for (int i = 1; i < s; ++i) {
            x = mulmod64_host(x, x, n);
            if (x == n - 1) { composite = false; break; }
        }
        if (composite) return false;
    }
    return true;
}

Field make_field(uint32_t p) {
    Field f;
    f.p = p;
    f.mu = ~0ull / p;                              // floor((2^64 - 1) / p) = floor(2^64 / p), p odd
    f.c32 = (uint32_t)((1ull << 32) % p);
    f.half = (p - 1) / 2;
    // Bound of a folded accumulator H*c32 + L, H in [-2^31, 2^31), L in [0, 2^32).
    const unsigned __int128 afold = (unsigned __int128)((1ull << 31) - 1) * f.c32 + 0xFFFFFFFFull;
    const unsigned __int128 afold_neg = (unsigned __int128)(1ull << 31) * f.c32;
    const unsigned __int128 amax = afold > afold_neg ? afold : afold_neg;
    const unsigned __int128 prod = (unsigned __int128)f.half * f.half;
    const unsigned __int128 room = (((unsigned __int128)1) << 63) - 1 - amax;
    unsigned __int128 k = prod ? room / prod : 1024;
    f.fold = (uint32_t)std::min<unsigned __int128>(k, 1024);
    // Montgomery constants: p^(-1) mod 2^32 by Newton's iteration (each step
    // doubles the number of correct low bits; p is odd, so p is its own
    // inverse mod 8), then R^2 mod p = (2^32 mod p)^2 mod p
    uint32_t inv = p;
    for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
    f.pinv = 0u - inv;
    f.r2 = (uint32_t)(((uint64_t)f.c32 * f.c32) % p);
    return f;
}

bool is_prime_u64(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t q : bases) {
        if (n == q) return true;
        if (n % q == 0) return false;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (uint64_t a : bases) {
        uint64_t x = powmod64_host(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool composite = true;
        for (int i = 1; i < s; ++i) {
            x = mulmod64_host(x, x, n);
            if (x == n - 1) { composite = false; break; }
        }
        if (composite) return false;
    }
    return true;
}

Field64 make_field64(uint64_t p) {
    Field64 f;
    f.p = p;
    // p^(-1) mod 2^64 by Newton's iteration: p is its own inverse mod 8 (3
    // bits) and each step doubles the correct low bits (3, 6, 12, 24, 48, 96)
    uint64_t inv = p;
    for (int i = 0; i < 5; ++i) inv *= 2ull - p * inv;
    f.pinv = 0ull - inv;
    f.r1 = (0ull - p) % p;                 // 2^64 - p is congruent to 2^64
    f.r2 = mulmod64_host(f.r1, f.r1, p);   // 2^128 mod p
    f.r3 = mulmod64_host(f.r2, f.r1, p);   // 2^192 mod p
    return f;
}

int fold_shifts(const Field& f, FoldShifts* fs) {
    uint32_t c = f.c32;
    int n = 0;
    fs->alu_reduce = 0;
    fs->pad = 0;
    for (int i = 0; i < 3; ++i) fs->e[i] = 0;
    for (int b = 0; b < 32; ++b)
        if ((c >> b) & 1u) {
            if (n == 3) {
                for (int i = 0; i < 3; ++i) fs->e[i] = 0;
                n = 0;
                break;
            }
            fs->e[n++] = (uint32_t)b;
        }
    for (int i = 0; i < 3; ++i) fs->s[i] = fs->e[i] == 0 ? 31u : 32u - fs->e[i];
    if (n > 0) {
        // bounds of reduce_alu (linac_device.cuh)
        const unsigned __int128 cc = c;
        const bool low_ok = cc * (cc + 1) / 2 <= f.p;
        const bool high_ok = (((unsigned __int128)1) << 32) - 1 + cc * (cc / 2 + 1) < (unsigned __int128)3 * f.p;
        fs->alu_reduce = low_ok && high_ok;
    }
    return n;
}

// ---------------------------------------------------------------------------
// Scratch memory

namespace {
struct ScratchBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_mu;
std::map<std::tuple<int, cudaStream_t, int>, ScratchBuf> g_scratch;
std::map<std::pair<int, cudaStream_t>, int*> g_status;
int g_sm_count[64] = {0};
int g_smem_optin[64] = {0};
}  // namespace

// Attribute of the CURRENT device, cached per device for the first 64
// device ordinals (queried every time beyond them).
static int device_attr(cudaDeviceAttr attr, int* cache) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    int v = 0;
    if (cudaDeviceGetAttribute(&v, attr, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    if (dev >= 0 && dev < 64) cache[dev] = v;
    return v;
}

int sm_count() {
    const int v = device_attr(cudaDevAttrMultiProcessorCount, g_sm_count);
    return v > 0 ? v : 1;
}

namespace {
std::atomic<long long> g_wait_cycles{0};
std::atomic<unsigned> g_wait_extra{0};
}  // namespace

WaitLimit wait_limit() {
    WaitLimit w;
    const long long c = g_wait_cycles.load();
    w.spin_cycles = c > 0 ? c : kSpinCycles;
    w.extra_arrivals = g_wait_extra.load();
    w.pad = 0;
    return w;
}

linac_status ensure_dynamic_smem(const void* fn, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> set;
    int dev = 0;
    LINAC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    int& cur = set[std::make_pair(dev, fn)];
    if (bytes > cur) {
        LINAC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        cur = bytes;
    }
    return LINAC_OK;
}

int auto_path(int64_t m, int64_t n) {
    // measured on GB300 (whole eliminations, p = 2^31 - 1): the hybrid update
    // beats the plain one by 3.5 % at 16384 x 16640 and 4.7 % at 32768 x
    // 33024, ties at 8192 x 8448 (its residue split costs what it gains) and
    // loses below
    return (m >= 16384 && n >= 16384) ? LINAC_PATH_HYBRID : LINAC_PATH_PLAIN;
}

int max_smem_optin() { return device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin, g_smem_optin); }

linac_status scratch_get_slot(cudaStream_t stream, int slot, size_t bytes, void** ptr) {
    int dev = 0;
    LINAC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchBuf& b = g_scratch[std::make_tuple(dev, stream, slot)];
    if (b.bytes < bytes) {
        if (b.ptr) {
            LINAC_CUDA_TRY(cudaStreamSynchronize(stream));
            cudaFree(b.ptr);
            b.ptr = nullptr;
            b.bytes = 0;
        }
        const size_t want = align_up(bytes, 1 << 20);
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return LINAC_ERR_NOMEM;
        }
        b.ptr = p;
        b.bytes = want;
    }
    *ptr = b.ptr;
    return LINAC_OK;
}

linac_status scratch_get(cudaStream_t stream, size_t bytes, void** ptr) {
    return scratch_get_slot(stream, 0, bytes, ptr);
}

int* status_word(cudaStream_t stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    int*& w = g_status[std::make_pair(dev, stream)];
    if (!w) {
        if (cudaMalloc(&w, 256) != cudaSuccess) {
            (void)cudaGetLastError();
            w = nullptr;
            return nullptr;
        }
        cudaMemset(w, 0, 256);
    }
    return w;
}

}  // namespace linac

using namespace linac;

namespace {

linac_status check_matrix(const void* d, int64_t m, int64_t n, int64_t ld) {
    if (m < 0 || n < 0 || ld < n || m > INT32_MAX || n > INT32_MAX) return LINAC_ERR_ARG;
    if (m > 0 && n > 0 && !d) return LINAC_ERR_ARG;
    if (ld % 4 != 0 || ((uintptr_t)d % 16) != 0) return LINAC_ERR_ALIGN;
    return LINAC_OK;
}

// uint64 matrices: ld a multiple of 2 elements (16-byte rows, section 3.4's
// ulonglong2 accesses) and a 16-byte aligned start.
linac_status check_matrix64(const void* d, int64_t m, int64_t n, int64_t ld) {
    if (m < 0 || n < 0 || ld < n || m > INT32_MAX || n > INT32_MAX) return LINAC_ERR_ARG;
    if (m > 0 && n > 0 && !d) return LINAC_ERR_ARG;
    if (ld % 2 != 0 || ((uintptr_t)d % 16) != 0) return LINAC_ERR_ALIGN;
    return LINAC_OK;
}

linac_status check_opts(const linac_options* o) {
    if (!o) return LINAC_OK;
    if (o->path < LINAC_PATH_AUTO || o->path > LINAC_PATH_HYBRID) return LINAC_ERR_ARG;
    if (o->nb < 0 || o->nb > NB_MAX || (o->nb % UPD_BK) != 0) return LINAC_ERR_ARG;
    return LINAC_OK;
}

int resolve_path(const linac_options* o, int64_t m, int64_t n) {
    const int p = o ? o->path : LINAC_PATH_AUTO;
    return p == LINAC_PATH_AUTO ? auto_path(m, n) : p;
}

linac_status reset_status(cudaStream_t stream) {
    int* s = status_word(stream);
    if (!s) return LINAC_ERR_NOMEM;
    LINAC_CUDA_TRY(cudaMemsetAsync(s, 0, sizeof(int), stream));
    return LINAC_OK;
}

}  // namespace

extern "C" {

linac_status linac_rref_ex(uint32_t* d_A, int64_t m, int64_t n, int64_t ld, uint32_t p,
                           int64_t ncols_search, int32_t* d_rank, int32_t* d_pivots,
                           const linac_options* opts, cudaStream_t stream) {
    linac_status s = check_matrix(d_A, m, n, ld);
    if (s != LINAC_OK) return s;
    if (ncols_search < 0 || ncols_search > n || !d_rank) return LINAC_ERR_ARG;
    if (std::min(m, ncols_search) > 0 && !d_pivots) return LINAC_ERR_ARG;
    if ((s = check_opts(opts)) != LINAC_OK) return s;
    if (!prime_ok(p)) return LINAC_ERR_PRIME;
    const Field f = make_field(p);
    if ((s = reset_status(stream)) != LINAC_OK) return s;
    if (opts && opts->validate) {
        s = validate_range(d_A, m, n, ld, p, status_word(stream), stream);
        if (s != LINAC_OK) return s;
    }
    return dense_rref(d_A, m, n, ld, f, ncols_search, d_rank, d_pivots, resolve_path(opts, m, n),
                      opts ? opts->nb : 0, stream);
}

linac_status linac_rref(uint32_t* d_A, int64_t m, int64_t n, int64_t ld, uint32_t p, int32_t* d_rank,
                        int32_t* d_pivots, cudaStream_t stream) {
    return linac_rref_ex(d_A, m, n, ld, p, n, d_rank, d_pivots, nullptr, stream);
}

linac_status linac_solve_ex(const uint32_t* d_A, int64_t m, int64_t nA, int64_t ldA, const uint32_t* d_B,
                            int64_t k, int64_t ldB, uint32_t p, uint32_t* d_X, int64_t ldX,
                            uint8_t* d_consistent, int32_t* d_rank, int32_t* d_pivots,
                            const linac_options* opts, cudaStream_t stream) {
    linac_status s = check_matrix(d_A, m, nA, ldA);
    if (s != LINAC_OK) return s;
    if ((s = check_matrix(d_B, m, k, ldB)) != LINAC_OK) return s;
    if (ldX < k || !d_rank || (std::min(m, nA) > 0 && !d_pivots)) return LINAC_ERR_ARG;
    if (k > 0 && nA > 0 && !d_X) return LINAC_ERR_ARG;
    if (k > 0 && !d_consistent) return LINAC_ERR_ARG;
    if (nA + k > INT32_MAX) return LINAC_ERR_ARG;
    if ((s = check_opts(opts)) != LINAC_OK) return s;
    if (!prime_ok(p)) return LINAC_ERR_PRIME;
    const Field f = make_field(p);
    if ((s = reset_status(stream)) != LINAC_OK) return s;
    if (opts && opts->validate) {
        if ((s = validate_range(d_A, m, nA, ldA, p, status_word(stream), stream)) != LINAC_OK) return s;
        if ((s = validate_range(d_B, m, k, ldB, p, status_word(stream), stream)) != LINAC_OK) return s;
    }
    const int64_t ldM = (int64_t)align_up((size_t)std::max<int64_t>(nA + k, 1), 4);
    void* buf = nullptr;
    if ((s = scratch_get_slot(stream, 1, (size_t)std::max<int64_t>(m, 1) * ldM * 4, &buf)) != LINAC_OK) return s;
    uint32_t* dM = (uint32_t*)buf;
    if ((s = solve_pack(d_A, m, nA, ldA, d_B, k, ldB, dM, ldM, stream)) != LINAC_OK) return s;
    s = dense_rref(dM, m, nA + k, ldM, f, nA, d_rank, d_pivots, resolve_path(opts, m, nA + k), opts ? opts->nb : 0,
                   stream);
    if (s != LINAC_OK) return s;
    return solve_extract(dM, m, nA, k, ldM, d_rank, d_pivots, d_X, ldX, d_consistent, stream);
}

linac_status linac_solve(const uint32_t* d_A, int64_t m, int64_t nA, int64_t ldA, const uint32_t* d_B,
                         int64_t k, int64_t ldB, uint32_t p, uint32_t* d_X, int64_t ldX,
                         uint8_t* d_consistent, int32_t* d_rank, int32_t* d_pivots, cudaStream_t stream) {
    return linac_solve_ex(d_A, m, nA, ldA, d_B, k, ldB, p, d_X, ldX, d_consistent, d_rank, d_pivots,
                          nullptr, stream);
}

linac_status linac_lup(const uint32_t* d_A, int64_t m, int64_t n, int64_t ldA, uint32_t p, uint32_t* d_L,
                       int64_t ldL, uint32_t* d_U, int64_t ldU, int32_t* d_perm, int32_t* d_rank,
                       int32_t* d_pivots, cudaStream_t stream) {
    linac_status s = check_matrix(d_A, m, n, ldA);
    if (s != LINAC_OK) return s;
    const int64_t mn = std::min(m, n);
    if (!d_rank || (m > 0 && !d_perm) || (mn > 0 && (!d_pivots || !d_L)) || (m > 0 && n > 0 && !d_U))
        return LINAC_ERR_ARG;
    if (ldL < mn || ldU < n) return LINAC_ERR_ARG;
    if (!prime_ok(p)) return LINAC_ERR_PRIME;
    if ((s = reset_status(stream)) != LINAC_OK) return s;
    return lup_factor(d_A, m, n, ldA, make_field(p), d_L, ldL, d_U, ldU, d_perm, d_rank, d_pivots, stream);
}

linac_status linac_rref_batched(uint32_t* d_data, const int64_t* d_offsets, const int32_t* d_m,
                                const int32_t* d_n, const int32_t* d_ld, const int32_t* d_nsearch,
                                int32_t batch, int32_t max_m, int32_t max_n, uint32_t p, uint32_t flags,
                                int32_t* d_ranks, int32_t* d_pivots, const int64_t* d_piv_offsets,
                                int32_t* d_status, cudaStream_t stream) {
    if (batch < 0 || max_m < 0 || max_n < 0) return LINAC_ERR_ARG;
    if (batch == 0) return LINAC_OK;
    if (!d_data || !d_offsets || !d_m || !d_n || !d_ld || !d_ranks || !d_pivots || !d_piv_offsets)
        return LINAC_ERR_ARG;
    if ((uintptr_t)d_data % 16) return LINAC_ERR_ALIGN;
    if (flags & ~LINAC_SHARED_PATTERN) return LINAC_ERR_ARG;
    if (max_n > 1024 || max_m > 1024) return LINAC_ERR_UNSUPPORTED;
    if (!prime_ok(p)) return LINAC_ERR_PRIME;
    const Field f = make_field(p);
    linac_status s = reset_status(stream);
    if (s != LINAC_OK) return s;
    return batched_rref(d_data, d_offsets, d_m, d_n, d_ld, d_nsearch, batch, max_m, max_n, f, flags,
                        d_ranks, d_pivots, d_piv_offsets, d_status, stream);
}

linac_status linac_batched_tune(uint32_t p, int32_t* nb_out, cudaStream_t stream) {
    if (!prime_ok(p)) return LINAC_ERR_PRIME;
    return batched_tune(make_field(p), nb_out, stream);
}

linac_status linac_batched_set_panel_widths(const int32_t* nb) {
    if (!nb) return LINAC_ERR_ARG;
    return batched_set_nb(nb);
}

linac_status linac_batched_panel_widths(int32_t* nb_out) {
    if (!nb_out) return LINAC_ERR_ARG;
    batched_get_nb(nb_out);
    return LINAC_OK;
}

linac_status linac_rref64_ex(uint64_t* d_A, int64_t m, int64_t n, int64_t ld, uint64_t p, int64_t ncols_search,
                             int32_t* d_rank, int32_t* d_pivots, const linac_options* opts, cudaStream_t stream) {
    linac_status s = check_matrix64(d_A, m, n, ld);
    if (s != LINAC_OK) return s;
    if (ncols_search < 0 || ncols_search > n || !d_rank) return LINAC_ERR_ARG;
    if (std::min(m, ncols_search) > 0 && !d_pivots) return LINAC_ERR_ARG;
    if (opts && (opts->path != LINAC_PATH_AUTO || opts->nb != 0)) return LINAC_ERR_ARG;
    if (!prime64_ok(p)) return LINAC_ERR_PRIME;
    if ((s = reset_status(stream)) != LINAC_OK) return s;
    if (opts && opts->validate) {
        s = validate64_range(d_A, m, n, ld, p, status_word(stream), stream);
        if (s != LINAC_OK) return s;
    }
    return dense64_rref(d_A, m, n, ld, make_field64(p), ncols_search, d_rank, d_pivots, stream);
}

linac_status linac_rref64(uint64_t* d_A, int64_t m, int64_t n, int64_t ld, uint64_t p, int32_t* d_rank,
                          int32_t* d_pivots, cudaStream_t stream) {
    return linac_rref64_ex(d_A, m, n, ld, p, n, d_rank, d_pivots, nullptr, stream);
}

linac_status linac_solve64(const uint64_t* d_A, int64_t m, int64_t nA, int64_t ldA, const uint64_t* d_B, int64_t k,
                           int64_t ldB, uint64_t p, uint64_t* d_X, int64_t ldX, uint8_t* d_consistent,
                           int32_t* d_rank, int32_t* d_pivots, cudaStream_t stream) {
    linac_status s = check_matrix64(d_A, m, nA, ldA);
    if (s != LINAC_OK) return s;
    if ((s = check_matrix64(d_B, m, k, ldB)) != LINAC_OK) return s;
    if (ldX < k || !d_rank || (std::min(m, nA) > 0 && !d_pivots)) return LINAC_ERR_ARG;
    if (k > 0 && nA > 0 && !d_X) return LINAC_ERR_ARG;
    if (k > 0 && !d_consistent) return LINAC_ERR_ARG;
    if (nA + k > INT32_MAX) return LINAC_ERR_ARG;
    if (!prime64_ok(p)) return LINAC_ERR_PRIME;
    if ((s = reset_status(stream)) != LINAC_OK) return s;
    const int64_t ldM = (int64_t)align_up((size_t)std::max<int64_t>(nA + k, 1), 2);
    void* buf = nullptr;
    if ((s = scratch_get_slot(stream, 7, (size_t)std::max<int64_t>(m, 1) * ldM * 8, &buf)) != LINAC_OK) return s;
    uint64_t* dM = (uint64_t*)buf;
    if ((s = solve64_pack(d_A, m, nA, ldA, d_B, k, ldB, dM, ldM, stream)) != LINAC_OK) return s;
    s = dense64_rref(dM, m, nA + k, ldM, make_field64(p), nA, d_rank, d_pivots, stream);
    if (s != LINAC_OK) return s;
    return solve64_extract(dM, m, nA, k, ldM, d_rank, d_pivots, d_X, ldX, d_consistent, stream);
}

size_t linac_workspace64_bytes(int64_t m, int64_t n) {
    if (m < 0 || n < 0) return 0;
    return dense64_workspace_bytes(m, n);
}

size_t linac_workspace_bytes(int64_t m, int64_t n, const linac_options* opts) {
    if (m < 0 || n < 0) return 0;
    const int nb = opts && opts->nb ? opts->nb : dense_default_nb(m, n);
    return dense_workspace_bytes(m, n, nb);
}

linac_status linac_last_device_status(cudaStream_t stream) {
    int* s = status_word(stream);
    if (!s) return LINAC_ERR_NOMEM;
    int v = 0;
    LINAC_CUDA_TRY(cudaStreamSynchronize(stream));
    LINAC_CUDA_TRY(cudaMemcpy(&v, s, sizeof(int), cudaMemcpyDeviceToHost));
    return (linac_status)v;
}

const char* linac_status_string(linac_status s) {
    switch (s) {
        case LINAC_OK: return "ok";
        case LINAC_ERR_ARG: return "invalid argument";
        case LINAC_ERR_PRIME: return "p is not an odd prime in the entry point's range";
        case LINAC_ERR_ALIGN: return "leading dimension or pointer misaligned";
        case LINAC_ERR_CUDA: return "CUDA runtime error";
        case LINAC_ERR_NOMEM: return "out of device memory";
        case LINAC_ERR_TIMEOUT: return "device-side wait timed out";
        case LINAC_ERR_RANGE: return "entry outside [0, p)";
        case LINAC_ERR_UNSUPPORTED: return "unsupported size or option";
    }
    return "unknown status";
}

linac_status linac_set_wait_limit(int64_t cycles) {
    if (cycles < 0) return LINAC_ERR_ARG;
    g_wait_cycles.store(cycles);
    return LINAC_OK;
}

void linac_debug_inject_wait_failure(int32_t on) { g_wait_extra.store(on ? 1u : 0u); }

int32_t linac_version(void) { return 200; }

}  // extern "C"
