/*
 * linac.h -- C ABI of the GB300 (sm_103a) exact mod-p row-reduction library.
 *
 * The library computes the reduced row-echelon form (RREF), rank, pivot
 * columns and particular solutions of linear systems over the prime field
 * Z/pZ for odd primes p < 2^31, with entries stored as uint32_t residues,
 * and (the *64 entry points near the end) for odd primes p < 2^64 with
 * uint64_t residues.
 * It follows the method of "Linac: linear algebra with CUDA over finite
 * fields": partially pivoted Gauss-Jordan elimination to RREF (section 3.2,
 * "Gaussian elimination on GPUs"), the RREF kept in the input's shape with
 * zero rows at the bottom (section 2.3), and solutions read off the reduced
 * augmented matrix (section 5.2, "Solving linear systems").
 *
 * Conventions shared by every entry point:
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device; the
 *    caller allocates and owns them.  Matrices are row-major with a leading
 *    dimension (ld, in elements) that is a multiple of 4 (of 2 for uint64
 *    residues) and >= the number of columns, and must start 16-byte aligned
 *    (section 3.2, "Number types": rows are padded so 128-bit accesses never
 *    cross a row).
 *  - Entries must be canonical residues in [0, p).  Larger entries are not
 *    reduced and give undefined results.
 *  - p must be an odd prime below 2^31 (below 2^64 for the *64 entry
 *    points), checked on the host with a deterministic Miller-Rabin test;
 *    otherwise LINAC_ERR_PRIME.
 *  - All calls are asynchronous and ordered on `stream` (0 = legacy default
 *    stream).  Argument errors are returned immediately; errors found on the
 *    device (a bounded wait that gave up) are written to the per-call device
 *    status word when one is given, otherwise reported by linac_last_device_status().
 *  - Scratch memory: the library keeps one growing scratch buffer per
 *    (device, stream), allocated with cudaMalloc on first use.  A call made
 *    while a stream is being captured into a CUDA graph must therefore be
 *    preceded by an uncaptured call of at least the same size on that stream.
 *  - Results are bit-exact: the field is exact, no floating point is used.
 */
#ifndef LINAC_H
#define LINAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cudaStream_t;

typedef enum {
    LINAC_OK = 0,
    LINAC_ERR_ARG = 1,        /* bad shape, null pointer, bad option */
    LINAC_ERR_PRIME = 2,      /* p is not an odd prime below 2^31 (below 2^64: *64 entry points) */
    LINAC_ERR_ALIGN = 3,      /* ld not a multiple of 4, or pointer not 16-byte aligned */
    LINAC_ERR_CUDA = 4,       /* a CUDA runtime call failed */
    LINAC_ERR_NOMEM = 5,      /* scratch allocation failed */
    LINAC_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up */
    LINAC_ERR_RANGE = 7,      /* an input entry is not in [0, p) (validation pass) */
    LINAC_ERR_UNSUPPORTED = 8 /* size or option outside what this build supports */
} linac_status;

/* Trailing-update arithmetic (the rank-k update C <- C - A*B mod p that
 * dominates the O(n^3) work). */
typedef enum {
    LINAC_PATH_AUTO = 0,   /* the fastest path measured on GB300 for the size:
                              LINAC_PATH_HYBRID when m and n are both at least
                              16384, LINAC_PATH_PLAIN otherwise */
    LINAC_PATH_PLAIN = 1,  /* CUDA cores: lazy signed 64-bit accumulation */
    LINAC_PATH_LIMB = 2,   /* integer tensor pipe: four u8 limbs per residue */
    LINAC_PATH_CRT = 3,    /* integer tensor pipe: residues modulo nine small
                              moduli (s8), exact Chinese-remainder
                              reconstruction of each output */
    LINAC_PATH_HYBRID = 4  /* both at once: CUDA-core and multi-modular tiles
                              on different warps of one block per SM */
} linac_path;

typedef struct {
    int32_t path;          /* linac_path */
    int32_t nb;            /* panel width; 0 = automatic (must be a multiple of 16, <= 128) */
    int32_t validate;      /* nonzero: check every entry is in [0, p) first */
    int32_t reserved;
} linac_options;

/*
 * linac_rref -- in-place reduced row-echelon form (section 3.2; section 2.3
 * for the output shape).
 *   d_A       m x n matrix, row-major, leading dimension ld; overwritten by its
 *             RREF: row t < rank has a 1 in column d_pivots[t], zeros in every
 *             other pivot column and in every column left of its pivot; rows
 *             rank..m-1 are zero.
 *   d_rank    one int32_t: the rank.
 *   d_pivots  min(m, n) int32_t: pivot columns in increasing order, -1 after
 *             the rank.
 * Pivots are searched over all n columns, as the paper's column loop does
 * (section 3.2, "Looping"), so an inconsistent augmented column becomes a
 * pivot (section 5.2).
 * Errors: LINAC_ERR_ARG (m or n < 0, null pointers with m*n > 0, ld < n),
 * LINAC_ERR_ALIGN, LINAC_ERR_PRIME, LINAC_ERR_NOMEM, LINAC_ERR_CUDA.
 */
linac_status linac_rref(uint32_t *d_A, int64_t m, int64_t n, int64_t ld, uint32_t p,
                        int32_t *d_rank, int32_t *d_pivots, cudaStream_t stream);

/*
 * linac_rref_noalloc -- linac_rref for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant.
 * linac_rref obtains its scratch with cudaMalloc on first use; callers whose
 * own pool allocator owns the whole device, latency-critical loops that
 * cannot absorb cudaMalloc's implicit synchronisation, and plugins hosted by
 * processes that forbid foreign device allocations cannot allow that.  This
 * entry point allocates nothing (with profiling off, the default): all
 * scratch is one fixed 4 MiB device array inside the library, reserved on
 * every device that loads it until the process exits.
 *   Same arguments, results and errors as linac_rref (plain CUDA-core
 *   update, default panel width), except:
 *   - m <= 2048 and n <= 2048, otherwise LINAC_ERR_UNSUPPORTED;
 *   - the first call on a device looks up the array's device address; make
 *     it before any stream capture on that device;
 *   - all calls share the array: calls that overlap on the GPU race and must
 *     be serialised by the caller;
 *   - a device-side failure (a bounded wait that gave up, see
 *     linac_set_wait_limit) is not reported by linac_last_device_status:
 *     *d_rank is then set to minus the status (-6 for LINAC_ERR_TIMEOUT),
 *     and the matrix and pivots are undefined.
 */
linac_status linac_rref_noalloc(uint32_t *d_A, int64_t m, int64_t n, int64_t ld, uint32_t p,
                                int32_t *d_rank, int32_t *d_pivots, cudaStream_t stream);

/*
 * linac_rref_host -- linac_rref of a matrix in page-locked HOST memory, with
 * the transfers inside the call: the matrix is copied to library scratch on
 * the device, reduced there exactly as linac_rref reduces it (section 3.2;
 * default options), and copied back in place.
 *   h_A       m x n, row-major, leading dimension ld (a multiple of 4, start
 *             16-byte aligned), in page-locked host memory (cudaHostAlloc or
 *             cudaHostRegister); overwritten by its RREF.
 *   h_rank    one int32_t, h_pivots min(m, n) int32_t (-1 after the rank):
 *             also page-locked host memory.
 * The call is asynchronous on `stream` like every other entry point: read
 * the outputs after synchronising it.  The copies are made by the SMs
 * through the host memory's device mapping rather than by the copy engines,
 * whose host-to-device rate drops after sustained GPU work on GB300.
 * Scratch: m * ld * 4 bytes plus the pivots, per stream (allocated on first
 * use as for linac_rref).  The paper has no counterpart (its matrices are
 * copied to the GPU by the Python layer, section 2.3).
 * Errors: as linac_rref; LINAC_ERR_ARG also when a pointer is not page-locked
 * host memory.
 */
linac_status linac_rref_host(uint32_t *h_A, int64_t m, int64_t n, int64_t ld, uint32_t p,
                             int32_t *h_rank, int32_t *h_pivots, cudaStream_t stream);

/* linac_rref with options (NULL = defaults).  ncols_search limits the pivot
 * search to columns [0, ncols_search) while still reducing all n columns
 * (pass n for plain RREF). */
linac_status linac_rref_ex(uint32_t *d_A, int64_t m, int64_t n, int64_t ld, uint32_t p,
                           int64_t ncols_search, int32_t *d_rank, int32_t *d_pivots,
                           const linac_options *opts, cudaStream_t stream);

/*
 * linac_solve -- particular solutions of A X = B over Z/pZ (section 5.2).
 *   d_A  m x nA (ldA), d_B m x k (ldB): read only.
 *   d_X  nA x k (ldX): X[pivots[t]][j] = reduced B[t][j], free variables 0
 *        (section 5.2: the particular solution sets the free variables to
 *        zero); an inconsistent column j of X is all zero.
 *   d_consistent  k bytes: 1 iff rank(A) == rank(A | b_j) (section 5.2).
 *   d_rank, d_pivots  rank of A and its pivot columns (min(m, nA) entries,
 *        -1 after the rank).
 * The augmented matrix [A | B] is reduced in library scratch memory with the
 * pivot search restricted to A's columns.  Same errors as linac_rref;
 * ldX must be >= k (a multiple of 4 is not required for X).
 */
linac_status linac_solve(const uint32_t *d_A, int64_t m, int64_t nA, int64_t ldA,
                         const uint32_t *d_B, int64_t k, int64_t ldB, uint32_t p,
                         uint32_t *d_X, int64_t ldX, uint8_t *d_consistent,
                         int32_t *d_rank, int32_t *d_pivots, cudaStream_t stream);

/* linac_solve with options (NULL = defaults). */
linac_status linac_solve_ex(const uint32_t *d_A, int64_t m, int64_t nA, int64_t ldA,
                            const uint32_t *d_B, int64_t k, int64_t ldB, uint32_t p,
                            uint32_t *d_X, int64_t ldX, uint8_t *d_consistent,
                            int32_t *d_rank, int32_t *d_pivots,
                            const linac_options *opts, cudaStream_t stream);

/*
 * linac_lup -- LUP factorisation P A = L U over Z/pZ, the option section 6
 * ("Conclusions and Outlook") names beside the rank decomposition.  The
 * elimination is the column loop of section 3.2 applied only to the rows not
 * yet used as pivots, without rescaling; the pivot of each column is the
 * lowest-index row, in the original order, among those rows with a nonzero
 * entry there.  This makes P, L and U unique:
 *   d_A      m x n (ldA), read only.
 *   d_perm   m int32: row i of P A is row d_perm[i] of A; the pivot rows come
 *            first in pivot order, then the other rows in increasing order.
 *   d_L      m x min(m, n) (ldL): the first min(m, n) columns of the m x m
 *            unit lower triangular factor (L[i][i] = 1; L[i][t] for i > t,
 *            t < rank is the multiplier row d_perm[i] took for pivot t;
 *            column t >= rank is the unit vector e_t).  The remaining columns
 *            of the m x m factor are those of the identity.
 *   d_U      m x n (ldU): row-echelon form; row t < rank is zero left of
 *            d_pivots[t] and nonzero there; rows rank..m-1 are zero.
 *   d_rank, d_pivots  rank and pivot columns (min(m, n) entries, -1 after
 *            the rank), the same as linac_rref's.
 * Scratch: about (m + 128) * n * 4 + m * 1.1 KB bytes per stream.  Errors: as
 * linac_rref; LINAC_ERR_ARG also for ldL < min(m, n) or ldU < n.
 */
linac_status linac_lup(const uint32_t *d_A, int64_t m, int64_t n, int64_t ldA, uint32_t p,
                       uint32_t *d_L, int64_t ldL, uint32_t *d_U, int64_t ldU, int32_t *d_perm,
                       int32_t *d_rank, int32_t *d_pivots, cudaStream_t stream);

/* Flags for linac_rref_batched. */
#define LINAC_SHARED_PATTERN 1u  /* all systems share one pivot pattern: find it
                                    with one probe elimination, reuse it, and fall
                                    back to a full search for any system where a
                                    reused pivot vanishes */

/*
 * linac_rref_batched -- in-place RREF of `batch` independent systems in one
 * launch sequence (no host synchronisation; capturable in a CUDA graph once
 * the scratch buffer exists).  The paper motivates many small systems by
 * evaluating polynomial ansatze at many points (section 3.3); each system is
 * reduced exactly as linac_rref would.
 *   d_data        packed matrices; system s is d_m[s] x d_n[s] with leading
 *                 dimension d_ld[s] (a multiple of 4) starting at element
 *                 d_offsets[s] (a multiple of 4).
 *   d_nsearch     per-system pivot-search limit (NULL = all columns).
 *   d_ranks       batch int32_t ranks.
 *   d_pivots      pivot columns of system s at d_pivots + d_piv_offsets[s]
 *                 (min(m, n) entries each, -1 after the rank).
 *   d_status      batch int32_t per-system status (NULL = not reported):
 *                 0 ok; with LINAC_SHARED_PATTERN, bit 8 (0x100) marks a
 *                 system that needed the full pivot search.
 *   max_m, max_n  upper bounds of d_m and d_n (host values, used to size the
 *                 launches); m > 1024 or n > 1024 is rejected.
 * Systems are counting-sorted by row count on the device and reduced one per
 * thread block, largest first, in per-size-bucket persistent launches whose
 * panel widths come from linac_batched_tune (or defaults).  With
 * LINAC_SHARED_PATTERN, system 0 is the probe: its pivot rows and columns are
 * reused for every system of the same shape reduced after them, and a system
 * whose reused pivot vanishes (or whose result leaves echelon form) is reduced
 * again with the search, starting from its partially reduced rows (row
 * operations preserve the RREF).  For batches larger than four times the
 * number of SMs the probe runs beside the first systems, which are reduced
 * with the search until its pattern is published; smaller batches run the
 * probe first.
 * Errors: as linac_rref; LINAC_ERR_UNSUPPORTED for sizes above the limits.
 */
linac_status linac_rref_batched(uint32_t *d_data, const int64_t *d_offsets,
                                const int32_t *d_m, const int32_t *d_n, const int32_t *d_ld,
                                const int32_t *d_nsearch, int32_t batch,
                                int32_t max_m, int32_t max_n, uint32_t p, uint32_t flags,
                                int32_t *d_ranks, int32_t *d_pivots, const int64_t *d_piv_offsets,
                                int32_t *d_status, cudaStream_t stream);

/*
 * linac_batched_tune -- autotuner of linac_rref_batched's panel width per
 * size bucket (row counts <= 64, 128, 256, 512, 1024).  For every bucket it
 * times each panel width that fits the GPU's shared memory (16, 32, 64) on
 * synthetic systems of that bucket's sizes (mod p) and keeps the fastest for
 * the current device; later linac_rref_batched calls on this device use the
 * table.  Allocates and frees its own buffers and synchronises `stream`: call
 * it once at start-up, outside any stream capture.  nb_out (5 entries, may
 * be NULL) receives the chosen widths.  Untuned buckets use 32.
 */
linac_status linac_batched_tune(uint32_t p, int32_t *nb_out, cudaStream_t stream);

/* Current panel width per size bucket (5 entries). */
linac_status linac_batched_panel_widths(int32_t *nb_out);

/* Sets the panel width per size bucket for the current device (5 entries,
 * each 16, 32 or 64, or 0 for the default 32), e.g. to reuse widths that
 * linac_batched_tune chose in an earlier run.  Errors: LINAC_ERR_ARG (another
 * value), LINAC_ERR_UNSUPPORTED (a width whose shared memory does not fit the
 * device for that bucket); nothing is changed on error. */
linac_status linac_batched_set_panel_widths(const int32_t *nb);

/*
 * linac_load_matrix -- build a linear system from monomials evaluated at
 * sampling points (section 3.3, "Building linear systems on GPUs"; section
 * 2.3, cuda_load_matrix):
 *     A[r][c] = prod_{t < d} bases[r][lindices[c][t]]  mod p.
 *   d_bases     n_rows x n_basis residues in [0, p), leading dimension
 *               ld_bases: row r holds the basis-variable values of point r.
 *   d_lindices  n_cols x d int32 indices into a row of bases (row-major,
 *               contiguous): column c is the monomial whose factors they
 *               name (pad lower-degree monomials with an index whose basis
 *               value is 1, as the paper does).  d = 0 gives all ones.
 *   d_A         n_rows x n_cols output, leading dimension ldA (any alignment).
 * An index outside [0, n_basis) is not read: its entry is written as 0 and
 * the device status word is set to LINAC_ERR_RANGE (linac_last_device_status).
 * Errors: LINAC_ERR_ARG (negative sizes, ld too small, null pointers),
 * LINAC_ERR_PRIME, LINAC_ERR_UNSUPPORTED (more than 524280 rows).
 */
linac_status linac_load_matrix(const uint32_t *d_bases, int64_t n_rows, int64_t n_basis, int64_t ld_bases,
                               const int32_t *d_lindices, int64_t n_cols, int32_t d, uint32_t p,
                               uint32_t *d_A, int64_t ldA, cudaStream_t stream);

/*
 * linac_matmul -- C = A B mod p for canonical residues: A is m x K (ldA),
 * B is K x n (ldB), C is m x n (ldC), all row-major, any alignment.  Exact:
 * the products of balanced residues accumulate in signed 64-bit registers
 * with periodic folds, and every output is reduced once.  With the monomial
 * values of many points as A and a template's coefficients as B, one call
 * evaluates a template of polynomial entries at every point (section 3.3); it
 * also states the identities A = C R and A K = 0 of section 5.1 on the device.
 * Errors: LINAC_ERR_ARG, LINAC_ERR_PRIME, LINAC_ERR_UNSUPPORTED (m above
 * 8388480).
 */
linac_status linac_matmul(const uint32_t *d_A, int64_t m, int64_t K, int64_t ldA,
                          const uint32_t *d_B, int64_t n, int64_t ldB, uint32_t p,
                          uint32_t *d_C, int64_t ldC, cudaStream_t stream);

/*
 * linac_null_space -- canonical basis of the null space read off an RREF
 * (section 5.1): ker(A) = ker(R); the non-pivot columns are the free
 * variables and their coefficients are fixed to minus the identity.
 *   d_R, m, n, ld   the RREF (as linac_rref leaves it); d_rank, d_pivots its
 *                   rank and pivot columns (device, as linac_rref writes them).
 *   d_K             n x kcols output (leading dimension ldK): column q < the
 *                   nullity n - rank belongs to the q-th free column f_q and
 *                   holds p - 1 (that is, -1) in row f_q, R[t][f_q] in row
 *                   pivots[t], and 0 elsewhere, so A K = 0; columns at or
 *                   beyond the nullity are zero.
 *   d_free          n int32: the free columns in increasing order, -1 after
 *                   the nullity.
 *   d_nullity       one int32: n - rank.
 * Nothing is synchronised: kcols is the caller's bound on the nullity (n
 * always suffices).  If the nullity exceeds kcols, the first kcols columns are
 * written and the device status word is set to LINAC_ERR_RANGE.  Uses n * 4
 * bytes of library scratch.
 * Errors: LINAC_ERR_ARG, LINAC_ERR_PRIME, LINAC_ERR_NOMEM.
 */
linac_status linac_null_space(const uint32_t *d_R, int64_t m, int64_t n, int64_t ld,
                              const int32_t *d_rank, const int32_t *d_pivots, uint32_t p,
                              uint32_t *d_K, int64_t kcols, int64_t ldK, int32_t *d_free,
                              int32_t *d_nullity, cudaStream_t stream);

/*
 * linac_rank_factor -- the left factor of the rank factorisation A = C R
 * (section 5.1): C = A[:, J], the pivot columns J of the ORIGINAL matrix
 * (keep a copy of A: linac_rref overwrites it), with R the RREF's first
 * rank rows.
 *   d_A, m, n, ld   the original matrix; d_rank, d_pivots from linac_rref.
 *   d_C             m x ccols output (ldC): column t < rank is A's column
 *                   pivots[t]; columns rank..ccols-1 are zero (ccols =
 *                   min(m, n) always suffices).
 * Errors: LINAC_ERR_ARG.
 */
linac_status linac_rank_factor(const uint32_t *d_A, int64_t m, int64_t n, int64_t ld,
                               const int32_t *d_rank, const int32_t *d_pivots,
                               uint32_t *d_C, int64_t ccols, int64_t ldC, cudaStream_t stream);

/* Scratch bytes linac_rref_ex needs for an m x n problem with these options
 * (the library allocates them itself; exposed for capacity planning). */
/*
 * uint64 residues: primes that do not fit 32 bits.  Section 2.3 ("Basic
 * Usage") selects uint64 storage for 2^32 - 1 < p <= 2^64 - 1; these entry
 * points accept every odd prime 3 <= p < 2^64 (so small primes can be
 * checked against the uint32 entry points).  Conventions as above, except:
 *   - matrices hold uint64_t residues in [0, p); the leading dimension is a
 *     multiple of 2 elements and the matrix starts 16-byte aligned (rows are
 *     read two residues at a time, section 3.4 "Optimisations");
 *   - the elimination is the same blocked Gauss-Jordan (section 3.2) with
 *     32-column panels, Montgomery arithmetic modulo 2^64 and exact 160-bit
 *     accumulation in the trailing update; the panel's pivots come from a
 *     window of the first 48 remaining rows, or from a search over all
 *     remaining rows when the window lacks one;
 *   - scratch: 32 (3 m + n) * 8 bytes plus a few KB, per stream
 *     (linac_workspace64_bytes), allocated on first use as for linac_rref;
 *   - the panel kernels run on a second, highest-priority stream that the
 *     library creates on first use per (device, stream) and forks from and
 *     joins back to `stream` with events; as with scratch memory, make one
 *     uncaptured call on a stream before capturing calls on it;
 *   - no tensor-core path: the options' path and nb must be 0.
 */

/* In-place RREF of the m x n uint64 matrix (same outputs as linac_rref). */
linac_status linac_rref64(uint64_t *d_A, int64_t m, int64_t n, int64_t ld, uint64_t p,
                          int32_t *d_rank, int32_t *d_pivots, cudaStream_t stream);

/* linac_rref64 with a pivot-search limit [0, ncols_search) and options
 * (NULL = defaults; only `validate` may be set: it checks every entry is
 * below p first and sets the device status word to LINAC_ERR_RANGE). */
linac_status linac_rref64_ex(uint64_t *d_A, int64_t m, int64_t n, int64_t ld, uint64_t p,
                             int64_t ncols_search, int32_t *d_rank, int32_t *d_pivots,
                             const linac_options *opts, cudaStream_t stream);

/* Particular solutions of A X = B with uint64 residues (section 5.2); same
 * arguments and results as linac_solve.  [A | B] is reduced in library
 * scratch (m * (nA + k) * 8 bytes); A and B are not modified. */
linac_status linac_solve64(const uint64_t *d_A, int64_t m, int64_t nA, int64_t ldA,
                           const uint64_t *d_B, int64_t k, int64_t ldB, uint64_t p,
                           uint64_t *d_X, int64_t ldX, uint8_t *d_consistent,
                           int32_t *d_rank, int32_t *d_pivots, cudaStream_t stream);

/* linac_null_space and linac_rank_factor (section 5.1) for uint64 residues:
 * same arguments, outputs and errors, with uint64 matrices (d_R, d_K, d_A,
 * d_C) and p an odd prime below 2^64 (the free columns' -1 is p - 1). */
linac_status linac_null_space64(const uint64_t *d_R, int64_t m, int64_t n, int64_t ld,
                                const int32_t *d_rank, const int32_t *d_pivots, uint64_t p,
                                uint64_t *d_K, int64_t kcols, int64_t ldK, int32_t *d_free,
                                int32_t *d_nullity, cudaStream_t stream);
linac_status linac_rank_factor64(const uint64_t *d_A, int64_t m, int64_t n, int64_t ld,
                                 const int32_t *d_rank, const int32_t *d_pivots,
                                 uint64_t *d_C, int64_t ccols, int64_t ldC, cudaStream_t stream);

/* Scratch bytes linac_rref64 uses for an m x n matrix (0 for negative sizes). */
size_t linac_workspace64_bytes(int64_t m, int64_t n);

size_t linac_workspace_bytes(int64_t m, int64_t n, const linac_options *opts);

/* Status word written by device-side checks of the most recent call on this
 * host thread (LINAC_OK when none fired); synchronises `stream`. */
linac_status linac_last_device_status(cudaStream_t stream);

/* Human-readable name of a status code (static string). */
const char *linac_status_string(linac_status s);

/* Profiling.  When enabled, every kernel launch of the library is bracketed
 * by CUDA events recorded on its own stream, accumulated per kernel class
 * ("panel", "trsm", "update_plain", ...).  linac_profile_read synchronises
 * the recorded events and fills up to max_entries entries (classes with at
 * least one timed launch), returning how many were written.  Launches are
 * counted whether or not profiling is enabled. */
typedef struct {
    const char *name;      /* static string */
    long long launches;
    double total_ms;
} linac_profile_entry;

void linac_profile_enable(int on);
void linac_profile_reset(void);
int linac_profile_read(linac_profile_entry *out, int max_entries);
long long linac_launch_count(void);

/*
 * Failure detection.  Every wait of one thread block on others (the arrival
 * barrier of the dense elimination's full-height pivot search, section 3.2
 * "Pivoting") is bounded: after the limit it records LINAC_ERR_TIMEOUT in the
 * device status word (linac_last_device_status; for linac_rref_noalloc, a
 * negative rank) and every block returns, so a fault elsewhere never hangs
 * the device.  The results of a call that timed out are not defined; the
 * next call starts afresh.
 *
 * linac_set_wait_limit -- limit of those waits in SM clock cycles for every
 * later launch from this process (0 restores the default of 4e9 cycles,
 * about 2 s).  Errors: LINAC_ERR_ARG for a negative value.
 */
linac_status linac_set_wait_limit(int64_t cycles);

/*
 * linac_debug_inject_wait_failure -- test support (the paper has no
 * counterpart).  While on, the arrival barrier of the full-height pivot
 * search waits for one more arrival than its blocks make: nothing ever
 * completes it, so every block's wait runs out after the wait limit and the
 * call reports LINAC_ERR_TIMEOUT.  It lets tests check the timeout path
 * without faulting or hanging the GPU.  Off by default; 0 turns it off.
 */
void linac_debug_inject_wait_failure(int32_t on);

/* Library version as major*10000 + minor*100 + patch. */
int32_t linac_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LINAC_H */
