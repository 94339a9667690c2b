// batched.cu -- many independent systems of uneven size, each reduced to RREF
// by one thread block, in persistent launches with no inter-block traffic.
//
// Per system the block runs the same blocked Gauss-Jordan elimination as the
// dense driver (paper section 3.2, blocked by panels of NB columns):
//   panel    fraction-free elimination of the panel columns of the rows not
//            yet used (shared memory), recording pivot rows, pivot columns and
//            multipliers -- or, in shared-pattern mode, the pivot rows and
//            columns of a probe system and an elimination of the k pivot rows
//            only;
//   inverses batched inverses of the k pivot heads;
//   E        the k x k matrix E = G^{-1} (G = the pivot rows at the pivot
//            columns), obtained by running the panel's fraction-free
//            recurrence, the scaling and the back substitution on the identity;
//   tiles    for each 64-column tile right of the panel start: R = E W (W the
//            pivot rows' tile), move the displaced rows, and update every
//            other row: A[d] <- A[d] - F[d] R with lazy signed 64-bit
//            accumulation (F = the rows' entries at the pivot columns).
// Systems are counting-sorted by row count on the device and launched per
// size bucket (shared memory is sized by the bucket's largest system); within
// a bucket blocks pull systems, largest first, from a device work counter.
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "linac_host.h"
#include "profile.h"

namespace linac {

constexpr int BT_THREADS = 256;
constexpr int BT_TB = 64;              // column tile of the update
constexpr int BT_NBUCKETS = 5;         // m <= 64, 128, 256, 512, 1024
// largest row count of bucket b: 64, 128, 256, 512, 1024
__host__ __device__ constexpr int bt_bucket_max(int b) { return 64 << b; }
constexpr int BT_FLAG_FALLBACK = 0x100;

// Per-call device scratch of the batched driver.
struct BatchScratch {
    unsigned int counters[2 * BT_NBUCKETS];   // work counters (search pass, fallback pass)
    int bbeg[BT_NBUCKETS], bend[BT_NBUCKETS]; // bucket segments of `order`
    int probe_m, probe_n, probe_ns;           // shape of the probe system
    int nfallback;                            // systems that left the shared pattern
    int pattern_ok;                           // the probe produced a usable pattern
    int pattern_k[1024 / 16 + 1];             // pivots per panel of the probe
};

// ---------------------------------------------------------------------------
// Sorting by row count (one block): order[] lists systems by bucket, and by
// decreasing m within a bucket.

__global__ void __launch_bounds__(1024)
batch_sort_kernel(const int32_t* __restrict__ dm, int batch, int32_t* __restrict__ order,
                  BatchScratch* bs, int skip_first) {
    __shared__ int cnt[1025];
    __shared__ int pos[1025];
    for (int i = threadIdx.x; i < 1025; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int s = threadIdx.x + skip_first; s < batch; s += blockDim.x) atomicAdd(&cnt[min(max(dm[s], 0), 1024)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        // descending m: pos[v] = number of systems with a key above v
        int acc = 0;
        for (int v = 1024; v >= 0; --v) {
            pos[v] = acc;
            acc += cnt[v];
        }
        // bucket b holds m in (max[b-1], max[b]]: positions [pos[max[b]], pos[max[b-1]])
        for (int b = 0; b < BT_NBUCKETS; ++b) {
            bs->bbeg[b] = pos[bt_bucket_max(b)];
            bs->bend[b] = b ? pos[bt_bucket_max(b - 1)] : acc;
        }
        for (int i = 0; i < 2 * BT_NBUCKETS; ++i) bs->counters[i] = 0;
        bs->nfallback = 0;
    }
    __syncthreads();
    for (int s = threadIdx.x + skip_first; s < batch; s += blockDim.x) {
        const int v = min(max(dm[s], 0), 1024);
        order[atomicAdd(&pos[v], 1)] = s;
    }
}

// ---------------------------------------------------------------------------
// Shared-memory layout of one block (sized by the bucket's largest m).

struct BtLayout {
    int mmax, ldF;
    size_t off_ft, off_p, off_pu, off_e, off_isp, total;
};

__host__ __device__ inline BtLayout bt_layout(int mmax, int nb) {
    BtLayout L;
    L.mmax = mmax;
    L.ldF = (mmax + 3) / 4 * 4;
    size_t o = 0;
    L.off_ft = o;  o += (size_t)nb * L.ldF * 4;                       // Ft[t][row], balanced
    L.off_p = o;
    const size_t panel = (size_t)mmax * (nb + 1) * 4;                  // panel slab
    const size_t tiles = (size_t)3 * nb * BT_TB * 4;                   // V, X, R tiles
    o += panel > tiles ? panel : tiles;
    L.off_pu = o;  o += (size_t)nb * nb * 4;                           // pivot rows' panel entries
    L.off_e = o;   o += (size_t)nb * nb * 4;                           // E = G^{-1}
    L.off_isp = o; o += (size_t)((mmax + 15) / 16 * 16);              // pivot flags
    L.total = (o + 15) / 16 * 16;
    return L;
}

template <int NB>
struct BtSmall {
    int J[NB], Pi[NB], own[NB], srcs[NB], dsts[NB];
    uint32_t hinv[NB], hs[NB];
    int red[BT_THREADS / 32];
    int s_min, s_sys, s_npairs, s_fail;
};

// Lowest index i in [0, cnt) with pred(i), block-wide (INT_MAX if none).
template <int NB, typename Pred>
__device__ __forceinline__ int block_first(int cnt, Pred pred, BtSmall<NB>& sm) {
    int ci = INT_MAX;
    for (int i = threadIdx.x; i < cnt; i += BT_THREADS)
        if (pred(i)) { ci = i; break; }
    for (int o = 16; o; o >>= 1) ci = min(ci, __shfl_xor_sync(0xffffffffu, ci, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm.red[warp] = ci;
    __syncthreads();
    if (warp == 0) {
        int v = lane < BT_THREADS / 32 ? sm.red[lane] : INT_MAX;
        for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sm.s_min = v;
    }
    __syncthreads();
    return sm.s_min;
}

// Reduce system A (m x n, leading dimension ld) in place.  mode 0: pivot
// search; mode 1: reuse the probe's pattern (pat_J / pat_Pi / pat_k per
// panel) and report failure (returns false) when a reused pivot vanishes or
// the result leaves echelon form.  Returns true on success; writes rank and
// pivots.
template <int NB>
__device__ bool bt_reduce(uint32_t* __restrict__ A, int m, int n, int64_t ld, int ns, const Field& f,
                          int32_t* __restrict__ piv, int* rank_out, uint8_t* smem, const BtLayout& L,
                          BtSmall<NB>& sm, int mode, const int32_t* pat_J, const int32_t* pat_Pi,
                          const int* pat_k, int32_t* rec_J, int32_t* rec_Pi, int* rec_k) {
    int32_t* Ft = (int32_t*)(smem + L.off_ft);
    uint32_t* P = (uint32_t*)(smem + L.off_p);
    uint32_t* PU = (uint32_t*)(smem + L.off_pu);
    uint32_t* E = (uint32_t*)(smem + L.off_e);
    unsigned char* isp = smem + L.off_isp;
    uint32_t* V = P;                                  // tiles alias the panel slab
    uint32_t* X = P + NB * BT_TB;
    int32_t* Rt = (int32_t*)(P + 2 * NB * BT_TB);
    const int tid = threadIdx.x;
    const int SW = NB + 1;

    const int npiv = min(m, ns);
    for (int i = tid; i < npiv; i += BT_THREADS) piv[i] = -1;
    int r = 0;
    int panel = 0;
    for (int c0 = 0; c0 < ns && r < m; c0 += NB, ++panel) {
        const int w = min(NB, ns - c0);
        int k = 0;
        if (mode == 0) {
            const int rows = m - r;
            for (int e = tid; e < rows * w; e += BT_THREADS) {
                const int i = e / w, j = e % w;
                P[i * SW + j] = A[(int64_t)(r + i) * ld + c0 + j];
            }
            for (int i = tid; i < rows; i += BT_THREADS) isp[i] = 0;
            __syncthreads();
            for (int cc = 0; cc < w; ++cc) {
                const int q = block_first<NB>(rows, [&](int i) { return !isp[i] && P[i * SW + cc] != 0; }, sm);
                if (q == INT_MAX) continue;
                if (tid == 0) {
                    isp[q] = 1;
                    sm.J[k] = c0 + cc;
                    sm.Pi[k] = r + q;
                    sm.own[k] = q;
                }
                const uint32_t h = P[q * SW + cc];
                for (int i = tid / 32; i < rows; i += BT_THREADS / 32) {
                    if (i == q || isp[i]) continue;
                    uint32_t* row = P + i * SW;
                    const uint32_t fi = row[cc];
                    if (fi == 0) continue;
                    const uint32_t nf = f.p - fi;
                    for (int j = cc + 1 + (tid & 31); j < w; j += 32)
                        row[j] = mul2add(h, row[j], nf, P[q * SW + j], f);
                }
                ++k;
                __syncthreads();
            }
            for (int e = tid; e < k * w; e += BT_THREADS) {
                const int t = e / w, j = e % w;
                PU[t * NB + j] = P[sm.own[t] * SW + j];
            }
            if (rec_k && tid == 0) {
                rec_k[panel] = k;
                for (int t = 0; t < k; ++t) {
                    rec_J[panel * NB + t] = sm.J[t];
                    rec_Pi[panel * NB + t] = sm.Pi[t];
                }
            }
        } else {
            // shared pattern: pivot rows and columns of the probe; eliminate the
            // k pivot rows among themselves (the same recurrence the search
            // would have applied to them)
            k = pat_k[panel];
            for (int t = tid; t < k; t += BT_THREADS) {
                sm.J[t] = pat_J[panel * NB + t];
                sm.Pi[t] = pat_Pi[panel * NB + t];
            }
            if (tid == 0) sm.s_fail = 0;
            __syncthreads();
            for (int e = tid; e < k * w; e += BT_THREADS) {
                const int t = e / w, j = e % w;
                PU[t * NB + j] = A[(int64_t)sm.Pi[t] * ld + c0 + j];
            }
            __syncthreads();
            for (int s = 0; s < k; ++s) {
                const int cs = sm.J[s] - c0;
                const uint32_t h = PU[s * NB + cs];
                if (h == 0) { if (tid == 0) sm.s_fail = 1; }
                for (int t = s + 1 + tid / 32; t < k; t += BT_THREADS / 32) {
                    uint32_t* row = PU + t * NB;
                    const uint32_t fi = row[cs];
                    if (fi == 0 || h == 0) continue;
                    const uint32_t nf = f.p - fi;
                    for (int j = cs + 1 + (tid & 31); j < w; j += 32)
                        row[j] = mul2add(h, row[j], nf, PU[s * NB + j], f);
                }
                __syncthreads();
            }
            if (sm.s_fail) return false;
        }
        if (k == 0) continue;
        // multipliers F (original entries at the pivot columns), inverses, E
        for (int e = tid; e < k * m; e += BT_THREADS) {
            const int t = e / m, i = e % m;
            Ft[t * L.ldF + i] = to_balanced(A[(int64_t)i * ld + sm.J[t]], f);
        }
        for (int t = tid; t < k; t += BT_THREADS) {
            sm.hs[t] = PU[t * NB + (sm.J[t] - c0)];
            sm.hinv[t] = inverse_mod(sm.hs[t], f.p);
        }
        for (int e = tid; e < k * k; e += BT_THREADS) E[(e / k) * NB + (e % k)] = (e / k == e % k) ? 1u : 0u;
        if (tid == 0) {
            // move plan: rows of [r, r+k) without a pivot go to the pivot rows' old places
            unsigned char occ[NB];
            for (int d = 0; d < k; ++d) occ[d] = 0;
            for (int t = 0; t < k; ++t)
                if (sm.Pi[t] >= r && sm.Pi[t] < r + k) occ[sm.Pi[t] - r] = 1;
            int a = 0, b = 0;
            for (int d = 0; d < k; ++d)
                if (!occ[d]) sm.srcs[a++] = r + d;
            for (int t = 0; t < k; ++t)
                if (sm.Pi[t] < r || sm.Pi[t] >= r + k) sm.dsts[b++] = sm.Pi[t];
            sm.s_npairs = a;
        }
        __syncthreads();
        // E <- forward fraction-free recurrence, scaling, back substitution
        for (int s = 0; s + 1 < k; ++s) {
            const uint32_t h = sm.hs[s];
            const int cs = sm.J[s] - c0;
            for (int e = tid; e < (k - 1 - s) * k; e += BT_THREADS) {
                const int t = s + 1 + e / k, j = e % k;
                const uint32_t fts = PU[t * NB + cs];
                if (fts) E[t * NB + j] = mul2add(h, E[t * NB + j], f.p - fts, E[s * NB + j], f);
            }
            __syncthreads();
        }
        for (int e = tid; e < k * k; e += BT_THREADS) {
            const int t = e / k, j = e % k;
            E[t * NB + j] = mulmod(E[t * NB + j], sm.hinv[t], f);
        }
        __syncthreads();
        for (int s = k - 1; s >= 1; --s) {
            const int cs = sm.J[s] - c0;
            for (int e = tid; e < s * k; e += BT_THREADS) {
                const int t = e / k, j = e % k;
                const uint32_t c = mulmod(PU[t * NB + cs], sm.hinv[t], f);
                if (c) E[t * NB + j] = mul2add(1u, E[t * NB + j], f.p - c, E[s * NB + j], f);
            }
            __syncthreads();
        }
        const int npairs = sm.s_npairs;
        for (int e = tid; e < npairs * k; e += BT_THREADS) {
            const int a = e / k, t = e % k;
            Ft[t * L.ldF + sm.dsts[a]] = Ft[t * L.ldF + sm.srcs[a]];
        }
        // E to balanced form for the tile products
        for (int e = tid; e < k * k; e += BT_THREADS) {
            const int t = e / k, j = e % k;
            E[t * NB + j] = (uint32_t)to_balanced(E[t * NB + j], f);
        }
        __syncthreads();
        // column tiles
        for (int j0 = c0; j0 < n; j0 += BT_TB) {
            const int tw = min(BT_TB, n - j0);
            for (int e = tid; e < k * tw; e += BT_THREADS) {
                const int t = e / tw, j = e % tw;
                V[t * BT_TB + j] = (uint32_t)to_balanced(A[(int64_t)sm.Pi[t] * ld + j0 + j], f);
            }
            for (int e = tid; e < npairs * tw; e += BT_THREADS) {
                const int a = e / tw, j = e % tw;
                X[a * BT_TB + j] = A[(int64_t)sm.srcs[a] * ld + j0 + j];
            }
            __syncthreads();
            // R = E V (balanced operands, lazy signed accumulation)
            for (int e = tid; e < k * tw; e += BT_THREADS) {
                const int t = e / tw, j = e % tw;
                int64_t acc = 0;
                for (int s = 0; s < k; ++s) {
                    mac_s64(acc, (int32_t)E[t * NB + s], (int32_t)V[s * BT_TB + j]);
                    if ((s & 3) == 3) acc = fold64_fast(acc, f);
                }
                Rt[t * BT_TB + j] = to_balanced(reduce_signed(acc, f), f);
            }
            for (int e = tid; e < npairs * tw; e += BT_THREADS) {
                const int a = e / tw, j = e % tw;
                A[(int64_t)sm.dsts[a] * ld + j0 + j] = X[a * BT_TB + j];
            }
            __syncthreads();
            // update: rows in [r, r+k) receive R, every other row A -= F R
            const int rgroups = (m + 3) / 4;
            const int cq = (tw + 3) / 4;
            for (int e = tid; e < rgroups * cq; e += BT_THREADS) {
                const int d0 = (e / cq) * 4, jq = (e % cq) * 4;
                int64_t acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
                for (int t = 0; t < k; ++t) {
                    const int4 fv = *reinterpret_cast<const int4*>(Ft + t * L.ldF + d0);
                    const int4 rv = *reinterpret_cast<const int4*>(Rt + t * BT_TB + jq);
                    const int fa[4] = {fv.x, fv.y, fv.z, fv.w};
                    const int rb[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) mac_s64(acc[a][b], fa[a], rb[b]);
                    if ((t & 3) == 3) {
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int b = 0; b < 4; ++b) acc[a][b] = fold64_fast(acc[a][b], f);
                    }
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int d = d0 + a;
                    if (d >= m) continue;
                    uint32_t* row = A + (int64_t)d * ld + j0;
                    const bool prow = d >= r && d < r + k;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int j = jq + b;
                        if (j >= tw) continue;
                        uint32_t v;
                        if (prow) v = from_balanced(Rt[(d - r) * BT_TB + j], f);
                        else v = submod(row[j], reduce_signed(acc[a][b], f), f);
                        row[j] = v;
                        // shared pattern: rows below the new rank must vanish in the panel
                        if (mode == 1 && d >= r + k && j0 + j < c0 + w && v != 0) sm.s_fail = 1;
                    }
                }
            }
            __syncthreads();
        }
        for (int t = tid; t < k; t += BT_THREADS) piv[r + t] = sm.J[t];
        r += k;
        __syncthreads();
        if (mode == 1) {
            // echelon shape: a pivot row is zero left of its pivot within the panel
            for (int e = tid; e < k * w; e += BT_THREADS) {
                const int t = e / w, j = e % w;
                if (c0 + j < sm.J[t] && A[(int64_t)(r - k + t) * ld + c0 + j] != 0) sm.s_fail = 1;
            }
            __syncthreads();
            if (sm.s_fail) return false;
        }
    }
    if (mode == 1 && r < m) {
        // the probe's rank was reached: every remaining row must be zero in
        // the searched columns, or this system has a different pattern
        for (int e = tid; e < (m - r) * ns; e += BT_THREADS) {
            const int i = r + e / ns, j = e % ns;
            if (A[(int64_t)i * ld + j] != 0) sm.s_fail = 1;
        }
        __syncthreads();
        if (sm.s_fail) return false;
    }
    *rank_out = r;
    return true;
}

// Persistent kernel over one bucket.  pass 0: the bucket's systems (search,
// or the shared pattern); pass 1: systems that failed the pattern (search).
template <int NB>
__global__ void __launch_bounds__(BT_THREADS)
batched_kernel(uint32_t* __restrict__ data, const int64_t* __restrict__ offsets, const int32_t* __restrict__ dm,
               const int32_t* __restrict__ dn, const int32_t* __restrict__ dld, const int32_t* __restrict__ dns,
               const int32_t* __restrict__ order, int bucket, int mmax, Field f, int32_t* __restrict__ ranks,
               int32_t* __restrict__ pivots, const int64_t* __restrict__ piv_off, int32_t* __restrict__ sys_status,
               BatchScratch* bs, int pass, int use_pattern, const int32_t* pat_J, const int32_t* pat_Pi,
               int32_t* fallback) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ BtSmall<NB> sm;
    const BtLayout L = bt_layout(mmax, NB);
    int begin, end;
    if (pass == 0) {
        begin = bs->bbeg[bucket];
        end = bs->bend[bucket];
    } else {
        begin = 0;
        end = bs->nfallback;
    }
    unsigned int* counter = &bs->counters[pass * BT_NBUCKETS + bucket];
    if (use_pattern && pass == 0 && !bs->pattern_ok) use_pattern = 0;
    for (;;) {
        if (threadIdx.x == 0) sm.s_sys = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int idx = begin + sm.s_sys;
        __syncthreads();
        if (idx >= end) return;
        const int s = pass == 0 ? order[idx] : fallback[idx];
        const int m = dm[s], n = dn[s];
        if (pass == 1 && mmax < m) continue;           // fallback systems are split by bucket too
        if (pass == 1 && bucket > 0 && m <= bt_bucket_max(bucket - 1)) continue;
        const int ns = dns ? min(dns[s], n) : n;
        uint32_t* A = data + offsets[s];
        int32_t* piv = pivots + piv_off[s];
        int rank = 0;
        bool ok;
        // the pattern applies only to systems shaped like the probe
        const bool same_shape = m == bs->probe_m && n == bs->probe_n && ns == bs->probe_ns;
        if (use_pattern && pass == 0 && !same_shape) {
            ok = false;
            if (threadIdx.x == 0) fallback[atomicAdd(&bs->nfallback, 1)] = s;
        } else if (use_pattern && pass == 0) {
            ok = bt_reduce<NB>(A, m, n, dld[s], ns, f, piv, &rank, smem, L, sm, 1, pat_J, pat_Pi,
                               bs->pattern_k, nullptr, nullptr, nullptr);
            if (!ok && threadIdx.x == 0) fallback[atomicAdd(&bs->nfallback, 1)] = s;
        } else {
            ok = bt_reduce<NB>(A, m, n, dld[s], ns, f, piv, &rank, smem, L, sm, 0, nullptr, nullptr, nullptr,
                               nullptr, nullptr, nullptr);
        }
        __syncthreads();
        if (ok && threadIdx.x == 0) {
            ranks[s] = rank;
            if (sys_status) sys_status[s] = pass == 1 ? BT_FLAG_FALLBACK : 0;
        }
        __syncthreads();
    }
}

// Probe: system 0 with the pivot search, recording its pattern.
template <int NB>
__global__ void __launch_bounds__(BT_THREADS)
batched_probe_kernel(uint32_t* __restrict__ data, const int64_t* __restrict__ offsets, const int32_t* __restrict__ dm,
                     const int32_t* __restrict__ dn, const int32_t* __restrict__ dld, const int32_t* __restrict__ dns,
                     int mmax, Field f, int32_t* __restrict__ ranks, int32_t* __restrict__ pivots,
                     const int64_t* __restrict__ piv_off, int32_t* __restrict__ sys_status, BatchScratch* bs,
                     int32_t* pat_J, int32_t* pat_Pi) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ BtSmall<NB> sm;
    const BtLayout L = bt_layout(mmax, NB);
    const int m = dm[0], n = dn[0];
    const int ns = dns ? min(dns[0], n) : n;
    for (int i = threadIdx.x; i < 1024 / 16 + 1; i += BT_THREADS) bs->pattern_k[i] = 0;
    __syncthreads();
    int rank = 0;
    bt_reduce<NB>(data + offsets[0], m, n, dld[0], ns, f, pivots + piv_off[0], &rank, smem, L, sm, 0, nullptr,
                  nullptr, nullptr, pat_J, pat_Pi, bs->pattern_k);
    __syncthreads();
    if (threadIdx.x == 0) {
        ranks[0] = rank;
        if (sys_status) sys_status[0] = 0;
        bs->probe_m = m;
        bs->probe_n = n;
        bs->probe_ns = ns;
        bs->pattern_ok = 1;
    }
}

// ---------------------------------------------------------------------------
// Host side: per-bucket panel width (autotuned table, see linac_batched_tune)

namespace {
std::mutex g_bt_mu;
int g_bt_nb[64][BT_NBUCKETS];   // 0 = default
}

static int bt_default_nb(int b) { return b >= 4 ? 16 : 32; }

int bt_bucket_nb(int b) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_bt_mu);
    const int v = (dev >= 0 && dev < 64) ? g_bt_nb[dev][b] : 0;
    return v ? v : bt_default_nb(b);
}

void bt_set_bucket_nb(int b, int nb) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_bt_mu);
    if (dev >= 0 && dev < 64 && b >= 0 && b < BT_NBUCKETS) g_bt_nb[dev][b] = nb;
}

template <int NB>
static linac_status launch_bucket(int b, int pass, int use_pattern, uint32_t* d_data, const int64_t* d_offsets,
                                  const int32_t* d_m, const int32_t* d_n, const int32_t* d_ld,
                                  const int32_t* d_nsearch, const int32_t* order, const Field& f,
                                  int32_t* d_ranks, int32_t* d_pivots, const int64_t* d_piv_offsets,
                                  int32_t* d_status, BatchScratch* bs, const int32_t* pat_J,
                                  const int32_t* pat_Pi, int32_t* fallback, cudaStream_t stream) {
    const int mmax = bt_bucket_max(b);
    const BtLayout L = bt_layout(mmax, NB);
    LINAC_CUDA_TRY(cudaFuncSetAttribute(batched_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)L.total));
    int occ = 0;
    LINAC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel<NB>, BT_THREADS, L.total));
    if (occ < 1) return LINAC_ERR_UNSUPPORTED;
    const int grid = occ * sm_count();
    ProfScope ps(stream, use_pattern ? PROF_PATTERN : PROF_BATCHED);
    batched_kernel<NB><<<grid, BT_THREADS, L.total, stream>>>(d_data, d_offsets, d_m, d_n, d_ld, d_nsearch, order, b,
                                                              mmax, f, d_ranks, d_pivots, d_piv_offsets, d_status, bs,
                                                              pass, use_pattern, pat_J, pat_Pi, fallback);
    LINAC_CUDA_TRY(cudaGetLastError());
    return LINAC_OK;
}

static linac_status launch_bucket_nb(int nb, int b, int pass, int use_pattern, uint32_t* d_data,
                                     const int64_t* d_offsets, const int32_t* d_m, const int32_t* d_n,
                                     const int32_t* d_ld, const int32_t* d_nsearch, const int32_t* order,
                                     const Field& f, int32_t* d_ranks, int32_t* d_pivots,
                                     const int64_t* d_piv_offsets, int32_t* d_status, BatchScratch* bs,
                                     const int32_t* pat_J, const int32_t* pat_Pi, int32_t* fallback,
                                     cudaStream_t stream) {
#define LINAC_BT_ARGS b, pass, use_pattern, d_data, d_offsets, d_m, d_n, d_ld, d_nsearch, order, f, d_ranks, \
                      d_pivots, d_piv_offsets, d_status, bs, pat_J, pat_Pi, fallback, stream
    switch (nb) {
        case 16: return launch_bucket<16>(LINAC_BT_ARGS);
        case 32: return launch_bucket<32>(LINAC_BT_ARGS);
        case 64: return launch_bucket<64>(LINAC_BT_ARGS);
        default: return LINAC_ERR_ARG;
    }
#undef LINAC_BT_ARGS
}

size_t bt_shared_bytes(int b, int nb) { return bt_layout(bt_bucket_max(b), nb).total; }

linac_status batched_rref(uint32_t* d_data, const int64_t* d_offsets, const int32_t* d_m,
                          const int32_t* d_n, const int32_t* d_ld, const int32_t* d_nsearch,
                          int32_t batch, int32_t max_m, int32_t max_n, const Field& f, uint32_t flags,
                          int32_t* d_ranks, int32_t* d_pivots, const int64_t* d_piv_offsets,
                          int32_t* d_status, cudaStream_t stream) {
    (void)max_n;
    const bool pattern = (flags & LINAC_SHARED_PATTERN) != 0 && batch > 1;
    // scratch: BatchScratch | order[batch] | fallback[batch] | pattern J, Pi
    const size_t pat_words = (size_t)(1024 / 16 + 1) * 64;
    const size_t bytes = align_up(sizeof(BatchScratch), 256) + align_up((size_t)batch * 4, 256) * 2 +
                         2 * pat_words * 4;
    void* buf = nullptr;
    linac_status s = scratch_get_slot(stream, 2, bytes, &buf);
    if (s != LINAC_OK) return s;
    char* p = (char*)buf;
    BatchScratch* bs = (BatchScratch*)p;
    p += align_up(sizeof(BatchScratch), 256);
    int32_t* order = (int32_t*)p;
    p += align_up((size_t)batch * 4, 256);
    int32_t* fallback = (int32_t*)p;
    p += align_up((size_t)batch * 4, 256);
    int32_t* pat_J = (int32_t*)p;
    int32_t* pat_Pi = pat_J + pat_words;

    {
        ProfScope ps(stream, PROF_BATCHED);
        batch_sort_kernel<<<1, 1024, 0, stream>>>(d_m, batch, order, bs, pattern ? 1 : 0);
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    LINAC_CUDA_TRY(cudaMemsetAsync(&bs->pattern_ok, 0, sizeof(int), stream));
    int top = 0;
    while (top + 1 < BT_NBUCKETS && max_m > bt_bucket_max(top)) ++top;
    if (pattern) {
        // the probe runs with the widest panel the bucket of system 0 may need
        const int nb = bt_bucket_nb(top);
        const BtLayout L = bt_layout(bt_bucket_max(top), nb);
        ProfScope ps(stream, PROF_PATTERN);
        switch (nb) {
#define LINAC_PROBE(NBV)                                                                                        \
    case NBV:                                                                                                   \
        LINAC_CUDA_TRY(cudaFuncSetAttribute(batched_probe_kernel<NBV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                            (int)L.total));                                                     \
        batched_probe_kernel<NBV><<<1, BT_THREADS, L.total, stream>>>(d_data, d_offsets, d_m, d_n, d_ld, d_nsearch, \
                                                                      bt_bucket_max(top), f, d_ranks, d_pivots,  \
                                                                      d_piv_offsets, d_status, bs, pat_J, pat_Pi); \
        break;
            LINAC_PROBE(16)
            LINAC_PROBE(32)
            LINAC_PROBE(64)
#undef LINAC_PROBE
            default: return LINAC_ERR_ARG;
        }
        LINAC_CUDA_TRY(cudaGetLastError());
    }
    // every bucket uses the pattern's panel width when a pattern is shared
    const int pat_nb = pattern ? bt_bucket_nb(top) : 0;
    for (int b = top; b >= 0; --b) {
        const int nb = pattern ? pat_nb : bt_bucket_nb(b);
        s = launch_bucket_nb(nb, b, 0, pattern ? 1 : 0, d_data, d_offsets, d_m, d_n, d_ld, d_nsearch, order, f,
                             d_ranks, d_pivots, d_piv_offsets, d_status, bs, pat_J, pat_Pi, fallback, stream);
        if (s != LINAC_OK) return s;
    }
    if (pattern) {
        for (int b = top; b >= 0; --b) {
            s = launch_bucket_nb(bt_bucket_nb(b), b, 1, 0, d_data, d_offsets, d_m, d_n, d_ld, d_nsearch, order, f,
                                 d_ranks, d_pivots, d_piv_offsets, d_status, bs, pat_J, pat_Pi, fallback, stream);
            if (s != LINAC_OK) return s;
        }
    }
    return LINAC_OK;
}

}  // namespace linac
