// Annihilation, part 2, and the estimators (Sec. III.C annihilation; Sec. IV.A
// initiator rule; Sec. III.A estimators).
//
// The sorted list L_t (unique keys, populations already updated by
// death/clone) and the sorted spawn records S (repeated keys) are merged
// along the merge path, L first on equal keys.  In the merged order every
// configuration forms one run: its L_t entry (if present) followed by all its
// spawn records.  Each run is summed under the initiator rule -- records whose
// parent was not an initiator count only when the configuration is occupied
// in L_t or diagonal -- and non-zero sums are compacted into L_{t+1} in order;
// every kept entry is added to the integer estimator numerators on the way out.
//
// Work is cut into tiles of MG_TILE merged positions, one tile per warp at a
// time, assigned statically (tiles never wait for one another): the warp
// brings its tile's list and spawn ranges into shared memory with two bulk
// copies, merges MG_IPT positions per lane in registers, sums runs as
// differences of a warp-wide prefix sum (the partition kernel has already
// located the spawn records that continue the tile's last run past its end;
// the warp sums them with coalesced loads) and writes its output entries,
// uncompacted, into the tile's own slot of a scratch array with their count.
// Runs whose head lies in an earlier tile are left to that tile.  Then one
// kernel scans the tile counts (decoupled look-back over chunks of MC_TILES
// tiles) and another copies every tile's entries to their place in L_{t+1}.
#pragma once

#include "common.cuh"
#include "radix.cuh"

namespace ddq {

constexpr int MG_TPB = 256;
constexpr int MG_WARPS = MG_TPB / 32;
constexpr int MG_IPT = 9;                  // odd: the lanes' merge cursors spread over the banks
constexpr int MG_TILE = 32 * MG_IPT;       // merged positions per warp tile

// ---- keys ----------------------------------------------------------------
// One-word records compare their packed key (bra << N | ket); two-word
// records compare (bra, ket) as a 128-bit number.
struct K128 {
    uint64_t lo, hi;            // ket word, bra word
};
__device__ __forceinline__ bool operator<=(const K128 &a, const K128 &b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}
__device__ __forceinline__ bool operator>(const K128 &a, const K128 &b) { return !(a <= b); }
__device__ __forceinline__ bool operator==(const K128 &a, const K128 &b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(const K128 &a, const K128 &b) { return !(a == b); }

// Keys of the merge tile: 32-bit when spawn records are packed (2N <= 32).
template <typename T> struct MergeKey { using type = uint64_t; };
template <> struct MergeKey<uint64_t> { using type = uint32_t; };
template <> struct MergeKey<P40> { using type = uint64_t; };
template <> struct MergeKey<RecW> { using type = K128; };

template <typename KT> __device__ __forceinline__ KT list_key(const Rec &v) { return (KT)v.key; }
template <typename KT> __device__ __forceinline__ KT list_key(const RecW &v) { return K128{v.lo, v.hi}; }
template <typename KT, typename T> __device__ __forceinline__ KT spawn_key(const T &v) {
    return (KT)RecTraits<T>::key(v);
}
template <> __device__ __forceinline__ K128 spawn_key<K128, RecW>(const RecW &v) { return K128{v.lo, v.hi}; }

// ket and bra words of a key
// (hmask: the hashed order's mask of the ket hash in a two-word key's stored
// bra word; 0 for one-word keys; a batch's covers the N spin bits at most)
__device__ __forceinline__ void key_words(uint64_t k, uint64_t nmask, int N, uint64_t &i, uint64_t &j,
                                          uint64_t = 0) {
    i = k & nmask;
    j = k >> N;
}
__device__ __forceinline__ void key_words(uint32_t k, uint64_t nmask, int N, uint64_t &i, uint64_t &j,
                                          uint64_t = 0) {
    key_words((uint64_t)k, nmask, N, i, j);
}
__device__ __forceinline__ void key_words(const K128 &k, uint64_t, int, uint64_t &i, uint64_t &j,
                                          uint64_t hmask = 0) {
    i = k.lo;
    j = bra_swap(k.lo, k.hi, hmask);
}

__device__ __forceinline__ uint64_t shfl_key(uint64_t v, int src) { return __shfl_sync(0xFFFFFFFFu, v, src); }
__device__ __forceinline__ uint32_t shfl_key(uint32_t v, int src) { return __shfl_sync(0xFFFFFFFFu, v, src); }
__device__ __forceinline__ K128 shfl_key(const K128 &v, int src) {
    return K128{__shfl_sync(0xFFFFFFFFu, v.lo, src), __shfl_sync(0xFFFFFFFFu, v.hi, src)};
}

// high word of a key, where a batch keeps the run id
__device__ __forceinline__ uint64_t key_high(uint64_t k) { return k; }
__device__ __forceinline__ uint64_t key_high(uint32_t k) { return (uint64_t)k; }
__device__ __forceinline__ uint64_t key_high(const K128 &k) { return k.hi; }

__device__ __forceinline__ void set_list(Rec &v, uint64_t key) { v.key = key; }
__device__ __forceinline__ void set_list(Rec &v, uint32_t key) { v.key = (uint64_t)key; }
__device__ __forceinline__ void set_list(RecW &v, const K128 &key) { v.lo = key.lo; v.hi = key.hi; }

// merge-path split of output diagonal `diag`: number of L elements among the
// first `diag` merged elements (L before S on equal keys)
template <typename T, typename LT>
__device__ __forceinline__ int64_t merge_split(const LT *L, int64_t M, const T *S, int64_t R, int64_t diag) {
    using KT = typename MergeKey<T>::type;
    int64_t lo = diag > R ? diag - R : 0;
    int64_t hi = diag < M ? diag : M;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (list_key<KT>(L[mid]) <= spawn_key<KT>(S[diag - 1 - mid])) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// For every tile boundary t: the merge-path split, and the end of the spawn
// records that continue the last run of tile t-1 past the boundary (the
// records S[b, rem_end[t]) share the key of the merged element before the
// boundary; rem_end[t] = b when the run stops there).  One thread per
// boundary in groups of MG_PGROUP consecutive boundaries: the first thread of
// a group searches the whole path, the others then search in parallel inside
// the window that bound gives (a split moves by at most MG_TILE per
// boundary), so each thread makes about one full and one short search.
constexpr int MG_PGROUP = 8;
template <typename T>
__global__ void k_merge_partition(const typename ListOf<T>::type *__restrict__ L, const T *__restrict__ S,
                                  DevState *__restrict__ st, int64_t *__restrict__ splits,
                                  int64_t *__restrict__ rem_end, int64_t rcap) {
    using KT = typename MergeKey<T>::type;
    if (st->status) return;
    const int64_t M = st->M;
    int64_t R = st->R;
    if (R > rcap) R = rcap;
    const int64_t tot = M + R;
    const int64_t ntiles = (tot + MG_TILE - 1) / MG_TILE;
    const int lane = threadIdx.x & 31, g = lane & (MG_PGROUP - 1);
    // the grid strides in whole warps, so the lanes of a group stay together
    const int64_t span = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 <= ntiles; t0 += span) {
        const int64_t t = t0 + lane;
        const int64_t tg = t - g;                         // first boundary of the group
        int64_t diag = t * MG_TILE;
        if (diag > tot) diag = tot;
        int64_t a0 = 0;
        if (g == 0 && t <= ntiles) a0 = merge_split(L, M, S, R, diag);
        a0 = __shfl_sync(0xFFFFFFFFu, a0, lane & ~(MG_PGROUP - 1));
        if (t > ntiles) continue;
        int64_t a = a0;
        if (g != 0) {
            const int64_t dg = tg * MG_TILE;
            int64_t lo = a0, hi = a0 + (diag - dg);
            if (lo < diag - R) lo = diag - R;
            if (hi > diag) hi = diag;
            if (hi > M) hi = M;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (list_key<KT>(L[mid]) <= spawn_key<KT>(S[diag - 1 - mid])) lo = mid + 1;
                else hi = mid;
            }
            a = lo;
        }
        const int64_t b = diag - a;
        splits[t] = a;
        int64_t e = b;
        if (b < R && diag > 0) {
            KT last{};
            if (a > 0) last = list_key<KT>(L[a - 1]);
            if (b > 0) {
                const KT k2 = spawn_key<KT>(S[b - 1]);
                if (a == 0 || k2 > last) last = k2;
            }
            if (spawn_key<KT>(S[b]) == last) {
                // first record after b with a larger key: gallop, then bisect
                // invariant: S[b, lo) all carry the key; the first other key is in [lo, hi]
                int64_t lo = b + 1, step = 1, hi = R;
                for (;;) {
                    if (lo >= R || spawn_key<KT>(S[lo]) != last) { hi = lo < R ? lo : R; break; }
                    const int64_t nxt = lo + step;
                    if (nxt >= R || spawn_key<KT>(S[nxt]) != last) { hi = nxt < R ? nxt : R; ++lo; break; }
                    lo = nxt + 1;
                    step <<= 1;
                }
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (spawn_key<KT>(S[mid]) == last) lo = mid + 1;
                    else hi = mid;
                }
                e = lo;
            }
        }
        rem_end[t] = e;
    }
}

// Shared memory of one warp tile: the tile's list and spawn ranges as raw
// records (one bulk copy each, the element before each range included), later
// the tile's output entries.
template <typename T>
struct MergeTile {
    using LT = typename ListOf<T>::type;
    static constexpr int LS = (int)sizeof(LT), SS = (int)sizeof(T);
    static constexpr int MAXS = LS > SS ? LS : SS;
    // two ranges of at most MG_TILE + 1 records in all, each widened by at most 30 bytes
    static constexpr int BYTES = ((MG_TILE + 2) * MAXS + 64 + 15) & ~15;
};

template <typename T>
struct MergeShared {
    alignas(128) unsigned char buf[MG_WARPS][MergeTile<T>::BYTES];
    uint64_t bar[MG_WARPS];
    int64_t rem[MG_WARPS][4];         // sums of the records past the tile: initiator re, im; others re, im
    unsigned long long est[NOBS_MAX];
    uint64_t bond_m[MAXB];
    int8_t bond_a[MAXB], bond_b[MAXB];
    int8_t pair_bond[MAXN * MAXN];
};

// est: the block's shared-memory numerators of the entry's run
template <typename T>
__device__ __forceinline__ void add_estimators(MergeShared<T> &s, unsigned long long *est, const RunParams &P,
                                               uint64_t i, uint64_t j, int32_t re, int32_t im) {
    const int N = P.N, B = P.B;
    if (i == j) {
        atomicAdd(&est[0], (unsigned long long)(int64_t)re);
        atomicAdd(&est[1], (unsigned long long)(int64_t)im);
        atomicAdd(&est[2], (unsigned long long)(int64_t)(re < 0 ? -re : re));
        for (int k = 0; k < N; ++k)
            atomicAdd(&est[5 + k], (unsigned long long)(int64_t)(((i >> k) & 1ull) ? re : -re));
        for (int b = 0; b < B; ++b) {
            const bool al = ((i >> s.bond_a[b]) & 1ull) == ((i >> s.bond_b[b]) & 1ull);
            atomicAdd(&est[5 + N + b], (unsigned long long)(int64_t)(al ? re : -re));
        }
    } else {
        const uint64_t d = i ^ j;
        if (__popcll(d) == 1) {
            // sigma^x_k, sigma^y_k (configurations of odd parity: only with a field)
            const int k = __ffsll((long long)d) - 1;
            const int ox = 5 + N + 3 * B + 4;
            atomicAdd(&est[ox + k], (unsigned long long)(int64_t)re);
            atomicAdd(&est[ox + N + k], (unsigned long long)(int64_t)(((i >> k) & 1ull) ? -im : im));
        } else if (__popcll(d) == 2) {
            const int a = __ffsll((long long)d) - 1;
            const int b2 = 63 - __clzll((long long)d);
            const int b = s.pair_bond[a * N + b2];
            if (b >= 0) {
                const bool al = ((i >> s.bond_a[b]) & 1ull) == ((i >> s.bond_b[b]) & 1ull);
                atomicAdd(&est[5 + N + B + b], (unsigned long long)(int64_t)re);
                atomicAdd(&est[5 + N + 2 * B + b], (unsigned long long)(int64_t)(al ? -re : re));
            }
        }
    }
}

// Exact warp sum of int32 values (two 32-bit reductions of the 16-bit
// halves, so no partial sum leaves the int32 range).
__device__ __forceinline__ int64_t warp_sum_i32(int32_t v) {
    const uint32_t lo = (uint32_t)v & 0xFFFFu;
    const int32_t hi = v >> 16;
    const uint32_t slo = __reduce_add_sync(0xFFFFFFFFu, lo);
    const int32_t shi = (int32_t)__reduce_add_sync(0xFFFFFFFFu, (uint32_t)hi);
    return (int64_t)shi * 65536 + (int64_t)slo;
}

// The diagonal numerators (Tr re, Tr im, N_w, sigma^z per site, zz per bond)
// of the warp's diagonal entries, all of one run (entries elsewhere give 0):
// summed over the warp, then one shared-memory atomic per observable.
template <typename T>
__device__ __forceinline__ void add_diagonal_warp(MergeShared<T> &s, unsigned long long *est, const RunParams &P,
                                                  bool diag, uint64_t i, int32_t re, int32_t im, int lane) {
    const int N = P.N, B = P.B;
    const int32_t x = diag ? re : 0;
    int64_t t;
    t = warp_sum_i32(x);
    if (lane == 0 && t) atomicAdd(&est[0], (unsigned long long)t);
    t = warp_sum_i32(diag ? im : 0);
    if (lane == 0 && t) atomicAdd(&est[1], (unsigned long long)t);
    t = warp_sum_i32(x < 0 ? -x : x);
    if (lane == 0 && t) atomicAdd(&est[2], (unsigned long long)t);
    for (int k = 0; k < N; ++k) {
        t = warp_sum_i32(((i >> k) & 1ull) ? x : -x);
        if (lane == 0 && t) atomicAdd(&est[5 + k], (unsigned long long)t);
    }
    for (int b = 0; b < B; ++b) {
        const bool al = ((i >> s.bond_a[b]) & 1ull) == ((i >> s.bond_b[b]) & 1ull);
        t = warp_sum_i32(al ? x : -x);
        if (lane == 0 && t) atomicAdd(&est[5 + N + b], (unsigned long long)t);
    }
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    return v;
}
// resident blocks per SM the merge is compiled for: 4 for a single run with
// packed records (64 registers a thread: a few spills, measured faster than
// 3 at 80), 2 for 128-bit keys, else 3
template <typename T, bool BATCH> struct MergeBlocks {
    static constexpr int value = std::is_same<T, RecW>::value ? 2
                                 : ((std::is_same<T, uint64_t>::value && !BATCH) ? 4 : 3);
};

__device__ __forceinline__ int64_t shfl_up_i64(int64_t v, int off) {
    return (int64_t)__shfl_up_sync(0xFFFFFFFFu, (long long)v, off);
}

// configuration (ket, bra) of a merge key, the batch run id stripped
template <typename KT, bool BATCH>
__device__ __forceinline__ bool key_diagonal(const KT &k, uint64_t nmask, int N, uint64_t hmask) {
    uint64_t i, j;
    key_words(k, nmask, N, i, j, hmask);
    if (BATCH) j &= nmask;
    return i == j;
}

// BATCH: the lists hold several runs (run id in the key's high bits); each
// run has its own initiator threshold (Pr[r]) and estimator numerators
// (rs[r]), summed per block in dynamic shared memory past MergeShared (nruns
// x nobs words).  A single run passes Pr = Pp and rs = st (unread).
//
// One warp tile of MG_TILE merged positions: lane 0 issues two bulk copies
// (list range [a0 - 1, a1), spawn range [b0 - 1, b1), each widened to 16-byte
// boundaries) completing on the warp's mbarrier; each lane merges its MG_IPT
// positions in registers; whether a run holds its L_t entry travels from the
// lane of its head by ballot and shuffle; run sums are differences of one
// warp-wide int64 prefix sum of the counted contributions (L_t entries and
// initiator records always, other records when the run is open: L_t entry
// present, diagonal, or no initiator rule).  The outputs are staged in the
// tile buffer and leave with one bulk store into the tile's slot
// (slots + tile * MG_TILE), their number into counts[tile].
// Sums of the spawn records S[b1, rem_e) (initiator re, im, other re, im)
// over one warp, into out (lane 0 writes).
template <typename T>
__device__ __noinline__ void rem_sums(const T *__restrict__ S, int64_t b1, int64_t rem_e, int lane, int64_t *out) {
    using TR = RecTraits<T>;
    int64_t f0 = 0, f1 = 0, u0 = 0, u1 = 0;
    for (int64_t q = b1 + lane; q < rem_e; q += 32) {
        const T g = S[q];
        if (TR::flag(g)) { f0 += TR::re(g); f1 += TR::im(g); }
        else { u0 += TR::re(g); u1 += TR::im(g); }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        f0 += __shfl_xor_sync(0xFFFFFFFFu, f0, off);
        f1 += __shfl_xor_sync(0xFFFFFFFFu, f1, off);
        u0 += __shfl_xor_sync(0xFFFFFFFFu, u0, off);
        u1 += __shfl_xor_sync(0xFFFFFFFFu, u1, off);
    }
    if (lane == 0) { out[0] = f0; out[1] = f1; out[2] = u0; out[3] = u1; }
}

template <typename T, bool BATCH>
__global__ void __launch_bounds__(MG_TPB, (MergeBlocks<T, BATCH>::value))
k_merge(const RunParams *__restrict__ Pp, const typename ListOf<T>::type *__restrict__ L, const T *__restrict__ S,
        typename ListOf<T>::type *__restrict__ slots, uint32_t *__restrict__ counts, DevState *__restrict__ st,
        const int64_t *__restrict__ splits, const int64_t *__restrict__ rem_end, int64_t rcap,
        const RunParams *__restrict__ Pr, DevState *__restrict__ rs) {
    using TR = RecTraits<T>;
    using KT = typename MergeKey<T>::type;
    using LT = typename ListOf<T>::type;
    constexpr int LS = MergeTile<T>::LS, SS = MergeTile<T>::SS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MergeShared<T> &s = *reinterpret_cast<MergeShared<T> *>(smem_raw);
    const RunParams &P = *Pp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (block_stopped(st)) return;
    const int64_t M = st->M;
    int64_t R = st->R;
    if (R > rcap) R = rcap;
    const int64_t tot = M + R;
    const int64_t ntiles = (tot + MG_TILE - 1) / MG_TILE;
    const int N = P.N;
    const uint64_t nmask = P.nmask;
    const uint64_t xmask = P.hash_mask;     // hashed order of two-word keys
    const bool no_init = P.n_a == 0;
    const int nruns = P.nruns, run_shift = P.run_shift, nobs = P.nobs;
    unsigned long long *best = reinterpret_cast<unsigned long long *>(smem_raw + sizeof(MergeShared<T>));

    for (int q = tid; q < NOBS_MAX; q += MG_TPB) s.est[q] = 0ull;
    if (BATCH)
        for (int q = tid; q < nruns * nobs; q += MG_TPB) best[q] = 0ull;
    for (int q = tid; q < P.B; q += MG_TPB) {
        s.bond_m[q] = P.bond_m[q];
        s.bond_a[q] = (int8_t)P.bond_a[q];
        s.bond_b[q] = (int8_t)P.bond_b[q];
    }
    for (int q = tid; q < N * N; q += MG_TPB) s.pair_bond[q] = P.pair_bond[q];
    if (lane == 0) mbar_init(&s.bar[warp], 1);
    __syncthreads();
    unsigned char *buf = s.buf[warp];
    uint64_t *bar = &s.bar[warp];
    uint32_t phase = 0;
    bool store_pending = false;          // lane 0: a bulk store still reads buf
    int64_t my_w = 0, my_m = 0;
    uint32_t local_status = 0;

    const int64_t nwarps = (int64_t)gridDim.x * MG_WARPS;
    int64_t tile = (int64_t)blockIdx.x * MG_WARPS + warp;
    // bounds of the next tile, loaded one tile ahead
    int64_t na0 = 0, na1 = 0, nrem = 0;
    if (tile < ntiles) { na0 = splits[tile]; na1 = splits[tile + 1]; nrem = rem_end[tile + 1]; }
    for (; tile < ntiles; tile += nwarps) {
        const int64_t d0 = tile * MG_TILE;
        const int64_t d1 = (d0 + MG_TILE < tot) ? d0 + MG_TILE : tot;
        const int64_t a0 = na0, a1 = na1, rem_e = nrem;
        const int64_t b0 = d0 - a0, b1 = d1 - a1;
        const int na = (int)(a1 - a0), nb = (int)(b1 - b0), nt = na + nb;
        // byte ranges of the two copies (from the element before each range)
        const int64_t gl0 = ((a0 > 0 ? a0 - 1 : 0) * LS) & ~15ll, gl1 = (a1 * LS + 15) & ~15ll;
        const int64_t gs0 = ((b0 > 0 ? b0 - 1 : 0) * SS) & ~15ll, gs1 = (b1 * SS + 15) & ~15ll;
        const uint32_t lbytes = (uint32_t)(gl1 - gl0), sbytes = (uint32_t)(gs1 - gs0);
        __syncwarp();                    // every lane is done with the previous tile's buffer
        if (lane == 0) {
            if (store_pending) { bulk_wait_read(); store_pending = false; }
            fence_proxy_async();
            mbar_arrive_expect_tx(bar, lbytes + sbytes);
            if (lbytes) bulk_load(buf, reinterpret_cast<const unsigned char *>(L) + gl0, lbytes, bar);
            if (sbytes) bulk_load(buf + lbytes, reinterpret_cast<const unsigned char *>(S) + gs0, sbytes, bar);
        }
        if (tile + nwarps < ntiles) {
            na0 = splits[tile + nwarps];
            na1 = splits[tile + nwarps + 1];
            nrem = rem_end[tile + nwarps + 1];
        }
        // spawn records past the tile end that continue its last run.  Up to
        // 32 (the usual case): one per lane, loaded now so that the load
        // overlaps the copies and the merge, and summed just before the run
        // ends.  More: summed here.
        const bool rem_any = rem_e > b1, rem_long = rem_e - b1 > 32;
        T g0 = TR::empty();
        if (rem_long) rem_sums<T>(S, b1, rem_e, lane, s.rem[warp]);
        else if (b1 + lane < rem_e) g0 = S[b1 + lane];
        const bool has_lprev = a0 > 0, has_sprev = b0 > 0;
        const bool arrived = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (!__all_sync(0xFFFFFFFFu, arrived)) {
            // the copies did not complete: report, give them one more bounded
            // wait (the buffer must not be left while they may still land), stop
            if (lane == 0) atomicOr(&st->status, ST_TIMEOUT);
            mbar_wait_bounded(bar, phase ^ 1u);
            break;
        }
        // Lt[q] = L[a0 + q], St[q] = S[b0 + q] for q >= -1
        const LT *Lt = reinterpret_cast<const LT *>(buf + (a0 * LS - gl0));
        const T *St = reinterpret_cast<const T *>(buf + lbytes + (b0 * SS - gs0));

        // ---- 1. merge: this lane's MG_IPT merged positions, in registers ----
        const int dloc = lane * MG_IPT;
        KT ik[MG_IPT];
        int2 iv[MG_IPT];
        uint32_t hmask = 0, lmask = 0, fmask = 0;   // run heads, elements of L_t, initiator records
        int nk = 0;
#pragma unroll
        for (int k = 0; k < MG_IPT; ++k) { ik[k] = KT{}; iv[k] = make_int2(0, 0); }
        if (dloc < nt) {
            int lo = dloc > nb ? dloc - nb : 0;
            int hi = dloc < na ? dloc : na;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (list_key<KT>(Lt[mid]) <= spawn_key<KT, T>(St[dloc - 1 - mid])) lo = mid + 1;
                else hi = mid;
            }
            int ia = lo, ib = dloc - lo;
            // the merged element before this lane's first position
            KT prev{};
            bool hprev = false;
            if (ia > 0 || has_lprev) { prev = list_key<KT>(Lt[ia - 1]); hprev = true; }
            if (ib > 0 || has_sprev) {
                const KT k2 = spawn_key<KT, T>(St[ib - 1]);
                if (!hprev || k2 > prev) prev = k2;
                hprev = true;
            }
            nk = nt - dloc < MG_IPT ? nt - dloc : MG_IPT;
#pragma unroll
            for (int k = 0; k < MG_IPT; ++k) {
                if (k < nk) {
                    bool fromL;
                    if (ia >= na) fromL = false;
                    else if (ib >= nb) fromL = true;
                    else fromL = list_key<KT>(Lt[ia]) <= spawn_key<KT, T>(St[ib]);
                    KT key;
                    if (fromL) {
                        const LT v = Lt[ia];
                        key = list_key<KT>(v);
                        iv[k] = make_int2(v.re, v.im);
                        lmask |= 1u << k;
                        ++ia;
                    } else {
                        const T v = St[ib];
                        key = spawn_key<KT, T>(v);
                        iv[k] = make_int2(TR::re(v), TR::im(v));
                        if (TR::flag(v)) fmask |= 1u << k;
                        ++ib;
                    }
                    ik[k] = key;
                    if (!hprev || key != prev) hmask |= 1u << k;
                    prev = key;
                    hprev = true;
                }
            }
        }
        // ---- 2. runs: L_t entry of the open run, counted contributions ------
        // the run open at this lane's start has its head in the nearest
        // earlier lane with a head (none: it began in an earlier tile and is
        // that tile's to finish)
        const int last_head = hmask ? 31 - __clz(hmask) : 0;
        const uint32_t last_head_L = (lmask >> last_head) & 1u;
        const unsigned heads = __ballot_sync(0xFFFFFFFFu, hmask != 0u);
        const unsigned below = heads & ((1u << lane) - 1u);
        const int src = below ? 31 - __clz(below) : 0;
        const uint32_t carry_L = __shfl_sync(0xFFFFFFFFu, last_head_L, src);
        const bool carry_owned = below != 0u;
        uint32_t cmask = 0;              // counted contributions
        int64_t lre = 0, lim = 0;        // lane sums of the counted contributions
        int64_t hre = 0, him = 0;        // lane prefix before its last head
        {
            uint32_t hasL = carry_L;
#pragma unroll
            for (int k = 0; k < MG_IPT; ++k) {
                if (k < nk) {
                    if ((hmask >> k) & 1u) { hasL = (lmask >> k) & 1u; hre = lre; him = lim; }
                    bool counted = (((lmask | fmask) >> k) & 1u) || hasL;
                    if (!counted) {
                        bool ni = no_init;
                        if constexpr (BATCH) ni = Pr[batch_run(key_high(ik[k]), run_shift, nruns)].n_a == 0;
                        counted = ni || key_diagonal<KT, BATCH>(ik[k], nmask, N, xmask);
                    }
                    if (counted) {
                        cmask |= 1u << k;
                        lre += iv[k].x;
                        lim += iv[k].y;
                    }
                }
            }
        }
        // exclusive warp prefix of the lane sums
        int64_t ere = lre, eim = lim;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t yr = shfl_up_i64(ere, off), yi = shfl_up_i64(eim, off);
            if (lane >= off) { ere += yr; eim += yi; }
        }
        ere -= lre;
        eim -= lim;
        // prefix before the head of the run open at this lane's start
        const int64_t cb_re = (int64_t)__shfl_sync(0xFFFFFFFFu, (long long)(ere + hre), src);
        const int64_t cb_im = (int64_t)__shfl_sync(0xFFFFFFFFu, (long long)(eim + him), src);
        const int my_first_head = nk > 0 ? (int)(hmask & 1u) : 1;
        const int next_first_head = __shfl_down_sync(0xFFFFFFFFu, my_first_head, 1);

        // sums of those records (initiator and other), for the tile's last run
        if (!rem_long) {
            const bool f = TR::flag(g0);
            int64_t f0 = f ? TR::re(g0) : 0, f1 = f ? TR::im(g0) : 0;
            int64_t u0 = f ? 0 : TR::re(g0), u1 = f ? 0 : TR::im(g0);
            if (rem_any) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    f0 += __shfl_xor_sync(0xFFFFFFFFu, f0, off);
                    f1 += __shfl_xor_sync(0xFFFFFFFFu, f1, off);
                    u0 += __shfl_xor_sync(0xFFFFFFFFu, u0, off);
                    u1 += __shfl_xor_sync(0xFFFFFFFFu, u1, off);
                }
            }
            if (lane == 0) { s.rem[warp][0] = f0; s.rem[warp][1] = f1; s.rem[warp][2] = u0; s.rem[warp][3] = u1; }
        }
        __syncwarp();
        // ---- 3. run ends: sums and the initiator rule; outputs replace iv ----
        uint32_t omask = 0;
        {
            int64_t pre = ere, pim = eim, bre = cb_re, bim = cb_im;
            uint32_t hasL = carry_L;
            bool owned = carry_owned;
#pragma unroll
            for (int k = 0; k < MG_IPT; ++k) {
                if (k < nk) {
                    if ((hmask >> k) & 1u) { bre = pre; bim = pim; hasL = (lmask >> k) & 1u; owned = true; }
                    if ((cmask >> k) & 1u) { pre += iv[k].x; pim += iv[k].y; }
                    const bool tile_last = dloc + k + 1 == nt;
                    bool ends;
                    if (k + 1 < nk) ends = ((hmask >> (k + 1)) & 1u) != 0u;
                    else ends = tile_last || next_first_head != 0;
                    if (ends && owned) {
                        int64_t sre = pre - bre, sim = pim - bim;
                        if (tile_last) {
                            // the records of the last run that lie past the tile
                            sre += s.rem[warp][0];
                            sim += s.rem[warp][1];
                            bool open = hasL != 0u;
                            if (!open) {
                                bool ni = no_init;
                                if constexpr (BATCH) ni = Pr[batch_run(key_high(ik[k]), run_shift, nruns)].n_a == 0;
                                open = ni || key_diagonal<KT, BATCH>(ik[k], nmask, N, xmask);
                            }
                            if (open) { sre += s.rem[warp][2]; sim += s.rem[warp][3]; }
                        }
                        bool keep = sre != 0 || sim != 0;
                        if constexpr (BATCH) keep = keep && Pr[batch_run(key_high(ik[k]), run_shift, nruns)].active != 0;
                        if (keep) {
                            if (iabs64(sre) > 2147483647ll || iabs64(sim) > 2147483647ll) local_status |= ST_OVERFLOW;
                            omask |= 1u << k;
                            iv[k] = make_int2((int32_t)sre, (int32_t)sim);
                        }
                    }
                }
            }
        }
        // ---- 4. compaction: warp scan of the output counts, staging ---------
        const int nout = __popc(omask);
        int x = nout;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += y;
        }
        const uint32_t total = (uint32_t)__shfl_sync(0xFFFFFFFFu, x, 31);
        __syncwarp();                    // every lane is done reading the tile
        LT *stage = reinterpret_cast<LT *>(buf);
        {
            uint32_t my_off = (uint32_t)(x - nout);
#pragma unroll
            for (int k = 0; k < MG_IPT; ++k) {
                if ((omask >> k) & 1u) {
                    LT v;
                    set_list(v, ik[k]);
                    v.re = iv[k].x;
                    v.im = iv[k].y;
                    stage[my_off++] = v;
                }
            }
        }
        __syncwarp();
        // estimator numerators of the outputs (walkers, entries; diagonal and
        // nearest-neighbour terms).  A single run sums walkers and entries in
        // registers; a batch sums them per run while consecutive entries stay
        // in one run, and when many lanes hold diagonal entries of one run
        // (the small runs batches are made of: most entries) it sums their
        // diagonal terms over the warp before the shared-memory atomics.
        if constexpr (!BATCH) {
            for (uint32_t q = lane; q < total; q += 32) {
                const LT v = stage[q];
                uint64_t i, j;
                key_words(list_key<KT>(v), nmask, N, i, j, xmask);
                my_w += iabs64(v.re) + iabs64(v.im);
                my_m += 1;
                if (i == j || __popcll(i ^ j) <= 2) add_estimators(s, s.est, P, i, j, v.re, v.im);
            }
        } else {
            int brun = -1;
            int64_t bw = 0, bm = 0;
            for (uint32_t q0 = 0; q0 < total; q0 += 32) {
                const uint32_t q = q0 + lane;
                const bool valid = q < total;
                LT v;
                set_list(v, KT{});
                v.re = 0;
                v.im = 0;
                if (valid) v = stage[q];
                uint64_t i, j;
                key_words(list_key<KT>(v), nmask, N, i, j, xmask);
                const int rr = batch_run(key_high(list_key<KT>(v)), run_shift, nruns);
                j &= nmask;
                unsigned long long *est = best + (size_t)rr * nobs;
                if (valid) {
                    if (rr != brun) {
                        if (brun >= 0) {
                            atomicAdd(&best[(size_t)brun * nobs + 3], (unsigned long long)bw);
                            atomicAdd(&best[(size_t)brun * nobs + 4], (unsigned long long)bm);
                        }
                        brun = rr;
                        bw = 0;
                        bm = 0;
                    }
                    bw += iabs64(v.re) + iabs64(v.im);
                    bm += 1;
                }
                const bool diag = valid && i == j;
                const unsigned dm = __ballot_sync(0xFFFFFFFFu, diag);
                bool warp_diag = false;
                if (__popc(dm) >= 4) {
                    const int r0 = __shfl_sync(0xFFFFFFFFu, rr, __ffs(dm) - 1);
                    warp_diag = __all_sync(0xFFFFFFFFu, !diag || rr == r0);
                    if (warp_diag) add_diagonal_warp(s, best + (size_t)r0 * nobs, P, diag, i, v.re, v.im, lane);
                }
                if (valid && (diag ? !warp_diag : __popcll(i ^ j) <= 2)) add_estimators(s, est, P, i, j, v.re, v.im);
            }
            if (brun >= 0) {
                atomicAdd(&best[(size_t)brun * nobs + 3], (unsigned long long)bw);
                atomicAdd(&best[(size_t)brun * nobs + 4], (unsigned long long)bm);
            }
        }
        // ---- 5. the tile's slot: one bulk store, the count ------------------
        fence_proxy_async();             // the staged entries, before the async proxy reads them
        __syncwarp();
        if (lane == 0) {
            counts[tile] = total;
            if (total > 0) {
                // rounded up to 16 bytes: an odd number of 24-byte entries
                // carries 8 more bytes, inside the buffer and inside the slot
                bulk_store(slots + tile * MG_TILE, buf, (total * (uint32_t)LS + 15u) & ~15u);
                bulk_commit();
                store_pending = true;
            }
        }
    }
    if (lane == 0 && store_pending) bulk_wait_all();
    __syncwarp();
    // flush the block's estimator partials
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        my_w += __shfl_xor_sync(0xFFFFFFFFu, my_w, off);
        my_m += __shfl_xor_sync(0xFFFFFFFFu, my_m, off);
    }
    if (lane == 0) {
        atomicAdd(&s.est[3], (unsigned long long)my_w);
        atomicAdd(&s.est[4], (unsigned long long)my_m);
    }
    if (local_status) atomicOr(&st->status, local_status);
    __syncthreads();
    if (BATCH) {
        for (int q = tid; q < nruns * nobs; q += MG_TPB)
            if (best[q]) atomicAdd((unsigned long long *)&rs[q / nobs].est[q % nobs], best[q]);
    } else {
        for (int q = tid; q < P.nobs; q += MG_TPB)
            if (s.est[q]) atomicAdd((unsigned long long *)&st->est[q], s.est[q]);
    }
}

constexpr int MC_TPB = 256;
constexpr int MC_PER_THREAD = 4;
constexpr int MC_TILES = MC_TPB * MC_PER_THREAD;   // merge tiles per scan chunk

// Output offsets of the merge's tiles: a persistent grid takes chunks of
// MC_TILES tile counts in order from a ticket, scans each chunk in the
// block, finds the chunk's offset by decoupled look-back over earlier chunks
// (bounded waits) and writes every tile's offset into tile_off.  The last
// chunk records the merged length; one longer than mcap sets the capacity
// status (and the copy kernel then writes nothing).
__global__ void __launch_bounds__(MC_TPB)
k_merge_scan(const uint32_t *__restrict__ counts, int64_t *__restrict__ tile_off, DevState *__restrict__ st,
             uint64_t *__restrict__ lookback, int64_t rcap, int64_t mcap) {
    __shared__ uint32_t warp_sum[MC_TPB / 32];
    __shared__ int64_t s_base, s_chunk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (block_stopped(st)) return;
    const int64_t M = st->M;
    int64_t R = st->R;
    if (R > rcap) R = rcap;
    const int64_t ntiles = (M + R + MG_TILE - 1) / MG_TILE;
    const int64_t nchunks = (ntiles + MC_TILES - 1) / MC_TILES;
    const uint32_t epoch = st->epoch + (uint32_t)MAXPASS;
    for (;;) {
        if (tid == 0) s_chunk = (int64_t)atomicAdd(&st->tickets[MAXPASS], 1u);
        __syncthreads();
        const int64_t chunk = s_chunk;
        if (chunk >= nchunks) break;
        const int64_t t0 = chunk * MC_TILES + (int64_t)tid * MC_PER_THREAD;
        uint32_t c[MC_PER_THREAD], sum = 0;
#pragma unroll
        for (int k = 0; k < MC_PER_THREAD; ++k) {
            c[k] = t0 + k < ntiles ? counts[t0 + k] : 0u;
            sum += c[k];
        }
        uint32_t x = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        uint32_t pre = 0, all = 0;
        for (int w = 0; w < MC_TPB / 32; ++w) {
            if (w < warp) pre += warp_sum[w];
            all += warp_sum[w];
        }
        if (warp == 0) {
            uint64_t *myw = lookback + chunk;
            if (lane == 0) lb_store(myw, lb_pack(epoch, chunk == 0 ? LB_INC : LB_AGG, all));
            uint64_t excl = 0;
            if (chunk > 0) {
                for (int64_t jt = chunk - 1;; jt -= 32) {
                    const int64_t jj = jt - lane;
                    const uint64_t w = jj >= 0 ? lb_wait(lookback + jj, epoch, &st->status) : lb_pack(epoch, LB_INC, 0u);
                    const unsigned inc = __ballot_sync(0xFFFFFFFFu, ((w >> 32) & 3ull) != LB_AGG);
                    if (inc) {
                        const int first = __ffs(inc) - 1;
                        excl += warp_sum_u64(lane <= first ? (uint64_t)(uint32_t)w : 0ull);
                        break;
                    }
                    excl += warp_sum_u64((uint64_t)(uint32_t)w);
                }
                if (lane == 0) lb_store(myw, lb_pack(epoch, LB_INC, (uint32_t)(excl + all)));
            }
            if (lane == 0) {
                s_base = (int64_t)excl;
                if (chunk == nchunks - 1) {
                    st->M_next = (int64_t)(excl + all);
                    if ((int64_t)(excl + all) > mcap) atomicOr(&st->status, ST_CAPACITY | ST_CAP_LIST);
                }
            }
        }
        __syncthreads();
        int64_t o = s_base + (int64_t)(pre + x - sum);
#pragma unroll
        for (int k = 0; k < MC_PER_THREAD; ++k) {
            if (t0 + k < ntiles) tile_off[t0 + k] = o;
            o += c[k];
        }
        __syncthreads();
    }
}

// Copy of every tile's entries from its slot to its place in L_{t+1}: one
// tile per warp at a time, grid-strided, every lane's loads of the tile
// issued before its stores.
template <typename LT>
__global__ void __launch_bounds__(MC_TPB)
k_merge_copy(const LT *__restrict__ slots, const uint32_t *__restrict__ counts, const int64_t *__restrict__ tile_off,
             LT *__restrict__ out, const DevState *__restrict__ st, int64_t rcap) {
    const int lane = threadIdx.x & 31;
    if (*(volatile const uint32_t *)&st->status) return;
    const int64_t M = st->M;
    int64_t R = st->R;
    if (R > rcap) R = rcap;
    const int64_t ntiles = (M + R + MG_TILE - 1) / MG_TILE;
    const int64_t nwarps = (int64_t)gridDim.x * (MC_TPB / 32);
    for (int64_t t = (int64_t)blockIdx.x * (MC_TPB / 32) + (threadIdx.x >> 5); t < ntiles; t += nwarps) {
        const uint32_t n = counts[t];
        const int64_t o = tile_off[t];
        const LT *src = slots + t * MG_TILE;
        LT v[MG_IPT];
#pragma unroll
        for (int k = 0; k < MG_IPT; ++k)
            if ((uint32_t)(lane + 32 * k) < n) v[k] = src[lane + 32 * k];
#pragma unroll
        for (int k = 0; k < MG_IPT; ++k)
            if ((uint32_t)(lane + 32 * k) < n) out[o + lane + 32 * k] = v[k];
    }
}

}  // namespace ddq
