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
// time, with no block-wide synchronisation: the warp takes a ticket, loads
// its tile, merges MG_IPT positions per lane, sums runs with a segmented scan
// over the lanes (the partition kernel has already located the spawn records
// that continue the tile's last run past its end; the warp sums them with
// coalesced loads), and finds its output offset by a warp-parallel decoupled
// look-back over earlier tiles.  Runs whose head lies in an earlier tile are
// left to that tile.
#pragma once

#include "common.cuh"
#include "radix.cuh"

namespace ddq {

constexpr int MG_TPB = 256;
constexpr int MG_WARPS = MG_TPB / 32;
constexpr int MG_IPT = 9;                  // odd: the lanes' merge cursors spread over the banks
constexpr int MG_TILE = 32 * MG_IPT;       // merged positions per warp tile
constexpr int MG_PCHUNK = 8;               // tile boundaries per partition thread

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
template <> struct MergeKey<RecW> { using type = K128; };

template <typename KT> __device__ __forceinline__ KT list_key(const Rec &v) { return (KT)v.key; }
template <typename KT> __device__ __forceinline__ KT list_key(const RecW &v) { return K128{v.lo, v.hi}; }
template <typename KT, typename T> __device__ __forceinline__ KT spawn_key(const T &v) {
    return (KT)RecTraits<T>::key(v);
}
template <> __device__ __forceinline__ K128 spawn_key<K128, RecW>(const RecW &v) { return K128{v.lo, v.hi}; }

// ket and bra words of a key
__device__ __forceinline__ void key_words(uint64_t k, uint64_t nmask, int N, uint64_t &i, uint64_t &j) {
    i = k & nmask;
    j = k >> N;
}
__device__ __forceinline__ void key_words(uint32_t k, uint64_t nmask, int N, uint64_t &i, uint64_t &j) {
    key_words((uint64_t)k, nmask, N, i, j);
}
__device__ __forceinline__ void key_words(const K128 &k, uint64_t, int, uint64_t &i, uint64_t &j) {
    i = k.lo;
    j = k.hi;
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
// boundary; rem_end[t] = b when the run stops there).
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
    // each thread takes MG_PCHUNK consecutive boundaries: after the first full
    // search the next split lies within one tile of the previous one
    const int64_t nchunks = (ntiles + MG_PCHUNK) / MG_PCHUNK;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks; ch += (int64_t)gridDim.x * blockDim.x)
    for (int64_t t = ch * MG_PCHUNK, aprev = -1; t <= ntiles && t < (ch + 1) * MG_PCHUNK; ++t) {
        int64_t diag = t * MG_TILE;
        if (diag > tot) diag = tot;
        int64_t a;
        if (aprev < 0) {
            a = merge_split(L, M, S, R, diag);
        } else {
            // merge path split of diag inside [aprev, aprev + MG_TILE]
            int64_t lo = aprev, hi = aprev + MG_TILE;
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
        aprev = a;
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

// Aggregate of a partial run for the segmented reduction: h = a run head lies
// in the aggregated range, hasL = that head is the L_t entry, f = L_t
// population plus initiator records, u = non-initiator records.
struct SegAgg {
    int32_t h, hasL;
    int64_t fre, fim, ure, uim;
};

__device__ __forceinline__ SegAgg seg_identity() {
    SegAgg a;
    a.h = 0; a.hasL = 0; a.fre = 0; a.fim = 0; a.ure = 0; a.uim = 0;
    return a;
}

__device__ __forceinline__ SegAgg seg_head(uint32_t fromL) {
    SegAgg a = seg_identity();
    a.h = 1;
    a.hasL = (int32_t)fromL;
    return a;
}

__device__ __forceinline__ void seg_add(SegAgg &a, int2 v, uint32_t counted) {
    if (counted) { a.fre += v.x; a.fim += v.y; }
    else { a.ure += v.x; a.uim += v.y; }
}

// a followed by b
__device__ __forceinline__ SegAgg seg_combine(const SegAgg &a, const SegAgg &b) {
    if (b.h) return b;
    SegAgg r;
    r.h = a.h; r.hasL = a.hasL;
    r.fre = a.fre + b.fre; r.fim = a.fim + b.fim; r.ure = a.ure + b.ure; r.uim = a.uim + b.uim;
    return r;
}

__device__ __forceinline__ SegAgg seg_shfl_up(const SegAgg &a, int off) {
    SegAgg r;
    r.h = __shfl_up_sync(0xFFFFFFFFu, a.h, off);
    r.hasL = __shfl_up_sync(0xFFFFFFFFu, a.hasL, off);
    r.fre = __shfl_up_sync(0xFFFFFFFFu, a.fre, off);
    r.fim = __shfl_up_sync(0xFFFFFFFFu, a.fim, off);
    r.ure = __shfl_up_sync(0xFFFFFFFFu, a.ure, off);
    r.uim = __shfl_up_sync(0xFFFFFFFFu, a.uim, off);
    return r;
}

// Exclusive segmented scan over the lanes of a warp.
__device__ __forceinline__ SegAgg seg_warp_exclusive(const SegAgg &mine, int lane) {
    SegAgg inc = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const SegAgg o = seg_shfl_up(inc, off);
        if (lane >= off) inc = seg_combine(o, inc);
    }
    SegAgg exc = seg_shfl_up(inc, 1);
    if (lane == 0) exc = seg_identity();
    return exc;
}

template <typename T>
struct MergeWarp {
    typename MergeKey<T>::type key[MG_TILE];   // L keys, then S keys; later the output keys
    int2 val[MG_TILE];                          // (re, im) of the same elements; later the output populations
    uint32_t sflag[(MG_TILE + 31) / 32];        // initiator flags of the S elements, bit q of word q/32
};

template <typename T>
struct MergeShared {
    MergeWarp<T> w[MG_WARPS];
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

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    return v;
}

// resident blocks per SM the merge is compiled for: 128-bit keys need more registers
template <typename T> struct MergeBlocks { static constexpr int value = 4; };
template <> struct MergeBlocks<RecW> { static constexpr int value = 3; };

// BATCH: the lists hold several runs (run id in the key's high bits); each
// run has its own initiator threshold (Pr[r]) and estimator numerators
// (rs[r]), summed per block in dynamic shared memory past MergeShared (nruns
// x nobs words).  A single run passes Pr = Pp and rs = st (unread).
template <typename T, bool BATCH>
__global__ void __launch_bounds__(MG_TPB, MergeBlocks<T>::value)
k_merge(const RunParams *__restrict__ Pp, const typename ListOf<T>::type *__restrict__ L, const T *__restrict__ S,
        typename ListOf<T>::type *__restrict__ out, DevState *__restrict__ st, const int64_t *__restrict__ splits,
        const int64_t *__restrict__ rem_end, uint64_t *__restrict__ lookback, int64_t rcap, int64_t mcap,
        const RunParams *__restrict__ Pr, DevState *__restrict__ rs) {
    using TR = RecTraits<T>;
    using KT = typename MergeKey<T>::type;
    using LT = typename ListOf<T>::type;
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
    const uint32_t epoch = st->epoch + (uint32_t)MAXPASS;
    const int N = P.N;
    const uint64_t nmask = P.nmask;
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
    __syncthreads();
    MergeWarp<T> &ws = s.w[warp];
    int64_t my_w = 0, my_m = 0;
    uint32_t local_status = 0;

    for (;;) {
        int64_t tile = 0;
        if (lane == 0) tile = (int64_t)atomicAdd(&st->tickets[MAXPASS], 1u);
        tile = __shfl_sync(0xFFFFFFFFu, tile, 0);
        if (tile >= ntiles) break;
        const int64_t d0 = tile * MG_TILE;
        const int64_t d1 = (d0 + MG_TILE < tot) ? d0 + MG_TILE : tot;
        const int64_t a0 = splits[tile], a1 = splits[tile + 1], rem_e = rem_end[tile + 1];
        const int64_t b0 = d0 - a0, b1 = d1 - a1;
        const int na = (int)(a1 - a0), nb = (int)(b1 - b0);
        // key of the merged element before the tile
        KT pk{};
        int hp = 0;
        if (lane == 0) {
            if (a0 > 0) { pk = list_key<KT>(L[a0 - 1]); hp = 1; }
            if (b0 > 0) {
                const KT k2 = spawn_key<KT>(S[b0 - 1]);
                if (!hp || k2 > pk) pk = k2;
                hp = 1;
            }
        }
        pk = shfl_key(pk, 0);
        hp = __shfl_sync(0xFFFFFFFFu, hp, 0);
        // load the tile's L and S elements; the S flags go to a bit mask
        for (int q = lane; q < na; q += 32) {
            const LT v = L[a0 + q];
            ws.key[q] = list_key<KT>(v);
            ws.val[q] = make_int2(v.re, v.im);
        }
        for (int q0 = 0; q0 < nb; q0 += 32) {
            const int q = q0 + lane;
            bool f = false;
            if (q < nb) {
                const T v = S[b0 + q];
                ws.key[na + q] = spawn_key<KT>(v);
                ws.val[na + q] = make_int2(TR::re(v), TR::im(v));
                f = TR::flag(v);
            }
            const unsigned fb = __ballot_sync(0xFFFFFFFFu, f);
            if (lane == 0) ws.sflag[q0 >> 5] = fb;
        }
        // spawn records past the tile end that continue its last run
        int64_t rf0 = 0, rf1 = 0, ru0 = 0, ru1 = 0;
        for (int64_t q = b1 + lane; q < rem_e; q += 32) {
            const T g = S[q];
            if (TR::flag(g)) { rf0 += TR::re(g); rf1 += TR::im(g); }
            else { ru0 += TR::re(g); ru1 += TR::im(g); }
        }
        if (rem_e > b1) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                rf0 += __shfl_xor_sync(0xFFFFFFFFu, rf0, off);
                rf1 += __shfl_xor_sync(0xFFFFFFFFu, rf1, off);
                ru0 += __shfl_xor_sync(0xFFFFFFFFu, ru0, off);
                ru1 += __shfl_xor_sync(0xFFFFFFFFu, ru1, off);
            }
        }
        __syncwarp();
        const KT *kL = ws.key;
        const KT *kS = ws.key + na;
        const int2 *vL = ws.val;
        const int2 *vS = ws.val + na;

        // ---- 1. merge: this lane's MG_IPT merged positions, in registers ----
        const int dloc = lane * MG_IPT;
        const int nt = na + nb;
        KT ik[MG_IPT];
        int2 iv[MG_IPT];
        uint32_t hmask = 0, lmask = 0, fmask = 0;   // run heads, elements of L_t, initiator records
        int nk = 0;
        if (dloc < nt) {
            int lo = dloc > nb ? dloc - nb : 0;
            int hi = dloc < na ? dloc : na;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (kL[mid] <= kS[dloc - 1 - mid]) lo = mid + 1;
                else hi = mid;
            }
            int ia = lo, ib = dloc - lo;
            KT prev{};
            bool hprev = false;
            if (dloc == 0) { prev = pk; hprev = hp != 0; }
            else {
                if (ia > 0) { prev = kL[ia - 1]; hprev = true; }
                if (ib > 0) {
                    const KT k2 = kS[ib - 1];
                    if (!hprev || k2 > prev) prev = k2;
                    hprev = true;
                }
            }
            nk = nt - dloc < MG_IPT ? nt - dloc : MG_IPT;
#pragma unroll
            for (int k = 0; k < MG_IPT; ++k) {
                ik[k] = KT{};
                iv[k] = make_int2(0, 0);
                if (k < nk) {
                    bool fromL;
                    if (ia >= na) fromL = false;
                    else if (ib >= nb) fromL = true;
                    else fromL = kL[ia] <= kS[ib];
                    const KT key = fromL ? kL[ia] : kS[ib];
                    ik[k] = key;
                    iv[k] = fromL ? vL[ia] : vS[ib];
                    if (!hprev || key != prev) hmask |= 1u << k;
                    if (fromL) lmask |= 1u << k;
                    else if ((ws.sflag[ib >> 5] >> (ib & 31)) & 1u) fmask |= 1u << k;
                    prev = key;
                    hprev = true;
                    if (fromL) ++ia; else ++ib;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < MG_IPT; ++k) { ik[k] = KT{}; iv[k] = make_int2(0, 0); }
        }
        // ---- 2. segmented reduction of the runs over the lanes ---------------
        SegAgg tail = seg_identity();
#pragma unroll
        for (int k = 0; k < MG_IPT; ++k) {
            if (k < nk) {
                if ((hmask >> k) & 1u) tail = seg_head((lmask >> k) & 1u);
                seg_add(tail, iv[k], ((lmask | fmask) >> k) & 1u);
            }
        }
        const SegAgg carry = seg_warp_exclusive(tail, lane);
        const int my_first_head = nk > 0 ? (int)(hmask & 1u) : 1;
        const int next_first_head = __shfl_down_sync(0xFFFFFFFFu, my_first_head, 1);
        SegAgg run = carry;
        bool owned = carry.h != 0;       // the open run has its head in this tile
        uint32_t omask = 0;
        int2 oval[MG_IPT];
#pragma unroll
        for (int k = 0; k < MG_IPT; ++k) {
            oval[k] = make_int2(0, 0);
            if (k < nk) {
                if ((hmask >> k) & 1u) { run = seg_head((lmask >> k) & 1u); owned = true; }
                seg_add(run, iv[k], ((lmask | fmask) >> k) & 1u);
                bool ends;
                if (k + 1 < nk) ends = ((hmask >> (k + 1)) & 1u) != 0u;
                else if (dloc + k + 1 < nt) ends = next_first_head != 0;
                else {
                    // the tile's last run: add its spawn records that follow the tile
                    ends = true;
                    run.fre += rf0;
                    run.fim += rf1;
                    run.ure += ru0;
                    run.uim += ru1;
                }
                if (ends && owned) {
                    uint64_t ki, kj;
                    key_words(ik[k], nmask, N, ki, kj);
                    bool ni = no_init;
                    if constexpr (BATCH) {
                        kj &= nmask;
                        ni = Pr[batch_run(key_high(ik[k]), run_shift, nruns)].n_a == 0;
                    }
                    const bool open = run.hasL || ni || ki == kj;
                    const int64_t sre = run.fre + (open ? run.ure : 0);
                    const int64_t sim = run.fim + (open ? run.uim : 0);
                    if (sre != 0 || sim != 0) {
                        if (iabs64(sre) > 2147483647ll || iabs64(sim) > 2147483647ll) local_status |= ST_OVERFLOW;
                        omask |= 1u << k;
                        oval[k] = make_int2((int32_t)sre, (int32_t)sim);
                    }
                }
            }
        }
        // ---- 3. compaction: warp scan of the output counts, look-back --------
        const int nout = __popc(omask);
        int x = nout;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += y;
        }
        const uint32_t total = (uint32_t)__shfl_sync(0xFFFFFFFFu, x, 31);
        __syncwarp();                    // every lane is done reading the tile
        uint32_t my_off = (uint32_t)(x - nout);
#pragma unroll
        for (int k = 0; k < MG_IPT; ++k) {
            if ((omask >> k) & 1u) {
                ws.key[my_off] = ik[k];
                ws.val[my_off] = oval[k];
                ++my_off;
            }
        }
        uint64_t *myw = lookback + tile;
        if (lane == 0) lb_store(myw, lb_pack(epoch, tile == 0 ? LB_INC : LB_AGG, total));
        uint64_t excl = 0;
        if (tile > 0) {
            for (int64_t jt = tile - 1;; jt -= 32) {
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
            if (lane == 0) lb_store(myw, lb_pack(epoch, LB_INC, (uint32_t)(excl + total)));
        }
        if (lane == 0 && tile == ntiles - 1) st->M_next = (int64_t)(excl + total);
        __syncwarp();
        const int64_t ob = (int64_t)excl;
        if (ob + (int64_t)total > mcap) {
            if (lane == 0) local_status |= ST_CAPACITY | ST_CAP_LIST;
        } else {
            for (uint32_t q = lane; q < total; q += 32) {
                LT v;
                set_list(v, ws.key[q]);
                v.re = ws.val[q].x;
                v.im = ws.val[q].y;
                out[ob + q] = v;
                uint64_t i, j;
                key_words(ws.key[q], nmask, N, i, j);
                unsigned long long *est = s.est;
                if constexpr (BATCH) {
                    j &= nmask;
                    est = best + (size_t)batch_run(key_high(ws.key[q]), run_shift, nruns) * nobs;
                    atomicAdd(&est[3], (unsigned long long)(iabs64(v.re) + iabs64(v.im)));
                    atomicAdd(&est[4], 1ull);
                } else {
                    my_w += iabs64(v.re) + iabs64(v.im);
                    my_m += 1;
                }
                if (i == j || __popcll(i ^ j) <= 2) add_estimators(s, est, P, i, j, v.re, v.im);
            }
        }
        __syncwarp();
    }
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

}  // namespace ddq
