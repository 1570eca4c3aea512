// Annihilation with two-word keys (more than 31 sites) in the hashed order
// (Sec. III.C, annihilation: only equal configurations must meet, so any
// total order of the keys serves, provided the walker list and the sorted
// spawn records share it).
//
// The stored bra word of a key is bra ^ (ket_mix(ket) & hash_mask); the list
// and the spawn records are ordered by (stored bra word, ket); a batch keeps
// its run id above the hash bits of that word.  The digit passes sort the
// spawn records on the stored bra word only (8 passes of 8 bits instead of
// up to 16 over both words).  Records with equal stored bra
// words are then in the order the passes left them; with a 64-bit hash two
// different keys share a stored bra word with probability about
// n^2 / 2^65 per step (n distinct keys).  Afterwards:
//   k_hash_check  marks every adjacent pair that shares a stored bra word and
//                 has its kets in decreasing order (none: already sorted);
//   k_hash_repair sorts each group of equal stored bra words that holds a
//                 marked pair by ket, one block per group: in shared memory
//                 (bitonic network) up to HO_SMEM_N records, else by
//                 odd-even transposition in place.
// Equal keys may stay in any order: the merge sums them.
#pragma once

#include "common.cuh"

namespace ddq {

constexpr int HO_TPB = 256;
constexpr int HO_MAXV = 16384;      // marked pairs recorded per step (more: capacity status)
constexpr int HO_SMEM_N = 1024;     // groups of at most this many records sort in shared memory

// Positions q of the sorted records S[0, R) with S[q].hi == S[q+1].hi and
// S[q].lo > S[q+1].lo into viol[0, min(count, HO_MAXV)), counted in st->hviol.
__global__ void __launch_bounds__(HO_TPB)
k_hash_check(const RecW *__restrict__ S, DevState *__restrict__ st, int64_t *__restrict__ viol, int64_t cap) {
    if (block_stopped(st)) return;
    int64_t R = st->R;
    if (R > cap) R = cap;
    for (int64_t q = (int64_t)blockIdx.x * HO_TPB + threadIdx.x; q + 1 < R; q += (int64_t)gridDim.x * HO_TPB) {
        const uint64_t h0 = S[q].hi, h1 = S[q + 1].hi;
        if (h0 == h1 && S[q].lo > S[q + 1].lo) {
            const uint32_t n = atomicAdd(&st->hviol, 1u);
            if (n < (uint32_t)HO_MAXV) viol[n] = q;
        }
    }
}

// Sort by ket each group of equal stored bra words holding a marked pair; the
// group of the smallest marked position in it is sorted by one block.
__global__ void __launch_bounds__(HO_TPB)
k_hash_repair(RecW *__restrict__ S, DevState *__restrict__ st, const int64_t *__restrict__ viol, int64_t cap) {
    __shared__ RecW buf[HO_SMEM_N];
    __shared__ uint16_t ix[HO_SMEM_N];
    __shared__ long long s_best;
    const int tid = threadIdx.x;
    if (block_stopped(st)) return;
    const uint32_t nv = st->hviol;
    if (nv > (uint32_t)HO_MAXV) {
        if (blockIdx.x == 0 && tid == 0) atomicOr(&st->status, ST_CAPACITY | ST_CAP_SPAWN);
        return;
    }
    int64_t R = st->R;
    if (R > cap) R = cap;
    for (uint32_t v = blockIdx.x; v < nv; v += gridDim.x) {
        const int64_t q = viol[v];
        if (q < 0 || q + 1 >= R) continue;      // not a pair of this step's records
        const uint64_t h = S[q].hi;
        // group [gs, ge): the records around q with stored bra word h
        int64_t gs = 0, ge = R;
        for (int64_t base = q; base > 0; base -= HO_TPB) {
            const int64_t p = base - 1 - tid;
            if (tid == 0) s_best = -1;
            __syncthreads();
            if (p >= 0 && S[p].hi != h) atomicMax(&s_best, (long long)p);
            __syncthreads();
            const int64_t b = s_best;
            __syncthreads();
            if (b >= 0) { gs = b + 1; break; }
        }
        for (int64_t base = q + 2; base < R; base += HO_TPB) {
            const int64_t p = base + tid;
            if (tid == 0) s_best = R;
            __syncthreads();
            if (p < R && S[p].hi != h) atomicMin(&s_best, (long long)p);
            __syncthreads();
            const int64_t b = s_best;
            __syncthreads();
            if (b < R) { ge = b; break; }
        }
        // another marked pair earlier in the group: that one's block sorts it
        bool later = false;
        for (uint32_t u = tid; u < nv; u += HO_TPB) {
            const int64_t o = viol[u];
            later |= o >= gs && o < q;
        }
        if (__syncthreads_or(later)) continue;
        const int64_t n = ge - gs;
        if (n <= HO_SMEM_N) {
            // bitonic sort of indices over the next power of two; indices past
            // n are padding and order last whatever their ket
            int np = 2;
            while (np < n) np <<= 1;
            for (int k = tid; k < np; k += HO_TPB) {
                if (k < n) buf[k] = S[gs + k];
                ix[k] = (uint16_t)k;
            }
            __syncthreads();
            for (int k = 2; k <= np; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int i = tid; i < np; i += HO_TPB) {
                        const int l = i ^ j;
                        if (l > i) {
                            const int a = ix[i], b = ix[l];
                            const bool pa = a >= n, pb = b >= n;
                            const bool greater = pa != pb ? pa : (!pa && buf[a].lo > buf[b].lo);
                            const bool up = (i & k) == 0;
                            if (greater == up) { ix[i] = (uint16_t)b; ix[l] = (uint16_t)a; }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int k = tid; k < n; k += HO_TPB) S[gs + k] = buf[ix[k]];
            __syncthreads();
        } else {
            // odd-even transposition in place: sorted once an even and an odd
            // round in a row exchange nothing
            int quiet = 0;
            for (int64_t round = 0; quiet < 2; ++round) {
                bool sw = false;
                for (int64_t k = gs + (round & 1) + 2 * (int64_t)tid; k + 1 < ge; k += 2 * HO_TPB) {
                    const RecW a = S[k], b = S[k + 1];
                    if (a.lo > b.lo) {
                        S[k] = b;
                        S[k + 1] = a;
                        sw = true;
                    }
                }
                quiet = __syncthreads_or(sw) ? 0 : quiet + 1;
            }
        }
    }
}

}  // namespace ddq
