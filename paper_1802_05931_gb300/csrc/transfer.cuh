// Walker lists in and out of the device in the caller's layout: four arrays
// (ket words, bra words, re, im; sorted by bra, then ket), copied over the
// host link as they are and converted to and from the packed list records on
// the device.  Nothing of the method's arithmetic happens here.
#pragma once

#include "common.cuh"

namespace ddq {

constexpr int TX_TPB = 256;

// hmask: the hashed order's mask of the ket hash in the stored bra word
// (two-word keys of a single run; 0 otherwise)
__device__ __forceinline__ void put_list(Rec &v, uint64_t ket, uint64_t bra, int N, uint64_t) {
    v.key = (bra << N) | ket;
}
__device__ __forceinline__ void put_list(RecW &v, uint64_t ket, uint64_t bra, int, uint64_t hmask) {
    v.lo = ket;
    v.hi = bra_swap(ket, bra, hmask);
}
__device__ __forceinline__ void get_list(const Rec &v, int N, uint64_t mask, uint64_t &ket, uint64_t &bra) {
    ket = v.key & mask;
    bra = (v.key >> N) & mask;
}
__device__ __forceinline__ void get_list(const RecW &v, int, uint64_t mask, uint64_t &ket, uint64_t &bra) {
    ket = v.lo;
    bra = v.hi & mask;
}

// Pack n caller entries into list records and check them: every word within
// the lattice's N bits, no empty entry, keys strictly increasing in (bra,
// ket) order.  acc[0] += sum |re| + |im|; acc[1] != 0 when any entry fails.
// With hmask != 0 the records carry the stored bra words of the hashed order
// and still need sorting in it.
template <typename LT>
__global__ void __launch_bounds__(TX_TPB)
k_import_pack(const uint64_t *__restrict__ ket, const uint64_t *__restrict__ bra, const int32_t *__restrict__ re,
              const int32_t *__restrict__ im, int64_t n, int N, uint64_t mask, uint64_t hmask, LT *__restrict__ out,
              unsigned long long *__restrict__ acc) {
    __shared__ unsigned long long s_w[TX_TPB / 32];
    int64_t w = 0;
    bool bad = false;
    for (int64_t q = (int64_t)blockIdx.x * TX_TPB + threadIdx.x; q < n; q += (int64_t)gridDim.x * TX_TPB) {
        const uint64_t k = ket[q], b = bra[q];
        const int32_t x = re[q], y = im[q];
        bad |= ((k | b) & ~mask) != 0ull || (x == 0 && y == 0);
        if (q > 0) {
            const uint64_t pk = ket[q - 1], pb = bra[q - 1];
            bad |= pb > b || (pb == b && pk >= k);
        }
        w += (int64_t)(x < 0 ? -(int64_t)x : x) + (int64_t)(y < 0 ? -(int64_t)y : y);
        LT v;
        put_list(v, k, b, N, hmask);
        v.re = x;
        v.im = y;
        out[q] = v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xFFFFFFFFu, w, off);
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(&acc[1], 1ull);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = (unsigned long long)w;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < TX_TPB / 32; ++k) t += s_w[k];
        if (t) atomicAdd(&acc[0], t);
    }
}

// Check n list records already in place (the caller's 16-byte records): key
// within kmask, no empty entry, keys strictly increasing.  acc as k_import_pack.
__global__ void __launch_bounds__(TX_TPB)
k_check_records(const Rec *__restrict__ L, int64_t n, uint64_t kmask, unsigned long long *__restrict__ acc) {
    __shared__ unsigned long long s_w[TX_TPB / 32];
    int64_t w = 0;
    bool bad = false;
    for (int64_t q = (int64_t)blockIdx.x * TX_TPB + threadIdx.x; q < n; q += (int64_t)gridDim.x * TX_TPB) {
        const Rec v = L[q];
        bad |= (v.key & ~kmask) != 0ull || (v.re == 0 && v.im == 0);
        if (q > 0) bad |= L[q - 1].key >= v.key;
        w += (int64_t)(v.re < 0 ? -(int64_t)v.re : v.re) + (int64_t)(v.im < 0 ? -(int64_t)v.im : v.im);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xFFFFFFFFu, w, off);
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(&acc[1], 1ull);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = (unsigned long long)w;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < TX_TPB / 32; ++k) t += s_w[k];
        if (t) atomicAdd(&acc[0], t);
    }
}

// The list records [0, m) as 12-byte records {u32 key, i32 re, i32 im} (keys
// of at most 32 bits), three words per entry.
__global__ void __launch_bounds__(TX_TPB)
k_pack_records32(const Rec *__restrict__ L, int64_t m, uint32_t *__restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * TX_TPB + threadIdx.x; q < m; q += (int64_t)gridDim.x * TX_TPB) {
        const Rec v = L[q];
        out[3 * q] = (uint32_t)v.key;
        out[3 * q + 1] = (uint32_t)v.re;
        out[3 * q + 2] = (uint32_t)v.im;
    }
}

// 12-byte records back into list records, with the checks of k_check_records.
__global__ void __launch_bounds__(TX_TPB)
k_unpack_records32(const uint32_t *__restrict__ in, int64_t n, uint64_t kmask, Rec *__restrict__ L,
                   unsigned long long *__restrict__ acc) {
    __shared__ unsigned long long s_w[TX_TPB / 32];
    int64_t w = 0;
    bool bad = false;
    for (int64_t q = (int64_t)blockIdx.x * TX_TPB + threadIdx.x; q < n; q += (int64_t)gridDim.x * TX_TPB) {
        Rec v;
        v.key = in[3 * q];
        v.re = (int32_t)in[3 * q + 1];
        v.im = (int32_t)in[3 * q + 2];
        bad |= (v.key & ~kmask) != 0ull || (v.re == 0 && v.im == 0);
        if (q > 0) bad |= (uint64_t)in[3 * (q - 1)] >= v.key;
        w += (int64_t)(v.re < 0 ? -(int64_t)v.re : v.re) + (int64_t)(v.im < 0 ? -(int64_t)v.im : v.im);
        L[q] = v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xFFFFFFFFu, w, off);
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(&acc[1], 1ull);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = (unsigned long long)w;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < TX_TPB / 32; ++k) t += s_w[k];
        if (t) atomicAdd(&acc[0], t);
    }
}

// Unpack list records [0, m) into the caller's layout (the batch run id, if
// any, dropped from the bra word).
template <typename LT>
__global__ void __launch_bounds__(TX_TPB)
k_export_unpack(const LT *__restrict__ L, int64_t m, int N, uint64_t mask, uint64_t *__restrict__ ket,
                uint64_t *__restrict__ bra, int32_t *__restrict__ re, int32_t *__restrict__ im) {
    for (int64_t q = (int64_t)blockIdx.x * TX_TPB + threadIdx.x; q < m; q += (int64_t)gridDim.x * TX_TPB) {
        const LT v = L[q];
        uint64_t k, b;
        get_list(v, N, mask, k, b);
        ket[q] = k;
        bra[q] = b;
        re[q] = v.re;
        im[q] = v.im;
    }
}

// Copy of a hashed-order list with its plain bra words (to be sorted in the
// (bra, ket) order of the caller's layout).
__global__ void __launch_bounds__(TX_TPB)
k_unhash(const RecW *__restrict__ L, int64_t m, uint64_t hmask, RecW *__restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * TX_TPB + threadIdx.x; q < m; q += (int64_t)gridDim.x * TX_TPB) {
        RecW v = L[q];
        v.hi = bra_swap(v.lo, v.hi, hmask);
        out[q] = v;
    }
}

// Entries [out[0], out[1]) of batch run k in a list sorted by (run, bra, ket):
// two binary searches on the run id (the key's high word from bit rs).
__device__ __forceinline__ uint64_t list_run(const Rec &v, int rs) { return v.key >> rs; }
__device__ __forceinline__ uint64_t list_run(const RecW &v, int rs) { return v.hi >> rs; }

template <typename LT>
__global__ void k_run_bounds(const LT *__restrict__ L, const DevState *__restrict__ st, int rs, uint64_t k,
                             int64_t *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int64_t M = st->M;
    int64_t lo = 0, hi = M;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (list_run(L[mid], rs) < k) lo = mid + 1; else hi = mid;
    }
    out[0] = lo;
    hi = M;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (list_run(L[mid], rs) <= k) lo = mid + 1; else hi = mid;
    }
    out[1] = lo;
}

}  // namespace ddq
