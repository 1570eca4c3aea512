// Annihilation, part 1: sort the spawn records of one step by configuration
// key (Sec. III.C, annihilation; Sec. II rule (iii)).
//
// Least-significant-digit radix sort in the single-pass ("onesweep") style:
// the digit histograms of every pass were counted by the spawn kernel, so a
// pass reads each record once and writes it once.  A persistent grid takes
// tiles in order from an atomic ticket; each tile ranks its records by digit
// with warp match/ballot multisplit (stable), publishes its per-digit counts,
// resolves its global per-digit offsets by decoupled look-back over earlier
// tiles (bounded waits), stages the tile in digit order in shared memory and
// writes runs of equal digits to consecutive global addresses.  The initiator
// flag is carried, never sorted.
//
// Two record layouts: 16-byte Rec (any key width), and 8-byte packed records
// for keys of at most 32 bits (2N <= 32):
//   bits 63..32 key, bit 31 initiator flag, bits 29..15 Delta im, 14..0 Delta re
// (15-bit two's complement each), which halves the bytes every pass moves.
#pragma once

#include "common.cuh"

namespace ddq {

template <typename T> struct RecTraits;

template <> struct RecTraits<Rec> {
    static constexpr int IPT = 8;      // records per thread in a radix tile
    static constexpr int MINB = 3;     // resident blocks per SM the pass is compiled for
    __device__ __forceinline__ static uint64_t key(const Rec &r) { return r.key & KEY_MASK; }
    __device__ __forceinline__ static uint32_t digit(const Rec &r, int shift) {
        return (uint32_t)((r.key & KEY_MASK) >> shift) & 0xFFu;
    }
    __device__ __forceinline__ static bool flag(const Rec &r) { return (r.key & FLAG_BIT) != 0ull; }
    __device__ __forceinline__ static int32_t re(const Rec &r) { return r.re; }
    __device__ __forceinline__ static int32_t im(const Rec &r) { return r.im; }
    __device__ __forceinline__ static Rec empty() { Rec r; r.key = 0; r.re = 0; r.im = 0; return r; }
};

// Two-word records: digits of the ket word at shifts 0..63, of the bra word at 64..127.
template <> struct RecTraits<RecW> {
    static constexpr int IPT = 8;      // at 3 blocks per SM: measured faster than 10 at 2 and 6 at 3
    static constexpr int MINB = 3;
    __device__ __forceinline__ static uint32_t digit(const RecW &r, int shift) {
        return (uint32_t)(shift < 64 ? (r.lo >> shift) : (r.hi >> (shift - 64))) & 0xFFu;
    }
    __device__ __forceinline__ static bool flag(const RecW &r) { return (r.re & 1) != 0; }
    __device__ __forceinline__ static int32_t re(const RecW &r) { return r.re >> 1; }
    __device__ __forceinline__ static int32_t im(const RecW &r) { return r.im; }
    __device__ __forceinline__ static RecW empty() { RecW r; r.lo = 0; r.hi = 0; r.re = 0; r.im = 0; return r; }
};

constexpr int PK_LIM = 16383;          // largest |Delta| of one packed record
constexpr int WK_LIM = 1 << 29;        // largest |Delta| of one two-word spawn record

template <> struct RecTraits<uint64_t> {
    static constexpr int IPT = 16;
    static constexpr int MINB = 3;
    __device__ __forceinline__ static uint64_t key(uint64_t r) { return r >> 32; }
    __device__ __forceinline__ static uint32_t digit(uint64_t r, int shift) {
        return (uint32_t)((r >> 32) >> shift) & 0xFFu;
    }
    __device__ __forceinline__ static bool flag(uint64_t r) { return ((r >> 31) & 1ull) != 0ull; }
    __device__ __forceinline__ static int32_t re(uint64_t r) { return ((int32_t)((uint32_t)r << 17)) >> 17; }
    __device__ __forceinline__ static int32_t im(uint64_t r) { return ((int32_t)((uint32_t)(r >> 15) << 17)) >> 17; }
    __device__ __forceinline__ static uint64_t empty() { return 0ull; }
};

// packed record; |re|, |im| <= PK_LIM
__device__ __forceinline__ uint64_t pack_rec(uint64_t key, bool flag, int re, int im) {
    return (key << 32) | (flag ? (1ull << 31) : 0ull) | ((uint64_t)((uint32_t)im & 0x7FFFu) << 15) |
           (uint64_t)((uint32_t)re & 0x7FFFu);
}

// 8-byte record for keys of 33 to 40 bits (lattices of 17 to 20 sites, and
// batches whose run id takes the key past 32 bits):
//   bits 63..24 key, bit 23 initiator flag, bits 22..12 Delta im, 11..0 Delta re
// (11- and 12-bit two's complement); larger aggregated counts become several
// records.
struct P40 {
    uint64_t v;
};
constexpr int P40_LIM = 1023;          // largest |Delta| of one such record

template <> struct RecTraits<P40> {
    static constexpr int IPT = 16;
    static constexpr int MINB = 3;
    __device__ __forceinline__ static uint64_t key(P40 r) { return r.v >> 24; }
    __device__ __forceinline__ static uint32_t digit(P40 r, int shift) {
        return (uint32_t)((r.v >> 24) >> shift) & 0xFFu;
    }
    __device__ __forceinline__ static bool flag(P40 r) { return ((r.v >> 23) & 1ull) != 0ull; }
    __device__ __forceinline__ static int32_t re(P40 r) { return ((int32_t)((uint32_t)r.v << 20)) >> 20; }
    __device__ __forceinline__ static int32_t im(P40 r) { return ((int32_t)((uint32_t)(r.v >> 12) << 21)) >> 21; }
    __device__ __forceinline__ static P40 empty() { return P40{0ull}; }
};

// |re|, |im| <= P40_LIM
__device__ __forceinline__ P40 pack_p40(uint64_t key, bool flag, int re, int im) {
    return P40{(key << 24) | (flag ? (1ull << 23) : 0ull) | ((uint64_t)((uint32_t)im & 0x7FFu) << 12) |
               (uint64_t)((uint32_t)re & 0xFFFu)};
}

constexpr int RX_TPB = 256;                  // one thread per digit value
constexpr int RX_WARPS = RX_TPB / 32;
constexpr int RX_TILE_MIN = RX_TPB * 6;      // smallest tile (sizes the look-back words)
constexpr int LB_BATCH = 16;                 // look-back words read together

// IPT: records per thread of a tile (default the record type's; the tuner
// picks among the instantiated alternatives)
template <typename T, int IPT = RecTraits<T>::IPT>
struct RadixShared {
    T stage[RX_TPB * IPT];
    uint32_t whist[RX_WARPS][256];
    uint32_t bucket[256];      // start of each digit's bucket in the output
    uint32_t dstart[256];      // start of each digit inside the staged tile
    int64_t gbase[256];        // output index of staged position 0 of each digit
    uint32_t scan_tmp[RX_WARPS];
    int64_t tile;
};

// Digit histograms of every pass over st->R records (used when the records do
// not come from the spawn kernel, which counts them as it writes them).  Pass
// p reads bits 8p.. of the key for p < nlo, and bits 64 + 8(p - nlo).. after
// (two-word records: the ket word, then the bra word).
template <typename T>
__global__ void __launch_bounds__(RX_TPB)
k_digit_histogram(const T *__restrict__ in, DevState *__restrict__ st, int npass, int nlo) {
    __shared__ uint32_t h[MAXPASS][256];
    const int tid = threadIdx.x;
    if (block_stopped(st)) return;
    for (int q = tid; q < MAXPASS * 256; q += RX_TPB) (&h[0][0])[q] = 0u;
    __syncthreads();
    const int64_t R = st->R;
    for (int64_t q = (int64_t)blockIdx.x * RX_TPB + tid; q < R; q += (int64_t)gridDim.x * RX_TPB) {
        const T r = in[q];
        for (int p = 0; p < npass; ++p)
            atomicAdd(&h[p][RecTraits<T>::digit(r, p < nlo ? 8 * p : 64 + 8 * (p - nlo))], 1u);
    }
    __syncthreads();
    for (int q = tid; q < npass * 256; q += RX_TPB)
        if ((&h[0][0])[q]) atomicAdd(&st->hist[q >> 8][q & 255], (&h[0][0])[q]);
}

// blocks per SM a tile size is compiled for: more records per thread need more registers
template <typename T, int IPT> struct RadixBlocks {
    static constexpr int value = IPT > RecTraits<T>::IPT ? 2 : RecTraits<T>::MINB;
};

template <typename T, int IPT = RecTraits<T>::IPT>
__global__ void __launch_bounds__(RX_TPB, (RadixBlocks<T, IPT>::value))
k_radix_pass(const T *__restrict__ in, T *__restrict__ out, DevState *__restrict__ st,
             uint64_t *__restrict__ lookback, int pass, int shift, int64_t cap) {
    using TR = RecTraits<T>;
    constexpr int TILE = RX_TPB * IPT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RadixShared<T, IPT> &s = *reinterpret_cast<RadixShared<T, IPT> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (block_stopped(st)) return;
    int64_t R = st->R;
    if (R > cap) R = cap;
    const int64_t ntiles = (R + TILE - 1) / TILE;
    const uint32_t epoch = st->epoch + (uint32_t)pass;

    // exclusive scan of this pass's global histogram -> bucket starts
    {
        const uint32_t v = st->hist[pass][tid];
        uint32_t x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) s.scan_tmp[warp] = x;
        __syncthreads();
        uint32_t pre = 0, all = 0;
        for (int w = 0; w < RX_WARPS; ++w) {
            if (w < warp) pre += s.scan_tmp[w];
            all += s.scan_tmp[w];
        }
        s.bucket[tid] = pre + x - v;
        // the counted records must be exactly the records to sort; otherwise
        // the bucket offsets would point outside the output (every block reads
        // the same histogram, so every block leaves here together)
        if ((int64_t)all != R) {
            if (blockIdx.x == 0 && tid == 0) atomicOr(&st->status, ST_CAPACITY | ST_CAP_SPAWN);
            return;
        }
        __syncthreads();
    }

    for (;;) {
        if (tid == 0) s.tile = (int64_t)atomicAdd(&st->tickets[pass], 1u);
        __syncthreads();
        const int64_t tile = s.tile;
        if (tile >= ntiles) break;
        const int64_t t0 = tile * TILE;
        for (int q = tid; q < RX_WARPS * 256; q += RX_TPB) (&s.whist[0][0])[q] = 0u;
        __syncthreads();

        // load: warp w owns records [t0 + w*32*IPT, +32*IPT), item q at + q*32 + lane
        T r[IPT];
        uint32_t dg[IPT];
        uint32_t rk[IPT];
        const int64_t wbase = t0 + (int64_t)warp * 32 * IPT;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int64_t idx = wbase + q * 32 + lane;
            if (idx < R) {
                r[q] = in[idx];
                dg[q] = TR::digit(r[q], shift);
            } else {
                r[q] = TR::empty();
                dg[q] = 0x100u + lane;            // unique sentinel, never counted
            }
        }
        // stable warp multisplit rank
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, dg[q]);
            const unsigned below = peers & ((1u << lane) - 1u);
            uint32_t base = 0;
            if (dg[q] < 256u) base = s.whist[warp][dg[q]];
            __syncwarp();
            if (dg[q] < 256u && below == 0u) s.whist[warp][dg[q]] = base + (uint32_t)__popc(peers);
            __syncwarp();
            rk[q] = base + (uint32_t)__popc(below);
        }
        __syncthreads();

        // per digit (thread tid = digit): warp offsets, tile count, tile-local start
        uint32_t cnt = 0;
        for (int w = 0; w < RX_WARPS; ++w) {
            const uint32_t c = s.whist[w][tid];
            s.whist[w][tid] = cnt;
            cnt += c;
        }
        uint64_t *my = lookback + (size_t)tile * 256 + tid;
        if (tile == 0) lb_store(my, lb_pack(epoch, LB_INC, cnt));
        else lb_store(my, lb_pack(epoch, LB_AGG, cnt));
        {
            uint32_t x = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
                if (lane >= off) x += y;
            }
            if (lane == 31) s.scan_tmp[warp] = x;
            __syncthreads();
            uint32_t pre = 0;
            for (int w = 0; w < warp; ++w) pre += s.scan_tmp[w];
            s.dstart[tid] = pre + x - cnt;
        }
        __syncthreads();
        // stage in digit order (tile-local positions need no look-back; the
        // records' registers are free again before it)
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (dg[q] < 256u) {
                const uint32_t pos = s.dstart[dg[q]] + s.whist[warp][dg[q]] + rk[q];
                s.stage[pos] = r[q];
            }
        }
        // decoupled look-back for this digit, reading LB_BATCH earlier tiles at a time
        uint64_t excl = 0;
        {
            bool done = tile == 0;
            for (int64_t jt = tile - 1; !done; jt -= LB_BATCH) {
                uint64_t w[LB_BATCH];
#pragma unroll
                for (int k = 0; k < LB_BATCH; ++k)
                    w[k] = jt - k >= 0 ? *(volatile const uint64_t *)(lookback + (size_t)(jt - k) * 256 + tid)
                                       : lb_pack(epoch, LB_INC, 0u);
#pragma unroll
                for (int k = 0; k < LB_BATCH; ++k) {
                    if (!done) {
                        uint64_t v = w[k];
                        if (!lb_ready(v, epoch)) v = lb_wait(lookback + (size_t)(jt - k) * 256 + tid, epoch, &st->status);
                        excl += (uint32_t)v;
                        if (((v >> 32) & 3ull) != LB_AGG) done = true;     // inclusive (or timed out)
                    }
                }
            }
        }
        if (tile > 0) lb_store(my, lb_pack(epoch, LB_INC, (uint32_t)(excl + cnt)));
        s.gbase[tid] = (int64_t)s.bucket[tid] + (int64_t)excl - (int64_t)s.dstart[tid];
        __syncthreads();
        int64_t nvalid = R - t0;
        if (nvalid > TILE) nvalid = TILE;
        bool bad = false;
        for (int q = tid; q < nvalid; q += RX_TPB) {
            const T v = s.stage[q];
            const uint32_t d = TR::digit(v, shift);
            const int64_t o = s.gbase[d] + q;
            // offsets come from the histograms and the look-back; one that
            // falls outside [0, R) (inconsistent counts, or a timed-out wait)
            // is reported, never written
            if ((uint64_t)o < (uint64_t)R) out[o] = v;
            else bad = true;
        }
        if (bad) atomicOr(&st->status, ST_CAPACITY | ST_CAP_SPAWN);
        __syncthreads();
    }
}

}  // namespace ddq
