// Shared definitions of the DDQMC GPU path: record layout, per-run constant
// tables, the device-resident step state, Philox4x32-10 and the series
// logarithm.  Nothing here is shared with the CPU oracle.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ddq {

constexpr int MAXN = 64;                      // sites: one 64-bit spin word per side
constexpr int NPACK = 31;                     // up to here ket and bra pack into one 62-bit key
constexpr int MAXB = 128;                     // bonds (2N for a periodic 2D lattice)
constexpr int MAXK = 2 * MAXB + 3 * MAXN;     // moves per configuration (bond flips, field flips, jumps)
constexpr int NOBS_MAX = 5 + MAXN + 3 * MAXB + 4 + 2 * MAXN + 2;
constexpr int LEVELS = 32;                    // blocking levels (block length 2^l)
constexpr int MAXPASS = 16;                   // radix passes of 8 bits over at most 128 key bits

constexpr uint32_t ST_CAPACITY = 1u, ST_OVERFLOW = 2u, ST_TIMEOUT = 4u;
constexpr uint32_t ST_CAP_LIST = 8u, ST_CAP_SPAWN = 16u;   // which capacity ran out (with ST_CAPACITY)

// Spawn records carry the parent's initiator flag in bit 63; list keys never do.
constexpr uint64_t FLAG_BIT = 1ull << 63;
constexpr uint64_t KEY_MASK = ~FLAG_BIT;

// One occupied configuration or one spawn record: packed key (bra << N | ket)
// and the signed real / imaginary walker populations.  16 bytes, so a whole
// record moves with one 128-bit load or store.
struct __align__(16) Rec {
    uint64_t key;
    int32_t re;
    int32_t im;
};

// Two-word record for N > 31 sites: lo = ket word, hi = bra word (canonical
// order: by hi, then lo), 24 bytes.  In a spawn record the re field holds
// 2 * Delta re + initiator flag; list entries hold plain populations.
struct __align__(8) RecW {
    uint64_t lo, hi;
    int32_t re;
    int32_t im;
};

// Mixing function of the hashed order of two-word keys: the 64-bit
// finalizer of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), a bijection
// of 64-bit words whose every output bit depends on every input bit.
__host__ __device__ __forceinline__ uint64_t ket_mix(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Stored bra word of a two-word key in the hashed order, and back (the same
// xor): the pair (ket, stored bra) still determines the key, so the list
// keeps 24-byte records and sorts the stored bra word as its leading word.
__host__ __device__ __forceinline__ uint64_t bra_swap(uint64_t ket, uint64_t bra, uint64_t hash_mask) {
    return hash_mask ? bra ^ (ket_mix(ket) & hash_mask) : bra;
}

// Walker-list record of each spawn-record type.
template <typename T> struct ListOf { using type = Rec; };
template <> struct ListOf<RecW> { using type = RecW; };

// Look-back status words: [epoch:30][flag:2][value:32].
constexpr uint64_t LB_AGG = 1ull, LB_INC = 2ull;
__device__ __forceinline__ uint64_t lb_pack(uint32_t epoch, uint64_t flag, uint32_t value) {
    return ((uint64_t)(epoch & 0x3FFFFFFFu) << 34) | (flag << 32) | (uint64_t)value;
}

// Per-run constants, computed on the host at create time.
struct RunParams {
    int32_t N, B, K, nobs, npass, n_a, guide_kind, control;
    int32_t sgn_h[2];          // sign of Jx - Jy (aligned bond) and Jx + Jy (anti-aligned)
    int32_t sgn_jz;
    int32_t pad0;
    uint64_t nmask;            // (1 << N) - 1
    uint64_t seed;
    int64_t target;
    int64_t t_eq_span;         // steps from the first variable-shift step to the first sample
    double gamma_half, dt, shift_gain;
    uint64_t jump_q;
    uint64_t bond_m[MAXB];
    int32_t bond_a[MAXB], bond_b[MAXB];
    uint64_t rate_q[MAXB][2][4];      // [bond][anti-aligned][importance class]
    uint32_t cross_int[2 * MAXB + 1];
    uint64_t cross_frac[2 * MAXB + 1];
    int8_t pair_bond[MAXN * MAXN];    // bond index of an (a, b) site pair, -1 if none
    // square-lattice geometry for the mask formulation of the rates
    int32_t Lx, shD;                  // row length; Lx * (Ly - 1)
    uint64_t ER, ED;                  // sites owning a bond to the right / below
    uint64_t LC, LR;                  // last column / last row
    int8_t rn[MAXN], dn[MAXN];        // right / lower neighbour of each site
    int32_t uniform;                  // 1 if every bond has the same rate table
    int32_t pad1;
    int32_t pass_shift[MAXPASS];      // key bit where the digit of each radix pass starts
    // in-plane field h sum_k sigma^x_k (axis 0), sigma^y_k (axis 1), or
    // (cos t sigma^x_k + sin t sigma^y_k) (axis 2: each flip is two moves, the
    // x part with the tables frate_q / ufrate.. and sign sgn_hf, then the y
    // part with frate_q2 / ufrate..2 and sign sgn_hf2)
    int32_t field_on, field_axis, sgn_hf, sgn_hf2;
    uint64_t frate_q[MAXN][4];        // site flip of site k, [importance class]
    uint64_t ufrate[4];               // the same when every site has the same table
    uint64_t Emorton;                 // bond-existence mask, bit 2k = right bond of k, 2k+1 = lower (sites < 32)
    uint64_t Emorton_hi;              // the same for sites 32..63 (bit 2(k-32), 2(k-32)+1)
    uint64_t urate8[8];               // rate of group 4*anti + class when every bond has the same table
    // A batch of runs shares one walker store with the run id in the key's
    // high bits (bit run_shift up: 2N for one-word keys; for two-word keys
    // N of the bra word, or in the hashed order above the hash bits if they
    // reach past N).  nruns = 0 for a single run.
    int32_t nruns, run_shift;
    // the uniform tables in the forms the light path reads (a single run
    // derives them in shared memory; a batch reads each run's copy)
    uint32_t urate32[8];
    float uinv[8];
    uint32_t ufrate32[4];
    float ufinv[4];
    float jinv;
    // a run of a batch that was retired (0): its configurations spawn nothing
    // and leave the list at the next merge; the other runs do not notice
    int32_t active;
    // Hashed order of two-word keys: the stored bra word is
    // bra ^ (ket_mix(ket) & hash_mask) (a batch's run id above the mask's
    // bits), the digit passes cover the stored bra word only, and a repair
    // kernel puts records with equal stored bra words in ket order
    // (hashed = 1).  hash_mask = 0, hashed = 0: the plain order.
    int32_t hashed;
    uint64_t hash_mask;
    uint64_t frate_q2[MAXN][4];       // axis 2: the y part of a site flip, [importance class]
    uint64_t ufrate2[4];
    uint32_t ufrate32_2[4];
    float ufinv2[4];
};

// Device-resident state of a run, updated by the kernels of each step.  A
// batch has one for the shared step machinery (list and spawn counts,
// tickets, histograms, status) and one per run (shift, population control,
// death table, estimators; M there counts the run's own entries).
struct DevState {
    int64_t t, t_var, t_eq, q_prev;
    double S;
    int32_t variable;
    uint32_t status;
    int64_t M;                 // entries of the current list
    int64_t M_next;            // entries of the merged list (written by the last merge tile)
    int64_t R;                 // spawn records of the step in progress
    int64_t R_last;            // spawn records of the last completed step
    uint32_t epoch;            // look-back epoch of the step in progress
    uint32_t hviol;            // hashed order: out-of-order neighbours found after the digit passes
    uint32_t tickets[MAXPASS + 16];   // tile tickets: [0, MAXPASS) radix passes, MAXPASS merge
    int64_t walker_steps;      // sum over completed steps of the walkers stepped
    int64_t W_cur;             // sum |re| + |im| of the current list
    int64_t n_app;             // samples accumulated for blocking
    int64_t sum_M, sum_R, sum_Mnext;   // totals over completed steps: entries stepped, spawn records, merged entries
    uint32_t d_int[2 * MAXN + 1];
    uint64_t d_frac[2 * MAXN + 1];
    int32_t d_sgn[2 * MAXN + 1];
    int64_t est[NOBS_MAX];     // estimator numerators of the step in progress
    int64_t last_est[NOBS_MAX];
    uint32_t hist[MAXPASS][256];
};

// One blocking cell: observable k at level l (block length 2^l).
struct BlkCell {
    int64_t n;                 // completed blocks
    int64_t sx;                // sum of block sums
    __int128 sxx;              // sum of squared block sums
    __int128 sxy;              // sum of block sum x trace block sum
    int64_t pend_x, pend_y;    // pending half-block
    int32_t has_pend;
    int32_t pad;
};

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with a Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t p0 = 0xD2511F53u * c.x, h0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t p1 = 0xCD9E8D57u * c.z, h1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(h1 ^ c.y ^ k0, p1, h0 ^ c.w ^ k1, p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Natural logarithm from log x = e ln2 + 2 atanh((m-1)/(m+1)), x = m 2^e,
// m in (1/sqrt2, sqrt2], atanh by its odd power series (15 terms), every
// operation an explicitly rounded IEEE double operation in a fixed order.
__device__ __forceinline__ double series_log(double x) {
    if (!(x > 0.0)) return 0.0;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    int e = (int)((bits >> 52) & 0x7FFull);
    if (e == 0) return 0.0;
    e -= 1023;
    double m = __longlong_as_double((long long)((bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
    if (m > 1.4142135623730951) { m = __dmul_rn(m, 0.5); e += 1; }
    const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double z = __dmul_rn(s, s);
    double p = __ddiv_rn(1.0, 29.0);
    for (int k = 13; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, z), __ddiv_rn(1.0, (double)(2 * k + 1)));
    return __dadd_rn(__dmul_rn((double)e, 0.6931471805599453), __dmul_rn(__dmul_rn(2.0, s), p));
}

__device__ __forceinline__ int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

// Block-uniform read of the sticky status: every thread of the block takes the
// same early exit, so no barrier is ever left waiting for an exited thread.
__device__ __forceinline__ bool block_stopped(const DevState *st) {
    __shared__ uint32_t s_stop;
    if (threadIdx.x == 0) s_stop = *(volatile const uint32_t *)&st->status;
    __syncthreads();
    const bool stop = s_stop != 0u;
    __syncthreads();
    return stop;
}

// A look-back word of this epoch with its flag set.
__device__ __forceinline__ bool lb_ready(uint64_t w, uint32_t epoch) {
    return (w >> 34) == (uint64_t)(epoch & 0x3FFFFFFFu) && ((w >> 32) & 3ull) != 0ull;
}

// Bounded spin on a look-back status word; returns the word or 0 on timeout
// (and records ST_TIMEOUT).
__device__ __forceinline__ uint64_t lb_wait(const uint64_t *p, uint32_t epoch, uint32_t *status) {
    const uint64_t want = (uint64_t)(epoch & 0x3FFFFFFFu);
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        const uint64_t w = *(volatile const uint64_t *)p;
        if ((w >> 34) == want && ((w >> 32) & 3ull) != 0ull) return w;
        if (it > 64) __nanosleep(64);
    }
    atomicOr(status, ST_TIMEOUT);
    return 0;
}

__device__ __forceinline__ void lb_store(uint64_t *p, uint64_t w) {
    *(volatile uint64_t *)p = w;
}

// ---- bulk asynchronous copies (TMA, non-tensor form) and mbarriers --------
// A copy moves a contiguous range between global and shared memory; both
// addresses 16-byte aligned, the size a multiple of 16.  Loads complete on an
// mbarrier (transaction bytes), stores on a bulk group.

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// one arrival that also announces `bytes` of transactions for the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Bounded wait for the phase of the given parity to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void bulk_store(void *dst_gmem, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 ::"l"(dst_gmem), "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory source of every committed bulk store has been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed bulk store has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// order this thread's generic-proxy shared-memory accesses with later async-proxy ones
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Run id of a batch key from its high word (the packed key, or the bra word
// of a two-word key), kept inside [0, nruns).
__device__ __forceinline__ int batch_run(uint64_t w, int shift, int nruns) {
    const uint64_t r = w >> shift;
    return r < (uint64_t)nruns ? (int)r : nruns - 1;
}

}  // namespace ddq
