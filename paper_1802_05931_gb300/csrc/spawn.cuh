// Spawn + death/clone kernel: steps (i) and (ii) of the DDQMC step (Sec. III.C).
//
// Every walker of every occupied configuration |i><j| draws one Philox block
// keyed by (seed, step) with counter (i, j, walker, part << 16 | block):
//   word 0  -> spawn attempt 0        word 1 -> death / cloning
//   word 2  -> on-site Re <-> Im      word 3 -> spawn attempt 1
// and blocks 1, 2, ... give attempts 4b-2 .. 4b+1 when the total spawning
// rate P_tot exceeds 1 (n_att = ceil(P_tot) attempts of rate P_tot / n_att).
// Per-walker categorical draws over the moves have the joint law of the
// binomial + multinomial scheme of Sec. III.B.
//
// Moves, in order: ket bond flips (child (i ^ m_b, j), A = -i h_b(i)), bra
// bond flips (child (i, j ^ m_b), A = +i h_b(j)), jumps (child (i - 2^k,
// j - 2^k), A = gamma, needs spin k up on both sides).  Rates are fixed-point
// integers (rate * 2^32, truncated), so the selection is integer-only.
//
// Children follow Delta rho_child = A rho_parent: a real parent of sign s
// makes a child of type sgn(Re A) / sgn(Im A) as in the four rules of
// Sec. III.C; the death / clone and Re <-> Im transfer act on the parent's own
// entry, which is updated in place.  Spawn records are appended through
// per-warp shared-memory staging (coalesced 16-byte stores) and counted into
// the radix histograms of every digit pass.
#pragma once

#include "common.cuh"

namespace ddq {

constexpr int SP_TPB = 256;
constexpr int SP_WARPS = SP_TPB / 32;
constexpr int SP_STAGE = 128;      // staged records per warp
constexpr int SP_FLUSH = 32;       // flush threshold at warp-uniform points
constexpr int SP_LIGHT = 8;        // entries with at most this many walkers run lane-per-entry

struct SpawnShared {
    uint64_t rate_q[MAXB][2][4];
    uint64_t bond_m[MAXB];
    uint64_t cross_frac[2 * MAXB + 1];
    uint64_t d_frac[2 * MAXN + 1];
    uint32_t cross_int[2 * MAXB + 1];
    uint32_t d_int[2 * MAXN + 1];
    int32_t d_sgn[2 * MAXN + 1];
    int8_t bond_a[MAXB], bond_b[MAXB];
    uint32_t hist[MAXPASS][256];
    int32_t stage_n[SP_WARPS];
    Rec stage[SP_WARPS][SP_STAGE];
    uint64_t cum[SP_WARPS][MAXK];
    int32_t cnt_re[SP_WARPS][MAXK];
    int32_t cnt_im[SP_WARPS][MAXK];
};

struct SpawnCtx {
    const SpawnShared *sh;
    int N, B, K, gk;
    uint64_t jump_q;
};

__device__ __forceinline__ int imp_class(int gk, uint64_t d, uint64_t m, int a, int b) {
    if (gk == 1) return d == 0 ? 1 : (d == m ? 2 : 0);
    if (gk == 2) return (int)((((d >> a) & 1ull) << 1) | ((d >> b) & 1ull));
    return 0;
}

// Rate of move m of configuration (i, j).
__device__ __forceinline__ uint64_t move_rate(const SpawnCtx &c, uint64_t i, uint64_t j, int m) {
    const SpawnShared &s = *c.sh;
    if (m < 2 * c.B) {
        const int b = m < c.B ? m : m - c.B;
        const uint64_t w = m < c.B ? i : j;
        const int a0 = s.bond_a[b], a1 = s.bond_b[b];
        const int anti = (int)(((w >> a0) ^ (w >> a1)) & 1ull);
        return s.rate_q[b][anti][imp_class(c.gk, i ^ j, s.bond_m[b], a0, a1)];
    }
    const int k = m - 2 * c.B;
    return (((i & j) >> k) & 1ull) ? c.jump_q : 0ull;
}

// Child key and signed (re, im) unit of move m for a walker of part `part`
// (0 real, 1 imaginary) and sign `sig`.
__device__ __forceinline__ void move_child(const SpawnCtx &c, const RunParams &P, uint64_t i, uint64_t j,
                                           int m, int part, int sig, uint64_t &ckey, int &dre, int &dim) {
    const SpawnShared &s = *c.sh;
    uint64_t ci = i, cj = j;
    dre = 0;
    dim = 0;
    if (m < 2 * c.B) {
        const bool ket = m < c.B;
        const int b = ket ? m : m - c.B;
        const uint64_t w = ket ? i : j;
        const int anti = (int)(((w >> s.bond_a[b]) ^ (w >> s.bond_b[b])) & 1ull);
        const int hs = P.sgn_h[anti];
        if (ket) ci ^= s.bond_m[b]; else cj ^= s.bond_m[b];
        // A = -i h (ket) or +i h (bra): Re parent -> Im child, Im parent -> Re child
        const int g = ket ? -hs : hs;
        if (part == 0) dim = sig * g; else dre = -sig * g;
    } else {
        const int k = m - 2 * c.B;
        ci &= ~(1ull << k);
        cj &= ~(1ull << k);
        if (part == 0) dre = sig; else dim = sig;
    }
    ckey = (cj << c.N) | ci;
}

__device__ __forceinline__ void count_digits(SpawnShared &s, uint64_t key, int npass) {
    for (int p = 0; p < npass; ++p) atomicAdd(&s.hist[p][(key >> (8 * p)) & 0xFFull], 1u);
}

// Append one record from a (possibly divergent) lane.
__device__ __forceinline__ void emit(SpawnShared &s, int warp, const Rec &r, Rec *out, int64_t cap,
                                     DevState *st, int npass) {
    const int pos = atomicAdd(&s.stage_n[warp], 1);
    if (pos < SP_STAGE) {
        s.stage[warp][pos] = r;
    } else {
        const unsigned long long idx = atomicAdd((unsigned long long *)&st->R, 1ull);
        if ((int64_t)idx < cap) {
            out[idx] = r;
            count_digits(s, r.key & KEY_MASK, npass);
        } else {
            atomicOr(&st->status, ST_CAPACITY);
        }
    }
}

// Warp-uniform flush of the warp's staged records.
__device__ __forceinline__ void flush(SpawnShared &s, int warp, int lane, Rec *out, int64_t cap,
                                      DevState *st, int npass, int min_n) {
    __syncwarp();
    int n = s.stage_n[warp];
    if (n > SP_STAGE) n = SP_STAGE;
    if (n >= min_n && n > 0) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd((unsigned long long *)&st->R, (unsigned long long)n);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (int k = lane; k < n; k += 32) {
            const Rec r = s.stage[warp][k];
            if ((int64_t)(base + k) < cap) {
                out[base + k] = r;
                count_digits(s, r.key & KEY_MASK, npass);
            }
        }
        if (lane == 0 && (int64_t)(base + n) > cap) atomicOr(&st->status, ST_CAPACITY);
        __syncwarp();
        if (lane == 0) s.stage_n[warp] = 0;
    }
    __syncwarp();
}

__device__ __forceinline__ uint32_t attempt_word(uint4 x0, uint4 &xb, uint32_t &blk, uint64_t a,
                                                 uint4 ctr, uint32_t k0, uint32_t k1) {
    if (a == 0) return x0.x;
    if (a == 1) return x0.w;
    const uint32_t want = 1u + (uint32_t)((a - 2) >> 2);
    if (want != blk) {
        blk = want;
        ctr.w = (ctr.w & 0xFFFF0000u) | want;
        xb = philox4x32_10(ctr, k0, k1);
    }
    switch ((a - 2) & 3) {
        case 0: return xb.x;
        case 1: return xb.y;
        case 2: return xb.z;
        default: return xb.w;
    }
}

__global__ void __launch_bounds__(SP_TPB)
k_spawn_death(const RunParams *__restrict__ Pp, DevState *__restrict__ st, Rec *__restrict__ L,
              Rec *__restrict__ out, int64_t cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpawnShared &s = *reinterpret_cast<SpawnShared *>(smem_raw);
    const RunParams &P = *Pp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (block_stopped(st)) return;
    const int N = P.N, B = P.B, K = P.K, npass = P.npass;
    // stage the constant tables
    for (int q = tid; q < B * 8; q += SP_TPB) (&s.rate_q[0][0][0])[q] = (&P.rate_q[0][0][0])[q];
    for (int q = tid; q < B; q += SP_TPB) {
        s.bond_m[q] = P.bond_m[q];
        s.bond_a[q] = (int8_t)P.bond_a[q];
        s.bond_b[q] = (int8_t)P.bond_b[q];
    }
    for (int q = tid; q <= 2 * B; q += SP_TPB) { s.cross_int[q] = P.cross_int[q]; s.cross_frac[q] = P.cross_frac[q]; }
    for (int q = tid; q <= 2 * N; q += SP_TPB) { s.d_int[q] = st->d_int[q]; s.d_frac[q] = st->d_frac[q]; s.d_sgn[q] = st->d_sgn[q]; }
    for (int q = tid; q < MAXPASS * 256; q += SP_TPB) (&s.hist[0][0])[q] = 0u;
    if (tid < SP_WARPS) s.stage_n[tid] = 0;
    __syncthreads();

    SpawnCtx c;
    c.sh = &s; c.N = N; c.B = B; c.K = K; c.gk = P.guide_kind; c.jump_q = P.jump_q;
    const int64_t M = st->M;
    const uint64_t t = (uint64_t)st->t;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32) ^ (uint32_t)t;
    const uint64_t nmask = P.nmask;
    const int n_a = P.n_a;
    uint32_t local_status = 0;

    const int64_t nwarps = (int64_t)gridDim.x * SP_WARPS;
    for (int64_t chunk = (int64_t)blockIdx.x * SP_WARPS + warp; chunk * 32 < M; chunk += nwarps) {
        const int64_t e = chunk * 32 + lane;
        Rec rec;
        rec.key = 0; rec.re = 0; rec.im = 0;
        if (e < M) rec = L[e];
        const uint64_t i = rec.key & nmask, j = rec.key >> N;
        const int64_t nre = iabs64(rec.re), nim = iabs64(rec.im);
        const int64_t nw = nre + nim;
        const bool heavy = (e < M) && nw > SP_LIGHT;
        const bool init = (n_a == 0) || (i == j) || (nw > (int64_t)n_a);
        const uint64_t fl = init ? FLAG_BIT : 0ull;

        // ---- light entries: one lane per configuration ----------------------
        if (e < M && !heavy) {
            uint64_t T = 0;
            int na_i = 0, na_j = 0;
            const uint64_t d = i ^ j;
            for (int b = 0; b < B; ++b) {
                const int a0 = s.bond_a[b], a1 = s.bond_b[b];
                const int ai = (int)(((i >> a0) ^ (i >> a1)) & 1ull);
                const int aj = (int)(((j >> a0) ^ (j >> a1)) & 1ull);
                const int cl = imp_class(c.gk, d, s.bond_m[b], a0, a1);
                T += s.rate_q[b][ai][cl] + s.rate_q[b][aj][cl];
                na_i += ai;
                na_j += aj;
            }
            T += (uint64_t)__popcll(i & j) * c.jump_q;
            uint64_t natt = (T + 0xFFFFFFFFull) >> 32;
            if (natt == 0) natt = 1;
            const int cd = __popcll(i) + __popcll(j);
            const int dz = 2 * (na_j - na_i);          // zsum(i) - zsum(j)
            const int adz = dz < 0 ? -dz : dz;
            const int sgn_d = (dz == 0) ? 0 : -P.sgn_jz * (dz > 0 ? 1 : -1);
            int64_t dre = 0, dim = 0;
            for (int part = 0; part < 2; ++part) {
                const int64_t pop = part == 0 ? rec.re : rec.im;
                const int64_t n = iabs64(pop);
                const int sig = pop < 0 ? -1 : 1;
                for (int64_t w = 0; w < n; ++w) {
                    const uint4 ctr = make_uint4((uint32_t)i, (uint32_t)j, (uint32_t)w, (uint32_t)part << 16);
                    const uint4 x = philox4x32_10(ctr, k0, k1);
                    const int64_t cnt = (int64_t)s.d_int[cd] + ((uint64_t)x.y < s.d_frac[cd] ? 1 : 0);
                    const int64_t cc = (int64_t)s.cross_int[adz] + ((uint64_t)x.z < s.cross_frac[adz] ? 1 : 0);
                    if (part == 0) { dre -= (int64_t)s.d_sgn[cd] * sig * cnt; dim += (int64_t)sig * sgn_d * cc; }
                    else { dim -= (int64_t)s.d_sgn[cd] * sig * cnt; dre -= (int64_t)sig * sgn_d * cc; }
                    uint4 xb = x;
                    uint32_t blk = 0;
                    for (uint64_t a = 0; a < natt; ++a) {
                        const uint32_t u = attempt_word(x, xb, blk, a, ctr, k0, k1);
                        const uint64_t v = (uint64_t)u * natt;
                        if (v >= T) continue;
                        uint64_t cum = 0;
                        int m = 0;
                        for (; m < K - 1; ++m) {
                            cum += move_rate(c, i, j, m);
                            if (v < cum) break;
                        }
                        Rec r;
                        int cre, cim;
                        move_child(c, P, i, j, m, part, sig, r.key, cre, cim);
                        r.key |= fl;
                        r.re = cre;
                        r.im = cim;
                        emit(s, warp, r, out, cap, st, npass);
                    }
                }
            }
            const int64_t re2 = (int64_t)rec.re + dre, im2 = (int64_t)rec.im + dim;
            if (iabs64(re2) > 2147483647ll || iabs64(im2) > 2147483647ll) local_status |= ST_OVERFLOW;
            *reinterpret_cast<int2 *>(&L[e].re) = make_int2((int32_t)re2, (int32_t)im2);
        }
        flush(s, warp, lane, out, cap, st, npass, SP_FLUSH);

        // ---- heavy entries: the whole warp on one configuration -------------
        unsigned hmask = __ballot_sync(0xFFFFFFFFu, heavy);
        while (hmask) {
            const int h = __ffs(hmask) - 1;
            hmask &= hmask - 1;
            const uint64_t hi = __shfl_sync(0xFFFFFFFFu, i, h);
            const uint64_t hj = __shfl_sync(0xFFFFFFFFu, j, h);
            const int32_t hre = __shfl_sync(0xFFFFFFFFu, rec.re, h);
            const int32_t him = __shfl_sync(0xFFFFFFFFu, rec.im, h);
            const bool hinit = __shfl_sync(0xFFFFFFFFu, init, h);
            const uint64_t hfl = hinit ? FLAG_BIT : 0ull;
            // cumulative thresholds over the K moves (warp scan)
            uint64_t carry = 0;
            for (int base = 0; base < K; base += 32) {
                const int m = base + lane;
                uint64_t r = m < K ? move_rate(c, hi, hj, m) : 0ull;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, r, off);
                    if (lane >= off) r += y;
                }
                if (m < K) s.cum[warp][m] = carry + r;
                carry += __shfl_sync(0xFFFFFFFFu, r, 31);
            }
            for (int m = lane; m < K; m += 32) { s.cnt_re[warp][m] = 0; s.cnt_im[warp][m] = 0; }
            __syncwarp();
            const uint64_t T = carry;
            uint64_t natt = (T + 0xFFFFFFFFull) >> 32;
            if (natt == 0) natt = 1;
            int na_i = 0, na_j = 0;
            for (int b = 0; b < B; ++b) {
                na_i += (int)(((hi >> s.bond_a[b]) ^ (hi >> s.bond_b[b])) & 1ull);
                na_j += (int)(((hj >> s.bond_a[b]) ^ (hj >> s.bond_b[b])) & 1ull);
            }
            const int cd = __popcll(hi) + __popcll(hj);
            const int dz = 2 * (na_j - na_i);
            const int adz = dz < 0 ? -dz : dz;
            const int sgn_d = (dz == 0) ? 0 : -P.sgn_jz * (dz > 0 ? 1 : -1);
            int64_t dre = 0, dim = 0;
            for (int part = 0; part < 2; ++part) {
                const int64_t pop = part == 0 ? hre : him;
                const int64_t n = iabs64(pop);
                const int sig = pop < 0 ? -1 : 1;
                for (int64_t w = lane; w < n; w += 32) {
                    const uint4 ctr = make_uint4((uint32_t)hi, (uint32_t)hj, (uint32_t)w, (uint32_t)part << 16);
                    const uint4 x = philox4x32_10(ctr, k0, k1);
                    const int64_t cnt = (int64_t)s.d_int[cd] + ((uint64_t)x.y < s.d_frac[cd] ? 1 : 0);
                    const int64_t cc = (int64_t)s.cross_int[adz] + ((uint64_t)x.z < s.cross_frac[adz] ? 1 : 0);
                    if (part == 0) { dre -= (int64_t)s.d_sgn[cd] * sig * cnt; dim += (int64_t)sig * sgn_d * cc; }
                    else { dim -= (int64_t)s.d_sgn[cd] * sig * cnt; dre -= (int64_t)sig * sgn_d * cc; }
                    uint4 xb = x;
                    uint32_t blk = 0;
                    for (uint64_t a = 0; a < natt; ++a) {
                        const uint32_t u = attempt_word(x, xb, blk, a, ctr, k0, k1);
                        const uint64_t v = (uint64_t)u * natt;
                        if (v >= T) continue;
                        int lo = 0, hi2 = K - 1;
                        while (lo < hi2) {
                            const int mid = (lo + hi2) >> 1;
                            if (v < s.cum[warp][mid]) hi2 = mid; else lo = mid + 1;
                        }
                        uint64_t ck;
                        int cre, cim;
                        move_child(c, P, hi, hj, lo, part, sig, ck, cre, cim);
                        if (cre) atomicAdd(&s.cnt_re[warp][lo], cre);
                        if (cim) atomicAdd(&s.cnt_im[warp][lo], cim);
                    }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                dre += __shfl_xor_sync(0xFFFFFFFFu, dre, off);
                dim += __shfl_xor_sync(0xFFFFFFFFu, dim, off);
            }
            const int64_t he = __shfl_sync(0xFFFFFFFFu, e, h);
            if (lane == 0) {
                const int64_t re2 = (int64_t)hre + dre, im2 = (int64_t)him + dim;
                if (iabs64(re2) > 2147483647ll || iabs64(im2) > 2147483647ll) local_status |= ST_OVERFLOW;
                *reinterpret_cast<int2 *>(&L[he].re) = make_int2((int32_t)re2, (int32_t)im2);
            }
            __syncwarp();
            for (int m = lane; m < K; m += 32) {
                const int32_t cre = s.cnt_re[warp][m], cim = s.cnt_im[warp][m];
                if (cre == 0 && cim == 0) continue;
                Rec r;
                int ure, uim;
                move_child(c, P, hi, hj, m, 0, 1, r.key, ure, uim);
                r.key |= hfl;
                r.re = cre;
                r.im = cim;
                emit(s, warp, r, out, cap, st, npass);
            }
            flush(s, warp, lane, out, cap, st, npass, SP_FLUSH);
        }
    }
    flush(s, warp, lane, out, cap, st, npass, 1);
    if (local_status) atomicOr(&st->status, local_status);
    __syncthreads();
    for (int q = tid; q < npass * 256; q += SP_TPB) {
        const uint32_t v = (&s.hist[0][0])[q];
        if (v) atomicAdd(&st->hist[q >> 8][q & 255], v);
    }
}

}  // namespace ddq
