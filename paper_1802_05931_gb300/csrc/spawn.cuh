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
// integers (rate * 2^32, truncated), so the move selection is integer-only.
//
// Children follow Delta rho_child = A rho_parent (the four sign rules of
// Sec. III.C); death / clone and the Re <-> Im transfer act on the parent's
// own entry, which is updated in place.
//
// Two paths share the work of a chunk of 32 configurations per warp:
//  * light configurations (few walkers): the walkers of the whole chunk are
//    spread over the 32 lanes, so every lane does the same per-walker work.
//    Rate totals and the move search use bond masks: with bit 2k the bond
//    from site k to its right neighbour and bit 2k+1 the bond to the one
//    below, bit order is move order, each bond's rate is a function of
//    (anti-aligned, importance class), and the cumulative rate up to a bit
//    position is a sum of popcounts times the six rates.  The selected move
//    is found by binary search over the 64 bit positions.
//  * heavy configurations (many walkers, or rate tables that differ per
//    bond): the whole warp on one configuration, with the cumulative rate
//    table in shared memory and the children aggregated per move.
// Spawn records are appended through per-warp shared-memory staging
// (coalesced 16-byte stores) and counted into the radix histograms of every
// digit pass.
#pragma once

#include "common.cuh"

namespace ddq {

constexpr int SP_TPB = 256;
constexpr int SP_WARPS = SP_TPB / 32;
constexpr int SP_STAGE = 128;      // staged records per warp
constexpr int SP_FLUSH = 32;       // flush threshold at warp-uniform points
constexpr int SP_HEAVY = 48;       // configurations with more walkers use the warp-cooperative path

// Parameters of one light configuration, staged for the lanes that run its walkers.
struct LightEntry {
    uint64_t Ai, Aj, C1, C2;   // anti-aligned (ket, bra) and importance-class bond masks
    uint64_t T_ket, T_bra, T;  // rate totals: ket moves, bra moves, all moves
    uint32_t i, j, natt;
    int32_t re, im, nre;
    int32_t cd, adz, sgn_d, init;
};

struct SpawnShared {
    uint64_t rate_q[MAXB][2][4];
    uint64_t bond_m[MAXB];
    uint64_t cross_frac[2 * MAXB + 1];
    uint64_t d_frac[2 * MAXN + 1];
    uint64_t urate[2][3];
    uint32_t cross_int[2 * MAXB + 1];
    uint32_t d_int[2 * MAXN + 1];
    int32_t d_sgn[2 * MAXN + 1];
    int8_t bond_a[MAXB], bond_b[MAXB];
    int8_t rn[MAXN + 1], dn[MAXN + 1];
    uint32_t hist[MAXPASS][256];
    int32_t stage_n[SP_WARPS];
    Rec stage[SP_WARPS][SP_STAGE];
    LightEntry le[SP_WARPS][32];
    int32_t incl[SP_WARPS][32];
    int32_t dre[SP_WARPS][32], dim[SP_WARPS][32];
    uint64_t cum[SP_WARPS][MAXK];
    int32_t cnt_re[SP_WARPS][MAXK];
    int32_t cnt_im[SP_WARPS][MAXK];
};

struct SpawnCtx {
    const SpawnShared *sh;
    int N, B, K, gk;
    uint64_t jump_q;
    uint32_t ER, ED, LC, LR;
    int Lx, shD;
    uint64_t Emorton;
};

__device__ __forceinline__ int imp_class(int gk, uint64_t d, uint64_t m, int a, int b) {
    if (gk == 1) return d == 0 ? 1 : (d == m ? 2 : 0);
    if (gk == 2) return (int)((((d >> a) & 1ull) << 1) | ((d >> b) & 1ull));
    return 0;
}

// ---- mask formulation -------------------------------------------------------

__device__ __forceinline__ uint64_t spread_bits(uint32_t x32) {
    uint64_t x = x32;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

// bond mask from per-direction site masks: bit 2k <- right bond of k, bit 2k+1 <- lower bond of k
__device__ __forceinline__ uint64_t bond_mask(uint32_t right, uint32_t down) {
    return spread_bits(right) | (spread_bits(down) << 1);
}

// word whose bit k is the spin of the right (resp. lower) neighbour of site k
__device__ __forceinline__ uint32_t nb_right(const SpawnCtx &c, uint32_t s) {
    return ((s >> 1) & ~c.LC) | ((s << (c.Lx - 1)) & c.LC);
}
__device__ __forceinline__ uint32_t nb_down(const SpawnCtx &c, uint32_t s) {
    return (s >> c.Lx) | ((s << c.shD) & c.LR);
}

__device__ __forceinline__ uint64_t anti_mask(const SpawnCtx &c, uint32_t s) {
    return bond_mask((s ^ nb_right(c, s)) & c.ER, (s ^ nb_down(c, s)) & c.ED);
}

// cumulative rate of the bonds selected by `low` (a prefix of bit positions)
__device__ __forceinline__ uint64_t seg_cum(uint64_t A, uint64_t E, uint64_t C1, uint64_t C2,
                                            const uint64_t (&R)[2][3], uint64_t low) {
    const uint64_t e = E & low, a = A & low, c1 = C1 & low, c2 = C2 & low;
    const uint64_t n = e & ~a, c0 = ~(c1 | c2);
    return R[1][0] * (uint64_t)__popcll(a & c0) + R[1][1] * (uint64_t)__popcll(a & c1) +
           R[1][2] * (uint64_t)__popcll(a & c2) + R[0][0] * (uint64_t)__popcll(n & c0) +
           R[0][1] * (uint64_t)__popcll(n & c1) + R[0][2] * (uint64_t)__popcll(n & c2);
}

// largest bit position p with seg_cum(prefix p) <= v (the selected bond), given v < segment total
__device__ __forceinline__ int seg_search(uint64_t A, uint64_t E, uint64_t C1, uint64_t C2,
                                          const uint64_t (&R)[2][3], uint64_t v) {
    int lo = 0, hi = 64;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (seg_cum(A, E, C1, C2, R, (1ull << mid) - 1ull) <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

// importance classes of every bond of configuration (i, j): C1, C2 bond masks
__device__ __forceinline__ void class_masks(const SpawnCtx &c, uint32_t i, uint32_t j, uint64_t &C1,
                                            uint64_t &C2) {
    const uint32_t d = i ^ j;
    C1 = 0;
    C2 = 0;
    if (c.gk == 1) {
        if (d == 0) { C1 = c.Emorton; return; }
        if (__popc(d) != 2) return;
        const int a = __ffs(d) - 1, b = 31 - __clz(d);
        const SpawnShared &s = *c.sh;
        // the bond whose two sites are exactly a and b (child diagonal)
        if ((c.ER >> a & 1u) && s.rn[a] == b) C2 = 1ull << (2 * a);
        else if ((c.ED >> a & 1u) && s.dn[a] == b) C2 = 1ull << (2 * a + 1);
        else if ((c.ER >> b & 1u) && s.rn[b] == a) C2 = 1ull << (2 * b);
        else if ((c.ED >> b & 1u) && s.dn[b] == a) C2 = 1ull << (2 * b + 1);
    } else if (c.gk == 2) {
        // class = number of the bond's two sites on which i and j differ
        const uint32_t ar = d & c.ER, br = nb_right(c, d) & c.ER;
        const uint32_t ad = d & c.ED, bd = nb_down(c, d) & c.ED;
        C1 = bond_mask(ar ^ br, ad ^ bd);
        C2 = bond_mask(ar & br, ad & bd);
    }
}

// ---- per-move tables (heavy path) -------------------------------------------

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

// Child key of move m of configuration (i, j) and the sign factor g of the
// move: a real parent of sign s makes an imaginary child of sign s*g and an
// imaginary parent a real child of sign -s*g (bond flips); jumps keep the type.
__device__ __forceinline__ void move_key(const SpawnCtx &c, const RunParams &P, uint64_t i, uint64_t j, int m,
                                         uint64_t &ckey, int &g, bool &jump) {
    const SpawnShared &s = *c.sh;
    uint64_t ci = i, cj = j;
    jump = m >= 2 * c.B;
    g = 1;
    if (!jump) {
        const bool ket = m < c.B;
        const int b = ket ? m : m - c.B;
        const uint64_t w = ket ? i : j;
        const int anti = (int)(((w >> s.bond_a[b]) ^ (w >> s.bond_b[b])) & 1ull);
        const int hs = P.sgn_h[anti];
        if (ket) ci ^= s.bond_m[b]; else cj ^= s.bond_m[b];
        g = ket ? -hs : hs;          // A = -i h (ket) or +i h (bra)
    } else {
        const int k = m - 2 * c.B;
        ci &= ~(1ull << k);
        cj &= ~(1ull << k);
    }
    ckey = (cj << c.N) | ci;
}

// ---- record output ----------------------------------------------------------

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
            atomicOr(&st->status, ST_CAPACITY | ST_CAP_SPAWN);
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
        if (lane == 0 && (int64_t)(base + n) > cap) atomicOr(&st->status, ST_CAPACITY | ST_CAP_SPAWN);
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
    for (int q = tid; q < N; q += SP_TPB) { s.rn[q] = P.rn[q]; s.dn[q] = P.dn[q]; }
    if (tid < 6) (&s.urate[0][0])[tid] = (&P.urate[0][0])[tid];
    for (int q = tid; q <= 2 * B; q += SP_TPB) { s.cross_int[q] = P.cross_int[q]; s.cross_frac[q] = P.cross_frac[q]; }
    for (int q = tid; q <= 2 * N; q += SP_TPB) { s.d_int[q] = st->d_int[q]; s.d_frac[q] = st->d_frac[q]; s.d_sgn[q] = st->d_sgn[q]; }
    for (int q = tid; q < MAXPASS * 256; q += SP_TPB) (&s.hist[0][0])[q] = 0u;
    if (tid < SP_WARPS) s.stage_n[tid] = 0;
    __syncthreads();

    SpawnCtx c;
    c.sh = &s; c.N = N; c.B = B; c.K = K; c.gk = P.guide_kind; c.jump_q = P.jump_q;
    c.ER = P.ER; c.ED = P.ED; c.LC = P.LC; c.LR = P.LR; c.Lx = P.Lx; c.shD = P.shD; c.Emorton = P.Emorton;
    const uint64_t(&R)[2][3] = s.urate;
    const bool uniform = P.uniform != 0;
    const int64_t M = st->M;
    const uint64_t t = (uint64_t)st->t;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32) ^ (uint32_t)t;
    const uint64_t nmask = P.nmask;
    const int n_a = P.n_a;
    const int sgn_jz = P.sgn_jz;
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
        const bool valid = e < M;
        const bool heavy = valid && (nw > SP_HEAVY || !uniform);
        const bool light = valid && !heavy;
        const bool init = (n_a == 0) || (i == j) || (nw > (int64_t)n_a);

        // ---- light configurations: per-configuration setup, one lane each ----
        int nl = 0;
        if (light) {
            LightEntry q;
            const uint32_t i32 = (uint32_t)i, j32 = (uint32_t)j;
            q.Ai = anti_mask(c, i32);
            q.Aj = anti_mask(c, j32);
            class_masks(c, i32, j32, q.C1, q.C2);
            q.T_ket = seg_cum(q.Ai, c.Emorton, q.C1, q.C2, R, ~0ull);
            q.T_bra = seg_cum(q.Aj, c.Emorton, q.C1, q.C2, R, ~0ull);
            q.T = q.T_ket + q.T_bra + (uint64_t)__popc(i32 & j32) * c.jump_q;
            uint64_t natt = (q.T + 0xFFFFFFFFull) >> 32;
            q.natt = natt == 0 ? 1u : (uint32_t)natt;
            q.i = i32;
            q.j = j32;
            q.re = rec.re;
            q.im = rec.im;
            q.nre = (int32_t)nre;
            q.cd = __popc(i32) + __popc(j32);
            const int dz = 2 * (__popcll(q.Aj) - __popcll(q.Ai));     // zsum(i) - zsum(j)
            q.adz = dz < 0 ? -dz : dz;
            q.sgn_d = (dz == 0) ? 0 : -sgn_jz * (dz > 0 ? 1 : -1);
            q.init = init ? 1 : 0;
            s.le[warp][lane] = q;
            nl = (int)nw;
        }
        s.dre[warp][lane] = 0;
        s.dim[warp][lane] = 0;
        int incl = nl;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off) incl += y;
        }
        s.incl[warp][lane] = incl;
        const int Wl = __shfl_sync(0xFFFFFFFFu, incl, 31);
        __syncwarp();

        // ---- light walkers, spread over the lanes ----------------------------
        for (int base = 0; base < Wl; base += 32) {
            const int g = base + lane;
            if (g < Wl) {
                int lo = 0, hi = 31;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s.incl[warp][mid] > g) hi = mid; else lo = mid + 1;
                }
                const int owner = lo;
                const LightEntry &q = s.le[warp][owner];
                const int local = g - (owner ? s.incl[warp][owner - 1] : 0);
                const int part = local < q.nre ? 0 : 1;
                const uint32_t w = (uint32_t)(part ? local - q.nre : local);
                const int sig = (part ? q.im : q.re) < 0 ? -1 : 1;
                const uint4 ctr = make_uint4(q.i, q.j, w, (uint32_t)part << 16);
                const uint4 x = philox4x32_10(ctr, k0, k1);
                const int cnt = (int)s.d_int[q.cd] + ((uint64_t)x.y < s.d_frac[q.cd] ? 1 : 0);
                const int cc = (int)s.cross_int[q.adz] + ((uint64_t)x.z < s.cross_frac[q.adz] ? 1 : 0);
                const int ddeath = -s.d_sgn[q.cd] * sig * cnt;
                const int dcross = sig * q.sgn_d * cc;
                if (part == 0) {
                    if (ddeath) atomicAdd(&s.dre[warp][owner], ddeath);
                    if (dcross) atomicAdd(&s.dim[warp][owner], dcross);
                } else {
                    if (ddeath) atomicAdd(&s.dim[warp][owner], ddeath);
                    if (dcross) atomicAdd(&s.dre[warp][owner], -dcross);
                }
                uint4 xb = x;
                uint32_t blk = 0;
                const uint64_t natt = q.natt;
                for (uint64_t a = 0; a < natt; ++a) {
                    const uint32_t u = attempt_word(x, xb, blk, a, ctr, k0, k1);
                    const uint64_t v = (uint64_t)u * natt;
                    if (v >= q.T) continue;
                    uint32_t ci = q.i, cj = q.j;
                    int cre = 0, cim = 0;
                    if (v < q.T_ket + q.T_bra) {
                        const bool ket = v < q.T_ket;
                        const uint64_t A = ket ? q.Ai : q.Aj;
                        const int p = seg_search(A, c.Emorton, q.C1, q.C2, R, ket ? v : v - q.T_ket);
                        const int k = p >> 1;
                        const int other = (p & 1) ? s.dn[k] : s.rn[k];
                        const uint32_t m = (1u << k) | (1u << other);
                        const int hs = P.sgn_h[(A >> p) & 1ull];
                        const int gsg = ket ? -hs : hs;
                        if (ket) ci ^= m; else cj ^= m;
                        if (part == 0) cim = sig * gsg; else cre = -sig * gsg;
                    } else {
                        uint64_t idx = (v - q.T_ket - q.T_bra) / c.jump_q;
                        uint32_t jm = q.i & q.j;
                        for (; idx > 0; --idx) jm &= jm - 1u;
                        const int k = __ffs(jm) - 1;
                        ci &= ~(1u << k);
                        cj &= ~(1u << k);
                        if (part == 0) cre = sig; else cim = sig;
                    }
                    Rec r;
                    r.key = ((uint64_t)cj << N) | (uint64_t)ci | (q.init ? FLAG_BIT : 0ull);
                    r.re = cre;
                    r.im = cim;
                    emit(s, warp, r, out, cap, st, npass);
                }
            }
        }
        __syncwarp();
        if (light) {
            const int64_t re2 = (int64_t)rec.re + s.dre[warp][lane], im2 = (int64_t)rec.im + s.dim[warp][lane];
            if (iabs64(re2) > 2147483647ll || iabs64(im2) > 2147483647ll) local_status |= ST_OVERFLOW;
            *reinterpret_cast<int2 *>(&L[e].re) = make_int2((int32_t)re2, (int32_t)im2);
        }
        flush(s, warp, lane, out, cap, st, npass, SP_FLUSH);

        // ---- heavy configurations: the whole warp on one configuration -------
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
            const int sgn_d = (dz == 0) ? 0 : -sgn_jz * (dz > 0 ? 1 : -1);
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
                        int gsg;
                        bool jump;
                        move_key(c, P, hi, hj, lo, ck, gsg, jump);
                        if (jump) {
                            if (part == 0) atomicAdd(&s.cnt_re[warp][lo], sig);
                            else atomicAdd(&s.cnt_im[warp][lo], sig);
                        } else {
                            if (part == 0) atomicAdd(&s.cnt_im[warp][lo], sig * gsg);
                            else atomicAdd(&s.cnt_re[warp][lo], -sig * gsg);
                        }
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
                int gsg;
                bool jump;
                move_key(c, P, hi, hj, m, r.key, gsg, jump);
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
