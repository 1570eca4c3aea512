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
// bond flips (child (i, j ^ m_b), A = +i h_b(j)), with the in-plane field of
// Sec. V.B ket and bra single-site flips (A = -i h / +i h along x, h (2 s_k - 1)
// along y), then jumps (child (i - 2^k, j - 2^k), A = gamma, needs spin k up
// on both sides).  Inside a bond-flip segment the moves are grouped by
// g = 4*anti + class (anti-aligned bond in the flipped word; importance class
// of the bond), groups in increasing g and bonds in bond order inside a
// group; site flips are grouped by the importance class of the site, sites in
// order.  Rates are fixed-point integers (rate * 2^32, truncated), so the
// move selection is integer-only.  Spin words are 32-bit up to 31 sites and
// 64-bit up to 64 (then bond masks are 128-bit pairs).
//
// Children follow Delta rho_child = A rho_parent (the four sign rules of
// Sec. III.C); death / clone and the Re <-> Im transfer act on the parent's
// own entry, which is updated in place.
//
// Two paths share the work of a chunk of 32 configurations per warp:
//  * light configurations (few walkers, every bond with the same rate
//    table): the walkers of the whole chunk are spread over the 32 lanes, so
//    every lane does the same per-walker work.  Bonds are bits of a mask
//    (bit 2k the bond from site k to its right neighbour, 2k+1 the one
//    below, which is bond order); a group is a mask, its rate total a popcount
//    times the group's rate, and a draw is resolved in O(1): the group from
//    eight running totals, the bond as the r-th set bit of the group's mask.
//  * heavy configurations (many walkers, or rate tables that differ per
//    bond): the whole warp on one configuration, with the cumulative rate
//    table of the group-ordered moves in shared memory and the children
//    aggregated per move.
// Spawn records are appended through per-warp shared-memory staging
// (coalesced stores) and counted into the radix histograms of every digit
// pass.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "radix.cuh"

namespace ddq {

constexpr int SP_TPB = 256;
constexpr int SP_WARPS = SP_TPB / 32;
constexpr int SP_STAGE = 128;      // staged records per warp (default)
constexpr int SP_FLUSH = 32;       // flush threshold at warp-uniform points
constexpr int SP_HEAVY = 1024;     // default: configurations with more walkers use the warp-cooperative path

// 128-bit bond mask (two-word keys: bonds 2k, 2k+1 of sites k < 32 in lo,
// of sites k >= 32 in hi).
struct U128 {
    uint64_t lo, hi;
};
__device__ __forceinline__ U128 operator&(const U128 &a, const U128 &b) { return U128{a.lo & b.lo, a.hi & b.hi}; }
__device__ __forceinline__ U128 operator|(const U128 &a, const U128 &b) { return U128{a.lo | b.lo, a.hi | b.hi}; }
__device__ __forceinline__ U128 operator~(const U128 &a) { return U128{~a.lo, ~a.hi}; }

// Site-word type SW and bond-mask type MT of the light path for each record
// type: 2N <= 32 (packed records), N <= 31, N <= 64.
template <typename T> struct LightTypes { using SW = uint32_t; using MT = uint64_t; };
template <> struct LightTypes<uint64_t> { using SW = uint32_t; using MT = uint32_t; };
template <> struct LightTypes<P40> { using SW = uint32_t; using MT = uint64_t; };
template <> struct LightTypes<RecW> { using SW = uint64_t; using MT = U128; };

// Parameters of the light configurations of one warp's chunk, one array per
// field (lanes that read different configurations hit different banks).
template <typename MT, typename SW>
struct LightSoA {
    MT Ai[32], Aj[32], X1[32], X2[32];         // anti-aligned bond masks (ket, bra), importance-class masks
    uint64_t Tket[32], Tbra[32], T[32];        // rate totals: ket moves, bra moves, all moves
    uint64_t gk[32], gb[32];                   // bonds per group (8 bytes), ket and bra
    SW i[32], j[32];
    uint64_t Tf[32];                           // field flips: rate total of one segment (ket or bra)
    uint32_t fc[32];                           // field flips: sites per importance class (8 bits each)
    uint32_t natt[32];
    int32_t re[32], im[32], nre[32];
    int32_t cd[32], adz[32], sgn_d[32], init[32];
};

// Tables of one warp-cooperative configuration: running rate sums of the
// moves in move order, the move index of each slot (ket b, bra B + b, jump
// 2B + k) and the children counted per slot.
template <int KM>
struct HeavyTables {
    uint64_t cum[KM];
    int32_t cnt_re[KM];
    int32_t cnt_im[KM];
    int16_t mv[KM];
};

// moves per configuration for one-word keys: 2 * 62 bonds + 3 * 31 sites
constexpr int MAXK_PACK = 2 * 2 * NPACK + 3 * NPACK + 1;

// Moves a warp's table holds: without the field's site flips a
// configuration has at most 2B + N moves (two-word keys: 320 against 448),
// which is what lets the two-word kernel keep two blocks per SM.
template <typename T, bool FIELD> struct HeavyCap {
    static constexpr int value = std::is_same<T, RecW>::value ? (FIELD ? MAXK : 2 * MAXB + MAXN)
                                                              : (FIELD ? MAXK_PACK : 2 * 2 * NPACK + NPACK);
};

// A warp's light-configuration parameters are dead before its heavy
// configurations start, so the two share storage.
template <typename T, bool FIELD>
union WarpScratch {
    LightSoA<typename LightTypes<T>::MT, typename LightTypes<T>::SW> le;
    HeavyTables<HeavyCap<T, FIELD>::value> hv;
};

// Constant tables of one step, staged in shared memory.
struct SpawnTables {
    uint64_t bond_m[MAXB];
    uint32_t cross_frac32[2 * MAXB + 1];  // fractional parts of the cross and death counts, x 2^32
    uint32_t d_frac32[2 * MAXN + 1];
    uint64_t urate8[8];
    uint32_t urate32[8];
    float uinv[8];
    float jinv;                       // 1 / jump rate (0 without jumps)
    int32_t sgn_h[2];
    uint32_t cross_int[2 * MAXB + 1];
    uint32_t d_int[2 * MAXN + 1];
    int32_t d_sgn[2 * MAXN + 1];
    int8_t bond_a[MAXB], bond_b[MAXB];
    int8_t rn[MAXN + 1], dn[MAXN + 1];
    int32_t pass_shift[MAXPASS];
    uint64_t ufrate[4];               // field flip rate of each importance class (uniform tables)
    uint32_t ufrate32[4];
    float ufinv[4];
    uint64_t ufrate2[4];              // the same for the y part of a flip at an angle (axis 2)
    uint32_t ufrate32_2[4];
    float ufinv2[4];
    int32_t field_on, field_axis, sgn_hf, sgn_hf2;
    int32_t fparts;                   // moves per site flip and segment: 2 when a run has axis 2
};

// Resident blocks per SM the spawn kernel is compiled for: four for a single
// run with packed records and for 40-bit-key records (64 registers a thread:
// a few spills, measured faster than three blocks at 80); two for two-word
// keys, whose shared memory allows no more (so up to 128 registers a thread);
// else three.
template <typename T, bool BATCH> struct SpawnBlocks {
    static constexpr int value = std::is_same<T, RecW>::value ? 2
                                 : (((std::is_same<T, uint64_t>::value && !BATCH) || std::is_same<T, P40>::value)
                                        ? 4 : 3);
};

// Shared memory of the spawn kernel for spawn records of type T, with or
// without the field's moves; packed records (keys of at most 32 bits) need at
// most four digit passes.
template <typename T, bool FIELD>
struct SpawnShared : SpawnTables {
    static constexpr int NP = std::is_same<T, uint64_t>::value ? 4
                              : (std::is_same<T, P40>::value ? 5 : (std::is_same<T, RecW>::value ? MAXPASS : 8));
    uint32_t hist[NP][256];
    int32_t stage_n[SP_WARPS];
    // staged records per warp (40-bit-key records: 64, for four blocks per SM)
    static constexpr int STAGE = std::is_same<T, P40>::value ? 64 : SP_STAGE;
    T stage[SP_WARPS][STAGE];
    WarpScratch<T, FIELD> ws[SP_WARPS];
    int32_t mark[SP_WARPS][32];       // first walker position of each configuration of the chunk
    int32_t dre[SP_WARPS][32], dim[SP_WARPS][32];
    uint64_t qv[SP_WARPS][64];        // queued spawn draws: scaled uniform v
    uint32_t qm[SP_WARPS][64];        //   and configuration | part << 5 | negative << 6
};

struct SpawnCtx {
    const SpawnTables *sh;
    int N, B, K, gk;
    uint64_t jump_q;
    uint64_t nmask;
    uint64_t ER, ED, LC, LR;
    int Lx, shD;
    uint64_t Emorton, Emorton_hi;
    uint64_t hmask;                 // hashed order of two-word keys: mask of the ket hash in the stored bra word
};

__device__ __forceinline__ int imp_class(int gk, uint64_t d, uint64_t m, int a, int b) {
    if (gk == 1) return d == 0 ? 1 : (d == m ? 2 : 0);
    if (gk == 2) return (int)((((d >> a) & 1ull) << 1) | ((d >> b) & 1ull));
    return 0;
}

// ---- mask formulation -------------------------------------------------------
// Bond masks are 32-bit words when N <= 16 (2N bond bits), 64-bit words when
// N <= 31 and 128-bit pairs up to N = 64; MT is the mask type, SW the type of
// a spin word (32 bits up to 31 sites, else 64).

__device__ __forceinline__ uint64_t spread32(uint32_t x32) {
    uint64_t x = x32;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

template <typename MT, typename SW> __device__ __forceinline__ MT spread_bits(SW x);
template <> __device__ __forceinline__ uint32_t spread_bits<uint32_t, uint32_t>(uint32_t x) {
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}
template <> __device__ __forceinline__ uint64_t spread_bits<uint64_t, uint32_t>(uint32_t x) { return spread32(x); }
template <> __device__ __forceinline__ U128 spread_bits<U128, uint64_t>(uint64_t x) {
    return U128{spread32((uint32_t)x), spread32((uint32_t)(x >> 32))};
}

__device__ __forceinline__ int popcount(uint32_t x) { return __popc(x); }
__device__ __forceinline__ int popcount(uint64_t x) { return __popcll(x); }
__device__ __forceinline__ int popcount(const U128 &x) { return __popcll(x.lo) + __popcll(x.hi); }

__device__ __forceinline__ uint32_t shl1(uint32_t x) { return x << 1; }
__device__ __forceinline__ uint64_t shl1(uint64_t x) { return x << 1; }
__device__ __forceinline__ U128 shl1(const U128 &x) { return U128{x.lo << 1, x.hi << 1}; }   // even bits to odd

__device__ __forceinline__ uint32_t mask_bit(uint32_t x, int p) { return (x >> p) & 1u; }
__device__ __forceinline__ uint32_t mask_bit(uint64_t x, int p) { return (uint32_t)(x >> p) & 1u; }
__device__ __forceinline__ uint32_t mask_bit(const U128 &x, int p) {
    return (uint32_t)((p < 64 ? (x.lo >> p) : (x.hi >> (p - 64))) & 1ull);
}

template <typename MT> __device__ __forceinline__ MT zero_mask() { return (MT)0; }
template <> __device__ __forceinline__ U128 zero_mask<U128>() { return U128{0ull, 0ull}; }
template <typename MT> __device__ __forceinline__ MT one_bit(int p) { return (MT)1 << p; }
template <> __device__ __forceinline__ U128 one_bit<U128>(int p) {
    return p < 64 ? U128{1ull << p, 0ull} : U128{0ull, 1ull << (p - 64)};
}
template <typename MT> __device__ __forceinline__ MT bond_exists(const SpawnCtx &c) { return (MT)c.Emorton; }
template <> __device__ __forceinline__ U128 bond_exists<U128>(const SpawnCtx &c) { return U128{c.Emorton, c.Emorton_hi}; }

__device__ __forceinline__ int low_bit(uint32_t x) { return __ffs(x) - 1; }
__device__ __forceinline__ int low_bit(uint64_t x) { return __ffsll((long long)x) - 1; }
__device__ __forceinline__ int high_bit(uint32_t x) { return 31 - __clz(x); }
__device__ __forceinline__ int high_bit(uint64_t x) { return 63 - __clzll((long long)x); }

// bond mask from per-direction site masks: bit 2k <- right bond of k, bit 2k+1 <- lower bond of k
template <typename MT, typename SW>
__device__ __forceinline__ MT bond_mask(SW right, SW down) {
    return spread_bits<MT, SW>(right) | shl1(spread_bits<MT, SW>(down));
}

// word whose bit k is the spin of the right (resp. lower) neighbour of site k
template <typename SW>
__device__ __forceinline__ SW nb_right(const SpawnCtx &c, SW s) {
    return ((s >> 1) & ~(SW)c.LC) | ((s << (c.Lx - 1)) & (SW)c.LC);
}
template <typename SW>
__device__ __forceinline__ SW nb_down(const SpawnCtx &c, SW s) {
    return (s >> c.Lx) | ((s << c.shD) & (SW)c.LR);
}

template <typename MT, typename SW>
__device__ __forceinline__ MT anti_mask(const SpawnCtx &c, SW s) {
    return bond_mask<MT, SW>((s ^ nb_right(c, s)) & (SW)c.ER, (s ^ nb_down(c, s)) & (SW)c.ED);
}

// importance-class masks of configuration (i, j): for the site-product guide
// X1 / X2 = bonds whose first / second site differs between i and j; for the
// uniform guide X1 = every bond when i == j, X2 = the bond whose flip makes
// the child diagonal
template <typename MT, typename SW>
__device__ __forceinline__ void class_masks(const SpawnCtx &c, SW i, SW j, MT &X1, MT &X2) {
    const SW d = i ^ j;
    X1 = zero_mask<MT>();
    X2 = zero_mask<MT>();
    if (c.gk == 1) {
        if (d == 0) { X1 = bond_exists<MT>(c); return; }
        if (popcount(d) != 2) return;
        const int a = low_bit(d), b = high_bit(d);
        const SpawnTables &s = *c.sh;
        if ((c.ER >> a & 1ull) && s.rn[a] == b) X2 = one_bit<MT>(2 * a);
        else if ((c.ED >> a & 1ull) && s.dn[a] == b) X2 = one_bit<MT>(2 * a + 1);
        else if ((c.ER >> b & 1ull) && s.rn[b] == a) X2 = one_bit<MT>(2 * b);
        else if ((c.ED >> b & 1ull) && s.dn[b] == a) X2 = one_bit<MT>(2 * b + 1);
    } else if (c.gk == 2) {
        X1 = bond_mask<MT, SW>(d & (SW)c.ER, d & (SW)c.ED);
        X2 = bond_mask<MT, SW>(nb_right(c, d) & (SW)c.ER, nb_down(c, d) & (SW)c.ED);
    }
}

// sites of each importance class of a field flip of (i, j) (nm: the N site bits):
// site-product guide: class 0 = sites where i and j agree, 1 = where they
// differ; uniform guide: class 1 = every site of a diagonal parent, class 2 =
// the one differing site, class 0 = the rest
template <typename SW>
__device__ __forceinline__ void field_masks(const SpawnCtx &c, SW i, SW j, SW (&fm)[4]) {
    const SW d = i ^ j, nm = (SW)c.nmask;
    fm[0] = 0; fm[1] = 0; fm[2] = 0; fm[3] = 0;
    if (c.gk == 2) {
        fm[0] = ~d & nm;
        fm[1] = d;
    } else if (c.gk == 1) {
        if (d == 0) fm[1] = nm;
        else if (popcount(d) == 1) { fm[2] = d; fm[0] = ~d & nm; }
        else fm[0] = nm;
    } else {
        fm[0] = nm;
    }
}

__device__ __forceinline__ int site_class(int gk, uint64_t d, int k) {
    if (gk == 1) return d == 0 ? 1 : (d == (1ull << k) ? 2 : 0);
    if (gk == 2) return (int)((d >> k) & 1ull);
    return 0;
}

// bonds of group g = 4*anti + class, given the anti mask A of the flipped word
template <typename MT>
__device__ __forceinline__ MT group_mask(const SpawnCtx &c, MT A, MT X1, MT X2, int g) {
    const int cls = g & 3;
    MT cm;
    if (c.gk == 2) cm = ((cls & 2) ? X1 : (MT)~X1) & ((cls & 1) ? X2 : (MT)~X2);
    else if (c.gk == 1) cm = cls == 0 ? (MT)~(X1 | X2) : (cls == 1 ? X1 : (cls == 2 ? X2 : zero_mask<MT>()));
    else cm = cls == 0 ? (MT)~zero_mask<MT>() : zero_mask<MT>();
    return ((g & 4) ? A : (MT)~A) & cm & bond_exists<MT>(c);
}

// the four importance-class masks of group_mask (class k: bonds of class k
// that exist), computed once per configuration
template <typename MT>
__device__ __forceinline__ void class_group_masks(const SpawnCtx &c, MT X1, MT X2, MT (&cm)[4]) {
    const MT E = bond_exists<MT>(c);
    if (c.gk == 2) {
        cm[0] = ~X1 & ~X2 & E;
        cm[1] = ~X1 & X2 & E;
        cm[2] = X1 & ~X2 & E;
        cm[3] = X1 & X2 & E;
    } else if (c.gk == 1) {
        cm[0] = ~(X1 | X2) & E;
        cm[1] = X1 & E;
        cm[2] = X2 & E;
        cm[3] = zero_mask<MT>();
    } else {
        cm[0] = E;
        cm[1] = zero_mask<MT>();
        cm[2] = zero_mask<MT>();
        cm[3] = zero_mask<MT>();
    }
}

// position of the r-th set bit (r from 0) of m, given r < popcount(m)
__device__ __forceinline__ int select_bit(uint32_t m, uint32_t r) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const uint32_t c = (uint32_t)__popc(m & ((1u << w) - 1u));
        if (r >= c) { r -= c; m >>= w; pos += w; }
    }
    return pos;
}
__device__ __forceinline__ int select_bit(uint64_t m, uint32_t r) {
    const uint32_t lo = (uint32_t)m;
    const uint32_t c = (uint32_t)__popc(lo);
    return r < c ? select_bit(lo, r) : 32 + select_bit((uint32_t)(m >> 32), r - c);
}
__device__ __forceinline__ int select_bit(const U128 &m, uint32_t r) {
    const uint32_t c = (uint32_t)__popcll(m.lo);
    return r < c ? select_bit(m.lo, r) : 64 + select_bit(m.hi, r - c);
}

// floor(v / q) for a quotient below 64, by integer bisection (no division:
// the FP64 and 64-bit integer division paths are slow on this GPU)
__device__ __forceinline__ uint32_t small_quotient(uint64_t v, uint64_t q) {
    uint32_t r = 0;
#pragma unroll
    for (uint32_t b = 32; b >= 1; b >>= 1)
        if ((uint64_t)(r + b) * q <= v) r += b;
    return r;
}

// bond bit of the draw v (0 <= v < segment total) in a segment with group counts cnt
template <typename MT>
__device__ __forceinline__ int seg_select(const SpawnCtx &c, const uint64_t *rate8, uint64_t cnt,
                                          MT A, MT X1, MT X2, uint64_t v) {
    int g = 0;
    for (; g < 7; ++g) {
        const uint64_t w = rate8[g] * ((cnt >> (8 * g)) & 0xFFull);
        if (v < w) break;
        v -= w;
    }
    return select_bit(group_mask<MT>(c, A, X1, X2, g), small_quotient(v, rate8[g]));
}

// Same for a segment whose total is below 2^32 (every group with bonds then
// has a rate below 2^32): 32-bit arithmetic, and the index inside the group
// from a float reciprocal estimate corrected to the exact integer quotient.
template <typename MT>
__device__ __forceinline__ int seg_select32(const SpawnCtx &c, const uint32_t *rate32, const float *rinv,
                                            uint64_t cnt, MT A, MT X1, MT X2, uint32_t v) {
    // inclusive prefix P of the eight group totals; the group is the number
    // of prefixes at or below v, found by a three-level search of selects
    // (no serial subtract chain, no divergence)
    uint32_t P[8], acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        acc += rate32[k] * (uint32_t)((cnt >> (8 * k)) & 0xFFull);
        P[k] = acc;
    }
    const bool h4 = v >= P[3];
    const bool h2 = v >= (h4 ? P[5] : P[1]);
    const bool h1 = v >= (h4 ? (h2 ? P[6] : P[4]) : (h2 ? P[2] : P[0]));
    const int g = (h4 ? 4 : 0) + (h2 ? 2 : 0) + (h1 ? 1 : 0);
    v -= h4 ? (h2 ? (h1 ? P[6] : P[5]) : (h1 ? P[4] : P[3])) : (h2 ? (h1 ? P[2] : P[1]) : (h1 ? P[0] : 0u));
    const uint32_t q = rate32[g];
    const float qi = rinv[g];
    uint32_t r = (uint32_t)((float)v * qi);
    const uint64_t pq = (uint64_t)r * q;
    if (pq > v) --r;
    else if (pq + q <= v) ++r;
    return select_bit(group_mask<MT>(c, A, X1, X2, g), r);
}

// ---- per-move tables (heavy path) -------------------------------------------

// Child (ci, cj) of move m of configuration (i, j).  Move ids: ket bond b,
// bra bond B + b, ket field flip 2B + k, bra field flip 2B + N + k (at an
// angle: their x parts), jump 2B + 2N + k, and at an angle the y parts of the
// ket and bra flips 2B + 3N + k, 2B + 4N + k.  same: the child has the parent's type (real / imaginary);
// a: the sign of the element's non-zero part -- a real parent of sign s makes
// a child of sign s*a, an imaginary parent one of sign s*a (same type) or
// -s*a (other type).  P: the run's parameters (a single run reads its field
// settings from the shared-memory copy, a batch from P).
template <bool BATCH>
__device__ __forceinline__ void move_child(const SpawnCtx &c, const RunParams &P, uint64_t i, uint64_t j, int m,
                                           uint64_t &ci, uint64_t &cj, bool &same, int &a) {
    const SpawnTables &s = *c.sh;
    const int field_axis = BATCH ? P.field_axis : s.field_axis;
    const int sgn_hf = BATCH ? P.sgn_hf : s.sgn_hf;
    const int sgn_hf2 = BATCH ? P.sgn_hf2 : s.sgn_hf2;
    ci = i;
    cj = j;
    const int B = c.B, N = c.N;
    if (m < 2 * B) {                 // bond flip: A = -i h_b (ket) or +i h_b (bra)
        const bool ket = m < B;
        const int b = ket ? m : m - B;
        const uint64_t w = ket ? i : j;
        const int anti = (int)(((w >> s.bond_a[b]) ^ (w >> s.bond_b[b])) & 1ull);
        const int hs = P.sgn_h[anti];
        if (ket) ci ^= s.bond_m[b]; else cj ^= s.bond_m[b];
        same = false;
        a = ket ? -hs : hs;
    } else if (m < 2 * B + 2 * N) {  // field flip: -i h (ket), +i h (bra) along x; h (2 s_k - 1) along y
        const bool ket = m < 2 * B + N;
        const int k = ket ? m - 2 * B : m - 2 * B - N;
        const uint64_t w = ket ? i : j;
        if (ket) ci ^= 1ull << k; else cj ^= 1ull << k;
        if (field_axis != 1) {
            same = false;
            a = ket ? -sgn_hf : sgn_hf;
        } else {
            same = true;
            a = ((w >> k) & 1ull) ? sgn_hf : -sgn_hf;
        }
    } else if (m < 2 * B + 3 * N) {  // jump: +gamma
        const int k = m - 2 * B - 2 * N;
        ci &= ~(1ull << k);
        cj &= ~(1ull << k);
        same = true;
        a = 1;
    } else {                         // y part of a flip at an angle: h sin t (2 s_k - 1)
        const bool ket = m < 2 * B + 4 * N;
        const int k = ket ? m - 2 * B - 3 * N : m - 2 * B - 4 * N;
        const uint64_t w = ket ? i : j;
        if (ket) ci ^= 1ull << k; else cj ^= 1ull << k;
        same = true;
        a = ((w >> k) & 1ull) ? sgn_hf2 : -sgn_hf2;
    }
}

// ---- record output ----------------------------------------------------------

// kp: the batch run id already shifted into place (0 for a single run)
template <typename T>
__device__ __forceinline__ T make_spawn(uint64_t ci, uint64_t cj, int N, bool flag, int re, int im, uint64_t kp);
template <>
__device__ __forceinline__ Rec make_spawn<Rec>(uint64_t ci, uint64_t cj, int N, bool flag, int re, int im,
                                               uint64_t kp) {
    Rec r;
    r.key = (kp | (cj << N) | ci) | (flag ? FLAG_BIT : 0ull);
    r.re = re;
    r.im = im;
    return r;
}
template <>
__device__ __forceinline__ uint64_t make_spawn<uint64_t>(uint64_t ci, uint64_t cj, int N, bool flag, int re, int im,
                                                         uint64_t kp) {
    return pack_rec(kp | (cj << N) | ci, flag, re, im);
}
template <>
__device__ __forceinline__ P40 make_spawn<P40>(uint64_t ci, uint64_t cj, int N, bool flag, int re, int im, uint64_t kp) {
    return pack_p40(kp | (cj << N) | ci, flag, re, im);
}
template <>
__device__ __forceinline__ RecW make_spawn<RecW>(uint64_t ci, uint64_t cj, int, bool flag, int re, int im,
                                                 uint64_t kp) {
    RecW r;
    r.lo = ci;
    r.hi = cj | kp;
    r.re = (int32_t)((uint32_t)re << 1) | (flag ? 1 : 0);
    r.im = im;
    return r;
}

template <typename T, bool F>
__device__ __forceinline__ void count_digits(SpawnShared<T, F> &s, const T &r, int npass) {
    // one-word keys: pass p reads bits 8p..8p+7; two-word keys: per-pass shifts
    for (int p = 0; p < npass; ++p) {
        const int shift = std::is_same<T, RecW>::value ? s.pass_shift[p] : 8 * p;
        atomicAdd(&s.hist[p][RecTraits<T>::digit(r, shift)], 1u);
    }
}

// Append one record from a (possibly divergent) lane.
template <typename T, bool F>
__device__ __forceinline__ void emit(SpawnShared<T, F> &s, int warp, const T &r, T *out, int64_t cap,
                                     DevState *st, int npass) {
    T *stage = &s.stage[warp][0];
    // one staging-counter update for all the lanes that emit together
    const unsigned am = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(am) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&s.stage_n[warp], __popc(am));
    base = __shfl_sync(am, base, leader);
    const int pos = base + __popc(am & ((1u << lane) - 1u));
    if (pos < SpawnShared<T, F>::STAGE) {
        stage[pos] = r;
    } else {
        const unsigned long long idx = atomicAdd((unsigned long long *)&st->R, 1ull);
        if ((int64_t)idx < cap) {
            out[idx] = r;
            count_digits(s, r, npass);
        } else {
            atomicOr(&st->status, ST_CAPACITY | ST_CAP_SPAWN);
        }
    }
}

// Append an aggregated child (any int32 counts): packed records carry at most
// PK_LIM walkers per part, 40-bit-key records P40_LIM and two-word records
// WK_LIM, so large counts become several records.
template <typename T, bool F>
__device__ __forceinline__ void emit_counts(SpawnShared<T, F> &s, int warp, uint64_t ci, uint64_t cj, int N, bool flag,
                                            int cre, int cim, T *out, int64_t cap, DevState *st, int npass,
                                            uint64_t kp) {
    if constexpr (std::is_same<T, Rec>::value) {
        emit(s, warp, make_spawn<T>(ci, cj, N, flag, cre, cim, kp), out, cap, st, npass);
    } else {
        constexpr int LIM = std::is_same<T, RecW>::value ? WK_LIM : (std::is_same<T, P40>::value ? P40_LIM : PK_LIM);
        while (cre != 0 || cim != 0) {
            const int pr = cre > LIM ? LIM : (cre < -LIM ? -LIM : cre);
            const int pi = cim > LIM ? LIM : (cim < -LIM ? -LIM : cim);
            emit(s, warp, make_spawn<T>(ci, cj, N, flag, pr, pi, kp), out, cap, st, npass);
            cre -= pr;
            cim -= pi;
        }
    }
}

// Warp-uniform flush of the warp's staged records.
template <typename T, bool F>
__device__ __forceinline__ void flush(SpawnShared<T, F> &s, int warp, int lane, T *out, int64_t cap,
                                      DevState *st, int npass, int min_n) {
    __syncwarp();
    const T *stage = &s.stage[warp][0];
    int n = s.stage_n[warp];
    if (n > SpawnShared<T, F>::STAGE) n = SpawnShared<T, F>::STAGE;
    if (n >= min_n && n > 0) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd((unsigned long long *)&st->R, (unsigned long long)n);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (int k = lane; k < n; k += 32) {
            const T r = stage[k];
            if ((int64_t)(base + k) < cap) {
                out[base + k] = r;
                count_digits(s, r, npass);
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

// Resolve the first n queued spawn draws of the warp, one per lane: the move
// (ket, bra or jump segment, then the group and the bond inside it), the child
// configuration and its signed unit, appended as a spawn record.  A single
// run reads its rate tables from shared memory; in a batch (BATCH) each
// configuration carries its run id and the tables are that run's (Pr).
template <typename T, typename MT, typename SW, bool FIELD, bool BATCH>
__device__ __forceinline__ void spawn_drain(SpawnShared<T, FIELD> &s, const SpawnCtx &c, const RunParams *__restrict__ Pr,
                                            int run_shift, int warp, int lane, int n, int N, T *out, int64_t cap,
                                            DevState *st, int npass) {
    if (lane < n) {
        const uint64_t v = s.qv[warp][lane];
        const uint32_t meta = s.qm[warp][lane];
        const int o = (int)(meta & 31u);
        const int part = (int)((meta >> 5) & 1u);
        const int sig = (meta & 64u) ? -1 : 1;
        const auto &q = s.ws[warp].le;
        const SW qi = q.i[o], qj = q.j[o];
        const uint64_t qT = q.T[o], qTket = q.Tket[o], qTbra = q.Tbra[o];
        // initiator flag in bit 0, batch run id above it
        const int qinit = q.init[o];
        const int orun = BATCH ? (qinit >> 1) : 0;
        const RunParams &R = Pr[orun];
        SW ci = qi, cj = qj;
        int cre = 0, cim = 0;
        if (v < qTket + qTbra) {
            const bool ket = v < qTket;
            const MT A = ket ? q.Ai[o] : q.Aj[o];
            const MT X1 = q.X1[o], X2 = q.X2[o];
            const uint64_t cnt8 = ket ? q.gk[o] : q.gb[o];
            const uint64_t vs = ket ? v : v - qTket;
            int p;
            if constexpr (BATCH)
                p = qT <= 0xFFFFFFFFull ? seg_select32<MT>(c, R.urate32, R.uinv, cnt8, A, X1, X2, (uint32_t)vs)
                                        : seg_select<MT>(c, R.urate8, cnt8, A, X1, X2, vs);
            else
                p = qT <= 0xFFFFFFFFull ? seg_select32<MT>(c, s.urate32, s.uinv, cnt8, A, X1, X2, (uint32_t)vs)
                                        : seg_select<MT>(c, s.urate8, cnt8, A, X1, X2, vs);
            const int k = p >> 1;
            const int other = (p & 1) ? s.dn[k] : s.rn[k];
            const SW m = ((SW)1 << k) | ((SW)1 << other);
            const int hs = BATCH ? R.sgn_h[mask_bit(A, p)] : s.sgn_h[mask_bit(A, p)];
            const int gsg = ket ? -hs : hs;
            if (ket) ci ^= m; else cj ^= m;
            if (part == 0) cim = sig * gsg; else cre = -sig * gsg;
        } else if (FIELD && v - qTket - qTbra < 2 * q.Tf[o]) {
            // field flip: ket segment, then bra segment; groups by importance class
            const uint64_t qTf = q.Tf[o];
            const uint32_t fcp = q.fc[o];
            const uint64_t vb = v - qTket - qTbra;
            const bool ket = vb < qTf;
            uint64_t vf = ket ? vb : vb - qTf;
            // at an angle: the x part of the segment's flips, then the y part
            const uint64_t *fr = BATCH ? R.ufrate : s.ufrate;
            const uint32_t *fr32 = BATCH ? R.ufrate32 : s.ufrate32;
            const float *fri = BATCH ? R.ufinv : s.ufinv;
            bool ypart = false;
            if (s.fparts == 2) {
                uint64_t tx = 0;
#pragma unroll
                for (int g = 0; g < 4; ++g) tx += fr[g] * (uint64_t)((fcp >> (8 * g)) & 0xFFu);
                if (vf >= tx) {
                    vf -= tx;
                    ypart = true;
                    fr = BATCH ? R.ufrate2 : s.ufrate2;
                    fr32 = BATCH ? R.ufrate32_2 : s.ufrate32_2;
                    fri = BATCH ? R.ufinv2 : s.ufinv2;
                }
            }
            int g = 0;
            for (; g < 3; ++g) {
                const uint64_t w = fr[g] * (uint64_t)((fcp >> (8 * g)) & 0xFFu);
                if (vf < w) break;
                vf -= w;
            }
            uint32_t idx;
            if (qT <= 0xFFFFFFFFull) {
                const uint32_t rq = fr32[g];
                idx = (uint32_t)((float)(uint32_t)vf * fri[g]);
                const uint64_t pq = (uint64_t)idx * rq;
                if (pq > vf) --idx;
                else if (pq + rq <= vf) ++idx;
            } else {
                idx = small_quotient(vf, fr[g]);
            }
            SW fm[4];
            field_masks<SW>(c, qi, qj, fm);
            const int k = select_bit(fm[g], idx);
            const SW w = ket ? qi : qj;
            const int axis = BATCH ? R.field_axis : s.field_axis;
            const int shf = ypart ? (BATCH ? R.sgn_hf2 : s.sgn_hf2) : (BATCH ? R.sgn_hf : s.sgn_hf);
            if (ket) ci ^= (SW)1 << k; else cj ^= (SW)1 << k;
            if (!ypart && axis != 1) {           // -i h (ket), +i h (bra): the other type
                const int gsg = ket ? -shf : shf;
                if (part == 0) cim = sig * gsg; else cre = -sig * gsg;
            } else {                             // h (2 s_k - 1): the same type
                const int a = ((w >> k) & 1) ? shf : -shf;
                if (part == 0) cre = sig * a; else cim = sig * a;
            }
        } else {
            // jumps share one rate: the site index is the quotient by it
            const uint64_t vj = v - qTket - qTbra - (FIELD ? 2 * q.Tf[o] : 0ull);
            const uint64_t jq = BATCH ? R.jump_q : c.jump_q;
            uint32_t idx;
            if (qT <= 0xFFFFFFFFull) {
                idx = (uint32_t)((float)(uint32_t)vj * (BATCH ? R.jinv : s.jinv));
                const uint64_t pq = (uint64_t)idx * jq;
                if (pq > vj) --idx;
                else if (pq + jq <= vj) ++idx;
            } else {
                idx = small_quotient(vj, jq);
            }
            const int k = select_bit((SW)(qi & qj), idx);
            ci &= ~((SW)1 << k);
            cj &= ~((SW)1 << k);
            if (part == 0) cre = sig; else cim = sig;
        }
        const uint64_t kp = BATCH ? (uint64_t)orun << run_shift : 0ull;
        uint64_t cjs = (uint64_t)cj;
        if constexpr (std::is_same<T, RecW>::value) cjs = bra_swap((uint64_t)ci, cjs, c.hmask);
        emit(s, warp, make_spawn<T>((uint64_t)ci, cjs, N, (qinit & 1) != 0, cre, cim, kp), out, cap, st, npass);
    }
    __syncwarp();
}

// FIELD: the run has the in-plane field's site flips (a separate instantiation
// keeps them out of the runs without).  BATCH: the list holds several runs
// (run id in the key's high bits, see RunParams::nruns); Pp then holds the
// batch's shared geometry, Pr[r] and rs[r] run r's rates, shift and death
// table, and st the shared step counters.  A single run passes Pr = Pp and
// rs = st (unread).
template <typename T, bool FIELD, bool BATCH>
__global__ void __launch_bounds__(SP_TPB, (SpawnBlocks<T, BATCH>::value))
k_spawn_death(const RunParams *__restrict__ Pp, DevState *__restrict__ st, typename ListOf<T>::type *__restrict__ L,
              T *__restrict__ out, int64_t cap, const RunParams *__restrict__ Pr, const DevState *__restrict__ rs,
              int64_t heavy_walkers) {
    // mask and spin-word types of the light path: 32-bit masks for packed
    // records (2N <= 32), 64-bit up to 31 sites, 128-bit (two words) beyond
    using MT = typename LightTypes<T>::MT;
    using SW = typename LightTypes<T>::SW;
    using LT = typename ListOf<T>::type;
    constexpr bool WIDE = std::is_same<T, RecW>::value;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SpawnShared<T, FIELD> &s = *reinterpret_cast<SpawnShared<T, FIELD> *>(smem_raw);
    const RunParams &P = *Pp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (block_stopped(st)) return;
    const int N = P.N, B = P.B, K = P.K, npass = P.npass;
    // stage the constant tables
    for (int q = tid; q < B; q += SP_TPB) {
        s.bond_m[q] = P.bond_m[q];
        s.bond_a[q] = (int8_t)P.bond_a[q];
        s.bond_b[q] = (int8_t)P.bond_b[q];
    }
    for (int q = tid; q < N; q += SP_TPB) { s.rn[q] = P.rn[q]; s.dn[q] = P.dn[q]; }
    for (int q = tid; q < MAXPASS; q += SP_TPB) s.pass_shift[q] = P.pass_shift[q];
    if (tid < 8) {
        s.urate8[tid] = P.urate8[tid];
        s.urate32[tid] = (uint32_t)P.urate8[tid];
        s.uinv[tid] = P.urate8[tid] ? 1.0f / (float)P.urate8[tid] : 0.0f;
    }
    if (tid < 2) s.sgn_h[tid] = P.sgn_h[tid];
    if (tid == 0) s.jinv = P.jump_q ? 1.0f / (float)P.jump_q : 0.0f;
    if (tid < 4) {
        s.ufrate[tid] = P.ufrate[tid];
        s.ufrate32[tid] = (uint32_t)P.ufrate[tid];
        s.ufinv[tid] = P.ufrate[tid] ? 1.0f / (float)P.ufrate[tid] : 0.0f;
    }
    if (tid < 4) {
        s.ufrate2[tid] = P.ufrate2[tid];
        s.ufrate32_2[tid] = (uint32_t)P.ufrate2[tid];
        s.ufinv2[tid] = P.ufrate2[tid] ? 1.0f / (float)P.ufrate2[tid] : 0.0f;
    }
    if (tid == 0) {
        s.field_on = P.field_on;
        s.field_axis = P.field_axis;
        s.sgn_hf = P.sgn_hf;
        s.sgn_hf2 = P.sgn_hf2;
        s.fparts = P.K == 2 * P.B + 5 * P.N ? 2 : 1;
    }
    for (int q = tid; q <= 2 * B; q += SP_TPB) s.cross_int[q] = P.cross_int[q];
    for (int q = tid; q <= 2 * N; q += SP_TPB) { s.d_int[q] = st->d_int[q]; s.d_sgn[q] = st->d_sgn[q]; }
    for (int q = tid; q <= 2 * B; q += SP_TPB) s.cross_frac32[q] = (uint32_t)P.cross_frac[q];
    for (int q = tid; q <= 2 * N; q += SP_TPB) s.d_frac32[q] = (uint32_t)st->d_frac[q];
    for (int q = tid; q < SpawnShared<T, FIELD>::NP * 256; q += SP_TPB) (&s.hist[0][0])[q] = 0u;
    if (tid < SP_WARPS) s.stage_n[tid] = 0;
    __syncthreads();

    SpawnCtx c;
    c.sh = &s; c.N = N; c.B = B; c.K = K; c.gk = P.guide_kind; c.jump_q = P.jump_q; c.nmask = P.nmask;
    c.ER = P.ER; c.ED = P.ED; c.LC = P.LC; c.LR = P.LR; c.Lx = P.Lx; c.shD = P.shD;
    c.Emorton = P.Emorton; c.Emorton_hi = P.Emorton_hi;
    c.hmask = P.hash_mask;
    const bool uniform = P.uniform != 0;
    const int64_t M = st->M;
    const uint64_t t = (uint64_t)st->t;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32) ^ (uint32_t)t;
    const uint64_t nmask = P.nmask;
    const int n_a = P.n_a;
    const int sgn_jz = P.sgn_jz;
    const int nruns = P.nruns, run_shift = P.run_shift;
    uint32_t local_status = 0;

    const int64_t nwarps = (int64_t)gridDim.x * SP_WARPS;
    for (int64_t chunk = (int64_t)blockIdx.x * SP_WARPS + warp; chunk * 32 < M; chunk += nwarps) {
        const int64_t e = chunk * 32 + lane;
        LT rec;
        uint64_t i = 0, j = 0;
        int crun = 0;                    // batch run of this lane's configuration
        rec.re = 0;
        rec.im = 0;
        if (e < M) {
            rec = L[e];
            if constexpr (WIDE) { i = rec.lo; j = bra_swap(rec.lo, rec.hi, c.hmask); }
            else { i = rec.key & nmask; j = rec.key >> N; }
            if constexpr (BATCH) {
                // the run id: from bit run_shift of a two-word key's bra word
                // (above the spin and hash bits), from bit N of key >> N
                crun = batch_run(j, WIDE ? run_shift : N, nruns);
                j &= nmask;
            }
        }
        const RunParams &CR = Pr[crun];
        const int64_t nre = iabs64(rec.re), nim = iabs64(rec.im);
        const int64_t nw = nre + nim;
        const bool valid = e < M && (!BATCH || CR.active != 0);
        const bool heavy = valid && (nw > heavy_walkers || !(BATCH ? CR.uniform != 0 : uniform));
        const bool light = valid && !heavy;
        const int na_r = BATCH ? CR.n_a : n_a;
        const bool init = (na_r == 0) || (i == j) || (nw > (int64_t)na_r);

        // ---- light configurations: per-configuration setup, one lane each ----
        int nl = 0;
        if (light) {
            auto &q = s.ws[warp].le;
            const SW i32 = (SW)i, j32 = (SW)j;
            const MT Ai = anti_mask<MT, SW>(c, i32), Aj = anti_mask<MT, SW>(c, j32);
            MT X1, X2;
            class_masks<MT, SW>(c, i32, j32, X1, X2);
            MT cm[4];
            class_group_masks<MT>(c, X1, X2, cm);
            uint64_t Tket = 0, Tbra = 0, gkp = 0, gbp = 0;
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const int ck = popcount(((g & 4) ? Ai : (MT)~Ai) & cm[g & 3]);
                const int cb = popcount(((g & 4) ? Aj : (MT)~Aj) & cm[g & 3]);
                gkp |= (uint64_t)ck << (8 * g);
                gbp |= (uint64_t)cb << (8 * g);
                const uint64_t rg = BATCH ? CR.urate8[g] : s.urate8[g];
                Tket += rg * (uint64_t)ck;
                Tbra += rg * (uint64_t)cb;
            }
            uint64_t Tf = 0;
            uint32_t fcp = 0;
            if constexpr (FIELD) {
                SW fm[4];
                field_masks<SW>(c, i32, j32, fm);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const int cf = popcount(fm[g]);
                    fcp |= (uint32_t)cf << (8 * g);
                    // both parts of a flip at an angle (the y part's rates are 0 otherwise)
                    Tf += ((BATCH ? CR.ufrate[g] : s.ufrate[g]) + (BATCH ? CR.ufrate2[g] : s.ufrate2[g])) *
                          (uint64_t)cf;
                }
            }
            const uint64_t Tall = Tket + Tbra + 2 * Tf + (uint64_t)popcount((SW)(i32 & j32)) * (BATCH ? CR.jump_q : c.jump_q);
            const uint64_t natt = (Tall + 0xFFFFFFFFull) >> 32;
            q.Ai[lane] = Ai;
            q.Aj[lane] = Aj;
            q.X1[lane] = X1;
            q.X2[lane] = X2;
            q.Tket[lane] = Tket;
            q.Tbra[lane] = Tbra;
            q.T[lane] = Tall;
            if constexpr (FIELD) {
                q.Tf[lane] = Tf;
                q.fc[lane] = fcp;
            }
            q.gk[lane] = gkp;
            q.gb[lane] = gbp;
            q.natt[lane] = natt == 0 ? 1u : (uint32_t)natt;
            q.i[lane] = i32;
            q.j[lane] = j32;
            q.re[lane] = rec.re;
            q.im[lane] = rec.im;
            q.nre[lane] = (int32_t)nre;
            q.cd[lane] = popcount(i32) + popcount(j32);
            const int dz = 2 * (popcount(Aj) - popcount(Ai));     // zsum(i) - zsum(j)
            q.adz[lane] = dz < 0 ? -dz : dz;
            q.sgn_d[lane] = (dz == 0) ? 0 : -(BATCH ? CR.sgn_jz : sgn_jz) * (dz > 0 ? 1 : -1);
            q.init[lane] = (crun << 1) | (init ? 1 : 0);
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
        const int excl = incl - nl;
        const int Wl = __shfl_sync(0xFFFFFFFFu, incl, 31);
        __syncwarp();

        // ---- light walkers, spread over the lanes ----------------------------
        // Death / cloning and the Re <-> Im transfer are applied per walker; a
        // draw that lands below the total rate is queued, and the move
        // searches run 32 at a time with every lane busy.
        int qn = 0;                      // queued spawn draws (same value in every lane)
        // the configurations' first walker positions, for the owner search
        __syncwarp();
        s.mark[warp][lane] = excl;
        __syncwarp();
        for (int base = 0; base < Wl; base += 32) {
            const bool last_base = base + 32 >= Wl;
            const int g = base + lane;
            const bool act = g < Wl;
            // owner of walker g: the last configuration starting at or before
            // g (binary search of the non-decreasing first positions)
            int owner = 0;
#pragma unroll
            for (int sft = 16; sft >= 1; sft >>= 1)
                if (s.mark[warp][owner + sft] <= g) owner += sft;
            const int owner_excl = __shfl_sync(0xFFFFFFFFu, excl, owner);
            int part = 0, sig = 1;
            uint32_t natt = 0;
            uint64_t qT = 0;
            uint4 x = make_uint4(0u, 0u, 0u, 0u), ctr = x;
            uint32_t wk0 = k0, wk1 = k1;     // Philox key of the owner's run
            if (act) {
                const auto &q = s.ws[warp].le;
                const int nre_o = q.nre[owner];
                const int local = g - owner_excl;
                part = local < nre_o ? 0 : 1;
                const uint32_t w = (uint32_t)(part ? local - nre_o : local);
                sig = (part ? q.im[owner] : q.re[owner]) < 0 ? -1 : 1;
                // counter words: the spin words, high halves folded in (zero up to 32 sites)
                const uint64_t oi = (uint64_t)q.i[owner], oj = (uint64_t)q.j[owner];
                ctr = make_uint4((uint32_t)oi ^ ((uint32_t)(oi >> 32) * 0x9E3779B9u),
                                 (uint32_t)oj ^ ((uint32_t)(oj >> 32) * 0x85EBCA6Bu), w, (uint32_t)part << 16);
                const int cd = q.cd[owner], adz = q.adz[owner];
                int cnt, cc, dsg;
                if constexpr (BATCH) {
                    const int orun = q.init[owner] >> 1;
                    const RunParams &OR = Pr[orun];
                    const DevState &OS = rs[orun];
                    wk0 = (uint32_t)OR.seed;
                    wk1 = (uint32_t)(OR.seed >> 32) ^ (uint32_t)t;
                    x = philox4x32_10(ctr, wk0, wk1);
                    cnt = (int)OS.d_int[cd] + ((uint64_t)x.y < OS.d_frac[cd] ? 1 : 0);
                    cc = (int)OR.cross_int[adz] + ((uint64_t)x.z < OR.cross_frac[adz] ? 1 : 0);
                    dsg = OS.d_sgn[cd];
                } else {
                    x = philox4x32_10(ctr, k0, k1);
                    cnt = (int)s.d_int[cd] + (x.y < s.d_frac32[cd] ? 1 : 0);
                    cc = (int)s.cross_int[adz] + (x.z < s.cross_frac32[adz] ? 1 : 0);
                    dsg = s.d_sgn[cd];
                }
                const int ddeath = -dsg * sig * cnt;
                const int dcross = sig * q.sgn_d[owner] * cc;
                if (part == 0) {
                    if (ddeath) atomicAdd(&s.dre[warp][owner], ddeath);
                    if (dcross) atomicAdd(&s.dim[warp][owner], dcross);
                } else {
                    if (ddeath) atomicAdd(&s.dim[warp][owner], ddeath);
                    if (dcross) atomicAdd(&s.dre[warp][owner], -dcross);
                }
                natt = q.natt[owner];
                qT = q.T[owner];
            }
            const uint32_t nmax = __reduce_max_sync(0xFFFFFFFFu, natt);
            uint4 xb = x;
            uint32_t blk = 0;
            for (uint32_t a = 0; a < nmax; ++a) {
                bool ev = false;
                uint64_t v = 0;
                if (a < natt) {
                    const uint32_t u = BATCH ? attempt_word(x, xb, blk, a, ctr, wk0, wk1)
                                             : attempt_word(x, xb, blk, a, ctr, k0, k1);
                    v = (uint64_t)u * natt;
                    ev = v < qT;
                }
                const unsigned em = __ballot_sync(0xFFFFFFFFu, ev);
                if (ev) {
                    const int pos = qn + __popc(em & ((1u << lane) - 1u));
                    s.qv[warp][pos] = v;
                    s.qm[warp][pos] = (uint32_t)owner | ((uint32_t)part << 5) | (sig < 0 ? 64u : 0u);
                }
                qn += __popc(em);
                // resolve full batches of 32, and what is left after the
                // chunk's last draw (the one place the draws are resolved)
                const bool fin = last_base && a + 1 == nmax;
                while (qn >= 32 || (fin && qn > 0)) {
                    __syncwarp();
                    // a drain adds up to 32 records: flush first when they
                    // might not fit, so that no record takes the one-by-one
                    // path through the global record counter
                    flush(s, warp, lane, out, cap, st, npass, SpawnShared<T, FIELD>::STAGE - 32 + 1);
                    const int nd = qn < 32 ? qn : 32;
                    spawn_drain<T, MT, SW, FIELD, BATCH>(s, c, Pr, run_shift, warp, lane, nd, N, out, cap, st, npass);
                    qn -= nd;
                    // move the rest of the queue to the front
                    uint64_t rv = 0;
                    uint32_t rm = 0;
                    if (lane < qn) { rv = s.qv[warp][32 + lane]; rm = s.qm[warp][32 + lane]; }
                    __syncwarp();
                    if (lane < qn) { s.qv[warp][lane] = rv; s.qm[warp][lane] = rm; }
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
            const int hrun = BATCH ? __shfl_sync(0xFFFFFFFFu, crun, h) : 0;
            const RunParams &HP = BATCH ? Pr[hrun] : P;         // the configuration's run
            const uint64_t hjump = BATCH ? HP.jump_q : c.jump_q;
            const uint64_t hkp = BATCH ? (uint64_t)hrun << run_shift : 0ull;
            const uint32_t hk0 = BATCH ? (uint32_t)HP.seed : k0;
            const uint32_t hk1 = BATCH ? ((uint32_t)(HP.seed >> 32) ^ (uint32_t)t) : k1;
            // rates of the K moves in move order (group-major inside each bond
            // segment, via ballots over the bonds), then their running sums
            {
                const uint64_t hd = hi ^ hj;
                const unsigned lt = (1u << lane) - 1u;
                int base = 0;
                // bond lane + 32 q of slot q; slots in order keep bond order in a group
                constexpr int NSLOT = (WIDE ? MAXB : 2 * NPACK + 2) / 32;
                for (int seg = 0; seg < 2; ++seg) {
                    const uint64_t w = seg == 0 ? hi : hj;
                    int gq[NSLOT];
                    uint64_t rq[NSLOT];
#pragma unroll
                    for (int q = 0; q < NSLOT; ++q) {
                        const int b = lane + 32 * q;
                        gq[q] = -1;
                        rq[q] = 0;
                        if (b < B) {
                            const int a0 = s.bond_a[b], a1 = s.bond_b[b];
                            const int anti = (int)(((w >> a0) ^ (w >> a1)) & 1ull);
                            const int cl = imp_class(c.gk, hd, s.bond_m[b], a0, a1);
                            gq[q] = 4 * anti + cl;
                            rq[q] = HP.rate_q[b][anti][cl];
                        }
                    }
                    for (int g = 0; g < 8; ++g) {
#pragma unroll
                        for (int q = 0; q < NSLOT; ++q) {
                            if (32 * q >= B) break;
                            const unsigned mq = __ballot_sync(0xFFFFFFFFu, gq[q] == g);
                            if (gq[q] == g) {
                                const int pos = base + __popc(mq & lt);
                                s.ws[warp].hv.cum[pos] = rq[q];
                                s.ws[warp].hv.mv[pos] = (int16_t)(seg * B + lane + 32 * q);
                            }
                            base += __popc(mq);
                        }
                    }
                }
                if (FIELD) {
                    // field flips: ket then bra; at an angle the x part of the
                    // segment, then its y part; groups by importance class, sites in order
                    for (int sp = 0; sp < 2 * s.fparts; ++sp) {
                        const int seg = sp / s.fparts, fp = sp % s.fparts;
                        int gq[2];
                        uint64_t rq[2];
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int k = lane + 32 * q;
                            gq[q] = -1;
                            rq[q] = 0;
                            if (k < N) {
                                gq[q] = site_class(c.gk, hd, k);
                                rq[q] = fp ? HP.frate_q2[k][gq[q]] : HP.frate_q[k][gq[q]];
                            }
                        }
                        // move ids: x part (or the axis) 2B + seg N + k, y part 2B + (3 + seg) N + k
                        const int mv0 = 2 * B + (fp ? 3 + seg : seg) * N;
                        for (int g = 0; g < 4; ++g) {
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                if (32 * q >= N) break;
                                const unsigned mq = __ballot_sync(0xFFFFFFFFu, gq[q] == g);
                                if (gq[q] == g) {
                                    const int pos = base + __popc(mq & lt);
                                    s.ws[warp].hv.cum[pos] = rq[q];
                                    s.ws[warp].hv.mv[pos] = (int16_t)(mv0 + lane + 32 * q);
                                }
                                base += __popc(mq);
                            }
                        }
                    }
                }
                for (int k = lane; k < N; k += 32) {
                    s.ws[warp].hv.cum[base + k] = (((hi & hj) >> k) & 1ull) ? hjump : 0ull;
                    s.ws[warp].hv.mv[base + k] = (int16_t)(2 * B + 2 * N + k);
                }
                __syncwarp();
            }
            uint64_t carry = 0;
            for (int base = 0; base < K; base += 32) {
                const int m = base + lane;
                uint64_t r = m < K ? s.ws[warp].hv.cum[m] : 0ull;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, r, off);
                    if (lane >= off) r += y;
                }
                if (m < K) s.ws[warp].hv.cum[m] = carry + r;
                carry += __shfl_sync(0xFFFFFFFFu, r, 31);
            }
            for (int m = lane; m < K; m += 32) { s.ws[warp].hv.cnt_re[m] = 0; s.ws[warp].hv.cnt_im[m] = 0; }
            __syncwarp();
            const uint64_t Ttot = carry;
            uint64_t natt = (Ttot + 0xFFFFFFFFull) >> 32;
            if (natt == 0) natt = 1;
            // anti-aligned bonds of each side (one bit per bond of the mask formulation)
            const int na_i = popcount(anti_mask<MT, SW>(c, (SW)hi)), na_j = popcount(anti_mask<MT, SW>(c, (SW)hj));
            const int cd = __popcll(hi) + __popcll(hj);
            const int dz = 2 * (na_j - na_i);
            const int adz = dz < 0 ? -dz : dz;
            const int sgn_d = (dz == 0) ? 0 : -(BATCH ? HP.sgn_jz : sgn_jz) * (dz > 0 ? 1 : -1);
            int64_t dre = 0, dim = 0;
            for (int part = 0; part < 2; ++part) {
                const int64_t pop = part == 0 ? hre : him;
                const int64_t n = iabs64(pop);
                const int sig = pop < 0 ? -1 : 1;
                for (int64_t w = lane; w < n; w += 32) {
                    // counter words: the spin words, their high halves folded in
                    // (zero for N <= 32)
                    const uint4 ctr = make_uint4((uint32_t)hi ^ ((uint32_t)(hi >> 32) * 0x9E3779B9u),
                                                 (uint32_t)hj ^ ((uint32_t)(hj >> 32) * 0x85EBCA6Bu), (uint32_t)w,
                                                 (uint32_t)part << 16);
                    const uint4 x = philox4x32_10(ctr, hk0, hk1);
                    int64_t cnt, cc, dsg;
                    if constexpr (BATCH) {
                        const DevState &HS = rs[hrun];
                        cnt = (int64_t)HS.d_int[cd] + ((uint64_t)x.y < HS.d_frac[cd] ? 1 : 0);
                        cc = (int64_t)HP.cross_int[adz] + ((uint64_t)x.z < HP.cross_frac[adz] ? 1 : 0);
                        dsg = HS.d_sgn[cd];
                    } else {
                        cnt = (int64_t)s.d_int[cd] + (x.y < s.d_frac32[cd] ? 1 : 0);
                        cc = (int64_t)s.cross_int[adz] + (x.z < s.cross_frac32[adz] ? 1 : 0);
                        dsg = s.d_sgn[cd];
                    }
                    if (part == 0) { dre -= dsg * sig * cnt; dim += (int64_t)sig * sgn_d * cc; }
                    else { dim -= dsg * sig * cnt; dre -= (int64_t)sig * sgn_d * cc; }
                    uint4 xb = x;
                    uint32_t blk = 0;
                    for (uint64_t a = 0; a < natt; ++a) {
                        const uint32_t u = attempt_word(x, xb, blk, a, ctr, hk0, hk1);
                        const uint64_t v = (uint64_t)u * natt;
                        if (v >= Ttot) continue;
                        int lo = 0, hi2 = K - 1;
                        while (lo < hi2) {
                            const int mid = (lo + hi2) >> 1;
                            if (v < s.ws[warp].hv.cum[mid]) hi2 = mid; else lo = mid + 1;
                        }
                        uint64_t ci, cj;
                        int gsg;
                        bool same;
                        move_child<BATCH>(c, HP, hi, hj, s.ws[warp].hv.mv[lo], ci, cj, same, gsg);
                        // child type (0 real, 1 imaginary) and signed unit
                        const int tgt = same ? part : 1 - part;
                        const int val = (same || part == 0) ? sig * gsg : -sig * gsg;
                        // one shared-memory update per distinct (move, type) among the lanes here
                        const unsigned am = __activemask();
                        const unsigned peers = __match_any_sync(am, (unsigned)(lo * 2 + tgt));
                        const unsigned posm = __ballot_sync(am, val > 0);
                        if (lane == __ffs(peers) - 1) {
                            const int sum = __popc(peers & posm) - __popc(peers & ~posm);
                            if (sum) atomicAdd(tgt ? &s.ws[warp].hv.cnt_im[lo] : &s.ws[warp].hv.cnt_re[lo], sum);
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
                const int32_t cre = s.ws[warp].hv.cnt_re[m], cim = s.ws[warp].hv.cnt_im[m];
                if (cre == 0 && cim == 0) continue;
                uint64_t ci, cj;
                int gsg;
                bool same;
                move_child<BATCH>(c, HP, hi, hj, s.ws[warp].hv.mv[m], ci, cj, same, gsg);
                if constexpr (WIDE) cj = bra_swap(ci, cj, c.hmask);
                emit_counts(s, warp, ci, cj, N, hinit, cre, cim, out, cap, st, npass, hkp);
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
