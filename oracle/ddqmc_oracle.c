/*
 * DDQMC oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of one step of the
 * driven-dissipative FCIQMC of Nagy & Savona (arXiv:1802.05931) for the
 * spin-1/2 XYZ lattice with sigma^- decay on every site.  Only the test
 * suite, the package smoke check and the benchmark's CPU-baseline leg may
 * build, load or call this file.  The CUDA library never links it, and the
 * two share no code, header, table or helper.
 *
 * What one step computes, in the paper's order (Sec. III.C):
 *   (i)   spawning along the off-diagonal elements of the shifted Liouvillian
 *         (Kronecker form and element equation of Sec. III.C), with the four
 *         real/imaginary parent/child sign rules;
 *   (ii)  clone/death from the real part of the diagonal element and the
 *         on-site Re<->Im transfer from its imaginary part;
 *   (iii) annihilation: all contributions to one configuration |i><j| are
 *         summed, real and imaginary parts separately, under the initiator
 *         survival rule of Sec. IV.A;
 *   then the estimators of Sec. III.A (ratio of traces) and the shift update
 *   of Sec. III.C.
 *
 * Fixed readings of what the paper leaves open (the CUDA path follows the same
 * written rules, from its own code):
 *   - basis: site k = x + Lx*y, bit k of a spin word set <=> spin up;
 *     a configuration is (ket i, bra j); canonical order is (bra, ket);
 *   - H = sum over bonds of Jx sx sx + Jy sy sy + Jz sz sz (Pauli matrices),
 *     decay gamma * D[sigma^-] on every site (Sec. V, XYZ model);
 *   - moves, in this order: ket bond flips, bra bond flips, ket site flips
 *     and bra site flips of the in-plane field (only when h != 0), then jumps
 *     by site; inside a bond-flip segment grouped by (anti-aligned,
 *     importance class) and in bond order inside a group; inside a site-flip
 *     segment grouped by importance class, in site order inside a group.  A
 *     field at a general angle (axis 2) has an element with a real and an
 *     imaginary part, so each site flip becomes two moves, one per part: a
 *     site-flip segment then holds the imaginary-part (cos) moves, then the
 *     real-part (sin) moves, each grouped as above;
 *   - per-walker categorical draws, which have the joint law of the
 *     binomial + multinomial scheme of Sec. III.B; n_att = ceil(P_tot)
 *     attempts when P_tot > 1;
 *   - rates are fixed-point integers: q(x) = (uint64)(x * 2^32), truncated;
 *   - Philox4x32-10 (Salmon et al., SC'11) with key (lo32(seed),
 *     hi32(seed) ^ lo32(t)) and counter (ket, bra, walker, part<<16 | block);
 *   - shift: S0 until the controlled weight first reaches the target, then
 *     the log update of Sec. III.C every step with a series logarithm.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_MAX_SITES 64
#define OR_MAX_BONDS 128
#define OR_MAX_MOVES (2 * OR_MAX_BONDS + 5 * OR_MAX_SITES)

/* error codes returned by or_step / or_import */
#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_OOM (-2)
#define OR_ERR_OVERFLOW (-4)

typedef struct {
    uint64_t ket, bra;
    int64_t re, im;     /* 64-bit while summing; range-checked against int32 */
} or_entry;

typedef struct {
    uint64_t ket, bra;
    int32_t dre, dim;
    int32_t init;       /* 1 if the parent was an initiator */
} or_spawn;

typedef struct {
    /* lattice and model */
    int Lx, Ly, periodic, N, B;
    int bond_a[OR_MAX_BONDS], bond_b[OR_MAX_BONDS];
    uint64_t bond_m[OR_MAX_BONDS];
    double Jx, Jy, Jz, gamma, dt;
    double h;               /* in-plane field strength (Sec. V.B), 0 = none */
    int field_axis;         /* 0: field along x (theta = 0), 1: along y (theta = pi/2), 2: angle theta */
    double theta;           /* field angle for axis 2 */
    int64_t target;
    int32_t n_a;
    int control;            /* 0: N_w = sum |Re rho_ii| (paper); 1: sum |re|+|im| */
    int guide_kind;         /* 0 none, 1 uniform w = exp(-p), 2 site product */
    double guide_p;
    double site_r[OR_MAX_SITES];
    uint64_t seed;
    double delta, S0;
    int64_t n0;
    int64_t t_eq_override;  /* < 0: derived */
    /* fixed-point rate tables */
    uint64_t rate_q[OR_MAX_BONDS][2][4];   /* [bond][aligned=0/anti=1][ratio class] */
    uint64_t jump_q;
    uint64_t frate_q[OR_MAX_SITES][4];     /* field flip of site k, [ratio class] */
    uint64_t frate_c[OR_MAX_SITES][4];     /* axis 2: the imaginary part, |h cos theta| */
    uint64_t frate_s[OR_MAX_SITES][4];     /* axis 2: the real part, |h sin theta| */
    uint32_t cross_int[2 * OR_MAX_BONDS + 1];
    uint64_t cross_frac[2 * OR_MAX_BONDS + 1];
    double shift_gain;      /* delta / dt */
    /* state */
    or_entry *L;
    int64_t M, capL;
    double S;
    int variable;
    int64_t Qprev;
    int64_t t, t_var, t_eq;
    /* per-step estimator series */
    int nobs;
    int64_t *series;
    int64_t nseries, capseries;
    int64_t last_spawns;    /* child-walker records made in the last step */
    /* uniform injection (hand-worked tests) */
    const uint32_t *inj;
    int64_t ninj, pinj;
    int inj_short;
} or_run;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its definition in Salmon, Moraes, Dror & Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3" (SC'11).                    */
/* ------------------------------------------------------------------------ */
static uint32_t or_mulhi32(uint32_t a, uint32_t b) {
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
}

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint32_t hi0 = or_mulhi32(M0, c0), lo0 = M0 * c0;
        uint32_t hi1 = or_mulhi32(M1, c2), lo1 = M1 * c2;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Deterministic natural logarithm: x = m 2^e with m in (1/sqrt2, sqrt2],     */
/* log m = 2 atanh(s), s = (m-1)/(m+1), atanh by its odd power series.       */
/* Every operation is a single IEEE-754 double operation in a fixed order.   */
/* ------------------------------------------------------------------------ */
double or_series_log(double x) {
    const double LN2 = 0.6931471805599453;      /* nearest double to ln 2 */
    const double SQRT2 = 1.4142135623730951;    /* nearest double to sqrt 2 */
    if (!(x > 0.0)) return 0.0;
    uint64_t bits;
    memcpy(&bits, &x, 8);
    int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) return 0.0;     /* subnormals never occur: inputs are ratios of counts */
    e -= 1023;
    uint64_t mb = (bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    double m;
    memcpy(&m, &mb, 8);
    if (m > SQRT2) { m = m * 0.5; e += 1; }
    double num = m - 1.0;
    double den = m + 1.0;
    double s = num / den;
    double z = s * s;
    /* sum_{k=0}^{14} z^k / (2k+1), Horner from the top term */
    double p = 1.0 / 29.0;
    for (int k = 13; k >= 0; --k) {
        double c = 1.0 / (double)(2 * k + 1);
        double pz = p * z;
        p = pz + c;
    }
    double two_s = 2.0 * s;
    double lm = two_s * p;
    double el = (double)e * LN2;
    return el + lm;
}

/* ------------------------------------------------------------------------ */
/* helpers                                                                   */
/* ------------------------------------------------------------------------ */
static int or_popc(uint64_t x) { int c = 0; while (x) { x &= x - 1; ++c; } return c; }
static int or_bit(uint64_t s, int k) { return (int)((s >> k) & 1u); }
static uint64_t or_q(double x) { return (uint64_t)(x * 4294967296.0); }

/* z-sum of a spin word: sum over bonds of z_a z_b (z = +1 up, -1 down) */
static int or_zsum(const or_run *r, uint64_t s) {
    int acc = 0;
    for (int b = 0; b < r->B; ++b)
        acc += (or_bit(s, r->bond_a[b]) == or_bit(s, r->bond_b[b])) ? 1 : -1;
    return acc;
}

/* off-diagonal element of H between s and s ^ m_b: Jx - Jy if the bond is
 * aligned in s (sy sy gives -1), Jx + Jy if anti-aligned (sy sy gives +1) */
static double or_hb(const or_run *r, uint64_t s, int b) {
    int aligned = or_bit(s, r->bond_a[b]) == or_bit(s, r->bond_b[b]);
    return aligned ? (r->Jx - r->Jy) : (r->Jx + r->Jy);
}

/* ratio class of a bond move applied to configuration (i, j) -- see rate table */
static int or_ratio_class(const or_run *r, uint64_t i, uint64_t j, int b) {
    uint64_t d = i ^ j;
    if (r->guide_kind == 1) {
        if (d == 0) return 1;                 /* diagonal parent -> off-diagonal child */
        if (d == r->bond_m[b]) return 2;      /* off-diagonal parent -> diagonal child */
        return 0;
    }
    if (r->guide_kind == 2)
        return 2 * or_bit(d, r->bond_a[b]) + or_bit(d, r->bond_b[b]);
    return 0;
}

/* ratio class of a site flip of the field at site k applied to (i, j) */
static int or_site_class(const or_run *r, uint64_t i, uint64_t j, int k) {
    uint64_t d = i ^ j;
    if (r->guide_kind == 1) {
        if (d == 0) return 1;                 /* diagonal parent -> off-diagonal child */
        if (d == (1ull << k)) return 2;       /* off-diagonal parent -> diagonal child */
        return 0;
    }
    if (r->guide_kind == 2) return or_bit(d, k);   /* 0: site k starts to differ, 1: stops */
    return 0;
}

/* ------------------------------------------------------------------------ */
/* construction                                                              */
/* ------------------------------------------------------------------------ */
static int or_build_lattice(or_run *r) {
    int Lx = r->Lx, Ly = r->Ly;
    if (Lx < 1 || Ly < 1 || Lx * Ly > OR_MAX_SITES) return OR_ERR_ARG;
    if (r->periodic && (Lx == 2 || Ly == 2)) return OR_ERR_ARG;
    r->N = Lx * Ly;
    int B = 0;
    for (int y = 0; y < Ly; ++y) {
        for (int x = 0; x < Lx; ++x) {
            int a = x + Lx * y;
            if (Lx > 1 && (x + 1 < Lx || r->periodic)) {
                r->bond_a[B] = a; r->bond_b[B] = ((x + 1) % Lx) + Lx * y; ++B;
            }
            if (Ly > 1 && (y + 1 < Ly || r->periodic)) {
                r->bond_a[B] = a; r->bond_b[B] = x + Lx * ((y + 1) % Ly); ++B;
            }
        }
    }
    r->B = B;
    for (int b = 0; b < B; ++b)
        r->bond_m[b] = (1ull << r->bond_a[b]) | (1ull << r->bond_b[b]);
    return OR_OK;
}

/* Fixed-point rate tables.  A bond move has |A| = |h_b| (aligned or
 * anti-aligned), times dt, times the importance-sampling ratio
 * w(child)/w(parent) of Sec. IV.B.  A jump has |A| = gamma and ratio 1
 * (it clears bit k on both sides, so i == j and the differing sites are
 * unchanged). */
static void or_build_rates(or_run *r) {
    double hv[2];
    hv[0] = fabs(r->Jx - r->Jy);
    hv[1] = fabs(r->Jx + r->Jy);
    double w_off = 1.0, w_inv = 1.0;
    if (r->guide_kind == 1) { w_off = exp(-r->guide_p); w_inv = 1.0 / w_off; }
    for (int b = 0; b < r->B; ++b) {
        for (int h = 0; h < 2; ++h) {
            double base = hv[h] * r->dt;
            for (int c = 0; c < 4; ++c) {
                double x = base;
                if (r->guide_kind == 1) {
                    if (c == 1) x = base * w_off;
                    else if (c == 2) x = base * w_inv;
                } else if (r->guide_kind == 2) {
                    double ra = r->site_r[r->bond_a[b]], rb = r->site_r[r->bond_b[b]];
                    double fa = (c & 2) ? (1.0 / ra) : ra;   /* site a differed -> becomes equal */
                    double fb = (c & 1) ? (1.0 / rb) : rb;
                    double ratio = fa * fb;
                    x = base * ratio;
                }
                r->rate_q[b][h][c] = or_q(x);
            }
        }
    }
    r->jump_q = or_q(r->gamma * r->dt);
    /* field site flips: |A| = |h|, times dt, times the ratio of the flipped site;
     * at a general angle the two parts |h cos theta| and |h sin theta| */
    for (int k = 0; k < r->N; ++k) {
        for (int part = 0; part < 3; ++part) {
            double amp = fabs(r->h);
            if (part == 1) amp = fabs(r->h * cos(r->theta));
            if (part == 2) amp = fabs(r->h * sin(r->theta));
            double base = amp * r->dt;
            for (int c = 0; c < 4; ++c) {
                double x = base;
                if (r->guide_kind == 1) {
                    if (c == 1) x = base * w_off;
                    else if (c == 2) x = base * w_inv;
                } else if (r->guide_kind == 2) {
                    if (c == 0) x = base * r->site_r[k];
                    else if (c == 1) x = base * (1.0 / r->site_r[k]);
                }
                if (part == 0) r->frate_q[k][c] = or_q(x);
                else if (part == 1) r->frate_c[k][c] = or_q(x);
                else r->frate_s[k][c] = or_q(x);
            }
        }
    }
    /* on-site cross term: q = dt |Jz| |zsum(i) - zsum(j)| */
    double cbase = r->dt * fabs(r->Jz);
    for (int c = 0; c <= 2 * r->B; ++c) {
        double x = cbase * (double)c;
        double ip = floor(x);
        r->cross_int[c] = (uint32_t)ip;
        r->cross_frac[c] = or_q(x - ip);
    }
    r->shift_gain = r->delta / r->dt;
}

void or_destroy(or_run *r) {
    if (!r) return;
    free(r->L);
    free(r->series);
    free(r);
}

or_run *or_create(int Lx, int Ly, int periodic, double Jx, double Jy, double Jz,
                  double gamma, double dt, int64_t target, int32_t n_a,
                  int guide_kind, double guide_p, const double *site_r,
                  uint64_t seed, double delta, double S0, int64_t n0,
                  int control, int64_t t_eq_override, double h, int field_axis, double theta) {
    or_run *r = (or_run *)calloc(1, sizeof(or_run));
    if (!r) return NULL;
    r->Lx = Lx; r->Ly = Ly; r->periodic = periodic;
    r->Jx = Jx; r->Jy = Jy; r->Jz = Jz; r->gamma = gamma; r->dt = dt;
    r->target = target; r->n_a = n_a; r->control = control;
    r->guide_kind = guide_kind; r->guide_p = guide_p;
    r->seed = seed; r->delta = delta; r->S0 = S0; r->n0 = n0;
    r->t_eq_override = t_eq_override;
    r->h = h;
    r->field_axis = field_axis;
    r->theta = theta;
    if (or_build_lattice(r) != OR_OK || !(dt > 0.0) || gamma < 0.0 || target <= 0 ||
        n_a < 0 || guide_kind < 0 || guide_kind > 2 || n0 < 0 || n0 > 2147483647 ||
        (control != 0 && control != 1) || !isfinite(h) || field_axis < 0 || field_axis > 2 ||
        !isfinite(theta)) {
        free(r);
        return NULL;
    }
    for (int k = 0; k < r->N; ++k) r->site_r[k] = 1.0;
    if (guide_kind == 2) {
        if (!site_r) { free(r); return NULL; }
        for (int k = 0; k < r->N; ++k) {
            if (!(site_r[k] > 0.0 && site_r[k] <= 1.0)) { free(r); return NULL; }
            r->site_r[k] = site_r[k];
        }
    }
    or_build_rates(r);
    r->nobs = 5 + r->N + 3 * r->B + 4 + 2 * r->N + 2;
    r->capL = 1024;
    r->L = (or_entry *)malloc(sizeof(or_entry) * (size_t)r->capL);
    if (!r->L) { free(r); return NULL; }
    /* initial state: n0 real walkers on |down...down><down...down| */
    r->M = 0;
    if (n0 > 0) { r->L[0].ket = 0; r->L[0].bra = 0; r->L[0].re = n0; r->L[0].im = 0; r->M = 1; }
    r->S = S0;
    r->variable = 0;
    r->t = 0;
    r->t_var = -1;
    r->t_eq = -1;
    r->Qprev = (control == 0) ? n0 : n0;   /* both measures equal n0 initially */
    return r;
}

/* ------------------------------------------------------------------------ */
/* draws                                                                     */
/* ------------------------------------------------------------------------ */
static void or_draw_block(or_run *r, uint64_t ket, uint64_t bra, uint32_t w, int part,
                          uint32_t block, uint32_t out[4]) {
    if (r->inj) {
        for (int q = 0; q < 4; ++q) {
            if (r->pinj < r->ninj) out[q] = r->inj[r->pinj++];
            else { out[q] = 0xFFFFFFFFu; r->inj_short = 1; }
        }
        return;
    }
    uint32_t ctr[4], key[2];
    ctr[0] = (uint32_t)ket;          /* N <= 32: the words themselves are unique */
    ctr[1] = (uint32_t)bra;
    if (r->N > 32) {                 /* wider words: fold the high halves in */
        ctr[0] ^= (uint32_t)(ket >> 32) * 0x9E3779B9u;
        ctr[1] ^= (uint32_t)(bra >> 32) * 0x85EBCA6Bu;
    }
    ctr[2] = w;
    ctr[3] = ((uint32_t)part << 16) | block;
    key[0] = (uint32_t)r->seed;
    key[1] = (uint32_t)(r->seed >> 32) ^ (uint32_t)r->t;
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* move enumeration (element rules derived from the Lindblad equation of     */
/* Sec. III.A and its Kronecker form in Sec. III.C)                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t cket, cbra;
    int kind;           /* 0 ket bond flip, 1 bra bond flip, 2 jump */
    double Are, Aim;    /* complex element A = L~[child, parent] */
    uint64_t rate;      /* q(|A| dt w_child / w_parent) */
} or_move;

/* Move order: the ket bond flips, then the bra bond flips, then the jumps.
 * Within each bond-flip segment the moves are grouped by g = 4*anti + class
 * (anti = 1 if the bond is anti-aligned in the flipped word, class = the
 * importance-sampling class of the bond), groups in increasing g, bonds in
 * bond order inside a group; jumps go by site. */
static int or_moves_of(const or_run *r, uint64_t i, uint64_t j, or_move *mv) {
    int K = 0;
    for (int g = 0; g < 8; ++g)                /* -i H rho: child (i ^ m_b, j), A = -i h_b(i) */
        for (int b = 0; b < r->B; ++b) {
            int al = or_bit(i, r->bond_a[b]) != or_bit(i, r->bond_b[b]);
            int cl = or_ratio_class(r, i, j, b);
            if (4 * al + cl != g) continue;
            double h = or_hb(r, i, b);
            mv[K].cket = i ^ r->bond_m[b]; mv[K].cbra = j; mv[K].kind = 0;
            mv[K].Are = 0.0; mv[K].Aim = -h;
            mv[K].rate = r->rate_q[b][al][cl];
            ++K;
        }
    for (int g = 0; g < 8; ++g)                /* +i rho H: child (i, j ^ m_b), A = +i h_b(j) */
        for (int b = 0; b < r->B; ++b) {
            int al = or_bit(j, r->bond_a[b]) != or_bit(j, r->bond_b[b]);
            int cl = or_ratio_class(r, i, j, b);
            if (4 * al + cl != g) continue;
            double h = or_hb(r, j, b);
            mv[K].cket = i; mv[K].cbra = j ^ r->bond_m[b]; mv[K].kind = 1;
            mv[K].Are = 0.0; mv[K].Aim = h;
            mv[K].rate = r->rate_q[b][al][cl];
            ++K;
        }
    if (r->h != 0.0 && r->field_axis == 2) {
        /* H_ext = h sum_k (cos theta sigma^x_k + sin theta sigma^y_k), Sec. V.B.
         * Ket flip: A = -i h (cos theta + i sin theta (2 s - 1))
         *             = -i h cos theta + h sin theta (2 s - 1);
         * bra flip: A = +i h (cos theta - i sin theta (2 s - 1))
         *             = +i h cos theta + h sin theta (2 s - 1)
         * (s the flipped word's bit before the flip).  Each flip is two moves:
         * the imaginary part, then (after all of them) the real part. */
        double hc = r->h * cos(r->theta), hs = r->h * sin(r->theta);
        for (int seg = 0; seg < 2; ++seg)
            for (int part = 0; part < 2; ++part)
                for (int g = 0; g < 4; ++g)
                    for (int k = 0; k < r->N; ++k) {
                        if (or_site_class(r, i, j, k) != g) continue;
                        uint64_t w = seg == 0 ? i : j;
                        mv[K].cket = seg == 0 ? (i ^ (1ull << k)) : i;
                        mv[K].cbra = seg == 0 ? j : (j ^ (1ull << k));
                        mv[K].kind = 3 + seg;
                        if (part == 0) {
                            mv[K].Are = 0.0;
                            mv[K].Aim = seg == 0 ? -hc : hc;
                            mv[K].rate = r->frate_c[k][g];
                        } else {
                            mv[K].Are = hs * (2.0 * (double)or_bit(w, k) - 1.0);
                            mv[K].Aim = 0.0;
                            mv[K].rate = r->frate_s[k][g];
                        }
                        ++K;
                    }
    } else if (r->h != 0.0) {
        /* -i H_ext rho and +i rho H_ext, H_ext = h sum_k sigma^x_k (axis 0) or
         * h sum_k sigma^y_k (axis 1), Sec. V.B: one site flipped in the ket
         * (A = -i <i'|H_ext|i>) or in the bra (A = +i <j|H_ext|j'>).  With
         * <up|sy|down> = -i and <down|sy|up> = +i, both give A = h (2 s_k - 1)
         * for the y axis, s the flipped word before the flip. */
        for (int seg = 0; seg < 2; ++seg)
            for (int g = 0; g < 4; ++g)
                for (int k = 0; k < r->N; ++k) {
                    if (or_site_class(r, i, j, k) != g) continue;
                    uint64_t w = seg == 0 ? i : j;
                    mv[K].cket = seg == 0 ? (i ^ (1ull << k)) : i;
                    mv[K].cbra = seg == 0 ? j : (j ^ (1ull << k));
                    mv[K].kind = 3 + seg;
                    if (r->field_axis == 0) {
                        mv[K].Are = 0.0;
                        mv[K].Aim = seg == 0 ? -r->h : r->h;
                    } else {
                        mv[K].Are = r->h * (2.0 * (double)or_bit(w, k) - 1.0);
                        mv[K].Aim = 0.0;
                    }
                    mv[K].rate = r->frate_q[k][g];
                    ++K;
                }
    }
    for (int k = 0; k < r->N; ++k) {           /* gamma sigma^- rho sigma^+: needs bit k up on both sides */
        int ok = or_bit(i, k) && or_bit(j, k);
        mv[K].cket = i & ~(1ull << k); mv[K].cbra = j & ~(1ull << k); mv[K].kind = 2;
        mv[K].Are = ok ? r->gamma : 0.0; mv[K].Aim = 0.0;
        mv[K].rate = ok ? r->jump_q : 0;
        ++K;
    }
    return K;
}

/* ------------------------------------------------------------------------ */
/* one step                                                                  */
/* ------------------------------------------------------------------------ */
static int or_cmp_key(uint64_t ka, uint64_t ba, uint64_t kb, uint64_t bb) {
    if (ba != bb) return ba < bb ? -1 : 1;
    if (ka != kb) return ka < kb ? -1 : 1;
    return 0;
}

static int or_spawn_cmp(const void *pa, const void *pb) {
    const or_spawn *a = (const or_spawn *)pa, *b = (const or_spawn *)pb;
    return or_cmp_key(a->ket, a->bra, b->ket, b->bra);
}

typedef struct { or_spawn *v; int64_t n, cap; } or_spawn_vec;

static int or_push(or_spawn_vec *sv, uint64_t ket, uint64_t bra, int32_t dre, int32_t dim, int init) {
    if (sv->n == sv->cap) {
        int64_t nc = sv->cap ? 2 * sv->cap : 4096;
        or_spawn *nv = (or_spawn *)realloc(sv->v, sizeof(or_spawn) * (size_t)nc);
        if (!nv) return OR_ERR_OOM;
        sv->v = nv; sv->cap = nc;
    }
    or_spawn *s = &sv->v[sv->n++];
    s->ket = ket; s->bra = bra; s->dre = dre; s->dim = dim; s->init = init;
    return OR_OK;
}

static void or_estimate(or_run *r, int64_t *est);
static int or_series_append(or_run *r, const int64_t *est);

/* Annihilation (Sec. III.C, rule (iii)) with the initiator rule of Sec. IV.A:
 * sort the spawned children by configuration, then walk L (sorted, unique)
 * and the children together; every configuration keeps the sum of its own
 * population and its children, except that children of non-initiator parents
 * count only on configurations occupied in L or on the diagonal (or when
 * n_a = 0, where every parent is an initiator).  Zero sums are dropped.
 * Sorts `sp` in place; *out is malloc'ed. */
static int or_merge_spawns(const or_entry *L, int64_t M, or_spawn *sp, int64_t R, int32_t n_a,
                           or_entry **out_p, int64_t *m_p) {
    if (R > 1) qsort(sp, (size_t)R, sizeof(or_spawn), or_spawn_cmp);
    int64_t cap = M + R + 1;
    or_entry *out = (or_entry *)malloc(sizeof(or_entry) * (size_t)cap);
    if (!out) return OR_ERR_OOM;
    int64_t a = 0, b = 0, m = 0;
    while (a < M || b < R) {
        uint64_t ket, bra;
        if (b >= R || (a < M && or_cmp_key(L[a].ket, L[a].bra, sp[b].ket, sp[b].bra) <= 0)) {
            ket = L[a].ket; bra = L[a].bra;
        } else {
            ket = sp[b].ket; bra = sp[b].bra;
        }
        int occupied = (a < M && L[a].ket == ket && L[a].bra == bra);
        int64_t sre = 0, sim = 0;
        if (occupied) { sre = L[a].re; sim = L[a].im; ++a; }
        int open = occupied || (ket == bra) || (n_a == 0);
        while (b < R && sp[b].ket == ket && sp[b].bra == bra) {
            if (open || sp[b].init) { sre += sp[b].dre; sim += sp[b].dim; }
            ++b;
        }
        if (sre == 0 && sim == 0) continue;
        if (sre > 2147483647LL || sre < -2147483647LL || sim > 2147483647LL || sim < -2147483647LL) {
            free(out);
            return OR_ERR_OVERFLOW;
        }
        out[m].ket = ket; out[m].bra = bra; out[m].re = sre; out[m].im = sim; ++m;
    }
    *out_p = out;
    *m_p = m;
    return OR_OK;
}



/* Death/clone table of the current step: p_c = dt ((gamma/2) c + S) for
 * c = n(i) + n(j); integer part, fixed-point fraction and sign. */
static void or_death_table(const or_run *r, uint32_t *d_int, uint64_t *d_frac, int *d_sgn) {
    double g2 = 0.5 * r->gamma;
    for (int c = 0; c <= 2 * r->N; ++c) {
        double a = g2 * (double)c;
        double b = a + r->S;
        double p = r->dt * b;
        double ap = fabs(p);
        double ip = floor(ap);
        d_int[c] = (uint32_t)ip;
        d_frac[c] = or_q(ap - ip);
        d_sgn[c] = (p > 0.0) ? 1 : ((p < 0.0) ? -1 : 0);
    }
}

/* Where the children of one entry go: all of them into a spawn vector (sv),
 * or, with sv NULL, only the sum of those landing on (want_ket, want_bra). */
typedef struct {
    or_spawn_vec *sv;
    uint64_t want_ket, want_bra;
    int64_t got_re, got_im;
} or_sink;

/* Steps (i) and (ii) for the walkers of one entry (i, j) with populations
 * (re, im): the change of the entry's own populations (death/clone and the
 * on-site transfer) in *dre_p, *dim_p, and its children into the sink. */
static int or_walk_entry(or_run *r, const uint32_t *d_int, const uint64_t *d_frac, const int *d_sgn,
                         uint64_t i, uint64_t j, int64_t re, int64_t im, or_move *mv,
                         int64_t *dre_p, int64_t *dim_p, or_sink *sink) {
    int err = OR_OK;
    int64_t nre = re < 0 ? -re : re, nim = im < 0 ? -im : im;
    int init = (r->n_a == 0) || (i == j) || (nre + nim > (int64_t)r->n_a);
    int K = or_moves_of(r, i, j, mv);
    uint64_t T = 0;
    for (int k = 0; k < K; ++k) T += mv[k].rate;
    uint64_t natt = (T + 0xFFFFFFFFull) >> 32;
    if (natt < 1) natt = 1;
    int cd = or_popc(i) + or_popc(j);
    int dz = or_zsum(r, i) - or_zsum(r, j);
    int adz = dz < 0 ? -dz : dz;
    /* Im part of the diagonal element, d = -(E(i) - E(j)) = -Jz dz */
    int sgn_d = 0;
    if (dz != 0 && r->Jz != 0.0) sgn_d = ((r->Jz > 0.0) == (dz > 0)) ? -1 : 1;
    int64_t dre = 0, dim = 0;
    for (int part = 0; part < 2 && err == OR_OK; ++part) {
        int64_t pop = part == 0 ? re : im;
        int64_t n = pop < 0 ? -pop : pop;
        int sig = pop < 0 ? -1 : 1;
        for (int64_t w = 0; w < n && err == OR_OK; ++w) {
            uint32_t x[4];
            or_draw_block(r, i, j, (uint32_t)w, part, 0, x);
            /* death (p > 0) or cloning (p < 0) on the walker's own part */
            int64_t cnt = (int64_t)d_int[cd] + ((uint64_t)x[1] < d_frac[cd] ? 1 : 0);
            if (part == 0) dre -= (int64_t)d_sgn[cd] * sig * cnt;
            else dim -= (int64_t)d_sgn[cd] * sig * cnt;
            /* on-site transfer from the imaginary part of the diagonal element */
            int64_t cc = (int64_t)r->cross_int[adz] + ((uint64_t)x[2] < r->cross_frac[adz] ? 1 : 0);
            if (part == 0) dim += (int64_t)sig * sgn_d * cc;
            else dre -= (int64_t)sig * sgn_d * cc;
            /* spawning attempts */
            uint32_t xb[4];
            uint32_t cur_block = 0;
            for (uint64_t a = 0; a < natt; ++a) {
                uint32_t u;
                if (a == 0) u = x[0];
                else if (a == 1) u = x[3];
                else {
                    uint32_t blk = 1u + (uint32_t)((a - 2) / 4);
                    if (blk != cur_block) { or_draw_block(r, i, j, (uint32_t)w, part, blk, xb); cur_block = blk; }
                    u = xb[(a - 2) % 4];
                }
                uint64_t v = (uint64_t)u * natt;
                if (v >= T) continue;
                uint64_t cum = 0;
                int k = 0;
                for (; k < K; ++k) { cum += mv[k].rate; if (v < cum) break; }
                /* child type and sign: Delta rho_child = A * rho_parent (Sec. III.C rules) */
                int32_t cre = 0, cim = 0;
                double Ar = mv[k].Are, Ai = mv[k].Aim;
                if (part == 0) {            /* real parent of sign sig */
                    if (Ar != 0.0) cre = sig * (Ar > 0.0 ? 1 : -1);
                    else cim = sig * (Ai > 0.0 ? 1 : -1);
                } else {                    /* imaginary parent i*sig */
                    if (Ar != 0.0) cim = sig * (Ar > 0.0 ? 1 : -1);
                    else cre = -sig * (Ai > 0.0 ? 1 : -1);
                }
                if (sink->sv) {
                    err = or_push(sink->sv, mv[k].cket, mv[k].cbra, cre, cim, init);
                    if (err != OR_OK) break;
                } else if (mv[k].cket == sink->want_ket && mv[k].cbra == sink->want_bra) {
                    sink->got_re += cre;
                    sink->got_im += cim;
                }
            }
        }
    }
    *dre_p = dre;
    *dim_p = dim;
    return err;
}

int or_step(or_run *r, int64_t nsteps) {
    or_move mv[OR_MAX_MOVES];
    for (int64_t it = 0; it < nsteps; ++it) {
        uint32_t d_int[2 * OR_MAX_SITES + 1];
        uint64_t d_frac[2 * OR_MAX_SITES + 1];
        int d_sgn[2 * OR_MAX_SITES + 1];
        or_death_table(r, d_int, d_frac, d_sgn);

        or_spawn_vec sv = {0, 0, 0};
        or_sink sink;
        memset(&sink, 0, sizeof(sink));
        sink.sv = &sv;
        int err = OR_OK;
        /* (i) spawning and (ii) death/clone, all from rho(t) and S(t) (Euler step) */
        for (int64_t e = 0; e < r->M && err == OR_OK; ++e) {
            int64_t dre = 0, dim = 0;
            err = or_walk_entry(r, d_int, d_frac, d_sgn, r->L[e].ket, r->L[e].bra, r->L[e].re, r->L[e].im, mv,
                                &dre, &dim, &sink);
            r->L[e].re += dre;
            r->L[e].im += dim;
        }
        if (err != OR_OK) { free(sv.v); return err; }
        r->last_spawns = sv.n;

        /* (iii) annihilation: sort the spawns, then one linear merge */
        or_entry *out = NULL;
        int64_t m = 0;
        int rc = or_merge_spawns(r->L, r->M, sv.v, sv.n, r->n_a, &out, &m);
        free(sv.v);
        if (rc != OR_OK) return rc;
        free(r->L);
        r->L = out; r->M = m; r->capL = m > 0 ? m : 1;

        /* estimators on rho(t+1), then the shift update of Sec. III.C */
        int64_t est[5 + OR_MAX_SITES + 3 * OR_MAX_BONDS + 4 + 2 * OR_MAX_SITES + 2];
        or_estimate(r, est);
        int64_t Q = (r->control == 0) ? est[2] : est[3];
        if (r->variable) {
            if (Q > 0 && r->Qprev > 0) {
                double ratio = (double)Q / (double)r->Qprev;
                double lg = or_series_log(ratio);
                double inc = r->shift_gain * lg;
                r->S = r->S + inc;
            }
        } else if (Q >= r->target) {
            r->variable = 1;
            r->t_var = r->t + 1;
            if (r->t_eq_override >= 0) r->t_eq = r->t_var + r->t_eq_override;
            else {
                double rate = r->gamma > 0.0 ? r->gamma : 1.0;
                double span = 10.0 / (rate * r->dt);
                r->t_eq = r->t_var + (int64_t)ceil(span);
            }
        }
        r->Qprev = Q;
        r->t += 1;
        if (r->variable && r->t >= r->t_eq) {
            int e2 = or_series_append(r, est);
            if (e2 != OR_OK) return e2;
        }
    }
    return OR_OK;
}

/* Estimator numerators over the current list, all integers (Sec. III.A):
 *   [0] Tr Re rho, [1] Tr Im rho, [2] N_w = sum |Re rho_ii|, [3] W = sum |re|+|im|,
 *   [4] M = occupied configurations,
 *   [5 .. 5+N)        sum_i z_k(i) Re rho_ii            (per-site sigma^z)
 *   [5+N .. +B)       sum_i z_a z_b Re rho_ii           (per-bond zz)
 *   [.. +B)           sum over i^j == m_b of Re rho_ij  (per-bond xx)
 *   [.. +B)           same with -1 if i is aligned on b, +1 if not (per-bond yy)
 *   [.. +4)           sums over sites / bonds of the four blocks above,
 *   [.. +N)           sum over i^j == 2^k of Re rho_ij   (per-site sigma^x)
 *   [.. +N)           same of +Im rho_ij if site k is down in i, -Im if up
 *                     (per-site sigma^y)
 *   [.. +2)           sums over sites of the two blocks above.
 * Importance weights divide the xx/yy/x/y numerators afterwards (Sec. IV.B).
 * Without a field every move flips an even number of spins, so the sigma^x
 * and sigma^y blocks stay zero. */
static void or_estimate(or_run *r, int64_t *est) {
    int N = r->N, B = r->B;
    int nobs = r->nobs;
    for (int k = 0; k < nobs; ++k) est[k] = 0;
    int oz = 5, ozz = 5 + N, oxx = 5 + N + B, oyy = 5 + N + 2 * B, oag = 5 + N + 3 * B;
    int ox = oag + 4, oy = ox + N, ofa = oy + N;
    for (int64_t e = 0; e < r->M; ++e) {
        uint64_t i = r->L[e].ket, j = r->L[e].bra;
        int64_t re = r->L[e].re, im = r->L[e].im;
        est[3] += (re < 0 ? -re : re) + (im < 0 ? -im : im);
        est[4] += 1;
        if (i == j) {
            est[0] += re;
            est[1] += im;
            est[2] += re < 0 ? -re : re;
            for (int k = 0; k < N; ++k) est[oz + k] += or_bit(i, k) ? re : -re;
            for (int b = 0; b < B; ++b)
                est[ozz + b] += (or_bit(i, r->bond_a[b]) == or_bit(i, r->bond_b[b])) ? re : -re;
        } else {
            uint64_t d = i ^ j;
            if (or_popc(d) == 1) {
                /* sigma^x_k: O_ji = 1; sigma^y_k: O_ji = -i if site k is down in i, +i if up */
                int k = 0;
                while (!((d >> k) & 1ull)) ++k;
                est[ox + k] += re;
                est[oy + k] += or_bit(i, k) ? -im : im;
            }
            if (or_popc(d) == 2) {
                for (int b = 0; b < B; ++b) {
                    if (r->bond_m[b] != d) continue;
                    est[oxx + b] += re;
                    int aligned = or_bit(i, r->bond_a[b]) == or_bit(i, r->bond_b[b]);
                    est[oyy + b] += aligned ? -re : re;
                }
            }
        }
    }
    for (int k = 0; k < N; ++k) est[oag + 0] += est[oz + k];
    for (int k = 0; k < N; ++k) {
        est[ofa + 0] += est[ox + k];
        est[ofa + 1] += est[oy + k];
    }
    for (int b = 0; b < B; ++b) {
        est[oag + 1] += est[ozz + b];
        est[oag + 2] += est[oxx + b];
        est[oag + 3] += est[oyy + b];
    }
}

static int or_series_append(or_run *r, const int64_t *est) {
    if (r->nseries == r->capseries) {
        int64_t nc = r->capseries ? 2 * r->capseries : 1024;
        int64_t *ns = (int64_t *)realloc(r->series, sizeof(int64_t) * (size_t)(nc * r->nobs));
        if (!ns) return OR_ERR_OOM;
        r->series = ns; r->capseries = nc;
    }
    memcpy(r->series + r->nseries * r->nobs, est, sizeof(int64_t) * (size_t)r->nobs);
    r->nseries += 1;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* accessors for the tests                                                   */
/* ------------------------------------------------------------------------ */
int or_nobs(const or_run *r) { return r->nobs; }
int or_nsites(const or_run *r) { return r->N; }
int or_nbonds(const or_run *r) { return r->B; }
int64_t or_size(const or_run *r) { return r->M; }
int64_t or_last_spawns(const or_run *r) { return r->last_spawns; }

void or_bonds(const or_run *r, int32_t *a, int32_t *b) {
    for (int k = 0; k < r->B; ++k) { a[k] = r->bond_a[k]; b[k] = r->bond_b[k]; }
}

/* scalar state: t, S, variable, Qprev, t_var, t_eq */
void or_get_state(const or_run *r, int64_t *t, double *S, int32_t *variable, int64_t *Qprev,
                  int64_t *t_var, int64_t *t_eq) {
    *t = r->t; *S = r->S; *variable = r->variable; *Qprev = r->Qprev; *t_var = r->t_var; *t_eq = r->t_eq;
}

void or_set_state(or_run *r, int64_t t, double S, int32_t variable, int64_t Qprev,
                  int64_t t_var, int64_t t_eq) {
    r->t = t; r->S = S; r->variable = variable; r->Qprev = Qprev; r->t_var = t_var; r->t_eq = t_eq;
}

int64_t or_export(const or_run *r, uint64_t *ket, uint64_t *bra, int32_t *re, int32_t *im, int64_t cap) {
    int64_t n = r->M < cap ? r->M : cap;
    for (int64_t e = 0; e < n; ++e) {
        ket[e] = r->L[e].ket; bra[e] = r->L[e].bra;
        re[e] = (int32_t)r->L[e].re; im[e] = (int32_t)r->L[e].im;
    }
    return r->M;
}

/* Replace the walker list; entries must be sorted by (bra, ket), unique and non-zero. */
int or_import(or_run *r, const uint64_t *ket, const uint64_t *bra, const int32_t *re,
              const int32_t *im, int64_t n) {
    for (int64_t e = 0; e < n; ++e) {
        if (re[e] == 0 && im[e] == 0) return OR_ERR_ARG;
        if (e > 0 && or_cmp_key(ket[e - 1], bra[e - 1], ket[e], bra[e]) >= 0) return OR_ERR_ARG;
        if (r->N < 64 && ((ket[e] >> r->N) || (bra[e] >> r->N))) return OR_ERR_ARG;
    }
    or_entry *L = (or_entry *)malloc(sizeof(or_entry) * (size_t)(n > 0 ? n : 1));
    if (!L) return OR_ERR_OOM;
    for (int64_t e = 0; e < n; ++e) { L[e].ket = ket[e]; L[e].bra = bra[e]; L[e].re = re[e]; L[e].im = im[e]; }
    free(r->L);
    r->L = L; r->M = n; r->capL = n > 0 ? n : 1;
    return OR_OK;
}

void or_estimates_now(or_run *r, int64_t *est) { or_estimate(r, est); }

int64_t or_series(const or_run *r, int64_t *out, int64_t cap_rows) {
    int64_t n = r->nseries < cap_rows ? r->nseries : cap_rows;
    if (out && n > 0) memcpy(out, r->series, sizeof(int64_t) * (size_t)(n * r->nobs));
    return r->nseries;
}

/* All moves of configuration (i, j) in move order, with the complex element
 * A = L~[child, parent] and the fixed-point rate.  Returns the move count. */
int or_moves(const or_run *r, uint64_t i, uint64_t j, uint64_t *cket, uint64_t *cbra,
             int32_t *kind, double *Are, double *Aim, uint64_t *rate) {
    or_move mv[OR_MAX_MOVES];
    int K = or_moves_of(r, i, j, mv);
    for (int k = 0; k < K; ++k) {
        cket[k] = mv[k].cket; cbra[k] = mv[k].cbra; kind[k] = mv[k].kind;
        Are[k] = mv[k].Are; Aim[k] = mv[k].Aim; rate[k] = mv[k].rate;
    }
    return K;
}

/* Diagonal element of the shifted Liouvillian at (i, j):
 * -(gamma/2)(n(i)+n(j)) - S - i (E(i) - E(j)),  E(s) = Jz zsum(s). */
void or_diag(const or_run *r, uint64_t i, uint64_t j, double *Dre, double *Dim) {
    double g2 = 0.5 * r->gamma;
    *Dre = -(g2 * (double)(or_popc(i) + or_popc(j))) - r->S;
    *Dim = -(r->Jz * (double)(or_zsum(r, i) - or_zsum(r, j)));
}

/* Inject a uniform stream: each Philox block draw takes the next four words
 * instead (in the order the step makes its draws).  NULL restores Philox.
 * Returns 1 if the last step ran past the end of the stream. */
int or_inject(or_run *r, const uint32_t *u, int64_t n) {
    int short_ = r->inj_short;
    r->inj = u; r->ninj = n; r->pinj = 0; r->inj_short = 0;
    return short_;
}
int64_t or_injected_used(const or_run *r) { return r->pinj; }

/* Standalone annihilation of arrays: list (m entries, sorted by (bra, ket),
 * unique) and spawn records (r entries, any order; init = parent initiator
 * flag).  Writes up to cap merged entries; returns the merged length, or a
 * negative error code. */
int64_t or_annihilate(const uint64_t *lket, const uint64_t *lbra, const int32_t *lre, const int32_t *lim,
                      int64_t m, const uint64_t *sket, const uint64_t *sbra, const int32_t *sre,
                      const int32_t *sim, const int32_t *sinit, int64_t r, int32_t n_a,
                      uint64_t *oket, uint64_t *obra, int32_t *ore, int32_t *oim, int64_t cap) {
    or_entry *L = (or_entry *)malloc(sizeof(or_entry) * (size_t)(m > 0 ? m : 1));
    or_spawn *sp = (or_spawn *)malloc(sizeof(or_spawn) * (size_t)(r > 0 ? r : 1));
    if (!L || !sp) { free(L); free(sp); return OR_ERR_OOM; }
    for (int64_t q = 0; q < m; ++q) { L[q].ket = lket[q]; L[q].bra = lbra[q]; L[q].re = lre[q]; L[q].im = lim[q]; }
    for (int64_t q = 0; q < r; ++q) {
        sp[q].ket = sket[q]; sp[q].bra = sbra[q]; sp[q].dre = sre[q]; sp[q].dim = sim[q]; sp[q].init = sinit[q] != 0;
    }
    or_entry *out = NULL;
    int64_t mo = 0;
    int rc = or_merge_spawns(L, m, sp, r, n_a, &out, &mo);
    free(L);
    free(sp);
    if (rc != OR_OK) return rc;
    for (int64_t q = 0; q < mo && q < cap; ++q) {
        oket[q] = out[q].ket; obra[q] = out[q].bra; ore[q] = (int32_t)out[q].re; oim[q] = (int32_t)out[q].im;
    }
    free(out);
    return mo;
}

/* The step of or_step evaluated at chosen configurations only ("gathered"):
 * for each target c = (tket[q], tbra[q]), its own walkers' death/clone and
 * on-site transfer (if c is occupied), plus every child that a walker of an
 * occupied parent sends to c -- the parents that can reach c are c with one
 * bond flipped in the ket or in the bra, and c with one site raised in both
 * words (the reverse of a jump) -- summed under the initiator rule of
 * Sec. IV.A.  Same draws, rates and rules as or_step, so the result equals
 * the entry of c in the stepped list (0, 0 when c is absent from it).
 * L_t: m entries sorted by (bra, ket), unique.  The run supplies the lattice,
 * the rate tables, t and S (its own list is not used). */
static int64_t or_find(const uint64_t *lket, const uint64_t *lbra, int64_t m, uint64_t ket, uint64_t bra) {
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (or_cmp_key(lket[mid], lbra[mid], ket, bra) < 0) lo = mid + 1;
        else hi = mid;
    }
    return (lo < m && lket[lo] == ket && lbra[lo] == bra) ? lo : -1;
}

int or_gather(or_run *r, const uint64_t *lket, const uint64_t *lbra, const int32_t *lre, const int32_t *lim,
              int64_t m, const uint64_t *tket, const uint64_t *tbra, int64_t nt, int64_t *out_re, int64_t *out_im) {
    if (r->inj) return OR_ERR_ARG;        /* an injected stream is consumed in list order */
    or_move mv[OR_MAX_MOVES];
    uint32_t d_int[2 * OR_MAX_SITES + 1];
    uint64_t d_frac[2 * OR_MAX_SITES + 1];
    int d_sgn[2 * OR_MAX_SITES + 1];
    or_death_table(r, d_int, d_frac, d_sgn);
    uint64_t wmask = (r->N >= 64) ? ~0ull : ((1ull << r->N) - 1ull);
    for (int64_t q = 0; q < nt; ++q) {
        uint64_t ci = tket[q], cj = tbra[q];
        int64_t own_re = 0, own_im = 0, fre = 0, fim = 0, ure = 0, uim = 0;
        int64_t e = or_find(lket, lbra, m, ci, cj);
        or_sink sink;
        memset(&sink, 0, sizeof(sink));
        sink.want_ket = ci;
        sink.want_bra = cj;
        if (e >= 0) {
            int64_t dre = 0, dim = 0;
            or_walk_entry(r, d_int, d_frac, d_sgn, ci, cj, lre[e], lim[e], mv, &dre, &dim, &sink);
            own_re = (int64_t)lre[e] + dre;
            own_im = (int64_t)lim[e] + dim;
        }
        /* candidate parents: 2B bond flips, up to N raised sites, and with a
         * field 2N single-site flips */
        int ncand = 2 * r->B + r->N + (r->h != 0.0 ? 2 * r->N : 0);
        for (int c = 0; c < ncand; ++c) {
            uint64_t pi = ci, pj = cj;
            if (c < r->B) pi ^= r->bond_m[c];
            else if (c < 2 * r->B) pj ^= r->bond_m[c - r->B];
            else if (c >= 2 * r->B + r->N) {
                int k = c - 2 * r->B - r->N;
                if (k < r->N) pi ^= 1ull << k;
                else pj ^= 1ull << (k - r->N);
            } else {
                int k = c - 2 * r->B;
                if (or_bit(ci, k) || or_bit(cj, k)) continue;
                pi |= 1ull << k;
                pj |= 1ull << k;
            }
            pi &= wmask;
            pj &= wmask;
            int64_t pe = or_find(lket, lbra, m, pi, pj);
            if (pe < 0) continue;
            int64_t pre = lre[pe], pim = lim[pe];
            int64_t npop = (pre < 0 ? -pre : pre) + (pim < 0 ? -pim : pim);
            int init = (r->n_a == 0) || (pi == pj) || (npop > (int64_t)r->n_a);
            int64_t dre = 0, dim = 0;
            sink.got_re = 0;
            sink.got_im = 0;
            or_walk_entry(r, d_int, d_frac, d_sgn, pi, pj, pre, pim, mv, &dre, &dim, &sink);
            if (init) { fre += sink.got_re; fim += sink.got_im; }
            else { ure += sink.got_re; uim += sink.got_im; }
        }
        int open = (e >= 0) || (ci == cj) || (r->n_a == 0);
        out_re[q] = own_re + fre + (open ? ure : 0);
        out_im[q] = own_im + fim + (open ? uim : 0);
    }
    return OR_OK;
}
