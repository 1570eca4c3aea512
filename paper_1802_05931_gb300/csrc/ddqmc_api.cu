// libddqmc.so: the C-ABI of the DDQMC GPU path (declared in include/ddqmc.h).
//
// One step (Sec. III.C) is five kinds of launch on the run's stream, none of
// which needs a host round trip: spawn + death/clone, npass onesweep radix
// passes, merge-path partition, merge + annihilation + estimators, finalize
// (shift update, blocking, resets).  Every size a kernel needs is read from
// the device-resident DevState.  A batch of runs (ddqmc_create_batch) issues
// the same launches once per step for all its runs, with the batch
// instantiations of the kernels and one finalize block per run.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <nvtx3/nvToolsExt.h>
#include <vector>

#include "../../include/ddqmc.h"
#include "common.cuh"
#include "finalize.cuh"
#include "hashorder.cuh"
#include "merge.cuh"
#include "radix.cuh"
#include "spawn.cuh"
#include "transfer.cuh"

using namespace ddq;

struct ddqmc_run {
    RunParams hp;
    RunParams *dP = nullptr;
    DevState *dS = nullptr;
    BlkCell *dBlk = nullptr;
    void *L[2] = {nullptr, nullptr};     // walker lists: Rec (N <= 31) or RecW records
    void *Sp[2] = {nullptr, nullptr};    // spawn records (radix ping-pong)
    uint64_t *lb_radix = nullptr;
    uint64_t *lb_merge = nullptr;
    int64_t *splits = nullptr;
    int64_t *rem_end = nullptr;
    void *slots = nullptr;               // the merge's per-tile output slots (list records)
    uint32_t *tile_counts = nullptr;     // entries in each slot
    int64_t mcap = 0, rcap = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int cur = 0;                 // which L buffer holds the current list
    int g_spawn = 0, g_radix = 0, g_part = 0, g_merge = 0, g_scan = 0, g_copy = 0;
    // launch shapes: SMs the grids are sized for, the most blocks per SM each
    // persistent kernel can hold (radix: per tile size of packed records),
    // and the shapes in use (defaults, a cached tuning, or ddqmc_tune's)
    int sms = 1;
    int occ_spawn = 1, occ_radix[3] = {1, 1, 1}, occ_merge = 1, occ_copy = 1, occ_scan = 1;
    ddqmc_tuning tune;
    size_t blk_cells = 0;        // blocking cells held in dBlk
    int g_radix_wide = 0;        // radix grid of 16-byte records (standalone annihilation)
    int g_merge_ann = 0;         // merge grid of 16-byte records (standalone annihilation)
    int g_copy_ann = 0;          // compaction copy grid of 16-byte records (standalone annihilation)
    bool packed = false;         // 8-byte spawn records (2N <= 32) on the step path
    bool wide = false;           // two-word keys (N > 31): RecW lists and spawn records
    bool p40 = false;            // 8-byte spawn records of 33- to 40-bit keys (P40) on the step path
    int guide_kind = 0;
    double w_bond[MAXB];         // importance weight of a configuration differing on bond b only
    double w_site[MAXN];         // importance weight of a configuration differing on site k only
    int host_status = 0;         // sticky host-visible status
    // optional per-kernel timing (CUDA events on the run's stream)
    bool timing = false;
    std::vector<cudaEvent_t> ev;     // 2 * NKCLASS events per step
    double kernel_ms[8] = {0};
    int64_t kernel_launches[8] = {0};
    // device arrays of the caller's layout for import / export (ket, bra
    // words, re, im), allocated on first use; small device scratch
    unsigned char *soa = nullptr;
    int64_t soa_cap = 0;         // entries
    unsigned long long *dxfer = nullptr;   // [0] walkers, [1] bad entry, [2..3] run bounds
    // counters of standalone annihilation calls (allocated on first use)
    DevState *dAnn = nullptr;
    uint32_t ann_calls = 0;
    // CUDA graphs of GRAPH_STEPS steps, one per starting list buffer, captured on first use
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool no_graph = false;       // capture failed once: plain launches from then on
    // a batch of runs in one walker store (nruns > 0): hp holds the shared
    // geometry and key layout, hpr / dPr each run's parameters, dRS each
    // run's state (dS then holds the shared step counters)
    int nruns = 0;
    std::vector<RunParams> hpr;
    RunParams *dPr = nullptr;
    DevState *dRS = nullptr;
    size_t mg_smem = 0;          // dynamic shared memory of the merge launch
    // hashed order of two-word keys: positions of out-of-order neighbours
    // found after the digit passes (HO_MAXV), grids of the check and repair
    int64_t *hviol = nullptr;
    int g_hcheck = 0, g_hrepair = 0;
};

namespace {

// 16-byte records are moved with 16-byte vector accesses and bulk copies:
// every record pointer a caller passes must be 16-byte aligned.
bool records_aligned(const void *a, const void *b, const void *c) {
    return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15u) == 0u;
}

int status_code(uint32_t st) {
    if (st & ST_TIMEOUT) return DDQMC_ERR_TIMEOUT;
    if (st & ST_OVERFLOW) return DDQMC_ERR_OVERFLOW;
    if (st & ST_CAPACITY) return DDQMC_ERR_CAPACITY;
    return DDQMC_OK;
}

uint64_t fixed_rate(double x) { return (uint64_t)(x * 4294967296.0); }

// Host-side death table for the shift S (same operation order as the device's).
void host_death_table(const RunParams &P, double S, DevState &st) {
    for (int c = 0; c <= 2 * P.N; ++c) {
        const double a = P.gamma_half * (double)c;
        const double b = a + S;
        const double p = P.dt * b;
        const double ap = std::fabs(p);
        const double ip = std::floor(ap);
        st.d_int[c] = (uint32_t)ip;
        st.d_frac[c] = (uint64_t)((ap - ip) * 4294967296.0);
        st.d_sgn[c] = p > 0.0 ? 1 : (p < 0.0 ? -1 : 0);
    }
}

// Parameters of one run into P; the guide's weights into r.
int build_params(ddqmc_run *r, RunParams &P, const ddqmc_lattice *lat, double Jx, double Jy, double Jz,
                 double gamma, double dt, int64_t target, int32_t n_a, const ddqmc_guide *guide,
                 const ddqmc_options &o) {
    std::memset(&P, 0, sizeof(P));
    P.active = 1;
    const int Lx = lat->Lx, Ly = lat->Ly, per = lat->periodic ? 1 : 0;
    if (Lx < 1 || Ly < 1 || (int64_t)Lx * Ly > 64) return DDQMC_ERR_INVALID_ARG;
    if (per && (Lx == 2 || Ly == 2)) return DDQMC_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !(gamma >= 0.0) || target <= 0 || n_a < 0) return DDQMC_ERR_INVALID_ARG;
    if (!std::isfinite(Jx) || !std::isfinite(Jy) || !std::isfinite(Jz) || !std::isfinite(gamma) || !std::isfinite(dt))
        return DDQMC_ERR_INVALID_ARG;
    if (o.n0 < 0 || o.n0 > 2147483647ll || (o.control != 0 && o.control != 1)) return DDQMC_ERR_INVALID_ARG;
    if (!std::isfinite(o.field_h) || o.field_axis < 0 || o.field_axis > 2 || !std::isfinite(o.field_theta))
        return DDQMC_ERR_INVALID_ARG;
    if (o.wide_sort_bits < -1 || o.wide_sort_bits > 64) return DDQMC_ERR_INVALID_ARG;
    const int N = Lx * Ly;
    if (N > MAXN) return DDQMC_ERR_UNSUPPORTED;
    P.N = N;
    int B = 0;
    // bonds: for each site in (y, x) order, the bond to the right, then the bond below
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            const int a = x + Lx * y;
            if (Lx > 1 && (x + 1 < Lx || per)) { P.bond_a[B] = a; P.bond_b[B] = (x + 1) % Lx + Lx * y; ++B; }
            if (Ly > 1 && (y + 1 < Ly || per)) { P.bond_a[B] = a; P.bond_b[B] = x + Lx * ((y + 1) % Ly); ++B; }
        }
    P.B = B;
    P.field_on = o.field_h != 0.0 ? 1 : 0;
    P.field_axis = o.field_axis;
    // amplitudes of the field's parts: h (axes 0, 1); h cos t and h sin t (axis 2)
    const double hx = o.field_axis == 2 ? o.field_h * std::cos(o.field_theta) : o.field_h;
    const double hy = o.field_axis == 2 ? o.field_h * std::sin(o.field_theta) : 0.0;
    P.sgn_hf = hx > 0.0 ? 1 : (hx < 0.0 ? -1 : 0);
    P.sgn_hf2 = hy > 0.0 ? 1 : (hy < 0.0 ? -1 : 0);
    P.K = 2 * B + N + (P.field_on ? (P.field_axis == 2 ? 4 * N : 2 * N) : 0);
    // the warp-cooperative path's move table
    if (P.K > (N > NPACK ? MAXK : MAXK_PACK)) return DDQMC_ERR_UNSUPPORTED;
    P.nobs = 5 + N + 3 * B + 4 + 2 * N + 2;
    if (N <= NPACK) {
        P.npass = (2 * N + 7) / 8;                 // digits of the packed key bra << N | ket
        for (int p = 0; p < P.npass; ++p) P.pass_shift[p] = 8 * p;
    } else if (o.wide_sort_bits >= 0) {
        // hashed order: digits of the stored bra word bra ^ (hash of ket), whose
        // low wide_sort_bits bits carry the hash; equal stored words are put
        // in ket order after the passes
        const int hb = o.wide_sort_bits;
        P.hashed = 1;
        P.hash_mask = hb >= 64 ? ~0ull : (1ull << hb) - 1ull;
        P.npass = ((hb > N ? hb : N) + 7) / 8;
        for (int p = 0; p < P.npass; ++p) P.pass_shift[p] = 64 + 8 * p;
    } else {
        const int nb = (N + 7) / 8;                // digits of the ket word, then of the bra word
        P.npass = 2 * nb;
        for (int p = 0; p < P.npass; ++p) P.pass_shift[p] = p < nb ? 8 * p : 64 + 8 * (p - nb);
    }
    P.n_a = n_a;
    P.control = o.control;
    P.nmask = N >= 64 ? ~0ull : (1ull << N) - 1ull;
    P.seed = o.seed;
    P.target = target;
    const double span_rate = gamma > 0.0 ? gamma : 1.0;
    P.t_eq_span = o.t_eq >= 0 ? o.t_eq : (int64_t)std::ceil(10.0 / (span_rate * dt));
    P.gamma_half = 0.5 * gamma;
    P.dt = dt;
    P.shift_gain = o.damping / dt;
    P.sgn_h[0] = (Jx - Jy) > 0.0 ? 1 : ((Jx - Jy) < 0.0 ? -1 : 0);
    P.sgn_h[1] = (Jx + Jy) > 0.0 ? 1 : ((Jx + Jy) < 0.0 ? -1 : 0);
    P.sgn_jz = Jz > 0.0 ? 1 : (Jz < 0.0 ? -1 : 0);
    for (int q = 0; q < N * N; ++q) P.pair_bond[q] = -1;
    for (int b = 0; b < B; ++b) {
        P.bond_m[b] = (1ull << P.bond_a[b]) | (1ull << P.bond_b[b]);
        const int lo = P.bond_a[b] < P.bond_b[b] ? P.bond_a[b] : P.bond_b[b];
        const int hi = P.bond_a[b] < P.bond_b[b] ? P.bond_b[b] : P.bond_a[b];
        P.pair_bond[lo * N + hi] = (int8_t)b;
    }
    // importance sampling (Sec. IV.B)
    int gk = guide ? guide->kind : 0;
    if (gk < 0 || gk > 2) return DDQMC_ERR_INVALID_ARG;
    double site_r[MAXN];
    for (int k = 0; k < N; ++k) site_r[k] = 1.0;
    double w_off = 1.0, w_inv = 1.0;
    if (gk == 1) {
        if (!std::isfinite(guide->p)) return DDQMC_ERR_INVALID_ARG;
        w_off = std::exp(-guide->p);
        w_inv = 1.0 / w_off;
    }
    if (gk == 2) {
        if (!guide->site_ratio) return DDQMC_ERR_INVALID_ARG;
        for (int k = 0; k < N; ++k) {
            const double v = guide->site_ratio[k];
            if (!(v > 0.0 && v <= 1.0)) return DDQMC_ERR_INVALID_ARG;
            site_r[k] = v;
        }
    }
    P.guide_kind = gk;
    r->guide_kind = gk;
    const double hval[2] = {std::fabs(Jx - Jy), std::fabs(Jx + Jy)};
    for (int k = 0; k < N; ++k) r->w_site[k] = gk == 1 ? w_off : (gk == 2 ? site_r[k] : 1.0);
    for (int b = 0; b < B; ++b) {
        r->w_bond[b] = gk == 1 ? w_off : (gk == 2 ? site_r[P.bond_a[b]] * site_r[P.bond_b[b]] : 1.0);
        for (int h = 0; h < 2; ++h) {
            const double base = hval[h] * dt;
            for (int c = 0; c < 4; ++c) {
                double x = base;
                if (gk == 1) {
                    if (c == 1) x = base * w_off;
                    else if (c == 2) x = base * w_inv;
                } else if (gk == 2) {
                    const double ra = site_r[P.bond_a[b]], rb = site_r[P.bond_b[b]];
                    const double fa = (c & 2) ? (1.0 / ra) : ra;
                    const double fb = (c & 1) ? (1.0 / rb) : rb;
                    const double ratio = fa * fb;
                    x = base * ratio;
                }
                P.rate_q[b][h][c] = fixed_rate(x);
            }
        }
    }
    P.jump_q = fixed_rate(gamma * dt);
    // field site flips: |A| times dt times the ratio of the flipped site;
    // |A| = |h| along an axis, |h cos t| and |h sin t| for the two parts at an angle
    auto field_rates = [&](double amp, uint64_t (*q)[4]) {
        for (int k = 0; k < N; ++k) {
            const double base = amp * dt;
            for (int c = 0; c < 4; ++c) {
                double x = base;
                if (gk == 1) {
                    if (c == 1) x = base * w_off;
                    else if (c == 2) x = base * w_inv;
                } else if (gk == 2) {
                    if (c == 0) x = base * site_r[k];
                    else if (c == 1) x = base * (1.0 / site_r[k]);
                }
                q[k][c] = fixed_rate(x);
            }
        }
    };
    field_rates(o.field_axis == 2 ? std::fabs(o.field_h * std::cos(o.field_theta)) : std::fabs(o.field_h), P.frate_q);
    if (o.field_axis == 2) field_rates(std::fabs(o.field_h * std::sin(o.field_theta)), P.frate_q2);
    // geometry masks and the bond-uniform rate table of the popcount formulation
    P.Lx = Lx;
    P.shD = Lx * (Ly - 1);
    for (int k = 0; k < N; ++k) {
        const int x = k % Lx, y = k / Lx;
        P.rn[k] = (int8_t)((x + 1) % Lx + Lx * y);
        P.dn[k] = (int8_t)(x + Lx * ((y + 1) % Ly));
    }
    // site and bond masks of the popcount formulation (light path)
    for (int k = 0; k < N; ++k) {
        const int x = k % Lx, y = k / Lx;
        if (Lx > 1 && (x + 1 < Lx || per)) P.ER |= 1ull << k;
        if (Ly > 1 && (y + 1 < Ly || per)) P.ED |= 1ull << k;
        if (x == Lx - 1) P.LC |= 1ull << k;
        if (y == Ly - 1) P.LR |= 1ull << k;
    }
    for (int k = 0; k < N; ++k) {
        uint64_t &E = k < 32 ? P.Emorton : P.Emorton_hi;
        const int kk = k & 31;
        if (P.ER >> k & 1ull) E |= 1ull << (2 * kk);
        if (P.ED >> k & 1ull) E |= 1ull << (2 * kk + 1);
    }
    bool uni = true;
    for (int b = 1; b < B; ++b)
        for (int h = 0; h < 2; ++h)
            for (int c = 0; c < 4; ++c) uni = uni && P.rate_q[b][h][c] == P.rate_q[0][h][c];
    for (int k = 1; k < N; ++k)
        for (int c = 0; c < 4; ++c)
            uni = uni && P.frate_q[k][c] == P.frate_q[0][c] && P.frate_q2[k][c] == P.frate_q2[0][c];
    P.uniform = uni ? 1 : 0;
    for (int g = 0; g < 8; ++g) {
        P.urate8[g] = P.rate_q[0][g >> 2][g & 3];
        P.urate32[g] = (uint32_t)P.urate8[g];
        P.uinv[g] = P.urate8[g] ? 1.0f / (float)P.urate8[g] : 0.0f;
    }
    for (int c = 0; c < 4; ++c) {
        P.ufrate[c] = P.frate_q[0][c];
        P.ufrate32[c] = (uint32_t)P.ufrate[c];
        P.ufinv[c] = P.ufrate[c] ? 1.0f / (float)P.ufrate[c] : 0.0f;
        P.ufrate2[c] = P.frate_q2[0][c];
        P.ufrate32_2[c] = (uint32_t)P.ufrate2[c];
        P.ufinv2[c] = P.ufrate2[c] ? 1.0f / (float)P.ufrate2[c] : 0.0f;
    }
    P.jinv = P.jump_q ? 1.0f / (float)P.jump_q : 0.0f;
    const double cbase = dt * std::fabs(Jz);
    for (int c = 0; c <= 2 * B; ++c) {
        const double x = cbase * (double)c;
        const double ip = std::floor(x);
        P.cross_int[c] = (uint32_t)ip;
        P.cross_frac[c] = fixed_rate(x - ip);
    }
    return DDQMC_OK;
}

template <typename T>
int dalloc(T **p, size_t n) {
    if (n == 0) n = 1;
    if (cudaMalloc((void **)p, n * sizeof(T)) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return DDQMC_ERR_OOM;
    }
    return DDQMC_OK;
}

int dalloc_bytes(void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return DDQMC_ERR_OOM;
    }
    return DDQMC_OK;
}

int occupancy(const void *fn, int tpb, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, tpb, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm;
}

int occupancy_grid(const void *fn, int tpb, size_t smem, int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, tpb, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * sms;
}

void free_run(ddqmc_run *r) {
    if (!r) return;
    for (cudaEvent_t e : r->ev) cudaEventDestroy(e);
    for (cudaGraphExec_t g : r->graph)
        if (g) cudaGraphExecDestroy(g);
    cudaFree(r->soa);
    cudaFree(r->dxfer);
    cudaFree(r->dP);
    cudaFree(r->dS);
    cudaFree(r->dPr);
    cudaFree(r->dRS);
    cudaFree(r->dBlk);
    cudaFree(r->L[0]);
    cudaFree(r->L[1]);
    cudaFree(r->Sp[0]);
    cudaFree(r->Sp[1]);
    cudaFree(r->lb_radix);
    cudaFree(r->lb_merge);
    cudaFree(r->splits);
    cudaFree(r->rem_end);
    cudaFree(r->slots);
    cudaFree(r->tile_counts);
    cudaFree(r->dAnn);
    cudaFree(r->hviol);
    if (r->own_stream && r->stream) cudaStreamDestroy(r->stream);
    delete r;
}

int read_status(ddqmc_run *r) {
    if (r->host_status) return r->host_status;
    uint32_t st = 0;
    if (cudaMemcpyAsync(&st, &r->dS->status, sizeof(st), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        r->host_status = DDQMC_ERR_CUDA;
        return r->host_status;
    }
    r->host_status = status_code(st);
    return r->host_status;
}

// Device arrays of the caller's layout for n entries (24 bytes each), grown
// on demand; nullptr when the allocation fails.
unsigned char *soa_scratch(ddqmc_run *r, int64_t n) {
    if (!r->dxfer && dalloc(&r->dxfer, 4) != DDQMC_OK) return nullptr;
    if (n <= r->soa_cap && r->soa) return r->soa;
    cudaFree(r->soa);
    r->soa = nullptr;
    r->soa_cap = 0;
    const int64_t cap = n > 4096 ? n : 4096;
    if (dalloc_bytes((void **)&r->soa, 24 * (size_t)cap) != DDQMC_OK) return nullptr;
    r->soa_cap = cap;
    return r->soa;
}

int grid_for(int64_t n) {
    const int64_t g = (n + TX_TPB - 1) / TX_TPB;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

// spawn kernel shared memory, without / with the field's moves
constexpr size_t SP_SMEM = sizeof(SpawnShared<Rec, false>), SP_SMEM_F = sizeof(SpawnShared<Rec, true>);
constexpr size_t SPP_SMEM = sizeof(SpawnShared<uint64_t, false>), SPP_SMEM_F = sizeof(SpawnShared<uint64_t, true>);
constexpr size_t RX_SMEM = sizeof(RadixShared<Rec>);
constexpr size_t RXP_SMEM = sizeof(RadixShared<uint64_t>);
constexpr size_t MG_SMEM = sizeof(MergeShared<Rec>);
constexpr size_t MGP_SMEM = sizeof(MergeShared<uint64_t>);
constexpr size_t SPW_SMEM = sizeof(SpawnShared<RecW, false>), SPW_SMEM_F = sizeof(SpawnShared<RecW, true>);
constexpr size_t SP4_SMEM = sizeof(SpawnShared<P40, false>), SP4_SMEM_F = sizeof(SpawnShared<P40, true>);
constexpr size_t RX4_SMEM = sizeof(RadixShared<P40>);
constexpr size_t MG4_SMEM = sizeof(MergeShared<P40>);
constexpr size_t RXW_SMEM = sizeof(RadixShared<RecW>);
// radix tile sizes (records per thread) of packed records the tuner chooses from
constexpr int RX_PK_IPT[3] = {12, 16, 24};
constexpr size_t RXP_SMEM_V[3] = {sizeof(RadixShared<uint64_t, 12>), sizeof(RadixShared<uint64_t, 16>),
                                  sizeof(RadixShared<uint64_t, 24>)};
const void *radix_packed_fn(int v) {
    return v == 0 ? (const void *)k_radix_pass<uint64_t, 12>
                  : (v == 2 ? (const void *)k_radix_pass<uint64_t, 24> : (const void *)k_radix_pass<uint64_t, 16>);
}
int radix_variant(int ipt) { return ipt == 12 ? 0 : (ipt == 24 ? 2 : 1); }
constexpr size_t MGW_SMEM = sizeof(MergeShared<RecW>);

// One step's launches for spawn records of type T (16-byte Rec, packed 8-byte,
// or two-word RecW), on the list buffers Lc (current) and Ln (next); BATCH:
// the lists hold a batch of runs.
template <typename T, bool BATCH>
void launch_step(ddqmc_run *r, void *Lcv, void *Lnv, const std::function<void(int, int)> &mark) {
    using LT = typename ListOf<T>::type;
    LT *Lc = reinterpret_cast<LT *>(Lcv), *Ln = reinterpret_cast<LT *>(Lnv);
    const RunParams &P = r->hp;
    T *sp0 = reinterpret_cast<T *>(r->Sp[0]);
    T *sp1 = reinterpret_cast<T *>(r->Sp[1]);
    const size_t rx_smem = sizeof(RadixShared<T>);
    const RunParams *Pr = BATCH ? r->dPr : r->dP;
    DevState *rs = BATCH ? r->dRS : r->dS;
    mark(0, 0);
    if (P.field_on)
        k_spawn_death<T, true, BATCH><<<r->g_spawn, SP_TPB, sizeof(SpawnShared<T, true>), r->stream>>>(
            r->dP, r->dS, Lc, sp0, r->rcap, Pr, rs, (int64_t)r->tune.heavy_walkers);
    else
        k_spawn_death<T, false, BATCH><<<r->g_spawn, SP_TPB, sizeof(SpawnShared<T, false>), r->stream>>>(
            r->dP, r->dS, Lc, sp0, r->rcap, Pr, rs, (int64_t)r->tune.heavy_walkers);
    mark(0, 1);
    mark(1, 0);
    for (int p = 0; p < P.npass; ++p) {
        const T *in = (p & 1) ? sp1 : sp0;
        T *outp = (p & 1) ? sp0 : sp1;
        if constexpr (std::is_same<T, uint64_t>::value) {
            const int v = radix_variant(r->tune.radix_records_per_thread);
            if (v == 0)
                k_radix_pass<T, 12><<<r->g_radix, RX_TPB, RXP_SMEM_V[0], r->stream>>>(in, outp, r->dS, r->lb_radix, p,
                                                                                    P.pass_shift[p], r->rcap);
            else if (v == 2)
                k_radix_pass<T, 24><<<r->g_radix, RX_TPB, RXP_SMEM_V[2], r->stream>>>(in, outp, r->dS, r->lb_radix, p,
                                                                                    P.pass_shift[p], r->rcap);
            else
                k_radix_pass<T, 16><<<r->g_radix, RX_TPB, RXP_SMEM_V[1], r->stream>>>(in, outp, r->dS, r->lb_radix, p,
                                                                                    P.pass_shift[p], r->rcap);
        } else {
            k_radix_pass<T><<<r->g_radix, RX_TPB, rx_smem, r->stream>>>(in, outp, r->dS, r->lb_radix, p,
                                                                       P.pass_shift[p], r->rcap);
        }
    }
    if constexpr (std::is_same<T, RecW>::value) {
        if (P.hashed) {
            // equal stored bra words into ket order
            RecW *srt = (P.npass & 1) ? sp1 : sp0;
            k_hash_check<<<r->g_hcheck, HO_TPB, 0, r->stream>>>(srt, r->dS, r->hviol, r->rcap);
            k_hash_repair<<<r->g_hrepair, HO_TPB, 0, r->stream>>>(srt, r->dS, r->hviol, r->rcap);
        }
    }
    mark(1, 1);
    const T *sorted = (P.npass & 1) ? sp1 : sp0;
    mark(2, 0);
    k_merge_partition<T><<<r->g_part, 256, 0, r->stream>>>(Lc, sorted, r->dS, r->splits, r->rem_end, r->rcap);
    mark(2, 1);
    mark(3, 0);
    k_merge<T, BATCH><<<r->g_merge, MG_TPB, r->mg_smem, r->stream>>>(
        r->dP, Lc, sorted, reinterpret_cast<LT *>(r->slots), r->tile_counts, r->dS, r->splits, r->rem_end, r->rcap,
        Pr, rs);
    mark(3, 1);
    // compaction: tile offsets (into splits, free once the merge has run), then the copy
    mark(5, 0);
    k_merge_scan<<<r->g_scan, MC_TPB, 0, r->stream>>>(r->tile_counts, r->splits, r->dS, r->lb_merge, r->rcap,
                                                      r->mcap);
    k_merge_copy<LT><<<r->g_copy, MC_TPB, 0, r->stream>>>(reinterpret_cast<const LT *>(r->slots), r->tile_counts,
                                                          r->splits, Ln, r->dS, r->rcap);
    mark(5, 1);
}

// Default capacities: with total-population control the list holds at most
// ~target entries and a step makes up to a few records per walker (P_tot > 1
// under importance sampling); with diagonal control the off-diagonal
// population is not held, so leave a wide margin.
int64_t default_list_capacity(int control, int64_t target) {
    return (control == 1 ? 2 * target : 64 * target) + 65536;
}
int64_t default_spawn_capacity(int control, int64_t target) {
    return (control == 1 ? 4 * target : 64 * target) + 65536;
}

// Step state of a run at t = 0: n0 real walkers on |0><0|, fixed shift S0.
void initial_state(const RunParams &P, double S0, int64_t n0, DevState &hs) {
    std::memset(&hs, 0, sizeof(hs));
    hs.t = 0;
    hs.t_var = -1;
    hs.t_eq = -1;
    hs.q_prev = n0;
    hs.S = S0;
    hs.variable = 0;
    hs.M = n0 > 0 ? 1 : 0;
    hs.W_cur = n0;
    hs.epoch = 16;
    host_death_table(P, S0, hs);
}

// ---- launch shapes --------------------------------------------------------
// Results never depend on the launch shapes (every draw is keyed by the
// configuration, tiles are taken by ticket and reduced in key order), so
// the shapes only change the time a step takes.

ddqmc_tuning default_tuning(const ddqmc_run *r) {
    ddqmc_tuning t;
    std::memset(&t, 0, sizeof(t));
    t.spawn_blocks_per_sm = r->occ_spawn;
    t.radix_blocks_per_sm = r->occ_radix[1];
    t.merge_blocks_per_sm = r->occ_merge;
    t.copy_blocks_per_sm = r->occ_copy;
    t.scan_blocks_per_sm = r->occ_scan;
    t.partition_blocks_per_sm = 4;
    t.heavy_walkers = SP_HEAVY;
    t.radix_records_per_thread = r->packed ? 16 : 0;
    return t;
}

int clamp_bps(int v, int hi) { return v < 1 ? 1 : (v > hi ? hi : v); }

// Grids of the shapes t, each clamped to what the kernel can hold; records
// the clamped shapes in r->tune and drops captured step graphs (they hold the
// old grids).
void apply_tuning(ddqmc_run *r, const ddqmc_tuning &t) {
    ddqmc_tuning c = t;
    if (!r->packed) c.radix_records_per_thread = 0;
    else if (c.radix_records_per_thread != 12 && c.radix_records_per_thread != 24) c.radix_records_per_thread = 16;
    const int rv = radix_variant(c.radix_records_per_thread);
    c.spawn_blocks_per_sm = clamp_bps(c.spawn_blocks_per_sm, r->occ_spawn);
    c.radix_blocks_per_sm = clamp_bps(c.radix_blocks_per_sm, r->occ_radix[rv]);
    c.merge_blocks_per_sm = clamp_bps(c.merge_blocks_per_sm, r->occ_merge);
    c.copy_blocks_per_sm = clamp_bps(c.copy_blocks_per_sm, r->occ_copy);
    c.scan_blocks_per_sm = clamp_bps(c.scan_blocks_per_sm, r->occ_scan);
    c.partition_blocks_per_sm = clamp_bps(c.partition_blocks_per_sm, 8);
    if (c.heavy_walkers < 32) c.heavy_walkers = 32;
    r->tune = c;
    r->g_spawn = c.spawn_blocks_per_sm * r->sms;
    r->g_radix = c.radix_blocks_per_sm * r->sms;
    r->g_merge = c.merge_blocks_per_sm * r->sms;
    r->g_copy = c.copy_blocks_per_sm * r->sms;
    r->g_scan = c.scan_blocks_per_sm * r->sms;
    r->g_part = c.partition_blocks_per_sm * r->sms;
    r->g_hcheck = 4 * r->sms;
    r->g_hrepair = r->sms;
    for (int k = 0; k < 2; ++k)
        if (r->graph[k]) {
            cudaGraphExecDestroy(r->graph[k]);
            r->graph[k] = nullptr;
        }
}

// Tunings found by ddqmc_tune in this process, by (sites, record kind, batch,
// SMs): a later run of the same kind starts with the last one found.
struct TuneKey {
    int N, kind, batch, sms;
    bool operator==(const TuneKey &o) const { return N == o.N && kind == o.kind && batch == o.batch && sms == o.sms; }
};
std::vector<std::pair<TuneKey, ddqmc_tuning>> g_tune_cache;

TuneKey tune_key(const ddqmc_run *r) {
    return TuneKey{r->hp.N, r->packed ? 1 : (r->wide ? 2 : (r->p40 ? 3 : 0)), r->nruns > 0 ? 1 : 0, r->sms};
}

bool cached_tuning(const ddqmc_run *r, ddqmc_tuning *out) {
    const TuneKey k = tune_key(r);
    for (const auto &e : g_tune_cache)
        if (e.first == k) { *out = e.second; return true; }
    return false;
}

void cache_tuning(const ddqmc_run *r, const ddqmc_tuning &t) {
    const TuneKey k = tune_key(r);
    for (auto &e : g_tune_cache)
        if (e.first == k) { e.second = t; return; }
    g_tune_cache.push_back({k, t});
}

// Stream, device buffers (capacities clamped to [4096, 2^31 - 1]), blocking
// cells, kernel attributes and persistent grid sizes of a run or a batch
// (r->hp, r->nruns, r->wide and r->packed already set).
int setup_device(ddqmc_run *r, const ddqmc_options &o, int64_t mcap, int64_t rcap, size_t blk_cells) {
    if (cudaGetDevice(&r->device) != cudaSuccess) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    if (mcap < 4096) mcap = 4096;
    if (rcap < 4096) rcap = 4096;
    const int64_t lim = (1ll << 31) - 1;
    if (mcap > lim) mcap = lim;
    if (rcap > lim) rcap = lim;
    r->mcap = mcap;
    r->rcap = rcap;
    if (o.cuda_stream) {
        r->stream = (cudaStream_t)o.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            r->stream = nullptr;
            return DDQMC_ERR_CUDA;
        }
        r->own_stream = true;
    }
    const int64_t rtiles = rcap / RX_TILE_MIN + 2;
    const int64_t mtiles = (mcap + rcap) / MG_TILE + 2;
    int rc = DDQMC_OK;
    rc |= dalloc(&r->dP, 1);
    rc |= dalloc(&r->dS, 1);
    rc |= dalloc(&r->dBlk, blk_cells);
    r->blk_cells = blk_cells;
    const size_t lsize = r->wide ? sizeof(RecW) : sizeof(Rec);
    const size_t ssize = r->wide ? sizeof(RecW) : sizeof(Rec);   // standalone annihilation uses 16-byte Rec
    // 64 bytes past the last record: the merge's bulk copies widen each range
    // to 16-byte boundaries, so 24-byte records are read up to 15 bytes past it
    rc |= dalloc_bytes(&r->L[0], lsize * (size_t)mcap + 64);
    rc |= dalloc_bytes(&r->L[1], lsize * (size_t)mcap + 64);
    rc |= dalloc_bytes(&r->Sp[0], ssize * (size_t)rcap + 64);
    rc |= dalloc_bytes(&r->Sp[1], ssize * (size_t)rcap + 64);
    rc |= dalloc(&r->lb_radix, (size_t)rtiles * 256);
    rc |= dalloc(&r->lb_merge, (size_t)mtiles);
    rc |= dalloc(&r->splits, (size_t)mtiles + 1);
    rc |= dalloc(&r->rem_end, (size_t)mtiles + 1);
    rc |= dalloc_bytes(&r->slots, lsize * (size_t)mtiles * MG_TILE + 64);
    rc |= dalloc(&r->tile_counts, (size_t)mtiles);
    if (r->wide) rc |= dalloc(&r->hviol, (size_t)HO_MAXV);
    if (rc != DDQMC_OK) return DDQMC_ERR_OOM;
    // kernel shapes
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, r->device);
    if (sms < 1) sms = 1;
    if (o.sm_limit > 0 && o.sm_limit < sms) sms = o.sm_limit;
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, r->device);
    bool ok = true;
    auto attr = [&](const void *fn, size_t bytes) {
        ok = ok && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
    };
    attr((const void *)k_spawn_death<Rec, true, false>, SP_SMEM_F);
    attr((const void *)k_spawn_death<Rec, false, false>, SP_SMEM);
    attr((const void *)k_spawn_death<uint64_t, true, false>, SPP_SMEM_F);
    attr((const void *)k_spawn_death<uint64_t, false, false>, SPP_SMEM);
    attr((const void *)k_spawn_death<RecW, true, false>, SPW_SMEM_F);
    attr((const void *)k_spawn_death<RecW, false, false>, SPW_SMEM);
    attr((const void *)k_spawn_death<Rec, true, true>, SP_SMEM_F);
    attr((const void *)k_spawn_death<Rec, false, true>, SP_SMEM);
    attr((const void *)k_spawn_death<uint64_t, true, true>, SPP_SMEM_F);
    attr((const void *)k_spawn_death<uint64_t, false, true>, SPP_SMEM);
    attr((const void *)k_spawn_death<RecW, true, true>, SPW_SMEM_F);
    attr((const void *)k_spawn_death<P40, true, false>, SP4_SMEM_F);
    attr((const void *)k_spawn_death<P40, false, false>, SP4_SMEM);
    attr((const void *)k_spawn_death<P40, true, true>, SP4_SMEM_F);
    attr((const void *)k_spawn_death<P40, false, true>, SP4_SMEM);
    attr((const void *)k_radix_pass<P40>, RX4_SMEM);
    attr((const void *)k_merge<P40, false>, MG4_SMEM);
    attr((const void *)k_spawn_death<RecW, false, true>, SPW_SMEM);
    attr((const void *)k_radix_pass<Rec>, RX_SMEM);
    attr((const void *)k_radix_pass<uint64_t>, RXP_SMEM);
    for (int v = 0; v < 3; ++v) attr(radix_packed_fn(v), RXP_SMEM_V[v]);
    attr((const void *)k_radix_pass<RecW>, RXW_SMEM);
    attr((const void *)k_merge<Rec, false>, MG_SMEM);
    attr((const void *)k_merge<uint64_t, false>, MGP_SMEM);
    attr((const void *)k_merge<RecW, false>, MGW_SMEM);
    // batch merges: per-run estimator sums past MergeShared, up to what the
    // device allows next to the kernel's static shared memory
    auto dyn_max = [&](const void *fn) -> size_t {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) { ok = false; return 0; }
        return (size_t)smem_max > fa.sharedSizeBytes ? (size_t)smem_max - fa.sharedSizeBytes : 0;
    };
    const size_t bmax_rec = dyn_max((const void *)k_merge<Rec, true>);
    const size_t bmax_pk = dyn_max((const void *)k_merge<uint64_t, true>);
    const size_t bmax_w = dyn_max((const void *)k_merge<RecW, true>);
    const size_t bmax_p4 = dyn_max((const void *)k_merge<P40, true>);
    attr((const void *)k_merge<Rec, true>, bmax_rec);
    attr((const void *)k_merge<uint64_t, true>, bmax_pk);
    attr((const void *)k_merge<RecW, true>, bmax_w);
    attr((const void *)k_merge<P40, true>, bmax_p4);
    if (!ok) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    const bool B = r->nruns > 0;
    const size_t est_bytes = B ? sizeof(unsigned long long) * (size_t)r->nruns * (size_t)r->hp.nobs : 0;
    const void *fs, *fr, *fm;
    size_t ss, sr, sm, bmax;
    const bool F = r->hp.field_on != 0;
    if (r->packed) {
        fs = F ? (B ? (const void *)k_spawn_death<uint64_t, true, true> : (const void *)k_spawn_death<uint64_t, true, false>)
               : (B ? (const void *)k_spawn_death<uint64_t, false, true> : (const void *)k_spawn_death<uint64_t, false, false>);
        fr = (const void *)k_radix_pass<uint64_t>;
        fm = B ? (const void *)k_merge<uint64_t, true> : (const void *)k_merge<uint64_t, false>;
        ss = F ? SPP_SMEM_F : SPP_SMEM; sr = RXP_SMEM; sm = MGP_SMEM; bmax = bmax_pk;
    } else if (r->p40) {
        fs = F ? (B ? (const void *)k_spawn_death<P40, true, true> : (const void *)k_spawn_death<P40, true, false>)
               : (B ? (const void *)k_spawn_death<P40, false, true> : (const void *)k_spawn_death<P40, false, false>);
        fr = (const void *)k_radix_pass<P40>;
        fm = B ? (const void *)k_merge<P40, true> : (const void *)k_merge<P40, false>;
        ss = F ? SP4_SMEM_F : SP4_SMEM; sr = RX4_SMEM; sm = MG4_SMEM; bmax = bmax_p4;
    } else if (r->wide) {
        fs = F ? (B ? (const void *)k_spawn_death<RecW, true, true> : (const void *)k_spawn_death<RecW, true, false>)
               : (B ? (const void *)k_spawn_death<RecW, false, true> : (const void *)k_spawn_death<RecW, false, false>);
        fr = (const void *)k_radix_pass<RecW>;
        fm = B ? (const void *)k_merge<RecW, true> : (const void *)k_merge<RecW, false>;
        ss = F ? SPW_SMEM_F : SPW_SMEM; sr = RXW_SMEM; sm = MGW_SMEM; bmax = bmax_w;
    } else {
        fs = F ? (B ? (const void *)k_spawn_death<Rec, true, true> : (const void *)k_spawn_death<Rec, true, false>)
               : (B ? (const void *)k_spawn_death<Rec, false, true> : (const void *)k_spawn_death<Rec, false, false>);
        fr = (const void *)k_radix_pass<Rec>;
        fm = B ? (const void *)k_merge<Rec, true> : (const void *)k_merge<Rec, false>;
        ss = F ? SP_SMEM_F : SP_SMEM; sr = RX_SMEM; sm = MG_SMEM; bmax = bmax_rec;
    }
    r->mg_smem = sm + est_bytes;
    if (B && r->mg_smem > bmax) return DDQMC_ERR_UNSUPPORTED;   // too many runs x observables
    r->sms = sms;
    r->occ_spawn = occupancy(fs, SP_TPB, ss);
    for (int v = 0; v < 3; ++v)
        r->occ_radix[v] = r->packed ? occupancy(radix_packed_fn(v), RX_TPB, RXP_SMEM_V[v]) : occupancy(fr, RX_TPB, sr);
    r->occ_merge = occupancy(fm, MG_TPB, r->mg_smem);
    r->g_merge_ann = occupancy_grid((const void *)k_merge<Rec, false>, MG_TPB, MG_SMEM, sms);
    r->g_radix_wide = occupancy_grid((const void *)k_radix_pass<Rec>, RX_TPB, RX_SMEM, sms);
    r->g_copy_ann = occupancy_grid((const void *)k_merge_copy<Rec>, MC_TPB, 0, sms);
    r->occ_scan = occupancy((const void *)k_merge_scan, MC_TPB, 0);
    r->occ_copy = occupancy(r->wide ? (const void *)k_merge_copy<RecW> : (const void *)k_merge_copy<Rec>, MC_TPB, 0);
    r->tune = default_tuning(r);
    cached_tuning(r, &r->tune);
    apply_tuning(r, r->tune);
    bool okc = cudaMemsetAsync(r->dBlk, 0, sizeof(BlkCell) * blk_cells, r->stream) == cudaSuccess;
    okc = okc && cudaMemsetAsync(r->lb_radix, 0, sizeof(uint64_t) * (size_t)rtiles * 256, r->stream) == cudaSuccess;
    okc = okc && cudaMemsetAsync(r->lb_merge, 0, sizeof(uint64_t) * (size_t)mtiles, r->stream) == cudaSuccess;
    if (!okc) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    return DDQMC_OK;
}

// kernel classes of the per-kernel timing
enum { KC_SPAWN = 0, KC_RADIX = 1, KC_PARTITION = 2, KC_MERGE = 3, KC_FINALIZE = 4, KC_COMPACT = 5, NKCLASS = 6 };

// Steps replayed from one captured graph: even, so that the list buffers end
// where they started and one graph per starting buffer suffices.
constexpr int64_t GRAPH_STEPS = 32;

void launch_one_step(ddqmc_run *r, const std::function<void(int, int)> &mark) {
    // one NVTX range per issued step (free without an attached tool)
    nvtxRangePushA("ddqmc step");
    void *Lc = r->L[r->cur], *Ln = r->L[r->cur ^ 1];
    if (r->nruns) {
        if (r->packed) launch_step<uint64_t, true>(r, Lc, Ln, mark);
        else if (r->p40) launch_step<P40, true>(r, Lc, Ln, mark);
        else if (r->wide) launch_step<RecW, true>(r, Lc, Ln, mark);
        else launch_step<Rec, true>(r, Lc, Ln, mark);
    } else {
        if (r->packed) launch_step<uint64_t, false>(r, Lc, Ln, mark);
        else if (r->p40) launch_step<P40, false>(r, Lc, Ln, mark);
        else if (r->wide) launch_step<RecW, false>(r, Lc, Ln, mark);
        else launch_step<Rec, false>(r, Lc, Ln, mark);
    }
    mark(KC_FINALIZE, 0);
    if (r->nruns) k_finalize<true><<<r->nruns, FN_TPB, 0, r->stream>>>(r->dPr, r->dS, r->dBlk, r->dRS);
    else k_finalize<false><<<1, FN_TPB, 0, r->stream>>>(r->dP, r->dS, r->dBlk, r->dS);
    mark(KC_FINALIZE, 1);
    nvtxRangePop();
    r->cur ^= 1;
}

// Capture GRAPH_STEPS steps starting from the current buffer (launch overhead
// dominates small runs; the graph replays the same launches).  false if
// capture is not possible on this stream.
bool capture_graph(ddqmc_run *r) {
    const int start = r->cur;
    std::function<void(int, int)> none = [](int, int) {};
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(r->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    for (int64_t s = 0; s < GRAPH_STEPS; ++s) launch_one_step(r, none);
    const bool ok = cudaStreamEndCapture(r->stream, &g) == cudaSuccess && g &&
                    cudaGraphInstantiate(&r->graph[start], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    r->cur = start;
    if (!ok) {
        cudaGetLastError();
        r->graph[start] = nullptr;
    }
    return ok;
}

int enqueue_steps(ddqmc_run *r, int64_t nsteps) {
    // whole graphs first (not while per-kernel events are recorded)
    while (!r->timing && !r->no_graph && nsteps >= GRAPH_STEPS) {
        if (!r->graph[r->cur] && !capture_graph(r)) { r->no_graph = true; break; }
        if (cudaGraphLaunch(r->graph[r->cur], r->stream) != cudaSuccess) {
            cudaGetLastError();
            r->host_status = DDQMC_ERR_CUDA;
            return r->host_status;
        }
        nsteps -= GRAPH_STEPS;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        cudaEvent_t *ev = nullptr;
        if (r->timing) {
            const size_t need = (size_t)(s + 1) * 2 * NKCLASS;
            while (r->ev.size() < need) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
                r->ev.push_back(e);
            }
            ev = &r->ev[(size_t)s * 2 * NKCLASS];
        }
        std::function<void(int, int)> mark = [&](int kc, int edge) {
            if (ev) cudaEventRecord(ev[2 * kc + edge], r->stream);
        };
        launch_one_step(r, mark);
    }
    if (cudaGetLastError() != cudaSuccess) {
        r->host_status = DDQMC_ERR_CUDA;
        return r->host_status;
    }
    return DDQMC_OK;
}

// Fold the recorded per-kernel times of the last nsteps steps into the totals
// (the stream must have been synchronised).
void collect_timing(ddqmc_run *r, int64_t nsteps) {
    if (!r->timing) return;
    for (int64_t s = 0; s < nsteps; ++s)
        for (int kc = 0; kc < NKCLASS; ++kc) {
            float ms = 0.f;
            const size_t b = (size_t)s * 2 * NKCLASS + 2 * kc;
            if (cudaEventElapsedTime(&ms, r->ev[b], r->ev[b + 1]) == cudaSuccess) {
                r->kernel_ms[kc] += ms;
                r->kernel_launches[kc] += (kc == KC_RADIX) ? r->hp.npass + (r->hp.hashed ? 2 : 0)
                                                           : (kc == KC_COMPACT ? 2 : 1);
            } else {
                cudaGetLastError();
            }
        }
}

struct LevelStat {
    int64_t n;
    double R, err;
};

// Delta-method variance of sum X / sum Y from exact integer moments of one level.
LevelStat level_stat(const BlkCell &cx, const BlkCell &cy) {
    LevelStat o;
    o.n = cx.n;
    o.R = cy.sx != 0 ? (double)cx.sx / (double)cy.sx : NAN;
    o.err = NAN;
    if (cx.n < 2 || cy.sx == 0) return o;
    const __int128 n = cx.n;
    const __int128 A = n * cx.sxx - (__int128)cx.sx * cx.sx;
    const __int128 C = n * cx.sxy - (__int128)cx.sx * cy.sx;
    const __int128 D = n * cy.sxx - (__int128)cy.sx * cy.sx;
    const long double X = (long double)cx.sx, Y = (long double)cy.sx;
    const long double num = (long double)A * Y * Y - 2.0L * X * Y * (long double)C + X * X * (long double)D;
    const long double den = (long double)(cx.n - 1) * Y * Y * Y * Y;
    const long double var = num / den;
    o.err = var >= 0 ? (double)std::sqrt(var) : NAN;
    return o;
}

// Blocked ratio estimate: R over all samples and the plateau error.
void blocked_ratio(const std::vector<BlkCell> &cells, int k, double &R, double &err) {
    std::vector<LevelStat> lv;
    for (int l = 0; l < LEVELS; ++l) {
        const BlkCell &cx = cells[(size_t)k * LEVELS + l];
        if (cx.n < 1) break;
        lv.push_back(level_stat(cx, cells[l]));
    }
    R = lv.empty() ? NAN : lv[0].R;
    err = NAN;
    std::vector<int> valid;
    for (int l = 0; l < (int)lv.size(); ++l)
        if (lv[l].n >= 16 && lv[l].err == lv[l].err) valid.push_back(l);
    if (valid.empty()) return;
    auto de = [&](int l) { return lv[l].err / std::sqrt(2.0 * (double)(lv[l].n - 1)); };
    for (size_t a = 0; a < valid.size(); ++a) {
        const int kk = valid[a];
        bool ok = true;
        for (size_t b = a + 1; b < valid.size() && ok; ++b) {
            const int q = valid[b];
            if (lv[q].err > lv[kk].err + 2.0 * std::sqrt(de(kk) * de(kk) + de(q) * de(q))) ok = false;
        }
        if (ok) { err = lv[kk].err; return; }
    }
    err = lv[valid.back()].err;
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch of ddqmc_annihilate_noalloc, in the library's own device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// already reserved by another allocator's pool (a serving engine or a
// framework's caching allocator that took it all up front), or a loop that
// must not take the driver's allocation path with its implicit
// synchronisation.  For them the annihilation stage can run out of this fixed
// array instead: every GPU that loads the library holds it until the process
// exits.  In host code the array's name is only a host-side stand-in; the
// device address comes from cudaGetSymbolAddress, looked up once per device.
// Every call shares the array and leaves its contents behind; the parts that
// must start at zero are cleared at the start of each call, and calls that
// overlap on the GPU (two streams at once) race on it.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NA_MAX_SPAWNS = 1ll << 18;     // spawn records per call
constexpr int64_t NA_MAX_LIST = 1ll << 20;       // list entries per call
constexpr int64_t NA_RTILES = NA_MAX_SPAWNS / RX_TILE_MIN + 2;
constexpr int64_t NA_MTILES = (NA_MAX_LIST + NA_MAX_SPAWNS) / MG_TILE + 3;

struct NoAllocScratch {
    RunParams P;
    DevState st;
    uint64_t lb_radix[NA_RTILES * 256];
    uint64_t lb_merge[NA_MTILES];
    int64_t splits[NA_MTILES + 1];
    int64_t rem_end[NA_MTILES + 1];
    uint32_t counts[NA_MTILES];
    Rec buf[2][NA_MAX_SPAWNS];
    Rec slots[NA_MTILES * MG_TILE];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int NA_MAX_DEVICES = 64;
NoAllocScratch *g_na_ptr[NA_MAX_DEVICES] = {nullptr};
int g_na_grid[NA_MAX_DEVICES][4];       // radix, partition (and tile-offset scan), merge, copy grids

// Once per device, with that device current: device address of the scratch
// array and the launch shapes.
int noalloc_setup(int dev) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return DDQMC_ERR_UNSUPPORTED;
    if (g_na_ptr[dev]) return DDQMC_OK;
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(k_radix_pass<Rec>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RX_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_merge<Rec, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MG_SMEM) !=
            cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    g_na_grid[dev][0] = occupancy_grid((const void *)k_radix_pass<Rec>, RX_TPB, RX_SMEM, sms);
    g_na_grid[dev][1] = 4 * sms;
    g_na_grid[dev][2] = occupancy_grid((const void *)k_merge<Rec, false>, MG_TPB, MG_SMEM, sms);
    g_na_grid[dev][3] = occupancy_grid((const void *)k_merge_copy<Rec>, MC_TPB, 0, sms);
    g_na_ptr[dev] = (NoAllocScratch *)ptr;
    return DDQMC_OK;
}

// Run k of a batch, or the run itself (k ignored) when not a batch.
DevState *run_state(ddqmc_run *r, int k) { return r->nruns ? r->dRS + k : r->dS; }
const RunParams &run_params(const ddqmc_run *r, int k) { return r->nruns ? r->hpr[(size_t)k] : r->hp; }
BlkCell *run_cells(ddqmc_run *r, int k) {
    return r->dBlk + (r->nruns ? (size_t)k * (size_t)r->hp.nobs * LEVELS : (size_t)0);
}

int raw_estimators_of(ddqmc_run *r, int k, int64_t *host_out, int32_t cap, int32_t *nobs) {
    const int n = run_params(r, k).nobs;
    if (nobs) *nobs = n;
    const int m = cap < n ? cap : n;
    if (m > 0) {
        if (cudaMemcpyAsync(host_out, run_state(r, k)->last_est, sizeof(int64_t) * (size_t)m,
                            cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
            cudaStreamSynchronize(r->stream) != cudaSuccess) {
            cudaGetLastError();
            return DDQMC_ERR_CUDA;
        }
    }
    return DDQMC_OK;
}

// Sort n two-word records in Sp[0] with the step's digit passes and the
// standalone counters (dAnn): npass passes of 8 bits, the first nlo over the
// ket word, the rest over the bra word; hashed: then equal bra words into ket
// order.  *sorted = the buffer holding the result.  Synchronises the stream.
int sort_records_wide(ddqmc_run *r, int64_t n, int npass, int nlo, bool hashed, RecW **sorted) {
    RecW *sp0 = reinterpret_cast<RecW *>(r->Sp[0]), *sp1 = reinterpret_cast<RecW *>(r->Sp[1]);
    *sorted = (npass & 1) ? sp1 : sp0;
    if (n > r->rcap) return DDQMC_ERR_CAPACITY;
    if (!r->dAnn && dalloc(&r->dAnn, 1) != DDQMC_OK) return DDQMC_ERR_OOM;
    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.R = n;
    // epochs of standalone calls carry bit 29, those of the run's steps do not
    hs.epoch = (1u << 29) | ((r->ann_calls++ * 16u) & ((1u << 29) - 1u));
    bool ok = cudaMemcpyAsync(r->dAnn, &hs, sizeof(DevState), cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
    if (n > 0) {
        k_digit_histogram<RecW><<<r->g_part, RX_TPB, 0, r->stream>>>(sp0, r->dAnn, npass, nlo);
        for (int p = 0; p < npass; ++p)
            k_radix_pass<RecW><<<r->g_radix, RX_TPB, RXW_SMEM, r->stream>>>(
                (p & 1) ? sp1 : sp0, (p & 1) ? sp0 : sp1, r->dAnn, r->lb_radix, p,
                p < nlo ? 8 * p : 64 + 8 * (p - nlo), r->rcap);
        if (hashed) {
            k_hash_check<<<r->g_hcheck, HO_TPB, 0, r->stream>>>(*sorted, r->dAnn, r->hviol, r->rcap);
            k_hash_repair<<<r->g_hrepair, HO_TPB, 0, r->stream>>>(*sorted, r->dAnn, r->hviol, r->rcap);
        }
        ok = ok && cudaGetLastError() == cudaSuccess;
    }
    ok = ok && cudaMemcpyAsync(&hs, r->dAnn, sizeof(DevState), cudaMemcpyDeviceToHost, r->stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(r->stream) == cudaSuccess;
    if (!ok) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    return hs.status ? status_code(hs.status) : DDQMC_OK;
}

// Canonical (ket, bra, re, im) of the current list: the whole list (k < 0),
// or the entries of batch run k (a contiguous range: the run id is the key's
// most significant part).  *n = the entries of that list or run.
template <typename LT>
int export_list(ddqmc_run *r, int k, uint64_t *ket, uint64_t *bra, int32_t *re, int32_t *im, int64_t cap,
                int64_t *n) {
    int64_t M = 0;
    if (cudaMemcpyAsync(&M, &r->dS->M, sizeof(M), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    const LT *L = reinterpret_cast<const LT *>(r->L[r->cur]);
    // [b0, b1): the exported range (run k's entries of a batch)
    int64_t b0 = 0, b1 = M;
    if (k >= 0 && M > 0) {
        if (!soa_scratch(r, 1)) return DDQMC_ERR_OOM;
        int64_t hb[2] = {0, 0};
        k_run_bounds<LT><<<1, 32, 0, r->stream>>>(L, r->dS, r->hp.run_shift, (uint64_t)k, (int64_t *)(r->dxfer + 2));
        if (cudaMemcpyAsync(hb, r->dxfer + 2, sizeof(hb), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
            cudaStreamSynchronize(r->stream) != cudaSuccess) {
            cudaGetLastError();
            return DDQMC_ERR_CUDA;
        }
        b0 = hb[0];
        b1 = hb[1];
    }
    *n = b1 - b0;
    int64_t m = b1 - b0;
    if (m > cap) m = cap > 0 ? cap : 0;     // only what the caller can take
    if (m <= 0) return DDQMC_OK;
    if constexpr (std::is_same<LT, RecW>::value) {
        if (r->hp.hashed) {
            // the hashed order is not the caller's: the exported range with
            // its plain bra words, then a sort on both words (Sp[0] holds the
            // copy; the entries of a batch run share their run bits, so the
            // bra word's digits need not reach them)
            const int64_t me = b1 - b0;
            if (me > r->rcap) return DDQMC_ERR_CAPACITY;
            k_unhash<<<grid_for(me), TX_TPB, 0, r->stream>>>(L + b0, me, r->hp.hash_mask,
                                                               reinterpret_cast<RecW *>(r->Sp[0]));
            const int nb = (r->hp.N + 7) / 8;
            RecW *srt = nullptr;
            const int rc = sort_records_wide(r, me, 2 * nb, nb, false, &srt);
            if (rc != DDQMC_OK) return rc;
            L = srt;
            b0 = 0;
        }
    }
    unsigned char *d = soa_scratch(r, m);
    if (!d) return DDQMC_ERR_OOM;
    uint64_t *dk = reinterpret_cast<uint64_t *>(d), *db = dk + m;
    int32_t *dr = reinterpret_cast<int32_t *>(db + m), *di = dr + m;
    k_export_unpack<LT><<<grid_for(m), TX_TPB, 0, r->stream>>>(L + b0, m, r->hp.N, r->hp.nmask, dk, db, dr, di);
    bool ok = cudaGetLastError() == cudaSuccess;
    ok = ok && cudaMemcpyAsync(ket, dk, 8 * (size_t)m, cudaMemcpyDeviceToHost, r->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(bra, db, 8 * (size_t)m, cudaMemcpyDeviceToHost, r->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(re, dr, 4 * (size_t)m, cudaMemcpyDeviceToHost, r->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(im, di, 4 * (size_t)m, cudaMemcpyDeviceToHost, r->stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(r->stream) == cudaSuccess;
    if (!ok) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    return DDQMC_OK;
}

// Walker list of run k (k < 0: the whole list of a single run) into the
// caller's arrays: unpacked on the device, then one copy per array.
int export_of(ddqmc_run *r, int k, uint64_t *ket, uint64_t *bra, int32_t *re, int32_t *im, int64_t cap,
              int64_t *n) {
    return r->wide ? export_list<RecW>(r, k, ket, bra, re, im, cap, n) : export_list<Rec>(r, k, ket, bra, re, im, cap, n);
}

// State of run k (the run itself when not a batch); the status word is the
// shared one.
int state_of(ddqmc_run *r, int k, ddqmc_state *out) {
    DevState hs;
    uint32_t status = 0;
    if (cudaMemcpyAsync(&hs, run_state(r, k), sizeof(DevState), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaMemcpyAsync(&status, &r->dS->status, sizeof(status), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    hs.status = status;
    out->t = hs.t;
    out->shift = hs.S;
    out->variable = hs.variable;
    out->q_prev = hs.q_prev;
    out->t_var = hs.t_var;
    out->t_eq = hs.t_eq;
    out->entries = hs.M;
    out->status = r->host_status ? r->host_status : status_code(hs.status);
    out->status_bits = (int32_t)hs.status;
    return DDQMC_OK;
}

// Estimates of run k (the run itself when not a batch).
int estimates_of(ddqmc_run *r, int k, ddqmc_estimates *out) {
    const RunParams &P = run_params(r, k);
    DevState hs;
    uint32_t status = 0;
    std::vector<BlkCell> cells((size_t)P.nobs * LEVELS);
    if (cudaMemcpyAsync(&hs, run_state(r, k), sizeof(DevState), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaMemcpyAsync(cells.data(), run_cells(r, k), sizeof(BlkCell) * cells.size(), cudaMemcpyDeviceToHost,
                        r->stream) != cudaSuccess ||
        cudaMemcpyAsync(&status, &r->dS->status, sizeof(status), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    hs.status = status;
    std::memset(out, 0, sizeof(*out));
    const int N = P.N, B = P.B, core = 5 + N + 3 * B;
    out->t = hs.t;
    out->shift = hs.S;
    out->variable = hs.variable;
    out->t_var = hs.t_var;
    out->t_eq = hs.t_eq;
    out->n_samples = hs.n_app;
    out->walkers = hs.last_est[3];
    out->entries = hs.M;
    out->nw = hs.last_est[2];
    out->trace_re = hs.last_est[0];
    out->trace_im = hs.last_est[1];
    out->nsites = N;
    out->nbonds = B;
    out->walker_steps = (double)hs.walker_steps;
    if (hs.t == 0) {            // nothing stepped yet: report the initial list
        out->walkers = hs.W_cur;
        out->nw = hs.W_cur;
        out->trace_re = hs.W_cur;
    }
    double R, e;
    blocked_ratio(cells, core + 0, R, e);
    out->mz = R / N;
    out->mz_err = e / N;
    for (int k = 0; k < N; ++k) {
        blocked_ratio(cells, 5 + k, R, e);
        out->sz[k] = R;
        out->sz_err[k] = e;
    }
    bool uniform_w = true;
    for (int b = 1; b < B; ++b) uniform_w = uniform_w && r->w_bond[b] == r->w_bond[0];
    for (int b = 0; b < B; ++b) {
        blocked_ratio(cells, 5 + N + b, R, e);
        out->bond_zz[b] = R;
        blocked_ratio(cells, 5 + N + B + b, R, e);
        out->bond_xx[b] = R / r->w_bond[b];
        blocked_ratio(cells, 5 + N + 2 * B + b, R, e);
        out->bond_yy[b] = R / r->w_bond[b];
    }
    blocked_ratio(cells, core + 1, R, e);
    out->zz = B ? R / B : NAN;
    out->zz_err = B ? e / B : NAN;
    const double w0 = B ? r->w_bond[0] : 1.0;
    blocked_ratio(cells, core + 2, R, e);
    out->xx = B ? R / (B * w0) : NAN;
    out->xx_err = B ? e / (B * w0) : NAN;
    blocked_ratio(cells, core + 3, R, e);
    out->yy = B ? R / (B * w0) : NAN;
    out->yy_err = B ? e / (B * w0) : NAN;
    // single-site sigma^x, sigma^y (non-zero only with a field): numerators / site weight
    {
        const int ox = core + 4, oy = ox + N;
        double sxs = 0, sys = 0, exs = 0, eys = 0;
        for (int k = 0; k < N; ++k) {
            double Rk, ek;
            blocked_ratio(cells, ox + k, Rk, ek);
            out->sx[k] = Rk / r->w_site[k];
            sxs += out->sx[k];
            exs += (ek / r->w_site[k]) * (ek / r->w_site[k]);
            blocked_ratio(cells, oy + k, Rk, ek);
            out->sy[k] = Rk / r->w_site[k];
            sys += out->sy[k];
            eys += (ek / r->w_site[k]) * (ek / r->w_site[k]);
        }
        bool uniform_s = true;
        for (int k = 1; k < N; ++k) uniform_s = uniform_s && r->w_site[k] == r->w_site[0];
        if (uniform_s) {        // the blocked error of the site sum
            blocked_ratio(cells, oy + N, R, e);
            out->mx = R / (N * r->w_site[0]);
            out->mx_err = e / (N * r->w_site[0]);
            blocked_ratio(cells, oy + N + 1, R, e);
            out->my = R / (N * r->w_site[0]);
            out->my_err = e / (N * r->w_site[0]);
        } else {
            out->mx = sxs / N;
            out->my = sys / N;
            out->mx_err = std::sqrt(exs) / N;
            out->my_err = std::sqrt(eys) / N;
        }
    }
    if (!uniform_w && B) {      // per-bond weights differ: average the per-bond estimates
        double sx = 0, sy = 0, ex = 0, ey = 0;
        for (int b = 0; b < B; ++b) {
            sx += out->bond_xx[b];
            sy += out->bond_yy[b];
            double Rb, eb;
            blocked_ratio(cells, 5 + N + B + b, Rb, eb);
            ex += (eb / r->w_bond[b]) * (eb / r->w_bond[b]);
            blocked_ratio(cells, 5 + N + 2 * B + b, Rb, eb);
            ey += (eb / r->w_bond[b]) * (eb / r->w_bond[b]);
        }
        out->xx = sx / B;
        out->yy = sy / B;
        out->xx_err = std::sqrt(ex) / B;
        out->yy_err = std::sqrt(ey) / B;
    }
    return r->host_status ? r->host_status : status_code(hs.status);
}

}  // namespace

namespace {

// Device state of a run saved for the tuning trials.
struct TuneBackup {
    DevState st;
    std::vector<DevState> rs;
    void *list = nullptr;
    BlkCell *blk = nullptr;
    int cur = 0;
    int64_t M = 0;
};

// Put the saved state back; the look-back epoch moves past every epoch the
// trials used, so no status word they left can match a later step.
int tune_restore(ddqmc_run *r, const TuneBackup &b) {
    const size_t lsize = r->wide ? sizeof(RecW) : sizeof(Rec);
    uint32_t ep = 0;
    bool ok = cudaMemcpyAsync(&ep, &r->dS->epoch, sizeof(ep), cudaMemcpyDeviceToHost, r->stream) == cudaSuccess &&
              cudaStreamSynchronize(r->stream) == cudaSuccess;
    DevState h = b.st;
    h.epoch = (ep + 16u) & 0x3FFFFFFFu;
    r->cur = b.cur;
    ok = ok && cudaMemcpyAsync(r->L[b.cur], b.list, lsize * (size_t)b.M, cudaMemcpyDeviceToDevice, r->stream) ==
                   cudaSuccess;
    ok = ok && cudaMemcpyAsync(r->dS, &h, sizeof(DevState), cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
    if (r->nruns)
        ok = ok && cudaMemcpyAsync(r->dRS, b.rs.data(), sizeof(DevState) * b.rs.size(), cudaMemcpyHostToDevice,
                                   r->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(r->dBlk, b.blk, sizeof(BlkCell) * r->blk_cells, cudaMemcpyDeviceToDevice,
                               r->stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(r->stream) == cudaSuccess;
    if (!ok) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    r->host_status = 0;
    return DDQMC_OK;
}

// One step with the shapes t from the saved state; kernel-class times into ms.
int tune_trial(ddqmc_run *r, const TuneBackup &b, const ddqmc_tuning &t, double *ms) {
    int rc = tune_restore(r, b);
    if (rc != DDQMC_OK) return rc;
    apply_tuning(r, t);
    for (int k = 0; k < 8; ++k) { r->kernel_ms[k] = 0.0; r->kernel_launches[k] = 0; }
    rc = enqueue_steps(r, 1);
    if (rc != DDQMC_OK) return rc;
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    collect_timing(r, 1);
    rc = read_status(r);
    if (rc != DDQMC_OK) return rc;
    for (int k = 0; k < NKCLASS; ++k) ms[k] = r->kernel_ms[k];
    return DDQMC_OK;
}

// Candidate shapes: every (blocks per SM, heavy threshold) of the spawn
// kernel and every (blocks per SM, tile) of the radix passes once, paired
// in one trial each, with the merge, partition and compaction shapes cycling.
std::vector<ddqmc_tuning> tune_candidates(const ddqmc_run *r) {
    std::vector<ddqmc_tuning> c;
    c.push_back(r->tune);
    const int heavy[3] = {256, 1024, 4096}, part[3] = {2, 4, 8};
    for (int i = 0; i < 9; ++i) {
        ddqmc_tuning t = r->tune;
        t.spawn_blocks_per_sm = 1 + i % 3;
        t.heavy_walkers = heavy[i / 3];
        t.radix_blocks_per_sm = 1 + i / 3;
        t.radix_records_per_thread = r->packed ? RX_PK_IPT[i % 3] : 0;
        t.merge_blocks_per_sm = 1 + (i + 1) % 3;
        t.partition_blocks_per_sm = part[i % 3];
        t.copy_blocks_per_sm = 2 + 2 * (i % 3);
        t.scan_blocks_per_sm = 1 + (i + 2) % 3;
        c.push_back(t);
    }
    return c;
}

}  // namespace

extern "C" {

int ddqmc_default_options(ddqmc_options *o) {
    if (!o) return DDQMC_ERR_INVALID_ARG;
    o->seed = 1;
    o->damping = 0.05;
    o->shift0 = -1.0;
    o->n0 = 1000;
    o->control = 0;
    o->t_eq = -1;
    o->capacity_entries = 0;
    o->capacity_spawns = 0;
    o->cuda_stream = nullptr;
    o->sm_limit = 0;
    o->field_h = 0.0;
    o->field_axis = 0;
    o->wide_sort_bits = 64;
    o->field_theta = 0.0;
    return DDQMC_OK;
}

int ddqmc_create(const ddqmc_lattice *lattice, double Jx, double Jy, double Jz, double gamma, double dt,
                 int64_t target_walkers, int32_t initiator_threshold, const ddqmc_guide *guide,
                 const ddqmc_options *opt, ddqmc_run **out) {
    if (!out) return DDQMC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!lattice) return DDQMC_ERR_INVALID_ARG;
    ddqmc_options o;
    ddqmc_default_options(&o);
    if (opt) o = *opt;
    ddqmc_run *r = new (std::nothrow) ddqmc_run();
    if (!r) return DDQMC_ERR_OOM;
    int rc = build_params(r, r->hp, lattice, Jx, Jy, Jz, gamma, dt, target_walkers, initiator_threshold, guide, o);
    if (rc != DDQMC_OK) { delete r; return rc; }
    // capacities
    int64_t mcap = o.capacity_entries, rcap = o.capacity_spawns;
    if (mcap <= 0) mcap = default_list_capacity(o.control, target_walkers);
    if (rcap <= 0) rcap = default_spawn_capacity(o.control, target_walkers);
    r->wide = r->hp.N > NPACK;
    r->packed = 2 * r->hp.N <= 32;
    r->p40 = !r->wide && !r->packed && 2 * r->hp.N <= 40;
    rc = setup_device(r, o, mcap, rcap, (size_t)NOBS_MAX * LEVELS);
    if (rc != DDQMC_OK) { free_run(r); return rc; }
    // initial state
    DevState hs;
    initial_state(r->hp, o.shift0, o.n0, hs);
    Rec first;
    first.key = 0;
    first.re = (int32_t)o.n0;
    first.im = 0;
    RecW firstw;
    firstw.lo = 0;
    firstw.hi = bra_swap(0ull, 0ull, r->hp.hash_mask);
    firstw.re = (int32_t)o.n0;
    firstw.im = 0;
    bool okc = cudaMemcpyAsync(r->dP, &r->hp, sizeof(RunParams), cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
    okc = okc && cudaMemcpyAsync(r->dS, &hs, sizeof(DevState), cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
    okc = okc && (r->wide ? cudaMemcpyAsync(r->L[0], &firstw, sizeof(RecW), cudaMemcpyHostToDevice, r->stream)
                          : cudaMemcpyAsync(r->L[0], &first, sizeof(Rec), cudaMemcpyHostToDevice, r->stream)) ==
                  cudaSuccess;
    okc = okc && cudaStreamSynchronize(r->stream) == cudaSuccess;
    if (!okc) { cudaGetLastError(); free_run(r); return DDQMC_ERR_CUDA; }
    r->cur = 0;
    *out = r;
    return DDQMC_OK;
}

int ddqmc_create_batch(const ddqmc_lattice *lattice, int32_t nruns, const ddqmc_run_spec *runs,
                       const ddqmc_guide *guide, const ddqmc_options *opt, ddqmc_run **out) {
    if (!out) return DDQMC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!lattice || !runs || nruns < 1 || nruns > DDQMC_MAX_BATCH) return DDQMC_ERR_INVALID_ARG;
    ddqmc_options o;
    ddqmc_default_options(&o);
    if (opt) o = *opt;
    ddqmc_run *r = new (std::nothrow) ddqmc_run();
    if (!r) return DDQMC_ERR_OOM;
    r->nruns = nruns;
    r->hpr.resize((size_t)nruns);
    int64_t mdef = 0, rdef = 0;
    for (int k = 0; k < nruns; ++k) {
        const ddqmc_run_spec &q = runs[k];
        ddqmc_options ok = o;
        ok.seed = q.seed;
        ok.damping = q.damping;
        ok.shift0 = q.shift0;
        ok.n0 = q.n0;
        ok.control = q.control;
        ok.t_eq = q.t_eq;
        ok.field_h = q.field_h;
        ok.field_axis = q.field_axis;
        ok.field_theta = q.field_theta;
        const int rc = build_params(r, r->hpr[k], lattice, q.Jx, q.Jy, q.Jz, q.gamma, q.dt, q.target_walkers,
                                    q.initiator_threshold, guide, ok);
        if (rc != DDQMC_OK) { delete r; return rc; }
        if (!std::isfinite(q.shift0) || !std::isfinite(q.damping)) { delete r; return DDQMC_ERR_INVALID_ARG; }
        mdef += default_list_capacity(q.control, q.target_walkers);
        rdef += default_spawn_capacity(q.control, q.target_walkers);
    }
    // key layout: the run id above the spin bits (2N of a one-word key, N of the bra word)
    RunParams &H = r->hp;
    H = r->hpr[0];
    const int N = H.N, B = H.B;
    int rbits = 0;
    while ((1ll << rbits) < (int64_t)nruns) ++rbits;
    r->wide = N > NPACK;
    // two-word keys in the hashed order (wide_sort_bits >= 0): the hash takes
    // the low bits of the stored bra word up to the run id, which sits above
    // both the N spin bits and the hash bits, so the runs stay contiguous;
    // the passes cover the stored bra word up to the run id's top bit.  The
    // hash takes at most hb = one digit byte more than the spin and run-id
    // bits fill, for one pass more than the minimum: at the default,
    // hb >= min(N + 8, 64 - run-id bits), and different keys of a run share
    // a stored bra word in about D^2 / 2^(hb + 1) pairs a step for D distinct
    // keys.  The plain order's passes cover the ket word, then the bra word.
    H.hashed = 0;
    H.hash_mask = 0;
    if (r->wide) {
        if (N + rbits > 64 || N >= 64) { delete r; return DDQMC_ERR_UNSUPPORTED; }
        const int nb = (N + 7) / 8, nbb = (N + rbits + 7) / 8;
        if (o.wide_sort_bits >= 0) {
            const int room = 64 - (rbits > 0 ? rbits : 1);      // the run id's shift stays below 64
            const int byte_more = 8 * nbb + 8 - rbits;
            int hb = o.wide_sort_bits;
            if (hb > byte_more) hb = byte_more;
            if (hb > room) hb = room;
            H.hashed = 1;
            H.hash_mask = (1ull << hb) - 1ull;
            H.run_shift = hb > N ? hb : N;
            H.npass = (H.run_shift + rbits + 7) / 8;
            for (int p = 0; p < H.npass; ++p) H.pass_shift[p] = 64 + 8 * p;
        } else {
            H.npass = nb + nbb;
            for (int p = 0; p < H.npass; ++p) H.pass_shift[p] = p < nb ? 8 * p : 64 + 8 * (p - nb);
            H.run_shift = N;
        }
    } else {
        if (2 * N + rbits > 63) { delete r; return DDQMC_ERR_UNSUPPORTED; }
        H.npass = (2 * N + rbits + 7) / 8;
        for (int p = 0; p < H.npass; ++p) H.pass_shift[p] = 8 * p;
        H.run_shift = 2 * N;
    }
    r->packed = 2 * N + rbits <= 32;
    r->p40 = !r->wide && !r->packed && 2 * N + rbits <= 40;
    H.nruns = nruns;
    H.field_on = 0;
    for (int k = 0; k < nruns; ++k) H.field_on |= r->hpr[k].field_on;
    bool axis2 = false;
    for (int k = 0; k < nruns; ++k) axis2 = axis2 || (r->hpr[k].field_on && r->hpr[k].field_axis == 2);
    H.K = 2 * B + N + (H.field_on ? (axis2 ? 4 * N : 2 * N) : 0);
    if (H.K > (N > NPACK ? MAXK : MAXK_PACK)) { delete r; return DDQMC_ERR_UNSUPPORTED; }
    for (int k = 0; k < nruns; ++k) {
        r->hpr[k].nruns = nruns;
        r->hpr[k].run_shift = H.run_shift;
        r->hpr[k].npass = H.npass;
        r->hpr[k].K = H.K;
        r->hpr[k].hashed = H.hashed;
        r->hpr[k].hash_mask = H.hash_mask;
    }
    int64_t mcap = o.capacity_entries > 0 ? o.capacity_entries : mdef;
    int64_t rcap = o.capacity_spawns > 0 ? o.capacity_spawns : rdef;
    int rc = setup_device(r, o, mcap, rcap, (size_t)nruns * H.nobs * LEVELS);
    if (rc != DDQMC_OK) { free_run(r); return rc; }
    rc |= dalloc(&r->dPr, (size_t)nruns);
    rc |= dalloc(&r->dRS, (size_t)nruns);
    if (rc != DDQMC_OK) { free_run(r); return DDQMC_ERR_OOM; }
    // per-run states, the shared counters and the first list (one entry per run with walkers, in run order)
    std::vector<DevState> rs((size_t)nruns);
    DevState ms;
    std::memset(&ms, 0, sizeof(ms));
    ms.epoch = 16;
    std::vector<Rec> first;
    std::vector<RecW> firstw;
    for (int k = 0; k < nruns; ++k) {
        initial_state(r->hpr[k], runs[k].shift0, runs[k].n0, rs[k]);
        if (runs[k].n0 > 0) {
            ms.M += 1;
            ms.W_cur += runs[k].n0;
            Rec e;
            e.key = (uint64_t)k << H.run_shift;
            e.re = (int32_t)runs[k].n0;
            e.im = 0;
            first.push_back(e);
            RecW w;
            w.lo = 0;
            w.hi = r->wide ? bra_swap(0ull, (uint64_t)k << H.run_shift, H.hash_mask) : 0ull;
            w.re = (int32_t)runs[k].n0;
            w.im = 0;
            firstw.push_back(w);
        }
    }
    if (ms.M > r->mcap) { free_run(r); return DDQMC_ERR_CAPACITY; }
    bool okc = cudaMemcpyAsync(r->dP, &H, sizeof(RunParams), cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
    okc = okc && cudaMemcpyAsync(r->dPr, r->hpr.data(), sizeof(RunParams) * (size_t)nruns, cudaMemcpyHostToDevice,
                                 r->stream) == cudaSuccess;
    okc = okc && cudaMemcpyAsync(r->dRS, rs.data(), sizeof(DevState) * (size_t)nruns, cudaMemcpyHostToDevice,
                                 r->stream) == cudaSuccess;
    okc = okc && cudaMemcpyAsync(r->dS, &ms, sizeof(DevState), cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
    if (ms.M > 0)
        okc = okc && (r->wide ? cudaMemcpyAsync(r->L[0], firstw.data(), sizeof(RecW) * firstw.size(),
                                                cudaMemcpyHostToDevice, r->stream)
                              : cudaMemcpyAsync(r->L[0], first.data(), sizeof(Rec) * first.size(),
                                                cudaMemcpyHostToDevice, r->stream)) == cudaSuccess;
    okc = okc && cudaStreamSynchronize(r->stream) == cudaSuccess;
    if (!okc) { cudaGetLastError(); free_run(r); return DDQMC_ERR_CUDA; }
    r->cur = 0;
    *out = r;
    return DDQMC_OK;
}

int ddqmc_step_async(ddqmc_run *r, int64_t nsteps) {
    if (!r || nsteps < 0) return DDQMC_ERR_INVALID_ARG;
    if (r->host_status) return r->host_status;
    return enqueue_steps(r, nsteps);
}

int ddqmc_sync(ddqmc_run *r) {
    if (!r) return DDQMC_ERR_INVALID_ARG;
    return read_status(r);
}

int ddqmc_step(ddqmc_run *r, int64_t nsteps) {
    if (!r || nsteps < 0) return DDQMC_ERR_INVALID_ARG;
    if (r->host_status) return r->host_status;
    // with timing on, steps are issued in batches whose events are folded in after each batch
    const int64_t batch = r->timing ? 256 : nsteps;
    for (int64_t done = 0; done < nsteps || (nsteps == 0 && done == 0); done += batch) {
        const int64_t n = nsteps - done < batch ? nsteps - done : batch;
        int rc = enqueue_steps(r, n);
        if (rc != DDQMC_OK) return rc;
        rc = read_status(r);
        collect_timing(r, n);
        if (rc != DDQMC_OK || nsteps == 0) return rc;
    }
    return DDQMC_OK;
}

int ddqmc_set_timing(ddqmc_run *r, int32_t enable) {
    if (!r) return DDQMC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    r->timing = enable != 0;
    for (int k = 0; k < 8; ++k) { r->kernel_ms[k] = 0.0; r->kernel_launches[k] = 0; }
    return DDQMC_OK;
}

int ddqmc_get_timing(ddqmc_run *r, double *ms, int64_t *launches, int32_t cap) {
    if (!r || cap < 0 || (cap > 0 && (!ms || !launches))) return DDQMC_ERR_INVALID_ARG;
    for (int k = 0; k < cap && k < NKCLASS; ++k) { ms[k] = r->kernel_ms[k]; launches[k] = r->kernel_launches[k]; }
    return DDQMC_OK;
}

int ddqmc_get_totals(ddqmc_run *r, int64_t *walker_steps, int64_t *entry_steps, int64_t *spawn_records,
                     int64_t *merged_entries) {
    if (!r) return DDQMC_ERR_INVALID_ARG;
    DevState hs;
    if (cudaMemcpyAsync(&hs, r->dS, sizeof(DevState), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    if (walker_steps) *walker_steps = hs.walker_steps;
    if (entry_steps) *entry_steps = hs.sum_M;
    if (spawn_records) *spawn_records = hs.sum_R;
    if (merged_entries) *merged_entries = hs.sum_Mnext;
    return DDQMC_OK;
}

int ddqmc_get_state(ddqmc_run *r, ddqmc_state *out) {
    if (!r || !out || r->nruns) return DDQMC_ERR_INVALID_ARG;
    return state_of(r, 0, out);
}

int ddqmc_batch_get_state(ddqmc_run *r, int32_t run, ddqmc_state *out) {
    if (!r || !out || run < 0 || run >= r->nruns) return DDQMC_ERR_INVALID_ARG;
    return state_of(r, run, out);
}


int ddqmc_get_counts(ddqmc_run *r, int64_t *spawn_records, int64_t *capacity_entries, int64_t *capacity_spawns) {
    if (!r) return DDQMC_ERR_INVALID_ARG;
    int64_t R = 0;
    if (cudaMemcpyAsync(&R, &r->dS->R_last, sizeof(R), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    if (spawn_records) *spawn_records = R;
    if (capacity_entries) *capacity_entries = r->mcap;
    if (capacity_spawns) *capacity_spawns = r->rcap;
    return DDQMC_OK;
}

int ddqmc_raw_estimators(ddqmc_run *r, int64_t *host_out, int32_t cap, int32_t *nobs) {
    if (!r || (cap > 0 && !host_out) || r->nruns) return DDQMC_ERR_INVALID_ARG;
    return raw_estimators_of(r, 0, host_out, cap, nobs);
}

int ddqmc_batch_raw_estimators(ddqmc_run *r, int32_t run, int64_t *host_out, int32_t cap, int32_t *nobs) {
    if (!r || (cap > 0 && !host_out) || run < 0 || run >= r->nruns) return DDQMC_ERR_INVALID_ARG;
    return raw_estimators_of(r, run, host_out, cap, nobs);
}

int ddqmc_blocking_moments(ddqmc_run *r, int32_t k, int32_t levels, int64_t *hn, int64_t *hsx, int64_t *hsxx,
                           int64_t *hsxy) {
    if (!r || k < 0 || k >= r->hp.nobs || levels < 0 || levels > LEVELS || r->nruns) return DDQMC_ERR_INVALID_ARG;
    std::vector<BlkCell> cells(LEVELS);
    if (cudaMemcpyAsync(cells.data(), r->dBlk + (size_t)k * LEVELS, sizeof(BlkCell) * LEVELS,
                        cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    for (int l = 0; l < levels; ++l) {
        if (hn) hn[l] = cells[l].n;
        if (hsx) hsx[l] = cells[l].sx;
        if (hsxx) {
            hsxx[2 * l] = (int64_t)(uint64_t)(unsigned __int128)cells[l].sxx;
            hsxx[2 * l + 1] = (int64_t)(uint64_t)((unsigned __int128)cells[l].sxx >> 64);
        }
        if (hsxy) {
            hsxy[2 * l] = (int64_t)(uint64_t)(unsigned __int128)cells[l].sxy;
            hsxy[2 * l + 1] = (int64_t)(uint64_t)((unsigned __int128)cells[l].sxy >> 64);
        }
    }
    return DDQMC_OK;
}

int ddqmc_estimators(ddqmc_run *r, ddqmc_estimates *out) {
    if (!r || !out || r->nruns) return DDQMC_ERR_INVALID_ARG;
    return estimates_of(r, 0, out);
}

int ddqmc_get_tuning(ddqmc_run *r, ddqmc_tuning *out) {
    if (!r || !out) return DDQMC_ERR_INVALID_ARG;
    *out = r->tune;
    return DDQMC_OK;
}

int ddqmc_set_tuning(ddqmc_run *r, const ddqmc_tuning *in) {
    if (!r || !in) return DDQMC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    apply_tuning(r, *in);
    return DDQMC_OK;
}

int ddqmc_tune(ddqmc_run *r, ddqmc_tuning *out) {
    if (!r) return DDQMC_ERR_INVALID_ARG;
    int rc = read_status(r);
    if (rc != DDQMC_OK) return rc;
    TuneBackup b;
    if (cudaMemcpyAsync(&b.st, r->dS, sizeof(DevState), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    if (r->nruns) {
        b.rs.resize((size_t)r->nruns);
        if (cudaMemcpyAsync(b.rs.data(), r->dRS, sizeof(DevState) * (size_t)r->nruns, cudaMemcpyDeviceToHost,
                            r->stream) != cudaSuccess) {
            cudaGetLastError();
            return DDQMC_ERR_CUDA;
        }
    }
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    b.M = b.st.M;
    b.cur = r->cur;
    if (b.M <= 0) return DDQMC_ERR_INVALID_ARG;
    const size_t lsize = r->wide ? sizeof(RecW) : sizeof(Rec);
    if (dalloc_bytes(&b.list, lsize * (size_t)b.M) != DDQMC_OK) return DDQMC_ERR_OOM;
    if (dalloc(&b.blk, r->blk_cells) != DDQMC_OK) { cudaFree(b.list); return DDQMC_ERR_OOM; }
    bool ok = cudaMemcpyAsync(b.list, r->L[b.cur], lsize * (size_t)b.M, cudaMemcpyDeviceToDevice, r->stream) ==
                  cudaSuccess &&
              cudaMemcpyAsync(b.blk, r->dBlk, sizeof(BlkCell) * r->blk_cells, cudaMemcpyDeviceToDevice, r->stream) ==
                  cudaSuccess &&
              cudaStreamSynchronize(r->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(b.list);
        cudaFree(b.blk);
        return DDQMC_ERR_CUDA;
    }
    const bool timing0 = r->timing;
    r->timing = true;
    const std::vector<ddqmc_tuning> cand = tune_candidates(r);
    // per kernel class: best time and the shape that gave it
    const int cls[5] = {KC_SPAWN, KC_RADIX, KC_PARTITION, KC_MERGE, KC_COMPACT};
    double best[5] = {1e300, 1e300, 1e300, 1e300, 1e300};
    ddqmc_tuning pick[5];
    double def_ms = 1e300;
    for (int rep = 0; rep < 2 && rc == DDQMC_OK; ++rep)
        for (size_t i = 0; i < cand.size() && rc == DDQMC_OK; ++i) {
            double ms[NKCLASS] = {0};
            rc = tune_trial(r, b, cand[i], ms);
            if (rc != DDQMC_OK) break;
            double tot = 0.0;                   // the tuned classes (finalize has no shape to tune)
            for (int q = 0; q < 5; ++q) tot += ms[cls[q]];
            if (i == 0 && tot < def_ms) def_ms = tot;
            for (int q = 0; q < 5; ++q)
                if (ms[cls[q]] < best[q]) { best[q] = ms[cls[q]]; pick[q] = r->tune; }
        }
    ddqmc_tuning t = r->tune;
    if (rc == DDQMC_OK) {
        t.spawn_blocks_per_sm = pick[0].spawn_blocks_per_sm;
        t.heavy_walkers = pick[0].heavy_walkers;
        t.radix_blocks_per_sm = pick[1].radix_blocks_per_sm;
        t.radix_records_per_thread = pick[1].radix_records_per_thread;
        t.partition_blocks_per_sm = pick[2].partition_blocks_per_sm;
        t.merge_blocks_per_sm = pick[3].merge_blocks_per_sm;
        t.copy_blocks_per_sm = pick[4].copy_blocks_per_sm;
        t.scan_blocks_per_sm = pick[4].scan_blocks_per_sm;
    } else {
        t = cand[0];
    }
    const int rrc = tune_restore(r, b);
    apply_tuning(r, t);
    r->timing = timing0;
    for (int k = 0; k < 8; ++k) { r->kernel_ms[k] = 0.0; r->kernel_launches[k] = 0; }
    cudaFree(b.list);
    cudaFree(b.blk);
    if (rc != DDQMC_OK) return rc;
    if (rrc != DDQMC_OK) return rrc;
    double tuned = 0.0;
    for (int q = 0; q < 5; ++q) tuned += best[q];
    r->tune.step_ms_default = def_ms;
    r->tune.step_ms_tuned = tuned;
    cache_tuning(r, r->tune);
    if (out) *out = r->tune;
    return DDQMC_OK;
}

int ddqmc_batch_retire(ddqmc_run *r, int32_t run) {
    if (!r || r->nruns == 0 || run < 0 || run >= r->nruns) return DDQMC_ERR_INVALID_ARG;
    r->hpr[(size_t)run].active = 0;
    // ordered on the batch's stream before every later step (the captured
    // graphs read the parameters from device memory when they run)
    if (cudaMemcpyAsync(&r->dPr[run].active, &r->hpr[(size_t)run].active, sizeof(int32_t), cudaMemcpyHostToDevice,
                        r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    return DDQMC_OK;
}

int ddqmc_batch_estimators(ddqmc_run *r, int32_t run, ddqmc_estimates *out) {
    if (!r || !out || run < 0 || run >= r->nruns) return DDQMC_ERR_INVALID_ARG;
    return estimates_of(r, run, out);
}


int ddqmc_export_walkers(ddqmc_run *r, uint64_t *ket, uint64_t *bra, int32_t *re, int32_t *im, int64_t cap,
                         int64_t *n) {
    if (!r || !n || (cap > 0 && (!ket || !bra || !re || !im)) || r->nruns) return DDQMC_ERR_INVALID_ARG;
    return export_of(r, -1, ket, bra, re, im, cap, n);
}

int ddqmc_batch_export_walkers(ddqmc_run *r, int32_t run, uint64_t *ket, uint64_t *bra, int32_t *re, int32_t *im,
                               int64_t cap, int64_t *n) {
    if (!r || !n || (cap > 0 && (!ket || !bra || !re || !im)) || run < 0 || run >= r->nruns)
        return DDQMC_ERR_INVALID_ARG;
    return export_of(r, run, ket, bra, re, im, cap, n);
}

// The imported list (n entries, W walkers) in the spare buffer becomes the
// current one, with the given step state; the look-back epoch keeps counting,
// so that no status word left by an earlier step can match a later one.
int finish_import(ddqmc_run *r, int64_t n, int64_t W, uint32_t old_epoch, int64_t t, double S, int32_t variable,
                  int64_t q_prev, int64_t t_var, int64_t t_eq) {
    r->cur ^= 1;
    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.t = t;
    hs.S = S;
    hs.variable = variable ? 1 : 0;
    hs.q_prev = q_prev;
    hs.t_var = t_var;
    hs.t_eq = t_eq;
    hs.M = n;
    hs.W_cur = W;
    hs.epoch = (old_epoch + 16u) & 0x3FFFFFFFu;
    host_death_table(r->hp, S, hs);
    bool ok = cudaMemcpyAsync(r->dS, &hs, sizeof(DevState), cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(r->dBlk, 0, sizeof(BlkCell) * (size_t)NOBS_MAX * LEVELS, r->stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(r->stream) == cudaSuccess;
    if (!ok) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    r->host_status = 0;
    return DDQMC_OK;
}

int ddqmc_import_walkers(ddqmc_run *r, const uint64_t *ket, const uint64_t *bra, const int32_t *re,
                         const int32_t *im, int64_t n, int64_t t, double S, int32_t variable, int64_t q_prev,
                         int64_t t_var, int64_t t_eq) {
    if (!r || n < 0 || (n > 0 && (!ket || !bra || !re || !im)) || t < 0 || !std::isfinite(S))
        return DDQMC_ERR_INVALID_ARG;
    if (r->nruns) return DDQMC_ERR_UNSUPPORTED;
    if (n > r->mcap || (r->hp.hashed && n > r->rcap)) return DDQMC_ERR_CAPACITY;
    const int N = r->hp.N;
    const uint64_t mask = r->hp.nmask;
    // the caller's arrays go over the link as they are, one copy each; the
    // device checks and packs them into the spare list buffer, so a rejected
    // list leaves the run as it was
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    unsigned char *d = soa_scratch(r, n > 0 ? n : 1);
    if (!d) return DDQMC_ERR_OOM;
    int64_t W = 0;
    uint32_t old_epoch = 0;
    {
        const int64_t m = n > 0 ? n : 1;
        uint64_t *dk = reinterpret_cast<uint64_t *>(d), *db = dk + m;
        int32_t *dr = reinterpret_cast<int32_t *>(db + m), *di = dr + m;
        unsigned long long acc[2] = {0ull, 0ull};
        bool ok = cudaMemsetAsync(r->dxfer, 0, 2 * sizeof(unsigned long long), r->stream) == cudaSuccess;
        if (n > 0) {
            ok = ok && cudaMemcpyAsync(dk, ket, 8 * (size_t)n, cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
            ok = ok && cudaMemcpyAsync(db, bra, 8 * (size_t)n, cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
            ok = ok && cudaMemcpyAsync(dr, re, 4 * (size_t)n, cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
            ok = ok && cudaMemcpyAsync(di, im, 4 * (size_t)n, cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
            // a hashed-order list is packed into Sp[0] and sorted into the spare buffer below
            if (r->wide)
                k_import_pack<RecW><<<grid_for(n), TX_TPB, 0, r->stream>>>(
                    dk, db, dr, di, n, N, mask, r->hp.hash_mask,
                    reinterpret_cast<RecW *>(r->hp.hashed ? r->Sp[0] : r->L[r->cur ^ 1]), r->dxfer);
            else
                k_import_pack<Rec><<<grid_for(n), TX_TPB, 0, r->stream>>>(
                    dk, db, dr, di, n, N, mask, 0ull, reinterpret_cast<Rec *>(r->L[r->cur ^ 1]), r->dxfer);
            ok = ok && cudaGetLastError() == cudaSuccess;
        }
        // the look-back epoch keeps counting, so that no status word left by
        // an earlier step can match a later one
        ok = ok && cudaMemcpyAsync(acc, r->dxfer, sizeof(acc), cudaMemcpyDeviceToHost, r->stream) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(&old_epoch, &r->dS->epoch, sizeof(old_epoch), cudaMemcpyDeviceToHost,
                                   r->stream) == cudaSuccess;
        ok = ok && cudaStreamSynchronize(r->stream) == cudaSuccess;
        if (!ok) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
        if (acc[1]) return DDQMC_ERR_INVALID_ARG;
        W = (int64_t)acc[0];
        if (r->hp.hashed && n > 0) {
            RecW *srt = nullptr;
            const int rc = sort_records_wide(r, n, r->hp.npass, 0, true, &srt);
            if (rc != DDQMC_OK) return rc;
            if (cudaMemcpyAsync(r->L[r->cur ^ 1], srt, sizeof(RecW) * (size_t)n, cudaMemcpyDeviceToDevice,
                                r->stream) != cudaSuccess) {
                cudaGetLastError();
                return DDQMC_ERR_CUDA;
            }
        }
    }
    return finish_import(r, n, W, old_epoch, t, S, variable, q_prev, t_var, t_eq);
}

int ddqmc_export_records(ddqmc_run *r, void *host_records, int64_t cap, int64_t *n) {
    if (!r || !n || cap < 0 || (cap > 0 && !host_records) || ((uintptr_t)host_records & 7u)) return DDQMC_ERR_INVALID_ARG;
    if (r->nruns || r->wide) return DDQMC_ERR_UNSUPPORTED;
    int64_t M = 0;
    if (cudaMemcpyAsync(&M, &r->dS->M, sizeof(M), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    *n = M;
    const int64_t m = M < cap ? M : cap;
    if (m <= 0) return DDQMC_OK;
    if (cudaMemcpyAsync(host_records, r->L[r->cur], sizeof(Rec) * (size_t)m, cudaMemcpyDeviceToHost, r->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    return DDQMC_OK;
}

int ddqmc_import_records(ddqmc_run *r, const void *host_records, int64_t n, int64_t t, double S, int32_t variable,
                         int64_t q_prev, int64_t t_var, int64_t t_eq) {
    if (!r || n < 0 || (n > 0 && !host_records) || ((uintptr_t)host_records & 7u) || t < 0 || !std::isfinite(S))
        return DDQMC_ERR_INVALID_ARG;
    if (r->nruns || r->wide) return DDQMC_ERR_UNSUPPORTED;
    if (n > r->mcap) return DDQMC_ERR_CAPACITY;
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    if (!soa_scratch(r, 1)) return DDQMC_ERR_OOM;
    // straight into the spare list buffer, checked there (a rejected list
    // leaves the run as it was)
    unsigned long long acc[2] = {0ull, 0ull};
    uint32_t old_epoch = 0;
    const int kbits = 2 * r->hp.N;
    bool ok = cudaMemsetAsync(r->dxfer, 0, 2 * sizeof(unsigned long long), r->stream) == cudaSuccess;
    if (n > 0) {
        ok = ok && cudaMemcpyAsync(r->L[r->cur ^ 1], host_records, sizeof(Rec) * (size_t)n, cudaMemcpyHostToDevice,
                                   r->stream) == cudaSuccess;
        k_check_records<<<grid_for(n), TX_TPB, 0, r->stream>>>(reinterpret_cast<const Rec *>(r->L[r->cur ^ 1]), n,
                                                                kbits >= 64 ? ~0ull : (1ull << kbits) - 1ull,
                                                                r->dxfer);
        ok = ok && cudaGetLastError() == cudaSuccess;
    }
    ok = ok && cudaMemcpyAsync(acc, r->dxfer, sizeof(acc), cudaMemcpyDeviceToHost, r->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(&old_epoch, &r->dS->epoch, sizeof(old_epoch), cudaMemcpyDeviceToHost, r->stream) ==
                   cudaSuccess;
    ok = ok && cudaStreamSynchronize(r->stream) == cudaSuccess;
    if (!ok) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    if (acc[1]) return DDQMC_ERR_INVALID_ARG;
    return finish_import(r, n, (int64_t)acc[0], old_epoch, t, S, variable, q_prev, t_var, t_eq);
}

int ddqmc_export_records32(ddqmc_run *r, void *host_records, int64_t cap, int64_t *n) {
    if (!r || !n || cap < 0 || (cap > 0 && !host_records) || ((uintptr_t)host_records & 3u)) return DDQMC_ERR_INVALID_ARG;
    if (r->nruns || 2 * r->hp.N > 32) return DDQMC_ERR_UNSUPPORTED;
    int64_t M = 0;
    if (cudaMemcpyAsync(&M, &r->dS->M, sizeof(M), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    *n = M;
    const int64_t m = M < cap ? M : cap;
    if (m <= 0) return DDQMC_OK;
    unsigned char *d = soa_scratch(r, m);
    if (!d) return DDQMC_ERR_OOM;
    k_pack_records32<<<grid_for(m), TX_TPB, 0, r->stream>>>(reinterpret_cast<const Rec *>(r->L[r->cur]), m,
                                                             reinterpret_cast<uint32_t *>(d));
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(host_records, d, 12 * (size_t)m, cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    return DDQMC_OK;
}

int ddqmc_import_records32(ddqmc_run *r, const void *host_records, int64_t n, int64_t t, double S, int32_t variable,
                           int64_t q_prev, int64_t t_var, int64_t t_eq) {
    if (!r || n < 0 || (n > 0 && !host_records) || ((uintptr_t)host_records & 3u) || t < 0 || !std::isfinite(S))
        return DDQMC_ERR_INVALID_ARG;
    if (r->nruns || 2 * r->hp.N > 32) return DDQMC_ERR_UNSUPPORTED;
    if (n > r->mcap) return DDQMC_ERR_CAPACITY;
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    unsigned char *d = soa_scratch(r, n > 0 ? n : 1);
    if (!d) return DDQMC_ERR_OOM;
    // over the link into scratch, unpacked and checked into the spare list
    // buffer (a rejected list leaves the run as it was)
    unsigned long long acc[2] = {0ull, 0ull};
    uint32_t old_epoch = 0;
    const int kbits = 2 * r->hp.N;
    bool ok = cudaMemsetAsync(r->dxfer, 0, 2 * sizeof(unsigned long long), r->stream) == cudaSuccess;
    if (n > 0) {
        ok = ok && cudaMemcpyAsync(d, host_records, 12 * (size_t)n, cudaMemcpyHostToDevice, r->stream) == cudaSuccess;
        k_unpack_records32<<<grid_for(n), TX_TPB, 0, r->stream>>>(reinterpret_cast<const uint32_t *>(d), n,
                                                                   kbits >= 64 ? ~0ull : (1ull << kbits) - 1ull,
                                                                   reinterpret_cast<Rec *>(r->L[r->cur ^ 1]),
                                                                   r->dxfer);
        ok = ok && cudaGetLastError() == cudaSuccess;
    }
    ok = ok && cudaMemcpyAsync(acc, r->dxfer, sizeof(acc), cudaMemcpyDeviceToHost, r->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(&old_epoch, &r->dS->epoch, sizeof(old_epoch), cudaMemcpyDeviceToHost, r->stream) ==
                   cudaSuccess;
    ok = ok && cudaStreamSynchronize(r->stream) == cudaSuccess;
    if (!ok) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    if (acc[1]) return DDQMC_ERR_INVALID_ARG;
    return finish_import(r, n, (int64_t)acc[0], old_epoch, t, S, variable, q_prev, t_var, t_eq);
}

int ddqmc_annihilate(ddqmc_run *r, const void *d_list, int64_t m, const void *d_spawns, int64_t nsp, void *d_out,
                     int64_t out_cap, int64_t *m_out) {
    if (!r || !m_out || m < 0 || nsp < 0 || out_cap < 0 || (m > 0 && !d_list) || (nsp > 0 && !d_spawns) ||
        (out_cap > 0 && !d_out) || !records_aligned(d_list, d_spawns, d_out))
        return DDQMC_ERR_INVALID_ARG;
    *m_out = 0;
    if (r->hp.N > NPACK || r->nruns) return DDQMC_ERR_UNSUPPORTED;   // one-word keys of a single run only
    if (nsp > r->rcap || m > r->mcap) return DDQMC_ERR_CAPACITY;
    if (!r->dAnn && dalloc(&r->dAnn, 1) != DDQMC_OK) return DDQMC_ERR_OOM;
    const RunParams &P = r->hp;
    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.M = m;
    hs.R = nsp;
    // epochs of standalone calls carry bit 29, those of the run's steps do not
    hs.epoch = (1u << 29) | ((r->ann_calls++ * 16u) & ((1u << 29) - 1u));
    if (cudaMemcpyAsync(r->dAnn, &hs, sizeof(DevState), cudaMemcpyHostToDevice, r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    const Rec *list = (const Rec *)d_list;
    const Rec *sp = (const Rec *)d_spawns;
    k_digit_histogram<Rec><<<r->g_part, RX_TPB, 0, r->stream>>>(sp, r->dAnn, P.npass, P.npass);
    const Rec *src = sp;
    for (int p = 0; p < P.npass; ++p) {
        Rec *dst = reinterpret_cast<Rec *>(r->Sp[p & 1]);
        k_radix_pass<Rec><<<r->g_radix_wide, RX_TPB, RX_SMEM, r->stream>>>(src, dst, r->dAnn, r->lb_radix, p, 8 * p,
                                                                          r->rcap);
        src = dst;
    }
    k_merge_partition<Rec><<<r->g_part, 256, 0, r->stream>>>(list, src, r->dAnn, r->splits, r->rem_end, r->rcap);
    k_merge<Rec, false><<<r->g_merge_ann, MG_TPB, MG_SMEM, r->stream>>>(r->dP, list, src, (Rec *)r->slots,
                                                                        r->tile_counts, r->dAnn, r->splits,
                                                                        r->rem_end, r->rcap, r->dP, r->dAnn);
    k_merge_scan<<<r->g_scan, MC_TPB, 0, r->stream>>>(r->tile_counts, r->splits, r->dAnn, r->lb_merge, r->rcap,
                                                      out_cap);
    k_merge_copy<Rec><<<r->g_copy_ann, MC_TPB, 0, r->stream>>>((const Rec *)r->slots, r->tile_counts, r->splits,
                                                               (Rec *)d_out, r->dAnn, r->rcap);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hs, r->dAnn, sizeof(DevState), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
        cudaStreamSynchronize(r->stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    *m_out = hs.M_next;
    return status_code(hs.status);
}

int ddqmc_annihilate_noalloc(const ddqmc_lattice *lattice, int32_t initiator_threshold, const void *d_list,
                             int64_t m, const void *d_spawns, int64_t nsp, void *d_out, int64_t out_cap,
                             int64_t *m_out, void *cuda_stream) {
    if (!lattice || !m_out || m < 0 || nsp < 0 || out_cap < 0 || (m > 0 && !d_list) || (nsp > 0 && !d_spawns) ||
        (out_cap > 0 && !d_out) || !records_aligned(d_list, d_spawns, d_out))
        return DDQMC_ERR_INVALID_ARG;
    *m_out = 0;
    if (nsp > NA_MAX_SPAWNS || m > NA_MAX_LIST) return DDQMC_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    int rc = noalloc_setup(dev);
    if (rc != DDQMC_OK) return rc;
    NoAllocScratch *sc = g_na_ptr[dev];
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // lattice tables (host only; couplings do not enter the annihilation)
    ddqmc_run host_ctx;
    ddqmc_options o;
    ddqmc_default_options(&o);
    rc = build_params(&host_ctx, host_ctx.hp, lattice, 0.0, 0.0, 0.0, 0.0, 1.0, 1, initiator_threshold, nullptr, o);
    if (rc != DDQMC_OK) return rc;
    const RunParams &P = host_ctx.hp;
    if (P.N > NPACK) return DDQMC_ERR_UNSUPPORTED;           // 16-byte records hold one-word keys only
    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.M = m;
    hs.R = nsp;
    hs.epoch = 16;
    // clear what must start at zero: counters, histograms, tickets, look-back words
    bool ok = cudaMemcpyAsync(&sc->P, &P, sizeof(RunParams), cudaMemcpyHostToDevice, stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(&sc->st, &hs, sizeof(DevState), cudaMemcpyHostToDevice, stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(sc->lb_radix, 0, sizeof(sc->lb_radix), stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(sc->lb_merge, 0, sizeof(sc->lb_merge), stream) == cudaSuccess;
    if (!ok) { cudaGetLastError(); return DDQMC_ERR_CUDA; }
    const Rec *list = (const Rec *)d_list;
    const Rec *src = (const Rec *)d_spawns;
    k_digit_histogram<Rec><<<g_na_grid[dev][1], RX_TPB, 0, stream>>>(src, &sc->st, P.npass, P.npass);
    for (int p = 0; p < P.npass; ++p) {
        Rec *dst = sc->buf[p & 1];
        k_radix_pass<Rec><<<g_na_grid[dev][0], RX_TPB, RX_SMEM, stream>>>(src, dst, &sc->st, sc->lb_radix, p, 8 * p,
                                                                           NA_MAX_SPAWNS);
        src = dst;
    }
    k_merge_partition<Rec><<<g_na_grid[dev][1], 256, 0, stream>>>(list, src, &sc->st, sc->splits, sc->rem_end,
                                                                   NA_MAX_SPAWNS);
    k_merge<Rec, false><<<g_na_grid[dev][2], MG_TPB, MG_SMEM, stream>>>(&sc->P, list, src, sc->slots, sc->counts,
                                                                        &sc->st, sc->splits, sc->rem_end,
                                                                        NA_MAX_SPAWNS, &sc->P, &sc->st);
    k_merge_scan<<<g_na_grid[dev][1], MC_TPB, 0, stream>>>(sc->counts, sc->splits, &sc->st, sc->lb_merge,
                                                           NA_MAX_SPAWNS, out_cap);
    k_merge_copy<Rec><<<g_na_grid[dev][3], MC_TPB, 0, stream>>>(sc->slots, sc->counts, sc->splits, (Rec *)d_out,
                                                                &sc->st, NA_MAX_SPAWNS);
    int64_t mo = 0;
    uint32_t status = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&mo, &sc->st.M_next, sizeof(mo), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaMemcpyAsync(&status, &sc->st.status, sizeof(status), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    *m_out = mo;
    return status_code(status);
}

// A look-back word that nothing ever publishes, and the status its bounded
// wait reports: the failure path of every device wait, exercised on purpose.
static __device__ uint64_t g_wait_word;
static __device__ uint32_t g_wait_status;

static __global__ void k_wait_selftest(uint32_t epoch) {
    if (threadIdx.x == 0) {
        g_wait_status = 0u;
        lb_wait(&g_wait_word, epoch, &g_wait_status);
    }
}

int ddqmc_wait_selftest(void *cuda_stream) {
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    uint32_t st = 0;
    k_wait_selftest<<<1, 32, 0, stream>>>(12345u);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyFromSymbolAsync(&st, g_wait_status, sizeof(st), 0, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return DDQMC_ERR_CUDA;
    }
    return status_code(st);
}

void ddqmc_destroy(ddqmc_run *r) {
    if (!r) return;
    if (r->stream) cudaStreamSynchronize(r->stream);
    free_run(r);
}

const char *ddqmc_strerror(int status) {
    switch (status) {
        case DDQMC_OK: return "success";
        case DDQMC_ERR_INVALID_ARG: return "invalid argument";
        case DDQMC_ERR_OOM: return "out of memory";
        case DDQMC_ERR_CAPACITY: return "walker list or spawn buffer capacity exceeded";
        case DDQMC_ERR_OVERFLOW: return "walker population left the int32 range";
        case DDQMC_ERR_TIMEOUT: return "a bounded device wait timed out";
        case DDQMC_ERR_CUDA: return "CUDA runtime error";
        case DDQMC_ERR_UNSUPPORTED: return "unsupported size (more than 31 sites)";
        default: return "unknown status";
    }
}

}  // extern "C"
