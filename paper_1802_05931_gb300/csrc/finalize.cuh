// End of a DDQMC step, one thread block per run: shift update (Sec. III.C), death /
// clone table for the next step, device-resident blocking accumulators of
// the estimator numerators (Sec. III.A time averages), and the resets that
// let the next step's kernels run without any host involvement.
#pragma once

#include "common.cuh"

namespace ddq {

constexpr int FN_TPB = 256;

// death / clone thresholds for p_c = dt ((gamma/2) c + S), c = n(i) + n(j)
__device__ __forceinline__ void death_entry(const RunParams &P, double S, int c, DevState *st) {
    const double a = __dmul_rn(P.gamma_half, (double)c);
    const double b = __dadd_rn(a, S);
    const double p = __dmul_rn(P.dt, b);
    const double ap = fabs(p);
    const double ip = floor(ap);
    st->d_int[c] = (uint32_t)ip;
    st->d_frac[c] = (uint64_t)__dmul_rn(__dsub_rn(ap, ip), 4294967296.0);
    st->d_sgn[c] = p > 0.0 ? 1 : (p < 0.0 ? -1 : 0);
}

// BATCH: one block per run r, with Pp = the runs' parameters, rs[r] the run's
// state and blocking cells at blk + r * nobs * LEVELS; block 0 also resets
// the shared step counters in st.  A single run: one block, rs = st.
template <bool BATCH>
__global__ void __launch_bounds__(FN_TPB)
k_finalize(const RunParams *__restrict__ Pp, DevState *__restrict__ st, BlkCell *__restrict__ blk,
           DevState *__restrict__ rs) {
    const int run = BATCH ? (int)blockIdx.x : 0;
    const RunParams &P = Pp[run];
    DevState *R = BATCH ? rs + run : st;         // the run's own state
    const bool machine = !BATCH || run == 0;     // this block resets the step counters
    __shared__ int64_t s_est[NOBS_MAX];
    __shared__ int s_append;
    __shared__ double s_S;
    const int tid = threadIdx.x;
    if (block_stopped(st)) return;
    const int N = P.N, B = P.B, nobs = P.nobs;
    // layout: [0, 5) totals, z per site, zz / xx / yy per bond, their 4 sums,
    // x and y per site, their 2 sums (the sums are formed here)
    const int core = 5 + N + 3 * B;
    const int ox = core + 4, oy = ox + N;
    for (int q = tid; q < nobs; q += FN_TPB) s_est[q] = R->est[q];
    __syncthreads();
    if (tid == 0) {
        int64_t sz = 0, szz = 0, sxx = 0, syy = 0, sx = 0, sy = 0;
        for (int k = 0; k < N; ++k) sz += s_est[5 + k];
        for (int b = 0; b < B; ++b) {
            szz += s_est[5 + N + b];
            sxx += s_est[5 + N + B + b];
            syy += s_est[5 + N + 2 * B + b];
        }
        for (int k = 0; k < N; ++k) {
            sx += s_est[ox + k];
            sy += s_est[oy + k];
        }
        s_est[core + 0] = sz;
        s_est[core + 1] = szz;
        s_est[core + 2] = sxx;
        s_est[core + 3] = syy;
        s_est[oy + N] = sx;
        s_est[oy + N + 1] = sy;
        // shift update on the controlled weight
        const int64_t Q = P.control == 0 ? s_est[2] : s_est[3];
        double S = R->S;
        if (R->variable) {
            if (Q > 0 && R->q_prev > 0) {
                const double ratio = __ddiv_rn((double)Q, (double)R->q_prev);
                S = __dadd_rn(S, __dmul_rn(P.shift_gain, series_log(ratio)));
            }
        } else if (Q >= P.target) {
            R->variable = 1;
            R->t_var = R->t + 1;
            R->t_eq = R->t_var + P.t_eq_span;
        }
        R->S = S;
        R->q_prev = Q;
        if (BATCH) {
            // the run's own totals; the batch's walker-steps are the sum over runs
            atomicAdd((unsigned long long *)&st->walker_steps, (unsigned long long)R->W_cur);
            R->walker_steps += R->W_cur;
            R->sum_M += R->M;
            R->M = s_est[4];
        } else {
            R->walker_steps += R->W_cur;
        }
        R->W_cur = s_est[3];
        R->t += 1;
        if (machine) {
            st->sum_M += st->M;
            st->sum_R += st->R;
            st->sum_Mnext += st->M_next;
            if (BATCH) st->t += 1;
            st->M = st->M_next;
            st->M_next = 0;
            st->R_last = st->R;
            st->R = 0;
            st->hviol = 0;
            st->epoch = (st->epoch + 16u) & 0x3FFFFFFFu;
        }
        s_S = S;
        s_append = (R->variable && R->t >= R->t_eq) ? 1 : 0;
        if (s_append) R->n_app += 1;
    }
    __syncthreads();
    for (int q = tid; q < nobs; q += FN_TPB) {
        R->last_est[q] = s_est[q];
        R->est[q] = 0;
    }
    if (machine) {
        for (int q = tid; q < MAXPASS + 16; q += FN_TPB) st->tickets[q] = 0u;
        for (int q = tid; q < MAXPASS * 256; q += FN_TPB) (&st->hist[0][0])[q] = 0u;
    }
    if (tid <= 2 * N) death_entry(P, s_S, tid, R);
    BlkCell *rcells = blk + (size_t)run * nobs * LEVELS;
    for (int q = tid; s_append && q < nobs; q += FN_TPB) {
        // binary-counter cascade of block sums for observable q against the trace
        int64_t x = s_est[q], y = s_est[0];
        BlkCell *cells = rcells + (size_t)q * LEVELS;
        for (int l = 0; l < LEVELS; ++l) {
            BlkCell &c = cells[l];
            c.n += 1;
            c.sx += x;
            c.sxx += (__int128)x * (__int128)x;
            c.sxy += (__int128)x * (__int128)y;
            if (!c.has_pend) {
                c.pend_x = x;
                c.pend_y = y;
                c.has_pend = 1;
                break;
            }
            x += c.pend_x;
            y += c.pend_y;
            c.has_pend = 0;
        }
    }
}

}  // namespace ddq
