// The integer fulfilment policies (greedy and bid-price) on one warp: replay of
// one Picard segment and the sequential simulation, shared by the
// single-trajectory and batch kernels.
#pragma once

#include "pic_picard.cuh"

namespace pic {
namespace picard {

// Replay one segment (all its runs, in order) with one warp.  Lane l owns
// warehouses l, l+32, ..., l+32(NPL-1).  fcp: first position of product k that
// changed in the previous pass (-1: every run is evaluated).
//
// Per run the state starts at max(0, x0 - D), D = counts of cached actions of
// this product before the run.  The walk keeps E = D + the run's actions so far
// per warehouse, and the stock is max(0, x0 - E): a warehouse at or below zero
// at the run's start is never chosen, so the clamp commutes with the run's
// decrements, and a warehouse has stock iff E < x0.  At a run's end E takes
// the correction for the orders whose new action differs from the cached one
// (rare once the iteration settles) and is the next run's D.
template <int NPL, bool DUAL, bool SMEM, bool FULL>
__device__ __forceinline__ bool replay_segment(const KArgs& a, const CostTable<SMEM>& ct, int s,
                                               const SegMeta& m, int fcp, int* fc_cur, int it,
                                               bool use_lam, unsigned long long& calls) {
    const int lane = lane_id();
    const int N = a.N, NP = a.NP;
    const int k = m.k;
    // key = score * 128 + n (ties to the lowest index); adj = n - 128 * lam[k][n]
    int D0[NPL], E[NPL], x0v[NPL], adj[NPL], corr[NPL], ctot[NPL];
    // prefix counts from earlier segments of this product (exclusive chain
    // prefix); none before pass 1 of an all-a^phi cache
    const bool chained = m.ce - m.cf > 1 && (it > 1 || a.first_dirty);
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        const bool in = FULL || n < N;
        corr[i] = 0;
        ctot[i] = 0;
        x0v[i] = in ? a.x0[(size_t)k * N + n] : 0;
        adj[i] = n - ((DUAL && use_lam && in) ? 128 * a.lam[(size_t)k * N + n] : 0);
        D0[i] = chained ? chain_prefix(a, s, m.cf, n) : 0;
        E[i] = D0[i];
    }
    const int j0 = m.j0, jend = m.jend;
    // Runs starting at or before fcp keep their cached actions (t_reset), so
    // walking them only advances D by the counts of those actions: without the
    // max_steps window they are skipped, and the counts taken in parallel (each
    // lane tallies its own warehouses over 32 cached actions at a time).
    int jst = j0, rst = m.r0;  // first position and run walked
    if (!a.run_chunk && j0 <= fcp) {
        int rs = m.r1;  // first run starting after fcp
        for (int w = m.r0 + 1; w < m.r1; w += 32) {
            const int st = w + lane < m.r1 ? a.run_start[w + lane] : INT_MAX;
            const unsigned b = __ballot_sync(kFull, st > fcp);
            if (b) {
                rs = w + __ffs(b) - 1;
                break;
            }
        }
        if (rs < m.r1) {
            rst = rs;
            jst = a.run_start[rs];
            int cnt[NPL];
#pragma unroll
            for (int i = 0; i < NPL; ++i) cnt[i] = 0;
            int v = j0 + lane < jst ? a.alpha_s[j0 + lane] : -1;
            for (int p = j0; p < jst; p += 32) {
                const int u = v;
                v = p + 32 + lane < jst ? a.alpha_s[p + 32 + lane] : -1;
#pragma unroll 8
                for (int q = 0; q < 32; ++q) {
                    const int aq = __shfl_sync(kFull, u, q);
#pragma unroll
                    for (int i = 0; i < NPL; ++i) cnt[i] += aq == lane + 32 * i;
                }
            }
#pragma unroll
            for (int i = 0; i < NPL; ++i) E[i] += cnt[i];
        }
    }
    // lane i holds the end (= next start) of run rwin + i
    int rwin = rst;
    int run_end = lane < m.r1 - rwin ? a.run_start[rwin + 1 + lane] : INT_MAX;
    int r = rst;
    int next_run = __shfl_sync(kFull, run_end, 0);
    // the max_steps window of this pass (none: INT_MAX)
    const int whi = a.run_chunk ? ld_volatile(&a.ctrl->win_hi) : INT_MAX;
    const int wprev = a.run_chunk ? ld_volatile(&a.ctrl->win_hi_prev) : INT_MAX;
    // this run's prefix changed in the previous pass (or it entered the window)
    bool eval = run_evaluated(a, whi, wprev, r, jst > fcp);
    unsigned long long evals = eval ? (unsigned long long)(next_run - jst) : 0ull;
    int first_chg = INT_MAX;
    int nreg = 0, nold = -1;
    if (lane < jend - jst) {
        nreg = a.reg_s[jst + lane];
        nold = a.alpha_s[jst + lane];
    }
    for (int base = jst; base < jend; base += 32) {
        const int cnt = min(32, jend - base);
        const int my_reg = nreg, my_old = nold;
        if (base + 32 + lane < jend) {  // prefetch the next batch of orders
            nreg = a.reg_s[base + 32 + lane];
            nold = a.alpha_s[base + 32 + lane];
        }
        int my_new = my_old;
        // order q's region, cached action and cost row are read during order q - 1,
        // off the loop-carried chain (stock -> decision -> stock)
        int rr_n = __shfl_sync(kFull, my_reg, 0), ao_n = __shfl_sync(kFull, my_old, 0);
        int c_n[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i)
            c_n[i] = (FULL || lane + 32 * i < N) ? ct.at(rr_n, lane + 32 * i) : 0;
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
            const int ao = ao_n;
            int c[NPL];
#pragma unroll
            for (int i = 0; i < NPL; ++i) c[i] = c_n[i];
            // lanes at or past cnt hold an earlier batch's (valid) region: read, unused
            const int q1 = q + 1 < 32 ? q + 1 : q;
            rr_n = __shfl_sync(kFull, my_reg, q1);
            ao_n = __shfl_sync(kFull, my_old, q1);
#pragma unroll
            for (int i = 0; i < NPL; ++i)
                c_n[i] = (FULL || lane + 32 * i < N) ? ct.at(rr_n, lane + 32 * i) : 0;
            if (base + q == next_run) {  // close run r, open run r+1
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    E[i] += corr[i];
                    ctot[i] += corr[i];
                    corr[i] = 0;
                }
                ++r;
                int idx = r - rwin;
                if (idx == 32) {  // next window of run ends
                    rwin += 32;
                    idx = 0;
                    run_end = lane < m.r1 - rwin ? a.run_start[rwin + 1 + lane] : INT_MAX;
                }
                const int nr = __shfl_sync(kFull, run_end, idx);
                eval = run_evaluated(a, whi, wprev, r, next_run > fcp);
                if (eval) evals += (unsigned long long)(nr - next_run);
                next_run = nr;
            }
            int act = ao;  // unchanged prefix: the cached action is the policy's
            if (eval) {
                int key = INT_MAX;
#pragma unroll
                for (int i = 0; i < NPL; ++i)
                    key = min(key, E[i] < x0v[i] ? c[i] * 128 + adj[i] : INT_MAX);
                const int best = __reduce_min_sync(kFull, key);
                act = best == INT_MAX ? -1 : (best & 127);
            }
#pragma unroll
            for (int i = 0; i < NPL; ++i) E[i] += (act == lane + 32 * i);
            if (act != ao) {  // warp-uniform: the cached action was not the new one
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    corr[i] += (ao == lane + 32 * i);
                    corr[i] -= (act == lane + 32 * i);
                }
            }
            if (lane == q) my_new = act;
        }
        if (lane < cnt) a.alpha_s[base + lane] = (int8_t)my_new;
        const unsigned chg = __ballot_sync(kFull, lane < cnt && my_new != my_old);
        if (chg && first_chg == INT_MAX) first_chg = base + __ffs(chg) - 1;
    }
    // the segment's histogram of actions: skipped runs' cached ones and the
    // evaluated runs' new ones, without the corrections applied to E
#pragma unroll
    for (int i = 0; i < NPL; ++i) a.agg[(size_t)s * NP + lane + 32 * i] = E[i] - D0[i] - ctot[i];
    if (lane == 0) {
        // many segments of a popular product change in the same pass: read before
        // the atomic so that only a new minimum contends for the word
        if (first_chg != INT_MAX && first_chg < ld_volatile(&fc_cur[k]))
            atomicMin(&fc_cur[k], first_chg);
        report_window_change(a, it, first_chg);
    }
    if (s == m.ce - 1) {  // last segment of the product: its end state is the final stock
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            if (FULL || n < N) a.xfin[(size_t)k * N + n] = max(0, x0v[i] - E[i]);
        }
    }
    calls += evals;
    return first_chg != INT_MAX;
}

}  // namespace picard

// Sequential simulation (Sec. 2 definition) on one warp: orders strictly one at
// a time.  The ids (product, region) of order t + 2*kAhead are fetched at step
// t; the stock row of order t + kAhead is fetched at step t and corrected, when
// used, for the decisions of the orders in between that hit the same product.
// cost_acc (lane-partial) and lost (warp-uniform) accumulate the order costs and
// a^phi count; lam may be null for the greedy policy.
constexpr int kAhead = 8;

template <int NPL, bool DUAL, bool SMEM>
__device__ __forceinline__ void seq_int_body(int T, int N, const int32_t* __restrict__ prod,
                                             const int32_t* __restrict__ reg,
                                             const int32_t* __restrict__ cost, const int16_t* s_cost,
                                             const int32_t* __restrict__ lam, int32_t* xw,
                                             int8_t* __restrict__ act_t, long long& cost_acc,
                                             long long& lost) {
    const int lane = lane_id();
    // slot p: order t = p (mod kAhead).  ik/ir: ids of order t + kAhead (next
    // occupant); rk/rr + Srow/Lrow: order t's ids and prefetched rows; dk/da:
    // product and decision of the order that used the slot last.
    int Srow[kAhead][NPL], Lrow[kAhead][NPL];
    int ik[kAhead], ir[kAhead], rk[kAhead], rrg[kAhead], dk[kAhead], da[kAhead];
#pragma unroll
    for (int p = 0; p < kAhead; ++p) {
        rk[p] = p < T ? __ldg(prod + p) : -1;
        rrg[p] = p < T ? __ldg(reg + p) : 0;
        ik[p] = p + kAhead < T ? __ldg(prod + p + kAhead) : -1;
        ir[p] = p + kAhead < T ? __ldg(reg + p + kAhead) : 0;
        dk[p] = -1;
        da[p] = -1;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            Srow[p][i] = (rk[p] >= 0 && n < N) ? xw[(size_t)rk[p] * N + n] : 0;
            Lrow[p][i] = (DUAL && lam && rk[p] >= 0 && n < N) ? __ldg(lam + (size_t)rk[p] * N + n) : 0;
        }
    }
    int my_act = -1;
    for (int t0 = 0; t0 < T; t0 += kAhead) {
#pragma unroll
        for (int p = 0; p < kAhead; ++p) {
            const int t = t0 + p;
            if (t < T) {
                const int k = rk[p];
                int S[NPL];
#pragma unroll
                for (int i = 0; i < NPL; ++i) S[i] = Srow[p][i];
#pragma unroll
                for (int d = 1; d < kAhead; ++d) {
                    const int q = (p - d + kAhead) % kAhead;
                    if (dk[q] == k) {
#pragma unroll
                        for (int i = 0; i < NPL; ++i) S[i] -= (da[q] == lane + 32 * i);
                    }
                }
                int c[NPL];
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int n = lane + 32 * i;
                    c[i] = n < N ? (SMEM ? (int)s_cost[rrg[p] * N + n]
                                         : __ldg(cost + (size_t)rrg[p] * N + n))
                                 : 0;
                }
                int key = INT_MAX;
#pragma unroll
                for (int i = 0; i < NPL; ++i)
                    key = min(key, S[i] > 0 ? (c[i] - Lrow[p][i]) * 128 + lane + 32 * i : INT_MAX);
                const int best = __reduce_min_sync(kFull, key);
                const int act = best == INT_MAX ? -1 : (best & 127);
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    if (act == lane + 32 * i) {
                        xw[(size_t)k * N + lane + 32 * i] = S[i] - 1;
                        cost_acc += c[i];
                    }
                }
                lost += act < 0;
                dk[p] = k;
                da[p] = act;
                if (lane == (t & 31)) my_act = act;
                if ((t & 31) == 31 || t == T - 1) {
                    const int tw = (t & ~31) + lane;
                    if (tw < T) act_t[tw] = (int8_t)my_act;
                }
                // this slot now takes order t + kAhead: row read after the store above
                const int nk = ik[p];
                rk[p] = nk;
                rrg[p] = ir[p];
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int n = lane + 32 * i;
                    Srow[p][i] = (nk >= 0 && n < N) ? xw[(size_t)nk * N + n] : 0;
                    Lrow[p][i] = (DUAL && lam && nk >= 0 && n < N) ? __ldg(lam + (size_t)nk * N + n) : 0;
                }
                const int t2 = t + 2 * kAhead;
                ik[p] = t2 < T ? __ldg(prod + t2) : -1;
                ir[p] = t2 < T ? __ldg(reg + t2) : 0;
            }
        }
    }
}

}  // namespace pic
