// Picard iteration (Algorithm 1) and the sequential baseline for the integer
// fulfilment policies:
//   greedy    a = argmin_{n : x[k][n] > 0} cost[r][n]                (Sec. 3.1)
//   bid-price a = argmin_{n : x[k][n] > 0} cost[r][n] - lam[k][n]    (Sec. 4.2, static prices)
// ties to the lowest warehouse index, a^phi (-1) when no warehouse has stock.
//
// One persistent cooperative launch runs every pass of Algorithm 1.  Each pass:
//   phase S  per product chain, per super-block of 32 segments: exclusive
//            prefix of the per-segment histograms of cached actions (the counts
//            d of the closed-form prefix max(0, x0 - d));
//   phase R  one warp per segment: start state of every run = max(0, x0 - d)
//            (the cached prefix of Algorithm 1 lines 5-7, applied in closed
//            form), then the run's orders replayed with fresh policy calls;
//            cache entries rewritten in place; histogram, cost and the first
//            changed position recorded;
// separated by grid barriers.  The loop ends at the first pass that changes no
// cached action (line 13).  A segment is replayed only if one of its runs starts
// after the first position of its product that changed in the previous pass
// (the t_reset optimisation of Appendix A.3, applied per product, which is
// exact because products never interact).
#include <cstdio>

#include "pic_device.cuh"

namespace pic {

namespace {

struct KArgs {
    int T, N, K, NP;
    const int32_t* __restrict__ reg_s;
    const int32_t* __restrict__ run_start;
    const int32_t* __restrict__ seg_run;
    const int32_t* __restrict__ seg_prod;
    const int32_t* __restrict__ seg_cf;
    const int32_t* __restrict__ seg_ce;
    const int32_t* __restrict__ x0;
    const int32_t* __restrict__ cost;
    const int32_t* __restrict__ lam;
    int8_t* alpha_s;
    int32_t* agg;
    int32_t* carry;
    int32_t* sbtot;
    int32_t* fc;
    int32_t* xfin;
    long long* seg_cost;
    int32_t* seg_lost;
    Ctrl* ctrl;
    int max_iters;
    int flags;
    int first_dirty;
    unsigned long long timeout_ns;
};

// Replay one segment (all its runs, in order) with one warp.  Lane l owns
// warehouses l, l+32, ..., l+32(NPL-1).
template <int NPL, bool DUAL>
__device__ __forceinline__ void replay_segment(const KArgs& a, int s, int k, int r0, int r1,
                                               int parity, int* fc_cur,
                                               unsigned long long& calls,
                                               unsigned long long& replays) {
    const int lane = lane_id();
    const int N = a.N, NP = a.NP;
    const int cf = a.seg_cf[s], ce = a.seg_ce[s];
    int D[NPL], x0v[NPL], lamv[NPL], S[NPL], S0[NPL], hist[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        D[i] = 0;
        hist[i] = 0;
        x0v[i] = n < N ? a.x0[(size_t)k * N + n] : 0;
        lamv[i] = (DUAL && n < N) ? a.lam[(size_t)k * N + n] : 0;
    }
    if (ce - cf > 1) {  // prefix counts from earlier segments of this product
#pragma unroll
        for (int i = 0; i < NPL; ++i) D[i] = a.carry[(size_t)s * NP + lane + 32 * i];
        const int nb = (s - cf) / kSuperBlock;
        for (int b = 0; b < nb; ++b) {
            const size_t h = (size_t)(cf + b * kSuperBlock) * NP;
#pragma unroll
            for (int i = 0; i < NPL; ++i) D[i] += a.sbtot[h + lane + 32 * i];
        }
    }
    const int j0 = a.run_start[r0], jend = a.run_start[r1];
    int r = r0;
    int next_run = a.run_start[r0 + 1];
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        S[i] = max(0, x0v[i] - D[i]);
        S0[i] = S[i];
    }
    long long cost_acc = 0;
    int lost_acc = 0;
    int first_chg = INT_MAX;
    int nreg = 0, nold = -1;
    if (lane < jend - j0) {
        nreg = a.reg_s[j0 + lane];
        nold = a.alpha_s[j0 + lane];
    }
    for (int base = j0; base < jend; base += 32) {
        const int cnt = min(32, jend - base);
        const int my_reg = nreg, my_old = nold;
        // prefetch the next batch of orders
        if (base + 32 + lane < jend) {
            nreg = a.reg_s[base + 32 + lane];
            nold = a.alpha_s[base + 32 + lane];
        }
        int my_new = my_old;
        int rr = __shfl_sync(kFull, my_reg, 0);
        int c[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            c[i] = n < N ? __ldg(a.cost + (size_t)rr * N + n) : 0;
        }
        for (int q = 0; q < cnt; ++q) {
            const int j = base + q;
            if (j == next_run) {  // close run r, open run r+1 (cached prefix now includes run r)
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    hist[i] += S0[i] - S[i];
                    S[i] = max(0, x0v[i] - D[i]);
                    S0[i] = S[i];
                }
                ++r;
                next_run = a.run_start[r + 1];
            }
            const int ao = __shfl_sync(kFull, my_old, q);
            // prefetch the next order's cost row
            const int rn = __shfl_sync(kFull, my_reg, q + 1 < cnt ? q + 1 : q);
            int cn[NPL];
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int n = lane + 32 * i;
                cn[i] = n < N ? __ldg(a.cost + (size_t)rn * N + n) : 0;
            }
            int key = INT_MAX;
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int n = lane + 32 * i;
                const int kk = (c[i] - lamv[i]) * 128 + n;
                if (S[i] > 0 && kk < key) key = kk;
            }
            const int best = __reduce_min_sync(kFull, key);
            const int act = best == INT_MAX ? -1 : (best & 127);
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int n = lane + 32 * i;
                if (act == n) {
                    S[i] -= 1;
                    cost_acc += c[i];
                }
                if (ao == n) D[i] += 1;
            }
            if (lane == q) my_new = act;
            lost_acc += act < 0;
#pragma unroll
            for (int i = 0; i < NPL; ++i) c[i] = cn[i];
        }
        if (lane < cnt) a.alpha_s[base + lane] = (int8_t)my_new;
        const unsigned chg = __ballot_sync(kFull, lane < cnt && my_new != my_old);
        if (chg && first_chg == INT_MAX) first_chg = base + __ffs(chg) - 1;
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        hist[i] += S0[i] - S[i];
        a.agg[(size_t)s * NP + lane + 32 * i] = hist[i];
    }
    cost_acc = warp_sum_i64(cost_acc);
    if (lane == 0) {
        a.seg_cost[s] = cost_acc;
        a.seg_lost[s] = lost_acc;
        if (first_chg != INT_MAX) {
            atomicMin(&fc_cur[k], first_chg);
            a.ctrl->changed[parity] = 1;
        }
    }
    if (s == ce - 1) {  // last segment of the product: its end state is the final stock
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            if (n < N) a.xfin[(size_t)k * N + n] = S[i];
        }
    }
    calls += (unsigned long long)(jend - j0);
    replays += 1;
}

template <int NPL, bool DUAL>
__global__ void __launch_bounds__(kThreads) k_picard_int(KArgs a) {
    const int lane = lane_id();
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    const int nseg = a.ctrl->nseg;
    const int NP = a.NP;
    unsigned long long calls = 0, replays = 0;
    int it = 1;
    bool ok = true, converged = false;
    for (; it <= a.max_iters; ++it) {
        const int parity = it & 1;
        const int* fc_prev = a.fc + (size_t)(parity ^ 1) * a.K;
        int* fc_cur = a.fc + (size_t)parity * a.K;
        // ---- phase S: super-block prefixes of cached-action histograms
        for (int k = gtid; k < a.K; k += gthreads) fc_cur[k] = INT_MAX;
        if (gtid == 0) a.ctrl->changed[parity] = 0;
        if (it > 1 || a.first_dirty) {
            for (int s = gwarp; s < nseg; s += nwarps) {
                const int cf = a.seg_cf[s], ce = a.seg_ce[s];
                if (ce - cf <= 1 || (s - cf) % kSuperBlock != 0) continue;
                if (it > 1 && fc_prev[a.seg_prod[s]] == INT_MAX) continue;
                const int send = min(s + kSuperBlock, ce);
                int acc[NPL];
#pragma unroll
                for (int i = 0; i < NPL; ++i) acc[i] = 0;
                for (int s2 = s; s2 < send; ++s2) {
#pragma unroll
                    for (int i = 0; i < NPL; ++i) {
                        const size_t o = (size_t)s2 * NP + lane + 32 * i;
                        const int g = a.agg[o];
                        a.carry[o] = acc[i];
                        acc[i] += g;
                    }
                }
#pragma unroll
                for (int i = 0; i < NPL; ++i) a.sbtot[(size_t)s * NP + lane + 32 * i] = acc[i];
            }
        }
        if (!grid_sync(a.ctrl, deadline)) { ok = false; break; }
        // ---- phase R: replay active segments
        for (int s = gwarp; s < nseg; s += nwarps) {
            const int k = a.seg_prod[s];
            const int r0 = a.seg_run[s], r1 = a.seg_run[s + 1];
            if (!(a.flags & PIC_FLAG_NO_RESET) && !(a.run_start[r1 - 1] > fc_prev[k])) continue;
            replay_segment<NPL, DUAL>(a, s, k, r0, r1, parity, fc_cur, calls, replays);
        }
        if (!grid_sync(a.ctrl, deadline)) { ok = false; break; }
        if (ld_volatile(&a.ctrl->changed[parity]) == 0) { converged = true; break; }
    }
    if (lane == 0 && calls) {
        atomicAdd(&a.ctrl->policy_calls, calls);
        atomicAdd(&a.ctrl->seg_replays, replays);
    }
    if (gtid == 0 && ok) {
        a.ctrl->iters = converged ? it : a.max_iters;
        a.ctrl->converged = converged ? 1 : 0;
    }
}

// Sequential simulation (Sec. 2 definition) on one warp: orders strictly one at
// a time.  Stock rows are prefetched kAhead orders in advance and corrected for
// the decisions of the orders in between that hit the same product, so the
// dependent row load does not stall every step.
constexpr int kAhead = 8;

template <int NPL, bool DUAL>
__global__ void __launch_bounds__(32) k_seq_int(int T, int N, const int32_t* __restrict__ prod,
                                                const int32_t* __restrict__ reg,
                                                const int32_t* __restrict__ cost,
                                                const int32_t* __restrict__ lam, int32_t* xw,
                                                int8_t* __restrict__ act_t, Ctrl* ctrl) {
    const int lane = lane_id();
    // ring of prefetched rows for orders t .. t+kAhead-1
    int Srow[kAhead][NPL], Crow[kAhead][NPL], Lrow[kAhead][NPL];
    int pk[kAhead], pa[kAhead], ok_[kAhead];
    long long cost_acc = 0, lost = 0;
    auto fetch = [&](int t, int slot_S[NPL], int slot_C[NPL], int slot_L[NPL], int& kk) {
        if (t < T) {
            kk = __ldg(prod + t);
            const int rr = __ldg(reg + t);
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int n = lane + 32 * i;
                slot_S[i] = n < N ? xw[(size_t)kk * N + n] : 0;
                slot_C[i] = n < N ? __ldg(cost + (size_t)rr * N + n) : 0;
                slot_L[i] = (DUAL && n < N) ? __ldg(lam + (size_t)kk * N + n) : 0;
            }
        } else {
            kk = -1;
        }
    };
#pragma unroll
    for (int p = 0; p < kAhead; ++p) {
        fetch(p, Srow[p], Crow[p], Lrow[p], ok_[p]);
        pk[p] = -1;
        pa[p] = -1;
    }
    int my_act = -1;
    for (int t0 = 0; t0 < T; t0 += kAhead) {
#pragma unroll
        for (int p = 0; p < kAhead; ++p) {
            const int t = t0 + p;
            if (t < T) {
                const int k = ok_[p];
                int S[NPL];
#pragma unroll
                for (int i = 0; i < NPL; ++i) S[i] = Srow[p][i];
                // decisions of the previous kAhead orders were not in the prefetched row
#pragma unroll
                for (int d = 1; d < kAhead; ++d) {
                    const int q = (p - d + kAhead) % kAhead;
                    if (pk[q] == k) {
#pragma unroll
                        for (int i = 0; i < NPL; ++i) S[i] -= (pa[q] == lane + 32 * i);
                    }
                }
                int key = INT_MAX;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int kk = (Crow[p][i] - Lrow[p][i]) * 128 + lane + 32 * i;
                    if (S[i] > 0 && kk < key) key = kk;
                }
                const int best = __reduce_min_sync(kFull, key);
                const int act = best == INT_MAX ? -1 : (best & 127);
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int n = lane + 32 * i;
                    if (act == n) {
                        xw[(size_t)k * N + n] = S[i] - 1;
                        cost_acc += Crow[p][i];
                    }
                }
                lost += act < 0;
                pk[p] = k;
                pa[p] = act;
                if (lane == (t & 31)) my_act = act;
                if ((t & 31) == 31 || t == T - 1) {
                    const int tw = t - (t & 31) + lane;
                    if (tw < T) act_t[tw] = (int8_t)my_act;
                }
                // refill this slot with order t + kAhead (row read after this store)
                fetch(t + kAhead, Srow[p], Crow[p], Lrow[p], ok_[p]);
            }
        }
    }
    cost_acc = warp_sum_i64(cost_acc);
    if (lane == 0) {
        ctrl->total_cost = cost_acc;
        ctrl->lost = lost;
        ctrl->iters = 1;
        ctrl->converged = 1;
        ctrl->policy_calls = (unsigned long long)T;
    }
}

template <int NPL, bool DUAL>
cudaError_t launch_picard(Instance* I, const KArgs& a, cudaStream_t st) {
    auto kern = k_picard_int<NPL, DUAL>;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0);
    if (e) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int grid = I->num_sms * (occ < 4 ? occ : 4);
    I->coop_blocks = grid;
    KArgs args = a;
    void* params[] = {&args};
    I->launches += 1;
    return cudaLaunchCooperativeKernel((const void*)kern, grid, kThreads, params, 0, st);
}

template <int NPL, bool DUAL>
cudaError_t launch_seq(Instance* I, cudaStream_t st) {
    I->launches += 1;
    k_seq_int<NPL, DUAL><<<1, 32, 0, st>>>(I->T, I->N, I->prod, I->reg, I->cost, I->lam, I->xwork,
                                           I->act_t, I->ctrl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t picard_int(Instance* I, int kind, int max_iters, int flags, const int8_t* alpha_init,
                       unsigned long long timeout_ns, cudaStream_t st) {
    KArgs a;
    a.T = I->T; a.N = I->N; a.K = I->K; a.NP = I->NP;
    a.reg_s = I->reg_s; a.run_start = I->run_start; a.seg_run = I->seg_run;
    a.seg_prod = I->seg_prod; a.seg_cf = I->seg_cf; a.seg_ce = I->seg_ce;
    a.x0 = I->x0; a.cost = I->cost; a.lam = I->lam;
    a.alpha_s = I->alpha_s; a.agg = I->agg; a.carry = I->carry; a.sbtot = I->sbtot;
    a.fc = I->fc; a.xfin = I->xfin; a.seg_cost = I->seg_cost; a.seg_lost = I->seg_lost;
    a.ctrl = I->ctrl; a.max_iters = max_iters; a.flags = flags;
    a.first_dirty = alpha_init != nullptr; a.timeout_ns = timeout_ns;
    const bool dual = kind == PIC_POLICY_DUAL;
    const int npl = (I->N + 31) / 32;
    if (npl == 1) return dual ? launch_picard<1, true>(I, a, st) : launch_picard<1, false>(I, a, st);
    if (npl == 2) return dual ? launch_picard<2, true>(I, a, st) : launch_picard<2, false>(I, a, st);
    return dual ? launch_picard<4, true>(I, a, st) : launch_picard<4, false>(I, a, st);
}

cudaError_t sequential_int(Instance* I, int kind, cudaStream_t st) {
    const bool dual = kind == PIC_POLICY_DUAL;
    const int npl = (I->N + 31) / 32;
    if (npl == 1) return dual ? launch_seq<1, true>(I, st) : launch_seq<1, false>(I, st);
    if (npl == 2) return dual ? launch_seq<2, true>(I, st) : launch_seq<2, false>(I, st);
    return dual ? launch_seq<4, true>(I, st) : launch_seq<4, false>(I, st);
}

}  // namespace pic
