// Picard iteration (Algorithm 1) and the sequential baseline for the integer
// fulfilment policies:
//   greedy    a = argmin_{n : x[k][n] > 0} cost[r][n]                (Sec. 3.1)
//   bid-price a = argmin_{n : x[k][n] > 0} cost[r][n] - lam[k][n]    (Sec. 4.2, static prices)
// ties to the lowest warehouse index, a^phi (-1) when no warehouse has stock.
//
// One persistent cooperative launch runs every pass of Algorithm 1.  Each pass:
//   phase S  per product chain: exclusive prefix, over the chain's segments, of
//            the per-segment histograms of cached actions (the counts d of the
//            closed-form prefix max(0, x0 - d)).  One warp per super-block of 32
//            segments; super-blocks of a chain chain their totals with a
//            decoupled look-back (publish the block total, then add
//            predecessors' totals until one with a published inclusive prefix);
//   phase R  one warp per segment: start state of every run = max(0, x0 - d)
//            (the cached prefix of Algorithm 1 lines 5-7, applied in closed
//            form), then the run's orders replayed with fresh policy calls;
//            cache entries rewritten in place; histogram, cost and the first
//            changed position recorded;
// separated by grid barriers.  The loop ends at the first pass that changes no
// cached action (line 13).
//
// t_reset (Appendix A.3), applied per product, which is exact because products
// never interact: a run whose first order is at or before the first position of
// its product that changed in the previous pass has the same cached prefix as
// in that pass, so its actions are the cached ones.  Such runs are walked
// without policy calls (to carry the state forward); a segment none of whose
// runs starts after that position is skipped entirely.
//
// The cost table is staged once per launch in shared memory (int16) when it
// fits, so the per-order score read is a shared-memory access.
#include <cstdio>

#include "pic_picard.cuh"

namespace pic {

namespace {

using namespace picard;

// Replay one segment (all its runs, in order) with one warp.  Lane l owns
// warehouses l, l+32, ..., l+32(NPL-1).  fcp: first position of product k that
// changed in the previous pass (-1: every run is evaluated).
//
// Per run the state starts at max(0, x0 - D), D = counts of cached actions of
// this product before the run.  D advances run by run: the run's own new
// actions (S0 - S at the run's end) plus a correction for the orders whose new
// action differs from the cached one (rare once the iteration settles).
template <int NPL, bool DUAL, bool SMEM, bool FULL>
__device__ __forceinline__ bool replay_segment(const KArgs& a, const CostTable<SMEM>& ct, int s,
                                               const SegMeta& m, int fcp, int* fc_cur,
                                               unsigned long long& calls,
                                               unsigned long long& replays) {
    const int lane = lane_id();
    const int N = a.N, NP = a.NP;
    const int k = m.k;
    // key = score * 128 + n (ties to the lowest index); adj = n - 128 * lam[k][n]
    int D[NPL], x0v[NPL], adj[NPL], S[NPL], S0[NPL], hist[NPL], corr[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        const bool in = FULL || n < N;
        hist[i] = 0;
        corr[i] = 0;
        x0v[i] = in ? a.x0[(size_t)k * N + n] : 0;
        adj[i] = n - ((DUAL && in) ? 128 * a.lam[(size_t)k * N + n] : 0);
        // prefix counts from earlier segments of this product (exclusive chain prefix)
        D[i] = m.ce - m.cf > 1 ? a.carry[(size_t)s * NP + n] : 0;
    }
    const int j0 = m.j0, jend = m.jend;
    // lane i holds the end (= next start) of run rwin + i
    int rwin = m.r0;
    int run_end = lane < m.r1 - rwin ? a.run_start[rwin + 1 + lane] : INT_MAX;
    int r = m.r0;
    int next_run = __shfl_sync(kFull, run_end, 0);
    bool eval = j0 > fcp;  // this run's prefix changed in the previous pass
    unsigned long long evals = eval ? (unsigned long long)(next_run - j0) : 0ull;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        S[i] = max(0, x0v[i] - D[i]);
        S0[i] = S[i];
    }
    int first_chg = INT_MAX;
    int nreg = 0, nold = -1;
    if (lane < jend - j0) {
        nreg = a.reg_s[j0 + lane];
        nold = a.alpha_s[j0 + lane];
    }
    for (int base = j0; base < jend; base += 32) {
        const int cnt = min(32, jend - base);
        const int my_reg = nreg, my_old = nold;
        if (base + 32 + lane < jend) {  // prefetch the next batch of orders
            nreg = a.reg_s[base + 32 + lane];
            nold = a.alpha_s[base + 32 + lane];
        }
        int my_new = my_old;
        for (int q = 0; q < cnt; ++q) {
            if (base + q == next_run) {  // close run r, open run r+1
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    hist[i] += S0[i] - S[i];
                    D[i] += S0[i] - S[i] + corr[i];
                    corr[i] = 0;
                    S[i] = max(0, x0v[i] - D[i]);
                    S0[i] = S[i];
                }
                ++r;
                int idx = r - rwin;
                if (idx == 32) {  // next window of run ends
                    rwin += 32;
                    idx = 0;
                    run_end = lane < m.r1 - rwin ? a.run_start[rwin + 1 + lane] : INT_MAX;
                }
                const int nr = __shfl_sync(kFull, run_end, idx);
                eval = next_run > fcp;
                if (eval) evals += (unsigned long long)(nr - next_run);
                next_run = nr;
            }
            const int rr = __shfl_sync(kFull, my_reg, q);
            const int ao = __shfl_sync(kFull, my_old, q);
            int c[NPL];
#pragma unroll
            for (int i = 0; i < NPL; ++i)
                c[i] = (FULL || lane + 32 * i < N) ? ct.at(rr, lane + 32 * i) : 0;
            int act = ao;  // unchanged prefix: the cached action is the policy's
            if (eval) {
                int key = INT_MAX;
#pragma unroll
                for (int i = 0; i < NPL; ++i)
                    key = min(key, S[i] > 0 ? c[i] * 128 + adj[i] : INT_MAX);
                const int best = __reduce_min_sync(kFull, key);
                act = best == INT_MAX ? -1 : (best & 127);
            }
#pragma unroll
            for (int i = 0; i < NPL; ++i) S[i] -= (act == lane + 32 * i);
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
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        hist[i] += S0[i] - S[i];
        a.agg[(size_t)s * NP + lane + 32 * i] = hist[i];
    }
    if (lane == 0) {
        // many segments of a popular product change in the same pass: read before
        // the atomic so that only a new minimum contends for the word
        if (first_chg != INT_MAX && first_chg < ld_volatile(&fc_cur[k]))
            atomicMin(&fc_cur[k], first_chg);
    }
    if (s == m.ce - 1) {  // last segment of the product: its end state is the final stock
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            if (FULL || n < N) a.xfin[(size_t)k * N + n] = S[i];
        }
    }
    calls += evals;
    replays += 1;
    return first_chg != INT_MAX;
}

template <int NPL, bool SMEM>
struct PicardShape {
    // with the staged cost table: one CTA per SM sharing it (85 or 128 registers/thread)
    static constexpr int threads = SMEM ? (NPL >= 4 ? 512 : 768) : kThreads;
};

template <int NPL, bool DUAL, bool SMEM, bool FULL>
__global__ void __launch_bounds__(PicardShape<NPL, SMEM>::threads, 1) k_picard_int(KArgs a) {
    __shared__ int s_changed;
    // per warp: the 32 segments it is examining (metadata, previous-pass first change)
    __shared__ SegMeta s_meta[kMaxWarpsPerCta][32];
    __shared__ int s_fcp[kMaxWarpsPerCta][32];
    const CostTable<SMEM> ct = stage_cost<SMEM>(a);
    const int lane = lane_id();
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    const int nseg = a.ctrl->nseg;
    const bool no_reset = (a.flags & PIC_FLAG_NO_RESET) != 0;
    if (threadIdx.x == 0) s_changed = 0;
    unsigned long long calls = 0, replays = 0;
    const unsigned long long t_start = globaltimer_ns();
    int it = 1;
    bool ok = true, converged = false;
    for (; it <= a.max_iters; ++it) {
        const int parity = it & 1;
        long long* tr = (a.trace && it <= kTraceCap) ? a.trace + 4 * (it - 1) : nullptr;
        const unsigned long long calls0 = calls, replays0 = replays;
        const int* fc_prev = a.fc + (size_t)(parity ^ 1) * a.K;
        int* fc_cur = a.fc + (size_t)parity * a.K;
        // ---- phase S: chain prefixes of cached-action histograms.  This warp's
        // segments gwarp + j * nwarps are examined 32 at a time, one per lane.
        for (int k = gtid; k < a.K; k += gthreads) fc_cur[k] = INT_MAX;
        if (gtid == 0) a.ctrl->changed[parity] = 0;
        if (it > 1 || a.first_dirty) {
            for (int j0 = 0; gwarp + j0 * nwarps < nseg; j0 += 32) {
                const int sl = gwarp + (j0 + lane) * nwarps;
                bool head = false;
                if (sl < nseg) {
                    const SegMeta m = load_meta(a.meta + sl);
                    head = m.ce - m.cf > 1 && (sl - m.cf) % kSuperBlock == 0;
                    const int f = it > 1 ? fc_prev[m.k] : -1;
                    if (head && it > 1) head = f != INT_MAX;
                    if (head) {
                        s_meta[threadIdx.x >> 5][lane] = m;
                        s_fcp[threadIdx.x >> 5][lane] = f;
                    }
                }
                unsigned todo = __ballot_sync(kFull, head);
                while (todo) {  // increasing segment order (lane order)
                    const int src = __ffs(todo) - 1;
                    todo &= todo - 1;
                    const SegMeta mm = smem_meta(&s_meta[threadIdx.x >> 5][src]);
                    superblock_prefix<NPL>(a, gwarp + (j0 + src) * nwarps, mm, it,
                                           s_fcp[threadIdx.x >> 5][src], deadline);
                }
                __syncwarp();
            }
        }
        if (!grid_sync(a.ctrl, deadline)) { ok = false; break; }
        if (tr && gtid == 0) tr[0] = (long long)(globaltimer_ns() - t_start);
        // ---- phase R: replay active segments.  Positions of the longest-first
        // order are dealt to warps in a snake (w, 2W-1-w, 2W+w, ...), examined 32
        // at a time per warp.
        bool chg = false;
        for (int j0 = 0; j0 * nwarps < nseg; j0 += 32) {
            const int j = j0 + lane;
            const int pos = j * nwarps + ((j & 1) ? nwarps - 1 - gwarp : gwarp);
            int sl = nseg;
            bool act = false;
            if (pos < nseg) {
                sl = a.lpt[pos];
                const SegMeta m = load_meta(a.meta + sl);
                const int fcp = no_reset ? -1 : fc_prev[m.k];
                act = m.last_start > fcp;
                if (act) {
                    s_meta[threadIdx.x >> 5][lane] = m;
                    s_fcp[threadIdx.x >> 5][lane] = fcp;
                }
            }
            unsigned todo = __ballot_sync(kFull, act);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const SegMeta mm = smem_meta(&s_meta[threadIdx.x >> 5][src]);
                const int f = s_fcp[threadIdx.x >> 5][src];
                const int seg = __shfl_sync(kFull, sl, src);
                chg |= replay_segment<NPL, DUAL, SMEM, FULL>(a, ct, seg, mm, f, fc_cur, calls,
                                                             replays);
            }
            __syncwarp();
        }
        if (tr && lane == 0 && replays != replays0) {
            atomicAdd((unsigned long long*)&tr[2], calls - calls0);
            atomicAdd((unsigned long long*)&tr[3], replays - replays0);
        }
        if (chg && lane == 0) s_changed = 1;  // one global write per CTA, below
        __syncthreads();
        if (threadIdx.x == 0 && s_changed) {
            a.ctrl->changed[parity] = 1;
            s_changed = 0;
        }
        if (!grid_sync(a.ctrl, deadline)) { ok = false; break; }
        if (tr && gtid == 0) tr[1] = (long long)(globaltimer_ns() - t_start);
        if (ld_volatile(&a.ctrl->changed[parity]) == 0) { converged = true; break; }
    }
    if (lane == 0 && replays) {
        atomicAdd(&a.ctrl->policy_calls, calls);
        atomicAdd(&a.ctrl->seg_replays, replays);
    }
    if (gtid == 0 && ok) {
        a.ctrl->iters = converged ? it : a.max_iters;
        a.ctrl->converged = converged ? 1 : 0;
    }
}

// Sequential simulation (Sec. 2 definition) on one warp: orders strictly one at
// a time.  The ids (product, region) of order t + 2*kAhead are fetched at step
// t; the stock row of order t + kAhead is fetched at step t and corrected, when
// used, for the decisions of the orders in between that hit the same product.
constexpr int kAhead = 8;

template <int NPL, bool DUAL, bool SMEM>
__global__ void __launch_bounds__(32) k_seq_int(int T, int N, int R,
                                                const int32_t* __restrict__ prod,
                                                const int32_t* __restrict__ reg,
                                                const int32_t* __restrict__ cost,
                                                const int32_t* __restrict__ lam, int32_t* xw,
                                                int8_t* __restrict__ act_t, Ctrl* ctrl) {
    extern __shared__ int16_t s_cost[];
    const int lane = lane_id();
    if (SMEM) {
        for (int i = lane; i < R * N; i += 32) s_cost[i] = (int16_t)cost[i];
        __syncwarp();
    }
    // slot p: order t = p (mod kAhead).  ik/ir: ids of order t + kAhead (next
    // occupant); rk/rr + Srow/Lrow: order t's ids and prefetched rows; dk/da:
    // product and decision of the order that used the slot last.
    int Srow[kAhead][NPL], Lrow[kAhead][NPL];
    int ik[kAhead], ir[kAhead], rk[kAhead], rrg[kAhead], dk[kAhead], da[kAhead];
    long long cost_acc = 0, lost = 0;
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
            Lrow[p][i] = (DUAL && rk[p] >= 0 && n < N) ? __ldg(lam + (size_t)rk[p] * N + n) : 0;
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
                    Lrow[p][i] = (DUAL && nk >= 0 && n < N) ? __ldg(lam + (size_t)nk * N + n) : 0;
                }
                const int t2 = t + 2 * kAhead;
                ik[p] = t2 < T ? __ldg(prod + t2) : -1;
                ir[p] = t2 < T ? __ldg(reg + t2) : 0;
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

template <int NPL, bool DUAL, bool SMEM, bool FULL>
cudaError_t launch_picard(Instance* I, const KArgs& a, cudaStream_t st) {
    auto kern = k_picard_int<NPL, DUAL, SMEM, FULL>;
    const int threads = PicardShape<NPL, SMEM>::threads;
    const size_t smem = SMEM ? (size_t)I->R * I->N * sizeof(int16_t) : 0;
    cudaError_t e;
    if (SMEM) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e) return e;
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = SMEM ? 1 : (occ < 4 ? occ : 4);
    const int grid = I->num_sms * per_sm;
    I->coop_blocks = grid;
    KArgs args = a;
    void* params[] = {&args};
    I->launches += 1;
    return cudaLaunchCooperativeKernel((const void*)kern, grid, threads, params, smem, st);
}

template <int NPL, bool DUAL, bool SMEM>
cudaError_t launch_seq(Instance* I, cudaStream_t st) {
    auto kern = k_seq_int<NPL, DUAL, SMEM>;
    const size_t smem = SMEM ? (size_t)I->R * I->N * sizeof(int16_t) : 0;
    if (SMEM) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e) return e;
    }
    I->launches += 1;
    kern<<<1, 32, smem, st>>>(I->T, I->N, I->R, I->prod, I->reg, I->cost, I->lam, I->xwork,
                              I->act_t, I->ctrl);
    return cudaGetLastError();
}

template <int NPL, bool DUAL>
cudaError_t picard_dispatch(Instance* I, const KArgs& a, cudaStream_t st) {
    const bool full = I->N == 32 * NPL;  // every lane owns real warehouses: no bounds checks
    if (smem_cost_ok(I))
        return full ? launch_picard<NPL, DUAL, true, true>(I, a, st)
                    : launch_picard<NPL, DUAL, true, false>(I, a, st);
    return full ? launch_picard<NPL, DUAL, false, true>(I, a, st)
                : launch_picard<NPL, DUAL, false, false>(I, a, st);
}

template <int NPL, bool DUAL>
cudaError_t seq_dispatch(Instance* I, cudaStream_t st) {
    return smem_cost_ok(I) ? launch_seq<NPL, DUAL, true>(I, st) : launch_seq<NPL, DUAL, false>(I, st);
}

}  // namespace

bool smem_cost_ok(const Instance* I) {
    return I->cost16 && (size_t)I->R * I->N * sizeof(int16_t) <= kSmemCostMax;
}

cudaError_t picard_run(Instance* I, const pic_policy* pol, int max_iters, int flags,
                       const int8_t* alpha_init, unsigned long long timeout_ns, bool trace,
                       cudaStream_t st) {
    const int kind = pol->kind;
    KArgs a;
    a.T = I->T; a.N = I->N; a.K = I->K; a.NP = I->NP; a.R = I->R;
    a.reg_s = I->reg_s; a.run_start = I->run_start; a.seg_run = I->seg_run;
    a.seg_prod = I->seg_prod; a.seg_cf = I->seg_cf; a.seg_ce = I->seg_ce;
    a.x0 = I->x0; a.cost = I->cost; a.lam = I->lam;
    a.alpha_s = I->alpha_s; a.agg = I->agg; a.carry = I->carry;
    a.sbagg = I->sbagg; a.sbincl = I->sbincl; a.meta = I->seg_meta; a.lpt = I->seg_lpt;
    a.fc = I->fc; a.xfin = I->xfin;
    a.ctrl = I->ctrl; a.max_iters = max_iters; a.flags = flags;
    a.first_dirty = alpha_init != nullptr; a.timeout_ns = timeout_ns;
    a.trace = trace ? I->trace : nullptr;
    if (kind == PIC_POLICY_MLP || kind == PIC_POLICY_GUMBEL) return picard_mlp(I, a, pol, st);
    const bool dual = kind == PIC_POLICY_DUAL;
    if ((flags & PIC_FLAG_GROUP_KERNEL) && grp_ok(I)) return picard_grp(I, a, dual, st);
    const int npl = (I->N + 31) / 32;
    if (npl == 1) return dual ? picard_dispatch<1, true>(I, a, st) : picard_dispatch<1, false>(I, a, st);
    if (npl == 2) return dual ? picard_dispatch<2, true>(I, a, st) : picard_dispatch<2, false>(I, a, st);
    return dual ? picard_dispatch<4, true>(I, a, st) : picard_dispatch<4, false>(I, a, st);
}

cudaError_t sequential_int(Instance* I, int kind, cudaStream_t st) {
    const bool dual = kind == PIC_POLICY_DUAL;
    const int npl = (I->N + 31) / 32;
    if (npl == 1) return dual ? seq_dispatch<1, true>(I, st) : seq_dispatch<1, false>(I, st);
    if (npl == 2) return dual ? seq_dispatch<2, true>(I, st) : seq_dispatch<2, false>(I, st);
    return dual ? seq_dispatch<4, true>(I, st) : seq_dispatch<4, false>(I, st);
}

}  // namespace pic
