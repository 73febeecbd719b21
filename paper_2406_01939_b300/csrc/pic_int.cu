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

#include "pic_replay.cuh"

namespace pic {

namespace {

using namespace picard;

template <int NPL, bool SMEM>
struct PicardShape {
    // with the staged cost table: one CTA per SM sharing it (85 or 128 registers/thread)
    static constexpr int threads = SMEM ? (NPL >= 4 ? 512 : 768) : kThreads;
};

template <int NPL, bool DUAL, bool SMEM, bool FULL>
__global__ void __launch_bounds__(PicardShape<NPL, SMEM>::threads, 1) k_picard_int(KArgs a) {
    const CostTable<SMEM> ct = stage_cost<SMEM>(a);
    unsigned long long calls = 0;
    picard_passes<NPL, PicardShape<NPL, SMEM>::threads / 32>(
        a, calls, [&](int seg, const SegMeta& m, int fcp, int* fc_cur, int it) {
            return replay_segment<NPL, DUAL, SMEM, FULL>(a, ct, seg, m, fcp, fc_cur, it, true, calls);
        });
}

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
    long long cost_acc = 0, lost = 0;
    seq_int_body<NPL, DUAL, SMEM>(T, N, prod, reg, cost, s_cost, lam, xw, act_t, cost_acc, lost);
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
    I->cta_threads = threads;
    I->ctas_per_sm = per_sm;
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
                       int max_steps, cudaStream_t st) {
    const int kind = pol->kind;
    KArgs a;
    a.T = I->T; a.N = I->N; a.K = I->K; a.NP = I->NP; a.R = I->R;
    a.reg_s = I->reg_s; a.run_start = I->run_start; a.seg_run = I->seg_run;
    a.seg_prod = I->seg_prod; a.seg_cf = I->seg_cf; a.seg_ce = I->seg_ce;
    a.x0 = I->x0; a.cost = I->cost; a.lam = I->lam;
    a.alpha_s = I->alpha_s; a.agg = I->agg; a.carry = I->carry; a.sbexc = I->sbexc;
    a.sbagg = I->sbagg; a.sbincl = I->sbincl; a.meta = I->seg_meta; a.lpt = I->seg_lpt;
    a.fc = I->fc; a.xfin = I->xfin;
    a.ctrl = I->ctrl; a.max_iters = max_iters; a.flags = flags;
    a.first_dirty = alpha_init != nullptr; a.timeout_ns = timeout_ns;
    a.trace = trace ? I->trace : nullptr;
    a.run_chunk = max_steps > 0 ? I->run_chunk : nullptr;
    a.perm = I->perm;
    a.win_steps = max_steps;
    a.M = I->tables_m;
    a.L = I->tables_m ? (int)(((long long)I->T + I->tables_m - 1) / I->tables_m) : 1;
    if (kind == PIC_POLICY_MLP || kind == PIC_POLICY_GUMBEL) return picard_mlp(I, a, pol, st);
    const bool dual = kind == PIC_POLICY_DUAL;
    // the group kernel has no max_steps window
    if ((flags & PIC_FLAG_GROUP_KERNEL) && grp_ok(I) && max_steps <= 0) return picard_grp(I, a, dual, st);
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
