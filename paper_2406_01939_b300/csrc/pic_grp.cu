// Picard iteration (Algorithm 1) for the integer policies, group-per-segment
// layout.  Same passes as the warp-per-segment kernel (phase S: chain prefixes
// of cached-action histograms; phase R: replay of every segment whose prefix
// changed), but a segment is replayed by a group of G lanes, each lane owning 8
// consecutive warehouses, so one warp advances 32/G segments at once.  The
// policy of one order then costs one 16-byte shared-memory read of the cost row
// slice, 8 masked keys per lane and a log2(G)-step shuffle minimum inside the
// group; the order stream and the run boundaries are staged per group in shared
// memory, 32 at a time.
//
// Requirements (checked by the dispatcher): every cost fits int16 and the cost
// table, padded to 8G columns, fits in shared memory next to the staging areas.
#include "pic_picard.cuh"

namespace pic {

namespace {

using namespace picard;

constexpr int kWpl = 8;           // warehouses per lane
constexpr int kGrpThreads = 512;  // 16 warps, up to 128 registers per thread
constexpr int kBatch = 32;        // orders (and run ends) staged per group

template <int G>
struct GrpLayout {
    static constexpr int gpw = 32 / G;  // groups per warp
    static constexpr int warps = kGrpThreads / 32;
    static constexpr int groups = kGrpThreads / G;
    static constexpr int per_lane = kBatch / G;  // staged orders each lane loads
};

__device__ __forceinline__ int lo16(unsigned w) { return (int)(short)(w & 0xffffu); }
__device__ __forceinline__ int hi16(unsigned w) { return (int)w >> 16; }

template <int G>
__device__ __forceinline__ int group_min(int v, unsigned gmask) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(gmask, v, off, G));
    return v;
}

// Replay one segment with the G lanes of gmask; j = lane index in the group.
// Returns whether any cached action of the segment changed.
template <int G, bool DUAL>
__device__ __forceinline__ bool replay_group(const KArgs& a, const int16_t* __restrict__ s_cost,
                                             int NP8, int s, const SegMeta& m, int fcp,
                                             int* fc_cur, int2* ord, int* runend,
                                             signed char* newa, unsigned gmask, int j,
                                             int it, unsigned long long& calls) {
    using Lay = GrpLayout<G>;
    const int N = a.N, NP = a.NP;
    const int k = m.k;
    const int nb = j * kWpl;  // first warehouse of this lane
    // D: counts of cached actions of product k before the current run; S: stock;
    // hist: new actions of this segment; corr: (cached - new) counts in the run
    int S[kWpl], D[kWpl], x0v[kWpl], adj[kWpl], hist[kWpl], corr[kWpl];
    // prefix counts of earlier segments; none before pass 1 of an all-a^phi cache
    const bool chained = m.ce - m.cf > 1 && (it > 1 || a.first_dirty);
#pragma unroll
    for (int i = 0; i < kWpl; ++i) {
        const int n = nb + i;
        const bool in = n < N;
        x0v[i] = in ? a.x0[(size_t)k * N + n] : 0;
        adj[i] = n - ((DUAL && in) ? 128 * a.lam[(size_t)k * N + n] : 0);  // key = score*128 + n
        D[i] = (chained && in) ? chain_prefix(a, s, m.cf, n) : 0;
        hist[i] = 0;
        corr[i] = 0;
    }
    int rwin = m.r0;  // runend[u] = end of run rwin + u
    for (int u = j; u < kBatch; u += G)
        runend[u] = u < m.r1 - rwin ? a.run_start[rwin + 1 + u] : INT_MAX;
    int pre_reg[Lay::per_lane], pre_old[Lay::per_lane];
#pragma unroll
    for (int v = 0; v < Lay::per_lane; ++v) {
        const int jj = m.j0 + j + v * G;
        pre_reg[v] = jj < m.jend ? a.reg_s[jj] : 0;
        pre_old[v] = jj < m.jend ? a.alpha_s[jj] : -1;
    }
    __syncwarp(gmask);
    int r = m.r0;
    int next_run = runend[0];
    bool eval = m.j0 > fcp;  // the run's cached prefix changed in the previous pass
    unsigned long long evals = eval ? (unsigned long long)(next_run - m.j0) : 0ull;
#pragma unroll
    for (int i = 0; i < kWpl; ++i) S[i] = max(0, x0v[i] - D[i]);
    int first_chg = INT_MAX;
    for (int base = m.j0; base < m.jend; base += kBatch) {
        const int cnt = min(kBatch, m.jend - base);
#pragma unroll
        for (int v = 0; v < Lay::per_lane; ++v) {
            const int u = j + v * G;
            if (u < cnt) ord[u] = make_int2(pre_reg[v], pre_old[v]);
        }
#pragma unroll
        for (int v = 0; v < Lay::per_lane; ++v) {  // prefetch the next batch
            const int jj = base + kBatch + j + v * G;
            if (jj < m.jend) {
                pre_reg[v] = a.reg_s[jj];
                pre_old[v] = a.alpha_s[jj];
            }
        }
        __syncwarp(gmask);
        for (int q = 0; q < cnt; ++q) {
            if (base + q == next_run) {  // close run r, open run r+1
#pragma unroll
                for (int i = 0; i < kWpl; ++i) {
                    const int s0 = max(0, x0v[i] - D[i]);
                    hist[i] += s0 - S[i];
                    D[i] += s0 - S[i] + corr[i];
                    corr[i] = 0;
                    S[i] = max(0, x0v[i] - D[i]);
                }
                ++r;
                int idx = r - rwin;
                if (idx == kBatch) {  // next window of run ends
                    rwin += kBatch;
                    idx = 0;
                    __syncwarp(gmask);
                    for (int u = j; u < kBatch; u += G)
                        runend[u] = u < m.r1 - rwin ? a.run_start[rwin + 1 + u] : INT_MAX;
                    __syncwarp(gmask);
                }
                const int nr = runend[idx];
                eval = next_run > fcp;
                if (eval) evals += (unsigned long long)(nr - next_run);
                next_run = nr;
            }
            const int2 o = ord[q];
            const uint4 cw = *reinterpret_cast<const uint4*>(s_cost + (size_t)o.x * NP8 + nb);
            const int c[kWpl] = {lo16(cw.x), hi16(cw.x), lo16(cw.y), hi16(cw.y),
                                 lo16(cw.z), hi16(cw.z), lo16(cw.w), hi16(cw.w)};
            int act = o.y;  // unchanged prefix: the cached action is the policy's
            if (eval) {
                int key = INT_MAX;
#pragma unroll
                for (int i = 0; i < kWpl; ++i) key = min(key, S[i] > 0 ? c[i] * 128 + adj[i] : INT_MAX);
                key = group_min<G>(key, gmask);
                act = key == INT_MAX ? -1 : (key & 127);
            }
            const int sel = act - nb;
#pragma unroll
            for (int i = 0; i < kWpl; ++i) S[i] -= (sel == i);
            if (act != o.y) {  // group-uniform
                const int osel = o.y - nb;
#pragma unroll
                for (int i = 0; i < kWpl; ++i) corr[i] += (osel == i) - (sel == i);
            }
            if (j == 0) newa[q] = (signed char)act;
        }
        __syncwarp(gmask);
        int fcl = INT_MAX;  // first change in this batch
        for (int u = j; u < cnt; u += G) {
            const int na = newa[u];
            a.alpha_s[base + u] = (int8_t)na;
            if (na != ord[u].y) fcl = min(fcl, base + u);
        }
        first_chg = min(first_chg, group_min<G>(fcl, gmask));
        __syncwarp(gmask);
    }
#pragma unroll
    for (int i = 0; i < kWpl; ++i) {
        const int s0 = max(0, x0v[i] - D[i]);
        hist[i] += s0 - S[i];
        if (nb + i < NP) a.agg[(size_t)s * NP + nb + i] = hist[i];
    }
    // many segments of a popular product change in the same pass: read before
    // the atomic so that only a new minimum contends for the word
    if (j == 0 && first_chg != INT_MAX && first_chg < ld_volatile(&fc_cur[k]))
        atomicMin(&fc_cur[k], first_chg);
    if (s == m.ce - 1) {  // last segment of the product: its end state is the final stock
#pragma unroll
        for (int i = 0; i < kWpl; ++i)
            if (nb + i < N) a.xfin[(size_t)k * N + nb + i] = S[i];
    }
    if (j == 0) calls += evals;
    return first_chg != INT_MAX;
}

template <int G, int NPL, bool DUAL>
__global__ void __launch_bounds__(kGrpThreads, 1) k_picard_grp(KArgs a, int NP8) {
    using Lay = GrpLayout<G>;
    extern __shared__ __align__(16) unsigned char s_dyn[];  // int16 cost table [R][NP8]
    int16_t* s_cost = reinterpret_cast<int16_t*>(s_dyn);
    __shared__ int s_changed;
    // per warp: the active segments of the 32 positions being examined
    __shared__ SegMeta s_meta[Lay::warps][32];
    __shared__ int s_fcp[Lay::warps][32];
    __shared__ int s_seg[Lay::warps][32];
    // per group: staged orders (region, cached action), run ends, new actions
    __shared__ int2 s_ord[Lay::groups][kBatch];
    __shared__ int s_runend[Lay::groups][kBatch];
    __shared__ signed char s_new[Lay::groups][kBatch];

    const int N = a.N;
    for (int i = threadIdx.x; i < a.R * NP8; i += blockDim.x) {
        const int rr = i / NP8, n = i - rr * NP8;
        s_cost[i] = n < N ? (int16_t)a.cost[(size_t)rr * N + n] : (int16_t)0;
    }
    if (threadIdx.x == 0) s_changed = 0;
    __syncthreads();

    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;  // warp in block
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    const int g = lane / G, jg = lane % G;
    const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << (g * G));
    const int gib = threadIdx.x / G;  // group in block
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    const int nseg = a.ctrl->nseg;
    const bool no_reset = (a.flags & PIC_FLAG_NO_RESET) != 0;
    const unsigned tag_base = ld_volatile(&a.ctrl->tag_base);
    unsigned long long calls = 0, replays = 0;
    const unsigned long long t_start = globaltimer_ns();
    int it = 1;
    bool ok = true, converged = false;
    for (; it <= a.max_iters; ++it) {
        const int parity = it & 1;
        long long* tr = (a.trace && it <= kTraceCap) ? a.trace + kTraceCols * (it - 1) : nullptr;
        const unsigned long long calls0 = calls, replays0 = replays;
        const int* fc_prev = a.fc + (size_t)(parity ^ 1) * a.K;
        int* fc_cur = a.fc + (size_t)parity * a.K;
        // ---- phase S: chain prefixes (warp per super-block, natural segment order)
        for (int k = gtid; k < a.K; k += gthreads) fc_cur[k] = INT_MAX;
        if (gtid == 0) a.ctrl->changed[parity] = 0;
        if (it > 1 || a.first_dirty)
            chain_prefixes<NPL>(a, it, fc_prev, tag_base + (unsigned)it, deadline, s_meta[wib],
                                s_fcp[wib]);
        if (!grid_sync(a.ctrl, deadline)) { ok = false; break; }
        if (tr && gtid == 0) tr[0] = (long long)(globaltimer_ns() - t_start);
        // ---- phase R: longest-first positions dealt to warps in a snake; each
        // warp queues the active ones of 32 positions and its groups take turns
        bool chg = false;
        for (int j0 = 0; j0 * nwarps < nseg; j0 += 32) {
            const int jj = j0 + lane;
            const int pos = jj * nwarps + ((jj & 1) ? nwarps - 1 - gwarp : gwarp);
            bool act = false;
            int sl = 0, fcp = -1;
            SegMeta m;
            if (pos < nseg) {
                sl = a.lpt[pos];
                m = load_meta(a.meta + sl);
                fcp = no_reset ? -1 : fc_prev[m.k];
                act = m.last_start > fcp;
            }
            const unsigned bal = __ballot_sync(kFull, act);
            if (act) {
                const int e = __popc(bal & ((1u << lane) - 1u));
                s_meta[wib][e] = m;
                s_fcp[wib][e] = fcp;
                s_seg[wib][e] = sl;
            }
            __syncwarp();
            const int qn = __popc(bal);
            for (int e = g; e < qn; e += Lay::gpw) {
                const SegMeta mm = smem_meta(&s_meta[wib][e]);
                chg |= replay_group<G, DUAL>(a, s_cost, NP8, s_seg[wib][e], mm, s_fcp[wib][e],
                                             fc_cur, s_ord[gib], s_runend[gib], s_new[gib], gmask,
                                             jg, it, calls);
                if (jg == 0) replays += 1;
            }
            __syncwarp();
        }
        if (tr) {
            const unsigned dc = __reduce_add_sync(kFull, (unsigned)(calls - calls0));
            const unsigned dr = __reduce_add_sync(kFull, (unsigned)(replays - replays0));
            if (lane == 0 && dr) {
                atomicAdd((unsigned long long*)&tr[2], (unsigned long long)dc);
                atomicAdd((unsigned long long*)&tr[3], (unsigned long long)dr);
            }
        }
        if (__any_sync(kFull, chg) && lane == 0) s_changed = 1;  // one global write per CTA, below
        __syncthreads();
        if (threadIdx.x == 0 && s_changed) {
            a.ctrl->changed[parity] = 1;
            s_changed = 0;
        }
        if (!grid_sync(a.ctrl, deadline)) { ok = false; break; }
        if (tr && gtid == 0) tr[1] = (long long)(globaltimer_ns() - t_start);
        if (ld_volatile(&a.ctrl->changed[parity]) == 0) { converged = true; break; }
    }
    // totals: each lane counted only its own group's work (group lane 0)
    unsigned long long c = calls, rp = replays;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(kFull, c, o);
        rp += __shfl_xor_sync(kFull, rp, o);
    }
    if (lane == 0 && rp) {
        atomicAdd(&a.ctrl->policy_calls, c);
        atomicAdd(&a.ctrl->seg_replays, rp);
    }
    if (gtid == 0 && ok) {
        a.ctrl->iters = converged ? it : a.max_iters;
        a.ctrl->converged = converged ? 1 : 0;
    }
}

template <int G, int NPL, bool DUAL>
cudaError_t launch_grp(Instance* I, const KArgs& a, cudaStream_t st) {
    auto kern = k_picard_grp<G, NPL, DUAL>;
    const int NP8 = G * kWpl;
    const size_t smem = (size_t)I->R * NP8 * sizeof(int16_t);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kGrpThreads, smem);
    if (e) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int grid = I->num_sms;  // one CTA per SM: every SM stages the cost table once
    I->coop_blocks = grid;
    I->cta_threads = kGrpThreads;
    I->ctas_per_sm = 1;
    KArgs args = a;
    int np8 = NP8;
    void* params[] = {&args, &np8};
    I->launches += 1;
    return cudaLaunchCooperativeKernel((const void*)kern, grid, kGrpThreads, params, smem, st);
}

template <int G, int NPL>
cudaError_t grp_dual(Instance* I, const KArgs& a, bool dual, cudaStream_t st) {
    return dual ? launch_grp<G, NPL, true>(I, a, st) : launch_grp<G, NPL, false>(I, a, st);
}

}  // namespace

int grp_lanes(int N) { return N <= 32 ? 4 : (N <= 64 ? 8 : 16); }

bool grp_ok(const Instance* I) {
    if (!I->cost16 || I->N < 17) return false;
    const int G = grp_lanes(I->N);
    const size_t dyn = (size_t)I->R * G * kWpl * sizeof(int16_t);
    return dyn <= kGrpSmemMax;
}

cudaError_t picard_grp(Instance* I, const KArgs& a, bool dual, cudaStream_t st) {
    const int npl = (I->N + 31) / 32;
    switch (grp_lanes(I->N)) {
        case 4: return grp_dual<4, 1>(I, a, dual, st);
        case 8: return npl == 1 ? grp_dual<8, 1>(I, a, dual, st) : grp_dual<8, 2>(I, a, dual, st);
        default:
            return npl <= 2 ? (npl == 2 ? grp_dual<16, 2>(I, a, dual, st) : grp_dual<16, 1>(I, a, dual, st))
                            : (npl == 3 ? grp_dual<16, 3>(I, a, dual, st) : grp_dual<16, 4>(I, a, dual, st));
    }
}

}  // namespace pic
