// Pieces shared by the Picard kernels (warp-per-segment and group-per-segment):
// the argument block, the staged cost table, packed segment metadata, and the
// phase that turns per-segment histograms of cached actions into per-segment
// prefix counts (decoupled look-back over super-blocks of 32 segments).
#pragma once

#include "pic_device.cuh"

namespace pic {
namespace picard {

struct KArgs {
    int T, N, K, NP, R;
    const int32_t* __restrict__ reg_s;
    const int32_t* __restrict__ run_start;
    const int32_t* __restrict__ seg_run;
    const int32_t* __restrict__ seg_prod;
    const int32_t* __restrict__ seg_cf;
    const int32_t* __restrict__ seg_ce;
    const SegMeta* __restrict__ meta;
    const int32_t* __restrict__ lpt;
    const int32_t* __restrict__ x0;
    const int32_t* __restrict__ cost;
    const int32_t* __restrict__ lam;
    int8_t* alpha_s;
    int32_t* __restrict__ agg;
    int32_t* __restrict__ carry;
    int32_t* __restrict__ sbexc;
    unsigned long long* sbagg;   // tagged super-block totals
    unsigned long long* sbincl;  // tagged inclusive prefixes
    int32_t* fc;
    int32_t* xfin;
    Ctrl* ctrl;
    int max_iters;
    int flags;
    int first_dirty;
    unsigned long long timeout_ns;
    long long* trace;  // per-pass record or nullptr
    // max_steps window (Appendix A.3), or run_chunk == nullptr: no window
    const int32_t* __restrict__ run_chunk;  // [runs] time block of each run
    const int32_t* __restrict__ perm;       // [T] sorted position -> time
    int win_steps;                          // max_steps
    int M, L;                               // chunks and chunk length
};

// Whether a run is evaluated in this pass.  Without a window: its start lies
// after its product's first change of the previous pass (t_reset).  With the
// window [0, hi) in chunks: the run's chunk is inside it, and either t_reset
// says so or the chunk was outside the previous pass's window (its cache was
// not computed from the current prefix).
__device__ __forceinline__ bool run_evaluated(const KArgs& a, int whi, int wprev, int r,
                                              bool after_change) {
    if (!a.run_chunk) return after_change;
    const int c = __ldg(a.run_chunk + r);
    return c < whi && (after_change || c >= wprev);
}

// A replay that changed a cached action reports the time of its first change
// (lane 0; sorted position j) for the window's t_reset.
__device__ __forceinline__ void report_window_change(const KArgs& a, int it, int j) {
    if (a.run_chunk && j != INT_MAX) atomicMin(&a.ctrl->win_fct[it & 1], __ldg(a.perm + j));
}

template <bool SMEM>
struct CostTable {
    const int32_t* __restrict__ g;
    const int16_t* s;
    int N;
    __device__ __forceinline__ int at(int r, int n) const {
        if (SMEM) return s[r * N + n];
        return __ldg(g + (size_t)r * N + n);
    }
};

template <bool SMEM>
__device__ __forceinline__ CostTable<SMEM> stage_cost(const KArgs& a) {
    extern __shared__ int16_t s_cost[];
    CostTable<SMEM> ct{a.cost, s_cost, a.N};
    if (SMEM) {
        const int n = a.R * a.N;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s_cost[i] = (int16_t)a.cost[i];
        __syncthreads();
    }
    return ct;
}

__device__ __forceinline__ SegMeta load_meta(const SegMeta* p) {
    const int4* q = reinterpret_cast<const int4*>(p);
    const int4 u = __ldg(q), v = __ldg(q + 1);
    SegMeta m;
    m.k = u.x; m.r0 = u.y; m.r1 = u.z; m.j0 = u.w;
    m.jend = v.x; m.last_start = v.y; m.cf = v.z; m.ce = v.w;
    return m;
}

__device__ __forceinline__ SegMeta smem_meta(const SegMeta* p) {
    const int4* q = reinterpret_cast<const int4*>(p);
    const int4 u = q[0], v = q[1];
    SegMeta m;
    m.k = u.x; m.r0 = u.y; m.r1 = u.z; m.j0 = u.w;
    m.jend = v.x; m.last_start = v.y; m.cf = v.z; m.ce = v.w;
    return m;
}

// The exclusive chain prefix of agg at segment s (chain from cf) for warehouse
// n: its super-block's prefix over the earlier super-blocks plus its own prefix
// inside the super-block.
__device__ __forceinline__ int chain_prefix(const KArgs& a, int s, int cf, int n) {
    const int head = s - (s - cf) % kSuperBlock;
    return a.carry[(size_t)s * a.NP + n] + a.sbexc[(size_t)head * a.NP + n];
}

constexpr int kMaxWarpsPerCta = 32;

// Look-back words carry a tag in the high half: (tag << 32) | value with tag =
// ctrl->tag_base + pass, unique over the calls on one instance, so a reader
// learns from the word itself whether it was written in this pass of this call
// (no clearing between calls).  The poll is a volatile relaxed load so that every spin really
// re-reads memory.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long tagged(unsigned tag, int v) {
    return ((unsigned long long)tag << 32) | (unsigned)v;
}

// Phase S for one super-block (head segment s of a chain whose product changed):
// its total, published; then the exclusive prefix of the chain's earlier
// super-blocks by decoupled look-back (an inclusive prefix ends the walk, a bare
// total is added and the walk continues); the inclusive prefix, published; then
// the exclusive prefix at every segment of the block.  A block whose orders all
// precede the product's first change (clean) keeps last pass's prefixes and only
// re-publishes them.  Waits are bounded by the deadline; on expiry the error is
// recorded and the pass is abandoned at the next grid barrier.
// ROWS: histogram rows loaded per round trip (a whole super-block when
// registers allow).
// SPLIT: carry holds the prefix inside the super-block (written while the
// totals are summed) and sbexc the super-block's prefix over the chain (read
// through chain_prefix); otherwise carry holds the whole chain prefix (a second
// pass over the super-block's rows; the capacity kernel, which reads one row per
// run).
template <int NPL, int ROWS = 16 / NPL, bool SPLIT = true>
__device__ __forceinline__ void superblock_prefix(const KArgs& a, int s, const SegMeta& m, int it,
                                                  unsigned tag, int fcp,
                                                  unsigned long long deadline) {
    const int lane = lane_id();
    const int NP = a.NP;
    const int send = min(s + kSuperBlock, m.ce);
    constexpr int kRows = ROWS;
    // the shortcut needs last pass's prefixes: pass 1 computes none unless the
    // cache started from alpha_init
    if (send < m.ce && (it > 2 || (it == 2 && a.first_dirty))) {
        const int next_j0 = __ldg(&a.meta[send].j0);
        if (next_j0 <= fcp) {  // clean: aggregates and prefixes unchanged
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const size_t o = (size_t)s * NP + lane + 32 * i;
                a.sbincl[o] = tagged(tag, (int)(unsigned)a.sbincl[o]);
            }
            return;
        }
    }
    // the super-block's total, writing every segment's prefix inside it on the way
    int tot[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) tot[i] = 0;
    for (int s2 = s; s2 < send; s2 += kRows) {
        int v[kRows][NPL];
#pragma unroll
        for (int u = 0; u < kRows; ++u)
#pragma unroll
            for (int i = 0; i < NPL; ++i)
                v[u][i] = s2 + u < send ? a.agg[(size_t)(s2 + u) * NP + lane + 32 * i] : 0;
#pragma unroll
        for (int u = 0; u < kRows; ++u)
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                if (SPLIT && s2 + u < send) a.carry[(size_t)(s2 + u) * NP + lane + 32 * i] = tot[i];
                tot[i] += v[u][i];
            }
    }
    int acc[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) acc[i] = 0;
    if (s > m.cf) {
#pragma unroll
        for (int i = 0; i < NPL; ++i) a.sbagg[(size_t)s * NP + lane + 32 * i] = tagged(tag, tot[i]);
        bool fail = false;
        for (int p = s - kSuperBlock; p >= m.cf && !fail; p -= kSuperBlock) {
            while (true) {
                unsigned long long wi[NPL], wa[NPL];
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    wi[i] = ld_relaxed_u64(a.sbincl + (size_t)p * NP + lane + 32 * i);
                    wa[i] = ld_relaxed_u64(a.sbagg + (size_t)p * NP + lane + 32 * i);
                }
                bool inc_ok = true, agg_ok = true;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    inc_ok &= (unsigned)(wi[i] >> 32) == tag;
                    agg_ok &= (unsigned)(wa[i] >> 32) == tag;
                }
                if (__all_sync(kFull, inc_ok)) {
#pragma unroll
                    for (int i = 0; i < NPL; ++i) acc[i] += (int)(unsigned)wi[i];
                    p = -1;  // walk done
                    break;
                }
                if (__all_sync(kFull, agg_ok)) {
#pragma unroll
                    for (int i = 0; i < NPL; ++i) acc[i] += (int)(unsigned)wa[i];
                    break;
                }
                if (globaltimer_ns() > deadline) {
                    if (lane == 0) atomicCAS(&a.ctrl->err, 0, (int)PIC_ERR_TIMEOUT);
                    fail = true;
                    break;
                }
                if (ld_volatile(&a.ctrl->err)) { fail = true; break; }
            }
            if (p < 0) break;
        }
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        a.sbincl[(size_t)s * NP + lane + 32 * i] = tagged(tag, acc[i] + tot[i]);
        if (SPLIT) a.sbexc[(size_t)s * NP + lane + 32 * i] = acc[i];
    }
    if (!SPLIT) {
        for (int s2 = s; s2 < send; s2 += kRows) {
            int v[kRows][NPL];
#pragma unroll
            for (int u = 0; u < kRows; ++u)
#pragma unroll
                for (int i = 0; i < NPL; ++i)
                    v[u][i] = s2 + u < send ? a.agg[(size_t)(s2 + u) * NP + lane + 32 * i] : 0;
#pragma unroll
            for (int u = 0; u < kRows; ++u)
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    if (s2 + u < send) a.carry[(size_t)(s2 + u) * NP + lane + 32 * i] = acc[i];
                    acc[i] += v[u][i];
                }
        }
    }
}


// Phase S of one pass, for every warp of the grid: the super-block heads of
// chains whose product changed in the previous pass (every chain in pass 1 of
// a cache started from alpha_init) are assigned to warps gwarp + j * nwarps, 32
// at a time, and run superblock_prefix.  s_meta / s_fcp: this warp's staging
// rows (32 entries each).
template <int NPL, int ROWS = 16 / NPL, bool SPLIT = true>
__device__ __forceinline__ void chain_prefixes(const KArgs& a, int it, const int* fc_prev,
                                               unsigned tag, unsigned long long deadline,
                                               SegMeta* s_meta, int* s_fcp) {
    const int lane = lane_id();
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nseg = a.ctrl->nseg;
    for (int j0 = 0; gwarp + j0 * nwarps < nseg; j0 += 32) {
        const int sl = gwarp + (j0 + lane) * nwarps;
        bool head = false;
        if (sl < nseg) {
            const SegMeta m = load_meta(a.meta + sl);
            head = m.ce - m.cf > 1 && (sl - m.cf) % kSuperBlock == 0;
            const int f = it > 1 ? fc_prev[m.k] : -1;
            if (head && it > 1) head = f != INT_MAX;
            if (head) {
                s_meta[lane] = m;
                s_fcp[lane] = f;
            }
        }
        unsigned todo = __ballot_sync(kFull, head);
        while (todo) {  // increasing segment order (lane order)
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const SegMeta mm = smem_meta(&s_meta[src]);
            superblock_prefix<NPL, ROWS, SPLIT>(a, gwarp + (j0 + src) * nwarps, mm, it, tag, s_fcp[src],
                                         deadline);
        }
        __syncwarp();
    }
}


// Algorithm 1's passes inside one persistent cooperative launch; every thread
// of the grid calls this.  Each pass:
//   phase S  chain prefixes of the per-segment histograms of cached actions
//            (superblock_prefix, one warp per super-block head of a chain whose
//            product changed in the previous pass);
//   phase R  active segments replayed, one warp each: positions of the
//            longest-first order are dealt to CTAs in a snake (c, 2C-1-c,
//            2C+c, ...); a CTA examines its positions with all its threads at
//            once, lists the active ones in order in shared memory, and its
//            warps take them one at a time (a shared-memory ticket), so that a
//            warp that finishes early takes the next unit of its CTA (GROUP > 1:
//            positions dealt to groups of warps in a snake, 32 at a time per
//            group);
//            replay(seg, meta, fcp, fc_cur, it) replays one of them and returns
//            whether it changed a cached action (warp-uniform; it adds its
//            policy calls to `calls` on lane 0); the trace records the pass's
//            largest unit (policy calls, orders walked), its critical path;
// separated by grid barriers.  The loop ends at the first pass that changes no
// cached action (line 13 of Algorithm 1), or after max_iters passes.
// GROUP > 1: work units go to groups of GROUP consecutive warps of a CTA (each
// warp of a group walks the same candidates and calls replay for the same
// segment; the replay shares its decisions); the group's first warp counts.
// CTA: phase R is one call for the whole CTA, replay(fc_prev, fc_cur, it, whi,
// wprev, replays, ucalls, uorders), which deals the pass's work units itself
// and returns whether it changed a cached action (CTA-uniform); its counts are
// kept by thread 0 (calls, replays, the largest unit's calls and orders), and
// phase S stages its segments in ext_meta / ext_fcp (WARPS x 32 entries, e.g.
// dynamic shared memory that phase R uses otherwise).
// SPLIT: the chain prefixes' layout (superblock_prefix); the replay reads them
// accordingly.
template <int NPL, int WARPS, class Replay, int GROUP = 1, bool CTA = false, bool SPLIT = true>
__device__ __forceinline__ void picard_passes(const KArgs& a, unsigned long long& calls,
                                              Replay&& replay, SegMeta* ext_meta = nullptr,
                                              int* ext_fcp = nullptr) {
    __shared__ int s_changed;
    // per warp: the 32 segments it is examining (metadata, previous-pass first
    // change); in phase R with GROUP == 1, the CTA's list of active units
    __shared__ SegMeta s_meta[CTA ? 1 : WARPS][32];
    __shared__ int s_fcp[CTA ? 1 : WARPS][32];
    __shared__ int s_seg[(CTA || GROUP > 1) ? 1 : WARPS * 32];
    __shared__ int s_wcnt[(CTA || GROUP > 1) ? 1 : WARPS];
    __shared__ int s_ticket;
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    const int nseg = a.ctrl->nseg;
    const bool no_reset = (a.flags & PIC_FLAG_NO_RESET) != 0;
    const unsigned tag_base = ld_volatile(&a.ctrl->tag_base);
    if (threadIdx.x == 0) s_changed = 0;
    __syncthreads();
    unsigned long long replays = 0;
    const unsigned long long t_start = globaltimer_ns();
    int it = 1;
    bool ok = true, converged = false;
    // max_steps window (identical in every thread): evaluated chunks [0, whi),
    // previous pass [0, wprev)
    const bool win = a.run_chunk != nullptr;
    long long wstart = 0;
    int wprev = win ? 0 : INT_MAX;
    int whi = win ? (int)min((long long)a.M, ((long long)a.win_steps + a.L - 1) / a.L) : INT_MAX;
    for (; it <= a.max_iters; ++it) {
        const int parity = it & 1;
        long long* tr = (a.trace && it <= kTraceCap) ? a.trace + kTraceCols * (it - 1) : nullptr;
        const unsigned long long calls0 = calls, replays0 = replays;
        const int* fc_prev = a.fc + (size_t)(parity ^ 1) * a.K;
        int* fc_cur = a.fc + (size_t)parity * a.K;
        // ---- phase S: this warp's segments gwarp + j * nwarps, 32 at a time
        for (int k = gtid; k < a.K; k += gthreads) fc_cur[k] = INT_MAX;
        if (gtid == 0) {
            a.ctrl->changed[parity] = 0;
            a.ctrl->win_fct[parity] = INT_MAX;
            a.ctrl->win_hi = whi;
            a.ctrl->win_hi_prev = wprev;
        }
        if (it > 1 || a.first_dirty)
            chain_prefixes<NPL, 16 / NPL, SPLIT>(a, it, fc_prev, tag_base + (unsigned)it, deadline,
                                CTA ? ext_meta + 32 * wib : s_meta[wib],
                                CTA ? ext_fcp + 32 * wib : s_fcp[wib]);
        if (!grid_sync(a.ctrl, deadline)) { ok = false; break; }
        if (tr && gtid == 0) tr[0] = (long long)(globaltimer_ns() - t_start);
        // ---- phase R
        bool chg = false;
        unsigned long long ucalls = 0, uorders = 0;  // largest unit of this warp (lane 0)
        const int unit = gwarp / GROUP, nunits = nwarps / GROUP;
        if constexpr (CTA) {
            chg = replay(fc_prev, fc_cur, it, whi, wprev, replays, ucalls, uorders);
        } else if constexpr (GROUP == 1) {
            // this CTA's positions j * C + (j odd ? C - 1 - b : b), a list of
            // WARPS * 32 at a time
            const int C = gridDim.x, b = blockIdx.x;
            const int npos = (nseg + C - 1) / C;  // rounds j; a position past nseg is skipped
            SegMeta* L_meta = &s_meta[0][0];
            int* L_fcp = &s_fcp[0][0];
            for (int base = 0; base < npos; base += WARPS * 32) {
                const int j = base + (int)threadIdx.x;
                bool act = false;
                SegMeta m;
                int sl = 0, fcp = 0;
                if (j < npos) {
                    const int pos = j * C + ((j & 1) ? C - 1 - b : b);
                    if (pos < nseg) {
                        sl = a.lpt[pos];
                        m = load_meta(a.meta + sl);
                        fcp = no_reset ? -1 : fc_prev[m.k];
                        act = m.last_start > fcp;  // some run starts after the first change
                        if (win) {  // ... or entered the window; and some run is inside it
                            const int c0 = __ldg(a.run_chunk + m.r0), c1 = __ldg(a.run_chunk + m.r1 - 1);
                            act = c0 < whi && (act || c1 >= wprev);
                        }
                    }
                }
                // the active units in position order: rank in the warp, then warp offsets
                const unsigned bal = __ballot_sync(kFull, act);
                if (lane == 0) s_wcnt[wib] = __popc(bal);
                if (threadIdx.x == 0) s_ticket = 0;
                __syncthreads();
                int off = 0, total = 0;
                for (int w = 0; w < WARPS; ++w) {
                    const int c = s_wcnt[w];
                    off += w < wib ? c : 0;
                    total += c;
                }
                if (act) {
                    const int idx = off + __popc(bal & ((1u << lane) - 1u));
                    L_meta[idx] = m;
                    L_fcp[idx] = fcp;
                    s_seg[idx] = sl;
                }
                __syncthreads();
                while (true) {
                    int u = 0;
                    if (lane == 0) u = atomicAdd(&s_ticket, 1);
                    u = __shfl_sync(kFull, u, 0);
                    if (u >= total) break;
                    const SegMeta mm = smem_meta(&L_meta[u]);
                    const unsigned long long cu0 = calls;
                    chg |= replay(s_seg[u], mm, L_fcp[u], fc_cur, it);
                    replays += 1;
                    if (calls - cu0 > ucalls) ucalls = calls - cu0;
                    if ((unsigned long long)(mm.jend - mm.j0) > uorders) uorders = mm.jend - mm.j0;
                }
                __syncthreads();  // the list is read until every warp is done
            }
        } else {
        for (int j0 = 0; j0 * nunits < nseg; j0 += 32) {
            const int j = j0 + lane;
            const int pos = j * nunits + ((j & 1) ? nunits - 1 - unit : unit);
            int sl = nseg;
            bool act = false;
            if (pos < nseg) {
                sl = a.lpt[pos];
                const SegMeta m = load_meta(a.meta + sl);
                const int fcp = no_reset ? -1 : fc_prev[m.k];
                act = m.last_start > fcp;  // some run starts after the first change
                if (win) {  // ... or entered the window; and some run is inside it
                    const int c0 = __ldg(a.run_chunk + m.r0), c1 = __ldg(a.run_chunk + m.r1 - 1);
                    act = c0 < whi && (act || c1 >= wprev);
                }
                if (act) {
                    s_meta[wib][lane] = m;
                    s_fcp[wib][lane] = fcp;
                }
            }
            unsigned todo = __ballot_sync(kFull, act);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const SegMeta mm = smem_meta(&s_meta[wib][src]);
                const int seg = __shfl_sync(kFull, sl, src);
                const unsigned long long cu0 = calls;
                chg |= replay(seg, mm, s_fcp[wib][src], fc_cur, it);
                if (wib % GROUP == 0) replays += 1;
                if (calls - cu0 > ucalls) ucalls = calls - cu0;
                if ((unsigned long long)(mm.jend - mm.j0) > uorders) uorders = mm.jend - mm.j0;
            }
            __syncwarp();
        }
        }
        if (tr && lane == 0 && replays != replays0) {
            atomicAdd((unsigned long long*)&tr[2], calls - calls0);
            atomicAdd((unsigned long long*)&tr[3], replays - replays0);
            atomicMax((unsigned long long*)&tr[4], ucalls);
            atomicMax((unsigned long long*)&tr[5], uorders);
        }
        if (chg && lane == 0) s_changed = 1;  // one global write per CTA, below
        __syncthreads();
        if (threadIdx.x == 0 && s_changed) {
            a.ctrl->changed[parity] = 1;
            s_changed = 0;
        }
        if (!grid_sync(a.ctrl, deadline)) { ok = false; break; }
        if (tr && gtid == 0) tr[1] = (long long)(globaltimer_ns() - t_start);
        const bool changed = ld_volatile(&a.ctrl->changed[parity]) != 0;
        if (!win) {
            if (!changed) { converged = true; break; }
            continue;
        }
        // the window: evaluated orders end at e; it restarts at the first change,
        // or moves past e once it changed nothing (Appendix A.3)
        const long long e = min((long long)a.T, (long long)whi * a.L);
        if (!changed) {
            if (e >= a.T) { converged = true; break; }
            wstart = e;
        } else {
            wstart = ld_volatile(&a.ctrl->win_fct[parity]);
        }
        wprev = whi;
        whi = (int)min((long long)a.M, (wstart + a.win_steps + a.L - 1) / a.L);
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

}  // namespace picard

// MLP Picard kernel (pic_mlp.cu).
cudaError_t picard_mlp(Instance* I, const picard::KArgs& a, const pic_policy* pol, cudaStream_t st);



// Group-per-segment Picard kernel (pic_grp.cu).
int grp_lanes(int N);
bool grp_ok(const Instance* I);
cudaError_t picard_grp(Instance* I, const picard::KArgs& a, bool dual, cudaStream_t st);

}  // namespace pic
