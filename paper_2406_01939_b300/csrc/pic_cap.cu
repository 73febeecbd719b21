// FO with node capacity (Sec. 3): the state is (x, c); an order of product k
// may go to node n only if x[k][n] > 0 and c[n] > 0, and f decrements both.
// Greedy and bid-price policies (the integer policies of pic_int.cu) choose over
// that feasible set.
//
// Capacity couples the products, so a time chunk of Algorithm 1 can no longer be
// split into independent per-product runs: process m (chunk m) replays its
// orders in time order.  Its start state is the cached prefix (Alg. 1 lines 5-7)
// in closed form.  While cached actions are replayed every decrement is
// conditional on positivity, and a node whose capacity reached 0 stays
// infeasible, so at the chunk start
//   x[k][n] = max(0, x0[k][n] - d[k][n])  at every node with c[n] > 0,
//   c[n]    = max(0, c_1[n] - q[n]),
// with d[k][n] the cached actions of product k naming n before the chunk (the
// per-run chain prefix of the inventory-only kernel, phase S) and q[n] those
// cached actions that found inventory.  Within one run of product k the cached
// actions naming n that found inventory number min(h[n], max(0, x0[k][n] -
// d[k][n])), h the run's histogram of cached actions, so q needs no walk over
// orders: it is a prefix over chunks of per-chunk sums.
//
// One persistent cooperative launch runs every pass:
//   phase S  chain prefixes d per run (superblock_prefix, with segments of one
//            run each);
//   phase C  one warp per chunk, chunks dealt in increasing order: stage the
//            start rows of the chunk's runs in shared memory and add up the
//            chunk's q; publish it, then take the prefix of q over earlier
//            chunks by a decoupled look-back (tagged words, as in phase S) and
//            publish the inclusive prefix; then replay the chunk's orders in
//            time order with fresh policy calls, write the cache, the runs'
//            histograms of new actions and the final stock of every product
//            whose last run is in the chunk;
// separated by grid barriers; the loop ends at the first pass that changes no
// cached action.  t_reset (Appendix A.3) is global here, because capacity
// couples all orders: with f the first time changed in the previous pass, a
// chunk that ends at or before f keeps its cache and its prefix of q, and a
// chunk that starts at or before f keeps its cache but recomputes its q.
#include "pic_picard.cuh"

namespace pic {

namespace {

using namespace picard;

constexpr int kCapWarps = 4;  // warps per CTA
constexpr int kAheadCap = 8;  // orders whose cost and price rows are loaded together

// Phase S loads a whole super-block of histogram rows per round trip when the
// registers allow (one run per segment makes phase S the larger part of a pass).
template <int NPL>
constexpr int kPrefixRows = NPL <= 2 ? kSuperBlock : 8;

// order-info bits (cap_info)
constexpr int kInfoSlot = 0xff;
constexpr int kInfoFirst = 1 << 8;     // first order of its run
constexpr int kInfoLastProd = 1 << 10; // last order of its product

struct CapArgs {
    int M, L;                              // chunks, chunk length
    const int32_t* __restrict__ prod;      // [T] time order
    const int32_t* __restrict__ reg;       // [T]
    const int32_t* __restrict__ info;      // [T] slot | flags
    const int32_t* __restrict__ run_t;     // [T] run of order t
    const int32_t* __restrict__ inv;       // [T] sorted position of order t
    const int32_t* __restrict__ cap;       // [N] c_1
    int8_t* act;                           // [T] the cache, time order
    unsigned long long* qagg;              // [M][NP] tagged chunk totals of q
    unsigned long long* qinc;              // [M][NP] tagged inclusive prefixes of q
};

// ---------------------------------------------------------------- tables
// Over sorted positions j: run and sorted position of order t = perm[j], and
// whether t is its run's first order.
__global__ void k_cap_order(const int32_t* __restrict__ perm, const int32_t* __restrict__ run_of,
                            const int32_t* __restrict__ run_start, int T, int32_t* __restrict__ run_t,
                            int32_t* __restrict__ inv, int32_t* __restrict__ first_t) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= T) return;
    const int t = perm[j], r = run_of[j];
    run_t[t] = r;
    inv[t] = (int)j;
    first_t[t] = run_start[r] == (int)j;
}

// Over times t: the slot of t's run in its chunk (runs numbered by their first
// order's time; first_ex = exclusive prefix of the first-order flags), and the
// flags first-of-run, last-of-run, last-of-product.
__global__ void k_cap_info(const int32_t* __restrict__ run_t, const int32_t* __restrict__ inv,
                           const int32_t* __restrict__ first_ex, const int32_t* __restrict__ run_start,
                           const int32_t* __restrict__ perm, const int32_t* __restrict__ prod,
                           const int32_t* __restrict__ pstart, int T, int L, int32_t* __restrict__ info) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int r = run_t[t], j = inv[t];
    const int j0 = run_start[r], j1 = run_start[r + 1];
    const int tf = perm[j0];  // first order of the run: same chunk as t
    const long long c0 = (t / L) * L;
    const int slot = first_ex[tf] - first_ex[c0];
    const int k = prod[t];
    info[t] = slot | (j == j0 ? kInfoFirst : 0) | (j == j1 - 1 ? (1 << 9) : 0) |
              (j == pstart[k + 1] - 1 ? kInfoLastProd : 0);
}

// The cache in time order from alpha_init (entries outside [-1, N) become a^phi;
// init_cache reports them).
__global__ void k_cap_cache(const int8_t* __restrict__ alpha_init, int T, int N,
                            int8_t* __restrict__ act) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int v = alpha_init[t];
    act[t] = (int8_t)((v < -1 || v >= N) ? -1 : v);
}

// ---------------------------------------------------------------- one chunk
// Prefix of q over chunks before m (decoupled look-back): adds to acc and
// returns false if the deadline passed or another CTA raised an error.
template <int NPL>
__device__ __forceinline__ bool lookback_q(const CapArgs& c, const KArgs& a, int m, unsigned tag,
                                           int acc[NPL], unsigned long long deadline) {
    const int lane = lane_id();
    const int NP = a.NP;
    for (int p = m - 1; p >= 0;) {
        unsigned long long wi[NPL], wa[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            wi[i] = ld_relaxed_u64(c.qinc + (size_t)p * NP + lane + 32 * i);
            wa[i] = ld_relaxed_u64(c.qagg + (size_t)p * NP + lane + 32 * i);
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
            return true;
        }
        if (__all_sync(kFull, agg_ok)) {
#pragma unroll
            for (int i = 0; i < NPL; ++i) acc[i] += (int)(unsigned)wa[i];
            --p;
            continue;
        }
        if (globaltimer_ns() > deadline) {
            if (lane == 0) atomicCAS(&a.ctrl->err, 0, (int)PIC_ERR_TIMEOUT);
            return false;
        }
        if (ld_volatile(&a.ctrl->err)) return false;
    }
    return true;
}

// Chunk m of pass `it`: q, its prefix, and (replay) the orders in time order;
// a replay adds its orders to calls and its runs to units.
// rows: this warp's [kCapChunk][NP] shared rows; s_run / s_k: run and product of
// each slot.  Returns whether a cached action changed.
template <int NPL, bool DUAL>
__device__ bool cap_chunk(const KArgs& a, const CapArgs& c, int m, int it, bool replay,
                          unsigned tag, unsigned long long deadline, int* rows, int* s_run,
                          int* s_k, int* fc_cur, int parity, unsigned long long& calls,
                          unsigned long long& units) {
    const int lane = lane_id();
    const int N = a.N, NP = a.NP;
    const int lo = m * c.L;
    const int cnt = min(a.T, lo + c.L) - lo;  // 1..kCapChunk
    // orders lo + lane and lo + 32 + lane
    int o_prod[2], o_reg[2], o_info[2], o_old[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = lane + 32 * h;
        const bool in = q < cnt;
        const int t = lo + q;
        o_prod[h] = in ? c.prod[t] : 0;
        o_reg[h] = in ? c.reg[t] : 0;
        o_info[h] = in ? c.info[t] : 0;
        o_old[h] = in ? (int)c.act[t] : -1;
        if (in && (o_info[h] & kInfoFirst)) {
            s_run[o_info[h] & kInfoSlot] = c.run_t[t];
            s_k[o_info[h] & kInfoSlot] = o_prod[h];
        }
    }
    __syncwarp();
    const int nslots = __popc(__ballot_sync(kFull, o_info[0] & kInfoFirst)) +
                       __popc(__ballot_sync(kFull, o_info[1] & kInfoFirst));
    // ---- start rows of the chunk's runs and the chunk's q.  The runs'
    // histograms of cached actions are rebuilt in the rows from the chunk's own
    // orders (no histogram loads), then each row is overwritten by its start state.
    const bool have_cache = it > 1 || a.first_dirty;
    int qsum[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) qsum[i] = 0;
    if (have_cache) {
        for (int s = 0; s < nslots; ++s)
#pragma unroll
            for (int i = 0; i < NPL; ++i) rows[s * NP + lane + 32 * i] = 0;
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (o_old[h] >= 0) atomicAdd(&rows[(o_info[h] & kInfoSlot) * NP + o_old[h]], 1);
        __syncwarp();
    }
#pragma unroll 8
    for (int s = 0; s < nslots; ++s) {
        const int r = s_run[s], k = s_k[s];
        // segments hold one run each: the run's chain is its product's segment range
        const bool chained = have_cache && __ldg(&a.meta[r].ce) - __ldg(&a.meta[r].cf) > 1;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            const int x0v = n < N ? __ldg(a.x0 + (size_t)k * N + n) : 0;
            const int d = chained ? a.carry[(size_t)r * NP + n] : 0;  // the whole chain prefix
            const int xs = max(0, x0v - d);
            if (have_cache) qsum[i] += min(rows[s * NP + n], xs);
            rows[s * NP + n] = xs;
        }
    }
    // ---- prefix of q: publish the total, look back, publish the inclusive prefix
    int pre[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) pre[i] = 0;
    if (have_cache) {
#pragma unroll
        for (int i = 0; i < NPL; ++i)
            c.qagg[(size_t)m * NP + lane + 32 * i] = tagged(tag, qsum[i]);
        if (!lookback_q<NPL>(c, a, m, tag, pre, deadline)) return false;
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i)
        c.qinc[(size_t)m * NP + lane + 32 * i] = tagged(tag, pre[i] + qsum[i]);
    if (!replay) return false;
    // ---- replay in time order from (rows, c)
    int cv[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        cv[i] = n < N ? max(0, __ldg(c.cap + n) - pre[i]) : 0;
    }
    // Start decision of every order: arg min of its key over the nodes feasible
    // at the chunk start.  Feasible sets only shrink along the chunk, so while
    // that node stays feasible it is also the arg min over the current set; the
    // walk below decides afresh only when it ran out inside the chunk.  Lane q
    // (q + 32) ends holding the start decision of order q (q + 32).
    int a0[2] = {-1, -1};
    for (int qb = 0; qb < cnt; qb += kAheadCap) {
        int ck[kAheadCap][NPL], sl[kAheadCap];
#pragma unroll
        for (int u = 0; u < kAheadCap; ++u) {
            const int q = min(qb + u, cnt - 1);
            const bool hh = q >= 32;
            const int k = __shfl_sync(kFull, hh ? o_prod[1] : o_prod[0], q & 31);
            const int r = __shfl_sync(kFull, hh ? o_reg[1] : o_reg[0], q & 31);
            sl[u] = __shfl_sync(kFull, hh ? o_info[1] : o_info[0], q & 31) & kInfoSlot;
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int n = lane + 32 * i;
                const int cst = n < N ? __ldg(a.cost + (size_t)r * N + n) : 0;
                const int l = (DUAL && n < N) ? __ldg(a.lam + (size_t)k * N + n) : 0;
                ck[u][i] = (cst - l) * 128 + n;
            }
        }
#pragma unroll
        for (int u = 0; u < kAheadCap; ++u) {
            const int q = qb + u;
            int key = INT_MAX;
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int n = lane + 32 * i;
                if (n < N && rows[sl[u] * NP + n] > 0 && cv[i] > 0) key = min(key, ck[u][i]);
            }
            key = __reduce_min_sync(kFull, key);
            const int act = key == INT_MAX ? -1 : (key & 127);
            if (q < cnt && lane == (q & 31)) {
                if (q >= 32) a0[1] = act;
                else a0[0] = act;
            }
        }
    }
    int my_new[2] = {o_old[0], o_old[1]};
    for (int q = 0; q < cnt; ++q) {
        const bool hh = q >= 32;
        const int src = q & 31;
        const int s = __shfl_sync(kFull, hh ? o_info[1] : o_info[0], src) & kInfoSlot;
        int act = __shfl_sync(kFull, hh ? a0[1] : a0[0], src);
        if (act >= 0) {
            bool still = false;  // only the lane owning node act can set it
#pragma unroll
            for (int i = 0; i < NPL; ++i)
                if (act == lane + 32 * i) still = rows[s * NP + act] > 0 && cv[i] > 0;
            if (!__any_sync(kFull, still)) {  // ran out inside the chunk: decide afresh
                const int k = __shfl_sync(kFull, hh ? o_prod[1] : o_prod[0], src);
                const int r = __shfl_sync(kFull, hh ? o_reg[1] : o_reg[0], src);
                int key = INT_MAX;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int n = lane + 32 * i;
                    if (n < N && rows[s * NP + n] > 0 && cv[i] > 0) {
                        const int l = DUAL ? __ldg(a.lam + (size_t)k * N + n) : 0;
                        key = min(key, (__ldg(a.cost + (size_t)r * N + n) - l) * 128 + n);
                    }
                }
                key = __reduce_min_sync(kFull, key);
                act = key == INT_MAX ? -1 : (key & 127);
            }
        }
#pragma unroll
        for (int i = 0; i < NPL; ++i)
            if (act == lane + 32 * i) {
                rows[s * NP + act] -= 1;
                cv[i] -= 1;
            }
        if (lane == src) {
            if (hh) my_new[1] = act;
            else my_new[0] = act;
        }
    }
    if (lane == 0) {
        calls += (unsigned long long)cnt;
        units += (unsigned long long)nslots;  // runs (segments of one run) replayed
    }
    // ---- cache, first changes (per product in sorted positions, and in time)
    bool chg = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = lane + 32 * h;
        const bool in = q < cnt;
        const bool ch = in && my_new[h] != o_old[h];
        if (in) c.act[lo + q] = (int8_t)my_new[h];
        if (ch) {
            const int j = c.inv[lo + q];
            if (j < ld_volatile(&fc_cur[o_prod[h]])) atomicMin(&fc_cur[o_prod[h]], j);
        }
        const unsigned b = __ballot_sync(kFull, ch);
        if (b) {
            chg = true;
            if (lane == 0) atomicMin(&a.ctrl->cap_fct[parity], lo + 32 * h + __ffs(b) - 1);
        }
    }
    // ---- final stock of products whose last run is in this chunk
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        unsigned b = __ballot_sync(kFull, (o_info[h] & kInfoLastProd) != 0);
        while (b) {
            const int src = __ffs(b) - 1;
            b &= b - 1;
            const int s = __shfl_sync(kFull, o_info[h], src) & kInfoSlot;
            const int k = __shfl_sync(kFull, o_prod[h], src);
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int n = lane + 32 * i;
                if (n < N) a.xfin[(size_t)k * N + n] = rows[s * NP + n];
            }
        }
    }
    // ---- histograms of the runs' new actions (the next pass's agg)
    __syncwarp();
    for (int s = 0; s < nslots; ++s)
#pragma unroll
        for (int i = 0; i < NPL; ++i) rows[s * NP + lane + 32 * i] = 0;
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = lane + 32 * h;
        if (q < cnt && my_new[h] >= 0) atomicAdd(&rows[(o_info[h] & kInfoSlot) * NP + my_new[h]], 1);
    }
    __syncwarp();
    for (int s = 0; s < nslots; ++s) {
        const int r = s_run[s];
#pragma unroll
        for (int i = 0; i < NPL; ++i) a.agg[(size_t)r * NP + lane + 32 * i] = rows[s * NP + lane + 32 * i];
    }
    __syncwarp();
    return chg;
}

// ---------------------------------------------------------------- the passes
template <int NPL, bool DUAL>
__global__ void __launch_bounds__(kCapWarps * 32) k_picard_cap(KArgs a, CapArgs c) {
    extern __shared__ int s_rows[];  // [kCapWarps][kCapChunk][NP]
    __shared__ SegMeta s_meta[kCapWarps][32];
    __shared__ int s_fcp[kCapWarps][32];
    __shared__ int s_run[kCapWarps][kCapChunk];
    __shared__ int s_k[kCapWarps][kCapChunk];
    __shared__ int s_changed;
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    int* rows = s_rows + (size_t)wib * kCapChunk * a.NP;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    const unsigned tag_base = ld_volatile(&a.ctrl->tag_base);
    if (threadIdx.x == 0) s_changed = 0;
    __syncthreads();
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
        const int f_prev = it > 1 ? ld_volatile(&a.ctrl->cap_fct[parity ^ 1]) : -1;
        const unsigned tag = tag_base + (unsigned)it;
        // ---- phase S
        for (int k = gtid; k < a.K; k += gthreads) fc_cur[k] = INT_MAX;
        if (gtid == 0) {
            a.ctrl->changed[parity] = 0;
            a.ctrl->cap_fct[parity] = INT_MAX;
        }
        if (it > 1 || a.first_dirty)
            chain_prefixes<NPL, kPrefixRows<NPL>, false>(a, it, fc_prev, tag, deadline, s_meta[wib],
                                                  s_fcp[wib]);
        if (!grid_sync(a.ctrl, deadline)) { ok = false; break; }
        if (tr && gtid == 0) tr[0] = (long long)(globaltimer_ns() - t_start);
        // ---- phase C
        bool chg = false;
        unsigned long long ucalls = 0;  // largest chunk of this warp (policy calls, lane 0)
        for (int m = gwarp; m < c.M; m += nwarps) {
            const int lo = m * c.L;
            const int hi = min(a.T, lo + c.L);
            if (hi <= f_prev) {  // cache and prefix unchanged: republish the prefix
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const size_t o = (size_t)m * a.NP + lane + 32 * i;
                    c.qinc[o] = tagged(tag, (int)(unsigned)c.qinc[o]);
                }
                continue;
            }
            const bool rep = lo > f_prev;
            const unsigned long long cu0 = calls;
            chg |= cap_chunk<NPL, DUAL>(a, c, m, it, rep, tag, deadline, rows, s_run[wib], s_k[wib],
                                        fc_cur, parity, calls, replays);
            if (calls - cu0 > ucalls) ucalls = calls - cu0;
        }
        if (tr && lane == 0 && replays != replays0) {
            atomicAdd((unsigned long long*)&tr[2], calls - calls0);
            atomicAdd((unsigned long long*)&tr[3], replays - replays0);
            atomicMax((unsigned long long*)&tr[4], ucalls);
            atomicMax((unsigned long long*)&tr[5], (unsigned long long)c.L);
        }
        if (chg && lane == 0) s_changed = 1;
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

// ---------------------------------------------------------------- sequential
// The sequential definition with capacity on one warp (lane l owns nodes
// l + 32 i): the speedup denominator.  xw starts as a copy of x0.
template <int NPL, bool DUAL>
__global__ void __launch_bounds__(32) k_seq_cap(int T, int N, const int32_t* __restrict__ prod,
                                                const int32_t* __restrict__ reg,
                                                const int32_t* __restrict__ cost,
                                                const int32_t* __restrict__ lam,
                                                const int32_t* __restrict__ cap, int32_t* xw,
                                                int8_t* __restrict__ act_t, Ctrl* ctrl) {
    const int lane = lane_id();
    int cv[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) cv[i] = lane + 32 * i < N ? cap[lane + 32 * i] : 0;
    long long cost_acc = 0, lost = 0;
    int k = T > 0 ? __ldg(prod) : 0, r = T > 0 ? __ldg(reg) : 0;
    for (int t = 0; t < T; ++t) {
        const int kn = t + 1 < T ? __ldg(prod + t + 1) : 0;
        const int rn = t + 1 < T ? __ldg(reg + t + 1) : 0;
        int key = INT_MAX, ccv[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            ccv[i] = 0;
            if (n < N) {
                const int xv = xw[(size_t)k * N + n];
                ccv[i] = __ldg(cost + (size_t)r * N + n);
                const int l = DUAL ? __ldg(lam + (size_t)k * N + n) : 0;
                if (xv > 0 && cv[i] > 0) key = min(key, (ccv[i] - l) * 128 + n);
            }
        }
        key = __reduce_min_sync(kFull, key);
        const int act = key == INT_MAX ? -1 : (key & 127);
#pragma unroll
        for (int i = 0; i < NPL; ++i)
            if (act == lane + 32 * i) {
                xw[(size_t)k * N + act] -= 1;
                cv[i] -= 1;
                cost_acc += ccv[i];
            }
        if (lane == 0) {
            act_t[t] = (int8_t)act;
            lost += act < 0;
        }
        k = kn;
        r = rn;
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

inline int nblk(long long n, int per) { return (int)((n + per - 1) / per); }

cudaError_t cap_tables(Instance* I, int M, cudaStream_t st) {
    if (I->cap_tables_m == M) return cudaSuccess;
    const int T = I->T;
    cudaError_t e;
    if (!I->cap_run_t) {
        if ((e = cudaMalloc((void**)&I->cap_run_t, sizeof(int32_t) * (size_t)T))) return e;
        if ((e = cudaMalloc((void**)&I->cap_info, sizeof(int32_t) * (size_t)T))) return e;
        if ((e = cudaMalloc((void**)&I->cap_inv, sizeof(int32_t) * (size_t)T))) return e;
    }
    const int L = (int)(((long long)T + M - 1) / M);
    k_cap_order<<<nblk(T, 256), 256, 0, st>>>(I->perm, I->run_of, I->run_start, T, I->cap_run_t,
                                              I->cap_inv, I->tmp_a);
    if ((e = scan_exclusive(I->tmp_a, I->tmp_b, T, nullptr, I->scan_blk, st, &I->ctrl->err))) return e;
    k_cap_info<<<nblk(T, 256), 256, 0, st>>>(I->cap_run_t, I->cap_inv, I->tmp_b, I->run_start,
                                             I->perm, I->prod, I->pstart, T, L, I->cap_info);
    I->launches += 3;
    if ((e = cudaGetLastError())) return e;
    I->cap_tables_m = M;
    return cudaSuccess;
}

template <int NPL, bool DUAL>
cudaError_t launch_cap(Instance* I, const KArgs& a, const CapArgs& c, cudaStream_t st) {
    auto kern = k_picard_cap<NPL, DUAL>;
    const int threads = kCapWarps * 32;
    const size_t smem = (size_t)kCapWarps * kCapChunk * I->NP * sizeof(int);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem))) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int grid = I->num_sms * occ;
    I->coop_blocks = grid;
    I->cta_threads = threads;
    I->ctas_per_sm = occ;
    KArgs aa = a;
    CapArgs cc = c;
    void* params[] = {&aa, &cc};
    I->launches += 1;
    return cudaLaunchCooperativeKernel((const void*)kern, grid, threads, params, smem, st);
}

template <int NPL, bool DUAL>
cudaError_t launch_seq_cap(Instance* I, cudaStream_t st) {
    I->launches += 1;
    k_seq_cap<NPL, DUAL><<<1, 32, 0, st>>>(I->T, I->N, I->prod, I->reg, I->cost, I->lam, I->cap,
                                           I->xwork, I->act_t, I->ctrl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t picard_cap(Instance* I, const pic_policy* pol, int M, int max_iters, int flags,
                       const int8_t* alpha_init, unsigned long long timeout_ns, bool trace,
                       cudaStream_t st) {
    const int T = I->T;
    cudaError_t e;
    if ((e = cap_tables(I, M, st))) return e;
    const size_t words = (size_t)M * I->NP;
    if (!I->cap_qagg || I->cap_qrows < M) {
        if (I->cap_qagg) {
            cudaFree(I->cap_qagg);
            cudaFree(I->cap_qinc);
            I->cap_qagg = I->cap_qinc = nullptr;
        }
        if ((e = cudaMalloc((void**)&I->cap_qagg, sizeof(unsigned long long) * words))) return e;
        if ((e = cudaMalloc((void**)&I->cap_qinc, sizeof(unsigned long long) * words))) return e;
        I->cap_qrows = M;
    }
    // the q words carry this call's tags (unique per instance until the tag space
    // is renewed); clearing them keeps words of earlier calls from matching
    if ((e = cudaMemsetAsync(I->cap_qagg, 0, sizeof(unsigned long long) * words, st))) return e;
    if ((e = cudaMemsetAsync(I->cap_qinc, 0, sizeof(unsigned long long) * words, st))) return e;
    // the cache in time order
    if (alpha_init) {
        k_cap_cache<<<nblk(T, 256), 256, 0, st>>>(alpha_init, T, I->N, I->act_t);
        I->launches += 1;
        if ((e = cudaGetLastError())) return e;
    } else if ((e = cudaMemsetAsync(I->act_t, 0xFF, (size_t)T, st))) {
        return e;
    }
    KArgs a;
    a.T = T; a.N = I->N; a.K = I->K; a.NP = I->NP; a.R = I->R;
    a.reg_s = I->reg_s; a.run_start = I->run_start; a.seg_run = I->seg_run;
    a.seg_prod = I->seg_prod; a.seg_cf = I->seg_cf; a.seg_ce = I->seg_ce;
    a.x0 = I->x0; a.cost = I->cost; a.lam = I->lam;
    a.alpha_s = I->alpha_s; a.agg = I->agg; a.carry = I->carry; a.sbexc = I->sbexc;
    a.sbagg = I->sbagg; a.sbincl = I->sbincl; a.meta = I->seg_meta; a.lpt = I->seg_lpt;
    a.fc = I->fc; a.xfin = I->xfin;
    a.ctrl = I->ctrl; a.max_iters = max_iters; a.flags = flags;
    a.first_dirty = alpha_init != nullptr; a.timeout_ns = timeout_ns;
    a.trace = trace ? I->trace : nullptr;
    a.run_chunk = nullptr;  // no max_steps window
    a.perm = nullptr;
    a.win_steps = 0;
    a.M = a.L = 0;
    CapArgs c;
    c.M = M;
    c.L = (int)(((long long)T + M - 1) / M);
    c.prod = I->prod; c.reg = I->reg; c.info = I->cap_info; c.run_t = I->cap_run_t;
    c.inv = I->cap_inv; c.cap = I->cap; c.act = I->act_t; c.qagg = I->cap_qagg; c.qinc = I->cap_qinc;
    const bool dual = pol->kind == PIC_POLICY_DUAL;
    const int npl = (I->N + 31) / 32;
    if (npl == 1) return dual ? launch_cap<1, true>(I, a, c, st) : launch_cap<1, false>(I, a, c, st);
    if (npl == 2) return dual ? launch_cap<2, true>(I, a, c, st) : launch_cap<2, false>(I, a, c, st);
    return dual ? launch_cap<4, true>(I, a, c, st) : launch_cap<4, false>(I, a, c, st);
}

cudaError_t sequential_cap(Instance* I, int kind, cudaStream_t st) {
    const bool dual = kind == PIC_POLICY_DUAL;
    const int npl = (I->N + 31) / 32;
    if (npl == 1) return dual ? launch_seq_cap<1, true>(I, st) : launch_seq_cap<1, false>(I, st);
    if (npl == 2) return dual ? launch_seq_cap<2, true>(I, st) : launch_seq_cap<2, false>(I, st);
    return dual ? launch_seq_cap<4, true>(I, st) : launch_seq_cap<4, false>(I, st);
}

}  // namespace pic
