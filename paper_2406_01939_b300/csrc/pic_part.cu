// Algorithm 1 for partitions of the orders other than contiguous time chunks,
// greedy and bid-price policies:
//   picard_products  the product partition (Sec. 3: all orders of a product go
//                    to one process), with or without node capacity;
//   picard_assigned  any caller-given assignment proc[t] (e.g. the uniform
//                    random partition of Sec. 4.1), without capacity.
// Each pass, Algorithm 1 has every process replay the horizon, taking its own
// orders' actions from the policy and every other order's action from the
// cache.  Here a process visits only its own orders: what the foreign cached
// actions do to its state is read from per-pass lists of the cache.
//
// Product partition.  Processor m owns the products k with k mod P = m.
// Only the processor's own products' stock matters to its decisions (foreign
// actions never touch it), and node capacity follows from counts: the capacity
// of node j before order t, in processor m's view, is
//   max(0, c_j - q_j),  q_j = successes of cached actions to j before t
//                            - those of m's own cached actions + m's fresh ones,
// where a cached action "succeeds" when its product still has stock at j under
// that product's cached actions alone (once a node's capacity is spent, whether
// later actions to it find stock no longer matters).  So with S_j(n) the time of
// the n-th cached success at node j (time order), node j has capacity at t iff
//   S_j(c_j + own_cached_j - fresh_j) >= t   (or fewer successes than that).
// A pass therefore needs, from the cache: every cached action's success (its
// rank among the cached actions of its product and node, against x0), the
// successes listed per node in time order, then one warp per processor walking
// its own orders with a threshold S_j(.) per node, refreshed only when its own
// cached or fresh successes move it.
#include <climits>

#include "pic_device.cuh"

namespace pic {

namespace {

constexpr int kPartWarps = 4;   // warps (processors) per CTA of the walk
constexpr int kPartBatch = 32;  // own orders staged per warp at a time

// key of each cached action: product * N + node, or K N for a^phi (and for a
// value outside [0, N), which the call reports as an invalid initial cache), so
// that every key lies in [0, K N]
__global__ void k_part_keys(int T, int N, int KN, const int32_t* __restrict__ prod,
                            const int8_t* __restrict__ act, int32_t* __restrict__ key) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = act[t];
        key[t] = a >= 0 && a < N ? prod[t] * N + a : KN;
    }
}

__device__ __forceinline__ int lower_bound_i32(const int32_t* __restrict__ v, int n, int x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Success of each cached action (stable sort by key keeps time order inside a
// key): rank within (product, node) below x0[product][node].  succ[t] = node, or
// N when the action is a^phi or finds no stock.
__global__ void k_part_succ(int T, int N, int KN, const int32_t* __restrict__ key_s,
                            const int32_t* __restrict__ t_s, const int32_t* __restrict__ x0,
                            int32_t* __restrict__ succ) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < T;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = key_s[i];
        int node = N;
        if (k < KN) {
            const int rank = (int)i - lower_bound_i32(key_s, T, k);
            if (rank < x0[k]) node = k % N;  // x0 is [K][N]: x0[k] = x0[product][node]
        }
        succ[t_s[i]] = node;
    }
}

// first position of each value 0..nv in a sorted array (offsets, nv + 1 entries)
__global__ void k_part_offsets(const int32_t* __restrict__ sorted, int n, int nv,
                               int32_t* __restrict__ off) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v <= nv) off[v] = lower_bound_i32(sorted, n, v);
}

// processor key of each order
__global__ void k_part_pkey(int T, int P, const int32_t* __restrict__ prod, int32_t* __restrict__ pk) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
         t += (long long)gridDim.x * blockDim.x)
        pk[t] = prod[t] % P;
}

__global__ void k_part_check_init(int T, int N, const int8_t* __restrict__ a, Ctrl* ctrl) {
    int b = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
         t += (long long)gridDim.x * blockDim.x)
        if (a[t] < -1 || a[t] >= N) b = 1;
    if (b) atomicOr(&ctrl->pad0, 64);
}

// 4-byte asynchronous global -> shared copy (completed by cp.async.wait_group)
__device__ __forceinline__ void part_copy4(int32_t* dst, const int32_t* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// S_j(n), the time of the n-th cached success at node j (list at S + base, cnt
// entries): -1 when n <= 0 (no capacity left), INT_MAX past the list (capacity
// left for the whole horizon).
__device__ __forceinline__ int part_sval(const int32_t* __restrict__ S, int base, int cnt, int n) {
    return n <= 0 ? -1 : (n > cnt ? INT_MAX : __ldg(S + base + n - 1));
}

// One warp per processor m (grid-stride): its orders in time order.  Lane l
// holds warehouses j = l + 32 q.  The decision is the arg min of cost (- lam)
// over warehouses with stock and capacity, ties to the lowest index, a^phi if
// none.  Per lane and warehouse: the stock of the current product (each
// product belongs to one processor, so the row is this warp's alone), and for
// capacity n = c_j + own cached successes - fresh actions so far with
// th = S_j(n) (capacity at t iff th >= t) and its neighbours S_j(n -/+ 1),
// prefetched so that a one-step change of n needs no load.  Orders are taken
// kPartBatch at a time: their indices are loaded one batch ahead and their
// cost rows staged in shared memory, so the per-order chain is shuffles,
// shared loads and one warp reduction.
template <int NPL, bool DUAL, bool CAP>
__global__ void __launch_bounds__(kPartWarps * 32) k_part_walk(
    int P, int N, const int32_t* __restrict__ own_t, const int32_t* __restrict__ own_off,
    const int32_t* __restrict__ prod, const int32_t* __restrict__ reg,
    const int32_t* __restrict__ cost, const int32_t* __restrict__ lam,
    const int32_t* __restrict__ cap, const int32_t* __restrict__ succ,
    const int32_t* __restrict__ S, const int32_t* __restrict__ soff, int8_t* __restrict__ act,
    int32_t* __restrict__ xv, Ctrl* ctrl, int32_t* __restrict__ changed) {
    extern __shared__ int32_t part_smem[];
    constexpr int kRow = NPL * 32;
    const int lane = threadIdx.x & 31;
    int32_t* cst = part_smem + (threadIdx.x >> 5) * kPartBatch * kRow;  // [kPartBatch][kRow]
    const int nwarps = gridDim.x * kPartWarps;
    int my_changed = 0;
    unsigned long long calls = 0;
    int sb[NPL], sc[NPL], cj[NPL];
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
        const int j = lane + 32 * q;
        sb[q] = 0, sc[q] = 0, cj[q] = 0;
        if (CAP && j < N) {
            sb[q] = soff[j];
            sc[q] = soff[j + 1] - sb[q];
            cj[q] = cap[j];
        }
    }
    for (int m = blockIdx.x * kPartWarps + (threadIdx.x >> 5); m < P; m += nwarps) {
        const int e0 = own_off[m], e1 = own_off[m + 1];
        if (e0 >= e1) continue;
        int n[NPL], th[NPL], tm[NPL], tp[NPL], xr[NPL], lr[NPL];
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
            n[q] = cj[q];
            th[q] = CAP ? part_sval(S, sb[q], sc[q], n[q]) : INT_MAX;
            tm[q] = CAP ? part_sval(S, sb[q], sc[q], n[q] - 1) : INT_MAX;
            tp[q] = CAP ? part_sval(S, sb[q], sc[q], n[q] + 1) : INT_MAX;
            xr[q] = 0, lr[q] = 0;
        }
        int kc = -1;
        // batch b's indices (bt .. bo) and batch b + 1's order times (nt)
        int bt = 0, bk = 0, br = 0, bs = N, bo = 0, nt = 0;
        if (lane < e1 - e0) {
            bt = own_t[e0 + lane];
            bk = prod[bt], br = reg[bt], bo = act[bt];
            if (CAP) bs = succ[bt];
        }
        if (e0 + kPartBatch + lane < e1) nt = own_t[e0 + kPartBatch + lane];
        for (int eb = e0; eb < e1; eb += kPartBatch) {
            const int nb = min(kPartBatch, e1 - eb);
            // next batch's indices (consumed after this batch's orders)
            int nk = 0, nr = 0, ns = N, no = 0, nnt = 0;
            if (eb + kPartBatch + lane < e1) {
                nk = prod[nt], nr = reg[nt], no = act[nt];
                if (CAP) ns = succ[nt];
            }
            if (eb + 2 * kPartBatch + lane < e1) nnt = own_t[eb + 2 * kPartBatch + lane];
            __syncwarp();  // the previous batch's reads of cst are done
            // all of the batch's cost rows in flight at once (asynchronous copies), one wait
#pragma unroll 8
            for (int i = 0; i < kPartBatch; ++i) {
                const int r = __shfl_sync(kFull, br, i);
                if (i < nb) {
#pragma unroll
                    for (int q = 0; q < NPL; ++q) {
                        const int j = lane + 32 * q;
                        if (j < N) part_copy4(cst + i * kRow + j, cost + (size_t)r * N + j);
                    }
                }
            }
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;\n" ::: "memory");
            __syncwarp();
            int bnew = -1;
            // order i's indices and cost row are read during order i - 1 (off the
            // loop-carried chain: stock and capacity -> decision -> update)
            int t_n = __shfl_sync(kFull, bt, 0), k_n = __shfl_sync(kFull, bk, 0);
            int sn_n = CAP ? __shfl_sync(kFull, bs, 0) : N;
            int cv_n[NPL];
#pragma unroll
            for (int q = 0; q < NPL; ++q) cv_n[q] = cst[lane + 32 * q];
            for (int i = 0; i < nb; ++i) {
                const int t = t_n, k = k_n, sn = sn_n;
                int cv[NPL];
#pragma unroll
                for (int q = 0; q < NPL; ++q) cv[q] = cv_n[q];
                const int i1 = i + 1 < kPartBatch ? i + 1 : i;  // row i1 >= nb: stale, unused
                t_n = __shfl_sync(kFull, bt, i1), k_n = __shfl_sync(kFull, bk, i1);
                if (CAP) sn_n = __shfl_sync(kFull, bs, i1);
#pragma unroll
                for (int q = 0; q < NPL; ++q) cv_n[q] = cst[i1 * kRow + lane + 32 * q];
                if (k != kc) {  // warp-uniform: switch the register row to product k
#pragma unroll
                    for (int q = 0; q < NPL; ++q) {
                        const int j = lane + 32 * q;
                        if (j < N) {
                            if (kc >= 0) xv[(size_t)kc * N + j] = xr[q];
                            xr[q] = xv[(size_t)k * N + j];
                            if (DUAL) lr[q] = __ldg(lam + (size_t)k * N + j);
                        }
                    }
                    kc = k;
                }
                int best = INT_MAX;
#pragma unroll
                for (int q = 0; q < NPL; ++q) {
                    const int j = lane + 32 * q;
                    if (j < N && xr[q] > 0 && th[q] >= t) {
                        int v = cv[q];
                        if (DUAL) v -= lr[q];
                        best = min(best, v * 128 + j);
                    }
                }
                best = __reduce_min_sync(kFull, best);
                const int a = best == INT_MAX ? -1 : (best & 127);
#pragma unroll
                for (int q = 0; q < NPL; ++q) {
                    const int j = lane + 32 * q;
                    if (j == a) xr[q] -= 1;  // the fresh action takes one unit of stock
                    if (CAP && j < N) {
                        // fresh action: one unit of capacity; this order's cached
                        // success (if any) no longer counts
                        const int dd = (j == sn ? 1 : 0) - (j == a ? 1 : 0);
                        if (dd > 0) {
                            n[q] += 1;
                            tm[q] = th[q], th[q] = tp[q];
                            tp[q] = part_sval(S, sb[q], sc[q], n[q] + 1);
                        } else if (dd < 0) {
                            n[q] -= 1;
                            tp[q] = th[q], th[q] = tm[q];
                            tm[q] = part_sval(S, sb[q], sc[q], n[q] - 1);
                        }
                    }
                }
                if (lane == i) bnew = a;
            }
            if (lane < nb) {
                act[bt] = (int8_t)bnew;
                my_changed |= bnew != bo;
            }
            calls += nb;
            bt = nt, bk = nk, br = nr, bs = ns, bo = no, nt = nnt;
        }
        if (kc >= 0) {
#pragma unroll
            for (int q = 0; q < NPL; ++q) {
                const int j = lane + 32 * q;
                if (j < N) xv[(size_t)kc * N + j] = xr[q];
            }
        }
    }
    my_changed = __any_sync(kFull, my_changed);
    if (lane == 0) {
        if (my_changed) atomicExch(changed, 1);
        if (calls) atomicAdd(&ctrl->policy_calls, calls);
    }
}

// ---------------------------------------------------------------- any assignment
// Algorithm 1 for an arbitrary assignment proc[t] of orders to processes, no
// capacity.  In process m's view the stock of (k, j) moves only by attempts on
// it: the cached actions of other processes' orders (applied while stock
// remains) and m's fresh actions (always feasible), so before order t it is
//   max(0, x0[k][j] - (C(t) - O(t) + F(t))),
// C the cached actions naming (k, j) before t (all orders), O those at m's own
// orders, F m's fresh actions naming j for product k before t.  m's orders of
// product k therefore form an independent chain (unit (k, m)), and stock > 0 at
// t iff the X-th cached action naming (k, j) comes at or after t, X = x0 - F + O.

// unit key m * K + k of each order; a process outside [0, P) sets Ctrl::pad0 bit 128
__global__ void k_assign_ukey(int T, int K, int P, const int32_t* __restrict__ proc,
                              const int32_t* __restrict__ prod, int32_t* __restrict__ ukey,
                              Ctrl* ctrl) {
    int bad = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
         t += (long long)gridDim.x * blockDim.x) {
        int m = proc[t];
        if (m < 0 || m >= P) {
            bad = 1;
            m = 0;
        }
        ukey[t] = m * K + prod[t];
    }
    if (bad) atomicOr(&ctrl->pad0, 128);
}

__global__ void k_assign_uflags(int n, const int32_t* __restrict__ uks, int32_t* __restrict__ flag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        flag[i] = i == 0 || uks[i] != uks[i - 1];
}

// ustart[u] = first sorted position of unit u; ustart[U] = n
__global__ void k_assign_ustart(int n, const int32_t* __restrict__ flag,
                                const int32_t* __restrict__ upos, int32_t* __restrict__ ustart) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (flag[i]) ustart[upos[i]] = (int)i;
        if (i == n - 1) ustart[upos[i] + flag[i]] = n;
    }
}

// Per (k, j) pair v: its list of cached actions (base, count) and the thresholds
// at X = x0 and x0 -/+ 1, so that a unit's start needs one coalesced row per
// field instead of offsets followed by list reads.
__global__ void k_assign_pairs(int KN, const int32_t* __restrict__ x0,
                               const int32_t* __restrict__ off, const int32_t* __restrict__ L,
                               int4* __restrict__ pr, int32_t* __restrict__ ptp,
                               int32_t* __restrict__ pth) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < KN;
         v += (long long)gridDim.x * blockDim.x) {
        const int b = off[v], c = off[v + 1] - b, X = x0[v];
        const int th = part_sval(L, b, c, X);
        pr[v] = make_int4(b, c, th, part_sval(L, b, c, X - 1));
        ptp[v] = part_sval(L, b, c, X + 1);
        pth[v] = th;
    }
}

// Per unit u (once per call): its first order, product and region, and whether
// it has more orders; the units with more are listed with their range after the
// first order, their product and first order.
__global__ void k_assign_units(int U, const int32_t* __restrict__ ustart,
                               const int32_t* __restrict__ uord, const int32_t* __restrict__ prod,
                               const int32_t* __restrict__ reg, int32_t* __restrict__ ft,
                               int32_t* __restrict__ fk, int32_t* __restrict__ fr,
                               int32_t* __restrict__ mflag) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < U;
         u += (long long)gridDim.x * blockDim.x) {
        const int e0 = ustart[u], t = uord[e0];
        ft[u] = t, fk[u] = prod[t], fr[u] = reg[t];
        mflag[u] = ustart[u + 1] - e0 > 1;
    }
}

__global__ void k_assign_mlist(int U, const int32_t* __restrict__ ustart,
                               const int32_t* __restrict__ ft, const int32_t* __restrict__ fk,
                               const int32_t* __restrict__ mflag, const int32_t* __restrict__ mpos,
                               int4* __restrict__ mu) {
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < U;
         u += (long long)gridDim.x * blockDim.x)
        if (mflag[u]) mu[mpos[u]] = make_int4(ustart[u] + 1, ustart[u + 1], fk[u], (int)u);
}

// The first order of every unit: its process has taken no own action of the
// product yet, so X = x0 and stock > 0 iff pth >= t.  One warp per 32 units:
// their first orders' indices lane-parallel, then each decision with lanes over
// the nodes (coalesced rows), the rows of four units loaded before their four
// decisions.  The order's cached action is kept in fold[u] for the walk of the
// unit's later orders.
template <int NPL, bool DUAL>
__global__ void __launch_bounds__(256) k_assign_first(
    int U, int N, const int32_t* __restrict__ ft, const int32_t* __restrict__ fk,
    const int32_t* __restrict__ fr, const int32_t* __restrict__ cost,
    const int32_t* __restrict__ lam, const int32_t* __restrict__ pth, int8_t* __restrict__ act,
    int8_t* __restrict__ fold, Ctrl* ctrl, int32_t* __restrict__ changed) {
    constexpr int G = 4;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int my_changed = 0;
    unsigned calls = 0;
    for (long long ub = (long long)gw * 32; ub < U; ub += (long long)nw * 32) {
        const int u = (int)ub + lane;
        int t = 0, k = 0, r = 0, c = -1;  // lanes past U: row 0 read, decision unused
        if (u < U) {
            t = ft[u], k = fk[u], r = fr[u];
            c = act[t];
        }
        const int nu = min(32, U - (int)ub);
        int anew = -1;
        for (int i0 = 0; i0 < nu; i0 += G) {
            int th[G][NPL], cv[G][NPL];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int kk = __shfl_sync(kFull, k, i0 + g), rr = __shfl_sync(kFull, r, i0 + g);
#pragma unroll
                for (int q = 0; q < NPL; ++q) {
                    const int j = lane + 32 * q;
                    th[g][q] = -1, cv[g][q] = 0;
                    if (j < N) {
                        th[g][q] = __ldg(pth + (size_t)kk * N + j);
                        cv[g][q] = __ldg(cost + (size_t)rr * N + j);
                        if (DUAL) cv[g][q] -= __ldg(lam + (size_t)kk * N + j);
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int tt = __shfl_sync(kFull, t, i0 + g);
                int key = INT_MAX;
#pragma unroll
                for (int q = 0; q < NPL; ++q)
                    if (th[g][q] >= tt) key = min(key, cv[g][q] * 128 + lane + 32 * q);
                key = __reduce_min_sync(kFull, key);
                if (lane == i0 + g) anew = key == INT_MAX ? -1 : (key & 127);
            }
        }
        if (u < U) {
            act[t] = (int8_t)anew;
            fold[u] = (int8_t)c;
            my_changed |= anew != c;
        }
        calls += nu;
    }
    my_changed = __any_sync(kFull, my_changed);
    if (lane == 0) {
        if (my_changed) atomicExch(changed, 1);
        if (calls) atomicAdd(&ctrl->policy_calls, (unsigned long long)calls);
    }
}

// final stock of a cache without capacity: max(0, x0 - its actions naming (k, j))
__global__ void k_assign_final(int KN, const int32_t* __restrict__ x0,
                               const int32_t* __restrict__ off, int32_t* __restrict__ xfin) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < KN;
         v += (long long)gridDim.x * blockDim.x)
        xfin[v] = max(0, x0[v] - (off[v + 1] - off[v]));
}

// One warp per unit (k, m) with more than one order, from its second order on
// (the first was decided by k_assign_first): its orders in time order, 32 at a
// time (indices one batch ahead, cost rows staged by asynchronous copies, the
// next order read during the current one).  Lane l holds nodes j = l + 32 q with
// X = x0 - F + O and th = L_kj(X), the time of the X-th cached action naming
// (k, j), and its neighbours L_kj(X -/+ 1), moved when a fresh action (X - 1)
// or the order's own cached action (X + 1) touches j.
template <int NPL, bool DUAL>
__global__ void __launch_bounds__(kPartWarps * 32) k_assign_walk(
    int MU, int N, const int4* __restrict__ mu, const int32_t* __restrict__ ft,
    const int8_t* __restrict__ fold, const int32_t* __restrict__ uord,
    const int32_t* __restrict__ reg,
    const int32_t* __restrict__ cost, const int32_t* __restrict__ lam,
    const int32_t* __restrict__ x0, const int32_t* __restrict__ L,
    const int4* __restrict__ pr, const int32_t* __restrict__ ptp, int8_t* __restrict__ act,
    Ctrl* ctrl, int32_t* __restrict__ changed) {
    extern __shared__ int32_t part_smem[];
    constexpr int kRow = NPL * 32;
    const int lane = threadIdx.x & 31;
    int32_t* cst = part_smem + (threadIdx.x >> 5) * kPartBatch * kRow;  // [kPartBatch][kRow]
    const int nwarps = gridDim.x * kPartWarps;
    int my_changed = 0;
    unsigned long long calls = 0;
    int i = blockIdx.x * kPartWarps + (threadIdx.x >> 5);
    int4 mn = make_int4(0, 0, 0, 0);  // the next unit {e0, e1, k, u}, read one unit ahead
    if (i < MU) mn = mu[i];
    for (; i < MU; i += nwarps) {
        const int e0 = mn.x, e1 = mn.y, k = mn.z, u = mn.w;
        if (i + nwarps < MU) mn = mu[i + nwarps];
        // the unit's first order: its fresh action (already in the cache) and the
        // cached action it replaced
        const int a1 = act[ft[u]], c1 = fold[u];
        int bt = 0, br = 0, bo = -1, nt = 0;
        if (lane < e1 - e0) {
            bt = uord[e0 + lane];
            br = reg[bt], bo = act[bt];
        }
        if (e0 + kPartBatch + lane < e1) nt = uord[e0 + kPartBatch + lane];
        int sb[NPL], sc[NPL], X[NPL], th[NPL], tm[NPL], tp[NPL], lr[NPL];
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
            const int j = lane + 32 * q;
            sb[q] = 0, sc[q] = 0, X[q] = 0, lr[q] = 0;
            th[q] = -1, tm[q] = -1, tp[q] = -1;
            if (j < N) {
                const size_t v = (size_t)k * N + j;
                const int4 w = pr[v];
                sb[q] = w.x, sc[q] = w.y, th[q] = w.z, tm[q] = w.w;
                tp[q] = ptp[v];
                X[q] = x0[v];
                if (DUAL) lr[q] = __ldg(lam + v);
                // after the first order: O + [j == c1], F + [j == a1]
                const int dd = (j == c1 ? 1 : 0) - (j == a1 ? 1 : 0);
                if (dd > 0) {
                    X[q] += 1;
                    tm[q] = th[q], th[q] = tp[q];
                    tp[q] = part_sval(L, sb[q], sc[q], X[q] + 1);
                } else if (dd < 0) {
                    X[q] -= 1;
                    tp[q] = th[q], th[q] = tm[q];
                    tm[q] = part_sval(L, sb[q], sc[q], X[q] - 1);
                }
            }
        }
        for (int eb = e0; eb < e1; eb += kPartBatch) {
            const int nb = min(kPartBatch, e1 - eb);
            int nr = 0, no = -1, nnt = 0;
            if (eb + kPartBatch + lane < e1) nr = reg[nt], no = act[nt];
            if (eb + 2 * kPartBatch + lane < e1) nnt = uord[eb + 2 * kPartBatch + lane];
            __syncwarp();  // the previous batch's reads of cst are done
#pragma unroll 8
            for (int i = 0; i < kPartBatch; ++i) {
                const int r = __shfl_sync(kFull, br, i);
                if (i < nb) {
#pragma unroll
                    for (int q = 0; q < NPL; ++q) {
                        const int j = lane + 32 * q;
                        if (j < N) part_copy4(cst + i * kRow + j, cost + (size_t)r * N + j);
                    }
                }
            }
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;\n" ::: "memory");
            __syncwarp();
            int bnew = -1;
            int t_n = __shfl_sync(kFull, bt, 0), c_n = __shfl_sync(kFull, bo, 0);
            int cv_n[NPL];
#pragma unroll
            for (int q = 0; q < NPL; ++q) cv_n[q] = cst[lane + 32 * q];
            for (int i = 0; i < nb; ++i) {
                const int t = t_n, c = c_n;
                int cv[NPL];
#pragma unroll
                for (int q = 0; q < NPL; ++q) cv[q] = cv_n[q];
                const int i1 = i + 1 < kPartBatch ? i + 1 : i;  // row i1 >= nb: stale, unused
                t_n = __shfl_sync(kFull, bt, i1), c_n = __shfl_sync(kFull, bo, i1);
#pragma unroll
                for (int q = 0; q < NPL; ++q) cv_n[q] = cst[i1 * kRow + lane + 32 * q];
                int best = INT_MAX;
#pragma unroll
                for (int q = 0; q < NPL; ++q) {
                    const int j = lane + 32 * q;
                    if (j < N && th[q] >= t) {
                        int v = cv[q];
                        if (DUAL) v -= lr[q];
                        best = min(best, v * 128 + j);
                    }
                }
                best = __reduce_min_sync(kFull, best);
                const int a = best == INT_MAX ? -1 : (best & 127);
#pragma unroll
                for (int q = 0; q < NPL; ++q) {
                    const int j = lane + 32 * q;
                    // fresh action: F + 1; the order's own cached action: O + 1
                    const int dd = (j < N && j == c ? 1 : 0) - (j == a ? 1 : 0);
                    if (dd > 0) {
                        X[q] += 1;
                        tm[q] = th[q], th[q] = tp[q];
                        tp[q] = part_sval(L, sb[q], sc[q], X[q] + 1);
                    } else if (dd < 0) {
                        X[q] -= 1;
                        tp[q] = th[q], th[q] = tm[q];
                        tm[q] = part_sval(L, sb[q], sc[q], X[q] - 1);
                    }
                }
                if (lane == i) bnew = a;
            }
            if (lane < nb) {
                act[bt] = (int8_t)bnew;
                my_changed |= bnew != bo;
            }
            calls += nb;
            bt = nt, br = nr, bo = no, nt = nnt;
        }
    }
    my_changed = __any_sync(kFull, my_changed);
    if (lane == 0) {
        if (my_changed) atomicExch(changed, 1);
        if (calls) atomicAdd(&ctrl->policy_calls, calls);
    }
}

__global__ void k_part_result(Ctrl* ctrl, int iters, int converged) {
    ctrl->iters = iters;
    ctrl->converged = converged;
}

}  // namespace

// Algorithm 1 with the product partition (processor of product k: k mod P) on
// the instance's orders.  The cache (time order, I->act_t) must hold alpha^0;
// returns with the last iterate there, the own products' final stock in
// I->xfin, and iters / converged in I->ctrl.
cudaError_t picard_products(Instance* I, const pic_policy* pol, int P, int iters_cap,
                            cudaStream_t st) {
    const int T = I->T, N = I->N, K = I->K, KN = K * N;
    const bool dual = pol->kind == PIC_POLICY_DUAL, cap = I->has_cap != 0;
    const int NPL = N <= 32 ? 1 : (N <= 64 ? 2 : 4);
    int32_t *key = nullptr, *key_s = nullptr, *t_s = nullptr, *succ = nullptr, *skey = nullptr,
            *S = nullptr, *pk = nullptr, *pks = nullptr, *own_t = nullptr, *soff = nullptr,
            *own_off = nullptr, *flag = nullptr;
    cudaError_t e = cudaSuccess;
    const size_t Tn = T > 0 ? (size_t)T : 1;
    auto A = [&](int32_t** p, size_t n) {
        if (!e) e = cudaMallocAsync(p, n * sizeof(int32_t), st);
    };
    A(&key, Tn); A(&key_s, Tn); A(&t_s, Tn); A(&succ, Tn); A(&skey, Tn); A(&S, Tn); A(&pk, Tn);
    A(&pks, Tn); A(&own_t, Tn); A(&soff, (size_t)N + 2); A(&own_off, (size_t)P + 1); A(&flag, 1);
    const int gb = (int)((Tn + 255) / 256) < 4 * I->num_sms ? (int)((Tn + 255) / 256) : 4 * I->num_sms;
    int iters = 0, converged = 0;
    if (!e && T > 0) {
        // each processor's orders in time order (stable sort by processor)
        k_part_pkey<<<gb, 256, 0, st>>>(T, P, I->prod, pk);
        e = sort_pairs(I, pk, T, P - 1, pks, own_t, I->tmp_a, I->tmp_b, st);
        if (!e) k_part_offsets<<<(P + 256) / 256, 256, 0, st>>>(pks, T, P, own_off);
        I->launches += 2;
    }
    const int blocks = (P + kPartWarps - 1) / kPartWarps;
    const int smem = kPartWarps * kPartBatch * NPL * 32 * (int)sizeof(int32_t);
    for (int pass = 1; !e && T > 0 && pass <= iters_cap; ++pass) {
        if (cap) {
            // which cached actions find stock, listed per node in time order
            k_part_keys<<<gb, 256, 0, st>>>(T, N, KN, I->prod, I->act_t, key);
            e = sort_pairs(I, key, T, KN, key_s, t_s, I->tmp_a, I->tmp_b, st);
            if (e) break;
            k_part_succ<<<gb, 256, 0, st>>>(T, N, KN, key_s, t_s, I->x0, succ);
            e = sort_pairs(I, succ, T, N, skey, S, I->tmp_a, I->tmp_b, st);
            if (e) break;
            k_part_offsets<<<1, 128, 0, st>>>(skey, T, N, soff);
            I->launches += 3;
        }
        if ((e = cudaMemcpyAsync(I->xfin, I->x0, sizeof(int32_t) * (size_t)K * N,
                                 cudaMemcpyDeviceToDevice, st)))
            break;
        if ((e = cudaMemsetAsync(flag, 0, sizeof(int32_t), st))) break;
#define PART_WALK(NP_, D_, C_)                                                              \
    do {                                                                                    \
        e = cudaFuncSetAttribute(k_part_walk<NP_, D_, C_>,                                 \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);       \
        if (!e)                                                                             \
            k_part_walk<NP_, D_, C_><<<blocks, kPartWarps * 32, smem, st>>>(               \
                P, N, own_t, own_off, I->prod, I->reg, I->cost, I->lam, I->cap, succ, S,   \
                soff, I->act_t, I->xfin, I->ctrl, flag);                                   \
    } while (0)
        if (NPL == 1) {
            if (dual) { if (cap) PART_WALK(1, true, true); else PART_WALK(1, true, false); }
            else { if (cap) PART_WALK(1, false, true); else PART_WALK(1, false, false); }
        } else if (NPL == 2) {
            if (dual) { if (cap) PART_WALK(2, true, true); else PART_WALK(2, true, false); }
            else { if (cap) PART_WALK(2, false, true); else PART_WALK(2, false, false); }
        } else {
            if (dual) { if (cap) PART_WALK(4, true, true); else PART_WALK(4, true, false); }
            else { if (cap) PART_WALK(4, false, true); else PART_WALK(4, false, false); }
        }
#undef PART_WALK
        if (e) break;
        I->launches += 1;
        int hf = 0;
        if ((e = cudaGetLastError())) break;
        if ((e = cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaStreamSynchronize(st))) break;
        iters = pass;
        if (!hf) {
            converged = 1;
            break;
        }
    }
    if (T == 0) {
        iters = 1;
        converged = 1;
        if (!e) e = cudaMemcpyAsync(I->xfin, I->x0, sizeof(int32_t) * (size_t)K * N,
                                    cudaMemcpyDeviceToDevice, st);
    }
    if (!e) {
        k_part_result<<<1, 1, 0, st>>>(I->ctrl, iters, converged);
        e = cudaGetLastError();
    }
    int32_t* bufs[] = {key, key_s, t_s, succ, skey, S, pk, pks, own_t, soff, own_off, flag};
    for (int32_t* b : bufs)
        if (b) cudaFreeAsync(b, st);
    return e;
}

// Algorithm 1 for the assignment proc[t] in [0, P) (DEVICE), no capacity, on the
// instance's orders.  Same contract as picard_products; a process outside
// [0, P) raises Ctrl::pad0 bit 128.
cudaError_t picard_assigned(Instance* I, const pic_policy* pol, const int32_t* proc, int P,
                            int iters_cap, cudaStream_t st) {
    const int T = I->T, N = I->N, K = I->K, KN = K * N;
    const bool dual = pol->kind == PIC_POLICY_DUAL;
    const int NPL = N <= 32 ? 1 : (N <= 64 ? 2 : 4);
    int32_t *ukey = nullptr, *uks = nullptr, *uord = nullptr, *flag = nullptr, *upos = nullptr,
            *ustart = nullptr, *key = nullptr, *key_s = nullptr, *t_s = nullptr, *off = nullptr,
            *cflag = nullptr, *total = nullptr;
    cudaError_t e = cudaSuccess;
    const size_t Tn = T > 0 ? (size_t)T : 1;
    auto A = [&](int32_t** p, size_t n) {
        if (!e) e = cudaMallocAsync(p, n * sizeof(int32_t), st);
    };
    A(&ukey, Tn); A(&uks, Tn); A(&uord, Tn); A(&flag, Tn); A(&upos, Tn); A(&ustart, Tn + 1);
    A(&key, Tn); A(&key_s, Tn); A(&t_s, Tn); A(&off, (size_t)KN + 1); A(&cflag, 1); A(&total, 1);
    int4 *pr = nullptr, *mu = nullptr;
    int32_t *ptp = nullptr, *pth = nullptr, *ft = nullptr, *fk = nullptr, *fr = nullptr,
            *mflag = nullptr, *mpos = nullptr;
    int8_t* fold = nullptr;
    A(&ptp, (size_t)KN); A(&pth, (size_t)KN);
    A(&ft, Tn); A(&fk, Tn); A(&fr, Tn); A(&mflag, Tn); A(&mpos, Tn);
    if (!e) e = cudaMallocAsync(&pr, sizeof(int4) * (size_t)KN, st);
    if (!e) e = cudaMallocAsync(&mu, sizeof(int4) * Tn, st);
    if (!e) e = cudaMallocAsync(&fold, Tn, st);
    const int gb = (int)((Tn + 255) / 256) < 4 * I->num_sms ? (int)((Tn + 255) / 256) : 4 * I->num_sms;
    int U = 0;
    if (!e && T > 0) {
        // units (k, m): orders sorted stably by m * K + k, so time order within a unit
        k_assign_ukey<<<gb, 256, 0, st>>>(T, K, P, proc, I->prod, ukey, I->ctrl);
        e = sort_pairs(I, ukey, T, P * K - 1, uks, uord, I->tmp_a, I->tmp_b, st);
        if (!e) {
            k_assign_uflags<<<gb, 256, 0, st>>>(T, uks, flag);
            e = scan_exclusive(flag, upos, T, total, I->scan_blk, st, &I->ctrl->err);
        }
        if (!e) {
            k_assign_ustart<<<gb, 256, 0, st>>>(T, flag, upos, ustart);
            e = cudaMemcpyAsync(&U, total, sizeof(int), cudaMemcpyDeviceToHost, st);
        }
        if (!e) e = cudaStreamSynchronize(st);
        I->launches += 4;
    }
    // per unit: first order, product, region; the units with more than one order
    int MU = 0;
    if (!e && T > 0) {
        const int gu = (U + 255) / 256 < 4 * I->num_sms ? (U + 255) / 256 : 4 * I->num_sms;
        k_assign_units<<<gu, 256, 0, st>>>(U, ustart, uord, I->prod, I->reg, ft, fk, fr, mflag);
        e = scan_exclusive(mflag, mpos, U, total, I->scan_blk, st, &I->ctrl->err);
        if (!e) {
            k_assign_mlist<<<gu, 256, 0, st>>>(U, ustart, ft, fk, mflag, mpos, mu);
            e = cudaMemcpyAsync(&MU, total, sizeof(int), cudaMemcpyDeviceToHost, st);
        }
        if (!e) e = cudaStreamSynchronize(st);
        I->launches += 3;
    }
    // the cached actions naming (k, j), listed per (k, j) in time order
    auto tables = [&]() {
        k_part_keys<<<gb, 256, 0, st>>>(T, N, KN, I->prod, I->act_t, key);
        cudaError_t r = sort_pairs(I, key, T, KN, key_s, t_s, I->tmp_a, I->tmp_b, st);
        if (!r) k_part_offsets<<<(KN + 256) / 256, 256, 0, st>>>(key_s, T, KN, off);
        I->launches += 2;
        return r ? r : cudaGetLastError();
    };
    const int gkn = (KN + 255) / 256 < 8 * I->num_sms ? (KN + 255) / 256 : 8 * I->num_sms;
    const int smem = kPartWarps * kPartBatch * NPL * 32 * (int)sizeof(int32_t);
    const int blocks = (MU + kPartWarps - 1) / kPartWarps;
    // one warp per 32 units: U / 32 warps, 8 per CTA
    const int gfirst = (U + 255) / 256 < 8 * I->num_sms ? (U + 255) / 256 : 8 * I->num_sms;
    int iters = 0, converged = 0;
    for (int pass = 1; !e && T > 0 && pass <= iters_cap; ++pass) {
        if ((e = tables())) break;
        k_assign_pairs<<<gkn, 256, 0, st>>>(KN, I->x0, off, t_s, pr, ptp, pth);
        I->launches += 1;
        if ((e = cudaMemsetAsync(cflag, 0, sizeof(int32_t), st))) break;
#define ASSIGN_FIRST(NP_, D_)                                                               \
    k_assign_first<NP_, D_><<<gfirst, 256, 0, st>>>(U, N, ft, fk, fr, I->cost, I->lam, pth,   \
                                                    I->act_t, fold, I->ctrl, cflag)
        if (NPL == 1) {
            if (dual) ASSIGN_FIRST(1, true); else ASSIGN_FIRST(1, false);
        } else if (NPL == 2) {
            if (dual) ASSIGN_FIRST(2, true); else ASSIGN_FIRST(2, false);
        } else {
            if (dual) ASSIGN_FIRST(4, true); else ASSIGN_FIRST(4, false);
        }
#undef ASSIGN_FIRST
        I->launches += 1;
        if ((e = cudaGetLastError())) break;
#define ASSIGN_WALK(NP_, D_)                                                                \
    do {                                                                                    \
        e = cudaFuncSetAttribute(k_assign_walk<NP_, D_>,                                   \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);       \
        if (!e)                                                                             \
            k_assign_walk<NP_, D_><<<blocks, kPartWarps * 32, smem, st>>>(                 \
                MU, N, mu, ft, fold, uord, I->reg, I->cost, I->lam, I->x0, t_s, pr, ptp,   \
                I->act_t, I->ctrl, cflag);                                                 \
    } while (0)
        if (MU > 0) {
            if (NPL == 1) {
                if (dual) ASSIGN_WALK(1, true); else ASSIGN_WALK(1, false);
            } else if (NPL == 2) {
                if (dual) ASSIGN_WALK(2, true); else ASSIGN_WALK(2, false);
            } else {
                if (dual) ASSIGN_WALK(4, true); else ASSIGN_WALK(4, false);
            }
            I->launches += 1;
        }
#undef ASSIGN_WALK
        if (e) break;
        int hf = 0;
        if ((e = cudaGetLastError())) break;
        if ((e = cudaMemcpyAsync(&hf, cflag, sizeof(int), cudaMemcpyDeviceToHost, st))) break;
        if ((e = cudaStreamSynchronize(st))) break;
        iters = pass;
        if (!hf) {
            converged = 1;
            break;
        }
    }
    if (T == 0) {
        iters = 1;
        converged = 1;
    }
    // final stock of the returned cache (the last pass's tables describe it when it
    // changed nothing)
    if (!e && T > 0 && !converged) e = tables();
    if (!e && T > 0) {
        k_assign_final<<<gb, 256, 0, st>>>(KN, I->x0, off, I->xfin);
        I->launches += 1;
        e = cudaGetLastError();
    } else if (!e) {
        e = cudaMemcpyAsync(I->xfin, I->x0, sizeof(int32_t) * (size_t)KN, cudaMemcpyDeviceToDevice,
                            st);
    }
    if (!e) {
        k_part_result<<<1, 1, 0, st>>>(I->ctrl, iters, converged);
        e = cudaGetLastError();
    }
    int32_t* bufs[] = {ukey, uks, uord, flag, upos, ustart, key, key_s, t_s, off, cflag, total,
                       ptp, pth, ft, fk, fr, mflag, mpos};
    for (int32_t* b : bufs)
        if (b) cudaFreeAsync(b, st);
    if (pr) cudaFreeAsync(pr, st);
    if (mu) cudaFreeAsync(mu, st);
    if (fold) cudaFreeAsync(fold, st);
    return e;
}

cudaError_t check_alpha_init(Instance* I, const int8_t* alpha, cudaStream_t st) {
    if (I->T == 0) return cudaSuccess;
    k_part_check_init<<<4 * I->num_sms, 256, 0, st>>>(I->T, I->N, alpha, I->ctrl);
    I->launches += 1;
    return cudaGetLastError();
}

}  // namespace pic
