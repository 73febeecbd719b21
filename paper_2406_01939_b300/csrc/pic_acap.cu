// Algorithm 1 for a caller's assignment of orders to processes (the uniform
// random partition of Sec. 4.1, Table 1) with node capacity, literally: every
// process replays the horizon from s_1 up to its last own order in its own
// state (x, c).  Its own orders take fresh policy calls; every other order
// applies its cached action when that action is feasible in the process's
// state (x[k][n] > 0 and c[n] > 0), else a^phi (Alg. 1 lines 4-7).
//
// Without capacity, or with product partitions, a process's view of other
// processes' orders has a closed form (the (product, process) chains and the
// per-node success lists of the other partition modes).  With capacity and an
// arbitrary partition it has none: whether a foreign cached action finds
// capacity depends on every earlier success at its node in this process's own
// view, which the process's fresh actions move, and a changed success changes
// later products' stock in turn.  So a pass costs sum over processes of their
// last own order: about P T order-steps against T for contiguous chunks.
//
// One warp per process.  Per pass the process's stock x[K][N] is a copy of x0
// in its own slice of a device scratch (P K N ints), its capacity row c[N]
// lives in shared memory.  The orders come 32 at a time: each lane loads one
// order and, for a foreign order, the stock entry its cached action would
// take; then the warp walks the 32 in time order, keeping those stock values
// current (a decrement applied at (k, n) lowers every later lane's copy of the
// same entry) and writing every decrement to the slice, where a fresh decision
// reads its product's row.
#include <climits>

#include "pic_device.cuh"

namespace pic {

namespace {

constexpr int kAcWarps = 4;
constexpr int kAcMaxN = 128;

__global__ void k_acap_last(int T, int P, const int32_t* __restrict__ proc, int32_t* last, Ctrl* ctrl) {
    int bad = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
         t += (long long)gridDim.x * blockDim.x) {
        const int m = proc[t];
        if (m < 0 || m >= P) bad = 1;
        else atomicMax(&last[m], (int)t);
    }
    if (bad) atomicOr(&ctrl->pad0, 128);
}

template <int NPL, bool DUAL>
__global__ void __launch_bounds__(32 * kAcWarps) k_acap_pass(
    int T, int N, int K, int P, const int32_t* __restrict__ proc, const int32_t* __restrict__ prod,
    const int32_t* __restrict__ reg, const int32_t* __restrict__ cost, const int32_t* __restrict__ lam,
    const int32_t* __restrict__ x0, const int32_t* __restrict__ cap, const int32_t* __restrict__ last,
    const int8_t* __restrict__ prev, int8_t* __restrict__ next, int32_t* xs, int* changed,
    unsigned long long* calls) {
    __shared__ int s_c[kAcWarps][kAcMaxN];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = blockIdx.x * kAcWarps + w;
    if (m >= P) return;
    const int lm = last[m];
    if (lm < 0) return;  // a process without orders
    int32_t* xm = xs + (size_t)m * K * N;
    for (size_t i = lane; i < (size_t)K * N; i += 32) xm[i] = x0[i];
    for (int n = lane; n < N; n += 32) s_c[w][n] = cap[n];
    __syncwarp();
    int* c = s_c[w];
    bool chg = false;
    unsigned long long ncalls = 0;
    for (int base = 0; base <= lm; base += 32) {
        const int cnt = min(32, lm + 1 - base);
        const int t = base + lane;
        int pk = 0, rg = 0, ao = -1, xv = 0;
        bool own = false;
        if (lane < cnt) {
            pk = prod[t];
            rg = reg[t];
            ao = prev[t];
            own = proc[t] == m;
            if (!own && ao >= 0) xv = xm[(size_t)pk * N + ao];
        }
        for (int q = 0; q < cnt; ++q) {
            const int k = __shfl_sync(kFull, pk, q);
            const int a0 = __shfl_sync(kFull, ao, q);
            const bool o = __shfl_sync(kFull, own ? 1 : 0, q) != 0;
            int act = -1;  // the action applied at order base + q (-1: none)
            if (o) {
                // a fresh decision in this process's state (lanes hold nodes lane + 32 i)
                const int r = __shfl_sync(kFull, rg, q);
                int best = INT_MAX;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int n = lane + 32 * i;
                    if (n < N && xm[(size_t)k * N + n] > 0 && c[n] > 0) {
                        int sc = cost[(size_t)r * N + n];
                        if (DUAL) sc -= lam[(size_t)k * N + n];
                        best = min(best, sc);
                    }
                }
                const int bs = __reduce_min_sync(kFull, best);
                int cand = INT_MAX;
                if (bs != INT_MAX) {
#pragma unroll
                    for (int i = 0; i < NPL; ++i) {
                        const int n = lane + 32 * i;
                        if (n < N && xm[(size_t)k * N + n] > 0 && c[n] > 0) {
                            int sc = cost[(size_t)r * N + n];
                            if (DUAL) sc -= lam[(size_t)k * N + n];
                            if (sc == bs) cand = min(cand, n);
                        }
                    }
                }
                const int nb = __reduce_min_sync(kFull, cand);
                act = nb == INT_MAX ? -1 : nb;
                if (lane == 0) {
                    next[base + q] = (int8_t)act;
                    chg |= act != a0;
                    ++ncalls;
                }
            } else if (a0 >= 0) {
                const int xq = __shfl_sync(kFull, xv, q);
                if (xq > 0 && c[a0] > 0) act = a0;  // the cached action is feasible
            }
            __syncwarp();
            if (act >= 0) {
                if (lane == 0) {
                    xm[(size_t)k * N + act] -= 1;
                    c[act] -= 1;
                }
                // later foreign orders of this batch that would take the same entry
                if (lane > q && !own && pk == k && ao == act) xv -= 1;
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        if (chg) atomicOr(changed, 1);
        if (ncalls) atomicAdd(calls, ncalls);
    }
}

__global__ void k_acap_xfin(int T, int N, const int32_t* __restrict__ prod, const int8_t* __restrict__ act,
                            int32_t* xfin) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = act[t];
        if (a >= 0) atomicSub(&xfin[(size_t)prod[t] * N + a], 1);
    }
}

__global__ void k_acap_result(Ctrl* ctrl, int iters, int converged, unsigned long long* calls) {
    ctrl->iters = iters;
    ctrl->converged = converged;
    ctrl->policy_calls = *calls;
}

}  // namespace

// Algorithm 1 with node capacity and process proc[t] owning order t, P
// processes; the cache (time order, I->act_t) must hold alpha^0.  Scratch
// (P K N stock entries and two caches) is taken with cudaMallocAsync on the
// call's stream.  On return I->act_t holds the last cache, I->xfin the stock
// after its actions, ctrl the pass count and convergence.
cudaError_t picard_assigned_cap(Instance* I, const pic_policy* pol, const int32_t* proc, int P,
                                int iters_cap, cudaStream_t st) {
    const int T = I->T, N = I->N, K = I->K;
    const bool dual = pol->kind == PIC_POLICY_DUAL;
    const int NPL = N <= 32 ? 1 : (N <= 64 ? 2 : 4);
    int32_t *last = nullptr, *xs = nullptr;
    int8_t* nxt = nullptr;
    int* changed = nullptr;
    unsigned long long* calls = nullptr;
    cudaError_t e = cudaSuccess;
    const size_t Tn = T > 0 ? (size_t)T : 1;
    if (!e) e = cudaMallocAsync(&last, sizeof(int32_t) * (size_t)P, st);
    if (!e) e = cudaMallocAsync(&xs, sizeof(int32_t) * (size_t)P * K * N, st);
    if (!e) e = cudaMallocAsync(&nxt, Tn, st);
    if (!e) e = cudaMallocAsync(&changed, sizeof(int), st);
    if (!e) e = cudaMallocAsync(&calls, sizeof(unsigned long long), st);
    const int gb = (int)((Tn + 255) / 256) < 4 * I->num_sms ? (int)((Tn + 255) / 256) : 4 * I->num_sms;
    int iters = 0, converged = 0;
    if (!e) e = cudaMemsetAsync(last, 0xff, sizeof(int32_t) * (size_t)P, st);
    if (!e) e = cudaMemsetAsync(calls, 0, sizeof(unsigned long long), st);
    if (!e && T > 0) {
        k_acap_last<<<gb, 256, 0, st>>>(T, P, proc, last, I->ctrl);
        I->launches += 1;
        e = cudaGetLastError();
    }
    if (!e && T > 0) {  // an out-of-range process is an error before any pass
        int bad = 0;
        e = cudaMemcpyAsync(&bad, &I->ctrl->pad0, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaStreamSynchronize(st);
        if (!e && (bad & 128)) iters_cap = 0;
    }
    const int blocks = (P + kAcWarps - 1) / kAcWarps;
    for (int pass = 1; !e && T > 0 && pass <= iters_cap; ++pass) {
        // orders whose owner does not write them this pass keep nothing stale:
        // every order has exactly one owner, which writes it
        if ((e = cudaMemsetAsync(changed, 0, sizeof(int), st))) break;
#define ACAP(NP_, D_)                                                                        \
    k_acap_pass<NP_, D_><<<blocks, 32 * kAcWarps, 0, st>>>(T, N, K, P, proc, I->prod, I->reg,   \
                                                          I->cost, I->lam, I->x0, I->cap, last, \
                                                          I->act_t, nxt, xs, changed, calls)
        if (NPL == 1) {
            if (dual) ACAP(1, true); else ACAP(1, false);
        } else if (NPL == 2) {
            if (dual) ACAP(2, true); else ACAP(2, false);
        } else {
            if (dual) ACAP(4, true); else ACAP(4, false);
        }
#undef ACAP
        I->launches += 1;
        if ((e = cudaGetLastError())) break;
        if ((e = cudaMemcpyAsync(I->act_t, nxt, (size_t)T, cudaMemcpyDeviceToDevice, st))) break;
        int hf = 0;
        if ((e = cudaMemcpyAsync(&hf, changed, sizeof(int), cudaMemcpyDeviceToHost, st))) break;
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
    if (!e) e = cudaMemcpyAsync(I->xfin, I->x0, sizeof(int32_t) * (size_t)K * N, cudaMemcpyDeviceToDevice, st);
    if (!e && T > 0) {
        k_acap_xfin<<<gb, 256, 0, st>>>(T, N, I->prod, I->act_t, I->xfin);
        I->launches += 1;
        e = cudaGetLastError();
    }
    if (!e) {
        k_acap_result<<<1, 1, 0, st>>>(I->ctrl, iters, converged, calls);
        I->launches += 1;
        e = cudaGetLastError();
    }
    if (last) cudaFreeAsync(last, st);
    if (xs) cudaFreeAsync(xs, st);
    if (nxt) cudaFreeAsync(nxt, st);
    if (changed) cudaFreeAsync(changed, st);
    if (calls) cudaFreeAsync(calls, st);
    return e;
}

}  // namespace pic
