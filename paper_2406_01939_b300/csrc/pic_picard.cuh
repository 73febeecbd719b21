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
};

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

constexpr int kMaxWarpsPerCta = 32;

// Look-back words carry their pass in the high half: (pass << 32) | value, so a
// reader learns from the word itself whether it was written in this pass.  The
// poll is a volatile relaxed load so that every spin really re-reads memory.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long tagged(int it, int v) {
    return ((unsigned long long)(unsigned)it << 32) | (unsigned)v;
}

// Phase S for one super-block (head segment s of a chain whose product changed):
// its total, published; then the exclusive prefix of the chain's earlier
// super-blocks by decoupled look-back (an inclusive prefix ends the walk, a bare
// total is added and the walk continues); the inclusive prefix, published; then
// the exclusive prefix at every segment of the block.  A block whose orders all
// precede the product's first change (clean) keeps last pass's prefixes and only
// re-publishes them.  Waits are bounded by the deadline; on expiry the error is
// recorded and the pass is abandoned at the next grid barrier.
template <int NPL>
__device__ __forceinline__ void superblock_prefix(const KArgs& a, int s, const SegMeta& m, int it,
                                                  int fcp, unsigned long long deadline) {
    const int lane = lane_id();
    const int NP = a.NP;
    const int send = min(s + kSuperBlock, m.ce);
    constexpr int kRows = 8 / NPL;  // rows per round trip
    if (send < m.ce && it > 1) {
        const int next_j0 = __ldg(&a.meta[send].j0);
        if (next_j0 <= fcp) {  // clean: aggregates and prefixes unchanged
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const size_t o = (size_t)s * NP + lane + 32 * i;
                a.sbincl[o] = tagged(it, (int)(unsigned)a.sbincl[o]);
            }
            return;
        }
    }
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
            for (int i = 0; i < NPL; ++i) tot[i] += v[u][i];
    }
    int acc[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) acc[i] = 0;
    if (s > m.cf) {
#pragma unroll
        for (int i = 0; i < NPL; ++i) a.sbagg[(size_t)s * NP + lane + 32 * i] = tagged(it, tot[i]);
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
                    inc_ok &= (int)(wi[i] >> 32) == it;
                    agg_ok &= (int)(wa[i] >> 32) == it;
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
    for (int i = 0; i < NPL; ++i)
        a.sbincl[(size_t)s * NP + lane + 32 * i] = tagged(it, acc[i] + tot[i]);
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


}  // namespace picard

// MLP Picard kernel (pic_mlp.cu).
cudaError_t picard_mlp(Instance* I, const picard::KArgs& a, const pic_policy* pol, cudaStream_t st);

// Group-per-segment Picard kernel (pic_grp.cu).
int grp_lanes(int N);
bool grp_ok(const Instance* I);
cudaError_t picard_grp(Instance* I, const picard::KArgs& a, bool dual, cudaStream_t st);

}  // namespace pic
