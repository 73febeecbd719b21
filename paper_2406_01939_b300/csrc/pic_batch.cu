// Batches of trajectories (pic_create_batch, pic_simulate_batch).
//
// A batch is held as one combined instance: trajectory b's orders, products
// and regions occupy their own index ranges, its ids shifted into them at
// creation.  Products never interact (Assumption 1 of Sec. 3.2) and no two
// trajectories share a product, so one Picard launch over the combined instance
// runs, trajectory by trajectory, exactly the passes each would run alone with
// the same chunks: trajectory b is cut into min(M, T_b) contiguous chunks of
// ceil(T_b / min(M, T_b)) orders, as pic_simulate would cut it.  The loop runs
// until no trajectory changes; each trajectory's own pass count is its last
// changing pass plus one, recorded on the device.  Trajectory parallelism is
// orthogonal to the Picard parallelism inside a trajectory (Sec. 3), and the
// single launch lets one pass serve every trajectory with one grid barrier.
//
// Each segment (work unit of one product) is replayed under its trajectory's
// policy: integer policies read the cost table from global memory, MLP
// policies share one weight set staged in shared memory.  The per-call device
// work can run as a CUDA graph (PIC_FLAG_GRAPH); the chunk count, CTA shape and
// segment window can be picked by a timing autotuner (num_chunks = 0).
#include <algorithm>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pic_mlp.cuh"
#include "pic_replay.cuh"

using namespace pic;

namespace {

using namespace pic::picard;
using namespace pic::mlp;

}  // namespace

namespace pic {
cudaError_t picard_wave_batch(Instance* I, const KArgs& a, const MlpPolicy& p,
                              const int32_t* traj_of_prod, const BatchPol* pol, const int32_t* toff,
                              int32_t* last_chg, cudaStream_t st);
}  // namespace pic

namespace {

using namespace pic::picard;
using namespace pic::mlp;

// ---------------------------------------------------------------------------- creation kernels
// Owner of global index i in an offset table off[0..B] (off[0] = 0, non-
// decreasing, off[B] > i): the largest b < B with off[b] <= i, which skips
// empty trajectories.
__device__ __forceinline__ int owner(const int32_t* __restrict__ off, int B, int i) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Local ids of every order checked against its trajectory's K_b and R_b (bits
// 1 and 2 of *bad), then shifted into the trajectory's ranges.
__global__ void k_batch_ids(int T, int B, const int32_t* __restrict__ toff,
                            const int32_t* __restrict__ koff, const int32_t* __restrict__ roff,
                            int32_t* prod, int32_t* reg, int* bad) {
    int bits = 0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = owner(toff, B, (int)t);
        const int k = prod[t], r = reg[t];
        if ((unsigned)k >= (unsigned)(koff[b + 1] - koff[b])) bits |= 1; else prod[t] = k + koff[b];
        if ((unsigned)r >= (unsigned)(roff[b + 1] - roff[b])) bits |= 2; else reg[t] = r + roff[b];
    }
    if (bits) atomicOr(bad, bits);
}

// own[i] = owner of i; local[i] = i - off[owner] (either may be null).
__global__ void k_owners(int n, int B, const int32_t* __restrict__ off, int32_t* own,
                         int32_t* local) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = owner(off, B, (int)i);
        if (own) own[i] = b;
        if (local) local[i] = (int)i - off[b];
    }
}

// ---------------------------------------------------------------------------- per-call kernels
// Cost and a^phi count of each trajectory from its actions in time order:
// CTA (b, s) sums slice s of gridDim.y slices of trajectory b into tres (zeroed
// before the launch); the batch totals are added to the control block.
constexpr int kReduceThreads = 256;

__global__ void __launch_bounds__(kReduceThreads) k_traj_reduce(
    const int8_t* __restrict__ act_t, const int32_t* __restrict__ reg,
    const int32_t* __restrict__ cost, int N, const int32_t* __restrict__ toff, long long* tres,
    Ctrl* ctrl) {
    __shared__ long long sc[kReduceThreads / 32], sl[kReduceThreads / 32];
    const int b = blockIdx.x;
    const int len = toff[b + 1] - toff[b], per = (len + (int)gridDim.y - 1) / (int)gridDim.y;
    const int t0 = toff[b] + min(len, (int)blockIdx.y * per), t1 = toff[b] + min(len, ((int)blockIdx.y + 1) * per);
    long long c = 0, l = 0;
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const int a = act_t[t];
        if (a >= 0) c += __ldg(cost + (size_t)reg[t] * N + a);
        else l += 1;
    }
    c = warp_sum_i64(c);
    l = warp_sum_i64(l);
    if ((threadIdx.x & 31) == 0) {
        sc[threadIdx.x >> 5] = c;
        sl[threadIdx.x >> 5] = l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        c = 0;
        l = 0;
        for (int w = 0; w < kReduceThreads / 32; ++w) {
            c += sc[w];
            l += sl[w];
        }
        if (c) atomicAdd((unsigned long long*)&tres[2 * b], (unsigned long long)c);
        if (l) atomicAdd((unsigned long long*)&tres[2 * b + 1], (unsigned long long)l);
        atomicAdd((unsigned long long*)&ctrl->total_cost, (unsigned long long)c);
        atomicAdd((unsigned long long*)&ctrl->lost, (unsigned long long)l);
    }
}

// Per-trajectory cost and lost count: enough slices per trajectory to give
// every SM a few CTAs.
inline cudaError_t traj_reduce(Instance& I, int B, cudaStream_t st) {
    Batch* bt = I.batch;
    cudaError_t e = cudaMemsetAsync(bt->tres, 0, sizeof(long long) * 2 * (size_t)B, st);
    if (e) return e;
    const int S = std::max(1, std::min(64, (4 * I.num_sms + B - 1) / B));
    k_traj_reduce<<<dim3(B, S), kReduceThreads, 0, st>>>(I.act_t, I.reg, I.cost, I.N, bt->toff, bt->tres,
                                                          I.ctrl);
    return cudaGetLastError();
}

// Sequential definition (Sec. 2) for every trajectory at once: one warp per
// trajectory, kSeqWarps trajectories per CTA sharing one staged copy of the MLP
// weights.  Only trajectory parallelism: the baseline the Picard launch is
// measured against.
constexpr int kSeqWarps = 4;

template <int NPL, bool SMEMW>
__global__ void __launch_bounds__(32 * kSeqWarps) k_seq_batch(
    int B, int N, const int32_t* __restrict__ toff, const int32_t* __restrict__ prod,
    const int32_t* __restrict__ reg, const int32_t* __restrict__ cost,
    const int32_t* __restrict__ lam, int32_t* xw, int8_t* __restrict__ act_t,
    const BatchPol* __restrict__ pol, MlpPolicy p, int has_mlp, Ctrl* ctrl) {
    extern __shared__ uint4 s_w[];
    __shared__ float s_fs[kSeqWarps][128];
    __shared__ __align__(16) float s_hs[kSeqWarps][kHidden];
    if (SMEMW && has_mlp) stage_weights(p, s_w);
    const uint4* W1p = SMEMW ? s_w : p.W1p;
    const uint4* W2p = SMEMW ? s_w + p.N * kHidden / 8 : p.W2p;
    const int w = threadIdx.x >> 5;
    const int b = blockIdx.x * kSeqWarps + w;
    if (b >= B) return;
    const int t0 = toff[b], T = toff[b + 1] - t0;
    const BatchPol bp = pol[b];
    if (bp.kind <= PIC_POLICY_DUAL) {
        long long c = 0, l = 0;  // costs come from k_traj_reduce
        seq_int_body<NPL, true, false>(T, N, prod + t0, reg + t0, cost, nullptr,
                                       bp.kind == PIC_POLICY_DUAL ? lam : nullptr, xw, act_t + t0,
                                       c, l);
    } else {
        MlpPolicy q = p;
        q.gumbel = bp.kind == PIC_POLICY_GUMBEL;
        q.seed = bp.seed;
        q.traj = bp.traj;
        MlpCounts mc{0, 0, 0, 0, 0};
        seq_mlp_body<NPL, SMEMW>(T, N, prod + t0, reg + t0, xw, act_t + t0, q, W1p, W2p, s_fs[w],
                                 s_hs[w], mc);
        if (lane_id() == 0 && mc.sat) atomicAdd(&ctrl->sat_rows, mc.sat);
        if (lane_id() == 0 && mc.near) atomicAdd(&ctrl->near_ties, mc.near);
    }
}

// ---------------------------------------------------------------------------- Picard launch
struct BatchArgs {
    const int32_t* __restrict__ traj_of_prod;
    const BatchPol* __restrict__ pol;
    const int32_t* __restrict__ toff;
    const int32_t* __restrict__ perm;
    int32_t* last_chg;
    int has_mlp;
};

// CTA shapes the launch (and the autotuner) can use, as (threads, CTAs per SM):
// 0 = (256, 1), 1 = (256, 2), 2 = (512, 1); see batch_shape.
constexpr int kNumShapes = 3;
constexpr int kDefaultShape = 2;

template <int NPL, int THREADS, int MINB, bool FULL, bool SPEC>
__global__ void __launch_bounds__(THREADS, MINB) k_picard_batch(KArgs a, MlpPolicy p, BatchArgs b) {
    constexpr bool SMEMW = true;  // the packed weights (N KB) fit in shared memory for any N
    constexpr int WARPS = THREADS / 32;
    extern __shared__ uint4 s_w[];
    __shared__ float s_fs[WARPS][128];
    __shared__ __align__(16) float s_hs[WARPS][kHidden];
    if (b.has_mlp) stage_weights(p, s_w);
    const uint4* W1p = s_w;
    const uint4* W2p = s_w + p.N * kHidden / 8;
    const CostTable<false> ct{a.cost, nullptr, a.N};
    const int wib = threadIdx.x >> 5;
    unsigned long long calls = 0;
    MlpCounts mc{0, 0, 0, 0, 0};
    picard_passes<NPL, WARPS>(a, calls, [&](int seg, const SegMeta& m, int fcp, int* fc_cur, int it) {
        const int tb = __ldg(b.traj_of_prod + m.k);
        const BatchPol bp = b.pol[tb];
        bool chg;
        if (bp.kind <= PIC_POLICY_DUAL) {
            chg = replay_segment<NPL, true, false, FULL>(a, ct, seg, m, fcp, fc_cur, it,
                                                         bp.kind == PIC_POLICY_DUAL, calls);
        } else {
            MlpPolicy q = p;
            q.gumbel = bp.kind == PIC_POLICY_GUMBEL;
            q.seed = bp.seed;
            q.traj = bp.traj;
            const unsigned long long m0 = mc.calls;
            chg = replay_segment_mlp<NPL, SMEMW, SPEC>(a, q, W1p, W2p, b.perm, seg, m, fcp, fc_cur, it,
                                                 __ldg(b.toff + tb), mc, s_fs[wib], s_hs[wib]);
            calls += mc.calls - m0;
        }
        // the trajectory's last changing pass (read first: many segments of one
        // trajectory change in the same pass)
        if (chg && lane_id() == 0 && ld_volatile(&b.last_chg[tb]) < it) atomicMax(&b.last_chg[tb], it);
        return chg;
    });
    if (lane_id() == 0 && mc.calls) {
        atomicAdd(&a.ctrl->mlp_calls, mc.calls);
        atomicAdd(&a.ctrl->rescored, mc.rescored);
        atomicAdd(&a.ctrl->tc_rows, mc.tc);
        atomicAdd(&a.ctrl->sat_rows, mc.sat);
        atomicAdd(&a.ctrl->near_ties, mc.near);
    }
}

template <int NPL, int THREADS, int MINB, bool FULL, bool SPEC>
cudaError_t launch_batch(Instance* I, const KArgs& a, const MlpPolicy& p, const BatchArgs& b,
                         cudaStream_t st) {
    auto kern = k_picard_batch<NPL, THREADS, MINB, FULL, SPEC>;
    const size_t smem = b.has_mlp ? packed_weight_bytes(I->N) : 0;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THREADS, smem))) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = occ < MINB ? occ : MINB;
    const int grid = I->num_sms * per_sm;
    I->coop_blocks = grid;
    I->cta_threads = THREADS;
    I->ctas_per_sm = per_sm;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the passes meet at grid barriers
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    I->launches += 1;
    return cudaLaunchKernelEx(&cfg, kern, a, p, b);
}

template <int NPL, bool FULL, bool SPEC>
cudaError_t batch_shape(Instance* I, int shape, const KArgs& a, const MlpPolicy& p,
                        const BatchArgs& b, cudaStream_t st) {
    if (shape == 0) return launch_batch<NPL, 256, 1, FULL, SPEC>(I, a, p, b, st);
    if (shape == 1) return launch_batch<NPL, 256, 2, FULL, SPEC>(I, a, p, b, st);
    return launch_batch<NPL, 512, 1, FULL, SPEC>(I, a, p, b, st);
}

// tc: MLP decisions through speculative tensor-core tiles (N <= 64)
cudaError_t batch_dispatch(Instance* I, int shape, bool tc, const KArgs& a, const MlpPolicy& p,
                           const BatchArgs& b, cudaStream_t st) {
    const int npl = (I->N + 31) / 32;
    const bool full = I->N == 32 * npl;  // every lane owns real warehouses
    if (npl == 1) {
        if (tc) return full ? batch_shape<1, true, true>(I, shape, a, p, b, st)
                            : batch_shape<1, false, true>(I, shape, a, p, b, st);
        return full ? batch_shape<1, true, false>(I, shape, a, p, b, st)
                    : batch_shape<1, false, false>(I, shape, a, p, b, st);
    }
    if (npl == 2) {
        if (tc) return full ? batch_shape<2, true, true>(I, shape, a, p, b, st)
                            : batch_shape<2, false, true>(I, shape, a, p, b, st);
        return full ? batch_shape<2, true, false>(I, shape, a, p, b, st)
                    : batch_shape<2, false, false>(I, shape, a, p, b, st);
    }
    return batch_shape<4, false, false>(I, shape, a, p, b, st);
}

template <int NPL>
cudaError_t launch_seq_batch(Instance* I, const MlpPolicy& p, bool has_mlp, cudaStream_t st) {
    constexpr bool SMEMW = true;  // the packed weights fit in shared memory for any N
    auto kern = k_seq_batch<NPL, SMEMW>;
    const size_t smem = has_mlp ? packed_weight_bytes(I->N) : 0;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const Batch* bt = I->batch;
    const int grid = (bt->B + kSeqWarps - 1) / kSeqWarps;
    I->launches += 1;
    kern<<<grid, 32 * kSeqWarps, smem, st>>>(bt->B, I->N, bt->toff, I->prod, I->reg, I->cost, I->lam,
                                             I->xwork, I->act_t, bt->pol, p, has_mlp ? 1 : 0,
                                             I->ctrl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------- host side
thread_local char t_msg[320];

pic_status fail(pic_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
pic_status fail(pic_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_msg, sizeof(t_msg), fmt, ap);
    va_end(ap);
    return record_error(s, t_msg);
}

pic_status cuda_fail(cudaError_t e, const char* what, int line) {
    return fail(e == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA, "%s failed: %s (pic_batch.cu:%d)",
                what, cudaGetErrorString(e), line);
}

#define BCU(call)                                                     \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call, __LINE__); \
    } while (0)

// Everything one Picard call of a batch depends on besides the per-trajectory
// policy selectors (which travel through bt->h_pol).
struct CallCfg {
    int M, W, shape, iters_cap, flags;
    bool tc;  // speculative tensor-core tiles for the MLP decisions
    const int8_t* alpha_init;
    bool trace;
    unsigned long long timeout_ns;
    bool has_mlp;
    pic_policy mlp;  // the shared MLP parameters (kind field unused)
};

// Layout of the pinned host staging block that receives a call's results.
size_t out_bytes(int B) { return sizeof(Ctrl) + (size_t)B * (2 * sizeof(long long) + sizeof(int32_t)); }

unsigned long long fnv(unsigned long long h, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

unsigned long long cfg_sig(const CallCfg& c) {
    unsigned long long h = 14695981039346656037ull;
    const long long v[] = {c.M, c.W, c.shape, c.tc, c.iters_cap, c.flags, (long long)(size_t)c.alpha_init,
                           c.trace, (long long)c.timeout_ns, c.has_mlp,
                           (long long)(size_t)c.mlp.W1, (long long)(size_t)c.mlp.b1,
                           (long long)(size_t)c.mlp.W2, (long long)(size_t)c.mlp.b2,
                           (long long)(size_t)c.mlp.E};
    return fnv(h, v, sizeof(v));
}

// Chunk lengths for M chunks per trajectory, then the order tables (if the
// chunking or window changed since they were built).
pic_status ensure_tables(Instance& I, int M, int W, cudaStream_t st) {
    Batch* bt = I.batch;
    if (I.tables_m == M && I.tables_w == W) return PIC_OK;
    std::vector<int32_t> L(bt->B);
    for (int b = 0; b < bt->B; ++b) {
        const long long Tb = bt->h_toff[b + 1] - bt->h_toff[b];
        const long long Mb = Tb < M ? (Tb > 0 ? Tb : 1) : M;
        L[b] = (int32_t)((Tb + Mb - 1) / Mb > 0 ? (Tb + Mb - 1) / Mb : 1);
    }
    BCU(cudaMemcpyAsync(bt->chunk_len, L.data(), sizeof(int32_t) * bt->B, cudaMemcpyHostToDevice, st));
    BCU(cudaStreamSynchronize(st));  // L is pageable and goes out of scope
    BCU(build_tables(&I, M, W, st));
    I.tables_m = M;
    I.tables_w = W;
    return PIC_OK;
}

// The per-call device work of a Picard call (graph-capturable: no allocation,
// no synchronisation, host memory only through pinned staging).
pic_status enqueue_picard(Instance& I, const CallCfg& c, cudaStream_t st) {
    Batch* bt = I.batch;
    const int B = bt->B;
    BCU(cudaMemcpyAsync(bt->pol, bt->h_pol, sizeof(BatchPol) * B, cudaMemcpyHostToDevice, st));
    BCU(cudaMemsetAsync(I.ctrl, 0, offsetof(Ctrl, nruns), st));
    BCU(take_tags(I, c.iters_cap, st));
    BCU(cudaMemsetAsync(bt->last_chg, 0, sizeof(int32_t) * B, st));
    BCU(build_lpt(&I, bt->pol, kMlpLptWeight, st));
    BCU(init_cache(I, c.alpha_init, st));
    if (c.has_mlp) BCU(mlp_prepare(&I, &c.mlp, st));
    if (c.trace) BCU(cudaMemsetAsync(I.trace, 0, sizeof(long long) * kTraceCols * kTraceCap, st));
    KArgs a;
    a.T = I.T; a.N = I.N; a.K = I.K; a.NP = I.NP; a.R = I.R;
    a.reg_s = I.reg_s; a.run_start = I.run_start; a.seg_run = I.seg_run;
    a.seg_prod = I.seg_prod; a.seg_cf = I.seg_cf; a.seg_ce = I.seg_ce;
    a.x0 = I.x0; a.cost = I.cost; a.lam = I.lam;
    a.alpha_s = I.alpha_s; a.agg = I.agg; a.carry = I.carry; a.sbexc = I.sbexc;
    a.sbagg = I.sbagg; a.sbincl = I.sbincl; a.meta = I.seg_meta; a.lpt = I.seg_lpt;
    a.fc = I.fc; a.xfin = I.xfin;
    a.ctrl = I.ctrl; a.max_iters = c.iters_cap; a.flags = c.flags;
    a.first_dirty = c.alpha_init != nullptr; a.timeout_ns = c.timeout_ns;
    a.trace = c.trace ? I.trace : nullptr;
    a.run_chunk = nullptr;  // no max_steps window
    a.perm = nullptr;
    a.win_steps = 0;
    a.M = a.L = 0;
    pic_policy mp = c.mlp;
    mp.kind = PIC_POLICY_MLP;
    const MlpPolicy p = make_policy_view(&I, &mp, c.flags);
    BatchArgs ba;
    ba.traj_of_prod = bt->traj_of_prod;
    ba.pol = bt->pol;
    ba.toff = bt->toff;
    ba.perm = I.perm;
    ba.last_chg = bt->last_chg;
    ba.has_mlp = c.has_mlp ? 1 : 0;
    if (c.has_mlp && (c.flags & PIC_FLAG_WAVE) && wave_applies(&I) && c.W == 1)  // one run per unit
        BCU(picard_wave_batch(&I, a, p, ba.traj_of_prod, ba.pol, ba.toff, ba.last_chg, st));
    else
        BCU(batch_dispatch(&I, c.shape, c.tc && I.N <= 64, a, p, ba, st));
    BCU(scatter_actions(&I, st));
    I.launches += 1;
    BCU(traj_reduce(I, B, st));
    unsigned char* h = bt->h_out;
    BCU(cudaMemcpyAsync(h, I.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    BCU(cudaMemcpyAsync(h + sizeof(Ctrl), bt->tres, sizeof(long long) * 2 * B, cudaMemcpyDeviceToHost, st));
    BCU(cudaMemcpyAsync(h + sizeof(Ctrl) + sizeof(long long) * 2 * B, bt->last_chg,
                        sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st));
    return PIC_OK;
}

// One Picard call of the batch with configuration c: tables, per-segment state,
// then the per-call work directly or through the cached graph.  Events ev[1],
// ev[2] bracket the per-call work.
pic_status run_picard(Instance& I, const CallCfg& c, bool graph, cudaStream_t st) {
    Batch* bt = I.batch;
    pic_status s = ensure_tables(I, c.M, c.W, st);
    if (s != PIC_OK) return s;
    BCU(prepare_picard_state(I, c.W, c.iters_cap, st));
    if (c.has_mlp) BCU(mlp_alloc(&I));
    if (!graph) {
        BCU(cudaEventRecord(I.ev[1], st));
        if ((s = enqueue_picard(I, c, st)) != PIC_OK) return s;
        BCU(cudaEventRecord(I.ev[2], st));
        return PIC_OK;
    }
    // the graph holds buffer addresses: a reallocation since capture needs a new one
    const void* bufs[] = {I.agg, I.carry, I.sbexc, I.sbagg, I.sbincl, I.mlp_P};
    const unsigned long long sig = fnv(cfg_sig(c), bufs, sizeof(bufs));
    if (!bt->gexec || bt->gsig != sig) {
        if (bt->gexec) {
            cudaGraphExecDestroy(bt->gexec);
            bt->gexec = nullptr;
        }
        if (!bt->cap_stream) BCU(cudaStreamCreateWithFlags(&bt->cap_stream, cudaStreamNonBlocking));
        const int l0 = I.launches;
        BCU(cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeThreadLocal));
        s = enqueue_picard(I, c, bt->cap_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(bt->cap_stream, &g);
        if (s != PIC_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (ec) return cuda_fail(ec, "cudaStreamEndCapture", __LINE__);
        const cudaError_t ei = cudaGraphInstantiate(&bt->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ei) {
            bt->gexec = nullptr;
            return cuda_fail(ei, "cudaGraphInstantiate", __LINE__);
        }
        bt->gsig = sig;
        bt->glaunches = I.launches - l0;
        I.launches = l0;  // counted when the graph runs
    }
    BCU(cudaEventRecord(I.ev[1], st));
    BCU(cudaGraphLaunch(bt->gexec, st));
    BCU(cudaEventRecord(I.ev[2], st));
    I.launches += bt->glaunches;
    return PIC_OK;
}

// Timing autotuner: chunk count M, then CTA shape, then segment window, each
// chosen by timing one full call of this batch (per-call work only; tables are
// built outside the timed region).  Cached per batch and policy mix.
pic_status autotune(Instance& I, CallCfg& c, cudaStream_t st) {
    Batch* bt = I.batch;
    unsigned long long sig = 14695981039346656037ull;
    for (int b = 0; b < bt->B; ++b) sig = fnv(sig, &bt->h_pol[b].kind, sizeof(int));
    sig = fnv(sig, &c.flags, sizeof(int));
    if (bt->tune_sig == sig && bt->tune_m > 0) {
        c.M = bt->tune_m;
        c.W = bt->tune_w;
        c.shape = bt->tune_shape;
        c.tc = bt->tune_tc != 0;
        if (bt->tune_wave) c.flags |= PIC_FLAG_WAVE;
        return PIC_OK;
    }
    const int max_t = bt->max_t > 0 ? bt->max_t : 1;
    auto trial = [&](int M, int W, int shape, bool tc, bool wv, float* ms) -> pic_status {
        CallCfg t = c;
        t.M = M;
        t.W = W;
        t.shape = shape;
        t.tc = tc;
        if (wv) t.flags |= PIC_FLAG_WAVE;
        t.iters_cap = (M < max_t ? M : max_t) + 1;
        t.trace = false;
        pic_status s = run_picard(I, t, false, st);
        if (s != PIC_OK) return s;
        BCU(cudaStreamSynchronize(st));
        const Ctrl* hc = reinterpret_cast<const Ctrl*>(bt->h_out);
        if (hc->err) return fail((pic_status)hc->err, "autotuner trial M=%d W=%d shape=%d: device wait "
                                 "exceeded the timeout", M, W, shape);
        BCU(cudaEventElapsedTime(ms, I.ev[1], I.ev[2]));
        return PIC_OK;
    };
    // the wave kernel (one run per unit, one CTA shape, no tiles): forced by
    // PIC_FLAG_WAVE, excluded by PIC_FLAG_NO_WAVE, otherwise a tuning choice
    const bool wave_ok = c.has_mlp && wave_applies(&I) && !(c.flags & PIC_FLAG_NO_WAVE);
    const bool wave_forced = wave_ok && (c.flags & PIC_FLAG_WAVE);
    const int w_def = c.has_mlp ? kSegWindowMlp : kSegWindow;
    // tensor-core tiles are a tuning choice unless a flag fixes them
    const bool tc_free = !wave_forced && c.has_mlp && I.N <= 64 &&
                         !(c.flags & (PIC_FLAG_TC | PIC_FLAG_NO_TC));
    bool bestT = c.tc, bestWave = false;
    int bestM = 0, bestW = w_def, bestS = kDefaultShape;
    float best = 3.4e38f;
    for (int M = 4; M <= 1024 && !wave_forced; M *= 2) {
        if (M > 4 && M / 2 >= max_t) break;  // larger M only repeats min(M, T_b) = T_b
        for (int tcv = 0; tcv < (tc_free ? 2 : 1); ++tcv) {
            const bool tc = tc_free ? tcv == 1 : c.tc;
            float ms;
            pic_status s = trial(M, w_def, kDefaultShape, tc, false, &ms);
            if (s != PIC_OK) return s;
            if (ms < best) { best = ms; bestM = M; bestT = tc; }
        }
    }
    for (int sh = 0; sh < kNumShapes && !wave_forced; ++sh) {
        if (sh == kDefaultShape) continue;
        float ms;
        pic_status s = trial(bestM, w_def, sh, bestT, false, &ms);
        if (s != PIC_OK) return s;
        if (ms < best) { best = ms; bestS = sh; }
    }
    const int wins_mlp[] = {4, 16, 32}, wins_int[] = {16, 32, 128};
    for (int i = 0; i < 3 && !wave_forced; ++i) {
        const int W = c.has_mlp ? wins_mlp[i] : wins_int[i];
        float ms;
        pic_status s = trial(bestM, W, bestS, bestT, false, &ms);
        if (s != PIC_OK) return s;
        if (ms < best) { best = ms; bestW = W; }
    }
    if (wave_ok) {
        for (int M = 4; M <= 4096; M *= 4) {
            if (M > 4 && M / 4 >= max_t) break;
            float ms;
            pic_status s = trial(M, 1, kDefaultShape, bestT, true, &ms);
            if (s != PIC_OK) return s;
            if (ms < best) { best = ms; bestM = M; bestW = 1; bestWave = true; }
        }
    }
    bt->tune_sig = sig;
    bt->tune_m = bestM;
    bt->tune_w = bestW;
    bt->tune_shape = bestS;
    bt->tune_tc = bestT ? 1 : 0;
    bt->tune_wave = bestWave ? 1 : 0;
    c.M = bestM;
    c.W = bestW;
    c.shape = bestS;
    c.tc = bestT;
    if (bestWave) c.flags |= PIC_FLAG_WAVE;
    return PIC_OK;
}

pic_status create_fail(pic_instance* h, pic_status s) {
    free_instance(h->I);
    delete h;
    return s;
}

// Copy every trajectory's inputs into the combined arrays (orders at toff[b],
// products at koff[b], regions at roff[b]; lam rows of trajectories without lam
// zero), shift its local product and region ids into its ranges, and check the
// ranges (ids, x0 >= 0, |cost|, |lam|, |cost - lam| < 2^23).  The descriptors'
// shapes must match the batch's.  Synchronises the stream.
pic_status load_inputs(Instance& I, const pic_instance_desc* descs, cudaStream_t st) {
    Batch* bt = I.batch;
    const int B = bt->B;
    const size_t N = I.N;
    int* bad = &I.ctrl->pad0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    for (int b = 0; b < B && !e; ++b) {
        const pic_instance_desc* d = descs + b;
        const cudaMemcpyKind kind = d->mem == PIC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        const size_t t0 = bt->h_toff[b], k0 = bt->h_koff[b], r0 = bt->h_roff[b];
        if (d->T) {
            e = cudaMemcpyAsync(I.prod + t0, d->prod, sizeof(int32_t) * d->T, kind, st);
            if (!e) e = cudaMemcpyAsync(I.reg + t0, d->reg, sizeof(int32_t) * d->T, kind, st);
        }
        if (!e) e = cudaMemcpyAsync(I.x0 + k0 * N, d->x0, sizeof(int32_t) * d->K * N, kind, st);
        if (!e) e = cudaMemcpyAsync(I.cost + r0 * N, d->cost, sizeof(int32_t) * d->R * N, kind, st);
        if (!e && I.has_lam) {
            e = d->lam ? cudaMemcpyAsync(I.lam + k0 * N, d->lam, sizeof(int32_t) * d->K * N, kind, st)
                       : cudaMemsetAsync(I.lam + k0 * N, 0, sizeof(int32_t) * d->K * N, st);
        }
    }
    if (e) return cuda_fail(e, "input copy", __LINE__);
    k_batch_ids<<<4 * I.num_sms, 256, 0, st>>>(I.T, B, bt->toff, bt->koff, bt->roff, I.prod, I.reg, bad);
    e = cudaGetLastError();
    int hb_ids = 0;
    if (!e) e = cudaMemcpyAsync(&hb_ids, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    // range checks of x0, cost, lam on the combined arrays (ids were checked above)
    if (!e) e = launch_validate(I, st);
    int hb = 0;
    if (!e) e = cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return cuda_fail(e, "validation", __LINE__);
    hb |= hb_ids;
    if (hb & 1) return fail(PIC_ERR_INVALID_ARG, "a trajectory has prod[t] outside [0, K)");
    if (hb & 2) return fail(PIC_ERR_INVALID_ARG, "a trajectory has reg[t] outside [0, R)");
    if (hb & 4) return fail(PIC_ERR_INVALID_ARG, "a trajectory's x0 has a negative entry");
    if (hb & (8 | 16 | 32))
        return fail(PIC_ERR_INVALID_ARG,
                    "|cost|, |lam| or |cost - lam| not below 2^23 (cost - lam is checked "
                    "over all trajectories' rows together)");
    return PIC_OK;
}

}  // namespace

namespace pic {
pic_status batch_tables(Instance& I, int M, int W, cudaStream_t st) {
    if (I.batch->invalid)
        return fail(PIC_ERR_INVALID_ARG, "the batch's last pic_batch_load failed: load valid inputs first");
    return ensure_tables(I, M, W, st);
}
}  // namespace pic

extern "C" {

pic_status pic_create_batch(const pic_instance_desc* descs, int32_t B, pic_instance** out) {
    clear_error();
    if (!out) return fail(PIC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || B < 1) return fail(PIC_ERR_INVALID_ARG, "descs is NULL or B < 1");
    long long T = 0, K = 0, R = 0;
    bool any_lam = false;
    const int N = descs[0].N;
    for (int b = 0; b < B; ++b) {
        const pic_instance_desc* d = descs + b;
        if (!desc_ok(d))
            return fail(PIC_ERR_INVALID_ARG, "trajectory %d: invalid descriptor (sizes, pointers or mem)", b);
        if (d->N != N) return fail(PIC_ERR_INVALID_ARG, "trajectory %d: N = %d differs from N = %d", b, d->N, N);
        if (d->cap) return fail(PIC_ERR_UNSUPPORTED, "trajectory %d: node capacity is not supported in a batch", b);
        T += d->T;
        K += d->K;
        R += d->R;
        any_lam |= d->lam != nullptr;
    }
    const long long lim = 0x7FFFFFFEll;
    if (T > lim || K > lim || R > lim)
        return fail(PIC_ERR_INVALID_ARG, "batch totals T=%lld K=%lld R=%lld must each stay below 2^31", T, K, R);
    pic_instance* h = new (std::nothrow) pic_instance();
    if (!h) return fail(PIC_ERR_OOM, "host allocation failed");
    Instance& I = h->I;
    memset(&I, 0, sizeof(I));
    Batch* bt = new (std::nothrow) Batch();
    if (!bt) {
        delete h;
        return fail(PIC_ERR_OOM, "host allocation failed");
    }
    memset(bt, 0, sizeof(Batch));
    I.batch = bt;
    bt->B = B;
    bt->h_toff = new (std::nothrow) int64_t[B + 1];
    bt->h_koff = new (std::nothrow) int64_t[B + 1];
    bt->h_roff = new (std::nothrow) int64_t[B + 1];
    bt->h_has_lam = new (std::nothrow) int8_t[B];
    if (!bt->h_toff || !bt->h_koff || !bt->h_roff || !bt->h_has_lam)
        return create_fail(h, fail(PIC_ERR_OOM, "host allocation failed"));
    bt->h_toff[0] = bt->h_koff[0] = bt->h_roff[0] = 0;
    for (int b = 0; b < B; ++b) {
        bt->h_toff[b + 1] = bt->h_toff[b] + descs[b].T;
        bt->h_koff[b + 1] = bt->h_koff[b] + descs[b].K;
        bt->h_roff[b + 1] = bt->h_roff[b] + descs[b].R;
        bt->h_has_lam[b] = descs[b].lam != nullptr;
        if (descs[b].T > bt->max_t) bt->max_t = descs[b].T;
    }
    cudaError_t e = alloc_instance(I, (int)T, N, (int)K, (int)R, any_lam);
    auto dm = [&](auto** p, size_t n) {
        if (!e) e = cudaMalloc((void**)p, sizeof(**p) * (n ? n : 1));
    };
    dm(&bt->toff, B + 1);
    dm(&bt->koff, B + 1);
    dm(&bt->roff, B + 1);
    dm(&bt->traj_of_prod, (size_t)K);
    dm(&bt->reg_local, (size_t)R);
    dm(&bt->chunk_len, B);
    dm(&bt->pol, B);
    dm(&bt->last_chg, B);
    dm(&bt->tres, 2 * (size_t)B);
    if (!e) e = cudaMallocHost((void**)&bt->h_pol, sizeof(BatchPol) * B);
    if (!e) e = cudaMallocHost((void**)&bt->h_out, out_bytes(B));
    if (e) return create_fail(h, cuda_fail(e, "allocation", __LINE__));
    cudaStream_t st = (cudaStream_t)descs[0].stream;
    std::vector<int32_t> off(3 * (size_t)(B + 1));
    for (int b = 0; b <= B; ++b) {
        off[b] = (int32_t)bt->h_toff[b];
        off[B + 1 + b] = (int32_t)bt->h_koff[b];
        off[2 * (B + 1) + b] = (int32_t)bt->h_roff[b];
    }
    e = cudaMemsetAsync(I.ctrl, 0, sizeof(Ctrl), st);
    if (!e) e = cudaMemcpyAsync(bt->toff, off.data(), sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(bt->koff, off.data() + B + 1, sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(bt->roff, off.data() + 2 * (B + 1), sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, st);
    if (e) return create_fail(h, cuda_fail(e, "offset copy", __LINE__));
    const int grid = 4 * I.num_sms;
    k_owners<<<grid, 256, 0, st>>>((int)K, B, bt->koff, bt->traj_of_prod, nullptr);
    k_owners<<<grid, 256, 0, st>>>((int)R, B, bt->roff, nullptr, bt->reg_local);
    if ((e = cudaGetLastError())) return create_fail(h, cuda_fail(e, "owner tables", __LINE__));
    const pic_status ls = load_inputs(I, descs, st);
    if (ls != PIC_OK) return create_fail(h, ls);
    I.cost16 = 0;  // the combined cost table is read from global memory
    *out = h;
    return PIC_OK;
}

pic_status pic_batch_load(pic_instance* h, const pic_instance_desc* descs, int32_t B) {
    clear_error();
    if (!h || !h->I.batch) return fail(PIC_ERR_INVALID_ARG, "not a batch instance (use pic_create_batch)");
    Instance& I = h->I;
    Batch* bt = I.batch;
    if (!descs || B != bt->B) return fail(PIC_ERR_INVALID_ARG, "descs is NULL or B differs from the batch's %d", bt->B);
    for (int b = 0; b < B; ++b) {
        const pic_instance_desc* d = descs + b;
        if (!desc_ok(d))
            return fail(PIC_ERR_INVALID_ARG, "trajectory %d: invalid descriptor (sizes, pointers or mem)", b);
        if (d->cap) return fail(PIC_ERR_UNSUPPORTED, "trajectory %d: node capacity is not supported in a batch", b);
        if (d->N != I.N || d->T != bt->h_toff[b + 1] - bt->h_toff[b] || d->K != bt->h_koff[b + 1] - bt->h_koff[b] ||
            d->R != bt->h_roff[b + 1] - bt->h_roff[b] || (d->lam != nullptr) != (bt->h_has_lam[b] != 0))
            return fail(PIC_ERR_INVALID_ARG, "trajectory %d: shape (T, N, K, R, lam) differs from the batch's", b);
    }
    // the order tables and the captured per-call graph describe the old inputs
    I.tables_m = 0;
    I.tables_w = 0;
    if (bt->gexec) {
        cudaGraphExecDestroy(bt->gexec);
        bt->gexec = nullptr;
        bt->gsig = 0;
    }
    bt->invalid = 1;
    const pic_status s = load_inputs(I, descs, (cudaStream_t)descs[0].stream);
    if (s == PIC_OK) bt->invalid = 0;
    return s;
}

pic_status pic_simulate_batch(pic_instance* h, const pic_policy* pols, const pic_sim_opts* opts,
                              int8_t* actions_out, int32_t* final_stock, pic_traj_result* traj,
                              pic_sim_result* res) {
    clear_error();
    if (!h || !h->I.batch) return fail(PIC_ERR_INVALID_ARG, "not a batch instance (use pic_create_batch)");
    Instance& I = h->I;
    Batch* bt = I.batch;
    const int B = bt->B;
    if (bt->invalid)
        return fail(PIC_ERR_INVALID_ARG, "the batch's last pic_batch_load failed: load valid inputs first");
    if (!pols || !opts || (!actions_out && I.T > 0))
        return fail(PIC_ERR_INVALID_ARG, "pols, opts and actions_out are required");
    if (opts->mode == PIC_MODE_PICARD_PRODUCTS || opts->mode == PIC_MODE_PICARD_ASSIGNED)
        return fail(PIC_ERR_UNSUPPORTED, "batches: PIC_MODE_PICARD or PIC_MODE_SEQUENTIAL only");
    if (opts->mode != PIC_MODE_PICARD && opts->mode != PIC_MODE_SEQUENTIAL)
        return fail(PIC_ERR_INVALID_ARG, "unknown mode %d", opts->mode);
    if (opts->out_mem != PIC_MEM_HOST && opts->out_mem != PIC_MEM_DEVICE)
        return fail(PIC_ERR_INVALID_ARG, "unknown out_mem %d", opts->out_mem);
    if (opts->num_chunks < 0 || opts->max_iters < 0 || opts->seg_window < 0)
        return fail(PIC_ERR_INVALID_ARG, "negative num_chunks, max_iters or seg_window");
    if (opts->max_steps != 0)
        return fail(PIC_ERR_UNSUPPORTED, "the max_steps window is for single instances (pic_simulate)");
    if (opts->flags & PIC_FLAG_GROUP_KERNEL)
        return fail(PIC_ERR_UNSUPPORTED, "PIC_FLAG_GROUP_KERNEL applies to pic_simulate only");
    CallCfg c;
    memset(&c, 0, sizeof(c));
    const pic_policy* first_mlp = nullptr;
    for (int b = 0; b < B; ++b) {
        const pic_policy& p = pols[b];
        if (p.kind < PIC_POLICY_GREEDY || p.kind > PIC_POLICY_GUMBEL)
            return fail(PIC_ERR_INVALID_ARG, "trajectory %d: unknown policy kind %d", b, p.kind);
        if (p.kind == PIC_POLICY_DUAL && !bt->h_has_lam[b])
            return fail(PIC_ERR_INVALID_ARG, "trajectory %d: bid-price policy needs lam", b);
        if (p.kind >= PIC_POLICY_MLP) {
            if (p.hidden != kHidden)
                return fail(PIC_ERR_UNSUPPORTED, "trajectory %d: MLP hidden width must be %d", b, kHidden);
            if (!p.W1 || !p.b1 || !p.W2 || !p.b2 || !p.E)
                return fail(PIC_ERR_INVALID_ARG, "trajectory %d: MLP policy needs W1, b1, W2, b2, E", b);
            if (!first_mlp) {
                first_mlp = &p;
            } else if (p.W1 != first_mlp->W1 || p.b1 != first_mlp->b1 || p.W2 != first_mlp->W2 ||
                       p.b2 != first_mlp->b2 || p.E != first_mlp->E) {
                return fail(PIC_ERR_UNSUPPORTED,
                            "trajectory %d: all MLP policies of a batch call must share one weight set", b);
            }
        }
        bt->h_pol[b].kind = p.kind;
        bt->h_pol[b].traj = p.traj;
        bt->h_pol[b].seed = p.seed;
    }
    c.has_mlp = first_mlp != nullptr;
    if (first_mlp) c.mlp = *first_mlp;
    cudaStream_t st = (cudaStream_t)opts->stream;
    const bool host_out = opts->out_mem == PIC_MEM_HOST;
    const cudaMemcpyKind okind = host_out ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const bool timing = (opts->flags & PIC_FLAG_TIMING) != 0;
    const size_t T = I.T, K = I.K, N = I.N;
    I.launches = 0;
    I.ran_wave = 0;
    if (c.has_mlp) BCU(mlp_alloc(&I));
    int32_t* stock_src = I.xfin;
    if (timing) BCU(cudaEventRecord(I.ev[0], st));
    if (opts->mode == PIC_MODE_SEQUENTIAL) {
        stock_src = I.xwork;
        BCU(cudaMemcpyAsync(bt->pol, bt->h_pol, sizeof(BatchPol) * B, cudaMemcpyHostToDevice, st));
        BCU(cudaMemsetAsync(I.ctrl, 0, offsetof(Ctrl, nruns), st));
        BCU(cudaMemcpyAsync(I.xwork, I.x0, sizeof(int32_t) * K * N, cudaMemcpyDeviceToDevice, st));
        pic_policy mp = c.mlp;
        mp.kind = PIC_POLICY_MLP;
        if (c.has_mlp) BCU(mlp_prepare(&I, &mp, st));
        BCU(cudaEventRecord(I.ev[1], st));
        const MlpPolicy p = make_policy_view(&I, &mp, opts->flags);
        const int npl = (I.N + 31) / 32;
        if (T) {
            if (npl == 1) BCU(launch_seq_batch<1>(&I, p, c.has_mlp, st));
            else if (npl == 2) BCU(launch_seq_batch<2>(&I, p, c.has_mlp, st));
            else BCU(launch_seq_batch<4>(&I, p, c.has_mlp, st));
        }
        BCU(cudaEventRecord(I.ev[2], st));
        I.launches += 1;
        BCU(traj_reduce(I, B, st));
        unsigned char* ho = bt->h_out;
        BCU(cudaMemcpyAsync(ho, I.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        BCU(cudaMemcpyAsync(ho + sizeof(Ctrl), bt->tres, sizeof(long long) * 2 * B, cudaMemcpyDeviceToHost, st));
        BCU(cudaMemsetAsync(bt->last_chg, 0, sizeof(int32_t) * B, st));
        BCU(cudaMemcpyAsync(ho + sizeof(Ctrl) + sizeof(long long) * 2 * B, bt->last_chg,
                            sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st));
    } else {
        c.flags = opts->flags & ~(PIC_FLAG_TIMING | PIC_FLAG_GRAPH | PIC_FLAG_REUSE_TABLES);
        c.tc = (opts->flags & PIC_FLAG_NO_TC) == 0 && I.N <= 64;
        c.alpha_init = opts->alpha_init;
        c.trace = opts->trace && opts->trace_cap > 0;
        c.timeout_ns = opts->timeout_ns ? opts->timeout_ns : 60000000000ull;
        c.shape = kDefaultShape;
        c.W = opts->seg_window ? opts->seg_window : (c.has_mlp ? kSegWindowMlp : kSegWindow);
        if (c.has_mlp && (c.flags & PIC_FLAG_WAVE) && wave_applies(&I)) c.W = 1;  // one run per unit
        if (opts->num_chunks) {
            c.M = opts->num_chunks;
        } else {
            pic_status s = autotune(I, c, st);
            if (s != PIC_OK) return s;
            if (opts->seg_window && !(c.flags & PIC_FLAG_WAVE)) c.W = opts->seg_window;
        }
        const int maxM = c.M < bt->max_t ? c.M : (bt->max_t > 0 ? bt->max_t : 1);
        c.iters_cap = opts->max_iters ? opts->max_iters : maxM + 1;
        pic_status s = run_picard(I, c, (opts->flags & PIC_FLAG_GRAPH) != 0, st);
        if (s != PIC_OK) return s;
    }
    if (T) BCU(cudaMemcpyAsync(actions_out, I.act_t, T, okind, st));
    if (final_stock) BCU(cudaMemcpyAsync(final_stock, stock_src, sizeof(int32_t) * K * N, okind, st));
    if (timing) BCU(cudaEventRecord(I.ev[3], st));
    BCU(cudaStreamSynchronize(st));
    Ctrl hc;
    memcpy(&hc, bt->h_out, sizeof(Ctrl));
    const long long* tres = reinterpret_cast<const long long*>(bt->h_out + sizeof(Ctrl));
    const int32_t* last = reinterpret_cast<const int32_t*>(bt->h_out + sizeof(Ctrl) + sizeof(long long) * 2 * B);
    const bool picard = opts->mode == PIC_MODE_PICARD;
    if (hc.pad0 & 64) return fail(PIC_ERR_INVALID_ARG, "alpha_init holds a value outside [-1, N)");
    if (hc.err) return fail((pic_status)hc.err, "device wait exceeded timeout (%llu ns)",
                            (unsigned long long)c.timeout_ns);
    const int passes = (picard && T) ? hc.iters : 1;
    if (picard && T && c.trace) {
        int rows = passes < opts->trace_cap ? passes : opts->trace_cap;
        if (rows > kTraceCap) rows = kTraceCap;
        if (rows > 0)
            BCU(cudaMemcpy(opts->trace, I.trace, sizeof(long long) * kTraceCols * rows, cudaMemcpyDeviceToHost));
    }
    if (traj) {
        for (int b = 0; b < B; ++b) {
            traj[b].total_cost = tres[2 * b];
            traj[b].lost = tres[2 * b + 1];
            if (!picard || !T) {
                traj[b].iters = 1;
                traj[b].converged = 1;
            } else {
                // a trajectory whose last change came in the final pass run, without
                // a global fixed point, has not been confirmed
                const bool conf = hc.converged || last[b] < passes;
                traj[b].iters = conf ? last[b] + 1 : passes;
                traj[b].converged = conf ? 1 : 0;
            }
        }
    }
    if (res) {
        res->total_cost = hc.total_cost;
        res->lost = hc.lost;
        res->policy_calls = picard ? (int64_t)hc.policy_calls : (int64_t)T;
        res->iters = passes;
        res->num_chunks = picard ? c.M : 1;
        res->rescored = (int64_t)hc.rescored;
        res->seg_replays = (int64_t)hc.seg_replays;
        res->launches = I.launches;
        res->mlp_calls = picard ? (int64_t)hc.mlp_calls : 0;
        res->tc_decisions = picard ? (int64_t)hc.tc_rows : 0;
        res->sat_decisions = (int64_t)hc.sat_rows;
        res->near_ties = (int64_t)hc.near_ties;
        res->wave = I.ran_wave;
        if (!picard)
            for (int b = 0; b < B; ++b)
                if (bt->h_pol[b].kind >= PIC_POLICY_MLP) res->mlp_calls += bt->h_toff[b + 1] - bt->h_toff[b];
        res->seg_window = picard ? c.W : 0;
        res->cta_threads = picard ? I.cta_threads : 32 * kSeqWarps;
        res->ctas_per_sm = picard ? I.ctas_per_sm : 0;
        res->prep_ms = res->sim_ms = res->total_ms = 0.0f;
        if (timing) {
            BCU(cudaEventElapsedTime(&res->prep_ms, I.ev[0], I.ev[1]));
            BCU(cudaEventElapsedTime(&res->sim_ms, I.ev[1], I.ev[2]));
            BCU(cudaEventElapsedTime(&res->total_ms, I.ev[0], I.ev[3]));
        }
    }
    if (picard && T && !hc.converged)
        return fail(PIC_ERR_NOT_CONVERGED, "no fixed point within %d passes", c.iters_cap);
    return PIC_OK;
}

}  // extern "C"
