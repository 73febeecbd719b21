// MLP policies (Sec. 4.1: an MLP scores the warehouses; the order goes to the
// best-scoring warehouse that holds stock) in a fixed FP32 operation order, and
// their Gumbel-max sampling variant.
//
// Score of warehouse n for an order of product k in region r with stock row S:
//   h_j = b1_j, then one fmaf per input: cost[r][n]/128 (n = 0..N-1), E[r][e]
//         (e = 0..15), min(S_n, 32)/32 (n = 0..N-1), weights W1 rows in that
//         input's position; h_j = max(h_j, 0);
//   s_n = b2_n, then one fmaf per hidden unit j = 0..255 with W2[j][n].
// Parameters are BF16 (exact in FP32).  The part of the h chain before the stock
// inputs depends only on the region, so it is evaluated once per call into
// P[r][j] (the same operations in the same order).  Argmax over stocked
// warehouses, ties to the lowest index; a^phi when nothing is stocked.
//
// Gumbel: s_n + g_n with g_n = -log(-log u), u = ((w >> 9) + 1/2) 2^-23 from
// Philox4x32-10 (Salmon et al., SC'11) with key = seed and counter = (t,
// trajectory, n / 4, 0), word n mod 4; log from IEEE operations only (x = m 2^e,
// log m = 2 atanh((m-1)/(m+1)) by its series to the 11th power, ln 2 split in
// two).  All floating-point steps use explicit round-to-nearest intrinsics so
// that no contraction changes the bits.
#include "pic_picard.cuh"

namespace pic {

namespace {

using namespace picard;

__device__ __forceinline__ float bf16f(uint16_t b) { return __uint_as_float((unsigned)b << 16); }

// ---------------------------------------------------------------- Philox / log / Gumbel
__device__ __forceinline__ void philox_round(unsigned c[4], unsigned k0, unsigned k1) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const unsigned n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

__device__ __forceinline__ void philox4x32_10(unsigned c[4], unsigned k0, unsigned k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        philox_round(c, k0, k1);
    }
}

__device__ __forceinline__ float ieee_log(float x) {
    const unsigned bits = __float_as_uint(x);
    int e = (int)((bits >> 23) & 0xFF) - 127;
    float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
    if (m > 1.41421356f) { m = __fmul_rn(m, 0.5f); e += 1; }
    const float f = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float f2 = __fmul_rn(f, f);
    float p = 0.09090909090909091f;
    p = fmaf(p, f2, 0.1111111111111111f);
    p = fmaf(p, f2, 0.14285714285714285f);
    p = fmaf(p, f2, 0.2f);
    p = fmaf(p, f2, 0.3333333333333333f);
    const float twof = __fmul_rn(2.0f, f);
    const float r = __fmul_rn(twof, f2);
    const float lm = fmaf(r, p, twof);
    const float ef = (float)e;
    return fmaf(ef, 0.693145751953125f, fmaf(ef, 1.4286068e-06f, lm));
}

// Gumbel noise for warehouses 4q .. 4q+3 of order t (one Philox block).
__device__ __forceinline__ void gumbel4(unsigned long long seed, int traj, int t, int q, float g[4]) {
    unsigned c[4] = {(unsigned)t, (unsigned)traj, (unsigned)q, 0u};
    philox4x32_10(c, (unsigned)seed, (unsigned)(seed >> 32));
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float u = __fmul_rn(__fadd_rn((float)(c[i] >> 9), 0.5f), 1.1920928955078125e-7f);
        g[i] = -ieee_log(-ieee_log(u));
    }
}

__device__ __forceinline__ float gumbel1(unsigned long long seed, int traj, int t, int n) {
    float g[4];
    gumbel4(seed, traj, t, n >> 2, g);
    return g[n & 3];
}

// monotone map of a float (not NaN) to unsigned; -0 is folded onto +0 first
__device__ __forceinline__ unsigned ord_key(float v) {
    const unsigned b = __float_as_uint(__fadd_rn(v, 0.0f));
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// ---------------------------------------------------------------- parameter preparation
struct MlpArgs {
    int N, R, H;
    const uint16_t *W1, *b1, *W2, *b2, *E;
    const int32_t* cost;
    float* P;     // [R][H] chain prefix before the stock inputs
    float* W1s;   // [N][H] stock rows of W1
    float* W2f;   // [H][N]
    float* b2f;   // [N]
};

__global__ void k_mlp_prefix(MlpArgs m) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int H = m.H, N = m.N;
    if (idx < m.R * H) {
        const int r = idx / H, j = idx - r * H;
        float a = bf16f(m.b1[j]);
        for (int n = 0; n < N; ++n)
            a = fmaf(bf16f(m.W1[(size_t)n * H + j]), __fdiv_rn((float)m.cost[(size_t)r * N + n], 128.0f), a);
        for (int e = 0; e < kEmb; ++e)
            a = fmaf(bf16f(m.W1[(size_t)(2 * N + e) * H + j]), bf16f(m.E[(size_t)r * kEmb + e]), a);
        m.P[idx] = a;
    }
    if (idx < N * H) {
        const int n = idx / H, j = idx - n * H;
        m.W1s[idx] = bf16f(m.W1[(size_t)(N + n) * H + j]);
        m.W2f[(size_t)j * N + n] = bf16f(m.W2[(size_t)j * N + n]);
    }
    if (idx < N) m.b2f[idx] = bf16f(m.b2[idx]);
}

// ---------------------------------------------------------------- one decision, one warp
struct MlpPolicy {
    int N, H;
    const float* __restrict__ P;
    const float* __restrict__ W1s;
    const float* __restrict__ W2f;
    const float* __restrict__ b2f;
    bool gumbel;
    unsigned long long seed;
    int traj;
};

// The warp evaluates the policy for stock row S (lane l holds warehouses l + 32 i)
// of an order in region r at time t; fs/hs: per-warp shared scratch (N and H
// floats).  Returns the action (warp-uniform).
template <bool SMEMW>
__device__ __forceinline__ float wld(const float* p) {
    if (SMEMW) return *p;  // shared-memory copy of the weights
    return __ldg(p);
}

template <int NPL, bool SMEMW>
__device__ __forceinline__ int mlp_decide(const MlpPolicy& p, const float* W1s, const float* W2f,
                                          const int S[NPL], int r, int t, float* fs, float* hs) {
    const int lane = lane_id();
    const int N = p.N, H = p.H;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        if (n < N) fs[n] = __fdiv_rn((float)min(S[i], 32), 32.0f);
    }
    __syncwarp();
    constexpr int kJ = kHidden / 32;  // hidden units per lane, advanced together
    float acc[kJ];
#pragma unroll
    for (int u = 0; u < kJ; ++u) acc[u] = __ldg(p.P + (size_t)r * H + lane + 32 * u);
#pragma unroll 2
    for (int n = 0; n < N; ++n) {
        const float f = fs[n];
        const float* w = W1s + (size_t)n * H + lane;
#pragma unroll
        for (int u = 0; u < kJ; ++u) acc[u] = fmaf(wld<SMEMW>(w + 32 * u), f, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kJ; ++u) hs[lane + 32 * u] = acc[u] > 0.0f ? acc[u] : 0.0f;
    __syncwarp();
    unsigned best_key = 0;
    int best_n = INT_MAX;
    bool any = false;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        if (n < N && S[i] > 0) {
            float s = __ldg(p.b2f + n);
#pragma unroll 8
            for (int j = 0; j < H; ++j) s = fmaf(wld<SMEMW>(W2f + (size_t)j * N + n), hs[j], s);
            if (p.gumbel) s = __fadd_rn(s, gumbel1(p.seed, p.traj, t, n));
            const unsigned kk = ord_key(s);
            if (!any || kk > best_key) { best_key = kk; best_n = n; any = true; }
        }
    }
    __syncwarp();  // fs / hs reused by the next call
    const unsigned kmax = __reduce_max_sync(kFull, any ? best_key : 0u);
    const bool stocked = __any_sync(kFull, any);
    const int n = __reduce_min_sync(kFull, (any && best_key == kmax) ? best_n : INT_MAX);
    return stocked ? n : -1;
}

// Copy the FP32 weights (W1 stock rows, then W2) into shared memory.
__device__ __forceinline__ void stage_weights(const MlpPolicy& p, float* sw) {
    const int n = 2 * p.N * p.H;
    const float* src0 = p.W1s;
    const float* src1 = p.W2f;
    const int half = p.N * p.H;
    for (int i = threadIdx.x; i < n; i += blockDim.x) sw[i] = i < half ? src0[i] : src1[i - half];
    __syncthreads();
}

// ---------------------------------------------------------------- sequential simulator
template <int NPL, bool SMEMW>
__global__ void __launch_bounds__(32) k_seq_mlp(int T, int N, const int32_t* __restrict__ prod,
                                                const int32_t* __restrict__ reg, int32_t* xw,
                                                int8_t* __restrict__ act_t, MlpPolicy p, Ctrl* ctrl) {
    __shared__ float fs[128];
    __shared__ float hs[kHidden];
    extern __shared__ float s_w[];
    if (SMEMW) stage_weights(p, s_w);
    const float* W1s = SMEMW ? s_w : p.W1s;
    const float* W2f = SMEMW ? s_w + (size_t)p.N * p.H : p.W2f;
    const int lane = lane_id();
    int my_act = -1;
    for (int t = 0; t < T; ++t) {
        const int k = __ldg(prod + t), r = __ldg(reg + t);
        int S[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            S[i] = n < N ? xw[(size_t)k * N + n] : 0;
        }
        const int act = mlp_decide<NPL, SMEMW>(p, W1s, W2f, S, r, t, fs, hs);
#pragma unroll
        for (int i = 0; i < NPL; ++i)
            if (act == lane + 32 * i) xw[(size_t)k * N + act] = S[i] - 1;
        if (lane == (t & 31)) my_act = act;
        if ((t & 31) == 31 || t == T - 1) {
            const int tw = (t & ~31) + lane;
            if (tw < T) act_t[tw] = (int8_t)my_act;
        }
        __syncwarp();
    }
    if (lane == 0) {
        ctrl->iters = 1;
        ctrl->converged = 1;
        ctrl->policy_calls = (unsigned long long)T;
    }
}

// ---------------------------------------------------------------- Picard, one warp per segment
template <int NPL, bool SMEMW>
__device__ bool replay_segment_mlp(const KArgs& a, const MlpPolicy& p, const float* W1s,
                                   const float* W2f, const int32_t* __restrict__ perm, int s,
                                   const SegMeta& m, int fcp, int* fc_cur,
                                   unsigned long long& calls, float* fs, float* hs) {
    const int lane = lane_id();
    const int N = a.N, NP = a.NP;
    const int k = m.k;
    int D[NPL], x0v[NPL], S[NPL], S0[NPL], hist[NPL], corr[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        x0v[i] = n < N ? a.x0[(size_t)k * N + n] : 0;
        D[i] = (m.ce - m.cf > 1) ? a.carry[(size_t)s * NP + n] : 0;
        S[i] = max(0, x0v[i] - D[i]);
        S0[i] = S[i];
        hist[i] = 0;
        corr[i] = 0;
    }
    int r = m.r0;
    int next_run = a.run_start[r + 1];
    bool eval = m.j0 > fcp;
    unsigned long long evals = 0;
    int first_chg = INT_MAX;
    for (int base = m.j0; base < m.jend; base += 32) {
        const int cnt = min(32, m.jend - base);
        const int my_reg = lane < cnt ? a.reg_s[base + lane] : 0;
        const int my_old = lane < cnt ? a.alpha_s[base + lane] : -1;
        const int my_t = lane < cnt ? perm[base + lane] : 0;
        int my_new = my_old;
        for (int q = 0; q < cnt; ++q) {
            if (base + q == next_run) {
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    hist[i] += S0[i] - S[i];
                    D[i] += S0[i] - S[i] + corr[i];
                    corr[i] = 0;
                    S[i] = max(0, x0v[i] - D[i]);
                    S0[i] = S[i];
                }
                eval = next_run > fcp;
                ++r;
                next_run = a.run_start[r + 1];
            }
            const int rr = __shfl_sync(kFull, my_reg, q);
            const int ao = __shfl_sync(kFull, my_old, q);
            const int tt = __shfl_sync(kFull, my_t, q);
            int act = ao;
            if (eval) {
                act = mlp_decide<NPL, SMEMW>(p, W1s, W2f, S, rr, tt, fs, hs);
                ++evals;
            }
#pragma unroll
            for (int i = 0; i < NPL; ++i) S[i] -= (act == lane + 32 * i);
            if (act != ao) {
#pragma unroll
                for (int i = 0; i < NPL; ++i) corr[i] += (ao == lane + 32 * i) - (act == lane + 32 * i);
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
    if (lane == 0 && first_chg != INT_MAX && first_chg < ld_volatile(&fc_cur[k]))
        atomicMin(&fc_cur[k], first_chg);
    if (s == m.ce - 1) {
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            if (n < N) a.xfin[(size_t)k * N + n] = S[i];
        }
    }
    if (lane == 0) calls += evals;
    return first_chg != INT_MAX;
}

constexpr int kMlpThreads = 256;

template <int NPL, bool SMEMW>
__global__ void __launch_bounds__(kMlpThreads, 1) k_picard_mlp(KArgs a, MlpPolicy p,
                                                              const int32_t* __restrict__ perm) {
    extern __shared__ float s_w[];
    if (SMEMW) stage_weights(p, s_w);
    const float* W1s = SMEMW ? s_w : p.W1s;
    const float* W2f = SMEMW ? s_w + (size_t)p.N * p.H : p.W2f;
    __shared__ int s_changed;
    __shared__ SegMeta s_meta[kMlpThreads / 32][32];
    __shared__ int s_fcp[kMlpThreads / 32][32];
    __shared__ float s_fs[kMlpThreads / 32][128];
    __shared__ float s_hs[kMlpThreads / 32][kHidden];
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    const unsigned long long deadline = globaltimer_ns() + a.timeout_ns;
    const int nseg = a.ctrl->nseg;
    const bool no_reset = (a.flags & PIC_FLAG_NO_RESET) != 0;
    if (threadIdx.x == 0) s_changed = 0;
    __syncthreads();
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
        for (int k = gtid; k < a.K; k += gthreads) fc_cur[k] = INT_MAX;
        if (gtid == 0) a.ctrl->changed[parity] = 0;
        if (it > 1 || a.first_dirty) {
            for (int j0 = 0; gwarp + j0 * nwarps < nseg; j0 += 32) {
                const int sl = gwarp + (j0 + lane) * nwarps;
                bool head = false;
                if (sl < nseg) {
                    const SegMeta mm = load_meta(a.meta + sl);
                    head = mm.ce - mm.cf > 1 && (sl - mm.cf) % kSuperBlock == 0;
                    const int f = it > 1 ? fc_prev[mm.k] : -1;
                    if (head && it > 1) head = f != INT_MAX;
                    if (head) {
                        s_meta[wib][lane] = mm;
                        s_fcp[wib][lane] = f;
                    }
                }
                unsigned todo = __ballot_sync(kFull, head);
                while (todo) {
                    const int src = __ffs(todo) - 1;
                    todo &= todo - 1;
                    const SegMeta mm = smem_meta(&s_meta[wib][src]);
                    superblock_prefix<NPL>(a, gwarp + (j0 + src) * nwarps, mm, it, s_fcp[wib][src],
                                           deadline);
                }
                __syncwarp();
            }
        }
        if (!grid_sync(a.ctrl, deadline)) { ok = false; break; }
        if (tr && gtid == 0) tr[0] = (long long)(globaltimer_ns() - t_start);
        bool chg = false;
        for (int j0 = 0; j0 * nwarps < nseg; j0 += 32) {
            const int jj = j0 + lane;
            const int pos = jj * nwarps + ((jj & 1) ? nwarps - 1 - gwarp : gwarp);
            int sl = nseg;
            bool act = false;
            if (pos < nseg) {
                sl = a.lpt[pos];
                const SegMeta mm = load_meta(a.meta + sl);
                const int fcp = no_reset ? -1 : fc_prev[mm.k];
                act = mm.last_start > fcp;
                if (act) {
                    s_meta[wib][lane] = mm;
                    s_fcp[wib][lane] = fcp;
                }
            }
            unsigned todo = __ballot_sync(kFull, act);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const SegMeta mm = smem_meta(&s_meta[wib][src]);
                const int seg = __shfl_sync(kFull, sl, src);
                chg |= replay_segment_mlp<NPL, SMEMW>(a, p, W1s, W2f, perm, seg, mm, s_fcp[wib][src],
                                                      fc_cur, calls, s_fs[wib], s_hs[wib]);
                if (lane == 0) replays += 1;
            }
            __syncwarp();
        }
        if (tr && lane == 0 && replays != replays0) {
            atomicAdd((unsigned long long*)&tr[2], calls - calls0);
            atomicAdd((unsigned long long*)&tr[3], replays - replays0);
        }
        if (__any_sync(kFull, chg) && lane == 0) s_changed = 1;
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

MlpPolicy make_policy_view(const Instance* I, const pic_policy* pol) {
    MlpPolicy p;
    p.N = I->N;
    p.H = kHidden;
    p.P = I->mlp_P;
    p.W1s = I->mlp_W1s;
    p.W2f = I->mlp_W2;
    p.b2f = I->mlp_b2;
    p.gumbel = pol->kind == PIC_POLICY_GUMBEL;
    p.seed = pol->seed;
    p.traj = pol->traj;
    return p;
}

// Weights fit in shared memory next to the kernels' static buffers.
bool smem_weights_ok(int N) { return (size_t)2 * N * kHidden * sizeof(float) <= 180 * 1024; }

template <int NPL, bool SMEMW>
cudaError_t launch_picard_mlp(Instance* I, const KArgs& a, const MlpPolicy& p, cudaStream_t st) {
    auto kern = k_picard_mlp<NPL, SMEMW>;
    const size_t smem = SMEMW ? (size_t)2 * I->N * kHidden * sizeof(float) : 0;
    cudaError_t e;
    if (SMEMW && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kMlpThreads, smem);
    if (e) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int grid = I->num_sms * (occ < 2 ? occ : 2);
    KArgs args = a;
    MlpPolicy pp = p;
    const int32_t* perm = I->perm;
    void* params[] = {&args, &pp, &perm};
    I->launches += 1;
    return cudaLaunchCooperativeKernel((const void*)kern, grid, kMlpThreads, params, smem, st);
}

template <int NPL, bool SMEMW>
cudaError_t launch_seq_mlp(Instance* I, const MlpPolicy& p, cudaStream_t st) {
    auto kern = k_seq_mlp<NPL, SMEMW>;
    const size_t smem = SMEMW ? (size_t)2 * I->N * kHidden * sizeof(float) : 0;
    cudaError_t e;
    if (SMEMW && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    I->launches += 1;
    kern<<<1, 32, smem, st>>>(I->T, I->N, I->prod, I->reg, I->xwork, I->act_t, p, I->ctrl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_prepare(Instance* I, const pic_policy* pol, cudaStream_t st) {
    MlpArgs m;
    m.N = I->N; m.R = I->R; m.H = kHidden;
    m.W1 = pol->W1; m.b1 = pol->b1; m.W2 = pol->W2; m.b2 = pol->b2; m.E = pol->E;
    m.cost = I->cost;
    m.P = I->mlp_P; m.W1s = I->mlp_W1s; m.W2f = I->mlp_W2; m.b2f = I->mlp_b2;
    const int n = I->R * kHidden > I->N * kHidden ? I->R * kHidden : I->N * kHidden;
    I->launches += 1;
    k_mlp_prefix<<<(n + 255) / 256, 256, 0, st>>>(m);
    return cudaGetLastError();
}

cudaError_t sequential_mlp(Instance* I, const pic_policy* pol, cudaStream_t st) {
    const MlpPolicy p = make_policy_view(I, pol);
    const int npl = (I->N + 31) / 32;
    const bool sw = smem_weights_ok(I->N);
    if (npl == 1) return sw ? launch_seq_mlp<1, true>(I, p, st) : launch_seq_mlp<1, false>(I, p, st);
    if (npl == 2) return sw ? launch_seq_mlp<2, true>(I, p, st) : launch_seq_mlp<2, false>(I, p, st);
    return sw ? launch_seq_mlp<4, true>(I, p, st) : launch_seq_mlp<4, false>(I, p, st);
}

cudaError_t picard_mlp(Instance* I, const KArgs& a, const pic_policy* pol, cudaStream_t st) {
    const MlpPolicy p = make_policy_view(I, pol);
    const int npl = (I->N + 31) / 32;
    const bool sw = smem_weights_ok(I->N);
    if (npl == 1) return sw ? launch_picard_mlp<1, true>(I, a, p, st) : launch_picard_mlp<1, false>(I, a, p, st);
    if (npl == 2) return sw ? launch_picard_mlp<2, true>(I, a, p, st) : launch_picard_mlp<2, false>(I, a, p, st);
    return sw ? launch_picard_mlp<4, true>(I, a, p, st) : launch_picard_mlp<4, false>(I, a, p, st);
}

}  // namespace pic
