// Kernels of the MLP and Gumbel-max policies (device code in pic_mlp.cuh).
#include "pic_mlp.cuh"

namespace pic {

namespace {

using namespace picard;
using namespace mlp;

// ---------------------------------------------------------------- parameter preparation
struct MlpArgs {
    int N, R, H;
    const uint16_t *W1, *b1, *W2, *b2, *E;
    const int32_t* cost;
    const int32_t* reg_local;  // region -> row of E (batch instances), or null (identity)
    float* P;     // [R][H] chain prefix before the stock inputs
    uint4* W1p;   // [N][32] packed stock rows of W1 (layout in pic_mlp.cuh)
    uint4* W2p;   // [H/8][N] packed W2
    float* b2f;   // [N]
};

__device__ __forceinline__ unsigned pack2(uint16_t lo, uint16_t hi) {
    return (unsigned)lo | ((unsigned)hi << 16);
}

__global__ void k_mlp_prefix(MlpArgs m) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int H = m.H, N = m.N;
    if (idx < m.R * H) {
        const int r = idx / H, j = idx - r * H;
        const int re = m.reg_local ? m.reg_local[r] : r;
        float a = bf16f(m.b1[j]);
        for (int n = 0; n < N; ++n)
            a = fmaf(bf16f(m.W1[(size_t)n * H + j]), __fdiv_rn((float)m.cost[(size_t)r * N + n], 128.0f), a);
        for (int e = 0; e < kEmb; ++e)
            a = fmaf(bf16f(m.W1[(size_t)(2 * N + e) * H + j]), bf16f(m.E[(size_t)re * kEmb + e]), a);
        m.P[idx] = a;
    }
    if (idx < N * 32) {  // W1p[n * 32 + l]
        const int n = idx >> 5, l = idx & 31;
        const uint16_t* row = m.W1 + (size_t)(N + n) * H;
        m.W1p[idx] = make_uint4(pack2(row[l], row[l + 32]), pack2(row[l + 64], row[l + 96]),
                                pack2(row[l + 128], row[l + 160]), pack2(row[l + 192], row[l + 224]));
    }
    if (idx < (H / 8) * N) {  // W2p[q * N + n]
        const int q = idx / N, n = idx - q * N;
        const uint16_t* c = m.W2 + (size_t)8 * q * N + n;
        m.W2p[idx] = make_uint4(pack2(c[0], c[N]), pack2(c[2 * N], c[3 * N]),
                                pack2(c[4 * N], c[5 * N]), pack2(c[6 * N], c[7 * N]));
    }
    if (idx < N) m.b2f[idx] = bf16f(m.b2[idx]);
}

// Error-bound constants.  c2[n] = sum_j |W2[j][n]| (the fast layer-2 order's
// bound), C1[j] = sum_n |W1s[n][j]| and the scalars bnd = {max_n c2[n],
// max_n |b2[n]|} (one block), then Emax[r] = max_j (|P[r][j]| + C1[j]) (one
// warp per region; the tensor-core tiles' bound).  Sums are rounded up by a
// relative 2^-16 so that they bound the exact values.
__global__ void k_mlp_consts(int N, const uint16_t* __restrict__ W1, const uint16_t* __restrict__ W2,
                             const uint16_t* __restrict__ b2, float* __restrict__ C1,
                             float* __restrict__ bnd, float* __restrict__ c2out) {
    __shared__ float red[2][kHidden];
    const int j = threadIdx.x;  // blockDim = kHidden
    float c1 = 0.f;
    for (int n = 0; n < N; ++n) c1 += fabsf(bf16f(W1[(size_t)(N + n) * kHidden + j]));
    C1[j] = c1 * (1.0f + 1.0f / 65536.0f);
    float c2 = 0.f, bb = 0.f;
    if (j < N) {
        for (int jj = 0; jj < kHidden; ++jj) c2 += fabsf(bf16f(W2[(size_t)jj * N + j]));
        bb = fabsf(bf16f(b2[j]));
        c2out[j] = c2 * (1.0f + 1.0f / 65536.0f);
    }
    red[0][j] = c2;
    red[1][j] = bb;
    __syncthreads();
    for (int o = kHidden / 2; o > 0; o >>= 1) {
        if (j < o) {
            red[0][j] = fmaxf(red[0][j], red[0][j + o]);
            red[1][j] = fmaxf(red[1][j], red[1][j + o]);
        }
        __syncthreads();
    }
    if (j == 0) {
        bnd[0] = red[0][0] * (1.0f + 1.0f / 65536.0f);
        bnd[1] = red[1][0];
    }
}

__global__ void k_mlp_emax(int R, const float* __restrict__ P, const float* __restrict__ C1,
                           float* __restrict__ Emax) {
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = gw; r < R; r += nw) {
        float m = 0.f;
        for (int j = lane; j < kHidden; j += 32) m = fmaxf(m, fabsf(P[(size_t)r * kHidden + j]) + C1[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
        if (lane == 0) Emax[r] = m * (1.0f + 1.0f / 65536.0f);
    }
}

// Scores of the saturated state (every warehouse at 32 units or more, so every
// stock feature is 1) for every region, in the reference order: one warp per
// region runs layer 1 as the scorer does, then each output's single chain.
constexpr int kSatWarps = 8;

template <int NPL>
__global__ void __launch_bounds__(32 * kSatWarps) k_mlp_sat(MlpPolicy p, int R, float* __restrict__ sat) {
    __shared__ float fs[kSatWarps][128];
    __shared__ __align__(16) float hs[kSatWarps][kHidden];
    const int w = threadIdx.x >> 5, lane = lane_id();
    const int r = blockIdx.x * kSatWarps + w;
    if (r >= R) return;
    int S[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) S[i] = 32;
    mlp_hidden<NPL, false>(p, p.W1p, S, r, fs[w], hs[w]);
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        if (n < p.N) sat[(size_t)r * p.N + n] = ref_score<false>(p, p.W2p, hs[w], n);
    }
}

// ---------------------------------------------------------------- sequential simulator
template <int NPL, bool SMEMW, int GROUP = 1>
__global__ void __launch_bounds__(32 * GROUP) k_seq_mlp(int T, int N, const int32_t* __restrict__ prod,
                                                        const int32_t* __restrict__ reg, int32_t* xw,
                                                        int8_t* __restrict__ act_t, MlpPolicy p,
                                                        Ctrl* ctrl) {
    __shared__ float fs[GROUP][128];
    __shared__ __align__(16) float hs[kHidden];
    __shared__ float ht[GROUP > 1 ? 128 : 1];
    __shared__ uint4 am[4];
    extern __shared__ uint4 s_w[];
    if (SMEMW) stage_weights(p, s_w);
    const uint4* W1p = SMEMW ? s_w : p.W1p;
    const uint4* W2p = SMEMW ? s_w + p.N * kHidden / 8 : p.W2p;
    const int w = threadIdx.x >> 5;
    const Group G{w, 1, hs, ht, am};
    MlpCounts mc{0, 0, 0, 0, 0};
    seq_mlp_body<NPL, SMEMW, GROUP>(T, N, prod, reg, xw, act_t, p, W1p, W2p, fs[w], hs, mc, &G);
    if (threadIdx.x == 0) {
        ctrl->iters = 1;
        ctrl->converged = 1;
        ctrl->policy_calls = (unsigned long long)T;
        ctrl->sat_rows = mc.sat;
        ctrl->near_ties = mc.near;
    }
}

constexpr int kMlpThreads = 256;

// GROUP = 4: four warps per segment, sharing each decision (N <= 64, no tiles).
template <int NPL, bool SMEMW, bool SPEC, int GROUP = 1>
__global__ void __launch_bounds__(kMlpThreads, 2) k_picard_mlp(KArgs a, MlpPolicy p,
                                                              const int32_t* __restrict__ perm) {
    constexpr int kWarps = kMlpThreads / 32;
    constexpr int kGroups = kWarps / GROUP;
    extern __shared__ uint4 s_w[];
    __shared__ float s_fs[kWarps][128];
    __shared__ __align__(16) float s_hs[GROUP > 1 ? kGroups : kWarps][kHidden];
    __shared__ float s_ht[kGroups][GROUP > 1 ? 128 : 1];
    __shared__ uint4 s_am[kGroups][4];
    if (SMEMW) stage_weights(p, s_w);
    const uint4* W1p = SMEMW ? s_w : p.W1p;
    const uint4* W2p = SMEMW ? s_w + p.N * kHidden / 8 : p.W2p;
    const int wib = threadIdx.x >> 5;
    const int grp = wib / GROUP;
    const Group G{wib % GROUP, 1 + grp, s_hs[GROUP > 1 ? grp : wib], s_ht[grp], s_am[grp]};
    unsigned long long calls = 0;
    MlpCounts mc{0, 0, 0, 0, 0};
    auto replay = [&](int seg, const SegMeta& m, int fcp, int* fc_cur, int it) {
        const unsigned long long c0 = mc.calls;
        const bool chg = replay_segment_mlp<NPL, SMEMW, SPEC, GROUP>(
            a, p, W1p, W2p, perm, seg, m, fcp, fc_cur, it, 0, mc, s_fs[wib], G.hs, &G);
        calls += mc.calls - c0;
        return chg;
    };
    picard_passes<NPL, kWarps, decltype(replay)&, GROUP>(a, calls, replay);
    if (lane_id() == 0 && (mc.rescored || mc.tc || mc.sat || mc.near)) {
        atomicAdd(&a.ctrl->rescored, mc.rescored);
        atomicAdd(&a.ctrl->tc_rows, mc.tc);
        atomicAdd(&a.ctrl->sat_rows, mc.sat);
        atomicAdd(&a.ctrl->near_ties, mc.near);
    }
}

template <int NPL, bool SMEMW, bool SPEC, int GROUP = 1>
cudaError_t launch_picard_mlp(Instance* I, const KArgs& a, const MlpPolicy& p, cudaStream_t st) {
    auto kern = k_picard_mlp<NPL, SMEMW, SPEC, GROUP>;
    const size_t smem = SMEMW ? packed_weight_bytes(I->N) : 0;
    cudaError_t e;
    if (SMEMW && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kMlpThreads, smem);
    if (e) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int grid = I->num_sms * (occ < 2 ? occ : 2);
    I->coop_blocks = grid;
    I->cta_threads = kMlpThreads;
    I->ctas_per_sm = occ < 2 ? occ : 2;
    KArgs args = a;
    MlpPolicy pp = p;
    const int32_t* perm = I->perm;
    void* params[] = {&args, &pp, &perm};
    I->launches += 1;
    return cudaLaunchCooperativeKernel((const void*)kern, grid, kMlpThreads, params, smem, st);
}

template <int NPL, bool SMEMW, int GROUP = 1>
cudaError_t launch_seq_mlp(Instance* I, const MlpPolicy& p, cudaStream_t st) {
    auto kern = k_seq_mlp<NPL, SMEMW, GROUP>;
    const size_t smem = SMEMW ? packed_weight_bytes(I->N) : 0;
    cudaError_t e;
    if (SMEMW && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    I->launches += 1;
    kern<<<1, 32 * GROUP, smem, st>>>(I->T, I->N, I->prod, I->reg, I->xwork, I->act_t, p, I->ctrl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_alloc(Instance* I) {
    if (I->mlp_P) return cudaSuccess;  // sized once per instance
    cudaError_t e = cudaMalloc((void**)&I->mlp_P, sizeof(float) * (size_t)I->R * kHidden);
    if (!e) e = cudaMalloc((void**)&I->mlp_W1p, sizeof(uint4) * (size_t)I->N * 32);
    if (!e) e = cudaMalloc((void**)&I->mlp_W2p, sizeof(uint4) * (size_t)I->N * (kHidden / 8));
    if (!e) e = cudaMalloc((void**)&I->mlp_b2, sizeof(float) * (size_t)I->N);
    if (!e) e = cudaMalloc((void**)&I->mlp_Emax, sizeof(float) * ((size_t)I->R + kHidden));
    if (!e) e = cudaMalloc((void**)&I->mlp_bnd, sizeof(float) * 2);
    if (!e) e = cudaMalloc((void**)&I->mlp_c2, sizeof(float) * (size_t)I->N);
    if (!e) e = cudaMalloc((void**)&I->mlp_sat, sizeof(float) * (size_t)I->R * I->N);
    return e;
}

cudaError_t mlp_prepare(Instance* I, const pic_policy* pol, cudaStream_t st) {
    MlpArgs m;
    m.N = I->N; m.R = I->R; m.H = kHidden;
    m.W1 = pol->W1; m.b1 = pol->b1; m.W2 = pol->W2; m.b2 = pol->b2; m.E = pol->E;
    m.cost = I->cost;
    m.reg_local = I->batch ? I->batch->reg_local : nullptr;
    m.P = I->mlp_P; m.W1p = I->mlp_W1p; m.W2p = I->mlp_W2p; m.b2f = I->mlp_b2;
    const int n = I->R * kHidden > I->N * kHidden ? I->R * kHidden : I->N * kHidden;
    I->launches += 3;
    k_mlp_prefix<<<(n + 255) / 256, 256, 0, st>>>(m);
    float* C1 = I->mlp_Emax + I->R;  // scratch after the per-region values
    k_mlp_consts<<<1, kHidden, 0, st>>>(I->N, pol->W1, pol->W2, pol->b2, C1, I->mlp_bnd, I->mlp_c2);
    k_mlp_emax<<<(I->R + 7) / 8, 256, 0, st>>>(I->R, I->mlp_P, C1, I->mlp_Emax);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    // the saturated-state score table, by the scorer itself (weights from global memory)
    MlpPolicy p = make_policy_view(I, pol, 0);
    p.sat = nullptr;
    const int npl = (I->N + 31) / 32;
    const int blocks = (I->R + kSatWarps - 1) / kSatWarps;
    I->launches += 1;
    if (npl == 1) k_mlp_sat<1><<<blocks, 32 * kSatWarps, 0, st>>>(p, I->R, I->mlp_sat);
    else if (npl == 2) k_mlp_sat<2><<<blocks, 32 * kSatWarps, 0, st>>>(p, I->R, I->mlp_sat);
    else k_mlp_sat<4><<<blocks, 32 * kSatWarps, 0, st>>>(p, I->R, I->mlp_sat);
    return cudaGetLastError();
}

cudaError_t sequential_mlp(Instance* I, const pic_policy* pol, int flags, cudaStream_t st) {
    const MlpPolicy p = make_policy_view(I, pol, flags);
    const int npl = (I->N + 31) / 32;
    const bool sw = smem_weights_ok(I->N);
    if ((flags & PIC_FLAG_WARP_GROUP) && npl <= 2)  // four warps per decision
        return npl == 1 ? launch_seq_mlp<1, true, 4>(I, p, st) : launch_seq_mlp<2, true, 4>(I, p, st);
    if (npl == 1) return sw ? launch_seq_mlp<1, true>(I, p, st) : launch_seq_mlp<1, false>(I, p, st);
    if (npl == 2) return sw ? launch_seq_mlp<2, true>(I, p, st) : launch_seq_mlp<2, false>(I, p, st);
    return sw ? launch_seq_mlp<4, true>(I, p, st) : launch_seq_mlp<4, false>(I, p, st);
}

cudaError_t picard_wave(Instance* I, const KArgs& a, const MlpPolicy& p, cudaStream_t st);

cudaError_t picard_mlp(Instance* I, const KArgs& a, const pic_policy* pol, cudaStream_t st) {
    const MlpPolicy p = make_policy_view(I, pol, a.flags);
    if ((a.flags & PIC_FLAG_WAVE) && wave_applies(I) && I->tables_w == 1)  // one run per unit
        return picard_wave(I, a, p, st);
    // the packed weights fit in shared memory for every N <= 127; tiles need N <= 64
    const bool tc = (a.flags & PIC_FLAG_NO_TC) == 0 && I->N <= 64;
    const int npl = (I->N + 31) / 32;
    if ((a.flags & PIC_FLAG_WARP_GROUP) && npl <= 2)  // four warps per decision, no tiles
        return npl == 1 ? launch_picard_mlp<1, true, false, 4>(I, a, p, st)
                        : launch_picard_mlp<2, true, false, 4>(I, a, p, st);
    if (npl == 1) return tc ? launch_picard_mlp<1, true, true>(I, a, p, st) : launch_picard_mlp<1, true, false>(I, a, p, st);
    if (npl == 2) return tc ? launch_picard_mlp<2, true, true>(I, a, p, st) : launch_picard_mlp<2, true, false>(I, a, p, st);
    return launch_picard_mlp<4, true, false>(I, a, p, st);
}

}  // namespace pic
