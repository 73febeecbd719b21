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

// ---------------------------------------------------------------- sequential simulator
template <int NPL, bool SMEMW>
__global__ void __launch_bounds__(32) k_seq_mlp(int T, int N, const int32_t* __restrict__ prod,
                                                const int32_t* __restrict__ reg, int32_t* xw,
                                                int8_t* __restrict__ act_t, MlpPolicy p, Ctrl* ctrl) {
    __shared__ float fs[128];
    __shared__ __align__(16) float hs[kHidden];
    extern __shared__ uint4 s_w[];
    if (SMEMW) stage_weights(p, s_w);
    const uint4* W1p = SMEMW ? s_w : p.W1p;
    const uint4* W2p = SMEMW ? s_w + p.N * kHidden / 8 : p.W2p;
    seq_mlp_body<NPL, SMEMW>(T, N, prod, reg, xw, act_t, p, W1p, W2p, fs, hs);
    if (lane_id() == 0) {
        ctrl->iters = 1;
        ctrl->converged = 1;
        ctrl->policy_calls = (unsigned long long)T;
    }
}

constexpr int kMlpThreads = 256;

template <int NPL, bool SMEMW>
__global__ void __launch_bounds__(kMlpThreads, 2) k_picard_mlp(KArgs a, MlpPolicy p,
                                                              const int32_t* __restrict__ perm) {
    extern __shared__ uint4 s_w[];
    __shared__ float s_fs[kMlpThreads / 32][128];
    __shared__ __align__(16) float s_hs[kMlpThreads / 32][kHidden];
    if (SMEMW) stage_weights(p, s_w);
    const uint4* W1p = SMEMW ? s_w : p.W1p;
    const uint4* W2p = SMEMW ? s_w + p.N * kHidden / 8 : p.W2p;
    const int wib = threadIdx.x >> 5;
    unsigned long long calls = 0;
    picard_passes<NPL, kMlpThreads / 32>(
        a, calls, [&](int seg, const SegMeta& m, int fcp, int* fc_cur, int it) {
            return replay_segment_mlp<NPL, SMEMW>(a, p, W1p, W2p, perm, seg, m, fcp, fc_cur, it, 0,
                                                  calls, s_fs[wib], s_hs[wib]);
        });
}

template <int NPL, bool SMEMW>
cudaError_t launch_picard_mlp(Instance* I, const KArgs& a, const MlpPolicy& p, cudaStream_t st) {
    auto kern = k_picard_mlp<NPL, SMEMW>;
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

template <int NPL, bool SMEMW>
cudaError_t launch_seq_mlp(Instance* I, const MlpPolicy& p, cudaStream_t st) {
    auto kern = k_seq_mlp<NPL, SMEMW>;
    const size_t smem = SMEMW ? packed_weight_bytes(I->N) : 0;
    cudaError_t e;
    if (SMEMW && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    I->launches += 1;
    kern<<<1, 32, smem, st>>>(I->T, I->N, I->prod, I->reg, I->xwork, I->act_t, p, I->ctrl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_alloc(Instance* I) {
    if (I->mlp_P) return cudaSuccess;  // sized once per instance
    cudaError_t e = cudaMalloc((void**)&I->mlp_P, sizeof(float) * (size_t)I->R * kHidden);
    if (!e) e = cudaMalloc((void**)&I->mlp_W1p, sizeof(uint4) * (size_t)I->N * 32);
    if (!e) e = cudaMalloc((void**)&I->mlp_W2p, sizeof(uint4) * (size_t)I->N * (kHidden / 8));
    if (!e) e = cudaMalloc((void**)&I->mlp_b2, sizeof(float) * (size_t)I->N);
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
