// MLP and Gumbel-max policies on one warp: the fixed-order FP32 scorer, the
// replay of one Picard segment and the sequential simulation, shared by the
// single-trajectory and batch kernels.
//
// MLP policies (Sec. 4.1: an MLP scores the warehouses; the order goes to the
// best-scoring warehouse that holds stock) in a fixed FP32 operation order, and
// their Gumbel-max sampling variant.
//
// Score of warehouse n for an order of product k in region r with stock row S:
//   h_j = b1_j, then one fmaf per input: cost[r][n]/128 (n = 0..N-1), E[r][e]
//         (e = 0..15), min(S_n, 32)/32 (n = 0..N-1), weights W1 rows in that
//         input's position; h_j = max(h_j, 0);
//   s_n = b2_n, then one fmaf per hidden unit j = 0, 1, ..., 255 with W2[j][n]
//         (the reference order: one sequential chain per output).
// Parameters are BF16 (exact in FP32).  The part of the h chain before the stock
// inputs depends only on the region, so it is evaluated once per call into
// P[r][j] (the same operations in the same order).  Argmax over stocked
// warehouses, ties to the lowest index; a^phi when nothing is stocked.
//
// Layer 1 runs in the reference order.  Layer 2 is scored fast first: eight
// partial chains over j = e mod 8 joined by a fixed tree (36 roundings per term
// at most, against 256 in the reference chain), so that one decision's latency
// stays short.  Both are FP32 evaluations of the same exact sum, hence
//   |s_fast - s_ref| <= (gamma_36 + gamma_256) (|b2_n| + sum_j |W2[j][n]| h_j)
//                    <= kScoreC (|b2_n| + hmax c2_n),
// gamma_m = m u / (1 - m u), u = 2^-24, hmax = max_j h_j, c2_n = sum_j |W2[j][n]|
// (rounded up).  The fast arg max stands when no other stocked warehouse can
// overtake it within these bounds; otherwise (a near tie) the winner and every
// warehouse within reach are re-scored in the reference order and the arg max
// is taken over those exact scores.  Either way the decision is the
// reference's.
//
// Gumbel: s_n + g_n with g_n = -log(-log u), u = ((w >> 9) + 1/2) 2^-23 from
// Philox4x32-10 (Salmon et al., SC'11) with key = seed and counter = (t,
// trajectory, n / 4, 0), word n mod 4; log from IEEE operations only (x = m 2^e,
// log m = 2 atanh((m-1)/(m+1)) by its series to the 11th power, ln 2 split in
// two).  All floating-point steps use explicit round-to-nearest intrinsics so
// that no contraction changes the bits.
#pragma once

#include <cuda_bf16.h>

#include "pic_picard.cuh"

namespace pic {
namespace mlp {

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

// ---------------------------------------------------------------- one decision, one warp
// W1p and W2p hold the BF16 weights packed in pairs (exact in FP32 after the
// 16-bit shift), in the order the scorer consumes them:
//   W1p[n * 32 + l] = {W1s[n][l + 64v] | W1s[n][l + 64v + 32] << 16, v = 0..3}
//                     (stock rows of W1; lane l's hidden units l + 32u, u = 0..7),
//   W2p[q * N + n]  = {W2[8q + 2v][n] | W2[8q + 2v + 1][n] << 16, v = 0..3}.
struct MlpPolicy {
    int N, H;
    const float* __restrict__ P;
    const uint4* __restrict__ W1p;
    const uint4* __restrict__ W2p;
    const float* __restrict__ b2f;
    // error-bound constants of the tensor-core scorer (k_mlp_bounds): Emax[r] =
    // max_j (|P[r][j]| + sum_n |W1s[n][j]|); bnd[0] = max_n sum_j |W2[j][n]|,
    // bnd[1] = max_n |b2[n]|
    const float* __restrict__ Emax;
    const float* __restrict__ bnd;
    // c2[n] = sum_j |W2[j][n]| rounded up (bound of the fast layer-2 order)
    const float* __restrict__ c2;
    // the caller's BF16 weights W1 [2N+16][H] and W2 [H][N] (tensor-core operands)
    const uint16_t* __restrict__ W1raw;
    const uint16_t* __restrict__ W2raw;
    // [R][N] FP32 scores (before the Gumbel term) of the saturated state, where
    // every warehouse holds at least 32 units (every stock feature is 1), in the
    // reference order; null: evaluate every decision
    const float* __restrict__ sat;
    bool gumbel;
    unsigned long long seed;
    int traj;
};

// Counters of one warp's MLP decisions: evaluations, tile rows re-scored in
// FP32, tile rows decided by the tensor-core scores, decisions taken from the
// saturated-state table, near ties re-scored in the reference order.
struct MlpCounts {
    unsigned long long calls, rescored, tc, sat, near;
};

// gamma_36 + gamma_256 = 1.7405e-5, rounded up with room for the FP32
// evaluation of the bound itself (a few roundings of relative 2^-24).
constexpr float kScoreC = 1.75e-5f;

// Packed weights read from shared memory (staged copy) or global memory.
template <bool SMEMW>
__device__ __forceinline__ uint4 wld4(const uint4* p) {
    if (SMEMW) return *p;
    return __ldg(p);
}
__device__ __forceinline__ float lo16(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi16(unsigned w) { return __uint_as_float(w & 0xFFFF0000u); }

// One stock input of layer 1 for the lane's 8 hidden units: acc[u] =
// fma(W1s[n][unit u], f, acc[u]), u in the W1p packing order (low then high half
// of w.x, w.y, w.z, w.w).  f is the feature's BF16 bit pattern: min(S, 32)/32 is
// exact in BF16, as are the weights.  The mixed-precision fma.rn.f32.bf16 forms
// the product of its two BF16 operands exactly and rounds the sum once to FP32,
// which is fmaf on the widened operands bit for bit, without the 8 unpacking
// instructions.
__device__ __forceinline__ void fma8_bf16(float acc[8], uint4 w, unsigned short f) {
    asm("{\n\t.reg .b16 l0, h0, l1, h1, l2, h2, l3, h3;\n\t"
        "mov.b32 {l0, h0}, %8;\n\tmov.b32 {l1, h1}, %9;\n\t"
        "mov.b32 {l2, h2}, %10;\n\tmov.b32 {l3, h3}, %11;\n\t"
        "fma.rn.f32.bf16 %0, l0, %12, %0;\n\tfma.rn.f32.bf16 %1, h0, %12, %1;\n\t"
        "fma.rn.f32.bf16 %2, l1, %12, %2;\n\tfma.rn.f32.bf16 %3, h1, %12, %3;\n\t"
        "fma.rn.f32.bf16 %4, l2, %12, %4;\n\tfma.rn.f32.bf16 %5, h2, %12, %5;\n\t"
        "fma.rn.f32.bf16 %6, l3, %12, %6;\n\tfma.rn.f32.bf16 %7, h3, %12, %7;\n\t}"
        : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3]), "+f"(acc[4]), "+f"(acc[5]),
          "+f"(acc[6]), "+f"(acc[7])
        : "r"(w.x), "r"(w.y), "r"(w.z), "r"(w.w), "h"(f));
}
// Two independent FP32 fmas in one instruction: c0 = fma(a0, b0, c0), c1 =
// fma(a1, b1, c1), each rounded once (fma.rn.f32x2; equal to two fmaf bit for
// bit, checked on the B300 over 1.05e9 random operand sets).
__device__ __forceinline__ void fma2(float& c0, float& c1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%0, %1};\n\t"
        "fma.rn.f32x2 rc, ra, rb, rc;\n\tmov.b64 {%0, %1}, rc;\n\t}"
        : "+f"(c0), "+f"(c1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

__device__ __forceinline__ unsigned short bf16_bits(float x) {
    return (unsigned short)(__float_as_uint(x) >> 16);  // exact for BF16-representable x
}

// Layer 1 in the reference order for stock row S (lane l holds warehouses
// l + 32 i) in region r: hs[j] = max(P[r][j] + stock chain, 0), every lane
// holding units l + 32 u.  fs/hs: per-warp shared scratch (N and H floats, hs
// 16-byte aligned).  Returns max_j hs[j] (warp-uniform).
template <int NPL, bool SMEMW>
__device__ __forceinline__ float mlp_hidden(const MlpPolicy& p, const uint4* W1p, const int S[NPL],
                                            int r, float* fs, float* hs) {
    const int lane = lane_id();
    const int N = p.N, H = p.H;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        if (n < N) fs[n] = __fdiv_rn((float)min(S[i], 32), 32.0f);
    }
    __syncwarp();
    constexpr int kJ = kHidden / 32;  // hidden units per lane (l + 32u), advanced together
    float acc[kJ];
#pragma unroll
    for (int u = 0; u < kJ; ++u) acc[u] = __ldg(p.P + (size_t)r * H + lane + 32 * u);
#pragma unroll 2
    for (int n = 0; n < N; ++n)
        fma8_bf16(acc, wld4<SMEMW>(W1p + n * 32 + lane), bf16_bits(fs[n]));
    float hm = 0.f;
#pragma unroll
    for (int u = 0; u < kJ; ++u) {
        const float h = acc[u] > 0.0f ? acc[u] : 0.0f;
        hs[lane + 32 * u] = h;
        hm = fmaxf(hm, h);
    }
    __syncwarp();
    // h >= 0: the bit patterns order like the values
    return __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(hm)));
}

// The reference-order score of warehouse n from the hidden layer hs: b2_n,
// then one fmaf per hidden unit in increasing j.
template <bool SMEMW>
__device__ __forceinline__ float ref_score(const MlpPolicy& p, const uint4* W2p, const float* hs,
                                           int n) {
    const float4* h4 = reinterpret_cast<const float4*>(hs);
    float s = __ldg(p.b2f + n);
#pragma unroll 4
    for (int q = 0; q < kHidden / 8; ++q) {
        const uint4 w = wld4<SMEMW>(W2p + q * p.N + n);
        const float4 ha = h4[2 * q], hb = h4[2 * q + 1];
        s = fmaf(lo16(w.x), ha.x, s);
        s = fmaf(hi16(w.x), ha.y, s);
        s = fmaf(lo16(w.y), ha.z, s);
        s = fmaf(hi16(w.y), ha.w, s);
        s = fmaf(lo16(w.z), hb.x, s);
        s = fmaf(hi16(w.z), hb.y, s);
        s = fmaf(lo16(w.w), hb.z, s);
        s = fmaf(hi16(w.w), hb.w, s);
    }
    return s;
}

// The fast layer-2 scores (eight chains and a fixed tree, before the Gumbel
// term) of the lane's warehouses n = lane + 32 i with want[i], from hs.
template <int NPL, bool SMEMW>
__device__ __forceinline__ void fast_scores(const MlpPolicy& p, const uint4* W2p, const float* hs,
                                            const bool want[NPL], float s_out[NPL]) {
    const int lane = lane_id();
    const int N = p.N;
    const float4* h4 = reinterpret_cast<const float4*>(hs);
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        if (want[i]) {
            // eight partial chains p_e over the hidden units 8q + e, then a fixed tree
            float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f, p4 = 0.f, p5 = 0.f, p6 = 0.f, p7 = 0.f;
#pragma unroll 4
            for (int q = 0; q < kHidden / 8; ++q) {
                const uint4 w = wld4<SMEMW>(W2p + q * N + n);
                const float4 ha = h4[2 * q], hb = h4[2 * q + 1];
                fma2(p0, p1, lo16(w.x), hi16(w.x), ha.x, ha.y);
                fma2(p2, p3, lo16(w.y), hi16(w.y), ha.z, ha.w);
                fma2(p4, p5, lo16(w.z), hi16(w.z), hb.x, hb.y);
                fma2(p6, p7, lo16(w.w), hi16(w.w), hb.z, hb.w);
            }
            const float v = __fadd_rn(__fadd_rn(__fadd_rn(p0, p1), __fadd_rn(p2, p3)),
                                      __fadd_rn(__fadd_rn(p4, p5), __fadd_rn(p6, p7)));
            s_out[i] = __fadd_rn(__ldg(p.b2f + n), v);
        }
    }
}

// Bound on |key_fast - key_ref| of warehouse n: the score bound, plus, with
// Gumbel noise, the two roundings of s + g (relative 2^-24 each).
__device__ __forceinline__ float key_bound(const MlpPolicy& p, int n, float hmax, float key) {
    const float bs = kScoreC * fmaf(hmax, __ldg(p.c2 + n), fabsf(__ldg(p.b2f + n)));
    return p.gumbel ? fmaf(bs, 1.0001f, ldexpf(fabsf(key), -22)) : bs;
}

// The decision from the scores s of the lane's warehouses: arg max over stocked
// warehouses of s (+ Gumbel noise for time t), ties to the lowest index, a^phi
// (-1) when nothing is stocked.  exact: s are reference-order scores (the
// saturated table).  Otherwise s are fast scores of the hidden layer in hs
// (hmax its largest unit), and near ties are re-scored in the reference order
// (counted in `near`, lane 0).  Warp-uniform.
template <int NPL, bool SMEMW>
__device__ __forceinline__ int mlp_pick(const MlpPolicy& p, const uint4* W2p, const int S[NPL],
                                        const float s_in[NPL], int t, bool exact, float hmax,
                                        const float* hs, unsigned long long& near) {
    const int lane = lane_id();
    float key[NPL], g[NPL];
    bool feas[NPL];
    unsigned best_key = 0;
    int best_n = INT_MAX;
    bool any = false;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        feas[i] = n < p.N && S[i] > 0;
        g[i] = 0.f;
        key[i] = 0.f;
        if (feas[i]) {
            float s = s_in[i];
            if (p.gumbel) {
                g[i] = gumbel1(p.seed, p.traj, t, n);
                s = __fadd_rn(s, g[i]);
            }
            key[i] = s;
            const unsigned kk = ord_key(s);
            if (!any || kk > best_key) { best_key = kk; best_n = n; any = true; }
        }
    }
    const unsigned kmax = __reduce_max_sync(kFull, any ? best_key : 0u);
    const bool stocked = __any_sync(kFull, any);
    const int nw = __reduce_min_sync(kFull, (any && best_key == kmax) ? best_n : INT_MAX);
    if (!stocked) return -1;
    if (exact) return nw;
    // the winner's key and bound, then every stocked warehouse that could reach it
    float kw_l = 0.f, bw_l = 0.f;
#pragma unroll
    for (int i = 0; i < NPL; ++i)
        if (lane + 32 * i == nw) { kw_l = key[i]; bw_l = key_bound(p, nw, hmax, key[i]); }
    const float kw = __shfl_sync(kFull, kw_l, nw & 31), bw = __shfl_sync(kFull, bw_l, nw & 31);
    bool cand[NPL];
    bool anyc = false;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        // key_n + B_n >= key_w - B_w, tested with directed roundings that never exclude
        cand[i] = feas[i] && n != nw &&
                  __fsub_rd(kw, __fadd_ru(key[i], key_bound(p, n, hmax, key[i]))) <= bw;
        anyc |= cand[i];
    }
    if (!__any_sync(kFull, anyc)) return nw;
    if (lane == 0) ++near;
    best_key = 0;
    best_n = INT_MAX;
    any = false;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        if (cand[i] || n == nw) {
            float s = ref_score<SMEMW>(p, W2p, hs, n);
            if (p.gumbel) s = __fadd_rn(s, g[i]);
            const unsigned kk = ord_key(s);
            if (!any || kk > best_key) { best_key = kk; best_n = n; any = true; }
        }
    }
    const unsigned km2 = __reduce_max_sync(kFull, any ? best_key : 0u);
    return __reduce_min_sync(kFull, (any && best_key == km2) ? best_n : INT_MAX);
}

// The warp evaluates the policy for stock row S (lane l holds warehouses l + 32 i)
// of an order in region r at time t; fs/hs: per-warp shared scratch (N and H
// floats, hs 16-byte aligned).  In the saturated state (every warehouse at 32
// units or more) the scores are row r of p.sat, which holds that state's
// reference-order scores, so the decision is the same.  Counts table decisions
// (cnt.sat) and near ties (cnt.near) on lane 0.  Returns the action
// (warp-uniform).
template <int NPL, bool SMEMW>
__device__ __forceinline__ int mlp_decide(const MlpPolicy& p, const uint4* W1p, const uint4* W2p,
                                          const int S[NPL], int r, int t, float* fs, float* hs,
                                          MlpCounts& cnt) {
    const int lane = lane_id();
    float s[NPL];
    bool sat = p.sat != nullptr;
#pragma unroll
    for (int i = 0; i < NPL; ++i)
        if (lane + 32 * i < p.N) sat &= S[i] >= 32;
    if (__all_sync(kFull, sat)) {
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            s[i] = n < p.N ? __ldg(p.sat + (size_t)r * p.N + n) : 0.0f;
        }
        if (lane == 0) ++cnt.sat;
        return mlp_pick<NPL, SMEMW>(p, W2p, S, s, t, true, 0.f, hs, cnt.near);
    }
    bool want[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) want[i] = lane + 32 * i < p.N && S[i] > 0;
    const float hmax = mlp_hidden<NPL, SMEMW>(p, W1p, S, r, fs, hs);
    fast_scores<NPL, SMEMW>(p, W2p, hs, want, s);
    const int act = mlp_pick<NPL, SMEMW>(p, W2p, S, s, t, false, hmax, hs, cnt.near);
    __syncwarp();  // fs / hs reused by the next call
    return act;
}

// ---------------------------------------------------------------- four warps per decision
// A group of four warps (128 threads) shares each decision, which shortens the
// latency of one decision (the critical path of a pass whose work is a few long
// runs).  The operations and their order are mlp_decide's exactly:
//   layer 1: thread (warp g, lane l) runs the 64-step chains of hidden units
//            l + 32 g and l + 32 g + 128 (units u = g and u = g + 4 of lane l);
//   layer 2 (fast order): thread (g, l) owns output n = l + 32 (g & 1) and the
//            four chains p_e, e = 4 (g >> 1) .. 4 (g >> 1) + 3, and forms their
//            half of the fixed tree, (p_0+p_1)+(p_2+p_3) or (p_4+p_5)+(p_6+p_7);
//   warps 0 and 1 add the halves, add b2 (and the Gumbel term), take their arg
//   max and publish it with its bound and the largest reach (key + bound) of
//   their other warehouses; every warp combines the two.  On a near tie every
//   warp re-scores the same candidates in the reference order (ref_score).
// N <= 64.  Each warp keeps its own copy of the stock row and its own feature
// scratch; the group shares hs (256 floats), ht (2 x 64) and am (4 entries),
// and synchronises with one named barrier (id bar, 128 threads) three times
// (four after a near tie).
struct Group {
    int g;        // warp index in the group (0..3)
    int bar;      // named barrier id
    float* hs;    // [256] hidden activations
    float* ht;    // [2][64] halves of the layer-2 tree
    uint4* am;    // [4]: per warp w = 0, 1: am[w] = {key order, index, any, hmax},
                  //      am[2 + w] = {key, bound, reach of the others, reach of all} (FP32 bits)
};

// Inverse of ord_key.
__device__ __forceinline__ float ord_inv(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ void group_sync(int bar) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(128) : "memory");
}

// acc = fma(w, f, acc) for one BF16 weight w and BF16 feature f (exact product,
// one rounding: fmaf on the widened operands)
__device__ __forceinline__ float fma1_bf16(float acc, unsigned short w, unsigned short f) {
    asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(acc) : "h"(w), "h"(f));
    return acc;
}

template <bool SMEMW>
__device__ __forceinline__ unsigned wld1(const unsigned* p) {
    if (SMEMW) return *p;
    return __ldg(p);
}
template <bool SMEMW>
__device__ __forceinline__ uint2 wld2(const uint2* p) {
    if (SMEMW) return *p;
    return __ldg(p);
}

template <int NPL, bool SMEMW>
__device__ __forceinline__ int mlp_decide_group(const MlpPolicy& p, const uint4* W1p,
                                                const uint4* W2p, const int S[NPL], int r, int t,
                                                float* fs, const Group& G, MlpCounts& cnt) {
    static_assert(NPL <= 2, "four-warp decisions need N <= 64");
    const int lane = lane_id();
    const int N = p.N, g = G.g;
    bool sat = p.sat != nullptr;
#pragma unroll
    for (int i = 0; i < NPL; ++i)
        if (lane + 32 * i < N) sat &= S[i] >= 32;
    if (__all_sync(kFull, sat)) {  // the same branch in every warp of the group
        float s[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            s[i] = n < N ? __ldg(p.sat + (size_t)r * N + n) : 0.0f;
        }
        if (lane == 0 && g == 0) ++cnt.sat;
        return mlp_pick<NPL, SMEMW>(p, W2p, S, s, t, true, 0.f, G.hs, cnt.near);
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        if (n < N) fs[n] = __fdiv_rn((float)min(S[i], 32), 32.0f);
    }
    __syncwarp();
    // layer 1: units j0 = lane + 32 g (word g >> 1 of W1p, half g & 1) and j1 = j0 + 128
    // (word 2 + (g >> 1))
    float a0 = __ldg(p.P + (size_t)r * kHidden + lane + 32 * g);
    float a1 = __ldg(p.P + (size_t)r * kHidden + lane + 32 * g + 128);
    const unsigned* W1w = reinterpret_cast<const unsigned*>(W1p) + 4 * lane + (g >> 1);
    const int sh = (g & 1) * 16;
#pragma unroll 4
    for (int n = 0; n < N; ++n) {
        const unsigned short f = bf16_bits(fs[n]);
        const unsigned u0 = wld1<SMEMW>(W1w + (size_t)n * 128);
        const unsigned u1 = wld1<SMEMW>(W1w + (size_t)n * 128 + 2);
        a0 = fma1_bf16(a0, (unsigned short)(u0 >> sh), f);
        a1 = fma1_bf16(a1, (unsigned short)(u1 >> sh), f);
    }
    G.hs[lane + 32 * g] = a0 > 0.0f ? a0 : 0.0f;
    G.hs[lane + 32 * g + 128] = a1 > 0.0f ? a1 : 0.0f;
    group_sync(G.bar);
    // layer 2: output n, chains 4 hf .. 4 hf + 3 (half hf of each packed uint4)
    const int n = lane + 32 * (g & 1), hf = g >> 1;
    if (n < N) {
        const uint2* W2h = reinterpret_cast<const uint2*>(W2p) + 2 * n + hf;
        const float4* h4 = reinterpret_cast<const float4*>(G.hs) + hf;
        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll 4
        for (int q = 0; q < kHidden / 8; ++q) {
            const uint2 w = wld2<SMEMW>(W2h + (size_t)2 * q * N);
            const float4 h = h4[2 * q];
            fma2(p0, p1, lo16(w.x), hi16(w.x), h.x, h.y);
            fma2(p2, p3, lo16(w.y), hi16(w.y), h.z, h.w);
        }
        G.ht[hf * 64 + n] = __fadd_rn(__fadd_rn(p0, p1), __fadd_rn(p2, p3));
    }
    group_sync(G.bar);
    if (hf == 0) {  // warps 0 and 1: outputs 0..31 and 32..63
        float hm = 0.f;
#pragma unroll
        for (int u = 0; u < kHidden / 32; ++u) hm = fmaxf(hm, G.hs[lane + 32 * u]);
        const float hmax = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(hm)));
        const int Sn = (NPL > 1 && (g & 1)) ? S[NPL - 1] : S[0];
        unsigned key = 0;
        float kf = 0.f, kb = 0.f;
        bool any = false;
        if (n < N && Sn > 0) {
            const float v = __fadd_rn(G.ht[n], G.ht[64 + n]);
            float s = __fadd_rn(__ldg(p.b2f + n), v);
            if (p.gumbel) s = __fadd_rn(s, gumbel1(p.seed, p.traj, t, n));
            kf = s;
            kb = key_bound(p, n, hmax, s);
            key = ord_key(s);
            any = true;
        }
        const unsigned kmax = __reduce_max_sync(kFull, any ? key : 0u);
        const bool wany = __any_sync(kFull, any);
        const int nmin = __reduce_min_sync(kFull, (any && key == kmax) ? n : INT_MAX);
        const int wl = nmin & 31;
        const float kw = __shfl_sync(kFull, kf, wl), bw = __shfl_sync(kFull, kb, wl);
        // reach = key + bound (rounded up) of this warp's other stocked warehouses, and of all
        const float reach = any ? __fadd_ru(kf, kb) : -INFINITY;
        const float rex = ord_inv(__reduce_max_sync(kFull, ord_key(lane != wl ? reach : -INFINITY)));
        const float rall = ord_inv(__reduce_max_sync(kFull, ord_key(reach)));
        if (lane == 0) {
            G.am[g] = make_uint4(kmax, (unsigned)nmin, wany ? 1u : 0u, __float_as_uint(hmax));
            G.am[2 + g] = make_uint4(__float_as_uint(kw), __float_as_uint(bw), __float_as_uint(rex),
                                     __float_as_uint(rall));
        }
    }
    group_sync(G.bar);
    const uint4 m0 = G.am[0], m1 = G.am[1];
    if (!m0.z && !m1.z) return -1;
    // the winner: the larger key, ties to the lower index (warp 0's)
    const int wi = !m0.z ? 1 : (!m1.z ? 0 : (m1.x > m0.x ? 1 : 0));
    const int nw = (int)(wi ? m1.y : m0.y);
    const uint4 fw = G.am[2 + wi], fo = G.am[3 - wi];
    const bool oany = (wi ? m0.z : m1.z) != 0;
    const float kw = __uint_as_float(fw.x), bw = __uint_as_float(fw.y);
    float reach = __uint_as_float(fw.z);
    if (oany) reach = fmaxf(reach, __uint_as_float(fo.w));
    if (!(__fsub_rd(kw, reach) <= bw)) return nw;  // nothing else can reach the winner
    // near tie: every warp scores the same candidates in the reference order
    const float hmax = __uint_as_float(m0.w);
    unsigned best_key = 0;
    int best_n = INT_MAX;
    bool any = false;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int nn = lane + 32 * i;
        if (nn < N && S[i] > 0) {
            const float gn = p.gumbel ? gumbel1(p.seed, p.traj, t, nn) : 0.f;
            float kf = __fadd_rn(__ldg(p.b2f + nn), __fadd_rn(G.ht[nn], G.ht[64 + nn]));
            if (p.gumbel) kf = __fadd_rn(kf, gn);
            const bool cand =
                nn == nw || __fsub_rd(kw, __fadd_ru(kf, key_bound(p, nn, hmax, kf))) <= bw;
            if (cand) {
                float sr = ref_score<SMEMW>(p, W2p, G.hs, nn);
                if (p.gumbel) sr = __fadd_rn(sr, gn);
                const unsigned kk = ord_key(sr);
                if (!any || kk > best_key) { best_key = kk; best_n = nn; any = true; }
            }
        }
    }
    const unsigned km = __reduce_max_sync(kFull, any ? best_key : 0u);
    const int res = __reduce_min_sync(kFull, (any && best_key == km) ? best_n : INT_MAX);
    if (lane == 0 && g == 0) ++cnt.near;
    group_sync(G.bar);  // hs / ht are read: the next decision may overwrite them
    return res;
}

// ---------------------------------------------------------------- speculative tensor-core tiles
// Inside one run the stock features min(x[k][n], 32)/32 stay the same from order
// to order until a decrement takes some warehouse below 32 units.  For the next
// L <= 16 orders of the run the warp therefore scores all of them at once from
// the current state: c = W1s^T f (FP32, shared by the rows), h_t = max(P[r_t] +
// c, 0) rounded to BF16, and s_t = h_t W2 (+ b2) and u_t = h_t |W2| with
// mma.sync m16n8k16 (BF16 inputs, FP32 accumulation).  A row's decision is the
// reference order's exactly when its top-2 margin among stocked warehouses
// exceeds max(1e-3, 2 B) with B a bound on |s_tc - s_ref| for that row:
//   |z_tc - z_ref| <= e1 = 2^-22 (N + 2) Emax[r]       (two FP32 chains of N terms),
//   B = 2.1e-3 max_n u_n + 1.01 e1 max_n sum_j |W2_jn| + 1.6e-5 max|b2| + 2^-21 |key|
// The terms cover, in order: the BF16 rounding of h (relative 2^-9) together
// with the two 256-term FP32 sums, the tensor-core accumulation and the
// reference chain from b2, each charged gamma_256 = 1.53e-5 relative (the
// first coefficient exceeds 2^-9 + 2 gamma_256 with the relative growth from
// h to its BF16 value); e1 propagated through layer 2; b2's own roundings in
// the reference chain; the roundings of the key.  Other rows are re-scored by
// mlp_decide.  Returns, on lane l < L, the action of row l (-2: re-score), and
// the lanes' state is unchanged.
constexpr int kTile = 16;
constexpr int kSpecMin = 8;          // shortest run remainder scored by a tile
constexpr float kTieMargin = 1e-3f;  // re-score rows whose top-2 margin is below this

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ void mma_bf16(float d[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Top-2 keys (and the arg max, lowest index on ties) of one row, merged over lanes.
struct Top2 {
    float k1, k2, um;
    int i1;
    __device__ __forceinline__ void add(float key, int n, float u) {
        if (key > k1 || (key == k1 && n < i1)) {
            k2 = k1;
            k1 = key;
            i1 = n;
        } else if (key > k2) {
            k2 = key;
        }
        um = fmaxf(um, u);
    }
    __device__ __forceinline__ void merge_xor(int m) {
        const float o1 = __shfl_xor_sync(kFull, k1, m), o2 = __shfl_xor_sync(kFull, k2, m);
        const float ou = __shfl_xor_sync(kFull, um, m);
        const int oi = __shfl_xor_sync(kFull, i1, m);
        if (o1 > k1 || (o1 == k1 && oi < i1)) {
            k2 = fmaxf(k1, o2);
            k1 = o1;
            i1 = oi;
        } else {
            k2 = fmaxf(k2, o1);
        }
        um = fmaxf(um, ou);
    }
};

template <int NPL, bool SMEMW>
__device__ __noinline__ int spec_tile(const MlpPolicy& p, const uint4* W1p, const uint4* W2p,
                                      int S0, int S1, int L, const int32_t* __restrict__ reg_s,
                                      const int32_t* __restrict__ perm, int j, int t_off, float* fs,
                                      float* hs) {
    const int lane = lane_id();
    const int N = p.N;
    const int S[2] = {S0, S1};  // warehouses lane and lane + 32 (N <= 64)
    const unsigned m0 = __ballot_sync(kFull, lane < N && S0 > 0);
    const unsigned m1 = NPL > 1 ? __ballot_sync(kFull, lane + 32 < N && S1 > 0) : 0u;
    const int nfeas = __popc(m0) + __popc(m1);
    if (nfeas <= 1)  // nothing to choose: a^phi, or the one stocked warehouse
        return nfeas == 0 ? -1 : (m0 ? __ffs(m0) - 1 : 32 + __ffs(m1) - 1);
    // c = W1s^T f, shared by the rows (the same chain as mlp_decide, from 0)
#pragma unroll
    for (int i = 0; i < (NPL < 2 ? NPL : 2); ++i) {
        const int n = lane + 32 * i;
        if (n < N) fs[n] = __fdiv_rn((float)min(S[i], 32), 32.0f);
    }
    __syncwarp();
    {
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int n = 0; n < N; ++n)
            fma8_bf16(acc, wld4<SMEMW>(W1p + n * 32 + lane), bf16_bits(fs[n]));
#pragma unroll
        for (int u = 0; u < 8; ++u) hs[lane + 32 * u] = acc[u];
    }
    __syncwarp();
    // rows g and g + 8 of the fragments
    const int g = lane >> 2, c = lane & 3;
    const bool okA = g < L, okB = g + 8 < L;
    const int rA = okA ? reg_s[j + g] : -1, rB = okB ? reg_s[j + g + 8] : -1;
    const int tA = okA ? perm[j + g] - t_off : 0, tB = okB ? perm[j + g + 8] - t_off : 0;
    const float* PA = p.P + (size_t)(rA < 0 ? 0 : rA) * kHidden;
    const float* PB = p.P + (size_t)(rB < 0 ? 0 : rB) * kHidden;
    const unsigned* W2u = reinterpret_cast<const unsigned*>(W2p);
    Top2 A{-INFINITY, -INFINITY, 0.f, INT_MAX}, Bq{-INFINITY, -INFINITY, 0.f, INT_MAX};
    const int ntiles = (N + 7) >> 3;
    for (int nt0 = 0; nt0 < ntiles; nt0 += 4) {
        float sacc[4][4], uacc[4][4];
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int e = 0; e < 4; ++e) sacc[t][e] = uacc[t][e] = 0.f;
#pragma unroll 2
        for (int kk = 0; kk < kHidden / 16; ++kk) {
            const int k0 = 16 * kk + 2 * c;
            const float2 c0 = *reinterpret_cast<const float2*>(hs + k0);
            const float2 c1 = *reinterpret_cast<const float2*>(hs + k0 + 8);
            float2 pa0 = make_float2(0.f, 0.f), pa1 = pa0, pb0 = pa0, pb1 = pa0;
            if (okA) {
                pa0 = __ldg(reinterpret_cast<const float2*>(PA + k0));
                pa1 = __ldg(reinterpret_cast<const float2*>(PA + k0 + 8));
            }
            if (okB) {
                pb0 = __ldg(reinterpret_cast<const float2*>(PB + k0));
                pb1 = __ldg(reinterpret_cast<const float2*>(PB + k0 + 8));
            }
            const unsigned a0 = pack_bf16(fmaxf(pa0.x + c0.x, 0.f), fmaxf(pa0.y + c0.y, 0.f));
            const unsigned a1 = pack_bf16(fmaxf(pb0.x + c0.x, 0.f), fmaxf(pb0.y + c0.y, 0.f));
            const unsigned a2 = pack_bf16(fmaxf(pa1.x + c1.x, 0.f), fmaxf(pa1.y + c1.y, 0.f));
            const unsigned a3 = pack_bf16(fmaxf(pb1.x + c1.x, 0.f), fmaxf(pb1.y + c1.y, 0.f));
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int n = 8 * (nt0 + t) + g;
                unsigned b0 = 0u, b1 = 0u;
                if (nt0 + t < ntiles && n < N) {
                    b0 = SMEMW ? W2u[((2 * kk) * N + n) * 4 + c] : __ldg(W2u + ((2 * kk) * N + n) * 4 + c);
                    b1 = SMEMW ? W2u[((2 * kk + 1) * N + n) * 4 + c]
                               : __ldg(W2u + ((2 * kk + 1) * N + n) * 4 + c);
                }
                mma_bf16(sacc[t], a0, a1, a2, a3, b0, b1);
                mma_bf16(uacc[t], a0, a1, a2, a3, b0 & 0x7FFF7FFFu, b1 & 0x7FFF7FFFu);
            }
        }
        // candidates of this lane: warehouses 8 (nt0 + t) + 2c + {0, 1}
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int n0 = 8 * (nt0 + t) + 2 * c;
            if (nt0 + t >= ntiles || n0 >= N) continue;
            float gA[4], gB[4];
            if (p.gumbel) {
                gumbel4(p.seed, p.traj, tA, n0 >> 2, gA);
                gumbel4(p.seed, p.traj, tB, n0 >> 2, gB);
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int n = n0 + e;
                if (n >= N) continue;
                const bool feas = ((n < 32 ? m0 >> n : m1 >> (n - 32)) & 1u) != 0;
                if (!feas) continue;
                const float b2 = __ldg(p.b2f + n);
                float kA = __fadd_rn(sacc[t][e], b2), kB = __fadd_rn(sacc[t][2 + e], b2);
                if (p.gumbel) {
                    kA = __fadd_rn(kA, gA[n & 3]);
                    kB = __fadd_rn(kB, gB[n & 3]);
                }
                A.add(kA, n, uacc[t][e]);
                Bq.add(kB, n, uacc[t][2 + e]);
            }
        }
    }
    A.merge_xor(1);
    A.merge_xor(2);
    Bq.merge_xor(1);
    Bq.merge_xor(2);
    const float c2max = __ldg(p.bnd), b2max = __ldg(p.bnd + 1);
    const float e1A = okA ? ldexpf((float)(N + 2), -22) * __ldg(p.Emax + rA) : 0.f;
    const float e1B = okB ? ldexpf((float)(N + 2), -22) * __ldg(p.Emax + rB) : 0.f;
    const float bA = 2.1e-3f * A.um + 1.01f * e1A * c2max + 1.6e-5f * b2max + ldexpf(fabsf(A.k1), -21);
    const float bB = 2.1e-3f * Bq.um + 1.01f * e1B * c2max + 1.6e-5f * b2max + ldexpf(fabsf(Bq.k1), -21);
    const int resA = (A.k1 - A.k2 > fmaxf(kTieMargin, 2.f * bA)) ? A.i1 : -2;
    const int resB = (Bq.k1 - Bq.k2 > fmaxf(kTieMargin, 2.f * bB)) ? Bq.i1 : -2;
    const int fromA = __shfl_sync(kFull, resA, (lane & 7) * 4);
    const int fromB = __shfl_sync(kFull, resB, (lane & 7) * 4);
    __syncwarp();  // hs / fs reused by the caller
    return lane < 8 ? fromA : fromB;
}

// Bytes of the packed weights (W1p then W2p).
__host__ __device__ __forceinline__ size_t packed_weight_bytes(int N) {
    return (size_t)2 * N * kHidden * sizeof(uint16_t);
}

// Copy the packed weights (W1p, then W2p) into shared memory.
__device__ __forceinline__ void stage_weights(const MlpPolicy& p, uint4* sw) {
    const int half = p.N * kHidden / 8;  // uint4 per packed matrix
    for (int i = threadIdx.x; i < 2 * half; i += blockDim.x)
        sw[i] = i < half ? p.W1p[i] : p.W2p[i - half];
    __syncthreads();
}

// Sequential simulation on one warp: orders strictly one at a time (time t
// counts from 0 within prod/reg/act_t).
// GROUP = 4: the four warps of a group run the loop together and share each
// decision (mlp_decide_group); every warp keeps the stock rows current (the
// same value written by each), warp 0 of the group writes the actions.
template <int NPL, bool SMEMW, int GROUP = 1>
__device__ __forceinline__ void seq_mlp_body(int T, int N, const int32_t* __restrict__ prod,
                                             const int32_t* __restrict__ reg, int32_t* xw,
                                             int8_t* __restrict__ act_t, const MlpPolicy& p,
                                             const uint4* W1p, const uint4* W2p, float* fs,
                                             float* hs, MlpCounts& cnt,
                                             const Group* G = nullptr) {
    const int lane = lane_id();
    const bool lead = GROUP == 1 || G->g == 0;
    int my_act = -1;
    for (int t = 0; t < T; ++t) {
        const int k = __ldg(prod + t), r = __ldg(reg + t);
        int S[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            S[i] = n < N ? xw[(size_t)k * N + n] : 0;
        }
        int act;
        if constexpr (GROUP > 1) {
            act = mlp_decide_group<NPL, SMEMW>(p, W1p, W2p, S, r, t, fs, *G, cnt);
            // every warp has read this order's stock row before it is decremented (a
            // table decision has no other barrier)
            group_sync(G->bar);
        } else {
            act = mlp_decide<NPL, SMEMW>(p, W1p, W2p, S, r, t, fs, hs, cnt);
        }
#pragma unroll
        for (int i = 0; i < NPL; ++i)
            if (act == lane + 32 * i) xw[(size_t)k * N + act] = S[i] - 1;
        if (lane == (t & 31)) my_act = act;
        if (lead && ((t & 31) == 31 || t == T - 1)) {
            const int tw = (t & ~31) + lane;
            if (tw < T) act_t[tw] = (int8_t)my_act;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- Picard, one warp per segment
// GROUP = 4: the four warps of a group replay the segment together, sharing
// each decision (mlp_decide_group; no tensor-core tiles); warp 0 of the group
// writes the cache, the histogram, the final stock and the counters.
template <int NPL, bool SMEMW, bool SPEC, int GROUP = 1>
__device__ bool replay_segment_mlp(const KArgs& a, const MlpPolicy& p, const uint4* W1p,
                                   const uint4* W2p, const int32_t* __restrict__ perm, int s,
                                   const SegMeta& m, int fcp, int* fc_cur, int it, int t_off,
                                   MlpCounts& cnt_out, float* fs, float* hs,
                                   const Group* G = nullptr) {
    static_assert(GROUP == 1 || !SPEC, "tiles are per warp");
    const bool lead = GROUP == 1 || G->g == 0;
    const int lane = lane_id();
    const int N = a.N, NP = a.NP;
    const int k = m.k;
    int D[NPL], x0v[NPL], S[NPL], S0[NPL], hist[NPL], corr[NPL];
    // prefix counts of earlier segments; none before pass 1 of an all-a^phi cache
    const bool chained = m.ce - m.cf > 1 && (it > 1 || a.first_dirty);
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int n = lane + 32 * i;
        x0v[i] = n < N ? a.x0[(size_t)k * N + n] : 0;
        D[i] = chained ? chain_prefix(a, s, m.cf, n) : 0;
        S[i] = max(0, x0v[i] - D[i]);
        S0[i] = S[i];
        hist[i] = 0;
        corr[i] = 0;
    }
    int r = m.r0;
    int next_run = a.run_start[r + 1];
    // the max_steps window of this pass (none: INT_MAX)
    const int whi = a.run_chunk ? ld_volatile(&a.ctrl->win_hi) : INT_MAX;
    const int wprev = a.run_chunk ? ld_volatile(&a.ctrl->win_hi_prev) : INT_MAX;
    bool eval = run_evaluated(a, whi, wprev, r, m.j0 > fcp);
    unsigned long long evals = 0, resc = 0, tcr = 0;
    MlpCounts dc{0, 0, 0, 0, 0};  // table decisions and near ties of mlp_decide
    int first_chg = INT_MAX;
    int spec_act = -2, spec_base = 0, spec_left = 0;  // current tile (rows left)
    for (int base = m.j0; base < m.jend; base += 32) {
        const int cnt = min(32, m.jend - base);
        const int my_reg = lane < cnt ? a.reg_s[base + lane] : 0;
        const int my_old = lane < cnt ? a.alpha_s[base + lane] : -1;
        const int my_t = lane < cnt ? perm[base + lane] - t_off : 0;  // time within the trajectory
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
                eval = run_evaluated(a, whi, wprev, r + 1, next_run > fcp);
                ++r;
                next_run = a.run_start[r + 1];
                spec_left = 0;  // the state jumps to the next run's start
            }
            const int rr = __shfl_sync(kFull, my_reg, q);
            const int ao = __shfl_sync(kFull, my_old, q);
            const int tt = __shfl_sync(kFull, my_t, q);
            int act = ao;
            if (eval) {
                ++evals;
                // a tile needs N <= 64 (two warehouses per lane), enough orders left in
                // the run, and every stocked warehouse above 32 units, so that no early
                // decrement can change a feature and waste the tile
                if (SPEC && NPL <= 2 && spec_left == 0 && next_run - (base + q) >= kSpecMin) {
                    bool low = false, empty = false;
#pragma unroll
                    for (int i = 0; i < NPL; ++i) {
                        low |= S[i] > 0 && S[i] <= 32;
                        empty |= lane + 32 * i < N && S[i] == 0;
                    }
                    // with no empty warehouse the saturated-state table is cheaper
                    if (!__any_sync(kFull, low) && (!p.sat || __any_sync(kFull, empty))) {
                        const int L = min(kTile, next_run - (base + q));
                        spec_act = spec_tile<NPL, SMEMW>(p, W1p, W2p, S[0], S[NPL > 1 ? 1 : 0], L,
                                                         a.reg_s, perm, base + q, t_off, fs, hs);
                        spec_base = base + q;
                        spec_left = L;
                    }
                }
                int sa = -3;  // -3: no tile; -2: tile row to re-score
                if (spec_left > 0) {
                    sa = __shfl_sync(kFull, spec_act, base + q - spec_base);
                    --spec_left;
                }
                if (sa < -1) {
                    if constexpr (GROUP > 1)
                        act = mlp_decide_group<NPL, SMEMW>(p, W1p, W2p, S, rr, tt, fs, *G, dc);
                    else
                        act = mlp_decide<NPL, SMEMW>(p, W1p, W2p, S, rr, tt, fs, hs, dc);
                    resc += sa == -2;
                } else {
                    act = sa;
                    ++tcr;
                }
            }
#pragma unroll
            for (int i = 0; i < NPL; ++i) S[i] -= (act == lane + 32 * i);
            if (spec_left > 0 && act >= 0) {
                // a warehouse below 32 units changes its feature: the tile is stale
                int sel = S[0];
#pragma unroll
                for (int i = 1; i < NPL; ++i)
                    if ((act >> 5) == i) sel = S[i];
                if (__shfl_sync(kFull, sel, act & 31) < 32) spec_left = 0;
            }
            if (act != ao) {
#pragma unroll
                for (int i = 0; i < NPL; ++i) corr[i] += (ao == lane + 32 * i) - (act == lane + 32 * i);
            }
            if (lane == q) my_new = act;
        }
        // every warp of a group has read this batch's cached actions before they
        // are overwritten (a batch without decisions has no other barrier)
        if constexpr (GROUP > 1) group_sync(G->bar);
        if (lead && lane < cnt) a.alpha_s[base + lane] = (int8_t)my_new;
        const unsigned chg = __ballot_sync(kFull, lane < cnt && my_new != my_old);
        if (chg && first_chg == INT_MAX) first_chg = base + __ffs(chg) - 1;
    }
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        hist[i] += S0[i] - S[i];
        if (lead) a.agg[(size_t)s * NP + lane + 32 * i] = hist[i];
    }
    if (lead && lane == 0 && first_chg != INT_MAX && first_chg < ld_volatile(&fc_cur[k]))
        atomicMin(&fc_cur[k], first_chg);
    if (lead && lane == 0) report_window_change(a, it, first_chg);
    if (lead && s == m.ce - 1) {
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int n = lane + 32 * i;
            if (n < N) a.xfin[(size_t)k * N + n] = S[i];
        }
    }
    if (lead && lane == 0) {
        cnt_out.calls += evals;
        cnt_out.rescored += resc;
        cnt_out.tc += tcr;
        cnt_out.sat += dc.sat;
        cnt_out.near += dc.near;
    }
    return first_chg != INT_MAX;
}


inline MlpPolicy make_policy_view(const Instance* I, const pic_policy* pol, int flags) {
    MlpPolicy p;
    p.N = I->N;
    p.H = kHidden;
    p.P = I->mlp_P;
    p.W1p = I->mlp_W1p;
    p.W2p = I->mlp_W2p;
    p.b2f = I->mlp_b2;
    p.Emax = I->mlp_Emax;
    p.bnd = I->mlp_bnd;
    p.c2 = I->mlp_c2;
    p.W1raw = static_cast<const uint16_t*>(pol->W1);
    p.W2raw = static_cast<const uint16_t*>(pol->W2);
    p.sat = (flags & PIC_FLAG_NO_SAT) ? nullptr : I->mlp_sat;
    p.gumbel = pol->kind == PIC_POLICY_GUMBEL;
    p.seed = pol->seed;
    p.traj = pol->traj;
    return p;
}

// Packed weights fit in shared memory next to the kernels' static buffers.
inline bool smem_weights_ok(int N) { return packed_weight_bytes(N) <= 150 * 1024; }

}  // namespace mlp
}  // namespace pic
