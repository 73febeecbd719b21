// REINFORCE gradient of the softmax MLP policy along simulated trajectories
// (pic_policy_grad).
//
// Objective: the policy-gradient surrogate of Sec. 4.2's training,
//   J(theta) = sum_b sum_t log pi_theta(a_t | s_t) G_t,
//   G_t = -(sum of trajectory b's order costs from t on)   (int64 suffix sums),
// pi_theta the softmax of the MLP scores over the feasible set F_t = {n :
// x_t[k_t][n] > 0}; orders with a_t = a^phi or |F_t| < 2 contribute nothing.
// The paths (s_t, a_t, G_t) are held fixed; the parameters are the BF16
// roundings of FP32 masters and the gradient with respect to those BF16 values
// is returned for the masters (straight-through).  Gumbel-max sampling draws a_t
// from exactly this softmax, so with Gumbel paths J's gradient is the REINFORCE
// estimate.
//
// Pipeline (all on the device):
//   1. BF16 rounding of the masters, the per-region prefix P[r] from them;
//   2. the paths: given, or simulated here by the batch Picard launch;
//   3. order costs, an int64 scan over time, G_t per order;
//   4. stock features per order: one warp per product walks the product's
//      orders in time order from x0 (min(x, 32) as int8; whether the order
//      counts), checking that every fulfilled action had stock;
//   5. the orders sorted by region;
//   6. k_pg_grad: tiles of 32 region-sorted orders.  Per tile the hidden layer
//      is recomputed (z = P[r] + W1s^T f; nothing of size T x 256 is stored),
//      then scores, softmax, ds = G (e_a - p), dW2 += h^T ds, dz = (W2 ds) *
//      [z > 0], dW1s += f^T dz (stock rows of W1), and DZ[r] = sum of dz over
//      the orders of region r;
//   7. the rows of dW1 for the cost and embedding inputs, db1 and dE depend on
//      an order only through its region, so they follow from DZ:
//      dW1[n][j] = sum_r cost[r][n]/128 DZ[r][j], dW1[2N+e][j] = sum_r
//      E[r][e] DZ[r][j], db1 = sum_r DZ[r], dE[r] = W1_E DZ[r].
// Products and sums are FP32 within a tile and a CTA; every sum across CTAs,
// DZ, J and the final reductions are FP64.
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>

#include <cuda_bf16.h>

#include "pic_device.cuh"
#include "pic_tc.cuh"

using namespace pic;

namespace pic {

// Device buffers of the gradient (sized at first use; see pg_alloc).
struct PgState {
    int64_t T, R, P;
    int e_rows;
    uint16_t* pbf;     // [P] BF16 parameters (flat layout of pic_grad_args.master)
    int8_t* acts;      // [T] paths simulated here
    long long* cost;   // [T] order costs (time order)
    long long* pex;    // [T + 1] exclusive prefix of cost
    long long* blk;    // scan block sums
    float* G;          // [T] G_t in sorted order
    int8_t* f8;        // [T][64] min(stock, 32) in sorted order
    uint8_t* ok;       // [T] order counts (fulfilled and |F| >= 2)
    int32_t* rq;       // [T] region of the q-th order in region order
    int32_t* jq;       // [T] sorted position of the q-th order in region order
    double* acc;       // [P] gradient accumulators
    double* dz;        // [R][256] per-region sums of dz
    double* J;         // objective
    int* bad;
    int32_t* npc;      // [K + 1] pieces of each product longer than kPgPiece orders (else 0)
    int32_t* poff;     // [K + 1] their exclusive prefix (poff[K]: all such pieces)
    int32_t* pcnt;     // [T / kPgPiece + K bounded: see pg_alloc][64] actions per warehouse of a piece
};

}  // namespace pic

namespace {

using namespace pic::tc;

constexpr int kPgN = 64;         // largest N the gradient kernel handles (f8 row stride)
constexpr int kPgT = 32;         // orders per tile
constexpr int kPgThreads = 512;  // 16 warps

__device__ __forceinline__ float lo16(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi16(unsigned w) { return __uint_as_float(w & 0xFFFF0000u); }

// Round-to-nearest-even of FP32 to BF16 on the bit pattern (NaN kept quiet).
__global__ void k_round_bf16(const float* __restrict__ in, long long n, uint16_t* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned u = __float_as_uint(in[i]);
        unsigned r;
        if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) r = (u >> 16) | 0x40u;
        else r = (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
        out[i] = (uint16_t)r;
    }
}

// ---------------------------------------------------------------- returns-to-go
__global__ void k_pg_cost(const int8_t* __restrict__ act, const int32_t* __restrict__ reg,
                          const int32_t* __restrict__ cost, int N, int T, long long* __restrict__ c) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = act[t];
        c[t] = a >= 0 ? (long long)cost[(size_t)reg[t] * N + a] : 0ll;
    }
}

constexpr int kS64Threads = 256, kS64Items = 8, kS64Tile = kS64Threads * kS64Items;

__device__ __forceinline__ long long block_exscan64(long long v, long long* total) {
    __shared__ long long ws[kS64Threads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        long long s = lane < kS64Threads / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kS64Threads / 32) ws[lane] = s;
    }
    __syncthreads();
    const long long before = w ? ws[w - 1] : 0;
    *total = ws[kS64Threads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan64_reduce(const long long* __restrict__ in, int n, long long* __restrict__ blk) {
    const long long base = (long long)blockIdx.x * kS64Tile + threadIdx.x * kS64Items;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kS64Items; ++i)
        if (base + i < n) s += in[base + i];
    long long tot;
    block_exscan64(s, &tot);
    if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

// Exclusive scan of the block sums in place; the grand total goes to *total.
__global__ void k_scan64_blocks(long long* blk, int nb, long long* total) {
    long long carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kS64Threads) {
        const int i = b0 + threadIdx.x;
        const long long v = i < nb ? blk[i] : 0;
        long long tot;
        const long long ex = block_exscan64(v, &tot);
        if (i < nb) blk[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan64_down(const long long* __restrict__ in, long long* __restrict__ out, int n,
                              const long long* __restrict__ blk) {
    const long long base = (long long)blockIdx.x * kS64Tile + threadIdx.x * kS64Items;
    long long v[kS64Items];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kS64Items; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    long long tot;
    long long ex = block_exscan64(s, &tot) + blk[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kS64Items; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
}

// G_t at sorted position j: -(total cost of the trajectory from time t on).
__global__ void k_pg_G(const int32_t* __restrict__ perm, const int32_t* __restrict__ prod_s,
                       const int32_t* __restrict__ traj_of_prod, const int32_t* __restrict__ toff,
                       const long long* __restrict__ pex, int T, float* __restrict__ G) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < T;
         j += (long long)gridDim.x * blockDim.x) {
        const int t = perm[j];
        const int b = traj_of_prod[prod_s[j]];
        G[j] = (float)(-(double)(pex[toff[b + 1]] - pex[t]));
    }
}

// ---------------------------------------------------------------- stock features
// The stock row of every order from x0 and the actions before it (per product,
// in sorted = time order): min(stock, 32) per warehouse (row stride kPgN, zero
// beyond N) and whether the order counts; bit 1 of *bad: a fulfilled action
// found no stock.  A product of at most kPgPiece orders is walked by one warp;
// a longer one is cut into pieces of kPgPiece orders, the actions of every
// piece but its last counted per warehouse (k_pg_pcount), and each piece walked
// by its own warp from x0 minus the counts of the pieces before it.
constexpr int kPgPiece = 1024;

__global__ void k_pg_npieces(int K, const int32_t* __restrict__ pstart, int32_t* __restrict__ npc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > K) return;
    const int len = k < K ? pstart[k + 1] - pstart[k] : 0;
    npc[k] = len > kPgPiece ? (len + kPgPiece - 1) / kPgPiece : 0;
}

// Product of piece p: the last k with poff[k] <= p (poff nondecreasing).
__device__ __forceinline__ int piece_product(const int32_t* __restrict__ poff, int K, int p) {
    int lo = 0, hi = K;  // poff[lo] <= p < poff[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(poff + mid) <= p) lo = mid; else hi = mid;
    }
    return lo;
}

// Walk orders [j0, j1) of one product from the stock row (S0, S1) (lanes hold
// warehouses lane and lane + 32).
__device__ __forceinline__ bool walk_stock(int j0, int j1, int S0, int S1,
                                           const int8_t* __restrict__ alpha_s, int8_t* __restrict__ f8,
                                           uint8_t* __restrict__ okf) {
    const int lane = lane_id();
    bool err = false;
    for (int base = j0; base < j1; base += 32) {
        const int cnt = min(32, j1 - base);
        const int my_a = lane < cnt ? alpha_s[base + lane] : -1;
        int my_ok = 0;
        for (int q = 0; q < cnt; ++q) {
            const int a = __shfl_sync(kFull, my_a, q);
            int8_t* row = f8 + (size_t)(base + q) * kPgN;
            row[lane] = (int8_t)max(-128, min(S0, 32));
            row[lane + 32] = (int8_t)max(-128, min(S1, 32));
            const int nf = __popc(__ballot_sync(kFull, S0 > 0)) + __popc(__ballot_sync(kFull, S1 > 0));
            if (a >= 0) {
                if (a == lane) { err |= S0 <= 0; S0 -= 1; }
                if (a == lane + 32) { err |= S1 <= 0; S1 -= 1; }
            }
            if (lane == q) my_ok = (a >= 0 && nf >= 2) ? 1 : 0;
        }
        if (lane < cnt) okf[base + lane] = (uint8_t)my_ok;
    }
    return err;
}

// Products of at most kPgPiece orders, one warp each.
__global__ void k_pg_stock(int K, int N, const int32_t* __restrict__ pstart,
                           const int8_t* __restrict__ alpha_s, const int32_t* __restrict__ x0,
                           int8_t* __restrict__ f8, uint8_t* __restrict__ okf, int* bad) {
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    bool err = false;
    for (int k = gw; k < K; k += nw) {
        const int j0 = pstart[k], j1 = pstart[k + 1];
        if (j1 - j0 > kPgPiece) continue;
        const int S0 = lane < N ? x0[(size_t)k * N + lane] : 0;
        const int S1 = lane + 32 < N ? x0[(size_t)k * N + lane + 32] : 0;
        err |= walk_stock(j0, j1, S0, S1, alpha_s, f8, okf);
    }
    if (__any_sync(kFull, err) && lane == 0) atomicOr(bad, 1);
}

// Actions per warehouse of every piece but the last of its product, one warp
// per piece (per-warp bins in shared memory).
__global__ void __launch_bounds__(256) k_pg_pcount(int K, const int32_t* __restrict__ pstart,
                                                   const int32_t* __restrict__ npc,
                                                   const int32_t* __restrict__ poff,
                                                   const int8_t* __restrict__ alpha_s,
                                                   int32_t* __restrict__ pcnt) {
    __shared__ int bins[8][kPgN];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int np = poff[K];
    for (int p = gw; p < np; p += nw) {
        const int k = piece_product(poff, K, p);
        const int i = p - poff[k];
        if (i == npc[k] - 1) continue;  // the last piece's counts are never needed
        bins[w][lane] = 0;
        bins[w][lane + 32] = 0;
        __syncwarp();
        const int j0 = pstart[k] + i * kPgPiece;
        for (int j = j0 + lane; j < j0 + kPgPiece; j += 32) {
            const int a = alpha_s[j];
            if (a >= 0 && a < kPgN) atomicAdd(&bins[w][a], 1);  // a path's actions are < N
        }
        __syncwarp();
        pcnt[(size_t)p * kPgN + lane] = bins[w][lane];
        pcnt[(size_t)p * kPgN + lane + 32] = bins[w][lane + 32];
        __syncwarp();
    }
}

// Pieces of the longer products, one warp each: x0 minus the counts of the
// product's earlier pieces, then the walk.
__global__ void k_pg_stock_pieces(int K, int N, const int32_t* __restrict__ pstart,
                                  const int32_t* __restrict__ poff, const int32_t* __restrict__ pcnt,
                                  const int8_t* __restrict__ alpha_s, const int32_t* __restrict__ x0,
                                  int8_t* __restrict__ f8, uint8_t* __restrict__ okf, int* bad) {
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int np = poff[K];
    bool err = false;
    for (int p = gw; p < np; p += nw) {
        const int k = piece_product(poff, K, p);
        const int p0 = poff[k];
        int S0 = lane < N ? x0[(size_t)k * N + lane] : 0;
        int S1 = lane + 32 < N ? x0[(size_t)k * N + lane + 32] : 0;
        for (int q = p0; q < p; ++q) {
            S0 -= pcnt[(size_t)q * kPgN + lane];
            S1 -= pcnt[(size_t)q * kPgN + lane + 32];
        }
        const int j0 = pstart[k] + (p - p0) * kPgPiece;
        const int j1 = min(pstart[k + 1], j0 + kPgPiece);
        err |= walk_stock(j0, j1, S0, S1, alpha_s, f8, okf);
    }
    if (__any_sync(kFull, err) && lane == 0) atomicOr(bad, 1);
}

// ---------------------------------------------------------------- the tile kernel
struct PgArgs {
    int N, Q;                                  // warehouses, orders
    const int32_t* __restrict__ rq;            // region-sorted orders: region
    const int32_t* __restrict__ jq;            //   and sorted position
    const int8_t* __restrict__ alpha_s;        // action per sorted position
    const float* __restrict__ G;               // G_t per sorted position
    const int8_t* __restrict__ f8;             // features per sorted position
    const uint8_t* __restrict__ ok;
    const float* __restrict__ P;               // [R][256] prefix b1 + cost + embedding rows
    const uint16_t* __restrict__ W1;           // BF16 [(2N+16)][256]
    const uint16_t* __restrict__ W2;           // BF16 [256][N]
    const uint16_t* __restrict__ b2;           // BF16 [N]
    double* accW1;                             // FP64 [(2N+16)][256] (stock rows written here)
    double* accW2;                             // FP64 [256][N]
    double* accb2;                             // FP64 [N]
    double* dz;                                // FP64 [R][256]
    double* J;
};

struct __align__(16) PgSmem {
    uint2 w1s[kPgN][64];     // stock rows of W1, [n][j/4] as 4 BF16
    uint2 w2[kHidden][16];   // W2 [j][n/4]
    uint2 w2t[kPgN][64];     // W2^T [n][j/4]
    float h[kPgT][kHidden];  // hidden activations, then dz
    float f[kPgT][kPgN];     // features [t][n]
    float fT[kPgN][kPgT];    // [n][t]
    float ds[kPgT][kPgN];    // scores, then ds [t][n]
    float dsT[kPgN][kPgT];   // [n][t]
    float b2[kPgN];
    float G[kPgT];
    int r[kPgT], a[kPgT], ok[kPgT], j[kPgT];
    double db2[kPgN];
};

__device__ __forceinline__ void unpack4(uint2 u, float w[4]) {
    w[0] = lo16(u.x); w[1] = hi16(u.x); w[2] = lo16(u.y); w[3] = hi16(u.y);
}

template <bool GRAD>
__global__ void __launch_bounds__(kPgThreads, 1) k_pg_grad(PgArgs p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PgSmem& s = *reinterpret_cast<PgSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int N = p.N;
    // ---- weights to shared memory (zero beyond N)
    for (int i = tid; i < kPgN * 64; i += kPgThreads) {
        const int n = i >> 6, q = i & 63;
        uint2 v = make_uint2(0, 0);
        if (n < N) {
            const uint16_t* row = p.W1 + (size_t)(N + n) * kHidden + 4 * q;
            v = make_uint2(row[0] | ((unsigned)row[1] << 16), row[2] | ((unsigned)row[3] << 16));
        }
        s.w1s[n][q] = v;
        uint16_t e[4];
        for (int c = 0; c < 4; ++c) e[c] = n < N ? p.W2[(size_t)(4 * q + c) * N + n] : 0;
        s.w2t[n][q] = make_uint2(e[0] | ((unsigned)e[1] << 16), e[2] | ((unsigned)e[3] << 16));
    }
    for (int i = tid; i < kHidden * 16; i += kPgThreads) {
        const int jj = i >> 4, q = i & 15;
        uint16_t e[4];
        for (int c = 0; c < 4; ++c) e[c] = 4 * q + c < N ? p.W2[(size_t)jj * N + 4 * q + c] : 0;
        s.w2[jj][q] = make_uint2(e[0] | ((unsigned)e[1] << 16), e[2] | ((unsigned)e[3] << 16));
    }
    if (tid < kPgN) {
        s.b2[tid] = tid < N ? lo16(p.b2[tid]) : 0.0f;
        s.db2[tid] = 0.0;
    }
    __syncthreads();
    // thread blocks of the two accumulated products: hidden units j0..j0+3,
    // warehouses n0..n0+7
    const int jq4 = tid & 63, j0 = 4 * jq4;
    const int nb8 = tid >> 6, n0 = 8 * nb8;
    float accW2[4][8], accW1[8][4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int i = 0; i < 8; ++i) accW2[c][i] = accW1[i][c] = 0.0f;
    double Jw = 0.0;
    int cur_r = -1;   // DZ run (threads < 256: column j = tid)
    float run = 0.0f;
    const int ntiles = (p.Q + kPgT - 1) / kPgT;
    const int tb0 = (int)((long long)blockIdx.x * ntiles / gridDim.x);
    const int tb1 = (int)((long long)(blockIdx.x + 1) * ntiles / gridDim.x);
    for (int tile = tb0; tile < tb1; ++tile) {
        // ---- orders of the tile
        if (tid < kPgT) {
            const int q = tile * kPgT + tid;
            int jj = -1, r = -1, a = -1, okv = 0;
            float g = 0.0f;
            if (q < p.Q) {
                jj = p.jq[q];
                r = p.rq[q];
                a = p.alpha_s[jj];
                g = p.G[jj];
                okv = p.ok[jj];
            }
            s.j[tid] = jj; s.r[tid] = r; s.a[tid] = a; s.G[tid] = g; s.ok[tid] = okv;
        }
        __syncthreads();
        {  // features: 32 rows x 64 warehouses, 4 per thread
            const int t = tid >> 4, n4 = (tid & 15) * 4;
            const int jj = s.j[t];
            char4 v = make_char4(0, 0, 0, 0);
            if (jj >= 0) v = *reinterpret_cast<const char4*>(p.f8 + (size_t)jj * kPgN + n4);
            const float f0 = v.x / 32.0f, f1 = v.y / 32.0f, f2 = v.z / 32.0f, f3 = v.w / 32.0f;
            *reinterpret_cast<float4*>(&s.f[t][n4]) = make_float4(f0, f1, f2, f3);
            s.fT[n4][t] = f0; s.fT[n4 + 1][t] = f1; s.fT[n4 + 2][t] = f2; s.fT[n4 + 3][t] = f3;
        }
        __syncthreads();
        {  // z = P[r] + W1s^T f, h = max(z, 0): orders t0..t0+3, hidden j0..j0+3
            const int t0 = 4 * (tid >> 6);
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = s.r[t0 + i];
                float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r >= 0) pv = __ldg(reinterpret_cast<const float4*>(p.P + (size_t)r * kHidden + j0));
                acc[i][0] = pv.x; acc[i][1] = pv.y; acc[i][2] = pv.z; acc[i][3] = pv.w;
            }
            for (int n = 0; n < N; ++n) {
                const float4 fv = *reinterpret_cast<const float4*>(&s.fT[n][t0]);
                float wv[4];
                unpack4(s.w1s[n][jq4], wv);
                const float fi[4] = {fv.x, fv.y, fv.z, fv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(wv[c], fi[i], acc[i][c]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
                *reinterpret_cast<float4*>(&s.h[t0 + i][j0]) =
                    make_float4(fmaxf(acc[i][0], 0.f), fmaxf(acc[i][1], 0.f), fmaxf(acc[i][2], 0.f),
                                fmaxf(acc[i][3], 0.f));
        }
        __syncthreads();
        {  // scores: order t, warehouses nq..nq+3
            const int t = tid >> 4, nq = tid & 15;
            float acc[4] = {s.b2[4 * nq], s.b2[4 * nq + 1], s.b2[4 * nq + 2], s.b2[4 * nq + 3]};
            for (int jj = 0; jj < kHidden; jj += 4) {
                const float4 hv = *reinterpret_cast<const float4*>(&s.h[t][jj]);
                const float hi[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float wv[4];
                    unpack4(s.w2[jj + u][nq], wv);
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[c] = fmaf(hi[u], wv[c], acc[c]);
                }
            }
            *reinterpret_cast<float4*>(&s.ds[t][4 * nq]) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        }
        __syncthreads();
        // ---- softmax over the feasible set, log pi(a), ds = G (e_a - p): one warp per order
        for (int t = w; t < kPgT; t += kPgThreads / 32) {
            const bool use = s.ok[t] != 0;
            const int a = s.a[t];
            const float G = s.G[t];
            float v[2], e[2];
            bool fe[2];
            float mx = -INFINITY;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int n = lane + 32 * i;
                v[i] = s.ds[t][n];
                fe[i] = n < N && s.f[t][n] > 0.0f;
                if (fe[i]) mx = fmaxf(mx, v[i]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
            float sum = 0.0f;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                e[i] = fe[i] ? expf(v[i] - mx) : 0.0f;
                sum += e[i];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
            const float lse = mx + logf(sum);
            // score of the taken action, from the lane that owns warehouse a
            const float va = __shfl_sync(kFull, a >= 32 ? v[1] : v[0], a >= 0 ? (a & 31) : 0);
            if (use && lane == 0) Jw += (double)G * (double)(va - lse);
            if (GRAD) {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int n = lane + 32 * i;
                    const float pr = e[i] / sum;
                    const float d = (use && fe[i]) ? G * ((n == a ? 1.0f : 0.0f) - pr) : 0.0f;
                    s.ds[t][n] = d;
                    s.dsT[n][t] = d;
                }
            }
        }
        if (!GRAD) {
            __syncthreads();
            continue;
        }
        __syncthreads();
        // ---- dW2 += h^T ds, db2 += sum ds
#pragma unroll 2
        for (int t = 0; t < kPgT; ++t) {
            const float4 hv = *reinterpret_cast<const float4*>(&s.h[t][j0]);
            const float4 d0 = *reinterpret_cast<const float4*>(&s.ds[t][n0]);
            const float4 d1 = *reinterpret_cast<const float4*>(&s.ds[t][n0 + 4]);
            const float hi[4] = {hv.x, hv.y, hv.z, hv.w};
            const float di[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int i = 0; i < 8; ++i) accW2[c][i] = fmaf(hi[c], di[i], accW2[c][i]);
        }
        if (tid < kPgN) {
            float sd = 0.0f;
            for (int t = 0; t < kPgT; ++t) sd += s.ds[t][tid];
            s.db2[tid] += (double)sd;
        }
        __syncthreads();
        {  // dz = (W2 ds) * [z > 0], written over h: orders t0..t0+3, hidden j0..j0+3
            const int t0 = 4 * (tid >> 6);
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[i][c] = 0.0f;
            for (int n = 0; n < N; ++n) {
                const float4 dv = *reinterpret_cast<const float4*>(&s.dsT[n][t0]);
                float wv[4];
                unpack4(s.w2t[n][jq4], wv);
                const float di[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(wv[c], di[i], acc[i][c]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float4 hv = *reinterpret_cast<const float4*>(&s.h[t0 + i][j0]);
                hv.x = hv.x > 0.f ? acc[i][0] : 0.f;
                hv.y = hv.y > 0.f ? acc[i][1] : 0.f;
                hv.z = hv.z > 0.f ? acc[i][2] : 0.f;
                hv.w = hv.w > 0.f ? acc[i][3] : 0.f;
                *reinterpret_cast<float4*>(&s.h[t0 + i][j0]) = hv;
            }
        }
        __syncthreads();
        // ---- dW1 (stock rows) += f^T dz
#pragma unroll 2
        for (int t = 0; t < kPgT; ++t) {
            const float4 f0 = *reinterpret_cast<const float4*>(&s.f[t][n0]);
            const float4 f1 = *reinterpret_cast<const float4*>(&s.f[t][n0 + 4]);
            const float4 zv = *reinterpret_cast<const float4*>(&s.h[t][j0]);
            const float fi[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
            const float zi[4] = {zv.x, zv.y, zv.z, zv.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c) accW1[i][c] = fmaf(fi[i], zi[c], accW1[i][c]);
        }
        // ---- DZ[r] += dz rows of region r (the tile is region-sorted)
        if (tid < kHidden) {
            for (int t = 0; t < kPgT; ++t) {
                const int r = s.r[t];
                if (r < 0) break;  // tail of the last tile
                if (r != cur_r) {
                    if (cur_r >= 0) atomicAdd(p.dz + (size_t)cur_r * kHidden + tid, (double)run);
                    cur_r = r;
                    run = 0.0f;
                }
                run += s.h[t][tid];
            }
        }
        __syncthreads();
    }
    // ---- flush
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Jw += __shfl_xor_sync(kFull, Jw, o);
    if (lane == 0 && Jw != 0.0) atomicAdd(p.J, Jw);
    if (!GRAD) return;
    if (tid < kHidden && cur_r >= 0) atomicAdd(p.dz + (size_t)cur_r * kHidden + tid, (double)run);
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int n = n0 + i;
            if (n < N) {
                atomicAdd(p.accW2 + (size_t)(j0 + c) * N + n, (double)accW2[c][i]);
                atomicAdd(p.accW1 + (size_t)(N + n) * kHidden + j0 + c, (double)accW1[i][c]);
            }
        }
    if (tid < N) atomicAdd(p.accb2 + tid, s.db2[tid]);
}

// ---------------------------------------------------------------- the tile kernel on tcgen05
// The same products on the 5th-generation tensor cores: 128 region-sorted orders
// per tile (one TMEM lane per order), the hidden layer in two halves of 128
// units.  Per tile and half h (F = stock features, exact in BF16; weights BF16):
//   phase 1  Z_h = F W1s_h (TMEM), h = max(Z_h + P[r], 0) split in BF16 hi + lo,
//            SC += h_hi W2_h + h_lo W2_h;
//            then softmax, log pi(a) G and ds = G (e_a - p) per order (FP32), ds
//            split into BF16 hi + lo;
//   phase 2  Z_h again, h split hi + lo; dW2_h += h_hi^T ds_hi + h_hi^T ds_lo +
//            h_lo^T ds_hi and dH_h = ds_hi W2_h^T + ds_lo W2_h^T; dz = dH_h [h > 0]
//            split hi + lo (over the h buffers); dW1s_h^T += dz_hi^T F + dz_lo^T F;
//            per-region sums of dz.
// The split products keep each term of the order sums within ~2^-16 of FP32.
// dW2 and dW1s^T accumulate in TMEM over all tiles of the CTA and are added to
// the FP64 accumulators once at the end.  Shared-memory operands use 8x8 core
// matrices (8 rows of 16 bytes) without swizzle: element (r, c) of an [R][C]
// buffer at (r/8)(C/8)128 + (c/8)128 + (r%8)16 + (c%8)2.  Read with its rows as
// the M/N index it is a K-major operand (LBO 128 B along K, SBO (C/8)128 B along
// M/N); read with its rows as the K index it is an MN-major operand (LBO
// (C/8)128 B along K, SBO 128 B along M/N).
constexpr int kTcRows = 128;     // orders per tile = TMEM lanes
constexpr int kTcThreads = 512;  // 16 warps: four per TMEM lane quadrant

struct __align__(16) TcSmem {
    unsigned char w1s[kHidden * kPgN * 2];   // [j][n] (B of Z: K = n, N = j)
    unsigned char w2[kPgN * kHidden * 2];    // [n][j] (B of SC: K = j, N = n; B of dH: MN-major)
    unsigned char f[kTcRows * kPgN * 2];     // [t][n] (A of Z; B of dW1s^T: MN-major)
    unsigned char hhi[kTcRows * 128 * 2];    // [t][j] of one half: h hi, then dz hi
    unsigned char hlo[kTcRows * 128 * 2];    // h lo, then dz lo
    unsigned char dshi[kTcRows * kPgN * 2];  // [t][n] ds hi (A of dH; B of dW2: MN-major)
    unsigned char dslo[kTcRows * kPgN * 2];
    float b2[kPgN];
    float red[4][kTcRows];  // softmax partials of the four column quarters of a row
    float G[kTcRows];
    int r[kTcRows], a[kTcRows], ok[kTcRows], j[kTcRows];
    unsigned long long mbar;
    unsigned tmem;
    int fail;
};

constexpr unsigned kColZ = 0, kColSC = 128, kColW2 = 192, kColW1 = 320;  // TMEM column bases

__device__ __forceinline__ void ld_p16(const float* Pr, int c, bool valid, float pv[16]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 q = valid ? __ldg(reinterpret_cast<const float4*>(Pr + c) + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        pv[4 * i] = q.x; pv[4 * i + 1] = q.y; pv[4 * i + 2] = q.z; pv[4 * i + 3] = q.w;
    }
}

// Column sums over the 32 lanes of a warp, V values per lane (V = 32 or 16), by
// recursive halving: at each step a lane keeps the half of its values selected
// by its lane bit and adds its partner's copy of that half.  V = 32: lane l ends
// with the total of value l in v[0]; V = 16: lanes l and l ^ 1 end with the
// total of value l >> 1.
template <int V>
__device__ __forceinline__ float warp_column_sum(float (&v)[V]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16, c = V; c > 1; o >>= 1, c >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < c / 2; ++i) {
            const float send = up ? v[i] : v[i + c / 2];
            const float keep = up ? v[i + c / 2] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
    if (V == 16) v[0] += __shfl_xor_sync(kFull, v[0], 1);
    return v[0];
}

// One tile row's inputs: sorted position, region, action, G, whether it counts,
// and this thread's 16 stock features (column quarter cq).
struct TileIn {
    int jj, r, a, ok;
    float g;
    char4 f[4];
};

__device__ __forceinline__ TileIn load_tile_in(const PgArgs& p, int q, int cq) {
    TileIn in;
    in.jj = q < p.Q ? __ldg(p.jq + q) : -1;
    in.r = -1; in.a = -1; in.ok = 0; in.g = 0.f;
    if (in.jj >= 0 && cq == 0) {
        in.r = __ldg(p.rq + q);
        in.a = p.alpha_s[in.jj];
        in.g = __ldg(p.G + in.jj);
        in.ok = p.ok[in.jj];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
        in.f[i] = in.jj >= 0 ? *reinterpret_cast<const char4*>(p.f8 + (size_t)in.jj * kPgN + 16 * cq + 4 * i)
                             : make_char4(0, 0, 0, 0);
    return in;
}

// Thread layout: 16 warps; warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows
// = orders, or hidden units for the accumulators) and the column quarter w / 4.
// Per tile the next tile's inputs are loaded during phase 2; db2 and the region
// sums of dz are column sums over the rows of a warp (warp_column_sum), kept per
// thread (quadrant of rows, column) until the region changes.
__global__ void __launch_bounds__(kTcThreads, 1) k_pg_tc(PgArgs p, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];  // 16-byte operand addresses suffice
    TcSmem& s = *reinterpret_cast<TcSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int t = 32 * (warp & 3) + (tid & 31);  // tile row of this thread
    const int cq = warp >> 2;                    // column quarter
    const int N = p.N;
    // ---- weights (zero beyond N), control
    for (int i = tid; i < kHidden * kPgN; i += kTcThreads) {
        const int jj = i / kPgN, n = i % kPgN;
        const uint16_t w1 = n < N ? p.W1[(size_t)(N + n) * kHidden + jj] : 0;
        const uint16_t w2 = n < N ? p.W2[(size_t)jj * N + n] : 0;
        *reinterpret_cast<uint16_t*>(s.w1s + lay(jj, n, kPgN)) = w1;
        *reinterpret_cast<uint16_t*>(s.w2 + lay(n, jj, kHidden)) = w2;
    }
    if (tid < kPgN) s.b2[tid] = tid < N ? lo16(p.b2[tid]) : 0.0f;
    double db2 = 0.0;  // even lanes: db2 of column 16 cq + lane / 2 over this warp's rows
    if (tid == 0) {
        s.fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&s.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s.tmem)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_sync_operands();
    const unsigned tm = s.tmem;
    const unsigned lane_base = (unsigned)(32 * (warp & 3)) << 16;  // this warp's TMEM lanes
    unsigned phase = 0;
    bool acc_started = false;  // the TMEM accumulators hold this CTA's sums
    double Jw = 0.0;
    // per-region dz sums of column 32 cq + lane of each half over this warp's rows
    int cur_r0 = -1, cur_r1 = -1;
    float run0 = 0.f, run1 = 0.f;
    const unsigned aF = su32(s.f), aW1 = su32(s.w1s), aW2 = su32(s.w2), aH = su32(s.hhi), aL = su32(s.hlo);
    const unsigned aSh = su32(s.dshi), aSl = su32(s.dslo);
    const int ntiles = (p.Q + kTcRows - 1) / kTcRows;
    const int tb0 = (int)((long long)blockIdx.x * ntiles / gridDim.x);
    const int tb1 = (int)((long long)(blockIdx.x + 1) * ntiles / gridDim.x);
    auto issue_z = [&](int h) {  // Z_h = F W1s_h into the Z columns
        for (int kk = 0; kk < kPgN / 16; ++kk)
            tc_mma(tm + kColZ, sdesc(aF + kk * 256, 128, 1024), sdesc(aW1 + h * 16384 + kk * 256, 128, 1024),
                   tc_idesc(128, 0, 0), kk > 0);
    };
    auto issue_sc = [&](int h) {  // SC += (h_hi + h_lo) W2_h
        for (int kk = 0; kk < 128 / 16; ++kk) {
            const unsigned long long bw = sdesc(aW2 + h * 2048 + kk * 256, 128, 4096);
            tc_mma(tm + kColSC, sdesc(aH + kk * 256, 128, 2048), bw, tc_idesc(kPgN, 0, 0), (h > 0 || kk > 0));
            tc_mma(tm + kColSC, sdesc(aL + kk * 256, 128, 2048), bw, tc_idesc(kPgN, 0, 0), 1);
        }
    };
    // h = max(Z + P[r], 0) of this thread's 32 columns of half h, split in BF16 hi + lo
    auto epi_h = [&](int h, const float* Pr, bool valid) {
        for (int c0 = 32 * cq; c0 < 32 * cq + 32; c0 += 16) {
            float v[16], pv[16], lo[16];
            tc_ld16(tm + lane_base + kColZ + c0, v);
            ld_p16(Pr, 128 * h + c0, valid, pv);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float x = valid ? fmaxf(v[i] + pv[i], 0.f) : 0.f;
                v[i] = __bfloat162float(__float2bfloat16_rn(x));
                lo[i] = x - v[i];
            }
            st_row16(s.hhi, t, c0, 128, v);
            st_row16(s.hlo, t, c0, 128, lo);
        }
    };
    bool ok_all = true;
    TileIn nxt = load_tile_in(p, tb0 * kTcRows + t, cq);
    for (int tile = tb0; tile < tb1 && ok_all; ++tile) {
        // ---- the tile's orders (warps 0-3: one row each) and features (16 columns per thread)
        {
            const TileIn& in = nxt;
            if (cq == 0) {
                s.j[t] = in.jj; s.r[t] = in.r; s.a[t] = in.a; s.G[t] = in.g; s.ok[t] = in.ok;
            }
            float fv[16];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                fv[4 * i] = in.f[i].x / 32.0f; fv[4 * i + 1] = in.f[i].y / 32.0f;
                fv[4 * i + 2] = in.f[i].z / 32.0f; fv[4 * i + 3] = in.f[i].w / 32.0f;
            }
            st_row16(s.f, t, 16 * cq, kPgN, fv);
        }
        tc_sync_operands();
        const int r = s.r[t];
        const bool valid = r >= 0;
        const float* Pr = p.P + (size_t)(valid ? r : 0) * kHidden;
        // ---- phase 1: scores.  Commits: {Z_0}, {SC_0, Z_1}, {SC_1, Z_0 again}
        if (tid == 0) { issue_z(0); tc_commit(&s.mbar); }
        if (!tc_wait(&s.mbar, phase)) s.fail = 1;
        epi_h(0, Pr, valid);
        tc_sync_operands();
        if (tid == 0) { issue_sc(0); issue_z(1); tc_commit(&s.mbar); }
        if (!tc_wait(&s.mbar, phase)) s.fail = 1;
        epi_h(1, Pr, valid);
        tc_sync_operands();
        if (tid == 0) { issue_sc(1); issue_z(0); tc_commit(&s.mbar); }
        if (!tc_wait(&s.mbar, phase)) s.fail = 1;
        // ---- softmax over the stocked warehouses (quarters of a row meet in shared
        // memory); ds = G (e_a - p), split in BF16 hi + lo
        {
            const int n0 = 16 * cq;
            float sc[16];
            tc_ld16(tm + lane_base + kColSC + n0, sc);
            const bool use = s.ok[t] != 0;
            const int a = s.a[t];
            const float G = s.G[t];
            float mx = -INFINITY;
            unsigned feas = 0;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = n0 + i;
                const float f = __uint_as_float((unsigned)*reinterpret_cast<const uint16_t*>(s.f + lay(t, n, kPgN)) << 16);
                sc[i] += s.b2[n];
                if (n < N && f > 0.f) {
                    feas |= 1u << i;
                    mx = fmaxf(mx, sc[i]);
                }
            }
            s.red[cq][t] = mx;
            __syncthreads();
            mx = fmaxf(fmaxf(s.red[0][t], s.red[1][t]), fmaxf(s.red[2][t], s.red[3][t]));
            float sum = 0.f, sa = 0.f;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (n0 + i == a) sa = sc[i];
                sc[i] = ((feas >> i) & 1u) ? expf(sc[i] - mx) : 0.f;
                sum += sc[i];
            }
            __syncthreads();  // everyone has read the maxima
            s.red[cq][t] = sum;
            __syncthreads();
            sum = (s.red[0][t] + s.red[1][t]) + (s.red[2][t] + s.red[3][t]);
            if (use && a >= n0 && a < n0 + 16) Jw += (double)G * (double)(sa - mx - logf(sum));
            const float inv = use ? 1.0f / sum : 0.f;
            float dhi[16], dlo[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = n0 + i;
                const float d = use && ((feas >> i) & 1u) ? G * ((n == a ? 1.0f : 0.0f) - sc[i] * inv) : 0.f;
                dhi[i] = __bfloat162float(__float2bfloat16_rn(d));
                dlo[i] = d - dhi[i];
                sc[i] = d;
            }
            st_row16(s.dshi, t, n0, kPgN, dhi);
            st_row16(s.dslo, t, n0, kPgN, dlo);
            db2 += (double)warp_column_sum<16>(sc);  // db2: the tile's column sums of ds
        }
        tc_sync_operands();
        // the next tile's inputs, loaded while phase 2 runs
        if (tile + 1 < tb1) nxt = load_tile_in(p, (tile + 1) * kTcRows + t, cq);
        // ---- phase 2: gradients.  Per half: {dW2_h, dH_h}, then {dW1_h (, Z_1)}
        for (int h = 0; h < 2; ++h) {
            epi_h(h, Pr, valid);  // Z_h is in the Z columns (issued with the previous group)
            tc_sync_operands();
            if (tid == 0) {
                const unsigned dW2 = tm + kColW2 + 64 * h;
                const unsigned id = tc_idesc(kPgN, 1, 1);
                for (int kk = 0; kk < kTcRows / 16; ++kk) {  // K = orders
                    const unsigned long long ah = sdesc(aH + kk * 4096, 2048, 128);
                    const unsigned long long al = sdesc(aL + kk * 4096, 2048, 128);
                    const unsigned long long bh = sdesc(aSh + kk * 2048, 1024, 128);
                    const unsigned long long bl = sdesc(aSl + kk * 2048, 1024, 128);
                    tc_mma(dW2, ah, bh, id, (acc_started || kk > 0));
                    tc_mma(dW2, ah, bl, id, 1);
                    tc_mma(dW2, al, bh, id, 1);
                }
                const unsigned idh = tc_idesc(128, 0, 1);
                for (int kk = 0; kk < kPgN / 16; ++kk) {  // K = warehouses
                    const unsigned long long bw = sdesc(aW2 + h * 2048 + kk * 8192, 4096, 128);
                    tc_mma(tm + kColZ, sdesc(aSh + kk * 256, 128, 1024), bw, idh, kk > 0);
                    tc_mma(tm + kColZ, sdesc(aSl + kk * 256, 128, 1024), bw, idh, 1);
                }
                tc_commit(&s.mbar);
            }
            if (!tc_wait(&s.mbar, phase)) s.fail = 1;
            // dz = dH [h > 0] over the h buffers (hi, lo): this thread's 32 columns
            float xs[32];
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int c0 = 32 * cq + 16 * g;
                float v[16], hi[16], lo[16];
                tc_ld16(tm + lane_base + kColZ + c0, v);
#pragma unroll
                for (int i = 0; i < 16; i += 8) {
                    const uint4 hq = *reinterpret_cast<const uint4*>(s.hhi + lay(t, c0 + i, 128));
                    const unsigned hw[4] = {hq.x, hq.y, hq.z, hq.w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float hh = (e & 1) ? hi16(hw[e >> 1]) : lo16(hw[e >> 1]);
                        const float x = hh > 0.f ? v[i + e] : 0.f;
                        hi[i + e] = __bfloat162float(__float2bfloat16_rn(x));
                        lo[i + e] = x - hi[i + e];
                        xs[16 * g + i + e] = x;
                    }
                }
                st_row16(s.hhi, t, c0, 128, hi);
                st_row16(s.hlo, t, c0, 128, lo);
            }
            // per-region sums of dz over this warp's rows (region-sorted: mostly one)
            {
                const int rt = s.r[t];
                const int r0 = __shfl_sync(kFull, rt, 0);  // rows without an order come last
                if (r0 >= 0) {
                    const int col = 128 * h + 32 * cq + (tid & 31);
                    if (__all_sync(kFull, rt == r0 || rt < 0)) {
                        const float tot = warp_column_sum<32>(xs);
                        int cr = h ? cur_r1 : cur_r0;
                        float rn = h ? run1 : run0;
                        if (cr != r0) {
                            if (cr >= 0) atomicAdd(p.dz + (size_t)cr * kHidden + col, (double)rn);
                            cr = r0;
                            rn = 0.f;
                        }
                        rn += tot;
                        if (h) { cur_r1 = cr; run1 = rn; } else { cur_r0 = cr; run0 = rn; }
                    } else if (rt >= 0) {  // several regions: each row adds to its own
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            atomicAdd(p.dz + (size_t)rt * kHidden + 128 * h + 32 * cq + i, (double)xs[i]);
                    }
                }
            }
            tc_sync_operands();
            if (tid == 0) {
                const unsigned dW1 = tm + kColW1 + 64 * h;
                const unsigned id = tc_idesc(kPgN, 1, 1);
                for (int kk = 0; kk < kTcRows / 16; ++kk) {
                    const unsigned long long bf = sdesc(aF + kk * 2048, 1024, 128);
                    tc_mma(dW1, sdesc(aH + kk * 4096, 2048, 128), bf, id, (acc_started || kk > 0));
                    tc_mma(dW1, sdesc(aL + kk * 4096, 2048, 128), bf, id, 1);
                }
                if (h == 0) issue_z(1);  // the dz columns were read above
                tc_commit(&s.mbar);
            }
            if (!tc_wait(&s.mbar, phase)) s.fail = 1;
            __syncthreads();
        }
        acc_started = true;
        ok_all = s.fail == 0;
        __syncthreads();
    }
    // ---- flush: objective, region sums, the TMEM accumulators (row t = hidden unit)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Jw += __shfl_xor_sync(kFull, Jw, o);
    if ((tid & 31) == 0 && Jw != 0.0) atomicAdd(p.J, Jw);
    if (cur_r0 >= 0) atomicAdd(p.dz + (size_t)cur_r0 * kHidden + 32 * cq + (tid & 31), (double)run0);
    if (cur_r1 >= 0) atomicAdd(p.dz + (size_t)cur_r1 * kHidden + 128 + 32 * cq + (tid & 31), (double)run1);
    {
        const int col = 16 * cq + ((tid & 31) >> 1);
        if ((tid & 1) == 0 && col < N && db2 != 0.0) atomicAdd(p.accb2 + col, db2);
    }
    if (acc_started && ok_all) {
        for (int h = 0; h < 2; ++h) {
            const int jj = 128 * h + t;
            const int c0 = 16 * cq;
            float v[16], u[16];
            tc_ld16(tm + lane_base + kColW2 + 64 * h + c0, v);
            tc_ld16(tm + lane_base + kColW1 + 64 * h + c0, u);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = c0 + i;
                if (n < N) {
                    atomicAdd(p.accW2 + (size_t)jj * N + n, (double)v[i]);
                    atomicAdd(p.accW1 + (size_t)(N + n) * kHidden + jj, (double)u[i]);
                }
            }
        }
    }
    if (!ok_all && tid == 0) atomicOr(err, 4);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(512));
}

// ---------------------------------------------------------------- reductions over regions
// dW1 rows of the cost inputs (n < N), of the embedding (2N + e), and db1, from
// DZ: acc[row][j] += sum_r coef(row, r) DZ[r][j].  Block: 256 threads = one per
// hidden unit; blockIdx.y picks a group of 16 rows; regions strided over blockIdx.x.
// The coefficients (cost / 128, BF16 embeddings, 1) are exact in FP32; DZ is
// rounded to FP32 and a block's partial sums (about R / 148 regions) are FP32,
// added to the FP64 accumulators once per block (FP64 arithmetic is slow here).
__global__ void __launch_bounds__(256) k_pg_rows(int N, int R, const double* __restrict__ dz,
                                                  const int32_t* __restrict__ cost,
                                                  const uint16_t* __restrict__ E,
                                                  const int32_t* __restrict__ reg_local,
                                                  double* accW1, double* accb1) {
    const int j = threadIdx.x;
    const int nrows = N + kEmb + 1;  // cost rows, embedding rows, b1
    const int row0 = blockIdx.y * 16;
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0.0f;
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        const float d = (float)dz[(size_t)r * kHidden + j];
        const int re = reg_local[r];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int row = row0 + i;
            float c = 0.0f;
            if (row < N) c = (float)cost[(size_t)r * N + row] * 0.0078125f;  // / 128, exact
            else if (row < N + kEmb) c = lo16(E[(size_t)re * kEmb + (row - N)]);
            else if (row == N + kEmb) c = 1.0f;
            acc[i] = fmaf(c, d, acc[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int row = row0 + i;
        if (row >= nrows || acc[i] == 0.0f) continue;
        if (row < N) atomicAdd(accW1 + (size_t)row * kHidden + j, (double)acc[i]);
        else if (row < N + kEmb) atomicAdd(accW1 + (size_t)(2 * N + row - N) * kHidden + j, (double)acc[i]);
        else atomicAdd(accb1 + j, (double)acc[i]);
    }
}

// dE[reg_local[r]] += W1_E DZ[r]: one warp per region, FP32 products and sums
// over the region's 256 hidden units (BF16 weights exact, DZ rounded), added to
// the FP64 accumulators.
__global__ void k_pg_dE(int N, int R, const double* __restrict__ dz, const uint16_t* __restrict__ W1,
                        const int32_t* __restrict__ reg_local, double* accE) {
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = gw; r < R; r += nw) {
        float u[kEmb];
#pragma unroll
        for (int e = 0; e < kEmb; ++e) u[e] = 0.0f;
        for (int j = lane; j < kHidden; j += 32) {
            const float d = (float)dz[(size_t)r * kHidden + j];
#pragma unroll
            for (int e = 0; e < kEmb; ++e) u[e] = fmaf(lo16(W1[(size_t)(2 * N + e) * kHidden + j]), d, u[e]);
        }
#pragma unroll
        for (int e = 0; e < kEmb; ++e) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u[e] += __shfl_xor_sync(kFull, u[e], o);
        }
        if (lane < kEmb) {
            float v = 0.0f;
#pragma unroll
            for (int e = 0; e < kEmb; ++e)
                if (e == lane) v = u[e];
            if (v != 0.0f) atomicAdd(accE + (size_t)reg_local[r] * kEmb + lane, (double)v);
        }
    }
}

__global__ void k_pg_out(const double* __restrict__ acc, long long n, double scale, float* __restrict__ g) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        g[i] = (float)(scale * acc[i]);
}

__global__ void k_gather_paths(const int8_t* __restrict__ act, const int32_t* __restrict__ perm, int T,
                               int N, int8_t* __restrict__ alpha_s, int* bad) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < T;
         j += (long long)gridDim.x * blockDim.x) {
        int a = act[perm[j]];
        if (a < -1 || a >= N) {
            atomicOr(bad, 2);
            a = -1;
        }
        alpha_s[j] = (int8_t)a;
    }
}

// ---------------------------------------------------------------- host side
thread_local char t_msg[320];

pic_status fail(pic_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
pic_status fail(pic_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_msg, sizeof(t_msg), fmt, ap);
    va_end(ap);
    return record_error(s, t_msg);
}

#define PCU(call)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA,           \
                        "%s failed: %s (pic_pg.cu:%d)", #call, cudaGetErrorString(e_), __LINE__); \
    } while (0)

int nblk(long long n, int per) { return (int)((n + per - 1) / per); }

pic_status pg_alloc(Instance& I, int e_rows, int64_t P) {
    PgState* g = I.pg;
    if (g && g->P == P && g->e_rows == e_rows) return PIC_OK;
    if (g) {
        void* ptrs[] = {g->pbf, g->acts, g->cost, g->pex, g->blk, g->G, g->f8, g->ok, g->rq, g->jq,
                        g->acc, g->dz, g->J, g->bad, g->npc, g->poff, g->pcnt};
        for (void* q : ptrs)
            if (q) cudaFree(q);
        delete g;
        I.pg = nullptr;
    }
    g = new (std::nothrow) PgState();
    if (!g) return fail(PIC_ERR_OOM, "host allocation failed");
    memset(g, 0, sizeof(PgState));
    I.pg = g;
    g->T = I.T;
    g->R = I.R;
    g->P = P;
    g->e_rows = e_rows;
    const size_t T = (size_t)(I.T ? I.T : 1);
    PCU(cudaMalloc((void**)&g->pbf, sizeof(uint16_t) * P));
    PCU(cudaMalloc((void**)&g->acts, T));
    PCU(cudaMalloc((void**)&g->cost, sizeof(long long) * T));
    PCU(cudaMalloc((void**)&g->pex, sizeof(long long) * (T + 1)));
    PCU(cudaMalloc((void**)&g->blk, sizeof(long long) * (T / kS64Tile + 2)));
    PCU(cudaMalloc((void**)&g->G, sizeof(float) * T));
    PCU(cudaMalloc((void**)&g->f8, (size_t)kPgN * T));
    PCU(cudaMalloc((void**)&g->ok, T));
    PCU(cudaMalloc((void**)&g->rq, sizeof(int32_t) * T));
    PCU(cudaMalloc((void**)&g->jq, sizeof(int32_t) * T));
    PCU(cudaMalloc((void**)&g->acc, sizeof(double) * P));
    PCU(cudaMalloc((void**)&g->dz, sizeof(double) * (size_t)I.R * kHidden));
    PCU(cudaMalloc((void**)&g->J, sizeof(double)));
    PCU(cudaMalloc((void**)&g->bad, sizeof(int)));
    // pieces: a product longer than kPgPiece has ceil(len / kPgPiece) <= 2 len / kPgPiece
    PCU(cudaMalloc((void**)&g->npc, sizeof(int32_t) * ((size_t)I.K + 1)));
    PCU(cudaMalloc((void**)&g->poff, sizeof(int32_t) * ((size_t)I.K + 1)));
    PCU(cudaMalloc((void**)&g->pcnt, sizeof(int32_t) * kPgN * (2 * T / kPgPiece + 1)));
    return PIC_OK;
}

}  // namespace

namespace pic {
void free_pg(Instance& I) {
    PgState* g = I.pg;
    if (!g) return;
    void* ptrs[] = {g->pbf, g->acts, g->cost, g->pex, g->blk, g->G, g->f8, g->ok, g->rq, g->jq,
                    g->acc, g->dz, g->J, g->bad, g->npc, g->poff, g->pcnt};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete g;
    I.pg = nullptr;
}
}  // namespace pic

extern "C" pic_status pic_policy_grad(pic_instance* h, const pic_policy* pols, const pic_grad_args* ga,
                                      const pic_sim_opts* opts, double* objective,
                                      pic_sim_result* res) {
    clear_error();
    if (!h || !h->I.batch)
        return fail(PIC_ERR_INVALID_ARG, "pic_policy_grad needs a batch instance (pic_create_batch)");
    if (!pols || !ga || !opts || !ga->master)
        return fail(PIC_ERR_INVALID_ARG, "pols, args, args->master and opts are required");
    Instance& I = h->I;
    Batch* bt = I.batch;
    const int B = bt->B, N = I.N;
    if (N > kPgN) return fail(PIC_ERR_UNSUPPORTED, "pic_policy_grad supports N <= %d (N = %d)", kPgN, N);
    int64_t max_r = 0;
    for (int b = 0; b < B; ++b) {
        if (pols[b].kind != PIC_POLICY_MLP && pols[b].kind != PIC_POLICY_GUMBEL)
            return fail(PIC_ERR_INVALID_ARG, "trajectory %d: the gradient needs an MLP or Gumbel policy", b);
        if (pols[b].hidden != kHidden)
            return fail(PIC_ERR_UNSUPPORTED, "trajectory %d: MLP hidden width must be %d", b, kHidden);
        const int64_t rb = bt->h_roff[b + 1] - bt->h_roff[b];
        if (rb > max_r) max_r = rb;
    }
    if (ga->e_rows < max_r)
        return fail(PIC_ERR_INVALID_ARG, "e_rows = %d is below the largest trajectory R = %lld", ga->e_rows,
                    (long long)max_r);
    const int64_t oW1 = 0, ob1 = (int64_t)(2 * N + kEmb) * kHidden, oW2 = ob1 + kHidden,
                  ob2 = oW2 + (int64_t)kHidden * N, oE = ob2 + N;
    const int64_t P = oE + (int64_t)ga->e_rows * kEmb;
    pic_status s = pg_alloc(I, ga->e_rows, P);
    if (s != PIC_OK) return s;
    PgState* g = I.pg;
    cudaStream_t st = (cudaStream_t)opts->stream;
    const int T = I.T;
    const int grid = 4 * I.num_sms;
    // 1. BF16 parameters
    k_round_bf16<<<grid, 256, 0, st>>>(ga->master, P, g->pbf);
    PCU(cudaGetLastError());
    pic_policy* pb = new (std::nothrow) pic_policy[B];
    if (!pb) return fail(PIC_ERR_OOM, "host allocation failed");
    for (int b = 0; b < B; ++b) {
        pb[b] = pols[b];
        pb[b].W1 = g->pbf + oW1;
        pb[b].b1 = g->pbf + ob1;
        pb[b].W2 = g->pbf + oW2;
        pb[b].b2 = g->pbf + ob2;
        pb[b].E = g->pbf + oE;
    }
    // 2. paths
    const int8_t* acts = ga->actions;
    pic_sim_result sr;
    memset(&sr, 0, sizeof(sr));
    PCU(cudaMemsetAsync(g->bad, 0, sizeof(int), st));
    if (!acts) {
        pic_sim_opts so = *opts;
        so.mode = PIC_MODE_PICARD;
        so.out_mem = PIC_MEM_DEVICE;
        int8_t* dst = ga->actions_out ? ga->actions_out : g->acts;
        s = pic_simulate_batch(h, pb, &so, dst, nullptr, nullptr, &sr);
        if (s != PIC_OK) {
            delete[] pb;
            return s;
        }
        acts = dst;
    } else {
        if (I.tables_m == 0) {
            s = batch_tables(I, 1, kSegWindow, st);
            if (s != PIC_OK) {
                delete[] pb;
                return s;
            }
        }
        if (T) k_gather_paths<<<grid, 256, 0, st>>>(acts, I.perm, T, N, I.alpha_s, g->bad);
        PCU(cudaGetLastError());
        if (ga->actions_out && T)
            PCU(cudaMemcpyAsync(ga->actions_out, acts, T, cudaMemcpyDeviceToDevice, st));
    }
    PCU(mlp_alloc(&I));
    cudaError_t e = mlp_prepare(&I, &pb[0], st);
    delete[] pb;
    PCU(e);
    PCU(cudaMemsetAsync(g->J, 0, sizeof(double), st));
    const bool want_grad = ga->grad != nullptr;
    if (want_grad) {
        PCU(cudaMemsetAsync(g->acc, 0, sizeof(double) * P, st));
        PCU(cudaMemsetAsync(g->dz, 0, sizeof(double) * (size_t)I.R * kHidden, st));
    }
    int launches = 3;
    if (T) {
        // 3. returns-to-go
        k_pg_cost<<<grid, 256, 0, st>>>(acts, I.reg, I.cost, N, T, g->cost);
        const int nb = nblk(T, kS64Tile);
        k_scan64_reduce<<<nb, kS64Threads, 0, st>>>(g->cost, T, g->blk);
        k_scan64_blocks<<<1, kS64Threads, 0, st>>>(g->blk, nb, g->pex + T);
        k_scan64_down<<<nb, kS64Threads, 0, st>>>(g->cost, g->pex, T, g->blk);
        k_pg_G<<<grid, 256, 0, st>>>(I.perm, I.prod_s, bt->traj_of_prod, bt->toff, g->pex, T, g->G);
        // 4. stock features: short products one warp each; long ones in pieces
        k_pg_npieces<<<nblk(I.K + 1, 256), 256, 0, st>>>(I.K, I.pstart, g->npc);
        PCU(scan_exclusive(g->npc, g->poff, I.K + 1, nullptr, I.scan_blk, st, &I.ctrl->err));
        k_pg_pcount<<<grid, 256, 0, st>>>(I.K, I.pstart, g->npc, g->poff, I.alpha_s, g->pcnt);
        k_pg_stock<<<grid, 256, 0, st>>>(I.K, N, I.pstart, I.alpha_s, I.x0, g->f8, g->ok, g->bad);
        k_pg_stock_pieces<<<grid, 256, 0, st>>>(I.K, N, I.pstart, g->poff, g->pcnt, I.alpha_s, I.x0,
                                                g->f8, g->ok, g->bad);
        launches += 4;
        PCU(cudaGetLastError());
        // 5. region order
        const int l0 = I.launches;
        PCU(sort_pairs(&I, I.reg_s, T, I.R - 1, g->rq, g->jq, I.tmp_a, I.tmp_b, st));
        launches += I.launches - l0;
        // 6. tiles
        PgArgs a;
        a.N = N; a.Q = T;
        a.rq = g->rq; a.jq = g->jq; a.alpha_s = I.alpha_s; a.G = g->G; a.f8 = g->f8; a.ok = g->ok;
        a.P = I.mlp_P;
        a.W1 = g->pbf + oW1; a.W2 = g->pbf + oW2; a.b2 = g->pbf + ob2;
        a.accW1 = g->acc + oW1; a.accW2 = g->acc + oW2; a.accb2 = g->acc + ob2;
        a.dz = g->dz; a.J = g->J;
        const size_t smem = sizeof(PgSmem);
        if (want_grad && !(opts->flags & PIC_FLAG_NO_TC)) {
            const size_t tsm = sizeof(TcSmem);
            PCU(cudaFuncSetAttribute(k_pg_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
            k_pg_tc<<<I.num_sms, kTcThreads, tsm, st>>>(a, g->bad);
        } else if (want_grad) {
            PCU(cudaFuncSetAttribute(k_pg_grad<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_pg_grad<true><<<I.num_sms, kPgThreads, smem, st>>>(a);
        } else {
            PCU(cudaFuncSetAttribute(k_pg_grad<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_pg_grad<false><<<I.num_sms, kPgThreads, smem, st>>>(a);
        }
        PCU(cudaGetLastError());
        launches += 7 + 1;
        // 7. rows that depend on the region only
        if (want_grad) {
            const int groups = (N + kEmb + 1 + 15) / 16;
            k_pg_rows<<<dim3(I.num_sms, groups), 256, 0, st>>>(N, I.R, g->dz, I.cost, g->pbf + oE,
                                                               bt->reg_local, g->acc + oW1, g->acc + ob1);
            k_pg_dE<<<grid, 256, 0, st>>>(N, I.R, g->dz, g->pbf + oW1, bt->reg_local, g->acc + oE);
            PCU(cudaGetLastError());
            launches += 2;
        }
    }
    if (want_grad) {
        k_pg_out<<<grid, 256, 0, st>>>(g->acc, P, ga->grad_scale, ga->grad);
        PCU(cudaGetLastError());
        launches += 1;
    }
    double J = 0.0;
    int bad = 0;
    PCU(cudaMemcpyAsync(&J, g->J, sizeof(double), cudaMemcpyDeviceToHost, st));
    PCU(cudaMemcpyAsync(&bad, g->bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    PCU(cudaStreamSynchronize(st));
    if (bad & 4) return fail(PIC_ERR_TIMEOUT, "gradient kernel: a tensor-core wait timed out");
    if (bad & 2) return fail(PIC_ERR_INVALID_ARG, "actions hold a value outside [-1, N)");
    if (bad & 1) return fail(PIC_ERR_INVALID_ARG, "actions are not a feasible path (an order took a unit "
                                                  "from a warehouse without stock)");
    if (objective) *objective = J;
    if (res) {
        *res = sr;
        res->launches = sr.launches + launches;
    }
    return PIC_OK;
}
