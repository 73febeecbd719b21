// Per-call preprocessing of one trajectory's order stream.
//
// Algorithm 1 assigns process m the contiguous orders [m*L, (m+1)*L).  Under
// inventory independence (Assumption 1 of Sec. 3.2) the orders of different
// products inside a process never interact, so a process splits into "runs":
// its orders of one product, replayed in time order.  The cached prefix that a
// run must apply before its first order involves only orders of the same
// product, so the kernels work in product-major order:
//   sorted position j  ->  (product, time) ascending (stable radix sort by product),
//   run   = maximal range of sorted positions with one product and one chunk,
//   segment = consecutive runs of one product whose first order falls in one
//             window of W sorted positions of that product (the unit one warp
//             replays), chain = all segments of one product.
// Everything here is rebuilt from the raw order stream on the device.
#include <cstddef>
#include <cstdio>

#include "pic_device.cuh"

namespace pic {

namespace {

constexpr int kScanThreads = 256;

constexpr int kRadixThreads = 256;           // 8 warps
constexpr int kRadixPerWarp = 512;           // 16 rounds of 32
constexpr int kRadixTile = 8 * kRadixPerWarp; // 4096 keys per CTA

__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
    __shared__ int warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    int before = w ? warp_sums[w - 1] : 0;
    *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

// Single-pass exclusive scan with decoupled look-back.  Tile b (= blockIdx.x)
// scans its kScanTile1 elements, publishes its total, walks back over the tiles
// before it (a warp reads 32 of them at a time) until it meets a published
// inclusive prefix, adding the totals on the way, and publishes its own.  The
// status words live in blk: blk[0] is an epoch counter, then per tile a total
// and an inclusive prefix, each (epoch + 1) << 32 | value, so words left by an
// earlier scan on the same scratch never match.  The last tile, which starts
// after all others and waits until each has published, advances the epoch.
// Waits are bounded: after kScanSpins failed polls the tile records
// PIC_ERR_TIMEOUT in *err (if given) and goes on with what it has.
constexpr int kScanItems1 = 32;
constexpr int kScanTile1 = kScanThreads * kScanItems1;  // 8192
constexpr int kScanSpins = 1 << 22;

__device__ __forceinline__ unsigned long long scan_ld(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void scan_st(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void __launch_bounds__(kScanThreads) k_scan_1pass(const int32_t* __restrict__ in,
                                                             int32_t* __restrict__ out, int n,
                                                             int32_t* blk, int32_t* total_dev,
                                                             int* err) {
    __shared__ int s_prefix;
    const int b = blockIdx.x, nb = gridDim.x;
    const unsigned tag = (unsigned)ld_volatile(blk) + 1u;
    unsigned long long* agg = reinterpret_cast<unsigned long long*>(blk + 2);
    unsigned long long* incl = agg + nb;
    const long long base = (long long)b * kScanTile1 + (long long)threadIdx.x * kScanItems1;
    const bool vec = (reinterpret_cast<uintptr_t>(in) & 15) == 0;  // 16-byte loads allowed
    int v[kScanItems1];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems1; i += 4) {
        if (vec && base + i + 3 < n) {
            const int4 q = *reinterpret_cast<const int4*>(in + base + i);
            v[i] = q.x; v[i + 1] = q.y; v[i + 2] = q.z; v[i + 3] = q.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) v[i + u] = base + i + u < n ? in[base + i + u] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) sum += v[i + u];
    }
    int tile_total;
    const int ex = block_exclusive_scan(sum, &tile_total);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int prefix = 0;
        if (b == 0) {
            if (lane == 0) scan_st(&incl[0], ((unsigned long long)tag << 32) | (unsigned)tile_total);
        } else {
            if (lane == 0) scan_st(&agg[b], ((unsigned long long)tag << 32) | (unsigned)tile_total);
            int p = b - 1, spins = 0;
            while (p >= 0) {
                const int q = p - lane;  // tile read by this lane (q < 0: an inclusive 0)
                unsigned long long wi = 0, wa = 0;
                if (q >= 0) {
                    wi = scan_ld(&incl[q]);
                    wa = scan_ld(&agg[q]);
                }
                const bool inc_ok = q < 0 || (unsigned)(wi >> 32) == tag;
                const bool agg_ok = inc_ok || (unsigned)(wa >> 32) == tag;
                const unsigned incm = __ballot_sync(kFull, inc_ok);
                const unsigned aggm = __ballot_sync(kFull, agg_ok);
                const int first = incm ? __ffs(incm) - 1 : 32;
                const unsigned need = first == 32 ? kFull : ((1u << first) - 1u) | (1u << first);
                if ((aggm & need) == need) {
                    int x = 0;
                    if (lane < first) x = (int)(unsigned)wa;
                    else if (lane == first && q >= 0) x = (int)(unsigned)wi;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
                    prefix += x;
                    if (first < 32) break;
                    p -= 32;
                } else if (++spins > kScanSpins) {
                    if (lane == 0 && err) atomicCAS(err, 0, (int)PIC_ERR_TIMEOUT);
                    break;
                } else {
                    __nanosleep(32);
                }
            }
            if (lane == 0)
                scan_st(&incl[b], ((unsigned long long)tag << 32) | (unsigned)(prefix + tile_total));
        }
        if (lane == 0) {
            s_prefix = prefix;
            if (b == nb - 1) {
                if (total_dev) *total_dev = prefix + tile_total;
                atomicAdd(blk, 1);  // every tile has read the epoch: it published
            }
        }
    }
    __syncthreads();
    int run = s_prefix + ex;
#pragma unroll
    for (int i = 0; i < kScanItems1; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

// --------------------------------------------------------------------------- radix sort
__global__ void k_radix_hist(const int32_t* __restrict__ keys, int n, int shift, int32_t* hist,
                             int nblk) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRadixTile;
    for (int i = threadIdx.x; i < kRadixTile; i += kRadixThreads) {
        long long idx = base + i;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: ranks inside the tile follow (warp, round, lane) = index order.
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in, int n, int shift,
    const int32_t* __restrict__ offs, int nblk, int32_t* __restrict__ keys_out,
    int32_t* __restrict__ vals_out) {
    __shared__ int wh[8][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 8 * 256; i += kRadixThreads) (&wh[0][0])[i] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRadixTile + (long long)w * kRadixPerWarp;
    int local[16];
    int dig[16];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int rd = 0; rd < 16; ++rd) {
        long long idx = base + rd * 32 + lane;
        bool valid = idx < n;
        int d = valid ? (keys_in[idx] >> shift) & 255 : 256 + lane;  // unique for invalid lanes
        unsigned peers = __match_any_sync(kFull, d);
        int rank = __popc(peers & lt);
        int off = valid ? wh[w][d] : 0;
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane) wh[w][d] += __popc(peers);
        __syncwarp();
        local[rd] = off + rank;
        dig[rd] = d;
    }
    __syncthreads();
    if (threadIdx.x < 256) {
        int run = 0;
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) {
            int tmp = wh[ww][threadIdx.x];
            wh[ww][threadIdx.x] = run;
            run += tmp;
        }
    }
    __syncthreads();
#pragma unroll
    for (int rd = 0; rd < 16; ++rd) {
        long long idx = base + rd * 32 + lane;
        if (idx < n) {
            int d = dig[rd];
            long long pos = (long long)offs[(long long)d * nblk + blockIdx.x] + wh[w][d] + local[rd];
            keys_out[pos] = keys_in[idx];
            vals_out[pos] = vals_in ? vals_in[idx] : (int32_t)idx;
        }
    }
}

// --------------------------------------------------------------------------- tables
// Region gather, first sorted position of every product (pstart, K + 1
// entries, pstart[K] = T: where the product changes between consecutive sorted
// positions, every product in between starts there) and run-start flags: a run
// starts where the product or the chunk changes between consecutive sorted
// positions.  The chunk of order t is t / L, or, in a batch, (t - toff[b]) /
// chunk_len[b] for the trajectory b that owns the product (consecutive
// positions of one product share b).
__global__ void k_run_flags(const int32_t* __restrict__ perm, const int32_t* __restrict__ prod_s,
                            const int32_t* __restrict__ reg, int32_t* __restrict__ reg_s, int T,
                            int K, int L, const int32_t* __restrict__ traj_of_prod,
                            const int32_t* __restrict__ toff, const int32_t* __restrict__ chunk_len,
                            int32_t* __restrict__ flag, int32_t* __restrict__ pstart) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= T) return;
    int t = perm[j];
    reg_s[j] = reg[t];
    const int kj = prod_s[j];
    const int kp = j > 0 ? prod_s[j - 1] : -1;
    for (int k = kp + 1; k <= kj; ++k) pstart[k] = (int)j;
    if (j == T - 1)
        for (int k = kj + 1; k <= K; ++k) pstart[k] = T;
    int f = 1;
    if (j > 0 && prod_s[j] == prod_s[j - 1]) {
        int tp = perm[j - 1], len = L;
        if (traj_of_prod) {
            const int b = traj_of_prod[prod_s[j]];
            t -= toff[b];
            tp -= toff[b];
            len = chunk_len[b];
        }
        f = t / len != tp / len;
    }
    flag[j] = f;
}

__global__ void k_runs(const int32_t* __restrict__ flag, const int32_t* __restrict__ ex, int T,
                       int32_t* __restrict__ run_of, int32_t* __restrict__ run_start, Ctrl* ctrl) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= T) return;
    int r = ex[j] + flag[j] - 1;
    run_of[j] = r;
    if (flag[j]) run_start[r] = (int)j;
    if (j == T - 1) {
        run_start[r + 1] = T;
        ctrl->nruns = r + 1;
    }
}

// Time block of each run (single instances): the chunk of its first order.
__global__ void k_run_chunk(const int32_t* __restrict__ run_start, const int32_t* __restrict__ perm,
                            int L, const Ctrl* ctrl, int T, int32_t* __restrict__ run_chunk) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= T || r >= ctrl->nruns) return;
    run_chunk[r] = perm[run_start[r]] / L;
}

__global__ void k_seg_flags(const int32_t* __restrict__ run_start, const int32_t* __restrict__ prod_s,
                            const int32_t* __restrict__ pstart, int W, int T, const Ctrl* ctrl,
                            int32_t* __restrict__ flag) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= T) return;
    const int nruns = ctrl->nruns;
    if (r >= nruns) { flag[r] = 0; return; }
    int j = run_start[r];
    int k = prod_s[j];
    int f = 1;
    if (r > 0) {
        int jp = run_start[r - 1];
        int kp = prod_s[jp];
        f = (k != kp) || ((j - pstart[k]) / W != (jp - pstart[kp]) / W);
    }
    flag[r] = f;
}

__global__ void k_segs(const int32_t* __restrict__ flag, const int32_t* __restrict__ ex, int T,
                       const int32_t* __restrict__ run_start, const int32_t* __restrict__ prod_s,
                       int32_t* __restrict__ seg_of_run, int32_t* __restrict__ seg_run,
                       int32_t* __restrict__ seg_prod, Ctrl* ctrl) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nruns = ctrl->nruns;
    if (r >= nruns) return;
    int s = ex[r] + flag[r] - 1;
    seg_of_run[r] = s;
    if (flag[r]) {
        seg_run[s] = (int)r;
        seg_prod[s] = prod_s[run_start[r]];
    }
    if (r == nruns - 1) {
        seg_run[s + 1] = nruns;
        ctrl->nseg = s + 1;
    }
}

__global__ void k_chains(const int32_t* __restrict__ seg_prod, const int32_t* __restrict__ seg_run,
                         const int32_t* __restrict__ run_start, const int32_t* __restrict__ pstart,
                         const int32_t* __restrict__ run_of, const int32_t* __restrict__ seg_of_run,
                         int T, const Ctrl* ctrl, int32_t* __restrict__ cf, int32_t* __restrict__ ce,
                         SegMeta* __restrict__ meta) {
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ctrl->nseg) return;
    const int k = seg_prod[s];
    const int c0 = seg_of_run[run_of[pstart[k]]];
    const int c1 = seg_of_run[run_of[pstart[k + 1] - 1]] + 1;
    cf[s] = c0;
    ce[s] = c1;
    SegMeta m;
    m.k = k;
    m.r0 = seg_run[s];
    m.r1 = seg_run[s + 1];
    m.j0 = run_start[m.r0];
    m.jend = run_start[m.r1];
    m.last_start = run_start[m.r1 - 1];
    m.cf = c0;
    m.ce = c1;
    meta[s] = m;
}

// Longest-first order of the segments: a counting sort, descending, on a
// bucket of the estimated work w = length (x mlp_weight for a segment of an MLP
// trajectory of a batch); order inside a bucket is arbitrary.  Buckets are
// exact below 32 and keep the leading 6 bits above (w = 1.m * 2^e with 5
// mantissa bits), so every 32-bit work value has one of fewer than 1024
// buckets.  Warps take segments from this order so that the long ones start
// first and the work evens out.
__device__ __forceinline__ int work_bucket(const SegMeta& m, const int32_t* __restrict__ traj_of_prod,
                                           const BatchPol* __restrict__ pol, int mlp_weight) {
    long long w = m.jend - m.j0;
    if (pol && pol[traj_of_prod[m.k]].kind >= PIC_POLICY_MLP) w *= mlp_weight;
    const unsigned v = (unsigned)min(w, 0x7FFFFFFFll);
    int key = (int)v;
    if (v >= 32) {
        const int e = 31 - __clz(v);
        key = (e - 4) * 32 + (int)((v >> (e - 5)) & 31);
    }
    return kLenBuckets - 1 - key;
}

__global__ void k_len_hist(const SegMeta* __restrict__ meta, const Ctrl* ctrl,
                           const int32_t* __restrict__ traj_of_prod, const BatchPol* __restrict__ pol,
                           int mlp_weight, int32_t* hist) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = s < ctrl->nseg;
    int b = -1 - (int)(threadIdx.x & 31);
    if (valid) b = work_bucket(meta[s], traj_of_prod, pol, mlp_weight);
    const unsigned peers = __match_any_sync(kFull, b);
    if (valid && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&hist[b], __popc(peers));
}

__global__ void k_len_scatter(const SegMeta* __restrict__ meta, const Ctrl* ctrl,
                              const int32_t* __restrict__ traj_of_prod,
                              const BatchPol* __restrict__ pol, int mlp_weight, int32_t* offs,
                              int32_t* __restrict__ lpt) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = s < ctrl->nseg;
    const int lane = threadIdx.x & 31;
    int b = -1 - lane;
    if (valid) b = work_bucket(meta[s], traj_of_prod, pol, mlp_weight);
    const unsigned peers = __match_any_sync(kFull, b);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (valid && leader == lane) base = atomicAdd(&offs[b], __popc(peers));
    base = __shfl_sync(kFull, base, leader);
    if (valid) lpt[base + __popc(peers & ((1u << lane) - 1u))] = (int)s;
}

__global__ void k_scatter_actions(const int8_t* __restrict__ alpha_s, const int32_t* __restrict__ perm,
                                  int T, int8_t* __restrict__ act_t) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < T) act_t[perm[j]] = alpha_s[j];
}

// Total cost sum_t cost[r_t][a_t] over fulfilled orders and the a^phi count,
// from the converged cache (in sorted order).
__global__ void k_reduce_costs(const int8_t* __restrict__ alpha_s, const int32_t* __restrict__ reg_s,
                               const int32_t* __restrict__ cost, int T, int N, Ctrl* ctrl) {
    long long c = 0, l = 0;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < T;
         j += (long long)gridDim.x * blockDim.x) {
        const int a = alpha_s[j];
        if (a >= 0) c += __ldg(cost + (size_t)reg_s[j] * N + a);
        else l += 1;
    }
    c = warp_sum_i64(c);
    l = warp_sum_i64(l);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd((unsigned long long*)&ctrl->total_cost, (unsigned long long)c);
        atomicAdd((unsigned long long*)&ctrl->lost, (unsigned long long)l);
    }
}

inline int nblocks(long long n, int per) { return (int)((n + per - 1) / per); }

}  // namespace

cudaError_t scan_exclusive(const int32_t* in, int32_t* out, int n, int32_t* total_dev, int32_t* blk,
                           cudaStream_t st, int* err) {
    if (n <= 0) return cudaSuccess;
    k_scan_1pass<<<nblocks(n, kScanTile1), kScanThreads, 0, st>>>(in, out, n, blk, total_dev, err);
    return cudaGetLastError();
}

int sort_hist_len(int n) { return 256 * nblocks(n, kRadixTile); }
int scan_blk_len(int n) { return 2 + 4 * nblocks(n > 0 ? n : 1, kScanTile1); }

cudaError_t sort_pairs(Instance* I, const int32_t* keys, int n, int max_key, int32_t* keys_out,
                       int32_t* vals_out, int32_t* tmp_k, int32_t* tmp_v, cudaStream_t st) {
    int passes = 1;
    while (passes < 4 && ((unsigned)max_key >> (8 * passes)) != 0) ++passes;
    I->launches += n > 0 ? passes * 3 : 0;
    return sort_pairs_raw(keys, n, max_key, keys_out, vals_out, tmp_k, tmp_v, I->hist,
                          I->scan_blk, st, &I->ctrl->err);
}

cudaError_t sort_pairs_raw(const int32_t* keys, int n, int max_key, int32_t* keys_out,
                           int32_t* vals_out, int32_t* tmp_k, int32_t* tmp_v, int32_t* hist,
                           int32_t* scan_blk, cudaStream_t st, int* err) {
    if (n <= 0) return cudaSuccess;
    // LSD radix, 8-bit digits, as many passes as max_key has bytes; the passes
    // alternate between (tmp_k, tmp_v) and (keys_out, vals_out) so that the last
    // one lands in (keys_out, vals_out)
    int passes = 1;
    while (passes < 4 && ((unsigned)max_key >> (8 * passes)) != 0) ++passes;
    const int nblk = nblocks(n, kRadixTile);
    const int32_t* kin = keys;
    const int32_t* vin = nullptr;
    cudaError_t e;
    for (int p = 0; p < passes; ++p) {
        const bool last_side = ((passes - 1 - p) & 1) == 0;
        int32_t* kout = last_side ? keys_out : tmp_k;
        int32_t* vout = last_side ? vals_out : tmp_v;
        const int shift = 8 * p;
        k_radix_hist<<<nblk, kRadixThreads, 0, st>>>(kin, n, shift, hist, nblk);
        if ((e = scan_exclusive(hist, hist, 256 * nblk, nullptr, scan_blk, st, err))) return e;
        k_radix_scatter<<<nblk, kRadixThreads, 0, st>>>(kin, vin, n, shift, hist, nblk, kout, vout);
        kin = kout;
        vin = vout;
    }
    return cudaGetLastError();
}

cudaError_t build_tables(Instance* I, int M, int W, cudaStream_t st) {
    const int T = I->T, K = I->K;
    cudaError_t e;
    if (T == 0) return cudaMemsetAsync(I->ctrl, 0, offsetof(Ctrl, tag_base), st);
    // 1. stable sort of (product, time) by product
    // kernel launches made below besides the sort: product offsets, run flags +
    // scan + runs, segment flags + scan + segments + chains
    I->launches += 3 + 4;
    if ((e = sort_pairs(I, I->prod, T, K - 1, I->prod_s, I->perm, I->tmp_a, I->tmp_b, st))) return e;
    // 2. first sorted position of every product, and runs for M chunks of L orders
    const long long L = ((long long)T + M - 1) / M;
    const Batch* bt = I->batch;
    k_run_flags<<<nblocks(T, 256), 256, 0, st>>>(I->perm, I->prod_s, I->reg, I->reg_s, T, K, (int)L,
                                                  bt ? bt->traj_of_prod : nullptr,
                                                  bt ? bt->toff : nullptr,
                                                  bt ? bt->chunk_len : nullptr, I->tmp_a, I->pstart);
    if ((e = scan_exclusive(I->tmp_a, I->tmp_b, T, nullptr, I->scan_blk, st, &I->ctrl->err))) return e;
    k_runs<<<nblocks(T, 256), 256, 0, st>>>(I->tmp_a, I->tmp_b, T, I->run_of, I->run_start, I->ctrl);
    if (!bt) {  // time block of each run (the max_steps window)
        k_run_chunk<<<nblocks(T, 256), 256, 0, st>>>(I->run_start, I->perm, (int)L, I->ctrl, T,
                                                     I->run_chunk);
        I->launches += 1;
    }
    // 4. segments (window W per product) and chains
    k_seg_flags<<<nblocks(T, 256), 256, 0, st>>>(I->run_start, I->prod_s, I->pstart, W, T, I->ctrl,
                                                  I->tmp_a);
    if ((e = scan_exclusive(I->tmp_a, I->tmp_b, T, nullptr, I->scan_blk, st, &I->ctrl->err))) return e;
    k_segs<<<nblocks(T, 256), 256, 0, st>>>(I->tmp_a, I->tmp_b, T, I->run_start, I->prod_s,
                                             I->seg_of_run, I->seg_run, I->seg_prod, I->ctrl);
    k_chains<<<nblocks(I->smax, 256), 256, 0, st>>>(I->seg_prod, I->seg_run, I->run_start,
                                                     I->pstart, I->run_of, I->seg_of_run, T, I->ctrl,
                                                     I->seg_cf, I->seg_ce, I->seg_meta);
    if ((e = cudaGetLastError())) return e;
    // 5. longest-first order of the segments (a batch rebuilds it per call, as
    // it depends on the trajectories' policies)
    return build_lpt(I, nullptr, 1, st);
}

cudaError_t build_lpt(Instance* I, const BatchPol* pol, int mlp_weight, cudaStream_t st) {
    if (I->T == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(I->len_hist, 0, sizeof(int32_t) * kLenBuckets, st);
    if (e) return e;
    const int sb = nblocks(I->smax, 256);
    const int32_t* top = I->batch ? I->batch->traj_of_prod : nullptr;
    I->launches += 3;
    k_len_hist<<<sb, 256, 0, st>>>(I->seg_meta, I->ctrl, top, pol, mlp_weight, I->len_hist);
    if ((e = scan_exclusive(I->len_hist, I->len_hist, kLenBuckets, nullptr, I->scan_blk, st,
                            &I->ctrl->err)))
        return e;
    k_len_scatter<<<sb, 256, 0, st>>>(I->seg_meta, I->ctrl, top, pol, mlp_weight, I->len_hist,
                                      I->seg_lpt);
    return cudaGetLastError();
}

cudaError_t reduce_costs(Instance* I, const int8_t* alpha, const int32_t* reg, cudaStream_t st) {
    if (I->T == 0) return cudaSuccess;
    I->launches += 1;
    k_reduce_costs<<<4 * I->num_sms, 256, 0, st>>>(alpha, reg, I->cost, I->T, I->N, I->ctrl);
    return cudaGetLastError();
}

cudaError_t scatter_actions(Instance* I, cudaStream_t st) {
    if (I->T == 0) return cudaSuccess;
    I->launches += 1;
    k_scatter_actions<<<nblocks(I->T, 256), 256, 0, st>>>(I->alpha_s, I->perm, I->T, I->act_t);
    return cudaGetLastError();
}

cudaError_t finish_outputs(Instance* I, cudaStream_t st) {
    if (I->T == 0) return cudaSuccess;
    cudaError_t e = scatter_actions(I, st);
    if (e) return e;
    return reduce_costs(I, I->alpha_s, I->reg_s, st);
}

}  // namespace pic
