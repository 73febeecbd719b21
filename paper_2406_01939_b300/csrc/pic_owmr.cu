// OWMR inventory control (Appendix B): Picard iteration with the retailer
// partition, and the sequential baseline, behind include/pic_owmr.h.
//
// A pass of Algorithm 1 runs as three phases of one persistent cooperative
// kernel, separated by grid barriers:
//   A  tile summaries of the cache alpha^{k-1} (time order),
//   B  per step t the prefix quantities of the cache before t --
//        Qc = sum of q,  LR = last step with r = 1,  D = sum of q after LR --
//      written with the cached action itself as pre[t] = {Qc, D, LR, alpha_t},
//   C  the walks: processor p (one lane of warp 0) visits only its own steps in
//      time order.  Between two own steps every step is cached, and the central
//      inventory only moves by "reset to S" and "subtract q, floor at 0", so
//        x0(t_b) = max(0, S - D[t_b])                          if LR[t_b] > t_a,
//                  max(0, x0(t_a + 1) - (Qc[t_b] - Qc[t_a + 1])) otherwise.
//      Retailer stock lives in shared memory (a retailer belongs to one lane).
//      With a network, a lane whose step needs a call (memo miss) parks it;
//      the CTA then evaluates all parked calls as one batched FP32 round.
// Nothing before the previous pass's first changed step w moved, so phase B
// keeps the tiles that end before w, and each walk resumes from a checkpoint
// at its last chunk whose lanes' states precede w.  With the max_steps window
// a pass evaluates only steps before w + max_steps.  The loop ends after the
// first pass that changed no cached action with the window covering the
// horizon.  Processors are interleaved over the CTAs' groups of 32 lanes.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "pic_device.cuh"
#include "pic_owmr.h"

using namespace pic;

namespace {

constexpr int kOwThreads = 256;             // 8 warps
constexpr int kLanes = 32;                  // processors per group (lanes of warp 0)
constexpr int kCh = 32;                     // steps per lane staged per chunk
constexpr int kItems = 16;                  // scan items per thread
constexpr int kTile = kOwThreads * kItems;  // steps per scan tile
constexpr int kMaxSlots = 4096;             // retailers per group (shared-memory stock)
constexpr int kMaxH = 512;

// Format the message pic_last_error() returns and pass the status through.
pic_status fail(pic_status s, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    return record_error(s, msg);
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA,   \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                      \
    } while (0)

// Device control block: pic::Ctrl's barrier and error fields, then per-pass
// statistics in three rotating slots (slot k % 3 is written in pass k, read
// after its last barrier, and cleared in pass k + 2 after a barrier).
struct OwCtrl {
    Ctrl c;
    int changed[3];
    int fct[3];  // first changed step of the pass (INT_MAX: none)
    long long lost[3], shipped[3], R[3];
    unsigned long long evals, rounds, near;
};

struct OwArgs {
    int T, N, P, B, ngroups, H, X0, s, S, ntiles, max_iters, rp;  // rp = ceil(N / P)
    int window;                                                   // max_steps, 0 = none
    int xs_len, nbuf;  // retailer-stock ints in shared memory; W2 buffers
    long long timeout_ns;
    const int32_t *cap, *sl, *Sl, *x0r;
    const int4* rec;        // interleaved [rows][32]: {t, n, d, e}, t = -1 pads
    const int32_t* gbase;   // [ngroups + 1] first row of each group
    int32_t* act;           // [T] cache, time order
    int4* pre;              // [T + 1]
    int4* tsum;             // [ntiles]
    int2* memo;             // interleaved like rec: {y, q} of the last evaluation
    const int32_t* cmax;    // [rows / 32] per chunk: latest first-step time over its lanes
    int4* ckpt;             // [rows / 32][2][32] walk state of each lane before each chunk
    int resume;             // walks resume at the last chunk that starts before w
    int32_t* xfin;          // [N] retailer stock after the last pass's walks
    OwCtrl* oc;
    const uint16_t *W1, *b1, *W2, *b2, *w3, *b3;
};

// ------------------------------------------------------------------ prefix monoid
// (sq, lr, da): sum of q, last replenishment index (-1 none), sum of q after it
// (the whole sum when lr = -1).  Combine left then right.
struct Mono {
    int sq, lr, da;
};

__device__ __forceinline__ Mono mono_id() { return {0, -1, 0}; }

__device__ __forceinline__ Mono mono_cat(const Mono& a, const Mono& b) {
    Mono r;
    r.sq = a.sq + b.sq;
    r.lr = b.lr >= 0 ? b.lr : a.lr;
    r.da = b.lr >= 0 ? b.da : a.da + b.sq;
    return r;
}

__device__ __forceinline__ Mono mono_step(const Mono& a, int t, int act) {
    const int q = act >> 1;
    Mono r;
    r.sq = a.sq + q;
    if (act & 1) {
        r.lr = t;
        r.da = 0;
    } else {
        r.lr = a.lr;
        r.da = a.da + q;
    }
    return r;
}

__device__ __forceinline__ Mono shfl_up_mono(const Mono& m, int o) {
    return {__shfl_up_sync(kFull, m.sq, o), __shfl_up_sync(kFull, m.lr, o),
            __shfl_up_sync(kFull, m.da, o)};
}

// Exclusive scan of one Mono per thread over the CTA, in thread order; *total
// receives the CTA's combination.  Uses the 9-entry shared array `ws`.
__device__ Mono block_exscan_mono(Mono v, Mono* total, Mono* ws) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Mono x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Mono y = shfl_up_mono(x, o);
        if (lane >= o) x = mono_cat(y, x);
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        Mono run = mono_id();
        for (int i = 0; i < kOwThreads / 32; ++i) {
            Mono nx = mono_cat(run, ws[i]);
            ws[i] = run;  // exclusive prefix of warp i
            run = nx;
        }
        ws[kOwThreads / 32] = run;
    }
    __syncthreads();
    Mono before = ws[w];
    const Mono incl_prev = shfl_up_mono(x, 1);  // every lane takes part in the shuffle
    Mono ex = lane ? mono_cat(before, incl_prev) : before;
    *total = ws[kOwThreads / 32];
    __syncthreads();
    return ex;
}

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float bf_lo(unsigned u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(unsigned u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ float bf1(uint16_t b) { return __uint_as_float((unsigned)b << 16); }

__device__ __forceinline__ int retailer_base(int y, int sl, int Sl) { return y <= sl ? Sl - y : 0; }

// q from the network output (the clamp of the retailer rule)
__device__ __forceinline__ int q_of(int base, int room, float z) {
    float v = floorf(__fadd_rn((float)base, z));
    v = v > 0.f ? v : 0.f;
    if (v > (float)room) v = (float)room;
    return (int)v;
}

constexpr int kMaxBufSlots = 2;  // mbarriers reserved for the W2 ring (kMaxBuf)

// Processors are interleaved over the groups (processor p: group p mod ngroups,
// lane p / ngroups) so that the busiest stores, which skewed demand puts at the
// low indices, fall into different CTAs.  Lanes of group g:
__device__ __forceinline__ int group_lanes(const OwArgs& a, int g) { return (a.P - 1 - g) / a.ngroups + 1; }

// Shared memory of the Picard kernel (dynamic; the network part only with H > 0).
struct __align__(16) OwSmem {
    int4 rec[kCh][kLanes];
    int4 pre[kCh][kLanes];
    int2 memo[kCh][kLanes];
    Mono ws[kOwThreads / 32 + 1];
    int feat_y[kLanes], feat_d[kLanes], feat_e[kLanes], feat_base[kLanes], feat_room[kLanes];
    int qout[kLanes];
    int rowidx[kLanes];
    int pend_any, pend_rows, all_done, abort, resume_q;
    unsigned long long full[kMaxBufSlots];  // W2 buffers: the copy landed
};

// Bytes of retailer stock in shared memory (16-byte multiple).
__host__ __device__ constexpr size_t xs_bytes(int n) { return ((size_t)n * 4 + 15) & ~(size_t)15; }

// ------------------------------------------------------------------ W2 staging
// W2 streams through shared memory in chunks of kKc rows (kKc * H BF16) moved
// by bulk asynchronous copies, nbuf buffers deep (as many as shared memory
// holds, at most kMaxBuf).  Chunk number `seq` (counted over the CTA's life,
// identically in every thread) uses buffer seq % nbuf; use u = seq / nbuf of
// that buffer completes phase u & 1 of its `full` mbarrier (the copy landed).
// 32 rows x 2 buffers measured fastest: a third buffer gains nothing, 16-row
// chunks pay one more barrier per chunk, and releasing buffers through
// per-warp mbarrier arrivals instead of __syncthreads was slower.
constexpr int kKc = 32;
constexpr int kMaxBuf = 2;
static_assert(kMaxBuf <= kMaxBufSlots, "one mbarrier per W2 buffer");

struct NetCtx {
    float *h1s, *W1s, *b1s, *b2s, *w3s;
    float2* zpart;  // [32][H/8] per row and 8-unit group: {sum w3 h2, sum |w3| h2}
    uint16_t* w2buf;  // [nbuf][kKc][H]
    unsigned long long* full;
    int nbuf;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void w2_issue(const NetCtx& nc, const uint16_t* W2, int H, int chunk,
                                         unsigned seq) {
    const int buf = seq % nc.nbuf;
    const unsigned bytes = (unsigned)(kKc * H * 2);
    unsigned long long* b = nc.full + buf;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(nc.w2buf + (size_t)buf * kKc * H)),
        "l"(W2 + (size_t)chunk * kKc * H), "r"(bytes), "r"(smem_u32(b))
        : "memory");
}

// Wait for phase `par` of mbarrier b; a wait past the kernel's deadline
// records a timeout and returns (the grid barrier then ends the kernel).
__device__ __forceinline__ void mbar_wait(unsigned long long* b, unsigned par, OwCtrl* oc,
                                          unsigned long long deadline) {
    for (unsigned it = 1;; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_u32(b)), "r"(par)
            : "memory");
        if (ok) return;
        if ((it & 1023u) == 0 && globaltimer_ns() > deadline) {
            atomicCAS(&oc->c.err, 0, (int)PIC_ERR_TIMEOUT);
            return;
        }
    }
}

// fma(a0, b0, c0) and fma(a1, b1, c1), each rounded once (fma.rn.f32x2: two
// fmaf results bit for bit).
__device__ __forceinline__ void fma2(float& c0, float& c1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%0, %1};\n\t"
        "fma.rn.f32x2 rc, ra, rb, rc;\n\tmov.b64 {%0, %1}, rc;\n\t}"
        : "+f"(c0), "+f"(c1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// Layer 2 for row groups of RPT compacted rows, CPT columns per thread
// (H / CPT threads per row group): acc = b2_j, then one fma per k in
// increasing k (the reference order); relu(acc) is written to the h2 table
// [row][H], which takes the place of h1s once every thread passed the last
// chunk.
template <int RPT, int CPT>
__device__ void net_layer2(const NetCtx& nc, const uint16_t* W2, int H, int nrowg,
                           unsigned& wuse, OwCtrl* oc, unsigned long long deadline) {
    const int tpr = H / CPT, nch = H / kKc;
    const bool active = (int)threadIdx.x < nrowg * tpr;
    const int rg = active ? (int)threadIdx.x / tpr : 0;
    const int col0 = ((int)threadIdx.x - rg * tpr) * CPT;
    float acc[RPT][CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const float bb = active ? nc.b2s[col0 + c] : 0.f;
#pragma unroll
        for (int r = 0; r < RPT; ++r) acc[r][c] = bb;
    }
    const unsigned nb = (unsigned)nc.nbuf;
    for (int ch = 0; ch < nch; ++ch) {
        const unsigned seq = wuse + ch;
        mbar_wait(nc.full + seq % nb, (seq / nb) & 1u, oc, deadline);
        if (active) {
            const uint16_t* wb = nc.w2buf + (size_t)(seq % nb) * kKc * H + col0;
            const float* hb = nc.h1s + (size_t)ch * kKc * kLanes + rg * RPT;
#pragma unroll 4
            for (int kk = 0; kk < kKc; ++kk) {
                float wf[CPT], hf[RPT];
                if constexpr (CPT == 8) {
                    const uint4 w = *reinterpret_cast<const uint4*>(wb + (size_t)kk * H);
                    wf[0] = bf_lo(w.x); wf[1] = bf_hi(w.x); wf[2] = bf_lo(w.y); wf[3] = bf_hi(w.y);
                    wf[4] = bf_lo(w.z); wf[5] = bf_hi(w.z); wf[6] = bf_lo(w.w); wf[7] = bf_hi(w.w);
                } else if constexpr (CPT == 4) {
                    const uint2 w = *reinterpret_cast<const uint2*>(wb + (size_t)kk * H);
                    wf[0] = bf_lo(w.x); wf[1] = bf_hi(w.x); wf[2] = bf_lo(w.y); wf[3] = bf_hi(w.y);
                } else {
                    const unsigned w = *reinterpret_cast<const unsigned*>(wb + (size_t)kk * H);
                    wf[0] = bf_lo(w); wf[1] = bf_hi(w);
                }
                if constexpr (RPT == 8) {
                    const float4 h0 = *reinterpret_cast<const float4*>(hb + kk * kLanes);
                    const float4 h1 = *reinterpret_cast<const float4*>(hb + kk * kLanes + 4);
                    hf[0] = h0.x; hf[1] = h0.y; hf[2] = h0.z; hf[3] = h0.w;
                    hf[4] = h1.x; hf[5] = h1.y; hf[6] = h1.z; hf[7] = h1.w;
                } else if constexpr (RPT == 4) {
                    const float4 h0 = *reinterpret_cast<const float4*>(hb + kk * kLanes);
                    hf[0] = h0.x; hf[1] = h0.y; hf[2] = h0.z; hf[3] = h0.w;
                } else if constexpr (RPT == 2) {
                    const float2 h0 = *reinterpret_cast<const float2*>(hb + kk * kLanes);
                    hf[0] = h0.x; hf[1] = h0.y;
                } else {
                    hf[0] = hb[kk * kLanes];
                }
                if constexpr (RPT % 2 == 0) {
                    // rows in pairs: two independent fmaf chains per instruction
#pragma unroll
                    for (int r = 0; r < RPT; r += 2)
#pragma unroll
                        for (int c = 0; c < CPT; ++c)
                            fma2(acc[r][c], acc[r + 1][c], wf[c], wf[c], hf[r], hf[r + 1]);
                } else {
#pragma unroll
                    for (int r = 0; r < RPT; ++r)
#pragma unroll
                        for (int c = 0; c < CPT; ++c) acc[r][c] = fmaf(wf[c], hf[r], acc[r][c]);
                }
            }
        }
        __syncthreads();  // every thread is done with buffer seq % nb: refill it
        if (threadIdx.x == 0 && ch + (int)nb < nch) w2_issue(nc, W2, H, ch + nb, seq + nb);
    }
    wuse += nch;
    __syncthreads();  // every warp is done with h1s and with this round's buffers
    if (active) {
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                nc.h1s[(size_t)(rg * RPT + r) * H + col0 + c] = acc[r][c] > 0.f ? acc[r][c] : 0.f;
    }
    __syncthreads();
}

// Layer 3 and the retailer rule for one row (h2: its H hidden values; zp: its
// H/8 group partials).  The fast output adds the partials in order,
// z = b3 + p_0 + p_1 + ... (each term rounded at most 8 + H/8 times, against H
// times in the reference chain z = b3, then one fma per unit), so
//   |z_fast - z_ref| <= (gamma_{8+H/8} + gamma_H) (|b3| + sum_j |w3_j| h2_j).
// q = clamp(floor(base + z), 0, room) is taken from z_fast when every z in
// that interval gives the same q (bounds rounded outwards); otherwise z is
// evaluated in the reference order.  Returns q; near: set on a re-score.
__device__ __forceinline__ int layer3_q(const NetCtx& nc, float b3, int H, const float* h2,
                                        const float2* zp, int base, int room, bool& near) {
    float z = b3, za = fabsf(b3);
    for (int g = 0; g < H / 8; ++g) {
        z = __fadd_rn(z, zp[g].x);
        za = __fadd_ru(za, zp[g].y);
    }
    // gamma_{8 + H/8} + gamma_H, with room for the partials' own roundings
    const float c = (float)(8 + H / 8 + H) * 5.9605e-8f * 1.002f;
    const float B = __fmul_ru(c, za);
    const float lo = floorf(__fadd_rd((float)base, __fsub_rd(z, B)));
    const float hi = floorf(__fadd_ru((float)base, __fadd_ru(z, B)));
    const float cl_lo = fminf(fmaxf(lo, 0.f), (float)room), cl_hi = fminf(fmaxf(hi, 0.f), (float)room);
    near = cl_lo != cl_hi;
    if (near) {
        z = b3;
        for (int j = 0; j < H; ++j) z = fmaf(nc.w3s[j], h2[j], z);
    }
    return q_of(base, room, z);
}

// One batched round of the network for the lanes flagged in `rows` (bit b =
// lane b, features in sm.feat_*).  The pending lanes are compacted; layer 1
// gives h1s [k][row] for nr rows, the smallest of 2, 4, 8, 16, 32 that holds
// them (ONE: a single row); layer 2 runs nr <= 8 rows x 2 columns per thread,
// or 8 rows x 4 / 8 columns for 16 / 32 rows; then the partials p_g (and their
// absolute counterparts) per (row, g) and layer3_q per row.  Every output
// follows the order documented in pic_owmr.h.
template <bool ONE>
__device__ void net_round(const OwArgs& a, OwSmem& sm, const NetCtx& nc, unsigned rows,
                          unsigned& wuse, unsigned long long deadline) {
    const int H = a.H, ncg = H >> 3, nch = H / kKc;
    const int m = __popc(rows);
    if (threadIdx.x == 0)
        for (int c = 0; c < nc.nbuf && c < nch; ++c) w2_issue(nc, a.W2, H, c, wuse + c);
    if (threadIdx.x < kLanes && ((rows >> threadIdx.x) & 1u))
        sm.rowidx[__popc(rows & ((1u << threadIdx.x) - 1u))] = threadIdx.x;
    __syncthreads();
    const int nr = ONE ? 1 : (m <= 2 ? 2 : (m <= 4 ? 4 : (m <= 8 ? 8 : (m <= 16 ? 16 : 32))));
    for (int idx = threadIdx.x; idx < H * nr; idx += blockDim.x) {
        const int k = idx / nr, i = idx - k * nr;
        float v = 0.f;
        if (i < m) {
            const int b = sm.rowidx[i];
            float acc = fmaf(nc.W1s[k], (float)sm.feat_y[b], nc.b1s[k]);
            acc = fmaf(nc.W1s[H + k], (float)sm.feat_d[b], acc);
            acc = fmaf(nc.W1s[2 * H + k], (float)sm.feat_e[b] * 0.000244140625f, acc);
            v = acc > 0.f ? acc : 0.f;
        }
        nc.h1s[k * kLanes + i] = v;
    }
    __syncthreads();
    if (ONE) {
        net_layer2<1, 2>(nc, a.W2, H, 1, wuse, a.oc, deadline);
    } else if (nr == 2) {
        net_layer2<2, 2>(nc, a.W2, H, 1, wuse, a.oc, deadline);
    } else if (nr == 4) {
        net_layer2<4, 2>(nc, a.W2, H, 1, wuse, a.oc, deadline);
    } else if (nr == 8) {
        net_layer2<8, 2>(nc, a.W2, H, 1, wuse, a.oc, deadline);
    } else if (nr == 16) {
        net_layer2<8, 4>(nc, a.W2, H, 2, wuse, a.oc, deadline);
    } else {
        net_layer2<8, 8>(nc, a.W2, H, 4, wuse, a.oc, deadline);
    }
    for (int idx = threadIdx.x; idx < m * ncg; idx += blockDim.x) {
        const int i = idx / ncg, g = idx - i * ncg;
        const float* h2 = nc.h1s + (size_t)i * H + 8 * g;
        float p = 0.f, pa = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            p = fmaf(nc.w3s[8 * g + c], h2[c], p);
            pa = fmaf(fabsf(nc.w3s[8 * g + c]), h2[c], pa);
        }
        nc.zpart[i * ncg + g] = make_float2(p, pa);
    }
    __syncthreads();
    if ((int)threadIdx.x < m) {
        const int b = sm.rowidx[threadIdx.x];
        bool near = false;
        sm.qout[b] = layer3_q(nc, bf1(a.b3[0]), H, nc.h1s + (size_t)threadIdx.x * H,
                              nc.zpart + threadIdx.x * ncg, sm.feat_base[b], sm.feat_room[b], near);
        if (near) atomicAdd(&a.oc->near, 1ull);
    }
    __syncthreads();
}

// Carve the network's shared memory after OwSmem: h1s [H][32] (h2 [32][H]
// later), zpart [32][H/8] (float2), W1s [3][H], b1s, b2s, w3s [H], W2 buffers;
// stage the small weights and initialise the mbarriers.
__device__ NetCtx net_setup(const OwArgs& a, unsigned char* smem_raw, OwSmem& sm) {
    NetCtx nc;
    const int H = a.H;
    nc.h1s = reinterpret_cast<float*>(smem_raw + sizeof(OwSmem) + xs_bytes(a.xs_len));
    nc.zpart = reinterpret_cast<float2*>(nc.h1s + H * kLanes);
    nc.W1s = reinterpret_cast<float*>(nc.zpart + kLanes * (H >> 3));
    nc.b1s = nc.W1s + 3 * H;
    nc.b2s = nc.b1s + H;
    nc.w3s = nc.b2s + H;
    nc.w2buf = reinterpret_cast<uint16_t*>(nc.w3s + H);
    nc.full = sm.full;
    nc.nbuf = a.nbuf;
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        nc.W1s[i] = bf1(a.W1[i]);
        nc.W1s[H + i] = bf1(a.W1[H + i]);
        nc.W1s[2 * H + i] = bf1(a.W1[2 * H + i]);
        nc.b1s[i] = bf1(a.b1[i]);
        nc.b2s[i] = bf1(a.b2[i]);
        nc.w3s[i] = bf1(a.w3[i]);
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < nc.nbuf; ++i) mbar_init(nc.full + i, 1);
        fence_mbar_init();
    }
    __syncthreads();
    return nc;
}

size_t net_fixed_smem(int H) {
    return sizeof(float) * ((size_t)H * kLanes + 2 * (size_t)kLanes * (H / 8) + 6 * (size_t)H);
}

// Phases A and B of pass `pass`: tile summaries of the cache, a grid barrier,
// then pre[t] = {Qc, D, LR, alpha_t} for the CTA's contiguous tiles (and
// pre[T]), and a second grid barrier.  Tiles that end at or before `wstart`
// (the previous pass's first change) keep last pass's summaries and records:
// the cache before wstart did not change.  Returns false when a barrier failed.
__device__ bool prefix_phases(const OwArgs& a, OwCtrl* oc, Mono* ws, int tile0, int tile1,
                              int pass, unsigned long long deadline, int wstart) {
    const int tid = threadIdx.x;
    const int tb = max(tile0, wstart / kTile);  // first tile this pass recomputes
    for (int tile = tb; tile < tile1; ++tile) {
        const long long base = (long long)tile * kTile + tid * kItems;
        Mono m = mono_id();
#pragma unroll 4
        for (int i = 0; i < kItems; ++i) {
            const long long t = base + i;
            if (t < a.T) m = mono_step(m, (int)t, a.act[t]);
        }
        Mono tot;
        block_exscan_mono(m, &tot, ws);
        if (tid == 0) a.tsum[tile] = make_int4(tot.sq, tot.lr, tot.da, 0);
    }
    if (!grid_sync(&oc->c, deadline)) return false;
    if (blockIdx.x == 0 && tid == 0) {
        const int nx = (pass + 1) % 3;
        oc->changed[nx] = 0;
        oc->fct[nx] = INT_MAX;
        oc->lost[nx] = oc->shipped[nx] = oc->R[nx] = 0;
    }
    if (tb < tile1 || (blockIdx.x == 0 && a.T == 0)) {
        // prefix of the tiles before tb
        Mono m = mono_id();
        const int per = (tb + kOwThreads - 1) / kOwThreads;
        for (int i = 0; i < per; ++i) {
            const int tl = tid * per + i;
            if (tl < tb) {
                const int4 s4 = a.tsum[tl];
                m = mono_cat(m, Mono{s4.x, s4.y, s4.z});
            }
        }
        Mono run;
        block_exscan_mono(m, &run, ws);
        for (int tile = tb; tile < tile1; ++tile) {
            const long long base = (long long)tile * kTile + tid * kItems;
            Mono loc = mono_id();
            for (int i = 0; i < kItems; ++i) {
                const long long t = base + i;
                if (t < a.T) loc = mono_step(loc, (int)t, a.act[t]);
            }
            Mono tot;
            Mono ex = block_exscan_mono(loc, &tot, ws);
            Mono cur = mono_cat(run, ex);
            for (int i = 0; i < kItems; ++i) {
                const long long t = base + i;
                if (t < a.T) {
                    const int v = a.act[t];
                    a.pre[t] = make_int4(cur.sq, cur.da, cur.lr, v);
                    cur = mono_step(cur, (int)t, v);
                    if (t == a.T - 1) a.pre[a.T] = make_int4(cur.sq, cur.da, cur.lr, 0);
                }
            }
            run = mono_cat(run, tot);
        }
        if (a.T == 0 && blockIdx.x == 0 && tid == 0) a.pre[0] = make_int4(0, 0, -1, 0);
    }
    return grid_sync(&oc->c, deadline);
}

// ------------------------------------------------------------------ Picard kernel
template <bool NET>
__global__ void __launch_bounds__(kOwThreads, 1) k_owmr_picard(OwArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OwSmem& sm = *reinterpret_cast<OwSmem*>(smem_raw);
    int* xs = reinterpret_cast<int*>(smem_raw + sizeof(OwSmem));  // [rp * 32] retailer stock
    OwCtrl* oc = a.oc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long deadline = globaltimer_ns() + (unsigned long long)a.timeout_ns;
    NetCtx nc{};
    unsigned wuse = 0;  // W2 chunks consumed by this CTA
    if (NET) nc = net_setup(a, smem_raw, sm);
    // contiguous tile range of this CTA (phases A and B)
    const int tpc = (a.ntiles + gridDim.x - 1) / gridDim.x;
    const int tile0 = min(a.ntiles, (int)blockIdx.x * tpc), tile1 = min(a.ntiles, tile0 + tpc);
    if (blockIdx.x == 0 && tid == 0)
        for (int i = 0; i < 3; ++i) oc->fct[i] = INT_MAX;
    int w = 0;  // window start (identical in every CTA)

    for (int pass = 1;; ++pass) {
        const int slot = pass % 3;
        const int whi = a.window > 0 ? (int)min((long long)a.T, (long long)w + a.window) : a.T;
        if (!prefix_phases(a, oc, sm.ws, tile0, tile1, pass, deadline, w)) break;
        // ---------------- phase C: walks
        int my_changed = 0, my_first = INT_MAX;
        long long my_lost = 0, my_ship = 0, my_R = 0;
        unsigned long long my_evals = 0, my_rounds = 0;
        for (int g = blockIdx.x; g < a.ngroups; g += gridDim.x) {
            const int nb = group_lanes(a, g);
            // stock of the group's retailers: slot j * 32 + lane for n = lane_proc + j P
            for (int i = tid; i < a.rp * kLanes; i += kOwThreads) {
                const int l = i & 31, j = i >> 5;
                const long long n = (long long)l * a.ngroups + g + (long long)j * a.P;
                if (l < nb && n < a.N) xs[i] = a.x0r[n];
            }
            // per-lane walk state (warp 0); gl_*: the lane's statistics over its steps
            int x0a = a.X0, ta = -1, qc_after = 0, done = 0, wdone = 0;
            int pend = 0, pt = 0, px0 = 0, py = 0, pold = 0, pqc = 0, pslot = 0;
            long long gl_lost = 0;
            int gl_ship = 0, gl_R = 0;
            const long long row0 = a.gbase[g], row1 = a.gbase[g + 1];
            long long rstart = row0;
            if (a.resume && w > 0) {
                // the last chunk whose lanes' states precede w (keys increase along the group)
                if (warp == 0) {
                    const int q0 = (int)(row0 / kCh), q1 = (int)(row1 / kCh);
                    int best = q0;
                    for (int qb = q0; qb < q1; qb += 32) {
                        const int q = qb + lane;
                        const unsigned m = __ballot_sync(kFull, q < q1 && a.cmax[q] < w);
                        if (m) best = qb + 31 - __clz(m);
                        if (m != kFull) break;
                    }
                    if (lane == 0) sm.resume_q = best;
                }
                __syncthreads();
                rstart = (long long)sm.resume_q * kCh;
                if (rstart > row0 && warp == 0 && lane < nb) {
                    const size_t q = (size_t)sm.resume_q * 2 * kLanes;
                    const int4 c0 = a.ckpt[q + lane], c1 = a.ckpt[q + kLanes + lane];
                    x0a = c0.x;
                    ta = c0.y;
                    qc_after = c0.z;
                    xs[lane] = c0.w;
                    gl_lost = (long long)(((unsigned long long)(unsigned)c1.y << 32) | (unsigned)c1.x);
                    gl_ship = c1.z;
                    gl_R = c1.w;
                }
            }
            for (long long r0 = rstart; r0 < row1; r0 += kCh) {
                if (a.resume && warp == 0 && lane < nb && !wdone) {
                    // state before this chunk (lanes that stopped at the window end excepted)
                    const size_t q = (size_t)(r0 / kCh) * 2 * kLanes;
                    a.ckpt[q + lane] = make_int4(x0a, ta, qc_after, xs[lane]);
                    a.ckpt[q + kLanes + lane] =
                        make_int4((int)(unsigned)(unsigned long long)gl_lost,
                                  (int)(unsigned)((unsigned long long)gl_lost >> 32), gl_ship, gl_R);
                }
                __syncthreads();
                for (int i = tid; i < kCh * kLanes; i += kOwThreads)
                    (&sm.rec[0][0])[i] = a.rec[r0 * kLanes + i];
                if (NET)
                    for (int i = tid; i < kCh * kLanes; i += kOwThreads)
                        (&sm.memo[0][0])[i] = a.memo[r0 * kLanes + i];
                __syncthreads();
                for (int i = tid; i < kCh * kLanes; i += kOwThreads) {
                    const int t = (&sm.rec[0][0])[i].x;
                    if (t >= 0) (&sm.pre[0][0])[i] = a.pre[t];
                }
                __syncthreads();
                int pos = 0;
                for (;;) {
                    if (warp == 0) {
                        bool parked = false;
                        if (lane < nb) {
                            if (NET && pend) {
                                // finish the parked step with the round's q
                                const int q = sm.qout[lane];
                                const long long mi = (r0 + pos) * kLanes + lane;
                                a.memo[mi] = make_int2(py, q);
                                const int r = px0 - q <= a.s;
                                const int recv = q < px0 ? q : px0;
                                xs[pslot] = py + recv;
                                gl_ship += recv;
                                gl_R += r;
                                x0a = r ? a.S : (px0 > q ? px0 - q : 0);
                                qc_after = pqc + (pold >> 1);
                                ta = pt;
                                const int nv = 2 * q + r;
                                if (nv != pold) {
                                    a.act[pt] = nv;
                                    if (!my_changed) my_first = pt;
                                    ++my_changed;
                                }
                                pend = 0;
                                ++pos;
                            }
                            while (pos < kCh) {
                                const int4 rc = sm.rec[pos][lane];
                                if (rc.x < 0 || rc.x >= whi) {  // list end or window end
                                    pos = kCh;
                                    done = 1;
                                    wdone = rc.x >= 0;
                                    break;
                                }
                                const int t = rc.x, n = rc.y, d = rc.z;
                                const int4 pr = sm.pre[pos][lane];  // {Qc, D, LR, old}
                                int x0 = pr.z > ta ? a.S - pr.y : x0a - (pr.x - qc_after);
                                x0 = x0 > 0 ? x0 : 0;
                                const int slotn = (n / a.P) * kLanes + lane;
                                const int xn = xs[slotn];
                                const int y = xn > d ? xn - d : 0;
                                gl_lost += d > xn ? d - xn : 0;
                                const int base = retailer_base(y, __ldg(a.sl + n), __ldg(a.Sl + n));
                                const int room = __ldg(a.cap + n) - y;
                                int q;
                                if (NET) {
                                    const int2 mm = sm.memo[pos][lane];
                                    if (mm.x != y) {
                                        pend = 1;
                                        pt = t; px0 = x0; py = y; pold = pr.w;
                                        pqc = pr.x; pslot = slotn;
                                        sm.feat_y[lane] = y;
                                        sm.feat_d[lane] = d;
                                        sm.feat_e[lane] = rc.w;
                                        sm.feat_base[lane] = base;
                                        sm.feat_room[lane] = room;
                                        parked = true;
                                        break;
                                    }
                                    q = mm.y;
                                } else {
                                    q = base < room ? base : room;
                                }
                                const int r = x0 - q <= a.s;
                                const int recv = q < x0 ? q : x0;
                                xs[slotn] = y + recv;
                                gl_ship += recv;
                                gl_R += r;
                                x0a = r ? a.S : (x0 > q ? x0 - q : 0);
                                qc_after = pr.x + (pr.w >> 1);
                                ta = t;
                                const int nv = 2 * q + r;
                                if (nv != pr.w) {
                                    a.act[t] = nv;
                                    if (!my_changed) my_first = t;
                                    ++my_changed;
                                }
                                ++pos;
                            }
                        }
                        const unsigned rows = __ballot_sync(kFull, parked);
                        const bool all = __all_sync(kFull, done || lane >= nb);
                        if (lane == 0) {
                            sm.pend_rows = (int)rows;
                            sm.pend_any = rows != 0u;
                            sm.all_done = all;
                            sm.abort = ld_volatile(&oc->c.err) != 0;  // one CTA-wide decision
                        }
                    }
                    __syncthreads();
                    if (!NET || !sm.pend_any || sm.abort) break;
                    const unsigned rows = (unsigned)sm.pend_rows;
                    net_round<false>(a, sm, nc, rows, wuse, deadline);
                    if (tid == 0) {
                        my_evals += __popc(rows);
                        ++my_rounds;
                    }
                }
                if (sm.all_done || sm.abort) break;  // lists or window done, or a wait timed out
            }
            __syncthreads();
            for (int i = tid; i < a.rp * kLanes; i += kOwThreads) {
                const int l = i & 31, j = i >> 5;
                const long long n = (long long)l * a.ngroups + g + (long long)j * a.P;
                if (l < nb && n < a.N) a.xfin[n] = xs[i];
            }
            my_lost += gl_lost;
            my_ship += gl_ship;
            my_R += gl_R;
        }
        // CTA totals
        if (warp == 0) {
            const int ch = __reduce_add_sync(kFull, my_changed);
            const int fmin = __reduce_min_sync(kFull, my_first);
            const long long lo = warp_sum_i64(my_lost), sh = warp_sum_i64(my_ship),
                            rr = warp_sum_i64(my_R);
            if (lane == 0) {
                if (ch) {
                    atomicAdd(&oc->changed[slot], ch);
                    atomicMin(&oc->fct[slot], fmin);
                }
                if (lo) atomicAdd((unsigned long long*)&oc->lost[slot], (unsigned long long)lo);
                if (sh) atomicAdd((unsigned long long*)&oc->shipped[slot], (unsigned long long)sh);
                if (rr) atomicAdd((unsigned long long*)&oc->R[slot], (unsigned long long)rr);
            }
        }
        if (tid == 0 && my_evals) {
            atomicAdd(&oc->evals, my_evals);
            atomicAdd(&oc->rounds, my_rounds);
        }
        if (!grid_sync(&oc->c, deadline)) break;
        const int changed = ld_volatile(&oc->changed[slot]);
        const bool fixed = changed == 0 && whi >= a.T;
        if (fixed || pass >= a.max_iters) {
            if (blockIdx.x == 0 && tid == 0) {
                oc->c.iters = pass;
                oc->c.converged = fixed;
                oc->c.pad0 = slot;
            }
            break;
        }
        w = changed ? ld_volatile(&oc->fct[slot]) : whi;
    }
}

// ------------------------------------------------------------------ sequential baseline
// One CTA walks the horizon one step at a time.  With a network, thread 0
// prepares each step and the CTA evaluates it as a one-row round (W2 streamed
// through shared memory, 2 layer-2 units per thread); without one, one warp
// runs the steps.  Retailer stock sits in shared memory when N <= 4096.
template <bool NET>
__global__ void __launch_bounds__(kOwThreads, 1) k_owmr_seq(OwArgs a, int32_t* xs_g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OwSmem& sm = *reinterpret_cast<OwSmem*>(smem_raw);
    int* xs = a.xs_len ? reinterpret_cast<int*>(smem_raw + sizeof(OwSmem)) : xs_g;
    const int tid = threadIdx.x;
    const unsigned long long deadline = globaltimer_ns() + (unsigned long long)a.timeout_ns;
    NetCtx nc{};
    unsigned wuse = 0;
    if (NET) nc = net_setup(a, smem_raw, sm);
    for (int n = tid; n < a.N; n += blockDim.x) xs[n] = a.x0r[n];
    __syncthreads();
    int x0 = a.X0;
    long long lost = 0, ship = 0, R = 0;
    unsigned long long evals = 0;
    if (!NET) {
        if (tid < 32) {
            for (long long t0 = 0; t0 < a.T; t0 += 32) {
                const long long tt = t0 + tid;
                const int4 rc = tt < a.T ? a.rec[tt] : make_int4(-1, 0, 0, 0);
                for (int j = 0; j < 32 && t0 + j < a.T; ++j) {
                    const int n = __shfl_sync(kFull, rc.y, j), d = __shfl_sync(kFull, rc.z, j);
                    if (tid == 0) {
                        const int xn = xs[n];
                        const int y = xn > d ? xn - d : 0;
                        lost += d > xn ? d - xn : 0;
                        const int base = retailer_base(y, a.sl[n], a.Sl[n]);
                        const int room = a.cap[n] - y;
                        const int q = base < room ? base : room;
                        const int r = x0 - q <= a.s;
                        const int recv = q < x0 ? q : x0;
                        xs[n] = y + recv;
                        ship += recv;
                        R += r;
                        x0 = r ? a.S : (x0 > q ? x0 - q : 0);
                        a.act[t0 + j] = 2 * q + r;
                    }
                }
            }
        }
    } else {
        for (long long t = 0; t < a.T; ++t) {
            int n = 0, y = 0;
            if (tid == 0) {
                const int4 rc = a.rec[t];
                n = rc.y;
                const int d = rc.z;
                const int xn = xs[n];
                y = xn > d ? xn - d : 0;
                lost += d > xn ? d - xn : 0;
                sm.feat_y[0] = y;
                sm.feat_d[0] = d;
                sm.feat_e[0] = rc.w;
                sm.feat_base[0] = retailer_base(y, a.sl[n], a.Sl[n]);
                sm.feat_room[0] = a.cap[n] - y;
            }
            __syncthreads();
            net_round<true>(a, sm, nc, 1u, wuse, deadline);
            if (tid == 0) {
                const int q = sm.qout[0];
                const int r = x0 - q <= a.s;
                const int recv = q < x0 ? q : x0;
                xs[n] = y + recv;
                ship += recv;
                R += r;
                x0 = r ? a.S : (x0 > q ? x0 - q : 0);
                a.act[t] = 2 * q + r;
                ++evals;
            }
            if (ld_volatile(&a.oc->c.err)) break;
        }
    }
    __syncthreads();
    for (int n = tid; n < a.N; n += blockDim.x) a.xfin[n] = xs[n];
    if (tid == 0) {
        OwCtrl* oc = a.oc;
        oc->lost[0] = lost;
        oc->shipped[0] = ship;
        oc->R[0] = R;
        oc->evals = evals;
        oc->c.pad0 = 0;
        oc->c.iters = 0;
        oc->c.converged = 1;
        a.pre[0] = make_int4(x0, 0, 0, 0);  // final central stock for the host
    }
}

// ------------------------------------------------------------------ tables
__global__ void k_ow_validate(int T, int N, const int32_t* __restrict__ ret,
                              const int32_t* __restrict__ dem, const int32_t* __restrict__ ex,
                              const int32_t* __restrict__ cap,
                              const int32_t* __restrict__ x0r, const int32_t* __restrict__ sl,
                              const int32_t* __restrict__ Sl, int* bad, int* maxcap) {
    int b = 0, mc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < T;
         i += (long long)gridDim.x * blockDim.x) {
        if (ret[i] < 0 || ret[i] >= N) b |= 1;
        if (dem[i] < 0 || dem[i] >= 32768) b |= 2;
        if (ex[i] < 0 || ex[i] >= 32768) b |= 32;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = cap[i];
        if (c < 0 || c >= (1 << 20)) b |= 4;
        if (x0r[i] < 0 || x0r[i] > c) b |= 8;
        if (sl[i] < 0 || Sl[i] < sl[i] || Sl[i] > c) b |= 16;
        mc = max(mc, c);
    }
    if (b) atomicOr(bad, b);
    if (mc) atomicMax(maxcap, mc);
}

__global__ void k_ow_keys(int T, int P, const int32_t* __restrict__ ret, int32_t* __restrict__ key,
                          int32_t* __restrict__ cnt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < T;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = ret[i] % P;
        key[i] = p;
        atomicAdd(cnt + p, 1);
    }
}

__global__ void k_ow_group_rows(int P, int B, int ngroups, const int32_t* __restrict__ cnt,
                                int32_t* __restrict__ rows) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngroups) return;
    int m = 0;
    for (long long p = g; p < P; p += ngroups) m = max(m, cnt[p]);  // lanes of group g
    rows[g] = (m + kCh - 1) / kCh * kCh;
}

__global__ void k_ow_rec(int T, int ngroups, const int32_t* __restrict__ key_s,
                         const int32_t* __restrict__ perm, const int32_t* __restrict__ off,
                         const int32_t* __restrict__ gbase, const int32_t* __restrict__ ret,
                         const int32_t* __restrict__ dem, const int32_t* __restrict__ ex,
                         int4* __restrict__ rec, int32_t* __restrict__ lastt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < T;
         i += (long long)gridDim.x * blockDim.x) {
        const int p = key_s[i], j = (int)(i - off[p]), g = p % ngroups, l = p / ngroups;
        const int t = perm[i];
        rec[((long long)gbase[g] + j) * kLanes + l] = make_int4(t, ret[t], dem[t], ex[t]);
        if (j == off[p + 1] - off[p] - 1) lastt[g * kLanes + l] = t;  // the lane's last step
    }
}

// Per chunk (kCh rows of one group), the latest over its lanes of the time that
// the lane's state before the chunk depends on: its first step in the chunk, or
// its last step when its list ended earlier (-1: no steps).  A lane's state
// before the chunk is unchanged by a pass whose first change is after that time.
__global__ void k_ow_cmax(const int32_t* __restrict__ gbase, const int4* __restrict__ rec,
                          const int32_t* __restrict__ lastt, int32_t* __restrict__ cmax) {
    const int g = blockIdx.x, lane = threadIdx.x;
    const int lt = lastt[g * kLanes + lane];
    for (long long r = gbase[g]; r < gbase[g + 1]; r += kCh) {
        int v = rec[r * kLanes + lane].x;
        if (v < 0) v = lt;
        v = __reduce_max_sync(kFull, v);
        if (lane == 0) cmax[r / kCh] = v;
    }
}

__global__ void k_ow_time_rec(int T, const int32_t* __restrict__ ret,
                              const int32_t* __restrict__ dem, const int32_t* __restrict__ ex,
                              int4* __restrict__ rec) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < T;
         i += (long long)gridDim.x * blockDim.x)
        rec[i] = make_int4((int)i, ret[i], dem[i], ex[i]);
}

__global__ void k_ow_check_init(int T, const int32_t* __restrict__ init, int maxcap, int* bad) {
    int b = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < T;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = init[i];
        if (v < 0 || (v >> 1) > maxcap) b = 1;
    }
    if (b) atomicOr(bad, 32);
}

inline int nblk(long long n, int per) { return (int)((n + per - 1) / per); }

}  // namespace

// ------------------------------------------------------------------ handle
struct pic_owmr {
    int T = 0, N = 0, X0 = 0, s = 0, S = 0, maxcap = 0, num_sms = 0, max_smem = 0;
    int32_t *ret = nullptr, *dem = nullptr, *ex = nullptr, *cap = nullptr, *x0r = nullptr, *sl = nullptr,
            *Sl = nullptr;
    int32_t* act = nullptr;
    int4* pre = nullptr;
    int32_t* xfin = nullptr;
    int* bad = nullptr;
    OwCtrl* oc = nullptr;
    // tables of the current processor count
    int P = 0, B = 0, ngroups = 0, ctas = 0;
    long long rows = 0;
    int4* rec = nullptr;   // interleaved step records of the Picard walks
    int4* trec = nullptr;  // time-order records for the sequential kernel
    int2* memo = nullptr;
    int32_t* cmax = nullptr;
    int32_t* lastt = nullptr;
    int4* ckpt = nullptr;
    int32_t* gbase = nullptr;
    int4* tsum = nullptr;
    int ntiles = 0;
};

namespace {

void free_tables(pic_owmr* h) {
    cudaFree(h->rec);
    cudaFree(h->memo);
    cudaFree(h->cmax);
    cudaFree(h->lastt);
    cudaFree(h->ckpt);
    h->cmax = h->lastt = nullptr;
    h->ckpt = nullptr;
    cudaFree(h->gbase);
    h->rec = nullptr;
    h->memo = nullptr;
    h->gbase = nullptr;
    h->P = 0;
}

pic_status build_tables(pic_owmr* h, int P, int ctas, cudaStream_t st, int* launches) {
    if (h->P == P && h->ctas == ctas) return PIC_OK;
    free_tables(h);
    const int T = h->T;
    int B = (P + ctas - 1) / ctas;
    B = B < 1 ? 1 : (B > kLanes ? kLanes : B);
    const int ngroups = (P + B - 1) / B;
    int32_t *key = nullptr, *key_s = nullptr, *perm = nullptr, *tk = nullptr, *tv = nullptr,
            *cnt = nullptr, *off = nullptr, *grows = nullptr, *hist = nullptr, *blk = nullptr,
            *serr = nullptr;  // set when a scan's look-back wait gives up
    const int Tn = T > 0 ? T : 1;
    const int hl = sort_hist_len(Tn);
    const int bl = scan_blk_len(hl > P + 1 ? hl : P + 1) + scan_blk_len(ngroups + 1) + 2;
    cudaError_t e = cudaSuccess;
    auto A = [&](int32_t** p, size_t n) {
        if (!e) e = cudaMalloc(p, n * sizeof(int32_t));
    };
    A(&key, Tn); A(&key_s, Tn); A(&perm, Tn); A(&tk, Tn); A(&tv, Tn); A(&cnt, (size_t)P + 1);
    A(&off, (size_t)P + 1); A(&grows, (size_t)ngroups + 1); A(&hist, hl); A(&blk, bl);
    A(&h->gbase, (size_t)ngroups + 1);
    A(&serr, 1);
    pic_status ps = PIC_OK;
    if (!e) e = cudaMemsetAsync(blk, 0, sizeof(int32_t) * (size_t)bl, st);  // scan epoch and words
    if (!e) e = cudaMemsetAsync(serr, 0, sizeof(int32_t), st);
    if (!e) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (P + 1), st);
    if (!e && T > 0) {
        k_ow_keys<<<nblk(T, 256) < 4096 ? nblk(T, 256) : 4096, 256, 0, st>>>(T, P, h->ret, key, cnt);
        e = sort_pairs_raw(key, T, P - 1, key_s, perm, tk, tv, hist, blk, st, serr);
        int passes = 1;
        while (passes < 4 && ((unsigned)(P - 1) >> (8 * passes)) != 0) ++passes;
        *launches += 1 + 3 * passes;
    }
    if (!e) e = scan_exclusive(cnt, off, P + 1, nullptr, blk, st, serr);
    if (!e) {
        k_ow_group_rows<<<nblk(ngroups, 256), 256, 0, st>>>(P, B, ngroups, cnt, grows);
        e = cudaMemsetAsync(grows + ngroups, 0, sizeof(int32_t), st);
    }
    if (!e) e = scan_exclusive(grows, h->gbase, ngroups + 1, nullptr, blk, st, serr);
    *launches += 3;
    int rows_total = 0, scan_err = 0;
    if (!e) e = cudaMemcpyAsync(&rows_total, h->gbase + ngroups, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaMemcpyAsync(&scan_err, serr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (!e && !scan_err) {  // rows_total sizes the record tables: only from a completed scan
        const size_t nrec = (size_t)(rows_total > 0 ? rows_total : 1) * kLanes;
        const size_t nchunk = nrec / ((size_t)kCh * kLanes) + 1;
        e = cudaMalloc(&h->rec, nrec * sizeof(int4));
        if (!e) e = cudaMalloc(&h->memo, nrec * sizeof(int2));
        if (!e) e = cudaMalloc(&h->cmax, nchunk * sizeof(int32_t));
        if (!e) e = cudaMalloc(&h->lastt, (size_t)ngroups * kLanes * sizeof(int32_t));
        if (!e) e = cudaMalloc(&h->ckpt, nchunk * 2 * kLanes * sizeof(int4));
        if (!e) e = cudaMemsetAsync(h->rec, 0xff, nrec * sizeof(int4), st);
        if (!e) e = cudaMemsetAsync(h->lastt, 0xff, (size_t)ngroups * kLanes * sizeof(int32_t), st);
        if (!e && T > 0) {
            k_ow_rec<<<nblk(T, 256) < 4096 ? nblk(T, 256) : 4096, 256, 0, st>>>(
                T, ngroups, key_s, perm, off, h->gbase, h->ret, h->dem, h->ex, h->rec, h->lastt);
            *launches += 1;
        }
        if (!e) {
            k_ow_cmax<<<ngroups, kLanes, 0, st>>>(h->gbase, h->rec, h->lastt, h->cmax);
            *launches += 1;
        }
    }
    if (!e) e = cudaStreamSynchronize(st);
    cudaFree(key); cudaFree(key_s); cudaFree(perm); cudaFree(tk); cudaFree(tv); cudaFree(cnt);
    cudaFree(off); cudaFree(grows); cudaFree(hist); cudaFree(blk); cudaFree(serr);
    if (!e && scan_err) {
        free_tables(h);
        return fail(PIC_ERR_TIMEOUT, "OWMR tables: a prefix scan's wait for an earlier tile exceeded its bound");
    }
    if (e) {
        free_tables(h);
        return fail(e == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA,
                    "OWMR tables: %s", cudaGetErrorString(e));
    }
    h->P = P;
    h->ctas = ctas;
    h->B = B;
    h->ngroups = ngroups;
    h->rows = rows_total;
    return ps;
}

// Dynamic shared memory: OwSmem, retailer stock, and with a network its fixed
// part plus nbuf W2 buffers (as many as the opt-in limit allows, 2..8).
size_t owmr_smem(int H, int xs_len, int max_smem, int* nbuf) {
    size_t s = sizeof(OwSmem) + xs_bytes(xs_len);
    *nbuf = 0;
    if (H) {
        s += net_fixed_smem(H);
        const size_t chunk = (size_t)kKc * H * 2;
        long long room = (long long)max_smem - 1024 - (long long)s;  // 1 KB for static smem
        int nb = room > 0 ? (int)(room / (long long)chunk) : 0;
        nb = nb > kMaxBuf ? kMaxBuf : nb;
        *nbuf = nb;
        s += (size_t)(nb > 0 ? nb : 0) * chunk;
    }
    return s;
}

}  // namespace

extern "C" {

pic_status pic_owmr_create(const pic_owmr_desc* d, pic_owmr** out) {
    if (!d || !out) return fail(PIC_ERR_INVALID_ARG, "desc and out are required");
    *out = nullptr;
    if (d->T < 0 || d->N < 1 || d->N > 65536)
        return fail(PIC_ERR_INVALID_ARG, "need 0 <= T and 1 <= N <= 65536");
    if ((d->T > 0 && (!d->ret || !d->dem || !d->ex)) || !d->cap || !d->x0r || !d->sl || !d->Sl)
        return fail(PIC_ERR_INVALID_ARG, "missing input array");
    if (d->mem != PIC_MEM_HOST && d->mem != PIC_MEM_DEVICE)
        return fail(PIC_ERR_INVALID_ARG, "unknown mem %d", d->mem);
    if (d->s < 0 || d->S <= d->s || d->S >= (1 << 30) || d->X0 < 0 || d->X0 >= (1 << 30))
        return fail(PIC_ERR_INVALID_ARG, "need 0 <= s < S < 2^30 and 0 <= X0 < 2^30");
    pic_owmr* h = new (std::nothrow) pic_owmr();
    if (!h) return fail(PIC_ERR_OOM, "host allocation failed");
    cudaStream_t st = (cudaStream_t)d->stream;
    h->T = d->T; h->N = d->N; h->X0 = d->X0; h->s = d->s; h->S = d->S;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaDeviceGetAttribute(&h->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t Tn = d->T > 0 ? (size_t)d->T : 1;
    auto A = [&](void** p, size_t bytes) {
        if (!e) e = cudaMalloc(p, bytes);
    };
    A((void**)&h->ret, Tn * 4); A((void**)&h->dem, Tn * 4); A((void**)&h->ex, Tn * 4); A((void**)&h->cap, (size_t)d->N * 4);
    A((void**)&h->x0r, (size_t)d->N * 4); A((void**)&h->sl, (size_t)d->N * 4);
    A((void**)&h->Sl, (size_t)d->N * 4); A((void**)&h->act, Tn * 4);
    A((void**)&h->pre, (Tn + 1) * sizeof(int4)); A((void**)&h->xfin, (size_t)d->N * 4);
    A((void**)&h->bad, 2 * sizeof(int)); A((void**)&h->oc, sizeof(OwCtrl));
    A((void**)&h->trec, Tn * sizeof(int4));
    h->ntiles = nblk(d->T, kTile);
    A((void**)&h->tsum, (size_t)(h->ntiles > 0 ? h->ntiles : 1) * sizeof(int4));
    const cudaMemcpyKind k = d->mem == PIC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (!e && d->T > 0) e = cudaMemcpyAsync(h->ret, d->ret, (size_t)d->T * 4, k, st);
    if (!e && d->T > 0) e = cudaMemcpyAsync(h->dem, d->dem, (size_t)d->T * 4, k, st);
    if (!e && d->T > 0) e = cudaMemcpyAsync(h->ex, d->ex, (size_t)d->T * 4, k, st);
    if (!e) e = cudaMemcpyAsync(h->cap, d->cap, (size_t)d->N * 4, k, st);
    if (!e) e = cudaMemcpyAsync(h->x0r, d->x0r, (size_t)d->N * 4, k, st);
    if (!e) e = cudaMemcpyAsync(h->sl, d->sl, (size_t)d->N * 4, k, st);
    if (!e) e = cudaMemcpyAsync(h->Sl, d->Sl, (size_t)d->N * 4, k, st);
    if (!e) e = cudaMemsetAsync(h->bad, 0, 2 * sizeof(int), st);
    if (!e) e = cudaMemsetAsync(h->oc, 0, sizeof(OwCtrl), st);
    int hb[2] = {0, 0};
    if (!e) {
        const long long n = d->T > d->N ? d->T : d->N;
        k_ow_validate<<<nblk(n, 256) < 1024 ? nblk(n, 256) : 1024, 256, 0, st>>>(
            d->T, d->N, h->ret, h->dem, h->ex, h->cap, h->x0r, h->sl, h->Sl, h->bad, h->bad + 1);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(hb, h->bad, sizeof(hb), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    pic_status ps = PIC_OK;
    if (e) ps = fail(e == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA, "OWMR create: %s",
                     cudaGetErrorString(e));
    else if (hb[0] & 1) ps = fail(PIC_ERR_INVALID_ARG, "ret[t] outside [0, N)");
    else if (hb[0] & 2) ps = fail(PIC_ERR_INVALID_ARG, "dem[t] outside [0, 32768)");
    else if (hb[0] & 32) ps = fail(PIC_ERR_INVALID_ARG, "ex[t] outside [0, 32768)");
    else if (hb[0] & 4) ps = fail(PIC_ERR_INVALID_ARG, "cap outside [0, 2^20)");
    else if (hb[0] & 8) ps = fail(PIC_ERR_INVALID_ARG, "x0r outside [0, cap]");
    else if (hb[0] & 16) ps = fail(PIC_ERR_INVALID_ARG, "need 0 <= sl <= Sl <= cap");
    else if ((long long)d->T * hb[1] >= (1ll << 31))
        ps = fail(PIC_ERR_INVALID_ARG, "T * max(cap) must be below 2^31");
    if (!ps && d->T > 0) {
        k_ow_time_rec<<<nblk(d->T, 256) < 4096 ? nblk(d->T, 256) : 4096, 256, 0, st>>>(
            d->T, h->ret, h->dem, h->ex, h->trec);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
            ps = fail(PIC_ERR_CUDA, "OWMR create: record table");
    }
    h->maxcap = hb[1];
    if (ps) {
        pic_owmr_destroy(h);
        return ps;
    }
    *out = h;
    return PIC_OK;
}

void pic_owmr_destroy(pic_owmr* h) {
    if (!h) return;
    free_tables(h);
    cudaFree(h->ret); cudaFree(h->dem); cudaFree(h->ex); cudaFree(h->cap); cudaFree(h->x0r); cudaFree(h->sl);
    cudaFree(h->Sl); cudaFree(h->act); cudaFree(h->pre); cudaFree(h->xfin); cudaFree(h->bad);
    cudaFree(h->oc); cudaFree(h->trec); cudaFree(h->tsum);
    delete h;
}

pic_status pic_owmr_simulate(pic_owmr* h, const pic_owmr_policy* pol, const pic_owmr_opts* o,
                             int32_t* actions_out, int32_t* state_out, int32_t out_mem,
                             pic_owmr_result* res, void* stream) {
    if (!h || !pol || !o || (!actions_out && h->T > 0))
        return fail(PIC_ERR_INVALID_ARG, "handle, policy, opts and actions_out are required");
    if (o->mode != PIC_MODE_PICARD && o->mode != PIC_MODE_SEQUENTIAL)
        return fail(PIC_ERR_INVALID_ARG, "unknown mode %d", o->mode);
    if (out_mem != PIC_MEM_HOST && out_mem != PIC_MEM_DEVICE)
        return fail(PIC_ERR_INVALID_ARG, "unknown out_mem %d", out_mem);
    const int H = pol->hidden;
    if (H != 0 && (H < 64 || H > kMaxH || H % 64))
        return fail(PIC_ERR_INVALID_ARG, "hidden must be 0 or a multiple of 64 in [64, 512]");
    if (H && (!pol->W1 || !pol->b1 || !pol->W2 || !pol->b2 || !pol->w3 || !pol->b3))
        return fail(PIC_ERR_INVALID_ARG, "network needs W1, b1, W2, b2, w3, b3 (device)");
    if (H && ((uintptr_t)pol->W2 & 15u))
        return fail(PIC_ERR_INVALID_ARG, "W2 must be 16-byte aligned");
    if (o->num_procs < 0 || o->num_procs > h->N || o->max_iters < 0 || o->timeout_ns < 0 ||
        o->max_steps < 0)
        return fail(PIC_ERR_INVALID_ARG,
                    "need 0 <= num_procs <= N, max_iters >= 0, timeout >= 0, max_steps >= 0");
    const int P = o->num_procs ? o->num_procs : h->N;
    const int rp = (h->N + P - 1) / P;
    if (o->mode == PIC_MODE_PICARD && rp > kMaxSlots / kLanes)
        return fail(PIC_ERR_UNSUPPORTED, "more than %d retailers per processor", kMaxSlots / kLanes);
    cudaStream_t st = (cudaStream_t)stream;
    int launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const bool timing = (o->flags & PIC_FLAG_TIMING) != 0;
    if (timing) {
        CU(cudaEventCreate(&ev0));
        CU(cudaEventCreate(&ev1));
        CU(cudaEventRecord(ev0, st));
    }
    CU(cudaMemsetAsync(h->oc, 0, sizeof(OwCtrl), st));
    CU(cudaMemsetAsync(h->bad, 0, sizeof(int), st));
    if (o->alpha_init && h->T > 0) {
        CU(cudaMemcpyAsync(h->act, o->alpha_init, (size_t)h->T * 4, cudaMemcpyDeviceToDevice, st));
        k_ow_check_init<<<nblk(h->T, 256) < 1024 ? nblk(h->T, 256) : 1024, 256, 0, st>>>(
            h->T, h->act, h->maxcap, h->bad);
        ++launches;
        int hb0 = 0;
        CU(cudaMemcpyAsync(&hb0, h->bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (hb0 & 32) return fail(PIC_ERR_INVALID_ARG, "alpha_init holds a negative value or q > max cap");
    } else if (h->T > 0) {
        CU(cudaMemsetAsync(h->act, 0, (size_t)h->T * 4, st));
    }
    OwArgs a{};
    a.T = h->T; a.N = h->N; a.P = P; a.H = H; a.X0 = h->X0; a.s = h->s; a.S = h->S;
    a.ntiles = h->ntiles; a.rp = rp;
    a.window = o->max_steps;
    {
        long long cap = (long long)h->T + 1;
        if (a.window > 0) cap += (long long)h->T / a.window + 1;
        a.max_iters = o->max_iters ? o->max_iters : (int)(cap < INT_MAX ? cap : INT_MAX);
    }
    a.timeout_ns = o->timeout_ns ? o->timeout_ns : 60000000000ll;
    a.cap = h->cap; a.sl = h->sl; a.Sl = h->Sl; a.x0r = h->x0r;
    a.act = h->act; a.pre = h->pre; a.tsum = h->tsum; a.xfin = h->xfin; a.oc = h->oc;
    a.W1 = pol->W1; a.b1 = pol->b1; a.W2 = pol->W2; a.b2 = pol->b2; a.w3 = pol->w3; a.b3 = pol->b3;
    if (o->mode == PIC_MODE_PICARD) {
        if (!(o->flags & PIC_FLAG_REUSE_TABLES)) free_tables(h);
        a.xs_len = rp * kLanes;
        const size_t smem = owmr_smem(H, a.xs_len, h->max_smem, &a.nbuf);
        if (H && a.nbuf < 2) return fail(PIC_ERR_UNSUPPORTED, "shared memory too small for the network");
        void (*kern)(OwArgs) = H ? k_owmr_picard<true> : k_owmr_picard<false>;
        CU(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int occ = 0;
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kOwThreads, smem));
        if (occ < 1) return fail(PIC_ERR_CUDA, "OWMR kernel does not fit an SM");
        const int grid = h->num_sms * occ;
        pic_status ps = build_tables(h, P, grid, st, &launches);
        if (ps) return ps;
        a.B = h->B; a.ngroups = h->ngroups; a.rec = h->rec; a.gbase = h->gbase; a.memo = h->memo;
        a.cmax = h->cmax; a.ckpt = h->ckpt;
        a.resume = rp == 1;  // checkpoints hold one store's stock per lane
        if (H) CU(cudaMemsetAsync(h->memo, 0xff, (size_t)(h->rows > 0 ? h->rows : 1) * kLanes * sizeof(int2), st));
        void* params[] = {&a};
        CU(cudaLaunchCooperativeKernel((const void*)kern, grid, kOwThreads, params, smem, st));
        ++launches;
    } else {
        a.rec = h->trec;
        const bool use_smem = h->N <= kMaxSlots;
        a.xs_len = use_smem ? h->N : 0;
        const size_t smem = owmr_smem(H, a.xs_len, h->max_smem, &a.nbuf);
        if (H && a.nbuf < 2) return fail(PIC_ERR_UNSUPPORTED, "shared memory too small for the network");
        int32_t* xs_g = nullptr;
        if (!use_smem) CU(cudaMallocAsync(&xs_g, (size_t)h->N * 4, st));
        void (*kern)(OwArgs, int32_t*) = H ? k_owmr_seq<true> : k_owmr_seq<false>;
        CU(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<1, kOwThreads, smem, st>>>(a, xs_g);
        CU(cudaGetLastError());
        ++launches;
        if (xs_g) CU(cudaFreeAsync(xs_g, st));
    }
    OwCtrl hc;
    int hbad = 0;
    int4 pT = make_int4(0, 0, -1, 0);
    CU(cudaMemcpyAsync(&hc, h->oc, sizeof(OwCtrl), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&hbad, h->bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&pT, h->pre + (o->mode == PIC_MODE_PICARD ? h->T : 0), sizeof(int4),
                       cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (hbad & 32) return fail(PIC_ERR_INVALID_ARG, "alpha_init holds a negative value or q > max cap");
    if (hc.c.err) return fail((pic_status)hc.c.err, "device wait exceeded timeout (%lld ns)", a.timeout_ns);
    const cudaMemcpyKind k = out_mem == PIC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (h->T > 0) CU(cudaMemcpyAsync(actions_out, h->act, (size_t)h->T * 4, k, st));
    if (state_out) {
        int x0f;
        if (o->mode == PIC_MODE_PICARD)
            x0f = pT.z >= 0 ? (h->S - pT.y > 0 ? h->S - pT.y : 0) : (h->X0 - pT.x > 0 ? h->X0 - pT.x : 0);
        else
            x0f = pT.x;
        if (out_mem == PIC_MEM_HOST) {
            state_out[0] = x0f;
        } else {
            CU(cudaMemcpyAsync(state_out, &x0f, sizeof(int), cudaMemcpyHostToDevice, st));
        }
        CU(cudaMemcpyAsync(state_out + 1, h->xfin, (size_t)h->N * 4, k, st));
    }
    if (timing) CU(cudaEventRecord(ev1, st));
    CU(cudaStreamSynchronize(st));
    const int sl = hc.c.pad0;
    if (res) {
        res->iters = hc.c.iters;
        res->procs = o->mode == PIC_MODE_PICARD ? P : 1;
        res->replenishments = hc.R[sl];
        res->lost = hc.lost[sl];
        res->shipped = hc.shipped[sl];
        res->policy_calls = (long long)hc.evals;
        res->eval_rounds = (long long)hc.rounds;
        res->near_ties = (long long)hc.near;
        res->launches = launches;
        res->ms_total = 0.f;
        if (timing) cudaEventElapsedTime(&res->ms_total, ev0, ev1);
    }
    if (timing) {
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
    }
    if (o->mode == PIC_MODE_PICARD && !hc.c.converged)
        return fail(PIC_ERR_NOT_CONVERGED, "no fixed point within %d passes", a.max_iters);
    return PIC_OK;
}

}  // extern "C"
