// MLP policies scored in CTA-wide waves on the tensor cores (tcgen05).
//
// Algorithm 1's replay phase (lines 4-9: every evaluated run of a pass replays
// its orders with fresh policy calls) has, inside one work unit (a segment of
// one product's runs), a chain of sequential decisions, and across work units
// none.  The per-warp kernels evaluate one decision at a time per warp; here a
// CTA keeps 128 work units in flight (slots, one per TMEM lane) and evaluates
// the pending decision of every slot at once, as the rows of one tile:
//   Z  = F W1s                       (F: the rows' stock features min(S,32)/32,
//                                     [128 x 64] BF16, exact; tcgen05, TMEM)
//   h' = max(Z + P[r], 0)            (P: the per-region chain prefix of layer 1,
//                                     FP32), split into BF16 hi + lo
//   SC = h'_hi W2 + h'_lo W2         (tcgen05, FP32 accumulation in TMEM)
// in two halves of 128 hidden units.  A row's decision is the arg max over its
// stocked warehouses of SC + b2 (+ Gumbel noise), kept when the top-2 margin
// exceeds twice a bound on |key_tc - key_ref| (the reference FP32 order: layer 1
// one fmaf chain from b1, layer 2 one chain from b2); other rows (near ties) go
// to the FP32 scorer (mlp_decide), which decides in the reference order.
//
// The bound.  Per hidden unit, Z + P differs from the reference pre-activation
// by at most e1 = 1.2e-5 Emax[r] (the tensor cores' 64-term sum charged 2u per
// addition, the reference chain's 64 roundings, the add of P; u = 2^-24;
// Emax[r] = max_j (|P[r][j]| + sum_n |W1s[n][j]|)); relu keeps it.  hi + lo is
// h' within 2^-18 h'.  The tensor cores' 512-term sum of SC (2u per addition),
// the reference chain's 256 roundings and the add of b2 give, with
// c2 = max_n sum_j |W2[j][n]| and hmax the row's largest h':
//   B = 1.01 (c2 (e1 + 8.5e-5 (hmax + e1)) + 1.6e-5 max|b2|)
// and with Gumbel noise the two roundings of s + g (2^-22 |key|).
//
// Rows that need no network are decided in the same wave from exact scores:
// saturated states (every warehouse at 32 units or more) from the per-region
// table of reference scores, and, in a batch, the greedy and bid-price
// trajectories' orders from the cost table (arg min, lowest index on ties).
//
// Slots: thread t < 128 (warps 0-3) owns slot t: it takes work units from the
// CTA's share of the pass's longest-first order (through a ring of active
// units), walks their orders (the new cache, the first changes) and stops at
// each order that needs a decision.  The stock rows S (current) and S0 (at the
// unit's start, the closed form max(0, x0 - D)) of each slot live in shared
// memory; all 16 warps build the start rows of the units taken in a wave, write
// the histograms S0 - S of the units finished (the next pass's prefix) and the
// rows' stock features.  All 16 warps take part in the epilogues: warp w reads
// TMEM lanes 32 (w % 4) .. + 31 and the column quarter w / 4.
#include <cstddef>

#include "pic_mlp.cuh"
#include "pic_tc.cuh"

namespace pic {

namespace {

using namespace picard;
using namespace mlp;
using namespace tc;

constexpr int kWRows = 128;     // slots = tile rows = TMEM lanes
constexpr int kWThreads = 512;  // 16 warps
constexpr int kWWarps = kWThreads / 32;
constexpr int kWN = 64;         // warehouses padded (stock features = K of Z, columns of SC)
constexpr int kWNp = kWN + 1;   // row stride of the per-slot arrays
constexpr unsigned kWColZ = 0, kWColSC = 128;  // TMEM columns: Z (one half, 128), SC (64)
constexpr float kWL1 = 1.2e-5f, kWL2 = 8.5e-5f, kWB2 = 1.6e-5f;
constexpr int kWSmall = 16;     // waves with at most this many network rows skip the tensor cores
constexpr int kRing = 512;      // active-unit ring of a CTA
constexpr int kRingScan = 256;  // candidates examined per refill round

// Row modes of a wave.
constexpr int kRowNone = 0, kRowNet = 1, kRowSat = 2, kRowGreedy = 3, kRowDual = 4;

struct __align__(16) WaveSmem {
    unsigned char w1s[kHidden * kWN * 2];  // [j][n]: B of Z (K = n, N = j)
    unsigned char w2[kWN * kHidden * 2];   // [n][j]: B of SC (K = j, N = n)
    union {
        unsigned char f[kWRows * kWN * 2];  // [t][n]: A of Z
        struct {                            // after the wave's last MMA: per-quarter top-2
            float rk1[4][kWRows], rk2[4][kWRows], rhm[4][kWRows];
            int rn1[4][kWRows];
        } red;
    };
    unsigned char hhi[kWRows * 128 * 2];   // [t][j] of one half: h' hi (A of SC); scratch
    unsigned char hlo[kWRows * 128 * 2];   // h' lo
    // per slot (row stride kWNp: the lanes of a warp, which own consecutive
    // slots, read the same warehouse of their rows from different banks)
    int S[kWRows][kWNp];                   // current stock row (0 beyond N)
    int S0[kWRows][kWNp];                  // stock row at the start of the unit
    float b2[kWN];
    int row_mode[kWRows], row_r[kWRows], row_t[kWRows], row_k[kWRows], row_act[kWRows];
    int row_traj[kWRows], row_gum[kWRows], row_near[kWRows];
    unsigned long long row_seed[kWRows];
    int near_list[kWRows];
    // active work units of the CTA's share, found ahead of the slots that take
    // them: {unit, product, first position, end | chained << 31}
    int4 ring[kRing];
    unsigned long long acc[4];
    // slots that finished a unit (its row's histogram to write) or started one
    // (its start row to build) in this wave's advance: done by all warps
    int fin_seg[kWRows], fin_row[kWRows];
    int st_row[kWRows], st_seg[kWRows], st_k[kWRows];
    unsigned char st_low[kWRows];  // warehouses below 32 units (at most 64)
    int n_fin, n_start;
    int n_near, fail, any_net;
    int ring_head, ring_tail, scan_i, share_done;
    unsigned long long mbar;
    unsigned tmem;
};

// The CTA's share of a pass's longest-first order: positions i G + c (i even)
// and i G + G - 1 - c (i odd) for CTA c of G.
__device__ __forceinline__ int cta_pos(int i) {
    const int G = gridDim.x, c = blockIdx.x;
    return i * G + ((i & 1) ? G - 1 - c : c);
}

struct WaveBatch {  // batch instances only
    const int32_t* __restrict__ traj_of_prod;
    const BatchPol* __restrict__ pol;
    const int32_t* __restrict__ toff;
    int32_t* last_chg;
};

// One slot's walk state (registers of its thread).  A work unit is one run
// (the tables are built with segment window 1), so every order of an active
// unit is evaluated.
struct Slot {
    int seg;          // current work unit, -1: none
    int k, j, jend;   // product, next sorted position, end
    int first_chg;    // first changed position in this unit
    int low;          // warehouses (n < N) below 32 units: 0 = saturated state
    unsigned long long evals;
    int t_off;        // batch: the trajectory's first order
    int kind;         // policy kind of the unit (PIC_POLICY_*)
    int traj;
    unsigned long long seed;
    int tb;           // batch: trajectory
    int ao;           // cached action of the pending order
    int nx_ao, nx_r, nx_t;  // the next order's cached action, region and time (loaded ahead)
};

template <bool BATCH>
struct WaveCtx {
    const KArgs& a;
    const MlpPolicy& p;
    const WaveBatch& b;
    WaveSmem& s;
    int whi, wprev, it;
    const int* fc_prev;
    int* fc_cur;
    bool no_reset;
};

// The data of order j (cached action, region, time within the trajectory).
__device__ __forceinline__ void load_order(const KArgs& a, int j, int t_off, int& ao, int& r, int& tt) {
    ao = a.alpha_s[j];
    r = __ldg(a.reg_s + j);
    tt = __ldg(a.perm + j) - t_off;
}

// Take the work unit e for the slot: its product, orders and policy, and the
// first order's data; the start row S0 = S = max(0, x0 - D) (D the cached
// actions of its product before it, the chain prefix) is built by rows_coop.
template <bool BATCH>
__device__ void slot_take(const WaveCtx<BATCH>& c, int t, Slot& sl, const int4 e) {
    const KArgs& a = c.a;
    WaveSmem& s = c.s;
    sl.seg = e.x;
    sl.k = e.y;
    sl.j = e.z;
    sl.jend = e.w & 0x7FFFFFFF;
    const bool chained = (e.w >> 31) & 1;
    const int i = atomicAdd(&s.n_start, 1);
    s.st_row[i] = t;
    s.st_seg[i] = chained ? sl.seg : -1 - sl.seg;  // -1 - seg: no chain prefix
    s.st_k[i] = sl.k;
    sl.first_chg = INT_MAX;
    sl.evals = 0;
    if constexpr (BATCH) {
        sl.tb = __ldg(c.b.traj_of_prod + sl.k);
        const BatchPol bp = c.b.pol[sl.tb];
        sl.kind = bp.kind;
        sl.traj = bp.traj;
        sl.seed = bp.seed;
        sl.t_off = __ldg(c.b.toff + sl.tb);
    } else {
        sl.kind = c.p.gumbel ? PIC_POLICY_GUMBEL : PIC_POLICY_MLP;
        sl.traj = c.p.traj;
        sl.seed = c.p.seed;
        sl.t_off = 0;
        sl.tb = 0;
    }
    load_order(a, sl.j, sl.t_off, sl.nx_ao, sl.nx_r, sl.nx_t);
}

// The rows of the slots listed by this wave's advance, one warp per row and
// lanes over warehouses (every thread of the CTA calls it): first the
// histograms of new actions of the finished units (S0 - S: every order of a
// unit was evaluated and each fresh action took one unit) for the next pass's
// prefix, then the start rows of the new units, S0 = S = max(0, x0 - D), and
// their count of warehouses below 32 units.
__device__ void rows_coop(const KArgs& a, WaveSmem& s) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = a.N, NP = a.NP;
    for (int i = warp; i < s.n_fin; i += kWWarps) {
        const int f = s.fin_row[i];
        int32_t* g = a.agg + (size_t)s.fin_seg[i] * NP;
        for (int n = lane; n < NP; n += 32) g[n] = s.S0[f][n] - s.S[f][n];
    }
    __syncthreads();
    // up to 4 rows per warp at a time, their loads issued together
    const int ns = s.n_start;
    for (int i0 = warp; i0 < ns; i0 += 4 * kWWarps) {
        int xv[4][kWN / 32], dv[4][kWN / 32];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * kWWarps;
            const int sg = i < ns ? s.st_seg[i] : -1, k = i < ns ? s.st_k[i] : 0;
            const int seg = sg >= 0 ? sg : -1 - sg;
#pragma unroll
            for (int h = 0; h < kWN / 32; ++h) {
                const int n = lane + 32 * h;
                const bool in = i < ns && n < N;
                xv[u][h] = in ? __ldg(a.x0 + (size_t)k * N + n) : 0;
                dv[u][h] = (in && sg >= 0) ? a.carry[(size_t)seg * NP + n] : 0;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * kWWarps;
            if (i >= ns) break;  // warp-uniform
            const int row = s.st_row[i];
            int low = 0;
#pragma unroll
            for (int h = 0; h < kWN / 32; ++h) {
                const int n = lane + 32 * h;
                const int v = max(0, xv[u][h] - dv[u][h]);
                s.S[row][n] = v;
                s.S0[row][n] = v;
                low += __popc(__ballot_sync(kFull, n < N && v < 32));
            }
            if (lane == 0) s.st_low[row] = (unsigned char)low;
        }
    }
    __syncthreads();
}

// The stock features min(S, 32) / 32 of every network row, one thread per row
// and group of 16 warehouses (every thread of the CTA calls it).
__device__ __forceinline__ void features_coop(WaveSmem& s) {
    const int row = threadIdx.x & (kWRows - 1), c0 = 16 * (threadIdx.x >> 7);
    if (s.row_mode[row] == kRowNet) {
        float fv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) fv[i] = (float)min(s.S[row][c0 + i], 32) * 0.03125f;  // exact
        st_row16(s.f, row, c0, kWN, fv);
    }
}

// Close the slot's work unit: list its row for the histogram of new actions
// (written by rows_coop) and keep the first-change records.  The final stock is computed
// after the passes from the final cache (k_wave_xfin).  Returns whether it
// changed a cached action.
template <bool BATCH>
__device__ bool slot_finish(const WaveCtx<BATCH>& c, int t, Slot& sl) {
    const KArgs& a = c.a;
    WaveSmem& s = c.s;
    const int i = atomicAdd(&s.n_fin, 1);  // its row's histogram: rows_coop
    s.fin_row[i] = t;
    s.fin_seg[i] = sl.seg;
    const bool chg = sl.first_chg != INT_MAX;
    if (chg) {
        if (sl.first_chg < ld_volatile(&c.fc_cur[sl.k])) atomicMin(&c.fc_cur[sl.k], sl.first_chg);
        report_window_change(a, c.it, sl.first_chg);
        if constexpr (BATCH)
            if (ld_volatile(&c.b.last_chg[sl.tb]) < c.it) atomicMax(&c.b.last_chg[sl.tb], c.it);
    }
    sl.seg = -1;
    return chg;
}

// Apply the decision of the order at sl.j and move on.
__device__ __forceinline__ void slot_apply(const KArgs& a, WaveSmem& s, int t, Slot& sl, int act) {
    if (act >= 0) {
        const int v = s.S[t][act] - 1;
        s.S[t][act] = v;
        sl.low += v == 31;
    }
    if (act != sl.ao) {
        a.alpha_s[sl.j] = (int8_t)act;
        if (sl.first_chg == INT_MAX) sl.first_chg = sl.j;
    }
    sl.j += 1;
}

// Refill the CTA's ring of active units (every thread calls it): rounds of
// kRingScan candidates of the share, one per thread, while the ring holds
// fewer than kRingScan units and the share is not done.
template <bool BATCH>
__device__ void ring_refill(const WaveCtx<BATCH>& c) {
    const KArgs& a = c.a;
    WaveSmem& s = c.s;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nseg = a.ctrl->nseg;
    for (int round = 0; round < 4; ++round) {
        __syncthreads();
        if (s.share_done || s.ring_tail - s.ring_head >= kRingScan) break;  // uniform
        bool act = false;
        int4 e = make_int4(0, 0, 0, 0);
        if (tid < kRingScan) {
            const int pos = cta_pos(s.scan_i + tid);
            if (pos < nseg) {
                const int seg = __ldg(a.lpt + pos);
                const SegMeta m = load_meta(a.meta + seg);
                const int fcp = c.no_reset ? -1 : c.fc_prev[m.k];
                // one run per unit: active = evaluated (after the product's first change
                // of the previous pass, or newly inside the window; and inside it)
                act = run_evaluated(a, c.whi, c.wprev, m.r0, m.j0 > fcp);
                const bool chained = m.ce - m.cf > 1 && (c.it > 1 || a.first_dirty);
                e = make_int4(seg, m.k, m.j0, m.jend | (chained ? (int)0x80000000 : 0));
            } else {
                s.share_done = 1;  // positions grow with the candidate index
            }
        }
        const unsigned am = __ballot_sync(kFull, act);
        int base = 0;
        if (lane == 0 && am) base = atomicAdd(&s.ring_tail, __popc(am));
        base = __shfl_sync(kFull, base, 0);
        if (act) s.ring[(base + __popc(am & ((1u << lane) - 1u))) % kRing] = e;
        __syncthreads();
        if (tid == 0) s.scan_i += kRingScan;
    }
    __syncthreads();
}

// Advance the slots of one warp (warps 0-3; every lane calls it), first half:
// finish the units whose orders are all decided; give every lane without a
// unit the next unit of the ring.  The rows of both are listed for rows_coop.
template <bool BATCH>
__device__ void slot_open(const WaveCtx<BATCH>& c, int t, Slot& sl,
                          bool& changed, unsigned long long& units, unsigned long long& calls,
                          unsigned long long& ucalls, unsigned long long& uorders) {
    WaveSmem& s = c.s;
    const int lane = t & 31;
    if (sl.seg >= 0 && sl.j == sl.jend) {
        changed |= slot_finish<BATCH>(c, t, sl);
        units += 1;
        calls += sl.evals;
        if (sl.evals > ucalls) ucalls = sl.evals;
        if (sl.evals > uorders) uorders = sl.evals;  // one run: every order evaluated
    }
    // lanes without a unit take the next entries of the ring
    const unsigned need = __ballot_sync(kFull, sl.seg < 0);
    if (need) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&s.ring_head, __popc(need));
        base = __shfl_sync(kFull, base, 0);
        const int idx = base + __popc(need & ((1u << lane) - 1u));
        if (sl.seg < 0 && idx < ld_volatile(&s.ring_tail)) slot_take<BATCH>(c, t, sl, s.ring[idx % kRing]);
    }
}

// Second half, after rows_coop: set up each busy lane's next order as a row of
// the wave (its features are written by features_coop).  started: the slot
// took its unit in this advance (its count of low warehouses comes from
// rows_coop).  Returns whether this lane has a pending decision.
template <bool BATCH>
__device__ bool slot_row(const WaveCtx<BATCH>& c, int t, Slot& sl, bool started) {
    const KArgs& a = c.a;
    WaveSmem& s = c.s;
    if (sl.seg < 0) return false;
    if (started) sl.low = s.st_low[t];
    const int ao = sl.nx_ao, r = sl.nx_r, tt = sl.nx_t;
    if (sl.j + 1 < sl.jend) load_order(a, sl.j + 1, sl.t_off, sl.nx_ao, sl.nx_r, sl.nx_t);
    sl.evals += 1;
    int mode;
    if (sl.kind == PIC_POLICY_GREEDY) mode = kRowGreedy;
    else if (sl.kind == PIC_POLICY_DUAL) mode = kRowDual;
    else mode = (c.p.sat != nullptr && sl.low == 0) ? kRowSat : kRowNet;
    s.row_mode[t] = mode;
    s.row_r[t] = r;
    s.row_k[t] = sl.k;
    s.row_t[t] = tt;
    s.row_gum[t] = sl.kind == PIC_POLICY_GUMBEL;
    s.row_seed[t] = sl.seed;
    s.row_traj[t] = sl.traj;
    sl.ao = ao;
    return true;
}

// Top-2 of one row's keys over the thread's 16 warehouses: k1 with the lowest
// index n1 among equal keys, and k2 the largest key of the other warehouses.
__device__ __forceinline__ void top2_add(float key, int n, float& k1, int& n1, float& k2) {
    if (key > k1) {
        k2 = k1;
        k1 = key;
        n1 = n;
    } else {
        k2 = fmaxf(k2, key);
    }
}

__device__ __forceinline__ float bf16_at(const unsigned char* buf, int r, int c, int C) {
    return __uint_as_float((unsigned)*reinterpret_cast<const uint16_t*>(buf + lay(r, c, C)) << 16);
}

// Decisions in the reference FP32 order for the rows listed in near_list[0..nn)
// (every thread of the CTA calls it; the half-h buffers are free): per row and
// hidden unit j, h_j = max(chain from P[r][j] over the stock inputs n = 0..N-1,
// 0); per row and stocked warehouse n, s_n = chain from b2_n over j = 0..255
// (plus its Gumbel noise); then the arg max, ties to the lowest index.  The
// weights come from the tensor cores' shared-memory operands (the same BF16
// values), 32 rows at a time.
template <bool BATCH>
__device__ void exact_rows(const WaveCtx<BATCH>& c, int nn) {
    const MlpPolicy& p = c.p;
    WaveSmem& s = c.s;
    const int tid = threadIdx.x, N = c.a.N;
    float* hb = reinterpret_cast<float*>(s.hhi);  // [32][256]
    float* kb = reinterpret_cast<float*>(s.hlo);  // [32][64]
    for (int e0 = 0; e0 < nn; e0 += 32) {
        const int ne = min(32, nn - e0);
        for (int q = tid; q < ne * kHidden; q += kWThreads) {
            const int e = q / kHidden, j = q % kHidden, row = s.near_list[e0 + e];
            float z = __ldg(p.P + (size_t)s.row_r[row] * kHidden + j);
            for (int n = 0; n < N; ++n)
                z = fmaf(bf16_at(s.w1s, j, n, kWN), (float)min(s.S[row][n], 32) * 0.03125f, z);
            hb[e * kHidden + j] = z > 0.0f ? z : 0.0f;
        }
        __syncthreads();
        for (int q = tid; q < ne * kWN; q += kWThreads) {
            const int e = q / kWN, n = q % kWN, row = s.near_list[e0 + e];
            float key = -INFINITY;
            if (n < N && s.S[row][n] > 0) {
                const float* h = hb + e * kHidden;
                float sc = s.b2[n];
#pragma unroll 8
                for (int j = 0; j < kHidden; ++j) sc = fmaf(bf16_at(s.w2, n, j, kHidden), h[j], sc);
                if (s.row_gum[row]) sc = __fadd_rn(sc, gumbel1(s.row_seed[row], s.row_traj[row], s.row_t[row], n));
                key = sc;
            }
            kb[e * kWN + n] = key;
        }
        __syncthreads();
        if (tid < ne) {
            const int row = s.near_list[e0 + tid];
            int best = -1;
            float bk = 0.f;
            for (int n = 0; n < N; ++n)
                if (s.S[row][n] > 0 && (best < 0 || kb[tid * kWN + n] > bk)) {
                    best = n;
                    bk = kb[tid * kWN + n];
                }
            s.row_act[row] = best;
        }
        __syncthreads();
    }
}

// The wave: scores of every pending row, decisions, near ties to the FP32
// scorer.  Every thread of the CTA calls it.  Returns false when a tensor-core
// wait timed out (CTA-uniform).
template <bool BATCH>
__device__ bool wave(const WaveCtx<BATCH>& c, unsigned tm, unsigned& phase, MlpCounts& mc) {
    const KArgs& a = c.a;
    const MlpPolicy& p = c.p;
    WaveSmem& s = c.s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t = 32 * (warp & 3) + lane;  // tile row of this thread
    const int cq = warp >> 2;              // column quarter
    const unsigned lane_base = (unsigned)(32 * (warp & 3)) << 16;
    const int N = a.N;
    const int mode = s.row_mode[t];
    float hm = 0.f;
    if (s.any_net) {
        const unsigned aF = su32(s.f), aW1 = su32(s.w1s), aW2 = su32(s.w2), aH = su32(s.hhi),
                       aL = su32(s.hlo);
        const bool net = mode == kRowNet;
        const float* Pr = p.P + (size_t)(net ? s.row_r[t] : 0) * kHidden;
        for (int h = 0; h < 2; ++h) {
            if (tid == 0) {
                if (h == 1)  // SC += h'_0 W2_0 (the half-0 operands are in place)
                    for (int kk = 0; kk < 128 / 16; ++kk) {
                        const unsigned long long bw = sdesc(aW2 + kk * 256, 128, 4096);
                        tc_mma(tm + kWColSC, sdesc(aH + kk * 256, 128, 2048), bw, tc_idesc(kWN, 0, 0), kk > 0);
                        tc_mma(tm + kWColSC, sdesc(aL + kk * 256, 128, 2048), bw, tc_idesc(kWN, 0, 0), 1);
                    }
                for (int kk = 0; kk < kWN / 16; ++kk)  // Z_h = F W1s_h
                    tc_mma(tm + kWColZ, sdesc(aF + kk * 256, 128, 1024),
                           sdesc(aW1 + h * 16384 + kk * 256, 128, 1024), tc_idesc(128, 0, 0), kk > 0);
                tc_commit(&s.mbar);
            }
            // P[r] of this thread's 32 columns, loaded while the tensor cores work
            float4 pq[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                pq[i] = net ? __ldg(reinterpret_cast<const float4*>(Pr + 128 * h + 32 * cq) + i)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
            if (!tc_wait(&s.mbar, phase)) s.fail = 1;
            // h' = max(Z_h + P[r], 0) of this thread's 32 columns, split in BF16 hi + lo
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int c0 = 32 * cq + 16 * hh;
                float v[16], lo[16];
                tc_ld16(tm + lane_base + kWColZ + c0, v);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 q = pq[4 * hh + i];
                    v[4 * i] += q.x; v[4 * i + 1] += q.y; v[4 * i + 2] += q.z; v[4 * i + 3] += q.w;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float x = net ? fmaxf(v[i], 0.f) : 0.f;
                    hm = fmaxf(hm, x);
                    v[i] = __bfloat162float(__float2bfloat16_rn(x));
                    lo[i] = x - v[i];
                }
                st_row16(s.hhi, t, c0, 128, v);
                st_row16(s.hlo, t, c0, 128, lo);
            }
            tc_sync_operands();
        }
        if (tid == 0) {  // SC += h'_1 W2_1
            for (int kk = 0; kk < 128 / 16; ++kk) {
                const unsigned long long bw = sdesc(aW2 + 2048 + kk * 256, 128, 4096);
                tc_mma(tm + kWColSC, sdesc(aH + kk * 256, 128, 2048), bw, tc_idesc(kWN, 0, 0), 1);
                tc_mma(tm + kWColSC, sdesc(aL + kk * 256, 128, 2048), bw, tc_idesc(kWN, 0, 0), 1);
            }
            tc_commit(&s.mbar);
        }
        if (!tc_wait(&s.mbar, phase)) s.fail = 1;
    }
    // ---- keys of this thread's 16 warehouses, top-2 per quarter
    {
        const int n0 = 16 * cq;
        float v[16];
        if (s.any_net) tc_ld16(tm + lane_base + kWColSC + n0, v);  // every warp (aligned load)
        float k1 = -INFINITY, k2 = -INFINITY;
        int n1 = INT_MAX;
        if (mode != kRowNone && (mode != kRowNet || s.any_net) && n0 < N) {
            const int r = s.row_r[t], k = s.row_k[t];
            const bool gum = (mode == kRowNet || mode == kRowSat) && s.row_gum[t];
            float g[16];
            if (gum) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    gumbel4(s.row_seed[t], s.row_traj[t], s.row_t[t], (n0 >> 2) + q, g + 4 * q);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = n0 + i;
                if (n >= N || s.S[t][n] <= 0) continue;
                float key;
                if (mode == kRowNet) {
                    key = __fadd_rn(v[i], s.b2[n]);
                } else if (mode == kRowSat) {
                    key = __ldg(p.sat + (size_t)r * N + n);
                } else {  // integer scores, minimised: keys -score are exact in FP32
                    int sc = __ldg(a.cost + (size_t)r * N + n);
                    if (mode == kRowDual) sc -= __ldg(a.lam + (size_t)k * N + n);
                    key = -(float)sc;
                }
                if (gum) key = __fadd_rn(key, g[i]);
                top2_add(key, n, k1, n1, k2);
            }
        }
        s.red.rk1[cq][t] = k1;
        s.red.rk2[cq][t] = k2;
        s.red.rn1[cq][t] = n1;
        s.red.rhm[cq][t] = hm;
    }
    __syncthreads();
    // ---- decisions (slot threads); near ties listed for the FP32 scorer
    if (tid < kWRows && mode != kRowNone) {
        float k1 = s.red.rk1[0][t], k2 = s.red.rk2[0][t], hmax = s.red.rhm[0][t];
        int n1 = s.red.rn1[0][t];
        for (int q = 1; q < 4; ++q) {
            const float o1 = s.red.rk1[q][t];
            if (o1 > k1) {  // quarters hold increasing warehouses: ties stay with the lower
                k2 = fmaxf(k1, s.red.rk2[q][t]);
                k1 = o1;
                n1 = s.red.rn1[q][t];
            } else {
                k2 = fmaxf(k2, fmaxf(o1, s.red.rk2[q][t]));
            }
            hmax = fmaxf(hmax, s.red.rhm[q][t]);
        }
        int act = n1 == INT_MAX ? -1 : n1;
        s.row_near[t] = 0;
        if (mode == kRowNet && !s.any_net) {  // a small wave: the FP32 scorer decides
            act = -2;
            s.row_near[t] = 2;
            s.near_list[atomicAdd(&s.n_near, 1)] = t;
        } else if (mode == kRowNet && act >= 0 && k2 > -INFINITY) {
            const float e1 = kWL1 * __ldg(p.Emax + s.row_r[t]);
            float B = 1.01f * (__ldg(p.bnd) * (e1 + kWL2 * (hmax + e1)) + kWB2 * __ldg(p.bnd + 1));
            if (s.row_gum[t]) B += ldexpf(fmaxf(fabsf(k1), fabsf(k2)), -22);
            if (!(__fsub_rd(k1, k2) > 2.0f * B)) {
                act = -2;
                s.row_near[t] = 1;
                s.near_list[atomicAdd(&s.n_near, 1)] = t;
            }
        }
        s.row_act[t] = act;
    }
    __syncthreads();
    // ---- near ties (and the rows of a small wave): the reference order
    const int nn = s.n_near;
    if (nn > 0) exact_rows<BATCH>(c, nn);
    return s.fail == 0;
}

// NPL: warehouses per lane of the warp-level phase S (N <= 32 NPL).
template <bool BATCH, int NPL>
__global__ void __launch_bounds__(kWThreads, 1) k_picard_wave(KArgs a, MlpPolicy p, WaveBatch b) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    WaveSmem& s = *reinterpret_cast<WaveSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int N = a.N;
    // ---- weights (zero beyond N), control, TMEM
    for (int i = tid; i < kHidden * kWN; i += kWThreads) {
        const int jj = i / kWN, n = i % kWN;
        const uint16_t w1 = (n < N && p.W1raw) ? p.W1raw[(size_t)(N + n) * kHidden + jj] : 0;
        const uint16_t w2 = (n < N && p.W2raw) ? p.W2raw[(size_t)jj * N + n] : 0;
        *reinterpret_cast<uint16_t*>(s.w1s + lay(jj, n, kWN)) = w1;
        *reinterpret_cast<uint16_t*>(s.w2 + lay(n, jj, kHidden)) = w2;
    }
    if (tid < kWN) s.b2[tid] = (tid < N && p.b2f) ? p.b2f[tid] : 0.0f;
    if (tid == 0) {
        s.fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&s.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s.tmem)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_sync_operands();
    const unsigned tm = s.tmem;
    unsigned phase = 0;
    unsigned long long calls = 0;
    MlpCounts mc{0, 0, 0, 0, 0};
    unsigned long long net_rows = 0, table_rows = 0;  // slot threads: decisions by the tile / by a table
    const bool no_reset = (a.flags & PIC_FLAG_NO_RESET) != 0;
    // waves with at most `small` network rows go to the FP32 scorer
    const int small = (a.flags & PIC_FLAG_TC) ? 0 : (a.flags & PIC_FLAG_NO_TC) ? INT_MAX : kWSmall;
    auto replay = [&](const int* fc_prev, int* fc_cur, int it, int whi, int wprev,
                      unsigned long long& replays, unsigned long long& ucalls,
                      unsigned long long& uorders) -> bool {
        const WaveCtx<BATCH> c{a, p, b, s, whi, wprev, it, fc_prev, fc_cur, no_reset};
        if (tid == 0) {
            s.ring_head = s.ring_tail = s.scan_i = 0;
            s.share_done = 0;
        }
        __syncthreads();
        Slot sl;
        sl.seg = -1;
        bool changed = false;
        unsigned long long units = 0, scalls = 0, umax = 0, omax = 0;
        bool ok = s.fail == 0;
        while (ok) {
            ring_refill<BATCH>(c);
            if (tid == 0) s.n_fin = s.n_start = 0;
            __syncthreads();
            bool started = false;
            if (tid < kWRows) {
                s.row_mode[tid] = kRowNone;
                const int seg0 = sl.seg;
                slot_open<BATCH>(c, tid, sl, changed, units, scalls, umax, omax);
                started = sl.seg >= 0 && sl.seg != seg0;  // a unit is never taken twice
            }
            __syncthreads();
            rows_coop(a, s);
            bool pend = false, net = false;
            if (tid < kWRows) {
                pend = slot_row<BATCH>(c, tid, sl, started);
                net = pend && s.row_mode[tid] == kRowNet;
            }
            if (tid == 0) s.n_near = 0;
            const int nnet = __syncthreads_count(net);
            // reservations beyond the ring's end took nothing
            if (tid == 0 && s.ring_head > s.ring_tail) s.ring_head = s.ring_tail;
            const int npend = __syncthreads_count(pend);
            if (npend == 0) {
                const bool more = !s.share_done || s.ring_tail > s.ring_head;
                __syncthreads();
                if (more) continue;
                break;
            }
            features_coop(s);
            // a few network rows are faster on the FP32 scorer, one warp each
            if (tid == 0) s.any_net = nnet > small;
            tc_sync_operands();  // the rows' features reach the tensor cores
            ok = wave<BATCH>(c, tm, phase, mc);
            if (tid < kWRows && pend) {
                const int md = s.row_mode[tid];
                if (md == kRowNet && s.row_near[tid] == 0) net_rows += 1;
                if (md == kRowNet && s.row_near[tid] == 1) mc.rescored += 1;
                if (md == kRowSat) table_rows += 1;
                if (md == kRowNet || md == kRowSat) mc.calls += 1;
                slot_apply(a, s, tid, sl, s.row_act[tid]);
            }
            __syncthreads();
        }
        if (!ok && tid == 0) atomicCAS(&a.ctrl->err, 0, (int)PIC_ERR_TIMEOUT);
        // CTA totals on thread 0
        if (tid == 0) s.acc[0] = s.acc[1] = s.acc[2] = s.acc[3] = 0;
        __syncthreads();
        if (tid < kWRows) {
            if (units) atomicAdd(&s.acc[0], units);
            if (scalls) atomicAdd(&s.acc[1], scalls);
            if (umax) atomicMax(&s.acc[2], umax);
            if (omax) atomicMax(&s.acc[3], omax);
        }
        const int any_chg = __syncthreads_count(changed);
        if (tid == 0) {
            replays += s.acc[0];
            calls += s.acc[1];
            if (s.acc[2] > ucalls) ucalls = s.acc[2];
            if (s.acc[3] > uorders) uorders = s.acc[3];
        }
        __syncthreads();
        return any_chg > 0;
    };
    // whole chain prefixes in carry: a unit's start row is one load per warehouse
    picard_passes<NPL, kWWarps, decltype(replay)&, 1, true, false>(a, calls, replay,
                                                            reinterpret_cast<SegMeta*>(s.hhi),
                                                            reinterpret_cast<int*>(s.hlo));
    // counters: decisions by the tensor-core tile, by the saturated-state table,
    // tile rows re-scored in FP32, near ties of that FP32 scorer, MLP calls
    if (tid < kWRows) {
        if (net_rows) atomicAdd(&a.ctrl->tc_rows, net_rows);
        if (table_rows) atomicAdd(&a.ctrl->sat_rows, table_rows);
        if (mc.rescored) atomicAdd(&a.ctrl->rescored, mc.rescored);
        if (BATCH && mc.calls) atomicAdd(&a.ctrl->mlp_calls, mc.calls);
    }
    if ((tid & 31) == 0 && mc.near) atomicAdd(&a.ctrl->near_ties, mc.near);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(256));
}

// Final stock of each product (one warp per product): x0 minus the actions of
// its orders in the cache (sorted positions pstart[k] .. pstart[k+1]).  At the
// fixed point every cached action is feasible, so this is the stock after the
// last order.
__global__ void k_wave_xfin(int K, int N, const int32_t* __restrict__ pstart,
                            const int8_t* __restrict__ alpha_s, const int32_t* __restrict__ x0,
                            int32_t* __restrict__ xfin) {
    __shared__ int cnt[8][kWN];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.x * 8 + w;
    if (k >= K) return;
    cnt[w][lane] = 0;
    cnt[w][lane + 32] = 0;
    __syncwarp();
    for (int j = pstart[k] + lane; j < pstart[k + 1]; j += 32) {
        const int v = alpha_s[j];
        if (v >= 0 && v < kWN) atomicAdd(&cnt[w][v], 1);
    }
    __syncwarp();
    for (int n = lane; n < N; n += 32) xfin[(size_t)k * N + n] = x0[(size_t)k * N + n] - cnt[w][n];
}

}  // namespace

// Shared memory of the wave kernel (dynamic: the WaveSmem block, 128-aligned).
size_t wave_smem_bytes() { return sizeof(WaveSmem) + 128; }
// dynamic (with the alignment slack) plus the kernel's static shared memory (the
// pass loop's CTA words, 128 B) within the 227 KB a CTA may opt into
static_assert(sizeof(WaveSmem) + 128 + 128 <= 232448, "wave kernel shared memory above 227 KB");

bool wave_applies(const Instance* I) { return I->N <= kWN; }

template <bool BATCH, int NPL>
cudaError_t launch_wave(Instance* I, const KArgs& a, const MlpPolicy& p, const WaveBatch& b,
                        cudaStream_t st) {
    auto kern = k_picard_wave<BATCH, NPL>;
    const size_t smem = wave_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWThreads, smem))) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int grid = I->num_sms;  // one CTA (and one TMEM allocation) per SM
    I->coop_blocks = grid;
    I->cta_threads = kWThreads;
    I->ctas_per_sm = 1;
    I->ran_wave = 1;
    KArgs args = a;
    args.perm = I->perm;  // sorted position -> time (the Gumbel counter), also for batches
    MlpPolicy pp = p;
    WaveBatch bb = b;
    void* params[] = {&args, &pp, &bb};
    I->launches += 1;
    e = cudaLaunchCooperativeKernel((const void*)kern, grid, kWThreads, params, smem, st);
    if (e) return e;
    // the final stock of every product from its actions in the final cache
    I->launches += 1;
    k_wave_xfin<<<(I->K + 7) / 8, 256, 0, st>>>(I->K, I->N, I->pstart, I->alpha_s, I->x0, I->xfin);
    return cudaGetLastError();
}

cudaError_t picard_wave(Instance* I, const KArgs& a, const MlpPolicy& p, cudaStream_t st) {
    const WaveBatch b{nullptr, nullptr, nullptr, nullptr};
    return I->N <= 32 ? launch_wave<false, 1>(I, a, p, b, st) : launch_wave<false, 2>(I, a, p, b, st);
}

cudaError_t picard_wave_batch(Instance* I, const KArgs& a, const MlpPolicy& p,
                              const int32_t* traj_of_prod, const BatchPol* pol, const int32_t* toff,
                              int32_t* last_chg, cudaStream_t st) {
    const WaveBatch b{traj_of_prod, pol, toff, last_chg};
    return I->N <= 32 ? launch_wave<true, 1>(I, a, p, b, st) : launch_wave<true, 2>(I, a, p, b, st);
}

}  // namespace pic
