// Internal (non-ABI) declarations shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pic.h"

namespace pic {

constexpr int kEmb = 16;           // region-embedding width of the MLP policy
constexpr int kHidden = 256;       // MLP hidden width
constexpr int kSegWindow = 64;     // default segment window (orders of one product), integer policies
constexpr int kSegWindowMlp = 8;   // default segment window, MLP policies
constexpr int kSuperBlock = 32;    // segments per carry super-block
constexpr int kThreads = 256;      // threads per CTA of the persistent kernels
constexpr size_t kSmemCostMax = 200 * 1024;  // largest int16 cost table staged in shared memory
constexpr int kTraceCap = 4096;    // passes recorded by the device-side trace
constexpr int kTraceCols = 6;      // int64 fields per recorded pass (see pic_sim_opts.trace)
constexpr int kLenBuckets = 1024;  // segment-length buckets of the longest-first order
constexpr size_t kGrpSmemMax = 150 * 1024;  // cost table budget of the group-per-segment kernel
constexpr int kMlpLptWeight = 64;  // work of an MLP order relative to an integer-policy order
constexpr int kCapChunk = 64;      // longest time chunk of the capacity kernel (orders)

// Device-side control block of one simulate call (zeroed before each launch).
struct Ctrl {
    unsigned int bar_count;  // grid barrier arrivals
    unsigned int bar_gen;    // grid barrier generation
    int err;                 // pic_status raised on the device (TIMEOUT)
    int iters;               // passes of Algorithm 1's loop
    int changed[2];          // "some cached action changed" per pass parity
    int converged;
    int pad0;
    unsigned long long policy_calls;
    long long total_cost;
    long long lost;
    unsigned long long rescored;
    unsigned long long seg_replays;
    unsigned long long mlp_calls;  // MLP / Gumbel policy evaluations (batch kernel)
    unsigned long long tc_rows;    // MLP decisions taken from tensor-core tile scores
    unsigned long long sat_rows;   // MLP decisions taken from the saturated-state table
    unsigned long long near_ties;  // MLP decisions re-scored in the reference order (near ties)
    int cap_fct[2];          // capacity kernel: first changed time of the pass, per parity
    int win_fct[2];          // max_steps window: first changed time of the pass, per parity
    int win_hi, win_hi_prev; // max_steps window of the current pass and of the previous one:
                             // runs of chunks below win_hi are evaluated; chunks at or above
                             // win_hi_prev were not evaluated in the previous pass
    int nruns;               // tables built by the preprocessing kernels
    int nseg;
    int last_m;              // chunk count the tables were built for
    int pad1;
    // look-back tags (kept across calls): a call's passes use tag_base + pass,
    // taken on the device by the call's first kernel from tag_next
    unsigned tag_base;
    unsigned tag_next;
};

// Per-segment metadata packed for one 32-byte load: product, run range, sorted
// position range, first order of the last run, chain (product) segment range.
struct __align__(32) SegMeta {
    int k, r0, r1, j0, jend, last_start, cf, ce;
};

// Per-trajectory policy selector of a batch call (device copy of pic_policy's
// kind, trajectory id and noise seed).
struct __align__(16) BatchPol {
    int kind;
    int traj;
    unsigned long long seed;
};

// A batch of trajectories held as one instance (pic_create_batch).  Trajectory
// b owns orders [toff[b], toff[b+1]), products [koff[b], koff[b+1]) and regions
// [roff[b], roff[b+1]) of the combined arrays: its product and region ids are
// shifted into those ranges at creation, so no two trajectories share state and
// one Picard launch over the combined instance runs every trajectory's own
// iteration (products never interact, Assumption 1 of Sec. 3.2).
struct Batch {
    int B;
    int64_t *h_toff, *h_koff, *h_roff;  // host [B+1]
    int8_t* h_has_lam;                  // host [B]: trajectory b was created with lam
    int32_t *toff, *koff, *roff;        // device [B+1]
    int32_t* traj_of_prod;              // [K] trajectory of each product
    int32_t* reg_local;                 // [R] region id within its trajectory
    int32_t* chunk_len;                 // [B] chunk length L_b of the current tables
    BatchPol* pol;                      // [B] policies of the current call
    BatchPol* h_pol;                    // pinned host staging of pol
    int32_t* last_chg;                  // [B] last pass that changed a cached action of b
    long long* tres;                    // [B][2] cost, a^phi count of trajectory b
    unsigned char* h_out;               // pinned host staging: Ctrl, tres, last_chg
    int max_t;                          // longest trajectory
    // graph of the per-call work (PIC_FLAG_GRAPH), the signature it was captured
    // for, the kernels it launches, and the stream captures are recorded on
    cudaGraphExec_t gexec;
    unsigned long long gsig;
    int glaunches;
    cudaStream_t cap_stream;
    // autotuner result and the policy signature it was tuned for
    unsigned long long tune_sig;
    int tune_m, tune_w, tune_shape, tune_tc, tune_wave;
    int invalid;  // the last pic_batch_load failed: its inputs are undefined
};

struct PgState;  // buffers of the policy gradient (pic_pg.cu)

// All device buffers of one instance.  Sizes: T orders, K products, N warehouses,
// R regions; NP = N rounded up to a multiple of 32.
struct Instance {
    int T, N, K, R, NP;
    int has_lam;
    int cost16;         // every cost fits int16 (the cost table can be staged in shared memory)
    cudaStream_t create_stream;
    // inputs
    int32_t *prod, *reg, *x0, *cost, *lam;
    // order tables (product-major sorted order; built per call)
    int32_t *perm;      // [T]   sorted position j -> time t
    int32_t *prod_s;    // [T]   product at sorted position j
    int32_t *reg_s;     // [T]   region at sorted position j
    int32_t *pcount;    // [K+1] orders per product
    int32_t *pstart;    // [K+1] first sorted position per product
    int32_t *run_start; // [T+1] first sorted position of each run (chunk x product)
    int32_t *run_of;    // [T]   run of sorted position j
    int32_t *run_chunk; // [T+1] chunk (time block) of each run (single instances)
    int32_t *seg_run;   // [SMAX+1] first run of each segment
    int32_t *seg_of_run;// [T]
    int32_t *seg_prod;  // [SMAX]
    int32_t *seg_cf;    // [SMAX] first segment of the segment's product (chain)
    int32_t *seg_ce;    // [SMAX] one past the last segment of the chain
    SegMeta *seg_meta;  // [SMAX] packed copy of the above for the simulation kernels
    int32_t *seg_lpt;   // [SMAX] segments in decreasing order of length (replay assignment)
    int32_t *len_hist;  // [kLenBuckets] counting-sort buckets
    int64_t smax;       // capacity of the segment tables (>= any segment count)
    int64_t smax_agg;   // capacity (segments) of agg/carry/sbtot
    int tables_m, tables_w;  // chunking the current tables were built for (0 = none)
    unsigned tag_next;  // host mirror of ctrl->tag_next (0: look-back words not cleared yet)
    // iteration state
    int8_t *alpha_s;    // [T]  action cache in sorted order
    int32_t *agg;       // [SMAX][NP] histogram of cached actions per segment
    int32_t *carry;     // [SMAX][NP] exclusive prefix of agg inside the segment's super-block
    int32_t *sbexc;     // [SMAX][NP] at a super-block's first segment: the exclusive prefix of
                        // agg over the chain's earlier super-blocks (a segment's chain prefix
                        // is its carry row plus its super-block's sbexc row)
    unsigned long long *sbagg;   // [SMAX][NP] super-block totals, (pass << 32) | value
    unsigned long long *sbincl;  // [SMAX][NP] inclusive chain prefix, (pass << 32) | value
    int32_t *fc;        // [2][K] first changed sorted position per product and pass parity
    int32_t *xfin;      // [K][N] final stock
    int32_t *xwork;     // [K][N] working stock of the sequential simulator
    int8_t *act_t;      // [T]  actions in time order (device staging)
    // MLP policy, per call: chain prefix per region and FP32 copies of the weights
    float *mlp_P;       // [R][256]
    uint4 *mlp_W1p;     // [N][32] packed BF16 stock rows of W1
    uint4 *mlp_W2p;     // [32][N] packed BF16 W2
    float *mlp_b2;      // [N]
    float *mlp_Emax;    // [R] error-bound constant per region (tensor-core tiles)
    float *mlp_bnd;     // [2] max column sum of |W2|, max |b2|
    float *mlp_c2;      // [N] column sums of |W2| (rounded up)
    float *mlp_sat;     // [R][N] reference-order scores of the saturated state (every stock
                        // feature 1)
    // scratch for the sort and scans
    int32_t *tmp_a, *tmp_b, *tmp_c;   // [T] each
    int32_t *scan_blk;                // block sums
    int32_t *hist;                    // radix histograms
    int64_t hist_cap;
    Ctrl *ctrl;
    long long *trace;                 // [kTraceCap][4] device-side per-pass record
    int num_sms;
    int coop_blocks;                  // persistent grid size of the last Picard launch
    int cta_threads, ctas_per_sm;     // its CTA shape
    int launches;                     // kernels launched by the current call
    int ran_wave;                     // the current call ran the wave kernel
    cudaEvent_t ev[4];                // phase timing events (created with the instance)
    // node capacity (pic_instance_desc.cap) and the capacity kernel's tables
    int has_cap;
    int32_t *cap;                     // [N] c_1
    int32_t *cap_run_t;               // [T] run of order t
    int32_t *cap_info;                // [T] slot in its chunk | first << 8 | last of run << 9 |
                                      //     last of product << 10
    int32_t *cap_inv;                 // [T] sorted position of order t
    unsigned long long *cap_qagg;     // [M][NP] tagged per-chunk totals of q
    unsigned long long *cap_qinc;     // [M][NP] tagged inclusive prefixes of q over chunks
    int64_t cap_qrows;                // chunks the q words are sized for
    int cap_tables_m;                 // chunk count the capacity tables describe (0 = none)
    Batch* batch;                     // non-null for a batch instance
    PgState* pg;                      // policy-gradient buffers (allocated at first use)
};

// Preprocessing (pic_prep.cu): sort orders by product (stable in time), region
// gather, per-product offsets, runs for M chunks and segments of window W (a
// batch instance chunks every trajectory by its own chunk_len), then the
// longest-first order of the segments.
cudaError_t build_tables(Instance* I, int M, int W, cudaStream_t st);
// Stable sort of n (key, index) pairs by key in [0, max_key] (LSD radix on the
// instance's histogram scratch); tmp_k / tmp_v are n-element scratch arrays.
cudaError_t sort_pairs(Instance* I, const int32_t* keys, int n, int max_key, int32_t* keys_out,
                       int32_t* vals_out, int32_t* tmp_k, int32_t* tmp_v, cudaStream_t st);
// The same LSD radix sort with explicit scratch: hist [sort_hist_len(n)] and
// scan_blk [scan_blk_len(sort_hist_len(n))], zeroed once when allocated (3
// launches per key byte); err as for scan_exclusive.
cudaError_t sort_pairs_raw(const int32_t* keys, int n, int max_key, int32_t* keys_out,
                           int32_t* vals_out, int32_t* tmp_k, int32_t* tmp_v, int32_t* hist,
                           int32_t* scan_blk, cudaStream_t st, int* err = nullptr);
int sort_hist_len(int n);
int scan_blk_len(int n);
// Longest-first order of the segments by estimated work: length, times
// mlp_weight for segments of trajectories whose policy (pol, batch only) is an
// MLP kind.
cudaError_t build_lpt(Instance* I, const BatchPol* pol, int mlp_weight, cudaStream_t st);
// Scatter the sorted cache to time order (act_t), and also reduce the costs.
cudaError_t scatter_actions(Instance* I, cudaStream_t st);
cudaError_t finish_outputs(Instance* I, cudaStream_t st);

// Picard passes for any policy (pic_int.cu dispatches to the integer or MLP kernels).
// max_steps > 0: the window of Appendix A.3 (integer and MLP warp kernels).
cudaError_t picard_run(Instance* I, const pic_policy* pol, int max_iters, int flags,
                       const int8_t* alpha_init, unsigned long long timeout_ns, bool trace,
                       int max_steps, cudaStream_t st);
// Wave kernel (pic_wave.cu): MLP decisions in CTA-wide tensor-core waves
// (N <= 64); its work units are single runs (segment window 1).
bool wave_applies(const Instance* I);

// MLP policies (pic_mlp.cu).  mlp_prepare evaluates the per-region chain
// prefix (E rows through reg_local for a batch) and the FP32 weight copies.
cudaError_t mlp_alloc(Instance* I);
cudaError_t mlp_prepare(Instance* I, const pic_policy* pol, cudaStream_t st);
cudaError_t sequential_mlp(Instance* I, const pic_policy* pol, int flags, cudaStream_t st);
// Algorithm 1 with the product partition (pic_part.cu): processor of product k
// is k mod P; the cache I->act_t (time order) holds alpha^0 on entry and the
// last iterate on return; final stock in I->xfin; iters and converged in I->ctrl.
cudaError_t picard_products(Instance* I, const pic_policy* pol, int P, int iters_cap,
                            cudaStream_t st);
// Algorithm 1 for the assignment proc[t] in [0, P) (DEVICE), no capacity
// (pic_part.cu); contract as picard_products; a process outside [0, P) raises
// Ctrl::pad0 bit 128.
cudaError_t picard_assigned(Instance* I, const pic_policy* pol, const int32_t* proc, int P,
                            int iters_cap, cudaStream_t st);
// The same with node capacity (pic_acap.cu): every process replays the horizon
// up to its last own order in its own state, one warp each.
cudaError_t picard_assigned_cap(Instance* I, const pic_policy* pol, const int32_t* proc, int P,
                                int iters_cap, cudaStream_t st);
// Flag (Ctrl::pad0 bit 64) an initial cache holding a value outside [-1, N).
cudaError_t check_alpha_init(Instance* I, const int8_t* alpha, cudaStream_t st);
// Node capacity (pic_cap.cu): Algorithm 1 on M contiguous chunks of at most
// kCapChunk orders with the state (x, c), and the sequential simulator.
cudaError_t picard_cap(Instance* I, const pic_policy* pol, int M, int max_iters, int flags,
                       const int8_t* alpha_init, unsigned long long timeout_ns, bool trace,
                       cudaStream_t st);
cudaError_t sequential_cap(Instance* I, int kind, cudaStream_t st);
// Total cost and a^phi count of an action array (any order) with its regions.
cudaError_t reduce_costs(Instance* I, const int8_t* alpha, const int32_t* reg, cudaStream_t st);
cudaError_t sequential_int(Instance* I, int kind, cudaStream_t st);
bool smem_cost_ok(const Instance* I);

// Order tables of a batch instance for M chunks per trajectory and window W
// (built only if the current ones differ; pic_batch.cu).
pic_status batch_tables(Instance& I, int M, int W, cudaStream_t st);

// Error message plumbing shared by the entry points (pic_api.cu).
pic_status record_error(pic_status s, const char* msg);
void clear_error();
// Sizes, pointers and memory kind of an instance descriptor are acceptable.
bool desc_ok(const pic_instance_desc* d);

// Instance memory (pic_api.cu): device buffers for T orders, K products, N
// warehouses, R regions; free_instance releases whatever is allocated.
cudaError_t alloc_instance(Instance& I, int T, int N, int K, int R, bool has_lam);
void free_instance(Instance& I);
void free_pg(Instance& I);  // pic_pg.cu
// Range checks of an instance's device inputs (bits: 1 prod, 2 reg, 4 x0,
// 8/16/32 cost, lam, cost - lam beyond 2^23, 128 a cost outside int16); the
// result is left in ctrl->pad0.
cudaError_t launch_validate(Instance& I, cudaStream_t st);
// Per-segment Picard state sized for window W, with the look-back words cleared
// when fresh or when a call of at most iters_cap passes would exhaust the tags.
cudaError_t prepare_picard_state(Instance& I, int W, int iters_cap, cudaStream_t st);
// First kernel of a call's per-call work: takes iters_cap + 1 tags on the device.
cudaError_t take_tags(Instance& I, int iters_cap, cudaStream_t st);
// Cache start (a^phi, or alpha_init gathered to sorted order with its segment
// histograms) and the per-call resets of fc and xfin.
cudaError_t init_cache(Instance& I, const int8_t* alpha_init, cudaStream_t st);

// Device-wide exclusive scan of int32 (n elements, one pass, decoupled
// look-back); total written to *total_dev (if given).  blk: scan_blk_len(n)
// ints, zeroed once when allocated (it carries an epoch counter between
// scans); a look-back wait that runs out records PIC_ERR_TIMEOUT in *err.
// in and out may be the same array.
cudaError_t scan_exclusive(const int32_t* in, int32_t* out, int n, int32_t* total_dev,
                           int32_t* blk, cudaStream_t st, int* err = nullptr);

}  // namespace pic

// The opaque handle of the C ABI: a single trajectory, or a batch (I.batch set).
struct pic_instance {
    pic::Instance I;
};
