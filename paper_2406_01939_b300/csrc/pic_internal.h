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
constexpr int kLenBuckets = 1024;  // segment-length buckets of the longest-first order
constexpr size_t kGrpSmemMax = 150 * 1024;  // cost table budget of the group-per-segment kernel

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
    int nruns;               // tables built by the preprocessing kernels
    int nseg;
    int last_m;              // chunk count the tables were built for
    int pad1;
};

// Per-segment metadata packed for one 32-byte load: product, run range, sorted
// position range, first order of the last run, chain (product) segment range.
struct __align__(32) SegMeta {
    int k, r0, r1, j0, jend, last_start, cf, ce;
};

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
    // iteration state
    int8_t *alpha_s;    // [T]  action cache in sorted order
    int32_t *agg;       // [SMAX][NP] histogram of cached actions per segment
    int32_t *carry;     // [SMAX][NP] in-super-block exclusive prefix of agg
    unsigned long long *sbagg;   // [SMAX][NP] super-block totals, (pass << 32) | value
    unsigned long long *sbincl;  // [SMAX][NP] inclusive chain prefix, (pass << 32) | value
    int32_t *fc;        // [2][K] first changed sorted position per product and pass parity
    int32_t *xfin;      // [K][N] final stock
    int32_t *xwork;     // [K][N] working stock of the sequential simulator
    int8_t *act_t;      // [T]  actions in time order (device staging)
    // MLP policy, per call: chain prefix per region and FP32 copies of the weights
    float *mlp_P;       // [R][256]
    float *mlp_W1s;     // [N][256] stock rows of W1
    float *mlp_W2;      // [256][N]
    float *mlp_b2;      // [N]
    // scratch for the sort and scans
    int32_t *tmp_a, *tmp_b, *tmp_c;   // [T] each
    int32_t *scan_blk;                // block sums
    int32_t *hist;                    // radix histograms
    int64_t hist_cap;
    Ctrl *ctrl;
    long long *trace;                 // [kTraceCap][4] device-side per-pass record
    int num_sms;
    int coop_blocks;                  // persistent grid size (integer kernel)
    int launches;                     // kernels launched by the current call
    cudaEvent_t ev[4];                // phase timing events (created with the instance)
};

// Preprocessing (pic_prep.cu): sort orders by product (stable in time), region
// gather, per-product offsets, runs for M chunks and segments of window W.
cudaError_t build_tables(Instance* I, int M, int W, cudaStream_t st);
// Scatter the sorted cache to time order and reduce segment costs.
cudaError_t finish_outputs(Instance* I, cudaStream_t st);

// Picard passes for any policy (pic_int.cu dispatches to the integer or MLP kernels).
cudaError_t picard_run(Instance* I, const pic_policy* pol, int max_iters, int flags,
                       const int8_t* alpha_init, unsigned long long timeout_ns, bool trace,
                       cudaStream_t st);
// MLP policies (pic_mlp.cu).
cudaError_t mlp_prepare(Instance* I, const pic_policy* pol, cudaStream_t st);
cudaError_t sequential_mlp(Instance* I, const pic_policy* pol, cudaStream_t st);
// Total cost and a^phi count of an action array (any order) with its regions.
cudaError_t reduce_costs(Instance* I, const int8_t* alpha, const int32_t* reg, cudaStream_t st);
cudaError_t sequential_int(Instance* I, int kind, cudaStream_t st);
bool smem_cost_ok(const Instance* I);

// Error message plumbing shared by the entry points (pic_api.cu).
pic_status record_error(pic_status s, const char* msg);
void clear_error();

// Simple device-wide exclusive scan of int32 (n elements); total written to *total_dev.
cudaError_t scan_exclusive(const int32_t* in, int32_t* out, int n, int32_t* total_dev,
                           int32_t* blk, cudaStream_t st);

}  // namespace pic
