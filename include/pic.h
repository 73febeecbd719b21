/*
 * pic.h -- C ABI of the B300 Picard-iteration policy simulator for the
 * fulfillment-optimization (FO) problem ("Speeding up Policy Simulation in
 * Supply Chain RL", Farias, Gijsbrechts, Khojandi, Peng, Zheng, ICML 2025).
 *
 * Problem (Sec. 2, policy simulation): given an initial state s_1, a horizon T
 * and disturbances w_1..w_T, compute the sample path of actions
 * a_t = pi(s_t, w_t), s_{t+1} = f(s_t, a_t, w_t).  Here (Sec. 3, FO model with
 * the node-capacity part left out) the state is the inventory x[K][N] of K
 * products at N warehouses (nodes), an order w_t = (product k_t, region r_t),
 * the action is a warehouse holding stock of k_t or a^phi (-1, do not fulfil),
 * and f decrements x[k_t][a_t].  Algorithm 1 (the Picard iteration) computes the
 * same path by iterating M parallel processes over a cache of actions.
 *
 * Conventions shared by every entry point
 *  - Every function returns a pic_status; on failure it writes no output and
 *    pic_last_error() returns a message (thread-local, valid until the next
 *    call on the same thread).
 *  - Array layouts are row-major, C-contiguous; sizes are element counts.
 *  - The caller owns every buffer it passes.  An instance owns the device
 *    copies it makes of its inputs (made at create / load time).
 *  - Device work is ordered on the CUDA stream given in the call (NULL = the
 *    legacy default stream); calls return after that work completed.
 *  - Actions: -1 = a^phi (no fulfilment), otherwise a 0-based warehouse index.
 *  - Limits: 1 <= N <= 127 (an action fits int8), 1 <= K <= 65535,
 *    1 <= R <= 65535, 0 <= T <= 2^31-1; x0 >= 0; for the integer policies
 *    |cost[r][n] - lam[k][n]| < 2^23.  Violations return PIC_ERR_INVALID_ARG.
 */
#ifndef PIC_H_
#define PIC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIC_OK = 0,
    PIC_ERR_INVALID_ARG = 1,   /* bad size, pointer, enum or value range */
    PIC_ERR_CUDA = 2,          /* a CUDA runtime call failed (message says which) */
    PIC_ERR_OOM = 3,           /* device allocation failed */
    PIC_ERR_NOT_CONVERGED = 4, /* max_iters passes without a fixed point */
    PIC_ERR_TIMEOUT = 5,       /* a device-side wait exceeded opts.timeout_ns */
    PIC_ERR_UNSUPPORTED = 6    /* valid request this build does not implement */
} pic_status;

/* Policy kinds (pic_policy.kind). */
enum {
    PIC_POLICY_GREEDY = 0, /* argmin_{n: x[k][n]>0} cost[r][n]; Sec. 3.1 greedy */
    PIC_POLICY_DUAL = 1,   /* argmin_{n: x[k][n]>0} cost[r][n] - lam[k][n]; bid-price, Sec. 4.2 */
    PIC_POLICY_MLP = 2,    /* argmax over stocked n of an MLP score, Sec. 4.1 */
    PIC_POLICY_GUMBEL = 3  /* argmax over stocked n of MLP score + Gumbel noise */
};

/* Simulation modes (pic_sim_opts.mode). */
enum {
    PIC_MODE_PICARD = 0,    /* Algorithm 1 on contiguous time chunks */
    PIC_MODE_SEQUENTIAL = 1, /* one order at a time on the GPU (the baseline of Sec. 4) */
    PIC_MODE_PICARD_PRODUCTS = 2 /* Algorithm 1 with the product partition of Sec. 3: processor
                                    m owns the orders of the products k with k mod P = m,
                                    P = num_chunks (0: K); greedy and bid-price policies, with
                                    or without node capacity; single instances; no max_steps.
                                    Same fixed point; Thm. 3.1 bounds the passes by |Q_T| + 2
                                    (Q_T: nodes whose capacity runs out) */,
    PIC_MODE_PICARD_ASSIGNED = 3 /* Algorithm 1 for a caller's assignment of orders to
                                    processes (opts.proc, P = num_chunks >= 1), e.g. the
                                    uniform random assignment of Sec. 4.1 (Table 1); greedy and
                                    bid-price policies, no capacity, single instances, no
                                    max_steps.  Same fixed point (Prop. 1) */
};

/* Where a pointer lives. */
enum { PIC_MEM_HOST = 0, PIC_MEM_DEVICE = 1 };

/* pic_sim_opts.flags bits */
enum {
    PIC_FLAG_NO_RESET = 1,   /* recompute every chunk on every pass (no t_reset skipping) */
    PIC_FLAG_REUSE_TABLES = 2, /* keep the order/run tables of the previous call if its
                                 chunking matches (skip the per-call preprocessing) */
    PIC_FLAG_TIMING = 4,       /* time the phases with CUDA events (pic_sim_result *_ms) */
    PIC_FLAG_GROUP_KERNEL = 8, /* tuning: replay each work unit with a group of 8 warehouses
                                  per lane instead of a whole warp (integer policies, costs
                                  that fit int16) */
    PIC_FLAG_GRAPH = 16,       /* pic_simulate_batch: run the per-call device work as a CUDA
                                  graph, captured at the first call and relaunched while the
                                  chunking, CTA shape, MLP weight pointers, alpha_init, trace,
                                  max_iters, timeout and flags stay the same */
    PIC_FLAG_NO_TC = 32,       /* MLP policies: score every decision with the FP32 scorer
                                  (no tensor-core tiles; see PIC_FLAG_TC) */
    PIC_FLAG_TC = 64,          /* MLP policies (N <= 64), the default unless PIC_FLAG_NO_TC:
                                  inside long runs of a product whose stocked warehouses all
                                  hold more than 32 units, score up to 16 orders at a time on
                                  the tensor cores (BF16 inputs, FP32 accumulation) and
                                  re-score in FP32 every order whose top-2 margin is below
                                  max(1e-3, twice a computed error bound); same results as the
                                  FP32 scorer.  With num_chunks = 0 the batch autotuner
                                  decides unless one of the two flags is given */
    PIC_FLAG_WARP_GROUP = 256, /* MLP policies with N <= 64, pic_simulate: four warps share
                                  each decision (two hidden units per thread, the layer-2
                                  chains split in two halves), which shortens the decisions
                                  on a pass's critical path; same operations in the same
                                  order, so the same actions; no tensor-core tiles.  Applies
                                  to the sequential mode as well */
    PIC_FLAG_NO_SAT = 128,     /* MLP policies: evaluate the network for every decision.  By
                                  default a decision whose product holds at least 32 units at
                                  every warehouse (every stock feature min(x,32)/32 equals 1)
                                  takes its FP32 scores from a per-region table computed at
                                  the start of the call by the same scorer in the same
                                  operation order, so the actions are the same */
    PIC_FLAG_WAVE = 512,       /* MLP policies with N <= 64 (pic_simulate,
                                  pic_simulate_batch, pic_policy_grad):
                                  replay the work units in CTA-wide waves, one unit per thread
                                  of 128, every pending decision of a wave scored at once on
                                  the tensor cores (tcgen05, BF16 operands with FP32
                                  accumulation) and kept when its top-2 margin exceeds twice
                                  a bound on the difference from the reference FP32 order,
                                  else re-scored by the FP32 scorer; the actions are the same.
                                  A wave with at most 16 network decisions runs them on the
                                  FP32 scorer instead (one warp each); with PIC_FLAG_TC every
                                  wave uses the tensor cores, with PIC_FLAG_NO_TC none does.
                                  Greedy and bid-price trajectories of a batch, and
                                  saturated-state decisions, are decided in the same waves.
                                  The work units are single runs (segment window 1).
                                  Ignored where it does not apply.  pic_simulate_batch and
                                  pic_policy_grad with num_chunks = 0 time this kernel as
                                  one of the autotuner's choices */
    PIC_FLAG_NO_WAVE = 1024    /* exclude the wave kernel from the autotuner's choices */
};

typedef struct pic_instance pic_instance;

/* One FO trajectory's inputs. */
typedef struct {
    int32_t T, N, K, R;
    const int32_t* prod; /* [T] product k_t of order t, 0 <= k_t < K */
    const int32_t* reg;  /* [T] region r_t of order t, 0 <= r_t < R */
    const int32_t* x0;   /* [K][N] initial inventory s_1, >= 0 */
    const int32_t* cost; /* [R][N] fulfilment cost (the paper's reward is -cost) */
    const int32_t* lam;  /* [K][N] dual prices for PIC_POLICY_DUAL, or NULL */
    int32_t mem;         /* PIC_MEM_HOST or PIC_MEM_DEVICE: where the arrays above live */
    void* stream;        /* cudaStream_t for the copies and preprocessing, or NULL */
    const int32_t* cap;  /* [N] node capacity c_1 >= 0 (Sec. 3's state (x, c)), or NULL: no
                            capacity constraint.  With capacity an order may go to node n only
                            if x[k][n] > 0 and c[n] > 0, and f decrements both; greedy and
                            bid-price policies only; single instances only (not batches) */
} pic_instance_desc;

/* Policy.  MLP parameters are BF16 bit patterns in DEVICE memory, borrowed for
 * the duration of the call: W1[2N+16][H] with rows [cost (N) | stock (N) |
 * region embedding (16)], b1[H], W2[H][N], b2[N], E[R][16]; H must be 256.
 * Features: cost[r][n]/128, min(x[k][n],32)/32, E[r][0..16). */
typedef struct {
    int32_t kind;   /* PIC_POLICY_* */
    int32_t hidden; /* H (MLP kinds only) */
    const uint16_t *W1, *b1, *W2, *b2, *E;
    uint64_t seed;  /* Gumbel noise key (PIC_POLICY_GUMBEL) */
    int32_t traj;   /* trajectory id in the noise counter (PIC_POLICY_GUMBEL) */
} pic_policy;

typedef struct {
    int32_t mode;             /* PIC_MODE_* */
    int32_t num_chunks;       /* M >= 1 time chunks (Picard); 0 = pick automatically.
                                 PIC_MODE_PICARD_PRODUCTS: P processors (product k -> k mod P;
                                 0 or P > K: K) */
    int32_t max_iters;        /* cap on passes; 0 = M + 1 (Prop. 1 bound plus the confirming pass);
                                 PIC_MODE_PICARD_PRODUCTS: 0 = T + 1 */
    int32_t flags;            /* PIC_FLAG_* */
    const int8_t* alpha_init; /* DEVICE [T] initial action cache, or NULL = all a^phi (Alg. 1) */
    uint64_t timeout_ns;      /* bound on the device-side waits of the simulation kernel,
                                 measured from its start; 0 = 10 s (60 s for a batch) */
    int32_t out_mem;          /* PIC_MEM_HOST / PIC_MEM_DEVICE for the output arrays */
    int32_t seg_window;       /* tuning: orders of one product per warp work unit; 0 = 64
                                 (greedy, bid-price) or 8 (MLP policies) */
    void* stream;             /* cudaStream_t or NULL */
    int64_t* trace;           /* PIC_MODE_PICARD: HOST [trace_cap][6] per-pass record, or NULL (the
                                 other modes leave it untouched): ns from the
                                 simulation kernel's start to the end of the pass's prefix
                                 phase, ns to the end of its replay phase, policy calls in the
                                 pass, work units replayed in the pass, policy calls of the
                                 pass's largest work unit, orders walked by its longest work
                                 unit (the last two: the pass's critical path of sequential
                                 decisions) */
    int32_t trace_cap;        /* rows available in trace */
    int32_t max_steps;        /* PIC_MODE_PICARD on a single instance without capacity: the
                                 window of Appendix A.3, or 0 for none.  A pass evaluates the
                                 policy only on the chunks that start before w + max_steps
                                 (whole chunks); w is 0 at first, then the first time changed
                                 by the previous pass, or, after a pass that changed nothing,
                                 the end of the chunks it evaluated.  The call returns after a
                                 pass that changed nothing and evaluated every chunk.  The
                                 result is still the sequential path; max_iters defaults to
                                 2 M + 2.  Batches reject it (UNSUPPORTED) */
    const int32_t* proc;      /* PIC_MODE_PICARD_ASSIGNED: DEVICE [T] process of each order,
                                 0 <= proc[t] < num_chunks (else INVALID_ARG), with
                                 num_chunks * K < 2^31; ignored by the other modes */
} pic_sim_opts;

typedef struct {
    int64_t total_cost;   /* sum of cost[r_t][a_t] over fulfilled orders */
    int64_t lost;         /* number of a^phi actions */
    int64_t policy_calls; /* policy evaluations performed, over all passes */
    int32_t iters;        /* passes of Algorithm 1's loop, including the confirming one
                             (1 for PIC_MODE_SEQUENTIAL); also the rows written to opts.trace
                             (at most trace_cap) */
    int32_t num_chunks;   /* M used (P with PIC_MODE_PICARD_PRODUCTS) */
    int64_t rescored;     /* MLP tile rows re-scored in FP32 (top-2 margin below the bound) */
    int64_t seg_replays;  /* warp work units (segments) replayed, over all passes */
    int32_t launches;     /* kernels this call launched */
    float prep_ms;        /* PIC_FLAG_TIMING: order tables (sort, runs, segments) */
    float sim_ms;         /* PIC_FLAG_TIMING: the simulation kernel (all passes) */
    float total_ms;       /* PIC_FLAG_TIMING: whole call on the device, first to last kernel */
    int32_t seg_window;   /* segment window used (Picard) */
    int32_t cta_threads;  /* threads per CTA of the Picard launch */
    int32_t ctas_per_sm;  /* CTAs per SM of the Picard launch */
    int64_t mlp_calls;    /* the policy_calls that evaluated an MLP / Gumbel policy */
    int64_t tc_decisions; /* MLP decisions taken from tensor-core tile scores (the rest of
                             mlp_calls ran the FP32 scorer; rescored counts tile rows sent
                             back to it because their top-2 margin was too small) */
    int64_t sat_decisions; /* MLP decisions taken from the saturated-state score table (see
                              PIC_FLAG_NO_SAT); mlp_calls - tc_decisions - sat_decisions ran
                              the FP32 scorer */
    int64_t near_ties;     /* FP32-scorer decisions whose fast layer-2 scores left a near tie
                              within their error bound, re-scored in the reference order
                              (one sequential fmaf chain per output, from the bias) */
    int32_t wave;          /* 1 if the MLP decisions ran in tensor-core waves (PIC_FLAG_WAVE,
                              set by the caller or chosen by the batch autotuner), else 0 */
} pic_sim_result;

/* Per-trajectory result of pic_simulate_batch. */
typedef struct {
    int64_t total_cost; /* sum of cost[r_t][a_t] over the trajectory's fulfilled orders */
    int64_t lost;       /* a^phi actions of the trajectory */
    int32_t iters;      /* passes after which the trajectory's cache stopped changing, plus
                           the confirming pass: what pic_simulate with min(M, T_b) chunks
                           reports for this trajectory alone (1 in PIC_MODE_SEQUENTIAL) */
    int32_t converged;  /* 1 if the trajectory reached its fixed point within the passes run */
} pic_traj_result;

/* Create an instance: validates and copies desc's arrays to the device, sized
 * for (T, N, K, R).  *out receives an owned handle (free with
 * pic_destroy_instance).  Errors: INVALID_ARG, OOM, CUDA. */
pic_status pic_create_instance(const pic_instance_desc* desc, pic_instance** out);

/* Replace an instance's inputs with new arrays of the same T, N, K, R (and lam,
 * cap present iff they were at create time), reusing its device memory.  Used to stream
 * new trajectories through one instance.  Errors: INVALID_ARG, CUDA. */
pic_status pic_instance_load(pic_instance* inst, const pic_instance_desc* desc);

/* Release an instance and its device memory (NULL is a no-op). */
void pic_destroy_instance(pic_instance* inst);

/* Simulate one trajectory (Sec. 2 policy simulation).  PIC_MODE_PICARD runs
 * Algorithm 1 with process m owning the contiguous orders
 * [m*L, min((m+1)*L, T)), L = ceil(T/M), the cache initialised to a^phi (or
 * opts.alpha_init), and stops at the first pass that changes no cached action;
 * the result equals the sequential path (Prop. 1).  PIC_MODE_SEQUENTIAL runs the
 * sequential definition directly.
 * With node capacity (desc.cap) each chunk replays its orders in time order,
 * because capacity couples products; its start state is the cached prefix in
 * closed form, x[k][n] = max(0, x0[k][n] - d[k][n]) and c[n] = max(0, c_1[n] - q[n])
 * with d the cached actions of product k naming n before the chunk and q those
 * of them that found inventory.  The chunk length ceil(T/M) must be at most 64
 * (num_chunks = 0 picks M = ceil(T/64)); seg_window and the MLP / group /
 * tensor-core flags do not apply.
 * PIC_MODE_PICARD_PRODUCTS runs Algorithm 1 with process m owning the orders of
 * the products k with k mod P = m (the product partition of Sec. 3): each pass a
 * process walks its own orders in time order, with its products' stock from its
 * own decisions and, with capacity, node n available before order t iff fewer
 * than c_1[n] cached actions found inventory at n before t once its own cached
 * ones are replaced by its fresh ones.  Greedy and bid-price policies only, no
 * max_steps (else UNSUPPORTED); device memory for the per-pass sorts is taken
 * with cudaMallocAsync on the call's stream.
 * PIC_MODE_PICARD_ASSIGNED runs Algorithm 1 with process proc[t] owning order t
 * (Sec. 4.1's uniform random partition, Table 1).  Without capacity, in a
 * process's view the stock of (k, n) before its order t is max(0, x0[k][n] -
 * attempts), the attempts being the cached actions naming (k, n) at other
 * processes' orders and its own fresh ones, so each (product, process) pair is
 * walked as an independent chain.  With node capacity no such closed form
 * exists (a foreign cached action's success depends on every earlier success
 * at its node in the process's own view), and every process replays the
 * horizon up to its last own order in its own state, one warp each: a pass
 * costs about num_chunks * T order-steps, and the scratch holds num_chunks * K *
 * N stock entries.  Same restrictions and allocation as
 * PIC_MODE_PICARD_PRODUCTS.
 *   actions_out  [T] int8 in opts.out_mem memory (required);
 *   final_stock  [K][N] int32 in opts.out_mem memory, or NULL;
 *   res          host struct, or NULL.
 * Errors: INVALID_ARG, UNSUPPORTED, NOT_CONVERGED (actions_out then holds the
 * last cache), TIMEOUT, CUDA. */
pic_status pic_simulate(pic_instance* inst, const pic_policy* pol, const pic_sim_opts* opts,
                        int8_t* actions_out, int32_t* final_stock, pic_sim_result* res);

/* Sequential simulation that allocates no device memory.  The paper has no
 * counterpart: this is a deployment variant of PIC_MODE_SEQUENTIAL for callers
 * that may not allocate device memory (a process whose own allocator owns all
 * device memory after start-up, or a latency-critical path that cannot absorb
 * cudaMalloc's implicit device synchronisation).  Instead of an instance it
 * reads the caller's DEVICE arrays in desc (desc->mem must be PIC_MEM_DEVICE)
 * and keeps its working stock and control block in a fixed 4 MiB array owned by
 * the library (a static device variable, held on every GPU that loads the
 * library until the process exits).
 *   kind         PIC_POLICY_GREEDY or PIC_POLICY_DUAL;
 *   actions_out  DEVICE [T] int8 (required when T > 0);
 *   final_stock  DEVICE [K][N] int32, or NULL;
 *   total_cost, lost  HOST, or NULL.
 * Limits: K*N <= 1,048,512 (else PIC_ERR_INVALID_ARG naming the limit);
 * |cost|, |lam| < 2^22.  The first call on each device resolves the array's
 * device address (with that device current) and should come before any stream
 * capture on it.  All calls share the array: calls whose work overlaps on the
 * same GPU race.  Synchronous on desc->stream.  Errors: INVALID_ARG,
 * UNSUPPORTED, CUDA. */
pic_status pic_simulate_sequential_static(const pic_instance_desc* desc, int32_t kind,
                                          int8_t* actions_out, int32_t* final_stock,
                                          int64_t* total_cost, int64_t* lost);

/* Create a batch instance from B trajectories' inputs (Sec. 4 simulates many
 * trajectories of one policy; each is its own FO instance).  All descs must
 * have the same N; T, K, R, lam presence and memory kind may differ per
 * trajectory; the work is ordered on descs[0].stream.  The batch is stored as
 * one combined instance: trajectory b's orders, products and regions occupy
 * their own index ranges in the order given, so trajectories never share state.
 * Limits: sum of T < 2^31, sum of K < 2^31, sum of R < 2^31.  Release with
 * pic_destroy_instance.  Errors: INVALID_ARG (names the trajectory), UNSUPPORTED
 * (a desc with cap), OOM, CUDA. */
pic_status pic_create_batch(const pic_instance_desc* descs, int32_t B, pic_instance** out);

/* Replace every trajectory's inputs of a batch instance with new arrays of the
 * same shapes, reusing its device memory: the batch analogue of
 * pic_instance_load, for a policy-gradient loop that samples new demand streams
 * each step (Sec. 4.2 estimates the gradient over such sampled trajectories).
 *   descs  HOST [B], B as at creation; desc b must have trajectory b's T, N, K,
 *          R and lam present iff it was at creation (no cap); its arrays are
 *          read (HOST or DEVICE per desc->mem) before the call returns, on
 *          descs[0].stream, which the call synchronises.
 * The same range checks as pic_create_batch run on the new inputs.  The order
 * tables and any captured per-call graph are rebuilt by the next call; the
 * autotuner's choice is kept.  Errors: INVALID_ARG (a shape mismatch or a
 * failed range check, naming it), UNSUPPORTED (cap), CUDA.  After a failed
 * check the batch's inputs are undefined: pic_simulate_batch and
 * pic_policy_grad return INVALID_ARG until a load succeeds. */
pic_status pic_batch_load(pic_instance* batch, const pic_instance_desc* descs, int32_t B);

/* Simulate every trajectory of a batch instance, each under its own policy,
 * in one persistent launch (PIC_MODE_PICARD) or one warp per trajectory
 * (PIC_MODE_SEQUENTIAL).
 *   pols         HOST [B]: policy of each trajectory.  Kinds may be mixed; every
 *                MLP / Gumbel policy of one call must use the same W1, b1, W2, b2,
 *                E pointers (seed and traj may differ), and E must then have
 *                max_b R_b rows (region r of trajectory b reads row r); bid-price
 *                needs the trajectory to have been created with lam.
 *   opts         as for pic_simulate, with num_chunks = M chunks per trajectory:
 *                trajectory b runs Algorithm 1 with min(M, T_b) contiguous chunks,
 *                exactly as pic_simulate would on it alone.  num_chunks = 0 runs
 *                the built-in autotuner (chunk count, CTA shape, segment window;
 *                timed trial launches on this batch, cached per batch and policy
 *                mix) and uses its choice; max_iters = 0 means (largest chunk
 *                count) + 1; alpha_init is DEVICE [sum T] in batch order.
 *   actions_out  [sum T] int8, trajectory b at offset T_0 + ... + T_{b-1};
 *   final_stock  [sum K][N] int32 in the same trajectory order, or NULL;
 *   traj         HOST [B] per-trajectory results, or NULL;
 *   res          HOST totals over the batch, or NULL (iters = passes run).
 * Errors: INVALID_ARG, UNSUPPORTED, NOT_CONVERGED, TIMEOUT, CUDA. */
pic_status pic_simulate_batch(pic_instance* batch, const pic_policy* pols,
                              const pic_sim_opts* opts, int8_t* actions_out, int32_t* final_stock,
                              pic_traj_result* traj, pic_sim_result* res);

/* Parameters and buffers of pic_policy_grad.  The flat parameter layout (FP32,
 * row-major) is W1 [(2N+16)][256] (rows: cost inputs, stock inputs, embedding
 * inputs) | b1 [256] | W2 [256][N] | b2 [N] | E [e_rows][16]. */
typedef struct {
    const float* master;   /* DEVICE FP32 parameters (masters), flat layout above */
    int32_t e_rows;        /* rows of E (>= every trajectory's R) */
    const int8_t* actions; /* DEVICE [sum T] paths to differentiate along (batch order), or
                              NULL to simulate them here (Picard, opts) under the policy
                              whose parameters are BF16(master) */
    int8_t* actions_out;   /* DEVICE [sum T] receives the paths used, or NULL */
    float* grad;           /* DEVICE FP32, flat layout: grad_scale * dJ/dtheta, or NULL to
                              compute the objective only */
    double grad_scale;
} pic_grad_args;

/* REINFORCE gradient of the MLP softmax policy along simulated paths (Sec. 4.2
 * trains its FO policy by policy gradient over simulated roll-outs):
 *   J = sum_b sum_t log pi(a_t | s_t) G_t,  G_t = -(sum of trajectory b's order
 *   costs cost[r_t'][a_t'] for t' >= t),
 * pi = softmax of the MLP scores over the warehouses holding stock; orders with
 * a_t = a^phi or fewer than 2 stocked warehouses contribute 0.  The paths are
 * held fixed; the policy's parameters are BF16(master) (round to nearest even)
 * and the gradient with respect to those BF16 values is returned for the
 * masters (straight-through).  With PIC_POLICY_GUMBEL paths, a_t is a sample of
 * pi, and dJ/dtheta is the REINFORCE estimate.  Hidden activations are
 * recomputed per order (no T x 256 storage).
 *   batch      a batch instance (pic_create_batch; one trajectory is a batch of 1),
 *              N <= 64;
 *   pols       HOST [B]: PIC_POLICY_MLP or PIC_POLICY_GUMBEL, hidden = 256, seed and
 *              traj per trajectory; weight pointers are ignored (BF16(master) is used);
 *   objective  HOST, or NULL: J.
 *   res        HOST, or NULL: the simulation's result when the paths are simulated here.
 * Errors: INVALID_ARG (also: given actions out of range or not a feasible path),
 * UNSUPPORTED, and those of pic_simulate_batch. */
pic_status pic_policy_grad(pic_instance* batch, const pic_policy* pols, const pic_grad_args* args,
                           const pic_sim_opts* opts, double* objective, pic_sim_result* res);

/* Message for the last non-OK status on this thread ("" if none). */
const char* pic_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H_ */
