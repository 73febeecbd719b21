/*
 * pic_owmr.h -- C ABI of the B300 Picard-iteration simulator for One-Warehouse
 * Multi-Retailer (OWMR) inventory control ("Speeding up Policy Simulation in
 * Supply Chain RL", Appendix B).
 *
 * Model (Appendix B.1), integer units.  State s_t = (x0, x_1..x_N): the central
 * warehouse and N retailers.  Step t brings demand d_t at retailer n_t.  The
 * action is a_t = (q_t, r_t): q_t units retailer n_t asks from the central
 * warehouse and r_t = 1 when the central warehouse replenishes up to S.  The
 * disturbance also carries e_t, the steps since the store's previous demand (the
 * demand history the retailer policy may use).  Any
 * action (fresh or cached) moves the state by
 *     y = max(0, x_n - d),  x_n <- y + min(q, x0),  x0 <- r ? S : max(0, x0 - q);
 * the demand lost at t is max(0, d - x_n).
 *
 * Policy (Appendix B.2).  The retailer's q depends only on its own inventory and
 * on the disturbance: base = (y <= s_n) ? S_n - y : 0 and, with a network,
 * q = clamp(floor(base + z), 0, c_n - y), z = MLP(y, d, e / 4096) in FP32 (the order is
 * given with pic_owmr_policy); without one, q = base.  The central warehouse
 * follows (s, S): r = [x0 - q <= s].
 *
 * Picard iteration (Algorithm 1 with the retailer partition of Appendix B.2).
 * Processor m owns the steps of retailers n with n mod P = m.  Each pass, every
 * processor runs the whole horizon from s_1.  It takes its own steps' actions
 * from the policy and every other step's action from the cache alpha^{k-1}.
 * alpha^k takes each step's action from the step's owner.  The call returns
 * after the first pass that changes nothing.  That result is the sequential path
 * (Prop. 1).  Under Theorem B.1's conditions (s >= every c_n, X0 > s) the cache
 * is the sequential path after at most 2R + 1 passes from an empty cache.  R is
 * the path's number of replenishments.  The call then takes one more pass to
 * confirm it.
 *
 * Conventions are those of pic.h: pic_status returns, pic_last_error(),
 * row-major arrays, caller-owned buffers, work ordered on the given stream
 * (calls return after it completed).  Actions are encoded as 2 q + r (int32).
 * Limits (else PIC_ERR_INVALID_ARG): 1 <= N <= 65,536; 0 <= T <= 2^31 - 1;
 * 0 <= d_t < 32,768; 0 <= e_t < 32,768; 0 <= x0_n <= c_n < 2^20; 0 <= s_n <= S_n <= c_n;
 * 0 <= s < S < 2^30; 0 <= X0 < 2^30; T * max(c_n) < 2^31 (prefix sums of q
 * fit int32).
 */
#ifndef PIC_OWMR_H_
#define PIC_OWMR_H_

#include <stdint.h>

#include "pic.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_owmr pic_owmr;

/* One OWMR trajectory's inputs. */
typedef struct {
    int32_t T, N;
    const int32_t* ret; /* [T] retailer n_t of step t, 0 <= n_t < N */
    const int32_t* dem; /* [T] demand d_t */
    const int32_t* ex;  /* [T] exogenous feature e_t (steps since the store's previous demand) */
    const int32_t* cap; /* [N] retailer capacity c_n */
    const int32_t* x0r; /* [N] initial retailer inventory */
    const int32_t* sl;  /* [N] retailer reorder point s_n */
    const int32_t* Sl;  /* [N] retailer order-up-to level S_n */
    int32_t X0;         /* initial central inventory */
    int32_t s, S;       /* central (s, S) policy */
    int32_t mem;        /* PIC_MEM_HOST or PIC_MEM_DEVICE: where the arrays above live */
    void* stream;       /* cudaStream_t for the copies and validation, or NULL */
} pic_owmr_desc;

/* Retailer network: 3 -> H -> H -> 1 with ReLU, BF16 bit patterns in DEVICE
 * memory, borrowed for the call.  W1 [3][H] and W2 [H][H] are input-major
 * (W2[k][j] connects hidden unit k of layer 1 to unit j of layer 2); b1, b2,
 * w3 [H]; b3 [1].  FP32 order, features y, d and g = e * 2^-12 as floats:
 *   h1_k = relu(fma(W1[2][k], g, fma(W1[1][k], d, fma(W1[0][k], y, b1_k))))
 *   h2_j = relu(acc), acc = b2_j, then acc = fma(W2[k][j], h1_k, acc) for k = 0..H-1
 *   z    = b3, then z = fma(w3_j, h2_j, z) for j = 0..H-1;  relu(v) = v > 0 ? v : 0.
 * Every output is one sequential chain from its bias.  The kernels add the
 * output layer in groups of 8 first (a shorter chain) and keep a bound on the
 * difference; a q whose floor that bound leaves undecided is taken from z in
 * the order above (counted in pic_owmr_result.near_ties).
 * hidden = 0: no network (q = base).  Otherwise 64 <= H <= 512, H % 64 == 0. */
typedef struct {
    int32_t hidden;
    const uint16_t *W1, *b1, *W2, *b2, *w3, *b3;
} pic_owmr_policy;

typedef struct {
    int32_t mode;              /* PIC_MODE_PICARD or PIC_MODE_SEQUENTIAL (one step at a time
                                  on the GPU, the baseline of Appendix B.3) */
    int32_t num_procs;         /* P processors (Picard), 1 <= P <= N; 0 = N (one per retailer) */
    int32_t max_iters;         /* pass limit; 0 = T + 1 (Prop. 1) */
    int32_t flags;             /* PIC_FLAG_TIMING; PIC_FLAG_REUSE_TABLES: keep the previous
                                  call's per-processor step tables when P is the same
                                  (otherwise every call rebuilds them) */
    const int32_t* alpha_init; /* [T] DEVICE, initial cache (2 q + r, q >= 0), or NULL: all 0 */
    int64_t timeout_ns;        /* bound on each device-side wait; 0 = 60 s */
    int32_t max_steps;         /* max_steps window of Appendix A.3, in steps: a pass calls
                                  the policy only at steps t < w + max_steps and keeps the
                                  cached actions of later steps; w starts at 0, becomes the
                                  first changed step after a pass that changed the cache, and
                                  the end of the evaluated range after one that did not; the
                                  call ends after a pass that changed nothing with the range
                                  covering the horizon (same result).  0 = no window; the
                                  default max_iters is then T + 1 + T / max_steps + 1 */
} pic_owmr_opts;

typedef struct {
    int32_t iters;          /* passes (Picard; 0 in sequential mode) */
    int32_t procs;          /* P used */
    int64_t replenishments; /* R = sum of r_t on the returned path */
    int64_t lost;           /* demand lost on the returned path */
    int64_t shipped;        /* units shipped to retailers, sum of min(q_t, x0_t) */
    int64_t policy_calls;   /* network evaluations made (memoised across passes) */
    int64_t eval_rounds;    /* batched network rounds (Picard) */
    int32_t launches;       /* kernels this call launched */
    float ms_total;         /* device time of the call (PIC_FLAG_TIMING) */
    int64_t near_ties;      /* network calls whose q the fast output layer left undecided
                               within its error bound, re-evaluated in the reference order */
} pic_owmr_result;

/* Copy and validate an instance.  *out is owned by the caller and freed with
 * pic_owmr_destroy. */
pic_status pic_owmr_create(const pic_owmr_desc* desc, pic_owmr** out);

/* Simulate the instance under pol.  actions_out [T] (2 q + r) and, if not NULL,
 * state_out [N + 1] (x0 then x_1..x_N after step T) are written in out_mem
 * (PIC_MEM_HOST or PIC_MEM_DEVICE).  res may be NULL.  Returns
 * PIC_ERR_NOT_CONVERGED (outputs = last iterate) when max_iters passes all
 * changed something, PIC_ERR_TIMEOUT when a device wait ran out,
 * PIC_ERR_UNSUPPORTED when P leaves a 32-processor group with more than 4,096
 * retailers. */
pic_status pic_owmr_simulate(pic_owmr* h, const pic_owmr_policy* pol, const pic_owmr_opts* opts,
                             int32_t* actions_out, int32_t* state_out, int32_t out_mem,
                             pic_owmr_result* res, void* stream);

void pic_owmr_destroy(pic_owmr* h);

#ifdef __cplusplus
}
#endif

#endif /* PIC_OWMR_H_ */
