/*
 * fo_oracle.c -- plain, slow, obviously-correct CPU oracle for Picard-iteration
 * policy simulation of the fulfillment-optimization (FO) problem
 * ("Speeding up Policy Simulation in Supply Chain RL", Farias et al., ICML 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file; only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or constant generator with the
 * CUDA implementation.
 *
 * What it computes (paper section / equation / algorithm cited per function):
 *   - the sequential simulation a^seq_t = pi(s_t, w_t), s_{t+1} = f(s_t, a_t, w_t)
 *     (Sec. 2, problem statement) with the FO dynamics of Sec. 3 restricted to
 *     inventory only (no node capacity): x_{t+1} = x_t - e_{i(w_t), a_t};
 *   - Algorithm 1 (the Picard iteration) verbatim, every process replaying the
 *     whole horizon from s_1 ("literal");
 *   - Algorithm 1 on contiguous time chunks with the prefix of cached actions
 *     applied in closed form ("chunked"), see orc_picard_chunked for the reading;
 *   - the policies: greedy (Sec. 3.1), bid-price / dual with static prices
 *     (Sec. 4.2), an MLP scorer in a fixed FP32 operation order, and Gumbel-max
 *     sampling from counter-based Philox4x32-10 noise (Salmon et al., SC'11).
 *
 * Conventions: action -1 is a^phi ("do not fulfil", which the paper writes as 0),
 * otherwise a 0-based node (warehouse) index.  Ties go to the lowest node index;
 * a^phi is taken only when no node has stock (Appendix A.3: ties are broken
 * against a^phi).  Costs are minimised: the paper's reward r_j(w) is -cost[r][j].
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC (all FP32 fused
 * multiply-adds are explicit fmaf calls; no other contraction is allowed).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NOT_CONVERGED 4

#define ORC_GREEDY 0
#define ORC_DUAL 1
#define ORC_MLP 2
#define ORC_GUMBEL 3

#define ORC_EMB 16 /* region embedding width */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11).  Multipliers and Weyl key increments as published there. */
/* ------------------------------------------------------------------------- */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Uniform in (0,1): the top 23 bits of a Philox word, centred in their cell:
 * u = (w >> 9 + 1/2) 2^-23, every step exact in FP32, so u lies in
 * [2^-24, 1 - 2^-24] and both logarithms of the Gumbel transform stay finite.
 * Counter = (t, trajectory, n / 4, 0), key = (seed low word, seed high word);
 * node n takes output word n mod 4. */
float orc_uniform(uint64_t seed, int32_t traj, int64_t t, int32_t n) {
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)traj, (uint32_t)(n >> 2), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint32_t word = w[n & 3];
    return ((float)(word >> 9) + 0.5f) * 1.1920928955078125e-7f; /* 2^-23 */
}

/* Natural logarithm in FP32 from IEEE operations only, so that any IEEE-754
 * platform evaluates it to the same bits.  Method: x = m * 2^e with m in
 * [sqrt(1/2), sqrt(2)); log m = 2 atanh(f), f = (m-1)/(m+1), with the atanh
 * Taylor series f + f^3/3 + ... + f^11/11 (|f| <= 0.1716 so the next term is
 * below 2^-25 relative); ln 2 is split hi+lo (Cody & Waite range reduction).
 * Defined for finite x > 0 (the only inputs the Gumbel transform produces). */
float orc_log(float x) {
    uint32_t bits;
    memcpy(&bits, &x, 4);
    int32_t e = (int32_t)((bits >> 23) & 0xFF) - 127;
    uint32_t mbits = (bits & 0x007FFFFFu) | 0x3F800000u; /* m in [1,2) */
    float m;
    memcpy(&m, &mbits, 4);
    if (m > 1.41421356f) { m = m * 0.5f; e += 1; }
    float f = (m - 1.0f) / (m + 1.0f);
    float f2 = f * f;
    float p = 0.09090909090909091f;           /* 1/11 */
    p = fmaf(p, f2, 0.1111111111111111f);     /* 1/9 */
    p = fmaf(p, f2, 0.14285714285714285f);    /* 1/7 */
    p = fmaf(p, f2, 0.2f);                    /* 1/5 */
    p = fmaf(p, f2, 0.3333333333333333f);     /* 1/3 */
    float r = (2.0f * f) * f2;                /* exact doubling */
    float lm = fmaf(r, p, 2.0f * f);          /* 2f + 2f^3 p(f^2) */
    float ef = (float)e;
    const float ln2_hi = 0.693145751953125f;  /* 2839/4096: ef*ln2_hi is exact */
    const float ln2_lo = 1.4286068e-06f;      /* ln 2 - ln2_hi, rounded to FP32 */
    return fmaf(ef, ln2_hi, fmaf(ef, ln2_lo, lm));
}

float orc_gumbel(uint64_t seed, int32_t traj, int64_t t, int32_t n) {
    float u = orc_uniform(seed, traj, t, n);
    return -orc_log(-orc_log(u));
}

/* ------------------------------------------------------------------------- */
/* MLP scorer (the policy network of Sec. 4.1: two dense layers with a ReLU,
 * one score per node).  Parameters are BF16 bit patterns (upcast to FP32
 * exactly).  Layout: W1[IN][H] with IN = 2N+16 rows ordered
 * [cost (N) | stock (N) | emb (16)], b1[H], W2[H][N], b2[N], E[R][16].
 * Features: cost[r][n]/128, min(S_n,32)/32, E[r][e].  The paper fixes no FP32
 * evaluation order (it runs 16-bit JAX); this is the plain one, a single
 * sequential fmaf chain per output:
 *   h_j = b1_j, then one fmaf per input over the cost rows, the embedding rows
 *         and the stock rows (in that order); h_j = max(h_j, 0);
 *   s_n = b2_n, then one fmaf per hidden unit j = 0, 1, ..., H-1 (W2[j][n] h_j). */
/* ------------------------------------------------------------------------- */
static inline float bf16f(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

typedef struct {
    int N, H;
    const uint16_t *W1, *b1, *W2, *b2, *E;
} mlp_t;

void orc_mlp_scores(int N, int H, const uint16_t* W1, const uint16_t* b1, const uint16_t* W2,
                    const uint16_t* b2, const uint16_t* E, const int32_t* cost_row, int32_t r,
                    const int32_t* stock_row, float* s_out) {
    float* h = (float*)malloc(sizeof(float) * (size_t)H);
    for (int j = 0; j < H; ++j) {
        float a = bf16f(b1[j]);
        for (int n = 0; n < N; ++n)
            a = fmaf(bf16f(W1[(size_t)n * H + j]), (float)cost_row[n] / 128.0f, a);
        for (int e = 0; e < ORC_EMB; ++e)
            a = fmaf(bf16f(W1[(size_t)(2 * N + e) * H + j]), bf16f(E[(size_t)r * ORC_EMB + e]), a);
        for (int n = 0; n < N; ++n) {
            int32_t s = stock_row[n] < 32 ? stock_row[n] : 32;
            a = fmaf(bf16f(W1[(size_t)(N + n) * H + j]), (float)s / 32.0f, a);
        }
        h[j] = a > 0.0f ? a : 0.0f;
    }
    for (int n = 0; n < N; ++n) {
        float a = bf16f(b2[n]);
        for (int j = 0; j < H; ++j) a = fmaf(bf16f(W2[(size_t)j * N + n]), h[j], a);
        s_out[n] = a;
    }
    free(h);
}

/* ------------------------------------------------------------------------- */
/* The policy pi(s, w) for one order (product k, region r) at time t, given the
 * inventory row S = x[k][*].  Feasible set F = {n : S[n] > 0} (Sec. 3 action
 * set with the capacity condition dropped).  Returns -1 (a^phi) iff F is empty. */
/* ------------------------------------------------------------------------- */
typedef struct {
    int kind, N, R;
    const int32_t* cost; /* [R][N] */
    const int32_t* lam;  /* [K][N] (dual only) */
    mlp_t mlp;
    uint64_t seed;
    int32_t traj;
    float* scratch; /* N floats */
} policy_t;

static int policy_eval(policy_t* P, const int32_t* S, int32_t k, int32_t r, int64_t t) {
    const int N = P->N;
    int best = -1;
    if (P->kind == ORC_GREEDY || P->kind == ORC_DUAL) {
        int64_t bv = 0;
        for (int n = 0; n < N; ++n) {
            if (S[n] <= 0) continue;
            int64_t v = P->cost[(size_t)r * N + n];
            if (P->kind == ORC_DUAL) v -= P->lam[(size_t)k * N + n];
            if (best < 0 || v < bv) { best = n; bv = v; }
        }
        return best;
    }
    /* MLP argmax / Gumbel-max over F */
    orc_mlp_scores(N, P->mlp.H, P->mlp.W1, P->mlp.b1, P->mlp.W2, P->mlp.b2, P->mlp.E,
                   P->cost + (size_t)r * N, r, S, P->scratch);
    float bv = 0.0f;
    for (int n = 0; n < N; ++n) {
        if (S[n] <= 0) continue;
        float v = P->scratch[n];
        if (P->kind == ORC_GUMBEL) v = v + orc_gumbel(P->seed, P->traj, t, n);
        if (best < 0 || v > bv) { best = n; bv = v; }
    }
    return best;
}

static int policy_init(policy_t* P, int kind, int N, int R, const int32_t* cost, const int32_t* lam,
                       int H, const uint16_t* W1, const uint16_t* b1, const uint16_t* W2,
                       const uint16_t* b2, const uint16_t* E, uint64_t seed, int32_t traj) {
    if (kind < ORC_GREEDY || kind > ORC_GUMBEL) return ORC_ERR_ARG;
    if (kind == ORC_DUAL && !lam) return ORC_ERR_ARG;
    if ((kind == ORC_MLP || kind == ORC_GUMBEL) && (!W1 || !b1 || !W2 || !b2 || !E || H <= 0))
        return ORC_ERR_ARG;
    P->kind = kind; P->N = N; P->R = R; P->cost = cost; P->lam = lam;
    P->mlp.N = N; P->mlp.H = H; P->mlp.W1 = W1; P->mlp.b1 = b1; P->mlp.W2 = W2;
    P->mlp.b2 = b2; P->mlp.E = E; P->seed = seed; P->traj = traj;
    P->scratch = (float*)malloc(sizeof(float) * (size_t)N);
    return ORC_OK;
}

static int check_instance(int T, int N, int K, int R, const int32_t* prod, const int32_t* reg,
                          const int32_t* x0) {
    if (T < 0 || N <= 0 || N > 127 || K <= 0 || R <= 0) return ORC_ERR_ARG;
    for (int64_t t = 0; t < T; ++t)
        if (prod[t] < 0 || prod[t] >= K || reg[t] < 0 || reg[t] >= R) return ORC_ERR_ARG;
    for (int64_t i = 0; i < (int64_t)K * N; ++i)
        if (x0[i] < 0) return ORC_ERR_ARG;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Sequential simulation (Sec. 2 problem statement; FO dynamics of Sec. 3).
 * Outputs: act[T]; x_final[K][N] (may be NULL); total cost (sum of cost[r_t][a_t]
 * over fulfilled orders, a^phi costs 0); number of a^phi actions. */
/* ------------------------------------------------------------------------- */
int orc_seq_sim(int32_t T, int32_t N, int32_t K, int32_t R, const int32_t* prod, const int32_t* reg,
                const int32_t* x0, const int32_t* cost, const int32_t* lam, int32_t kind, int32_t H,
                const uint16_t* W1, const uint16_t* b1, const uint16_t* W2, const uint16_t* b2,
                const uint16_t* E, uint64_t seed, int32_t traj, int8_t* act, int32_t* x_final,
                int64_t* total_cost, int64_t* lost) {
    int rc = check_instance(T, N, K, R, prod, reg, x0);
    if (rc) return rc;
    policy_t P;
    rc = policy_init(&P, kind, N, R, cost, lam, H, W1, b1, W2, b2, E, seed, traj);
    if (rc) return rc;
    int32_t* x = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * N);
    memcpy(x, x0, sizeof(int32_t) * (size_t)K * N);
    int64_t c = 0, nl = 0;
    for (int64_t t = 0; t < T; ++t) {
        int32_t k = prod[t], r = reg[t];
        int32_t* row = x + (size_t)k * N;
        int a = policy_eval(&P, row, k, r, t);
        act[t] = (int8_t)a;
        if (a >= 0) {
            row[a] -= 1;
            c += cost[(size_t)r * N + a];
        } else {
            nl += 1;
        }
    }
    if (x_final) memcpy(x_final, x, sizeof(int32_t) * (size_t)K * N);
    if (total_cost) *total_cost = c;
    if (lost) *lost = nl;
    free(x);
    free(P.scratch);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1, verbatim, with process m owning the contiguous time block
 * [m*L, min((m+1)*L, T)), L = ceil(T/M).  Each process restarts from s_1 = x0,
 * evaluates pi on its own block and, on every other time-step before the end of
 * its block, applies the cached action alpha^{k-1}_t if it is feasible in the
 * process's own state, else a^phi.  (Time-steps after the block cannot influence
 * the block, so the replay stops at the block's end.)  The cache is rewritten on
 * each block; the loop returns when no cached action changed.
 *   iters_out  = number of passes of the while-loop body, including the pass
 *                that found no change;
 *   iterates   = optional [max_iters][T] record of alpha^1, alpha^2, ...;
 *   alpha_init = optional initial cache (NULL: every entry a^phi, as in Alg. 1).
 * Returns ORC_ERR_NOT_CONVERGED if max_iters passes do not reach a fixed point. */
/* ------------------------------------------------------------------------- */
int orc_picard_literal(int32_t T, int32_t N, int32_t K, int32_t R, const int32_t* prod,
                       const int32_t* reg, const int32_t* x0, const int32_t* cost,
                       const int32_t* lam, int32_t kind, int32_t H, const uint16_t* W1,
                       const uint16_t* b1, const uint16_t* W2, const uint16_t* b2, const uint16_t* E,
                       uint64_t seed, int32_t traj, int32_t M, int32_t max_iters,
                       const int8_t* alpha_init, int8_t* act_out, int32_t* iters_out,
                       int8_t* iterates) {
    int rc = check_instance(T, N, K, R, prod, reg, x0);
    if (rc) return rc;
    if (M <= 0 || max_iters <= 0) return ORC_ERR_ARG;
    policy_t P;
    rc = policy_init(&P, kind, N, R, cost, lam, H, W1, b1, W2, b2, E, seed, traj);
    if (rc) return rc;
    const int64_t L = ((int64_t)T + M - 1) / M;
    int8_t* prev = (int8_t*)malloc((size_t)T + 1);
    int8_t* next = (int8_t*)malloc((size_t)T + 1);
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * N);
    for (int64_t t = 0; t < T; ++t) prev[t] = alpha_init ? alpha_init[t] : (int8_t)-1;
    int converged = 0, k;
    for (k = 1; k <= max_iters; ++k) {
        for (int32_t m = 0; m < M; ++m) {
            int64_t lo = (int64_t)m * L, hi = lo + L < T ? lo + L : T;
            if (lo >= hi) continue;
            memcpy(s, x0, sizeof(int32_t) * (size_t)K * N); /* s^{k,m}_1 = s_1 */
            for (int64_t t = 0; t < hi; ++t) {
                int32_t pk = prod[t], r = reg[t];
                int32_t* row = s + (size_t)pk * N;
                int a;
                if (t >= lo) {
                    a = policy_eval(&P, row, pk, r, t); /* t in T_m: evaluate pi */
                    next[t] = (int8_t)a;
                } else {
                    a = prev[t]; /* cached action if feasible, else a^phi */
                    if (a >= 0 && !(a < N && row[a] > 0)) a = -1;
                }
                if (a >= 0) row[a] -= 1; /* f: x_{t+1} = x_t - e_{i(w_t), a_t} */
            }
        }
        if (iterates) memcpy(iterates + (size_t)(k - 1) * T, next, (size_t)T);
        int same = 1;
        for (int64_t t = 0; t < T; ++t)
            if (next[t] != prev[t]) { same = 0; break; }
        int8_t* tmp = prev; prev = next; next = tmp;
        if (same) { converged = 1; break; }
    }
    memcpy(act_out, prev, (size_t)T);
    *iters_out = converged ? k : max_iters;
    free(prev); free(next); free(s); free(P.scratch);
    return converged ? ORC_OK : ORC_ERR_NOT_CONVERGED;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 on the same contiguous blocks, with the prefix replay of line 5-7
 * (cached actions on t < block start) written in closed form.  Under the
 * inventory-only dynamics every (product k, node n) counter changes only when a
 * cached action for an order of product k names node n, and the feasibility
 * fallback of line 6 turns a decrement of an empty counter into a^phi; d such
 * events applied to x0[k][n] therefore leave max(0, x0[k][n] - d).  Each block
 * starts from that state and replays its own orders with fresh policy calls, in
 * time order.  Same outputs and iteration count as orc_picard_literal.
 *   changed_out (optional, [max_iters]) = number of cache entries changed by
 *   each pass; first_changed_out (optional) = smallest changed t per pass (T if
 *   none). */
/* ------------------------------------------------------------------------- */
int orc_picard_chunked(int32_t T, int32_t N, int32_t K, int32_t R, const int32_t* prod,
                       const int32_t* reg, const int32_t* x0, const int32_t* cost,
                       const int32_t* lam, int32_t kind, int32_t H, const uint16_t* W1,
                       const uint16_t* b1, const uint16_t* W2, const uint16_t* b2, const uint16_t* E,
                       uint64_t seed, int32_t traj, int32_t M, int32_t max_iters,
                       const int8_t* alpha_init, int8_t* act_out, int32_t* iters_out,
                       int8_t* iterates, int64_t* changed_out, int64_t* first_changed_out) {
    int rc = check_instance(T, N, K, R, prod, reg, x0);
    if (rc) return rc;
    if (M <= 0 || max_iters <= 0) return ORC_ERR_ARG;
    policy_t P;
    rc = policy_init(&P, kind, N, R, cost, lam, H, W1, b1, W2, b2, E, seed, traj);
    if (rc) return rc;
    const int64_t L = ((int64_t)T + M - 1) / M;
    int8_t* prev = (int8_t*)malloc((size_t)T + 1);
    int8_t* next = (int8_t*)malloc((size_t)T + 1);
    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * N);   /* prefix counts */
    int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * N);   /* block-local rows */
    int32_t* stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);   /* block that built row */
    for (int64_t t = 0; t < T; ++t) prev[t] = alpha_init ? alpha_init[t] : (int8_t)-1;
    int converged = 0, k;
    for (k = 1; k <= max_iters; ++k) {
        memset(D, 0, sizeof(int32_t) * (size_t)K * N);
        for (int32_t i = 0; i < K; ++i) stamp[i] = -1;
        for (int32_t m = 0; m < M; ++m) {
            int64_t lo = (int64_t)m * L, hi = lo + L < T ? lo + L : T;
            if (lo >= hi) break;
            for (int64_t t = lo; t < hi; ++t) {
                int32_t pk = prod[t], r = reg[t];
                int32_t* row = S + (size_t)pk * N;
                if (stamp[pk] != m) { /* first order of product pk in this block */
                    for (int n = 0; n < N; ++n) {
                        int32_t v = x0[(size_t)pk * N + n] - D[(size_t)pk * N + n];
                        row[n] = v > 0 ? v : 0;
                    }
                    stamp[pk] = m;
                }
                int a = policy_eval(&P, row, pk, r, t);
                next[t] = (int8_t)a;
                if (a >= 0) row[a] -= 1;
            }
            /* extend the prefix by this block's cached (previous-pass) actions */
            for (int64_t t = lo; t < hi; ++t) {
                int a = prev[t];
                if (a >= 0 && a < N) D[(size_t)prod[t] * N + a] += 1;
            }
        }
        int64_t nchg = 0, first = T;
        for (int64_t t = 0; t < T; ++t)
            if (next[t] != prev[t]) { if (first == T) first = t; nchg++; }
        if (iterates) memcpy(iterates + (size_t)(k - 1) * T, next, (size_t)T);
        if (changed_out) changed_out[k - 1] = nchg;
        if (first_changed_out) first_changed_out[k - 1] = first;
        int8_t* tmp = prev; prev = next; next = tmp;
        if (nchg == 0) { converged = 1; break; }
    }
    memcpy(act_out, prev, (size_t)T);
    *iters_out = converged ? k : max_iters;
    free(prev); free(next); free(D); free(S); free(stamp); free(P.scratch);
    return converged ? ORC_OK : ORC_ERR_NOT_CONVERGED;
}

/* Stock row of the order at time t under a given action path (the state s_t
 * that the policy saw), for sampled full-size checks: x0[k] minus the fulfilled
 * actions of product k before t. */
int orc_state_before(int32_t T, int32_t N, const int32_t* prod, const int8_t* act,
                     const int32_t* x0, int64_t t, int32_t* row_out) {
    if (t < 0 || t >= T) return ORC_ERR_ARG;
    int32_t k = prod[t];
    for (int n = 0; n < N; ++n) row_out[n] = x0[(size_t)k * N + n];
    for (int64_t u = 0; u < t; ++u)
        if (prod[u] == k && act[u] >= 0) row_out[act[u]] -= 1;
    return ORC_OK;
}

/* One policy call, exposed for sampled checks and unit pins. */
int orc_policy_call(int32_t N, int32_t R, const int32_t* cost, const int32_t* lam, int32_t kind,
                    int32_t H, const uint16_t* W1, const uint16_t* b1, const uint16_t* W2,
                    const uint16_t* b2, const uint16_t* E, uint64_t seed, int32_t traj,
                    const int32_t* stock_row, int32_t k, int32_t r, int64_t t) {
    policy_t P;
    if (policy_init(&P, kind, N, R, cost, lam, H, W1, b1, W2, b2, E, seed, traj)) return -2;
    int a = policy_eval(&P, stock_row, k, r, t);
    free(P.scratch);
    return a;
}

/* ========================================================================= */
/* FO with node capacity (Sec. 3).  The state is (x, c): inventory x[K][N] and
 * node capacity c[N].  An order of product k may go to node n only if
 * x[k][n] > 0 and c[n] > 0; f decrements both.  The integer policies (greedy,
 * bid-price) choose over that feasible set with the same scores as above, so a
 * policy call sees the row m[n] = (x[k][n] > 0 && c[n] > 0).  The MLP policies
 * take stock features and are not defined here with capacity. */
/* ========================================================================= */
static int check_cap(int32_t N, const int32_t* cap, int32_t kind) {
    if (kind != ORC_GREEDY && kind != ORC_DUAL) return ORC_ERR_ARG;
    for (int n = 0; n < N; ++n)
        if (cap[n] < 0) return ORC_ERR_ARG;
    return ORC_OK;
}

/* policy call on the feasible set of (row, c); c == NULL: no capacity */
static int cap_policy(policy_t* P, const int32_t* row, const int32_t* c, int32_t* mask, int32_t k,
                      int32_t r, int64_t t) {
    if (!c) return policy_eval(P, row, k, r, t);
    for (int n = 0; n < P->N; ++n) mask[n] = (row[n] > 0 && c[n] > 0) ? 1 : 0;
    return policy_eval(P, mask, k, r, t);
}

/* Sequential simulation with capacity.  Outputs as orc_seq_sim plus c_final[N]
 * (may be NULL). */
int orc_seq_sim_cap(int32_t T, int32_t N, int32_t K, int32_t R, const int32_t* prod,
                    const int32_t* reg, const int32_t* x0, const int32_t* cap, const int32_t* cost,
                    const int32_t* lam, int32_t kind, int8_t* act, int32_t* x_final,
                    int32_t* c_final, int64_t* total_cost, int64_t* lost) {
    int rc = check_instance(T, N, K, R, prod, reg, x0);
    if (rc) return rc;
    if (!cap || check_cap(N, cap, kind)) return ORC_ERR_ARG;
    policy_t P;
    rc = policy_init(&P, kind, N, R, cost, lam, 0, NULL, NULL, NULL, NULL, NULL, 0, 0);
    if (rc) return rc;
    int32_t* x = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * N);
    int32_t* c = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    int32_t* mask = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    memcpy(x, x0, sizeof(int32_t) * (size_t)K * N);
    memcpy(c, cap, sizeof(int32_t) * (size_t)N);
    int64_t tc = 0, nl = 0;
    for (int64_t t = 0; t < T; ++t) {
        int32_t k = prod[t], r = reg[t];
        int32_t* row = x + (size_t)k * N;
        int a = cap_policy(&P, row, c, mask, k, r, t);
        act[t] = (int8_t)a;
        if (a >= 0) {
            row[a] -= 1;
            c[a] -= 1;
            tc += cost[(size_t)r * N + a];
        } else {
            nl += 1;
        }
    }
    if (x_final) memcpy(x_final, x, sizeof(int32_t) * (size_t)K * N);
    if (c_final) memcpy(c_final, c, sizeof(int32_t) * (size_t)N);
    if (total_cost) *total_cost = tc;
    if (lost) *lost = nl;
    free(x); free(c); free(mask); free(P.scratch);
    return ORC_OK;
}

/* Algorithm 1 verbatim for an arbitrary assignment of time-steps to processes:
 * proc[t] in [0, M) is the process that owns t (contiguous blocks, product
 * partitions T_m = union of T_i over i in I_m, or a uniform random assignment).
 * Process m restarts from s_1 = (x0, cap), walks t = 0 .. its last own step,
 * evaluates pi on its own steps and applies the cached action elsewhere if it
 * is feasible in its own state (else a^phi).  cap == NULL: no capacity (then
 * every policy kind is allowed).  Outputs as orc_picard_literal. */
int orc_picard_partition(int32_t T, int32_t N, int32_t K, int32_t R, const int32_t* prod,
                         const int32_t* reg, const int32_t* x0, const int32_t* cap,
                         const int32_t* cost, const int32_t* lam, int32_t kind, int32_t H,
                         const uint16_t* W1, const uint16_t* b1, const uint16_t* W2,
                         const uint16_t* b2, const uint16_t* E, uint64_t seed, int32_t traj,
                         const int32_t* proc, int32_t M, int32_t max_iters,
                         const int8_t* alpha_init, int8_t* act_out, int32_t* iters_out,
                         int8_t* iterates) {
    int rc = check_instance(T, N, K, R, prod, reg, x0);
    if (rc) return rc;
    if (M <= 0 || max_iters <= 0 || !proc) return ORC_ERR_ARG;
    if (cap && check_cap(N, cap, kind)) return ORC_ERR_ARG;
    for (int64_t t = 0; t < T; ++t)
        if (proc[t] < 0 || proc[t] >= M) return ORC_ERR_ARG;
    policy_t P;
    rc = policy_init(&P, kind, N, R, cost, lam, H, W1, b1, W2, b2, E, seed, traj);
    if (rc) return rc;
    int64_t* last = (int64_t*)malloc(sizeof(int64_t) * (size_t)M);
    for (int32_t m = 0; m < M; ++m) last[m] = -1;
    for (int64_t t = 0; t < T; ++t) last[proc[t]] = t;
    int8_t* prev = (int8_t*)malloc((size_t)T + 1);
    int8_t* next = (int8_t*)malloc((size_t)T + 1);
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * N);
    int32_t* c = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    int32_t* mask = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    for (int64_t t = 0; t < T; ++t) prev[t] = alpha_init ? alpha_init[t] : (int8_t)-1;
    int converged = 0, k;
    for (k = 1; k <= max_iters; ++k) {
        for (int32_t m = 0; m < M; ++m) {
            if (last[m] < 0) continue;
            memcpy(s, x0, sizeof(int32_t) * (size_t)K * N); /* s^{k,m}_1 = s_1 */
            if (cap) memcpy(c, cap, sizeof(int32_t) * (size_t)N);
            for (int64_t t = 0; t <= last[m]; ++t) {
                int32_t pk = prod[t], r = reg[t];
                int32_t* row = s + (size_t)pk * N;
                int a;
                if (proc[t] == m) {
                    a = cap_policy(&P, row, cap ? c : NULL, mask, pk, r, t);
                    next[t] = (int8_t)a;
                } else {
                    a = prev[t];
                    if (a >= 0 && !(a < N && row[a] > 0 && (!cap || c[a] > 0))) a = -1;
                }
                if (a >= 0) {
                    row[a] -= 1;
                    if (cap) c[a] -= 1;
                }
            }
        }
        if (iterates) memcpy(iterates + (size_t)(k - 1) * T, next, (size_t)T);
        int same = 1;
        for (int64_t t = 0; t < T; ++t)
            if (next[t] != prev[t]) { same = 0; break; }
        int8_t* tmp = prev; prev = next; next = tmp;
        if (same) { converged = 1; break; }
    }
    memcpy(act_out, prev, (size_t)T);
    *iters_out = converged ? k : max_iters;
    free(last); free(prev); free(next); free(s); free(c); free(mask); free(P.scratch);
    return converged ? ORC_OK : ORC_ERR_NOT_CONVERGED;
}

/* Algorithm 1 with capacity on contiguous blocks [m*L, min((m+1)*L, T)), the
 * cached-prefix replay written in closed form.  Replaying cached actions before
 * a block, every decrement is conditional on positivity, and a node whose
 * capacity reached 0 never becomes feasible again; hence at the block start
 *   x[k][n] = max(0, x0[k][n] - D[k][n]) for every node with c[n] > 0, and
 *   c[n]    = max(0, cap[n] - Q[n]),
 * with D[k][n] = cached actions of product k naming n before the block, and
 * Q[n] = those cached actions naming n that found inventory, i.e. were taken
 * while the running D[k][n] was below x0[k][n] (the rows of nodes with c[n] = 0
 * are never consulted: such nodes are infeasible).  Each block then replays its
 * own orders from that state with fresh policy calls.  Same outputs, iterates
 * and iteration count as orc_picard_partition with proc[t] = t / L. */
int orc_picard_chunked_cap(int32_t T, int32_t N, int32_t K, int32_t R, const int32_t* prod,
                           const int32_t* reg, const int32_t* x0, const int32_t* cap,
                           const int32_t* cost, const int32_t* lam, int32_t kind, int32_t M,
                           int32_t max_iters, const int8_t* alpha_init, int8_t* act_out,
                           int32_t* iters_out, int8_t* iterates, int64_t* changed_out,
                           int64_t* first_changed_out) {
    int rc = check_instance(T, N, K, R, prod, reg, x0);
    if (rc) return rc;
    if (M <= 0 || max_iters <= 0 || !cap || check_cap(N, cap, kind)) return ORC_ERR_ARG;
    policy_t P;
    rc = policy_init(&P, kind, N, R, cost, lam, 0, NULL, NULL, NULL, NULL, NULL, 0, 0);
    if (rc) return rc;
    const int64_t L = ((int64_t)T + M - 1) / M;
    int8_t* prev = (int8_t*)malloc((size_t)T + 1);
    int8_t* next = (int8_t*)malloc((size_t)T + 1);
    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * N);
    int32_t* Q = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * N);
    int32_t* c = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    int32_t* mask = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    int32_t* stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
    for (int64_t t = 0; t < T; ++t) prev[t] = alpha_init ? alpha_init[t] : (int8_t)-1;
    int converged = 0, k;
    for (k = 1; k <= max_iters; ++k) {
        memset(D, 0, sizeof(int32_t) * (size_t)K * N);
        memset(Q, 0, sizeof(int32_t) * (size_t)N);
        for (int32_t i = 0; i < K; ++i) stamp[i] = -1;
        for (int32_t m = 0; m < M; ++m) {
            int64_t lo = (int64_t)m * L, hi = lo + L < T ? lo + L : T;
            if (lo >= hi) break;
            for (int n = 0; n < N; ++n) {
                int32_t v = cap[n] - Q[n];
                c[n] = v > 0 ? v : 0;
            }
            for (int64_t t = lo; t < hi; ++t) {
                int32_t pk = prod[t], r = reg[t];
                int32_t* row = S + (size_t)pk * N;
                if (stamp[pk] != m) { /* first order of product pk in this block */
                    for (int n = 0; n < N; ++n) {
                        int32_t v = x0[(size_t)pk * N + n] - D[(size_t)pk * N + n];
                        row[n] = v > 0 ? v : 0;
                    }
                    stamp[pk] = m;
                }
                int a = cap_policy(&P, row, c, mask, pk, r, t);
                next[t] = (int8_t)a;
                if (a >= 0) {
                    row[a] -= 1;
                    c[a] -= 1;
                }
            }
            /* extend the prefix by this block's cached (previous-pass) actions */
            for (int64_t t = lo; t < hi; ++t) {
                int a = prev[t];
                if (a < 0 || a >= N) continue;
                int32_t* d = D + (size_t)prod[t] * N + a;
                if (*d < x0[(size_t)prod[t] * N + a]) Q[a] += 1;
                *d += 1;
            }
        }
        int64_t nchg = 0, first = T;
        for (int64_t t = 0; t < T; ++t)
            if (next[t] != prev[t]) { if (first == T) first = t; nchg++; }
        if (iterates) memcpy(iterates + (size_t)(k - 1) * T, next, (size_t)T);
        if (changed_out) changed_out[k - 1] = nchg;
        if (first_changed_out) first_changed_out[k - 1] = first;
        int8_t* tmp = prev; prev = next; next = tmp;
        if (nchg == 0) { converged = 1; break; }
    }
    memcpy(act_out, prev, (size_t)T);
    *iters_out = converged ? k : max_iters;
    free(prev); free(next); free(D); free(Q); free(S); free(c); free(mask); free(stamp);
    free(P.scratch);
    return converged ? ORC_OK : ORC_ERR_NOT_CONVERGED;
}

/* ========================================================================= */
/* Algorithm 1 with the max_steps window of Appendix A.3, on the contiguous
 * blocks [m*L, min((m+1)*L, T)) (no capacity).  A pass evaluates the policy
 * only on the blocks that start before w_end = w_start + max_steps; later blocks
 * keep their cached actions.  The window is counted in whole blocks: a block is
 * evaluated whole once its first order is inside the window, so a pass
 * evaluates the orders before e = min(T, ceil(w_end / L) L).  The window starts
 * at 0; after a pass that changed some action it starts at the first changed
 * time t_reset (earlier actions are final); after a pass that changed nothing it
 * moves on to e (the evaluated blocks reached their fixed point from an exact
 * prefix).  The loop returns after a pass that changed nothing with e = T.  Blocks are replayed from
 * the closed-form prefix, as in orc_picard_chunked.  With max_steps >= T the
 * passes are those of orc_picard_chunked.  Outputs as orc_picard_chunked. */
/* ========================================================================= */
int orc_picard_windowed(int32_t T, int32_t N, int32_t K, int32_t R, const int32_t* prod,
                        const int32_t* reg, const int32_t* x0, const int32_t* cost,
                        const int32_t* lam, int32_t kind, int32_t H, const uint16_t* W1,
                        const uint16_t* b1, const uint16_t* W2, const uint16_t* b2,
                        const uint16_t* E, uint64_t seed, int32_t traj, int32_t M,
                        int64_t max_steps, int32_t max_iters, const int8_t* alpha_init,
                        int8_t* act_out, int32_t* iters_out, int8_t* iterates,
                        int64_t* changed_out, int64_t* first_changed_out) {
    int rc = check_instance(T, N, K, R, prod, reg, x0);
    if (rc) return rc;
    if (M <= 0 || max_iters <= 0 || max_steps <= 0) return ORC_ERR_ARG;
    policy_t P;
    rc = policy_init(&P, kind, N, R, cost, lam, H, W1, b1, W2, b2, E, seed, traj);
    if (rc) return rc;
    const int64_t L = ((int64_t)T + M - 1) / M;
    int8_t* prev = (int8_t*)malloc((size_t)T + 1);
    int8_t* next = (int8_t*)malloc((size_t)T + 1);
    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * N);
    int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * N);
    int32_t* stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
    for (int64_t t = 0; t < T; ++t) prev[t] = alpha_init ? alpha_init[t] : (int8_t)-1;
    int converged = 0, k;
    int64_t w_start = 0;
    for (k = 1; k <= max_iters; ++k) {
        const int64_t w_end = w_start + max_steps;
        memcpy(next, prev, (size_t)T);
        memset(D, 0, sizeof(int32_t) * (size_t)K * N);
        for (int32_t i = 0; i < K; ++i) stamp[i] = -1;
        for (int32_t m = 0; m < M; ++m) {
            int64_t lo = (int64_t)m * L, hi = lo + L < T ? lo + L : T;
            if (lo >= hi || lo >= w_end) break; /* blocks from here on keep their cache */
            for (int64_t t = lo; t < hi; ++t) {
                int32_t pk = prod[t], r = reg[t];
                int32_t* row = S + (size_t)pk * N;
                if (stamp[pk] != m) {
                    for (int n = 0; n < N; ++n) {
                        int32_t v = x0[(size_t)pk * N + n] - D[(size_t)pk * N + n];
                        row[n] = v > 0 ? v : 0;
                    }
                    stamp[pk] = m;
                }
                int a = policy_eval(&P, row, pk, r, t);
                next[t] = (int8_t)a;
                if (a >= 0) row[a] -= 1;
            }
            for (int64_t t = lo; t < hi; ++t) {
                int a = prev[t];
                if (a >= 0 && a < N) D[(size_t)prod[t] * N + a] += 1;
            }
        }
        int64_t nchg = 0, first = T;
        for (int64_t t = 0; t < T; ++t)
            if (next[t] != prev[t]) { if (first == T) first = t; nchg++; }
        if (iterates) memcpy(iterates + (size_t)(k - 1) * T, next, (size_t)T);
        if (changed_out) changed_out[k - 1] = nchg;
        if (first_changed_out) first_changed_out[k - 1] = first;
        int8_t* tmp = prev; prev = next; next = tmp;
        /* end of the evaluated blocks: every block that starts before w_end */
        int64_t e = ((w_end + L - 1) / L) * L;
        if (e > T) e = T;
        if (nchg == 0) {
            if (e >= T) { converged = 1; break; }
            w_start = e; /* the window converged: move on past its blocks */
        } else {
            w_start = first;
        }
    }
    memcpy(act_out, prev, (size_t)T);
    *iters_out = converged ? k : max_iters;
    free(prev); free(next); free(D); free(S); free(stamp); free(P.scratch);
    return converged ? ORC_OK : ORC_ERR_NOT_CONVERGED;
}
