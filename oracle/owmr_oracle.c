/*
 * CPU oracle for the One-Warehouse-Multi-Retailer (OWMR) inventory-control
 * extension (Appendix B) -- TEST INFRASTRUCTURE.  Only tests, the smoke check
 * and the benchmark's CPU legs use it; it shares no code with the CUDA path.
 *
 * Model (Appendix B.1), integer units.  State s_t = (x0, x_1..x_N): central
 * warehouse and N retailers.  Disturbance w_t = (retailer n_t, demand d_t,
 * e_t = steps since the store's previous demand: the demand history the policy
 * may use).
 * Action a_t = (q_t, r_t): q_t >= 0 units retailer n_t asks from the central
 * warehouse, r_t = 1 when the central warehouse replenishes (order up to S).
 * Transition for any action (cached or fresh):
 *     y = max(0, x_n - d), x_n <- y + min(q, x0),  x0 <- r ? S : max(0, x0 - q)
 * Lost demand at t: max(0, d - x_n).  Actions are stored as 2 q + r.
 *
 * Policy (Appendix B.2): the retailer's q depends on its own inventory and on
 * the disturbance only; the central warehouse follows (s, S): r = [x0 - q <= s].
 * Retailer rule (a reading; the appendix fixes the network's size, not its
 * inputs or output map): base = (y <= s_n) ? S_n - y : 0; with a network,
 * q = clamp(floor(base + z), 0, c_n - y) where z = MLP(y, d, e / 4096) in FP32 in
 * the fixed operation order of owmr_mlp() below; without one, q = min(base, c_n - y).
 *
 * Picard iteration (Algorithm 1 with the retailer partition of Appendix B.2:
 * processor m owns the time steps of its retailers).  Pass k: every processor
 * replays the whole horizon from s_1, taking its own steps' actions from the
 * policy and every other step's action from the cache alpha^{k-1}; alpha^k
 * takes each step's action from its owner.  The loop returns after the first
 * pass that changed nothing.
 *
 * Parity status: every function here is pinned by tests/test_oracle_owmr.py
 * (sequential path against a hand-derived trace and closed forms; the literal
 * iteration against Prop. 1 and Theorem B.1's replenishment bound; the walk
 * against the literal iteration pass by pass; the network against an FP64
 * evaluation within its rounding bound).  None is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OK 0
#define ERR_ARG 1
#define ERR_NOT_CONVERGED 4

static float bf16f(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

typedef struct {
    int H;                   /* 0: no network */
    const uint16_t *W1;      /* [3][H]  input-major: W1[i*H + k] */
    const uint16_t *b1;      /* [H] */
    const uint16_t *W2;      /* [H][H]  input-major: W2[k*H + j] */
    const uint16_t *b2;      /* [H] */
    const uint16_t *w3;      /* [H] */
    const uint16_t *b3;      /* [1] */
} Net;

/* The network's FP32 output z for features (y, d, g = e * 2^-12), in this order:
 *   h1_k = relu(fma(W1[2][k], g, fma(W1[1][k], d, fma(W1[0][k], y, b1_k))))
 *   h2_j = relu(b2_j + sum_k W2[k][j] h1_k), one fma per k in increasing k
 *   z    = b3, then one fma per j in increasing j (w3_j h2_j),
 * relu(v) = v > 0 ? v : 0.  Every output is one sequential fma chain: the
 * appendix fixes no FP32 order, and this is the plain one. */
float owmr_mlp(const Net* net, int y, int d, int e, float* h1, float* h2) {
    const int H = net->H;
    const float fy = (float)y, fd = (float)d, fg = (float)e * 0.000244140625f; /* exact */
    for (int k = 0; k < H; ++k) {
        float a = fmaf(bf16f(net->W1[k]), fy, bf16f(net->b1[k]));
        a = fmaf(bf16f(net->W1[H + k]), fd, a);
        a = fmaf(bf16f(net->W1[2 * H + k]), fg, a);
        h1[k] = a > 0.f ? a : 0.f;
    }
    for (int j = 0; j < H; ++j) {
        float a = bf16f(net->b2[j]);
        for (int k = 0; k < H; ++k) a = fmaf(bf16f(net->W2[(size_t)k * H + j]), h1[k], a);
        h2[j] = a > 0.f ? a : 0.f;
    }
    float z = bf16f(net->b3[0]);
    for (int j = 0; j < H; ++j) z = fmaf(bf16f(net->w3[j]), h2[j], z);
    return z;
}

typedef struct {
    int T, N;
    const int32_t *ret, *dem, *ex, *cap, *x0r, *sl, *Sl;
    int X0, s, S;
    Net net;
    float *h1, *h2; /* scratch [H] */
} Model;

/* Retailer order quantity for post-demand inventory y (Appendix B.2's pi_n). */
static int retailer_q(Model* M, int n, int y, int d, int e, long long* evals) {
    const int base = y <= M->sl[n] ? M->Sl[n] - y : 0;
    const int room = M->cap[n] - y;
    if (M->net.H == 0) return base < room ? base : room;
    ++*evals;
    const float z = owmr_mlp(&M->net, y, d, e, M->h1, M->h2);
    float v = floorf((float)base + z);
    v = v > 0.f ? v : 0.f;               /* NaN-free: z is finite for finite weights */
    if (v > (float)room) v = (float)room;
    return (int)v;
}

static int check(const Model* M) {
    if (M->T < 0 || M->N < 1 || M->s < 0 || M->S <= M->s || M->X0 < 0) return ERR_ARG;
    if (M->net.H < 0 || M->net.H % 64 || M->net.H > 512) return ERR_ARG;
    for (int n = 0; n < M->N; ++n)
        if (M->cap[n] < 0 || M->x0r[n] < 0 || M->x0r[n] > M->cap[n] || M->sl[n] < 0 ||
            M->Sl[n] < M->sl[n] || M->Sl[n] > M->cap[n]) return ERR_ARG;
    for (int t = 0; t < M->T; ++t)
        if (M->ret[t] < 0 || M->ret[t] >= M->N || M->dem[t] < 0 || M->ex[t] < 0 ||
            M->ex[t] >= 32768) return ERR_ARG;
    return OK;
}

static int setup(Model* M, int T, int N, const int32_t* ret, const int32_t* dem,
                 const int32_t* ex, const int32_t* cap, const int32_t* x0r, const int32_t* sl, const int32_t* Sl,
                 int X0, int s, int S, int H, const uint16_t* W1, const uint16_t* b1,
                 const uint16_t* W2, const uint16_t* b2, const uint16_t* w3, const uint16_t* b3) {
    M->T = T; M->N = N; M->ret = ret; M->dem = dem; M->ex = ex; M->cap = cap; M->x0r = x0r;
    M->sl = sl; M->Sl = Sl; M->X0 = X0; M->s = s; M->S = S;
    M->net.H = H; M->net.W1 = W1; M->net.b1 = b1; M->net.W2 = W2; M->net.b2 = b2;
    M->net.w3 = w3; M->net.b3 = b3;
    M->h1 = M->h2 = NULL;
    int e = check(M);
    if (e) return e;
    if (H) {
        M->h1 = (float*)malloc(sizeof(float) * H);
        M->h2 = (float*)malloc(sizeof(float) * H);
    }
    return OK;
}

static void teardown(Model* M) {
    free(M->h1);
    free(M->h2);
}

/* Sequential simulation (the baseline of Appendix B.3): act[t] = 2 q_t + r_t,
 * xfin = (x0, x_1..x_N) after step T, stats = (R = sum r, lost units, shipped
 * units sum min(q, x0), policy evaluations). */
int orc_owmr_seq(int T, int N, const int32_t* ret, const int32_t* dem, const int32_t* ex,
                 const int32_t* cap,
                 const int32_t* x0r, const int32_t* sl, const int32_t* Sl, int X0, int s, int S,
                 int H, const uint16_t* W1, const uint16_t* b1, const uint16_t* W2,
                 const uint16_t* b2, const uint16_t* w3, const uint16_t* b3, int32_t* act,
                 int32_t* xfin, int64_t* stats) {
    Model M;
    int e = setup(&M, T, N, ret, dem, ex, cap, x0r, sl, Sl, X0, s, S, H, W1, b1, W2, b2, w3, b3);
    if (e) return e;
    int32_t* x = (int32_t*)malloc(sizeof(int32_t) * (N ? N : 1));
    memcpy(x, x0r, sizeof(int32_t) * N);
    long long x0 = X0, R = 0, lost = 0, shipped = 0, evals = 0;
    for (int t = 0; t < T; ++t) {
        const int n = ret[t], d = dem[t];
        const int y = x[n] > d ? x[n] - d : 0;
        lost += d > x[n] ? d - x[n] : 0;
        const int q = retailer_q(&M, n, y, d, ex[t], &evals);
        const int r = x0 - q <= s;
        const long long recv = q < x0 ? q : x0;
        shipped += recv;
        x[n] = (int32_t)(y + recv);
        x0 = r ? S : (x0 > q ? x0 - q : 0);
        R += r;
        act[t] = 2 * q + r;
    }
    if (xfin) {
        xfin[0] = (int32_t)x0;
        memcpy(xfin + 1, x, sizeof(int32_t) * N);
    }
    if (stats) { stats[0] = R; stats[1] = lost; stats[2] = shipped; stats[3] = evals; }
    free(x);
    teardown(&M);
    return OK;
}

static int check_procs(int N, int P, const int32_t* proc) {
    if (P < 1) return ERR_ARG;
    for (int n = 0; n < N; ++n)
        if (proc[n] < 0 || proc[n] >= P) return ERR_ARG;
    return OK;
}

/* The max_steps window (Appendix A.3).  A pass evaluates the policy only at
 * steps t < w + window; later steps keep their cached actions.  w starts at 0;
 * after a pass that changed the cache, w is the first changed step; after a
 * pass that changed nothing, w moves to the end of the evaluated range, and the
 * iteration ends once that range covered the horizon.  window = 0: no window. */
static int window_end(int T, int w, int window) {
    if (window <= 0) return T;
    const long long e = (long long)w + window;
    return e < T ? (int)e : T;
}

static int first_change(const int32_t* a, const int32_t* b, int T) {
    for (int t = 0; t < T; ++t)
        if (a[t] != b[t]) return t;
    return -1;
}

/* Algorithm 1, literally: every pass, every processor replays the whole horizon
 * from s_1 and calls the policy at each of its own steps.  init = alpha^0 (NULL:
 * q = 0, r = 0 everywhere).  record (optional, [max_iters][T]) receives alpha^k.
 * Returns ERR_NOT_CONVERGED if max_iters passes change something every time. */
int orc_owmr_picard_literal(int T, int N, const int32_t* ret, const int32_t* dem, const int32_t* ex,
                            const int32_t* cap, const int32_t* x0r, const int32_t* sl,
                            const int32_t* Sl, int X0, int s, int S, int H, const uint16_t* W1,
                            const uint16_t* b1, const uint16_t* W2, const uint16_t* b2,
                            const uint16_t* w3, const uint16_t* b3, int P, const int32_t* proc,
                            int max_iters, int window, const int32_t* init, int32_t* act,
                            int32_t* iters, int32_t* record, int64_t* evals_out) {
    Model M;
    int e = setup(&M, T, N, ret, dem, ex, cap, x0r, sl, Sl, X0, s, S, H, W1, b1, W2, b2, w3, b3);
    if (e) return e;
    if ((e = check_procs(N, P, proc))) { teardown(&M); return e; }
    int32_t* alpha = (int32_t*)calloc(T ? T : 1, sizeof(int32_t));
    int32_t* next = (int32_t*)calloc(T ? T : 1, sizeof(int32_t));
    int32_t* x = (int32_t*)malloc(sizeof(int32_t) * N);
    if (init) memcpy(alpha, init, sizeof(int32_t) * T);
    long long evals = 0;
    int k = 0, status = ERR_NOT_CONVERGED, w = 0;
    while (k < max_iters) {
        ++k;
        const int whi = window_end(T, w, window);
        memcpy(next, alpha, sizeof(int32_t) * T);
        for (int m = 0; m < P; ++m) {
            memcpy(x, x0r, sizeof(int32_t) * N);
            long long x0 = X0;
            for (int t = 0; t < T; ++t) {
                const int n = ret[t], d = dem[t];
                const int y = x[n] > d ? x[n] - d : 0;
                int q, r;
                if (proc[n] == m && t < whi) {
                    q = retailer_q(&M, n, y, d, ex[t], &evals);
                    r = x0 - q <= s;
                    next[t] = 2 * q + r;
                } else {
                    q = alpha[t] >> 1;
                    r = alpha[t] & 1;
                }
                const long long recv = q < x0 ? q : x0;
                x[n] = (int32_t)(y + recv);
                x0 = r ? S : (x0 > q ? x0 - q : 0);
            }
        }
        if (record) memcpy(record + (size_t)(k - 1) * T, next, sizeof(int32_t) * T);
        const int fc = first_change(alpha, next, T);
        memcpy(alpha, next, sizeof(int32_t) * T);
        if (fc < 0 && whi >= T) { status = OK; break; }
        w = fc >= 0 ? fc : whi;
    }
    memcpy(act, alpha, sizeof(int32_t) * T);
    *iters = k;
    if (evals_out) *evals_out = evals;
    free(alpha); free(next); free(x);
    teardown(&M);
    return status;
}

/* The same iteration computed the way the GPU path organises it; identical
 * iterates to orc_owmr_picard_literal.  Per pass, from the cache alpha^{k-1}:
 *   Qc[t] = sum_{u<t} q_u,  LR[t] = max{u < t : r_u = 1} (or -1),
 *   D[t]  = sum_{LR[t] < u < t} q_u.
 * A processor's x0 only moves by "reset to S" and "subtract q, floor at 0", so
 * between two of its own steps ta < tb (all other steps cached):
 *   x0(tb) = max(0, S - D[tb])                        if LR[tb] > ta,
 *            max(0, x0(ta + 1) - (Qc[tb] - Qc[ta + 1])) otherwise,
 * with ta = -1, x0(0) = X0 before the first own step.  Each processor then walks
 * only its own steps in time order.  A policy call whose input y (and step) is
 * the same as at the previous evaluation of that step reuses its result (the
 * policy is deterministic); evals_out counts the calls actually made.  With a
 * window, a processor stops its walk at the window's end. */
int orc_owmr_picard_walk(int T, int N, const int32_t* ret, const int32_t* dem, const int32_t* ex,
                         const int32_t* cap, const int32_t* x0r, const int32_t* sl,
                         const int32_t* Sl, int X0, int s, int S, int H, const uint16_t* W1,
                         const uint16_t* b1, const uint16_t* W2, const uint16_t* b2,
                         const uint16_t* w3, const uint16_t* b3, int P, const int32_t* proc,
                         int max_iters, int window, const int32_t* init, int32_t* act,
                         int32_t* iters, int32_t* record, int64_t* evals_out, int32_t* xfin,
                         int64_t* stats) {
    Model M;
    int e = setup(&M, T, N, ret, dem, ex, cap, x0r, sl, Sl, X0, s, S, H, W1, b1, W2, b2, w3, b3);
    if (e) return e;
    if ((e = check_procs(N, P, proc))) { teardown(&M); return e; }
    const size_t Tn = T ? (size_t)T : 1;
    int32_t* alpha = (int32_t*)calloc(Tn, sizeof(int32_t));
    int32_t* next = (int32_t*)calloc(Tn, sizeof(int32_t));
    long long* Qc = (long long*)malloc(sizeof(long long) * (Tn + 1));
    long long* D = (long long*)malloc(sizeof(long long) * (Tn + 1));
    int32_t* LR = (int32_t*)malloc(sizeof(int32_t) * (Tn + 1));
    int32_t* memo_y = (int32_t*)malloc(sizeof(int32_t) * Tn);
    int32_t* memo_q = (int32_t*)malloc(sizeof(int32_t) * Tn);
    int32_t* x = (int32_t*)malloc(sizeof(int32_t) * N);
    /* own steps of each processor, in time order */
    int32_t* off = (int32_t*)calloc((size_t)P + 1, sizeof(int32_t));
    int32_t* own = (int32_t*)malloc(sizeof(int32_t) * Tn);
    for (int t = 0; t < T; ++t) off[proc[ret[t]] + 1]++;
    for (int m = 0; m < P; ++m) off[m + 1] += off[m];
    {
        int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * ((size_t)P + 1));
        memcpy(fill, off, sizeof(int32_t) * ((size_t)P + 1));
        for (int t = 0; t < T; ++t) own[fill[proc[ret[t]]]++] = t;
        free(fill);
    }
    for (int t = 0; t < T; ++t) memo_y[t] = -1;
    if (init) memcpy(alpha, init, sizeof(int32_t) * T);
    long long evals = 0, lost = 0, shipped = 0;
    int k = 0, status = ERR_NOT_CONVERGED, w = 0;
    while (k < max_iters) {
        ++k;
        const int whi = window_end(T, w, window);
        /* prefix quantities of the cache */
        Qc[0] = 0; D[0] = 0; LR[0] = -1;
        for (int t = 0; t < T; ++t) {
            const int q = alpha[t] >> 1, r = alpha[t] & 1;
            Qc[t + 1] = Qc[t] + q;
            if (r) { LR[t + 1] = t; D[t + 1] = 0; }
            else { LR[t + 1] = LR[t]; D[t + 1] = D[t] + q; }
        }
        memcpy(next, alpha, sizeof(int32_t) * T);
        memcpy(x, x0r, sizeof(int32_t) * N);
        lost = shipped = 0;
        for (int m = 0; m < P; ++m) {
            long long x0a = X0;   /* x0 just after the previous own step */
            int ta = -1;
            for (int i = off[m]; i < off[m + 1] && own[i] < whi; ++i) {
                const int t = own[i], n = ret[t], d = dem[t];
                long long x0;
                if (LR[t] > ta) x0 = (long long)S - D[t];
                else x0 = x0a - (Qc[t] - Qc[ta + 1]);
                if (x0 < 0) x0 = 0;
                const int y = x[n] > d ? x[n] - d : 0;
                lost += d > x[n] ? d - x[n] : 0;
                int q;
                if (memo_y[t] == y) q = memo_q[t];
                else {
                    q = retailer_q(&M, n, y, d, ex[t], &evals);
                    memo_y[t] = y;
                    memo_q[t] = q;
                }
                const int r = x0 - q <= s;
                const long long recv = q < x0 ? q : x0;
                shipped += recv;
                x[n] = (int32_t)(y + recv);
                x0a = r ? S : (x0 > q ? x0 - q : 0);
                ta = t;
                next[t] = 2 * q + r;
            }
        }
        if (record) memcpy(record + (size_t)(k - 1) * T, next, sizeof(int32_t) * T);
        const int fc = first_change(alpha, next, T);
        memcpy(alpha, next, sizeof(int32_t) * T);
        if (fc < 0 && whi >= T) { status = OK; break; }
        w = fc >= 0 ? fc : whi;
    }
    memcpy(act, alpha, sizeof(int32_t) * T);
    *iters = k;
    if (evals_out) *evals_out = evals;
    if (xfin) {
        /* x0 after step T from the final cache, retailers from the last walk */
        long long x0 = X0;
        for (int t = 0; t < T; ++t) {
            const int q = alpha[t] >> 1;
            x0 = (alpha[t] & 1) ? S : (x0 > q ? x0 - q : 0);
        }
        xfin[0] = (int32_t)x0;
        memcpy(xfin + 1, x, sizeof(int32_t) * N);
    }
    if (stats) {
        long long R = 0;
        for (int t = 0; t < T; ++t) R += alpha[t] & 1;
        stats[0] = R; stats[1] = lost; stats[2] = shipped; stats[3] = evals;
    }
    free(alpha); free(next); free(Qc); free(D); free(LR); free(memo_y); free(memo_q);
    free(x); free(off); free(own);
    teardown(&M);
    return status;
}
