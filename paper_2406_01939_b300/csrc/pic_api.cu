// C ABI entry points (include/pic.h): instance management and the simulate call.
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>

#include "pic_device.cuh"

using namespace pic;

namespace {

thread_local char g_err[512] = "";

pic_status fail(pic_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA,   \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                      \
    } while (0)

// Validation of the value ranges the kernels rely on (one pass over the inputs).
__global__ void k_validate(int T, int N, int K, int R, const int32_t* __restrict__ prod,
                           const int32_t* __restrict__ reg, const int32_t* __restrict__ x0,
                           const int32_t* __restrict__ cost, const int32_t* __restrict__ lam,
                           int* bad) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    int b = 0;
    for (long long t = gid; t < T; t += stride) {
        if ((unsigned)prod[t] >= (unsigned)K) b |= 1;
        if ((unsigned)reg[t] >= (unsigned)R) b |= 2;
    }
    for (long long i = gid; i < (long long)K * N; i += stride)
        if (x0[i] < 0) b |= 4;
    const int lim = 1 << 23;
    for (long long i = gid; i < (long long)R * N; i += stride) {
        const int c = cost[i];
        if (c <= -lim || c >= lim) b |= 8;
        if (c < -32768 || c > 32767) b |= 128;  // not representable in int16
    }
    if (lam)
        for (long long i = gid; i < (long long)K * N; i += stride) {
            const int l = lam[i];
            if (l <= -lim || l >= lim) b |= 16;
        }
    if (b) atomicOr(bad, b);
}

// Exact check of |cost[r][n] - lam[k][n]| < 2^23 via per-warehouse extremes.
__global__ void k_validate_cap(int N, const int32_t* __restrict__ cap, int* bad) {
    for (int n = threadIdx.x; n < N; n += blockDim.x)
        if (cap[n] < 0) atomicOr(bad, 256);
}

__global__ void k_validate_dual(int N, int K, int R, const int32_t* __restrict__ cost,
                                const int32_t* __restrict__ lam, int* bad) {
    const int n = blockIdx.x;
    long long cmin = LLONG_MAX, cmax = LLONG_MIN, lmin = LLONG_MAX, lmax = LLONG_MIN;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        cmin = min(cmin, (long long)cost[(size_t)r * N + n]);
        cmax = max(cmax, (long long)cost[(size_t)r * N + n]);
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        lmin = min(lmin, (long long)lam[(size_t)k * N + n]);
        lmax = max(lmax, (long long)lam[(size_t)k * N + n]);
    }
    __shared__ long long red[4][32];
    for (int o = 16; o > 0; o >>= 1) {
        cmin = min(cmin, __shfl_xor_sync(kFull, cmin, o));
        cmax = max(cmax, __shfl_xor_sync(kFull, cmax, o));
        lmin = min(lmin, __shfl_xor_sync(kFull, lmin, o));
        lmax = max(lmax, __shfl_xor_sync(kFull, lmax, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = cmin; red[1][w] = cmax; red[2][w] = lmin; red[3][w] = lmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            cmin = min(cmin, red[0][i]); cmax = max(cmax, red[1][i]);
            lmin = min(lmin, red[2][i]); lmax = max(lmax, red[3][i]);
        }
        const long long lim = 1 << 23;
        if (cmax - lmin >= lim || cmin - lmax <= -lim) atomicOr(bad, 32);
    }
}

__global__ void k_gather_alpha(const int8_t* __restrict__ alpha_t, const int32_t* __restrict__ perm,
                               int T, int N, int8_t* __restrict__ alpha_s, int* bad) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= T) return;
    int a = alpha_t[perm[j]];
    if (a < -1 || a >= N) { atomicOr(bad, 64); a = -1; }
    alpha_s[j] = (int8_t)a;
}

// Histogram of the cache per segment (used when the cache starts from alpha_init).
__global__ void k_seg_hist(const int8_t* __restrict__ alpha_s, const int32_t* __restrict__ run_start,
                           const int32_t* __restrict__ seg_run, const Ctrl* ctrl, int NP,
                           int32_t* __restrict__ agg) {
    extern __shared__ int sh[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* h = sh + w * NP;
    const int nseg = ctrl->nseg;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = gw; s < nseg; s += nw) {
        for (int i = lane; i < NP; i += 32) h[i] = 0;
        __syncwarp();
        const int j0 = run_start[seg_run[s]], j1 = run_start[seg_run[s + 1]];
        for (int j = j0 + lane; j < j1; j += 32) {
            const int a = alpha_s[j];
            if (a >= 0) atomicAdd(&h[a], 1);
        }
        __syncwarp();
        for (int i = lane; i < NP; i += 32) agg[(size_t)s * NP + i] = h[i];
        __syncwarp();
    }
}

__global__ void k_set_tag(Ctrl* c, unsigned v) { c->tag_next = v; }

__global__ void k_take_tags(Ctrl* c, unsigned n) {
    c->tag_base = c->tag_next;
    c->tag_next += n;
}

bool valid_desc(const pic_instance_desc* d) {
    return d && d->T >= 0 && d->N >= 1 && d->N <= 127 && d->K >= 1 && d->K <= 65535 && d->R >= 1 &&
           d->R <= 65535 && (d->T == 0 || (d->prod && d->reg)) && d->x0 && d->cost &&
           (d->mem == PIC_MEM_HOST || d->mem == PIC_MEM_DEVICE);
}

template <typename T>
cudaError_t dmalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
}

pic_status copy_inputs(Instance& I, const pic_instance_desc* d, cudaStream_t st) {
    const cudaMemcpyKind kind = d->mem == PIC_MEM_HOST ? cudaMemcpyHostToDevice
                                                       : cudaMemcpyDeviceToDevice;
    if (I.T) {
        CU(cudaMemcpyAsync(I.prod, d->prod, sizeof(int32_t) * I.T, kind, st));
        CU(cudaMemcpyAsync(I.reg, d->reg, sizeof(int32_t) * I.T, kind, st));
    }
    CU(cudaMemcpyAsync(I.x0, d->x0, sizeof(int32_t) * I.K * I.N, kind, st));
    CU(cudaMemcpyAsync(I.cost, d->cost, sizeof(int32_t) * I.R * I.N, kind, st));
    if (I.has_lam) CU(cudaMemcpyAsync(I.lam, d->lam, sizeof(int32_t) * I.K * I.N, kind, st));
    if (I.has_cap) CU(cudaMemcpyAsync(I.cap, d->cap, sizeof(int32_t) * I.N, kind, st));
    CU(launch_validate(I, st));
    int* bad = &I.ctrl->pad0;
    int hb = 0;
    CU(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (hb & 1) return fail(PIC_ERR_INVALID_ARG, "prod[t] outside [0, K)");
    if (hb & 2) return fail(PIC_ERR_INVALID_ARG, "reg[t] outside [0, R)");
    if (hb & 4) return fail(PIC_ERR_INVALID_ARG, "x0 has a negative entry");
    if (hb & (8 | 16 | 32))
        return fail(PIC_ERR_INVALID_ARG, "|cost|, |lam| or |cost - lam| not below 2^23");
    if (hb & 256) return fail(PIC_ERR_INVALID_ARG, "cap has a negative entry");
    I.cost16 = (hb & 128) ? 0 : 1;
    return PIC_OK;
}

}  // namespace

namespace pic {
// Record the message pic_last_error() returns on this thread (for entry points
// defined in other translation units).
pic_status record_error(pic_status s, const char* msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg);
    return s;
}
void clear_error() { g_err[0] = 0; }

bool desc_ok(const pic_instance_desc* d) { return valid_desc(d); }

cudaError_t launch_validate(Instance& I, cudaStream_t st) {
    int* bad = &I.ctrl->pad0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (e) return e;
    k_validate<<<2 * I.num_sms, 256, 0, st>>>(I.T, I.N, I.K, I.R, I.prod, I.reg, I.x0, I.cost,
                                              I.has_lam ? I.lam : nullptr, bad);
    if (I.has_lam) k_validate_dual<<<I.N, 256, 0, st>>>(I.N, I.K, I.R, I.cost, I.lam, bad);
    if (I.has_cap) k_validate_cap<<<1, 128, 0, st>>>(I.N, I.cap, bad);
    return cudaGetLastError();
}

void free_instance(Instance& I) {
    free_pg(I);
    void* ptrs[] = {I.prod, I.reg, I.x0, I.cost, I.lam, I.perm, I.prod_s, I.reg_s, I.pcount,
                    I.pstart, I.run_start, I.run_of, I.run_chunk, I.seg_run, I.seg_of_run, I.seg_prod, I.seg_cf,
                    I.seg_ce, I.seg_meta, I.seg_lpt, I.len_hist, I.alpha_s, I.agg, I.carry, I.sbexc, I.sbagg,
                    I.sbincl, I.fc, I.xfin, I.xwork, I.act_t, I.tmp_a, I.tmp_b, I.tmp_c, I.scan_blk,
                    I.hist, I.ctrl, I.trace, I.mlp_P, I.mlp_W1p, I.mlp_W2p, I.mlp_b2, I.mlp_Emax, I.mlp_bnd, I.mlp_c2, I.mlp_sat,
                    I.cap, I.cap_run_t, I.cap_info, I.cap_inv, I.cap_qagg, I.cap_qinc};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < 4; ++i)
        if (I.ev[i]) cudaEventDestroy(I.ev[i]);
    if (Batch* b = I.batch) {
        void* dp[] = {b->toff, b->koff, b->roff, b->traj_of_prod, b->reg_local, b->chunk_len,
                      b->pol, b->last_chg, b->tres};
        for (void* p : dp)
            if (p) cudaFree(p);
        if (b->h_pol) cudaFreeHost(b->h_pol);
        if (b->h_out) cudaFreeHost(b->h_out);
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        delete[] b->h_toff;
        delete[] b->h_koff;
        delete[] b->h_roff;
        delete[] b->h_has_lam;
        delete b;
        I.batch = nullptr;
    }
}

cudaError_t alloc_instance(Instance& I, int T_, int N_, int K_, int R_, bool has_lam) {
    I.T = T_; I.N = N_; I.K = K_; I.R = R_;
    I.NP = ((N_ + 31) / 32) * 32;
    I.has_lam = has_lam;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&I.num_sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t T = (size_t)I.T, K = I.K, N = I.N;
    // segments <= runs <= T for any window; per-segment histograms are sized per window later
    I.smax = (int64_t)T + (int64_t)K + 2;
    const size_t nblk_radix = (T + 4095) / 4096 + 1;
    const size_t nscan = (T > 256 * nblk_radix ? T : 256 * nblk_radix) + K + 2;
    I.hist_cap = 256 * nblk_radix;
    const size_t S = (size_t)I.smax;
    if (!e) e = dmalloc(&I.prod, T);
    if (!e) e = dmalloc(&I.reg, T);
    if (!e) e = dmalloc(&I.x0, K * N);
    if (!e) e = dmalloc(&I.cost, (size_t)I.R * N);
    if (!e && I.has_lam) e = dmalloc(&I.lam, K * N);
    if (!e) e = dmalloc(&I.perm, T);
    if (!e) e = dmalloc(&I.prod_s, T);
    if (!e) e = dmalloc(&I.reg_s, T);
    if (!e) e = dmalloc(&I.pcount, K + 1);
    if (!e) e = dmalloc(&I.pstart, K + 1);
    if (!e) e = dmalloc(&I.run_start, T + 2);
    if (!e) e = dmalloc(&I.run_of, T + 1);
    if (!e) e = dmalloc(&I.run_chunk, T + 1);
    if (!e) e = dmalloc(&I.seg_run, S + 1);
    if (!e) e = dmalloc(&I.seg_of_run, T + 1);
    if (!e) e = dmalloc(&I.seg_prod, S);
    if (!e) e = dmalloc(&I.seg_cf, S);
    if (!e) e = dmalloc(&I.seg_ce, S);
    if (!e) e = dmalloc(&I.seg_meta, S);
    if (!e) e = dmalloc(&I.seg_lpt, S);
    if (!e) e = dmalloc(&I.len_hist, kLenBuckets);
    if (!e) e = dmalloc(&I.alpha_s, T);
    if (!e) e = dmalloc(&I.fc, 2 * K);
    if (!e) e = dmalloc(&I.xfin, K * N);
    if (!e) e = dmalloc(&I.xwork, K * N);
    if (!e) e = dmalloc(&I.act_t, T);
    if (!e) e = dmalloc(&I.tmp_a, T);
    if (!e) e = dmalloc(&I.tmp_b, T);
    if (!e) e = dmalloc(&I.scan_blk, (size_t)scan_blk_len((int)nscan));
    if (!e) e = cudaMemset(I.scan_blk, 0, sizeof(int32_t) * (size_t)scan_blk_len((int)nscan));
    if (!e) e = dmalloc(&I.hist, (size_t)I.hist_cap);
    if (!e) e = cudaMalloc((void**)&I.ctrl, sizeof(Ctrl));
    if (!e) e = cudaMalloc((void**)&I.trace, sizeof(long long) * kTraceCols * kTraceCap);
    for (int i = 0; i < 4 && !e; ++i) e = cudaEventCreate(&I.ev[i]);
    return e;
}

cudaError_t prepare_picard_state(Instance& I, int W, int iters_cap, cudaStream_t st) {
    const int64_t smax = (int64_t)2 * I.K + (int64_t)((int64_t)I.T + W - 1) / W + 2;
    cudaError_t e;
    if (!I.agg || smax > I.smax_agg) {
        if (I.agg) {
            cudaFree(I.agg); cudaFree(I.carry); cudaFree(I.sbexc); cudaFree(I.sbagg); cudaFree(I.sbincl);
        }
        I.agg = I.carry = I.sbexc = nullptr;
        I.sbagg = I.sbincl = nullptr;
        I.smax_agg = 0;
        if ((e = dmalloc(&I.agg, (size_t)smax * I.NP))) return e;
        if ((e = dmalloc(&I.carry, (size_t)smax * I.NP))) return e;
        if ((e = dmalloc(&I.sbexc, (size_t)smax * I.NP))) return e;
        if ((e = dmalloc(&I.sbagg, (size_t)smax * I.NP))) return e;
        if ((e = dmalloc(&I.sbincl, (size_t)smax * I.NP))) return e;
        I.smax_agg = smax;
        I.tag_next = 0;  // forces the clear below
    }
    // Look-back words carry tags that are never reused on this instance, so the
    // words of earlier calls need no clearing; they are cleared only for fresh
    // memory and when the 32-bit tag space runs out.  agg and carry need no
    // clearing either: pass 1 replays every segment (writing agg) and reads no
    // carry unless the cache starts from alpha_init, whose histograms and
    // prefixes are computed before use.
    if (I.tag_next == 0 || (unsigned long long)I.tag_next + iters_cap + 1 >= 0x7FFFFFFFull) {
        const size_t bytes = sizeof(unsigned long long) * (size_t)I.smax_agg * I.NP;
        if ((e = cudaMemsetAsync(I.sbagg, 0, bytes, st))) return e;
        if ((e = cudaMemsetAsync(I.sbincl, 0, bytes, st))) return e;
        k_set_tag<<<1, 1, 0, st>>>(I.ctrl, 1u);
        I.launches += 1;
        if ((e = cudaGetLastError())) return e;
        I.tag_next = 1;
    }
    // the host mirror runs ahead by one call; take_tags advances the device copy
    I.tag_next += (unsigned)iters_cap + 1;
    return cudaSuccess;
}

cudaError_t take_tags(Instance& I, int iters_cap, cudaStream_t st) {
    k_take_tags<<<1, 1, 0, st>>>(I.ctrl, (unsigned)iters_cap + 1);
    I.launches += 1;
    return cudaGetLastError();
}

cudaError_t init_cache(Instance& I, const int8_t* alpha_init, cudaStream_t st) {
    const size_t T = I.T, K = I.K, N = I.N;
    cudaError_t e;
    if ((e = cudaMemsetAsync(I.fc, 0xFF, sizeof(int32_t) * K, st))) return e;  // pass 0: all "changed"
    if ((e = cudaMemcpyAsync(I.xfin, I.x0, sizeof(int32_t) * K * N, cudaMemcpyDeviceToDevice, st)))
        return e;
    if (!T) return cudaSuccess;
    if (alpha_init) {
        int* bad = &I.ctrl->pad0;
        k_gather_alpha<<<(int)((T + 255) / 256), 256, 0, st>>>(alpha_init, I.perm, (int)T, (int)N,
                                                             I.alpha_s, bad);
        k_seg_hist<<<2 * I.num_sms, 256, 8 * I.NP * sizeof(int), st>>>(I.alpha_s, I.run_start,
                                                                       I.seg_run, I.ctrl, I.NP, I.agg);
        I.launches += 2;
        return cudaGetLastError();
    }
    return cudaMemsetAsync(I.alpha_s, 0xFF, T, st);  // a^phi everywhere (Alg. 1 line 1)
}
}  // namespace pic

extern "C" {

const char* pic_last_error(void) { return g_err; }

pic_status pic_create_instance(const pic_instance_desc* d, pic_instance** out) {
    g_err[0] = 0;
    if (!out) return fail(PIC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_desc(d)) return fail(PIC_ERR_INVALID_ARG, "invalid instance descriptor (sizes, pointers or mem)");
    pic_instance* h = new (std::nothrow) pic_instance();
    if (!h) return fail(PIC_ERR_OOM, "host allocation failed");
    Instance& I = h->I;
    memset(&I, 0, sizeof(I));
    cudaError_t e = alloc_instance(I, d->T, d->N, d->K, d->R, d->lam != nullptr);
    I.has_cap = d->cap != nullptr;
    if (!e && I.has_cap) e = dmalloc(&I.cap, (size_t)d->N);
    // per-segment histograms: allocated lazily at the first simulate (size depends on W)
    if (e) {
        free_instance(I);
        delete h;
        return fail(e == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA,
                    "allocation failed: %s", cudaGetErrorString(e));
    }
    cudaStream_t st = (cudaStream_t)d->stream;
    if (cudaMemsetAsync(I.ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) {
        free_instance(I);
        delete h;
        return fail(PIC_ERR_CUDA, "memset failed");
    }
    pic_status s = copy_inputs(I, d, st);
    if (s != PIC_OK) {
        free_instance(I);
        delete h;
        return s;
    }
    *out = h;
    return PIC_OK;
}

pic_status pic_instance_load(pic_instance* h, const pic_instance_desc* d) {
    g_err[0] = 0;
    if (!h) return fail(PIC_ERR_INVALID_ARG, "instance is NULL");
    if (!valid_desc(d)) return fail(PIC_ERR_INVALID_ARG, "invalid instance descriptor");
    Instance& I = h->I;
    if (I.batch) return fail(PIC_ERR_INVALID_ARG, "batch instance: inputs are fixed at pic_create_batch");
    if (d->T != I.T || d->N != I.N || d->K != I.K || d->R != I.R || (d->lam != nullptr) != (I.has_lam != 0) ||
        (d->cap != nullptr) != (I.has_cap != 0))
        return fail(PIC_ERR_INVALID_ARG, "shape differs from the instance's");
    I.tables_m = 0;  // the order tables describe the old stream
    I.cap_tables_m = 0;
    return copy_inputs(I, d, (cudaStream_t)d->stream);
}

void pic_destroy_instance(pic_instance* h) {
    if (!h) return;
    free_instance(h->I);
    delete h;
}

pic_status pic_simulate(pic_instance* h, const pic_policy* pol, const pic_sim_opts* opts,
                        int8_t* actions_out, int32_t* final_stock, pic_sim_result* res) {
    g_err[0] = 0;
    if (!h || !pol || !opts || (!actions_out && h->I.T > 0))
        return fail(PIC_ERR_INVALID_ARG, "instance, policy, opts and actions_out are required");
    Instance& I = h->I;
    if (I.batch) return fail(PIC_ERR_INVALID_ARG, "batch instance: use pic_simulate_batch");
    if (opts->mode != PIC_MODE_PICARD && opts->mode != PIC_MODE_SEQUENTIAL &&
        opts->mode != PIC_MODE_PICARD_PRODUCTS && opts->mode != PIC_MODE_PICARD_ASSIGNED)
        return fail(PIC_ERR_INVALID_ARG, "unknown mode %d", opts->mode);
    if (opts->out_mem != PIC_MEM_HOST && opts->out_mem != PIC_MEM_DEVICE)
        return fail(PIC_ERR_INVALID_ARG, "unknown out_mem %d", opts->out_mem);
    if (pol->kind < PIC_POLICY_GREEDY || pol->kind > PIC_POLICY_GUMBEL)
        return fail(PIC_ERR_INVALID_ARG, "unknown policy kind %d", pol->kind);
    if (pol->kind == PIC_POLICY_DUAL && !I.has_lam)
        return fail(PIC_ERR_INVALID_ARG, "bid-price policy needs an instance created with lam");
    const bool mlp = pol->kind == PIC_POLICY_MLP || pol->kind == PIC_POLICY_GUMBEL;
    if (mlp && pol->hidden != kHidden)
        return fail(PIC_ERR_UNSUPPORTED, "MLP hidden width must be %d", kHidden);
    if (mlp && (!pol->W1 || !pol->b1 || !pol->W2 || !pol->b2 || !pol->E))
        return fail(PIC_ERR_INVALID_ARG, "MLP policy needs W1, b1, W2, b2 and E (device pointers)");
    if (mlp && I.has_cap)
        return fail(PIC_ERR_UNSUPPORTED, "node capacity: greedy and bid-price policies only");
    if (opts->num_chunks < 0 || opts->max_iters < 0 || opts->seg_window < 0 || opts->max_steps < 0)
        return fail(PIC_ERR_INVALID_ARG, "negative num_chunks, max_iters, seg_window or max_steps");
    if (opts->max_steps > 0 && I.has_cap)
        return fail(PIC_ERR_UNSUPPORTED, "the max_steps window is not supported with node capacity");
    if (opts->mode == PIC_MODE_PICARD_PRODUCTS && (mlp || opts->max_steps > 0))
        return fail(PIC_ERR_UNSUPPORTED, "product partition: greedy and bid-price policies, no window");
    if (opts->mode == PIC_MODE_PICARD_ASSIGNED) {
        if (mlp || opts->max_steps > 0)
            return fail(PIC_ERR_UNSUPPORTED,
                        "assigned partition: greedy and bid-price policies, no window");
        if (opts->num_chunks < 1 || (long long)opts->num_chunks * I.K >= (1LL << 31))
            return fail(PIC_ERR_INVALID_ARG, "assigned partition: need 1 <= num_chunks and num_chunks * K < 2^31");
        if (I.T && !opts->proc) return fail(PIC_ERR_INVALID_ARG, "assigned partition: proc is NULL");
    }
    cudaStream_t st = (cudaStream_t)opts->stream;
    const size_t T = I.T, K = I.K, N = I.N;
    const bool host_out = opts->out_mem == PIC_MEM_HOST;
    const cudaMemcpyKind okind = host_out ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const bool timing = (opts->flags & PIC_FLAG_TIMING) != 0;
    I.launches = 0;
    I.ran_wave = 0;
    if (mlp) CU(mlp_alloc(&I));
    if (timing) CU(cudaEventRecord(I.ev[0], st));
    CU(cudaMemsetAsync(I.ctrl, 0, offsetof(Ctrl, nruns), st));
    if (mlp) CU(mlp_prepare(&I, pol, st));
    int M = 1, iters_cap = 1;
    if (opts->mode == PIC_MODE_SEQUENTIAL) {
        CU(cudaMemcpyAsync(I.xwork, I.x0, sizeof(int32_t) * K * N, cudaMemcpyDeviceToDevice, st));
        if (timing) CU(cudaEventRecord(I.ev[1], st));
        if (T && I.has_cap) {
            CU(sequential_cap(&I, pol->kind, st));
        } else if (T && mlp) {
            CU(sequential_mlp(&I, pol, opts->flags, st));
            CU(reduce_costs(&I, I.act_t, I.reg, st));
        } else if (T) {
            CU(sequential_int(&I, pol->kind, st));
        }
        if (timing) CU(cudaEventRecord(I.ev[2], st));
        if (T) CU(cudaMemcpyAsync(actions_out, I.act_t, T, okind, st));
        if (final_stock)
            CU(cudaMemcpyAsync(final_stock, I.xwork, sizeof(int32_t) * K * N, okind, st));
    } else if (opts->mode == PIC_MODE_PICARD_PRODUCTS || opts->mode == PIC_MODE_PICARD_ASSIGNED) {
        // products: processor of product k is k mod M, and M > K gives the same
        // assignment as M = K; assigned: M processes named by opts->proc
        if (opts->mode == PIC_MODE_PICARD_ASSIGNED)
            M = opts->num_chunks;
        else
            M = opts->num_chunks && opts->num_chunks < (int)K ? opts->num_chunks : (int)K;
        iters_cap = opts->max_iters ? opts->max_iters : (T < (size_t)INT_MAX ? (int)T + 1 : INT_MAX);
        if (T) {
            if (opts->alpha_init) {
                CU(cudaMemcpyAsync(I.act_t, opts->alpha_init, T, cudaMemcpyDeviceToDevice, st));
                CU(check_alpha_init(&I, I.act_t, st));
                // an invalid cache is rejected before any pass runs on it
                int bad = 0;
                CU(cudaMemcpyAsync(&bad, &I.ctrl->pad0, sizeof(int), cudaMemcpyDeviceToHost, st));
                CU(cudaStreamSynchronize(st));
                if (bad & 64) return fail(PIC_ERR_INVALID_ARG, "alpha_init holds a value outside [-1, N)");
            } else {
                CU(cudaMemsetAsync(I.act_t, 0xFF, T, st));  // a^phi everywhere (Alg. 1)
            }
        }
        if (timing) CU(cudaEventRecord(I.ev[1], st));
        if (opts->mode == PIC_MODE_PICARD_PRODUCTS)
            CU(picard_products(&I, pol, M, iters_cap, st));
        else
            CU(I.has_cap ? picard_assigned_cap(&I, pol, opts->proc, M, iters_cap, st)
                         : picard_assigned(&I, pol, opts->proc, M, iters_cap, st));
        if (timing) CU(cudaEventRecord(I.ev[2], st));
        if (T) {
            CU(reduce_costs(&I, I.act_t, I.reg, st));
            CU(cudaMemcpyAsync(actions_out, I.act_t, T, okind, st));
        }
        if (final_stock)
            CU(cudaMemcpyAsync(final_stock, I.xfin, sizeof(int32_t) * K * N, okind, st));
    } else if (I.has_cap) {
        // time chunks of at most kCapChunk orders, one run per segment
        M = opts->num_chunks ? opts->num_chunks : (int)((T + kCapChunk - 1) / kCapChunk);
        if (M < 1) M = 1;
        if (T && M > (int)T) M = (int)T;
        if (T && (T + M - 1) / M > (size_t)kCapChunk)
            return fail(PIC_ERR_INVALID_ARG,
                        "node capacity: chunk length ceil(T/M) = %zu exceeds %d (raise num_chunks)",
                        (T + M - 1) / M, kCapChunk);
        iters_cap = opts->max_iters ? opts->max_iters : M + 1;
        CU(prepare_picard_state(I, 1, iters_cap, st));
        const bool reuse = (opts->flags & PIC_FLAG_REUSE_TABLES) && I.tables_m == M && I.tables_w == 1;
        if (!reuse) {
            CU(build_tables(&I, M, 1, st));
            I.tables_m = M;
            I.tables_w = 1;
            I.cap_tables_m = 0;
        }
        CU(take_tags(I, iters_cap, st));
        CU(init_cache(I, opts->alpha_init, st));
        if (T) {
            if (timing) CU(cudaEventRecord(I.ev[1], st));
            const bool trace = opts->trace && opts->trace_cap > 0;
            if (trace) CU(cudaMemsetAsync(I.trace, 0, sizeof(long long) * kTraceCols * kTraceCap, st));
            CU(picard_cap(&I, pol, M, iters_cap, opts->flags, opts->alpha_init,
                          opts->timeout_ns ? opts->timeout_ns : 10000000000ull, trace, st));
            if (timing) CU(cudaEventRecord(I.ev[2], st));
            CU(reduce_costs(&I, I.act_t, I.reg, st));
            CU(cudaMemcpyAsync(actions_out, I.act_t, T, okind, st));
        }
        if (final_stock)
            CU(cudaMemcpyAsync(final_stock, I.xfin, sizeof(int32_t) * K * N, okind, st));
    } else {
        M = opts->num_chunks ? opts->num_chunks : (int)((T + 255) / 256);
        if (M < 1) M = 1;
        if (T && M > (int)T) M = (int)T;
        // default window: long work units amortise the cheap integer policy; the MLP
        // policy's per-order cost makes short units (short critical paths) better
        // the wave kernel takes one run per work unit
        const bool wave = mlp && (opts->flags & PIC_FLAG_WAVE) && wave_applies(&I);
        const int W = wave ? 1 : opts->seg_window ? opts->seg_window : (mlp ? kSegWindowMlp : kSegWindow);
        // the window needs at most two passes per block (one change, one confirmation)
        iters_cap = opts->max_iters ? opts->max_iters : (opts->max_steps > 0 ? 2 * M + 2 : M + 1);
        CU(prepare_picard_state(I, W, iters_cap, st));
        const bool reuse = (opts->flags & PIC_FLAG_REUSE_TABLES) && I.tables_m == M && I.tables_w == W;
        if (!reuse) {
            CU(build_tables(&I, M, W, st));
            I.tables_m = M;
            I.tables_w = W;
        }
        CU(take_tags(I, iters_cap, st));
        CU(init_cache(I, opts->alpha_init, st));
        if (T && opts->max_steps > 0 && !opts->alpha_init) {
            // segments outside the first windows are not replayed in pass 1: their
            // histograms and chain prefixes must start as those of the all-a^phi cache
            const size_t bytes = sizeof(int32_t) * (size_t)I.smax_agg * I.NP;
            CU(cudaMemsetAsync(I.agg, 0, bytes, st));
            CU(cudaMemsetAsync(I.carry, 0, bytes, st));
            CU(cudaMemsetAsync(I.sbexc, 0, bytes, st));
        }
        if (T) {
            if (timing) CU(cudaEventRecord(I.ev[1], st));
            const bool trace = opts->trace && opts->trace_cap > 0;
            if (trace) CU(cudaMemsetAsync(I.trace, 0, sizeof(long long) * kTraceCols * kTraceCap, st));
            CU(picard_run(&I, pol, iters_cap, opts->flags, opts->alpha_init,
                          opts->timeout_ns ? opts->timeout_ns : 10000000000ull, trace,
                          opts->max_steps, st));
            if (timing) CU(cudaEventRecord(I.ev[2], st));
            CU(finish_outputs(&I, st));
            CU(cudaMemcpyAsync(actions_out, I.act_t, T, okind, st));
        }
        if (final_stock)
            CU(cudaMemcpyAsync(final_stock, I.xfin, sizeof(int32_t) * K * N, okind, st));
    }
    if (timing) {
        if (!T) {
            CU(cudaEventRecord(I.ev[1], st));
            CU(cudaEventRecord(I.ev[2], st));
        }
        CU(cudaEventRecord(I.ev[3], st));
    }
    Ctrl hc;
    CU(cudaMemcpyAsync(&hc, I.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (hc.pad0 & 64) return fail(PIC_ERR_INVALID_ARG, "alpha_init holds a value outside [-1, N)");
    if (hc.pad0 & 128) return fail(PIC_ERR_INVALID_ARG, "proc holds a process outside [0, num_chunks)");
    if (hc.err) return fail((pic_status)hc.err, "device wait exceeded timeout (%llu ns)",
                            (unsigned long long)opts->timeout_ns);
    if (T && opts->mode == PIC_MODE_PICARD && opts->trace && opts->trace_cap > 0) {
        int rows = hc.iters < opts->trace_cap ? hc.iters : opts->trace_cap;
        if (rows > kTraceCap) rows = kTraceCap;
        if (rows > 0)
            CU(cudaMemcpy(opts->trace, I.trace, sizeof(long long) * kTraceCols * rows, cudaMemcpyDeviceToHost));
    }
    if (res) {
        res->total_cost = hc.total_cost;
        res->lost = hc.lost;
        res->policy_calls = (int64_t)hc.policy_calls;
        res->iters = T ? hc.iters : 1;  // (set for every Picard mode)
        res->num_chunks = M;
        res->mlp_calls = mlp ? res->policy_calls : 0;
        res->seg_window = opts->mode == PIC_MODE_PICARD ? I.tables_w : 0;
        res->cta_threads = opts->mode == PIC_MODE_PICARD ? I.cta_threads : 32;
        res->ctas_per_sm = opts->mode == PIC_MODE_PICARD ? I.ctas_per_sm : 1;
        res->rescored = (int64_t)hc.rescored;
        res->tc_decisions = (int64_t)hc.tc_rows;
        res->sat_decisions = (int64_t)hc.sat_rows;
        res->near_ties = (int64_t)hc.near_ties;
        res->wave = I.ran_wave;
        res->seg_replays = (int64_t)hc.seg_replays;
        res->launches = I.launches;
        res->prep_ms = res->sim_ms = res->total_ms = 0.0f;
        if (timing) {
            CU(cudaEventElapsedTime(&res->prep_ms, I.ev[0], I.ev[1]));
            CU(cudaEventElapsedTime(&res->sim_ms, I.ev[1], I.ev[2]));
            CU(cudaEventElapsedTime(&res->total_ms, I.ev[0], I.ev[3]));
        }
    }
    if (T && opts->mode != PIC_MODE_SEQUENTIAL && !hc.converged)
        return fail(PIC_ERR_NOT_CONVERGED, "no fixed point within %d passes", iters_cap);
    return PIC_OK;
}

}  // extern "C"
