// pic_simulate_sequential_static: the sequential simulator with its scratch in
// a fixed, library-owned device array, for callers that must not allocate
// device memory.
//
// Who needs it: a host process that hands all device memory to its own
// allocator at start-up and forbids driver allocations afterwards, and code on
// a latency-critical path where the implicit device-wide synchronisation of
// cudaMalloc / cudaFree is not acceptable.  pic_create_instance allocates; this
// entry point does not: it reads the caller's device arrays directly and keeps
// its working stock and its control block in g_static_scratch.
//
// The scratch array is a file-scope __device__ variable, so every GPU that
// loads the library holds kStaticScratchBytes of it until the process exits.
// In host code the name g_static_scratch is only a host-side stand-in, not a
// device address: on the first call on each device (with that device current)
// cudaGetSymbolAddress translates it once, and the translated pointer is what
// the kernels receive.  That first call should therefore come before any stream
// capture on the device.  Every call synchronizes its stream before it returns.
// Every call shares the one array and leaves the last call's contents in it;
// the parts that must start at zero are cleared at the start of each call.  Two
// calls whose work overlaps on the same GPU (different streams or threads) race
// on the array.
//
// The kernels read and write the caller's arrays directly, so every pointer is
// checked on the host before the first launch: it must be device memory of the
// current device (or managed memory), and the bytes the call touches must lie
// inside the allocation that holds it (cuMemGetAddressRange, reached through
// the runtime's driver entry point).  A host pointer, another device's pointer
// or a short array is INVALID_ARG, never a fault.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pic_device.cuh"

namespace {

using namespace pic;

// Layout: [Ctrl, padded to 256 B][working stock, int32 x K x N]
constexpr size_t kStaticScratchBytes = 4u << 20;  // 4 MiB
constexpr size_t kCtrlBytes = 256;
constexpr size_t kMaxStockEntries = (kStaticScratchBytes - kCtrlBytes) / sizeof(int32_t);
static_assert(sizeof(Ctrl) <= kCtrlBytes, "control block exceeds its slot");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices];  // device address of g_static_scratch per device (set on first use)

// Range checks the simulator relies on; bit 128 = a cost does not fit int16.
__global__ void k_static_validate(int T, int N, int K, int R, const int32_t* __restrict__ prod,
                                  const int32_t* __restrict__ reg, const int32_t* __restrict__ x0,
                                  const int32_t* __restrict__ cost, const int32_t* __restrict__ lam,
                                  int* bad) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lim = 1 << 22;  // |cost|, |lam| < 2^22 keeps |cost - lam| < 2^23
    int b = 0;
    for (long long t = gid; t < T; t += stride) {
        if ((unsigned)prod[t] >= (unsigned)K) b |= 1;
        if ((unsigned)reg[t] >= (unsigned)R) b |= 2;
    }
    for (long long i = gid; i < (long long)K * N; i += stride) {
        if (x0[i] < 0) b |= 4;
        if (lam && (lam[i] <= -lim || lam[i] >= lim)) b |= 8;
    }
    for (long long i = gid; i < (long long)R * N; i += stride) {
        const int c = cost[i];
        if (c <= -lim || c >= lim) b |= 8;
        if (c < -32768 || c > 32767) b |= 128;
    }
    if (b) atomicOr(bad, b);
}

pic_status cuda_fail(cudaError_t e, const char* what) {
    char msg[256];
    snprintf(msg, sizeof(msg), "%s failed: %s", what, cudaGetErrorString(e));
    return record_error(PIC_ERR_CUDA, msg);
}

// cuMemGetAddressRange (driver API): base and size of the allocation holding a
// device address.  Resolved once; null when the driver does not provide it.
typedef int (*AddressRangeFn)(unsigned long long* base, size_t* size, unsigned long long ptr);

AddressRangeFn address_range_fn() {
    static std::once_flag once;
    static AddressRangeFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<AddressRangeFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// Whether `bytes` bytes at p are device (or managed) memory that device `dev`
// may access: the pointer's memory type and device, then the extent of its
// allocation.  bytes == 0 accepts any pointer (nothing is touched).
bool device_range_ok(const void* p, size_t bytes, int dev) {
    if (bytes == 0) return true;
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice) {
        if (at.device != dev) return false;
    } else if (at.type != cudaMemoryTypeManaged) {
        return false;
    }
    if (AddressRangeFn fn = address_range_fn()) {
        unsigned long long base = 0;
        size_t size = 0;
        const unsigned long long a = (unsigned long long)(uintptr_t)p;
        if (fn(&base, &size, a) != 0) return false;
        if (a < base || bytes > size || a - base > size - bytes) return false;
    }
    return true;
}

}  // namespace

extern "C" pic_status pic_simulate_sequential_static(const pic_instance_desc* d, int32_t kind,
                                                     int8_t* actions_out, int32_t* final_stock,
                                                     int64_t* total_cost, int64_t* lost) {
    clear_error();
    if (!d || d->mem != PIC_MEM_DEVICE || d->T < 0 || d->N < 1 || d->N > 127 || d->K < 1 ||
        d->K > 65535 || d->R < 1 || d->R > 65535 || !d->x0 || !d->cost ||
        (d->T > 0 && (!d->prod || !d->reg || !actions_out)))
        return record_error(PIC_ERR_INVALID_ARG,
                            "pic_simulate_sequential_static: invalid descriptor (device arrays, "
                            "1<=N<=127, 1<=K,R<=65535, actions_out required when T>0)");
    if (kind != PIC_POLICY_GREEDY && kind != PIC_POLICY_DUAL)
        return record_error(PIC_ERR_UNSUPPORTED,
                            "pic_simulate_sequential_static: greedy and bid-price policies only");
    if (d->cap)
        return record_error(PIC_ERR_UNSUPPORTED,
                            "pic_simulate_sequential_static: node capacity needs an instance");
    if (kind == PIC_POLICY_DUAL && !d->lam)
        return record_error(PIC_ERR_INVALID_ARG, "pic_simulate_sequential_static: bid-price needs lam");
    if ((size_t)d->K * (size_t)d->N > kMaxStockEntries) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "pic_simulate_sequential_static: K*N = %lld exceeds the static scratch limit of %zu "
                 "stock entries",
                 (long long)d->K * d->N, kMaxStockEntries);
        return record_error(PIC_ERR_INVALID_ARG, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return record_error(PIC_ERR_UNSUPPORTED, "pic_simulate_sequential_static: device index too large");
    {
        const size_t T = (size_t)d->T, KN4 = (size_t)d->K * d->N * 4;
        struct { const void* p; size_t bytes; const char* name; } arrays[] = {
            {d->prod, 4 * T, "prod"}, {d->reg, 4 * T, "reg"}, {d->x0, KN4, "x0"},
            {d->cost, (size_t)d->R * d->N * 4, "cost"},
            {d->lam, kind == PIC_POLICY_DUAL ? KN4 : 0, "lam"},
            {actions_out, T, "actions_out"}, {final_stock, final_stock ? KN4 : 0, "final_stock"}};
        for (const auto& x : arrays)
            if (!device_range_ok(x.p, x.bytes, dev)) {
                char msg[200];
                snprintf(msg, sizeof(msg),
                         "pic_simulate_sequential_static: %s is not %zu bytes of device memory of "
                         "the current device",
                         x.name, x.bytes);
                return record_error(PIC_ERR_INVALID_ARG, msg);
            }
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev]) {  // once per device, with that device current
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
            g_addr[dev] = p;
        }
        base = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)d->stream;
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(base);
    int32_t* xwork = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(base) + kCtrlBytes);
    const size_t KN = (size_t)d->K * d->N;

    // the control block starts at zero; the flag word carries validation bits
    if ((e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st))) return cuda_fail(e, "cudaMemsetAsync");
    int dev_sms = 0;
    if ((e = cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev)))
        return cuda_fail(e, "cudaDeviceGetAttribute");
    k_static_validate<<<2 * dev_sms, 256, 0, st>>>(d->T, d->N, d->K, d->R, d->prod, d->reg, d->x0,
                                                   d->cost, kind == PIC_POLICY_DUAL ? d->lam : nullptr,
                                                   &ctrl->pad0);
    if ((e = cudaGetLastError())) return cuda_fail(e, "validation launch");
    int bad = 0;
    if ((e = cudaMemcpyAsync(&bad, &ctrl->pad0, sizeof(int), cudaMemcpyDeviceToHost, st)))
        return cuda_fail(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "cudaStreamSynchronize");
    if (bad & 1) return record_error(PIC_ERR_INVALID_ARG, "prod[t] outside [0, K)");
    if (bad & 2) return record_error(PIC_ERR_INVALID_ARG, "reg[t] outside [0, R)");
    if (bad & 4) return record_error(PIC_ERR_INVALID_ARG, "x0 has a negative entry");
    if (bad & 8) return record_error(PIC_ERR_INVALID_ARG, "|cost| or |lam| not below 2^22");

    if ((e = cudaMemcpyAsync(xwork, d->x0, sizeof(int32_t) * KN, cudaMemcpyDeviceToDevice, st)))
        return cuda_fail(e, "cudaMemcpyAsync");
    if ((e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st))) return cuda_fail(e, "cudaMemsetAsync");
    if (d->T > 0) {
        Instance I;
        memset(&I, 0, sizeof(I));
        I.T = d->T; I.N = d->N; I.K = d->K; I.R = d->R;
        I.NP = ((d->N + 31) / 32) * 32;
        I.has_lam = d->lam != nullptr;
        I.cost16 = (bad & 128) ? 0 : 1;
        I.prod = const_cast<int32_t*>(d->prod);
        I.reg = const_cast<int32_t*>(d->reg);
        I.x0 = const_cast<int32_t*>(d->x0);
        I.cost = const_cast<int32_t*>(d->cost);
        I.lam = const_cast<int32_t*>(d->lam);
        I.xwork = xwork;
        I.act_t = actions_out;
        I.ctrl = ctrl;
        I.num_sms = dev_sms;
        if ((e = sequential_int(&I, kind, st))) return cuda_fail(e, "sequential kernel launch");
    }
    if (final_stock &&
        (e = cudaMemcpyAsync(final_stock, xwork, sizeof(int32_t) * KN, cudaMemcpyDeviceToDevice, st)))
        return cuda_fail(e, "cudaMemcpyAsync");
    long long res[2] = {0, 0};
    if ((e = cudaMemcpyAsync(res, &ctrl->total_cost, sizeof(res), cudaMemcpyDeviceToHost, st)))
        return cuda_fail(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "cudaStreamSynchronize");
    if (total_cost) *total_cost = res[0];
    if (lost) *lost = res[1];
    return PIC_OK;
}
