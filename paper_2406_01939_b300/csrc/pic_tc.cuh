// Helpers for tcgen05 kernels with 128-row tiles (one TMEM lane per row):
// shared-memory operand layout and descriptors, the kind::f16 instruction
// descriptor, MMA issue, commit to an mbarrier, bounded waits, TMEM loads.
//
// Shared-memory operands use 8x8 core matrices (8 rows of 16 bytes) without
// swizzle: element (r, c) of an [R][C] BF16 buffer at (r/8)(C/8)128 + (c/8)128 +
// (r%8)16 + (c%8)2.  Read with its rows as the M/N index it is a K-major
// operand (LBO 128 B along K, SBO (C/8)128 B along M/N); read with its rows as
// the K index it is an MN-major operand (LBO (C/8)128 B along K, SBO 128 B along
// M/N).  Descriptors: start address, LBO and SBO in 16-byte units, version bits
// 46-47 = 1, no swizzle.
#pragma once

#include <cuda_bf16.h>

namespace pic {
namespace tc {

__device__ __forceinline__ int lay(int r, int c, int C) {
    return (r >> 3) * (C >> 3) * 128 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2;
}

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFF) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: BF16 A and B, FP32 D, M = 128
__host__ __device__ constexpr unsigned tc_idesc(int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)a_mn << 15) | ((unsigned)b_mn << 16) |
           ((unsigned)(N >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(unsigned long long* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(mbar)));
}

// Wait for the next phase of the CTA's mbarrier (bounded); false on time-out.
__device__ __forceinline__ bool tc_wait(unsigned long long* mbar, unsigned& phase) {
    unsigned done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(su32(mbar)), "r"(phase));
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    return done != 0;
}

__device__ __forceinline__ void tc_ld16(unsigned addr, float v[16]) {
    unsigned u[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
                   "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(u[i]);
}

// Shared-memory writes by the threads become visible to the tensor cores, and
// the threads meet (with the tcgen05 ordering fences around the barrier).
__device__ __forceinline__ void tc_sync_operands() {
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

__device__ __forceinline__ unsigned pack2bf(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&v);
}

// 16 BF16 values (columns c0..c0+15 of row t of a [R][C] core-matrix buffer)
__device__ __forceinline__ void st_row16(unsigned char* buf, int t, int c0, int C, const float v[16]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint4 q;
        q.x = pack2bf(v[8 * h + 0], v[8 * h + 1]);
        q.y = pack2bf(v[8 * h + 2], v[8 * h + 3]);
        q.z = pack2bf(v[8 * h + 4], v[8 * h + 5]);
        q.w = pack2bf(v[8 * h + 6], v[8 * h + 7]);
        *reinterpret_cast<uint4*>(buf + lay(t, c0 + 8 * h, C)) = q;
    }
}


}  // namespace tc
}  // namespace pic
