// Thin wrappers over the sm_100-family tensor-core instructions (tcgen05.*),
// shared-memory matrix descriptors and mbarriers, written as inline PTX.
//
// Operand tiles use the no-swizzle canonical layout: 8x8 "core matrices" of
// 16-bit elements (8 rows of 16 bytes, 128 contiguous bytes). A tile with CC
// columns stores its rows in strips of 8; a strip holds the CC/8 core matrices
// of those rows side by side. Descriptor strides (verified on the device):
//   K-major operand (rows = M or N, columns = K):   LBO = 128, SBO = CC/8 * 128
//   MN-major operand (rows = K, columns = M or N):  LBO = CC/8 * 128, SBO = 128
// i.e. LBO steps between core matrices along K, SBO along M/N.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vmapk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, c) in a core-matrix tile with CC columns
__host__ __device__ __forceinline__ int cm_off(int r, int c, int CC) {
    return ((r >> 3) * (CC >> 3) + (c >> 3)) * 128 + (r & 7) * 16 + (c & 7) * 2;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version for tcgen05; no swizzle, base offset 0
    return d;
}
// K-major tile with CC columns, starting at K column k0 (multiple of 8)
__device__ __forceinline__ uint64_t desc_kmajor(const void* tile, int CC, int k0) {
    return smem_desc(smem_u32(tile) + (k0 >> 3) * 128, 128, (CC >> 3) * 128);
}
// MN-major tile (rows = K) with CC columns, starting at K row k0 (multiple of 8)
__device__ __forceinline__ uint64_t desc_mnmajor(const void* tile, int CC, int k0) {
    return smem_desc(smem_u32(tile) + (k0 >> 3) * (CC >> 3) * 128, (CC >> 3) * 128, 128);
}

// instruction descriptor: kind::f16, BF16 x BF16 -> FP32, M x N, operand majors
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A * B, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"((int)acc));
}

// The same MMA, executed by all 32 lanes of a converged warp: every lane forms
// the operands (so they are warp-uniform values), the lane elect.sync picks
// (the lowest active lane, the same lane at every call of a converged warp)
// issues.
__device__ __forceinline__ void mma_bf16_w(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n.reg .pred p, e;\nelect.sync _|e, 0xffffffff;\nsetp.ne.b32 p, %4, 0;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"((int)acc));
}
// mma_commit by the elected lane of a converged warp (the lane that issued
// the warp's MMAs with mma_bf16_w)
__device__ __forceinline__ void mma_commit_w(uint64_t* mbar) {
    asm volatile(
        "{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}" ::"r"(smem_u32(mbar))
        : "memory");
}

// arrive on mbar once every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* m, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity, long long limit) {
    uint32_t ok = 0;
    for (long long it = 0; it < limit; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_u32(m)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// arrive once on mbar and raise its pending transaction count by `bytes`
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(m)),
                 "r"(bytes)
                 : "memory");
}

// bulk (non-tensor) async copy global -> shared of `bytes` (multiple of 16,
// both addresses 16-byte aligned); completes `bytes` transactions on mbar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, int ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 lanes x 16 consecutive 32-bit columns: thread t gets lane (base lane + t)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// bulk (non-tensor) async copy shared -> global of `bytes` (multiple of 16,
// 16-byte aligned), tracked in the issuing thread's bulk groups
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// this thread's bulk stores have finished reading shared memory (the source may be rewritten)
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Ampere-style asynchronous global -> shared copies (completion by wait_all)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// NC (8, 16 or 32) consecutive columns of this warp's 32 lanes, one wait
template <int NC>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[NC]) {
    static_assert(NC == 8 || NC == 16 || NC == 32, "columns per thread");
    if constexpr (NC == 8) {
        tmem_ld8(taddr, v);
    } else if constexpr (NC == 16) {
        tmem_ld16(taddr, v);
    } else {
        float a[16], b[16];
        tmem_ld16(taddr, a);
        tmem_ld16(taddr + 16, b);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            v[i] = a[i];
            v[16 + i] = b[i];
        }
    }
    tmem_ld_wait();
}

}  // namespace vmapk
