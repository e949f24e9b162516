// Tensor-core GEMMs of the warm-start hypernetwork's 128-wide shared layers
// (BF16 operands converted from FP32 on load, FP32 accumulation in TMEM).
//
//   k_hgemm_rows<B_MN, EPI>:  C[M][128] = A[M][128] op(B) (+ bias, ReLU)
//       A row-major FP32; B_MN = false: B is W [128 out][128 in] row-major and
//       op(B) = W^T (forward layers); B_MN = true: B is W [128][128] used as
//       is (input gradients dA = dZ W). One CTA per 128 rows of A.
//   k_hgemm_tn:  part[s][128][128] = sum over rows r of chunk s of
//       A[r][:]^T B[r][:]  (weight gradients dW = dZ^T h over all points);
//       the chunks' partial sums are added in chunk order afterwards.
//
// Operands go to shared memory in the no-swizzle core-matrix layout of
// vmap_tc.cuh; the MMAs are M = 128, N = 128, K = 16 (kind::f16, BF16 in,
// FP32 out); every mbarrier wait is bounded and a give-up sets *err.
#pragma once
#include <cuda_bf16.h>

#include "vmap_tc.cuh"

namespace vmapk {

constexpr int HG = 128;                      // the shared layers' width
constexpr long long HG_WAIT_LIMIT = 1LL << 26;

struct HgemmSmem {
    static constexpr int A = 0;              // [128][128] bf16
    static constexpr int B = HG * HG * 2;    // [128][128] bf16
    static constexpr int MBAR = 2 * HG * HG * 2;
    static constexpr int TSLOT = MBAR + 8;
    static constexpr int BYTES = TSLOT + 8;
};

// 8 FP32 values -> 4 packed BF16 pairs, written as 16 bytes
__device__ __forceinline__ void hg_store8(unsigned char* tile, int off, const float4& a, const float4& b) {
    __nv_bfloat162 p[4] = {__floats2bfloat162_rn(a.x, a.y), __floats2bfloat162_rn(a.z, a.w),
                           __floats2bfloat162_rn(b.x, b.y), __floats2bfloat162_rn(b.z, b.w)};
    *reinterpret_cast<uint4*>(tile + off) = *reinterpret_cast<const uint4*>(p);
}

// rows [r0, r0 + 128) of a row-major [*][128] FP32 matrix -> core-matrix tile (rows = tile rows)
__device__ __forceinline__ void hg_load_rows(unsigned char* tile, const float* __restrict__ src, long long r0,
                                             long long nrows) {
    for (int i = threadIdx.x; i < HG * (HG / 8); i += blockDim.x) {
        const int r = i / (HG / 8), c = (i % (HG / 8)) * 8;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (r0 + r < nrows) {
            const float4* p = reinterpret_cast<const float4*>(src + (r0 + r) * HG + c);
            a = p[0];
            b = p[1];
        }
        hg_store8(tile, cm_off(r, c, HG), a, b);
    }
}

__device__ __forceinline__ bool hg_mma_wait(uint64_t* mbar, uint32_t phase, int* err) {
    const bool ok = mbar_wait(mbar, phase, HG_WAIT_LIMIT);
    if (!ok) atomicExch(err, 1);
    return ok;
}

template <bool B_MN, int EPI>
__global__ void __launch_bounds__(128) k_hgemm_rows(long long M, const float* __restrict__ A,
                                                    const float* __restrict__ B, const float* __restrict__ bias,
                                                    float* __restrict__ C, int* err) {
    using S = HgemmSmem;
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::MBAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::TSLOT);
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long r0 = (long long)blockIdx.x * HG;
    if (tid == 0) mbar_init(mbar, 1);
    if (warp == 0) tmem_alloc(tslot, HG);
    hg_load_rows(sm + S::A, A, r0, M);
    hg_load_rows(sm + S::B, B, 0, HG);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
#pragma unroll
        for (int kc = 0; kc < HG / 16; ++kc) {
            const uint64_t bd = B_MN ? desc_mnmajor(sm + S::B, HG, 16 * kc) : desc_kmajor(sm + S::B, HG, 16 * kc);
            mma_bf16(tmem, desc_kmajor(sm + S::A, HG, 16 * kc), bd, idesc_bf16(HG, HG, 0, B_MN ? 1 : 0), kc > 0);
        }
        mma_commit(mbar);
    }
    const bool ok = hg_mma_wait(mbar, 0, err);
    tc_fence_after();
    const long long r = r0 + tid;          // TMEM lane = row of the tile
    if (ok && r < M) {
#pragma unroll 1
        for (int c0 = 0; c0 < HG; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if (EPI >= 1) v[j] += bias[c0 + j];
                if (EPI == 2) v[j] = fmaxf(v[j], 0.f);
            }
            float4* dst = reinterpret_cast<float4*>(C + r * HG + c0);
#pragma unroll
            for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
    } else if (!ok) {
        // the MMA may still be running: wait once more (bounded) before freeing TMEM
        if (tid == 0) mbar_wait(mbar, 0, HG_WAIT_LIMIT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, HG);
}

// split s takes rows [s * chunk, min(K, (s + 1) * chunk)), chunk a multiple of 128
__global__ void __launch_bounds__(128) k_hgemm_tn(long long K, long long chunk, const float* __restrict__ A,
                                                  const float* __restrict__ B, float* __restrict__ part, int* err) {
    using S = HgemmSmem;
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::MBAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::TSLOT);
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long k0 = (long long)blockIdx.x * chunk, k1 = min(K, k0 + chunk);
    if (tid == 0) mbar_init(mbar, 1);
    if (warp == 0) tmem_alloc(tslot, HG);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;
    bool ok = true;
    int nsub = 0;
#pragma unroll 1
    for (long long kb = k0; kb < k1 && ok; kb += HG, ++nsub) {
        // rows kb .. kb + 127 of A and B: tiles with rows = K, columns = M (A) or N (B): MN-major operands
        hg_load_rows(sm + S::A, A, kb, k1);
        hg_load_rows(sm + S::B, B, kb, k1);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int kc = 0; kc < HG / 16; ++kc)
                mma_bf16(tmem, desc_mnmajor(sm + S::A, HG, 16 * kc), desc_mnmajor(sm + S::B, HG, 16 * kc),
                         idesc_bf16(HG, HG, 1, 1), nsub > 0 || kc > 0);
            mma_commit(mbar);
        }
        ok = hg_mma_wait(mbar, phase, err);   // the tiles are reloaded next: wait for this MMA batch
        phase ^= 1;
        ok = __syncthreads_and(ok);
        tc_fence_after();
    }
    float* out = part + (long long)blockIdx.x * HG * HG + (long long)tid * HG;   // lane = row m of dW
    if (ok && nsub > 0) {
#pragma unroll 1
        for (int c0 = 0; c0 < HG; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
            tmem_ld_wait();
            float4* dst = reinterpret_cast<float4*>(out + c0);
#pragma unroll
            for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
    } else {
        for (int c = 0; c < HG; ++c) out[c] = 0.f;
        if (!ok && tid == 0) mbar_wait(mbar, phase ^ 1, HG_WAIT_LIMIT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, HG);
}

}  // namespace vmapk
