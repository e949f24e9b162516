// Ray picking and depth-guided sampling (vMAP section 3.3, Eq. 1 and Eq. 2).
#pragma once
#include "vmap_build.cuh"
#include "vmap_common.cuh"
#include "vmap_tc.cuh"

namespace vmapk {

// Largest j in [0, n) with off[j] <= i (off ascending, off[0] == 0).
__device__ __forceinline__ int upper_index(const int* off, int n, int i) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One warp per batch ray at a time (SAMPLE_RAYS_PER_BLOCK warps per block, the
// warps striding over the batch), one lane per sample slot. Writes the picked pool
// index (the ray's own index when the caller gives the rays) and S sorted depths.
// Philox words of a ray, in order (word w is lane w % 4 of block w / 4):
//   word 0          -> pick = floor(w * n_pool / 2^32)
//   words 1..N_c    -> u_j, t = t_n + (j + u_j) / N_c * (t_s + pad - t_n)      (Eq. 1)
//   next word pairs -> Box-Muller z = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2),
//                      t = max(t_s + d_sigma z, t_n)                            (Eq. 2)
// t_s is the ray's depth, or t_far when the depth is not positive. A ray off
// the object's mask (M = 0) ends at the surface it hits (the supplementary
// material's termination of rays that cross the box but belong to another
// surface): its stratified range stops at t_s, its Gaussian samples are
// clamped above at t_s. Slots
// 0..N_s-1 hold the surface samples, N_s.. the stratified ones, sorted ascending.
constexpr int SAMPLE_RAYS_PER_BLOCK = 8;
constexpr int SAMPLE_BLOCKS_PER_SM = 8;   // one wave: 64 warps per SM at 29 registers

__global__ void __launch_bounds__(32 * SAMPLE_RAYS_PER_BLOCK) k_sample(
    StepParams sp, const ObjDev* __restrict__ objs, const ObjBatch* __restrict__ obs, const int* __restrict__ bobj,
    const int* __restrict__ bray_off, const int* __restrict__ ray_obj, const int* __restrict__ counts,
    const float* __restrict__ src, int given, const int* __restrict__ steps, int* __restrict__ pick_out,
    float* __restrict__ t_out) {
    // a tile kernel launched behind the sampler may take SMs its last blocks
    // free; it waits for the sampler's completion before reading picks and depths
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int total_rays = counts[BC_RAYS];
    // warps stride over the batch's rays: a grid of one wave serves any batch size
    // (the grid is fixed when the step is captured, the ray count is the builder's)
    const int n_warps = gridDim.x * SAMPLE_RAYS_PER_BLOCK;
#pragma unroll 1
    for (int i = blockIdx.x * SAMPLE_RAYS_PER_BLOCK + (threadIdx.x >> 5); i < total_rays; i += n_warps) {
        // the ray's object: from the builder's per-ray table, or by search
        const int k = ray_obj ? ray_obj[i] : bobj[upper_index(bray_off, counts[BC_NB], i)];
        const ObjDev& ob = objs[k];
        const ObjBatch& bt = obs[k];
        const uint32_t r = (uint32_t)(i - bt.ray_off), step = (uint32_t)steps[k], stream = ob.stream;
        const int Ns = ob.n_surface, Nc = ob.n_strat, S = ob.S;

        // lane b computes Philox block b of the ray; words travel by shuffles
        const int nblk = (1 + Nc + 2 * ((Ns + 1) / 2) + 3) / 4;
        uint4 blk = make_uint4(0u, 0u, 0u, 0u);
        if (lane < nblk) blk = philox4x32_10(make_uint4(r, (uint32_t)lane, step, stream), sp.key0, sp.key1);
        auto word = [&](int w) {   // warp-collective: every lane asks for its own word w
            const int sl = w >> 2, c = w & 3;
            const uint32_t x = __shfl_sync(0xffffffffu, blk.x, sl), y = __shfl_sync(0xffffffffu, blk.y, sl);
            const uint32_t z = __shfl_sync(0xffffffffu, blk.z, sl), ww = __shfl_sync(0xffffffffu, blk.w, sl);
            return c == 0 ? x : c == 1 ? y : c == 2 ? z : ww;
        };
        // word 0 picks the ray; with caller-given rays it is drawn and dropped so
        // the depth draws keep their word positions
        const uint32_t w0 = word(0);
        const int p2 = lane >> 1;
        const uint32_t wa = word(lane < Ns ? 1 + Nc + 2 * p2 : (lane < S ? 1 + (lane - Ns) : 0));
        const uint32_t wb = word(lane < Ns ? 2 + Nc + 2 * p2 : 0);
        const long long pick = given ? (long long)r
                                     : (long long)(((unsigned long long)w0 * (unsigned long long)ob.pool_n) >> 32);
        if (lane == 0) pick_out[i] = (int)pick;
        const float depth = src[(bt.src_off + pick) * REC + 6];
        const bool on_mask = src[(bt.src_off + pick) * REC + 10] > 0.f;
        const float ts = depth > 0.f ? depth : sp.t_far;
        const float lo = sp.t_near;
        const float span = ts + (on_mask ? sp.depth_pad : 0.f) - lo;

        float t = INFINITY;
        if (lane < Ns) {
            const float u1 = word_to_unit(wa);
            const float u2 = word_to_unit(wb);
            const float rho = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
            t = fmaxf(ts + sp.d_sigma * (rho * ((lane & 1) ? sn : cs)), lo);
            if (!on_mask) t = fminf(t, ts);
        } else if (lane < S) {
            const int q = lane - Ns;
            const float u = word_to_unit(wa);
            t = lo + ((float)q + u) / (float)Nc * span;
        }
        // ascending order: a bitonic network over the warp's 32 lanes (lanes past S
        // hold +inf and sort last); equal values are interchangeable, so the
        // stored depths are the stable order's
    #pragma unroll
        for (int kb = 2; kb <= 32; kb <<= 1) {
    #pragma unroll
            for (int jb = kb >> 1; jb > 0; jb >>= 1) {
                const float o = __shfl_xor_sync(0xffffffffu, t, jb);
                const bool keep_min = ((lane & jb) == 0) == ((lane & kb) == 0);
                t = keep_min ? fminf(t, o) : fmaxf(t, o);
            }
        }
        if (lane < S) t_out[bt.sample_off + (long long)r * S + lane] = t;
    }
}

}  // namespace vmapk
