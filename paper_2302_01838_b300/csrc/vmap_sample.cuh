// Ray picking and depth-guided sampling (vMAP section 3.3, Eq. 1 and Eq. 2).
#pragma once
#include "vmap_build.cuh"
#include "vmap_common.cuh"

namespace vmapk {

// Sequential reader of one ray's Philox words: counter (ray, block, step, stream).
struct WordStream {
    uint32_t ctr0, ctr2, ctr3, k0, k1;
    uint32_t block;
    uint4 cur;
    int lane;
    __device__ WordStream(uint32_t ray, uint32_t step, uint32_t stream, uint32_t key0, uint32_t key1)
        : ctr0(ray), ctr2(step), ctr3(stream), k0(key0), k1(key1), block(0), lane(4) {}
    __device__ __forceinline__ uint32_t next() {
        if (lane == 4) {
            cur = philox4x32_10(make_uint4(ctr0, block, ctr2, ctr3), k0, k1);
            ++block;
            lane = 0;
        }
        const uint32_t w = lane == 0 ? cur.x : lane == 1 ? cur.y : lane == 2 ? cur.z : cur.w;
        ++lane;
        return w;
    }
};

// Largest j in [0, n) with off[j] <= i (off ascending, off[0] == 0).
__device__ __forceinline__ int upper_index(const int* off, int n, int i) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One thread per batch ray (fixed grid; threads past the batch exit). Writes
// the picked pool index (the ray's own index when the caller gives the rays)
// and S sorted depths.
//   word 0          -> pick = floor(w * n_pool / 2^32)
//   words 1..N_c    -> u_j, t = t_n + (j + u_j) / N_c * (t_s + pad - t_n)      (Eq. 1)
//   next word pairs -> Box-Muller z = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2),
//                      t = max(t_s + d_sigma z, t_n)                            (Eq. 2)
// t_s is the ray's depth, or t_far when the depth is not positive.
__global__ void __launch_bounds__(128) k_sample(StepParams sp, const ObjDev* __restrict__ objs,
                                                const ObjBatch* __restrict__ obs,
                                                const int* __restrict__ bobj,
                                                const int* __restrict__ bray_off,
                                                const int* __restrict__ counts,
                                                const float* __restrict__ src, int given,
                                                const int* __restrict__ steps,
                                                int* __restrict__ pick_out,
                                                float* __restrict__ t_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int total_rays = counts[BC_RAYS];
    const int nb = counts[BC_NB];
    if (i >= total_rays) return;
    const int j = upper_index(bray_off, nb, i);
    const int k = bobj[j];
    const ObjDev& ob = objs[k];
    const ObjBatch& bt = obs[k];
    const int r = i - bt.ray_off;
    WordStream ws((uint32_t)r, (uint32_t)steps[k], ob.stream, sp.key0, sp.key1);

    // word 0 picks the ray; with caller-given rays it is drawn and dropped so
    // the depth draws keep their word positions
    const uint32_t w0 = ws.next();
    const long long pick = given ? (long long)r
                                 : (long long)(((unsigned long long)w0 * (unsigned long long)ob.pool_n) >> 32);
    pick_out[i] = (int)pick;
    const float depth = src[(bt.src_off + pick) * REC + 6];
    const float ts = depth > 0.f ? depth : sp.t_far;
    const float lo = sp.t_near;
    const float span = ts + sp.depth_pad - lo;

    float t[SMAX];
    const int Ns = ob.n_surface, Nc = ob.n_strat, S = ob.S;
    for (int q = 0; q < Nc; ++q) {
        const float u = word_to_unit(ws.next());
        t[Ns + q] = lo + ((float)q + u) / (float)Nc * span;
    }
    for (int p = 0; 2 * p < Ns; ++p) {
        const float u1 = word_to_unit(ws.next());
        const float u2 = word_to_unit(ws.next());
        const float rho = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        t[2 * p] = fmaxf(ts + sp.d_sigma * (rho * cs), lo);
        if (2 * p + 1 < Ns) t[2 * p + 1] = fmaxf(ts + sp.d_sigma * (rho * sn), lo);
    }
    // stable insertion sort (surface samples first among equals)
    for (int a = 1; a < S; ++a) {
        const float v = t[a];
        int b = a - 1;
        while (b >= 0 && t[b] > v) { t[b + 1] = t[b]; --b; }
        t[b + 1] = v;
    }
    float* dst = t_out + bt.sample_off + (long long)r * S;
    for (int a = 0; a < S; ++a) dst[a] = t[a];
}

}  // namespace vmapk
