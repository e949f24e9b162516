// Compositional scene rendering (section 3.4): every object renders the rays
// inside its box (the eval mode of the tile kernel writes (O^, D^, C^) per
// ray and object); this kernel ranks the objects a ray meets by their
// expected hit depth D^_k / O^_k (ties: lower list position first; O^_k = 0
// skipped) and composes them front to back the way Eq. 3 composes samples:
//   D = sum_k A_k D^_k, C = sum_k A_k C^_k, O = sum_k A_k O^_k,
//   A_k = prod over the objects j ranked before k of (1 - O^_j).
#pragma once
#include "vmap_common.cuh"

namespace vmapk {

constexpr int COMPOSE_LOCAL = 32;   // objects per ray ranked in registers; more fall back to selection

// rec: [m][n][5] records; one thread per ray
__global__ void __launch_bounds__(256) k_compose(const float* __restrict__ rec, int m, long long n,
                                                 float* __restrict__ depth, float* __restrict__ rgb,
                                                 float* __restrict__ occ) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float key[COMPOSE_LOCAL];
        int idx[COMPOSE_LOCAL];
        int cnt = 0;
        for (int k = 0; k < m; ++k) {
            const float O = rec[((long long)k * n + i) * 5];
            if (O > 0.f) {
                if (cnt < COMPOSE_LOCAL) {
                    // insertion into (key, list position) order
                    const float kk = rec[((long long)k * n + i) * 5 + 1] / O;
                    int p = cnt;
                    while (p > 0 && key[p - 1] > kk) {
                        key[p] = key[p - 1];
                        idx[p] = idx[p - 1];
                        --p;
                    }
                    key[p] = kk;
                    idx[p] = k;
                }
                ++cnt;
            }
        }
        float A = 1.f, D = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Os = 0.f;
        auto take = [&](int k) {
            const float* e = rec + ((long long)k * n + i) * 5;
            D = fmaf(A, e[1], D);
            C0 = fmaf(A, e[2], C0);
            C1 = fmaf(A, e[3], C1);
            C2 = fmaf(A, e[4], C2);
            Os = fmaf(A, e[0], Os);
            A *= 1.f - e[0];
        };
        if (cnt <= COMPOSE_LOCAL) {
            for (int p = 0; p < cnt; ++p) take(idx[p]);
        } else {
            // more objects than registers: repeated selection of the next (key, position)
            float last = -INFINITY;
            int last_k = -1;
            for (int step = 0; step < cnt; ++step) {
                float best = INFINITY;
                int bk = -1;
                for (int k = 0; k < m; ++k) {
                    const float O = rec[((long long)k * n + i) * 5];
                    if (!(O > 0.f)) continue;
                    const float kk = rec[((long long)k * n + i) * 5 + 1] / O;
                    const bool after = kk > last || (kk == last && k > last_k);
                    if (after && (kk < best || (kk == best && k < bk))) {
                        best = kk;
                        bk = k;
                    }
                }
                if (bk < 0) break;
                take(bk);
                last = best;
                last_k = bk;
            }
        }
        depth[i] = D;
        if (rgb) {
            rgb[3 * i] = C0;
            rgb[3 * i + 1] = C1;
            rgb[3 * i + 2] = C2;
        }
        if (occ) occ[i] = Os;
    }
}

}  // namespace vmapk
