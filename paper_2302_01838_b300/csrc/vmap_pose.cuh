// Camera-pose refinement on the device, the map held fixed. A camera at
// position p with rotation R (world from camera) casts rays o = p,
// d = R d_c; the object's loss on those rays has per-ray gradients
// (dL/do, dL/dd) from the encoding backward, so dL/dp = sum_rays dL/do and,
// for the rotation update R <- exp([w]x) R, dL/dw = sum_rays d x dL/dd.
#pragma once
#include "vmap_common.cuh"

namespace vmapk {

// pose: [12] = p[3], R[9] row-major. Ray record i: origin p, direction
// R dc_i, then the measured depth, rgb and mask, then 0.
__global__ void k_pose_rays(const float* __restrict__ pose, const float* __restrict__ dc,
                            const float* __restrict__ meas, int n, float* __restrict__ rays) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* R = pose + 3;
    const float c0 = dc[3 * i], c1 = dc[3 * i + 1], c2 = dc[3 * i + 2];
    float* r = rays + (long long)i * REC;
    r[0] = pose[0];
    r[1] = pose[1];
    r[2] = pose[2];
    r[3] = fmaf(R[0], c0, fmaf(R[1], c1, R[2] * c2));
    r[4] = fmaf(R[3], c0, fmaf(R[4], c1, R[5] * c2));
    r[5] = fmaf(R[6], c0, fmaf(R[7], c1, R[8] * c2));
#pragma unroll
    for (int u = 0; u < 5; ++u) r[6 + u] = meas[5 * i + u];
    r[11] = 0.f;
}

constexpr int POSE_THREADS = 256;

// One block: the pose gradient (thread t sums rays t, t + 256, ... in order,
// then a fixed tree over the threads), then one Adam step (Kingma & Ba,
// epsilon added to the root of the corrected second moment) on (p, w) and
// R <- exp([w]x) R by Rodrigues' formula. adam: [13] = m[6], v[6], step count.
__global__ void __launch_bounds__(POSE_THREADS) k_pose_update(float* __restrict__ pose, float* __restrict__ adam,
                                                              const float* __restrict__ gr,
                                                              const float* __restrict__ rays, int n, float lr_t,
                                                              float lr_r, float beta1, float beta2, float eps) {
    __shared__ float part[6][POSE_THREADS];
    const int t = threadIdx.x;
    float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int i = t; i < n; i += POSE_THREADS) {
        const float* q = gr + 6LL * i;        // dL/do, dL/dd
        const float* d = rays + (long long)i * REC + 3;
        g[0] += q[0];
        g[1] += q[1];
        g[2] += q[2];
        g[3] += d[1] * q[5] - d[2] * q[4];    // d x dL/dd
        g[4] += d[2] * q[3] - d[0] * q[5];
        g[5] += d[0] * q[4] - d[1] * q[3];
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) part[c][t] = g[c];
    __syncthreads();
    for (int s = POSE_THREADS / 2; s > 0; s >>= 1) {
        if (t < s)
#pragma unroll
            for (int c = 0; c < 6; ++c) part[c][t] += part[c][t + s];
        __syncthreads();
    }
    if (t != 0) return;
    const float step_count = adam[12] + 1.f;
    const float c1 = 1.f - powf(beta1, step_count), c2 = 1.f - powf(beta2, step_count);
    float st[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const float gc = part[c][0];
        const float m = beta1 * adam[c] + (1.f - beta1) * gc;
        const float v = beta2 * adam[6 + c] + (1.f - beta2) * gc * gc;
        adam[c] = m;
        adam[6 + c] = v;
        st[c] = (m / c1) / (sqrtf(v / c2) + eps);
    }
    adam[12] = step_count;
    for (int a = 0; a < 3; ++a) pose[a] -= lr_t * st[a];
    // R <- exp([w]x) R with w = -lr_r * step (Rodrigues)
    const float w0 = -lr_r * st[3], w1 = -lr_r * st[4], w2 = -lr_r * st[5];
    const float th = sqrtf(w0 * w0 + w1 * w1 + w2 * w2);
    if (th < 1e-12f) return;
    const float k0 = w0 / th, k1 = w1 / th, k2 = w2 / th;
    const float s = sinf(th), c = 1.f - cosf(th);
    const float K[9] = {0.f, -k2, k1, k2, 0.f, -k0, -k1, k0, 0.f};
    float E[9];
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            float kk = 0.f;
            for (int u = 0; u < 3; ++u) kk += K[3 * r + u] * K[3 * u + q];
            E[3 * r + q] = (r == q ? 1.f : 0.f) + s * K[3 * r + q] + c * kk;
        }
    float* R = pose + 3;
    float Rn[9];
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) Rn[3 * r + q] = E[3 * r] * R[q] + E[3 * r + 1] * R[3 + q] + E[3 * r + 2] * R[6 + q];
    for (int u = 0; u < 9; ++u) R[u] = Rn[u];
}

}  // namespace vmapk
