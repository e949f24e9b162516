// Shared device-side definitions of the vMAP training library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vmapk {

constexpr int NF = 45;        // encoding frequencies (rows of B)
constexpr int DIN = 93;       // 3 + 2 * 45 encoded features
constexpr int DINP = 96;      // padded to a multiple of 4
constexpr int NOUT = 4;       // occupancy + rgb
constexpr int REC = 12;       // floats per ray record
constexpr int SMAX = 32;      // samples per ray, at most
constexpr int NTHREADS = 256; // threads of the per-tile kernels
constexpr int NEXTRA = 8;     // per-tile partial tail: depth, colour, occupancy sums, dc[3], 2 pad

// Scalars every kernel needs, passed by value (lives in the constant bank).
struct StepParams {
    float B[NF * 3];
    float t_near, depth_pad, d_sigma, t_far;
    float lam_c, lam_o;
    float lr, beta1, beta2, eps;
    uint32_t key0, key1;
};

// One object's fixed description, written by the host when the object is
// added or changed.
struct ObjDev {
    int hidden, S, n_surface, n_strat;
    float c[3];
    float scale;
    long long param_off;   // float offset into the parameter / moment arenas
    long long wt_off;      // float offset into the transposed-weight arena
    long long pool_off;    // record offset into the ray-pool arena
    long long pool_n;      // records in the pool
    unsigned stream;       // Philox stream id
    int active;            // 0: stopped by the caller
};

// One object's place in the current batch, written by the device-side batch
// builder (k_build) at every draw.
struct ObjBatch {
    int R;                 // rays this step (0: not in the batch)
    int ray_off;           // first batch ray
    long long sample_off;  // first batch sample
    long long src_off;     // record offset of its rays in the batch source
                           // (pool arena: pool_off; caller-given rays: ray_off)
    int tile_begin;        // first tile (within its width class)
    int n_runs;            // partial slots holding its gradient
    long long part_off;    // float offset of its first slot
};

// A tile: nr consecutive batch rays of one object, processed by one CTA.
struct TileDev {
    int obj;
    int ray0;         // first batch ray
    int nr;           // rays in the tile
    int pad;
    long long part;   // float offset of the slot of the run the tile belongs to
};

__host__ __device__ constexpr long long param_count(int H) {
    return (long long)DIN * H + H + 3LL * (H * H + H) + NOUT * H + NOUT;
}
// Transposed-weight shadow: W1^T [96][H] (rows 93..95 zero), W2..4^T [H][H], W5^T [H][4].
__host__ __device__ constexpr long long wt_count(int H) {
    return (long long)DINP * H + 3LL * H * H + (long long)H * NOUT;
}
// Offsets of W_l and b_l (l = 0..4) inside the canonical packed block.
__host__ __device__ constexpr long long w_off(int H, int l) {
    return l == 0 ? 0 : (long long)DIN * H + H + (long long)(l - 1) * (H * H + H);
}
__host__ __device__ constexpr long long b_off(int H, int l) {
    return l < 4 ? w_off(H, l) + (l == 0 ? (long long)DIN * H : (long long)H * H)
                 : w_off(H, 4) + (long long)NOUT * H;
}
__host__ __device__ constexpr long long wt_layer_off(int H, int l) {
    return l == 0 ? 0 : (long long)DINP * H + (long long)(l - 1) * H * H;
}

// programmatic dependent launch: let the next kernel of the stream (when it was
// launched with programmatic stream serialization) start; without such a
// dependent this has no effect
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// wait until the grids this one depends on have completed and their writes are
// visible (returns at once for a grid launched without programmatic dependences)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Open-interval uniform: (2 (w >> 9) + 1) 2^-24, exact in FP32.
__device__ __forceinline__ float word_to_unit(uint32_t w) {
    return (float)((w >> 9) * 2u + 1u) * 5.9604644775390625e-8f;
}

__device__ __forceinline__ float sigmoidf_(float y) { return 1.0f / (1.0f + expf(-y)); }

__device__ __forceinline__ float signf_(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

}  // namespace vmapk
