// Per-object gradient reduction + Adam, weight initialisation, and the
// transposed-weight shadow that the forward GEMMs stage from.
#pragma once
#include <cuda_bf16.h>

#include "vmap_build.cuh"
#include "vmap_common.cuh"
#include "vmap_tc.cuh"

namespace vmapk {

enum ReduceMode { RED_ADAM = 0, RED_GRAD = 1, RED_LOSS = 2 };

// index (in bf16 elements) of canonical parameter p inside the object's
// tensor-core weight image (W1 [H][96], W2..W4 [H][H], W5 [16][H], each a
// core-matrix tile), or -1 for a bias
__host__ __device__ inline long long img_index(int H, long long p) {
    for (int l = 0; l < 5; ++l) {
        const long long w0 = w_off(H, l);
        const int K = l == 0 ? DIN : H;
        const int N = l == 4 ? NOUT : H;
        if (p >= w0 && p < w0 + (long long)N * K) {
            const int n = (int)((p - w0) / K), k = (int)((p - w0) % K);
            const long long base = l == 0 ? 0 : (long long)H * DINP + (long long)(l - 1) * H * H;
            const int CC = l == 0 ? DINP : H;
            return base + cm_off(n, k, CC) / 2;
        }
    }
    return -1;
}
__host__ __device__ constexpr long long img_count(int H) { return (long long)H * DINP + 3LL * H * H + 16LL * H; }



// Weight element p of an object of width H (a power of two) -> (layer l,
// output row n, input column k), or -1 for a bias. 32-bit arithmetic; the
// only division is by the constant fan-in of layer 1.
__device__ __forceinline__ int weight_of(int H, int p, int& n, int& k) {
    const int lg = __ffs(H) - 1;
    if (p < DIN * H) {
        n = p / DIN;
        k = p - n * DIN;
        return 0;
    }
    int base = DIN * H + H;
    if (p < base) return -1;
#pragma unroll
    for (int l = 1; l < 4; ++l) {
        if (p < base + H * H) {
            const int q = p - base;
            n = q >> lg;
            k = q & (H - 1);
            return l;
        }
        base += H * H + H;
        if (p < base) return -1;
    }
    if (p < base + NOUT * H) {
        const int q = p - base;
        n = q >> lg;
        k = q & (H - 1);
        return 4;
    }
    return -1;
}

// index of canonical parameter p in the transposed shadow, or -1 for a bias
__device__ __forceinline__ long long wt_index(int H, long long p) {
#pragma unroll 1
    for (int l = 0; l < 5; ++l) {
        const long long w0 = w_off(H, l);
        const int K = l == 0 ? DIN : H;
        const int N = l == 4 ? NOUT : H;
        if (p >= w0 && p < w0 + (long long)N * K) {
            const long long q = p - w0;
            const long long n = q / K, k = q % K;
            return wt_layer_off(H, l) + k * N + n;
        }
    }
    return -1;
}

// Loss of an object from its run slots' sums (Eq. 4-5 as means). Called by
// a whole warp: lane l sums slots l, l + 32, ... in order, then a fixed
// butterfly combines the lanes (deterministic).
// Fixed grid of REDUCE_THREADS-thread blocks; each warp takes half of a
// reduce work item (object, chunk of REDUCE_CHUNK parameters) from the
// builder's list: 128 parameters, four consecutive ones per lane, moved as
// 16-byte vectors (parameter offsets, slot strides and every width's
// parameter count are multiples of four). It sums the object's run slots in
// slot order and, in the same warp, the object's loss terms (lane-strided
// over runs, then a butterfly); then (RED_ADAM) applies Adam with the
// object's step count + 1, or (RED_GRAD) writes grad_loss[k] * g. With
// RED_ADAM and per-object counters `done` (zero between launches), the last
// warp of an object to finish (every other one has read the step count)
// advances the object's step count unless it is frozen, and resets its counter.
constexpr int REDUCE_THREADS = 256;
constexpr int REDUCE_SLOT_LOADS = 4;    // slot loads in flight per lane (registers)
constexpr int REDUCE_STAGED_SLOTS = 8;  // slot copies in flight per lane (staged in shared memory)
constexpr int REDUCE_BLOCKS_PER_SM = 3; // the grid
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float& at4(float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

__global__ void __launch_bounds__(REDUCE_THREADS, REDUCE_BLOCKS_PER_SM) k_reduce(StepParams sp, const ObjDev* __restrict__ objs,
                                                           const ObjBatch* __restrict__ obs,
                                                           const int2* __restrict__ items,
                                                           const int* __restrict__ counts,
                                                           const float* part, float* params,
                                                           float* wt, float* mom, float* vel,
                                                           int* steps, int* status,
                                                           int mode, const float* __restrict__ grad_loss,
                                                           float* __restrict__ grad_out,
                                                           float* __restrict__ loss_out,
                                                           float* __restrict__ dcenter_out,
                                                           __nv_bfloat16* img, const long long* __restrict__ img_off,
                                                           int* done, const int* __restrict__ n_obj,
                                                           float* const* __restrict__ loss_user_pp,
                                                           const int* gave_up) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int n_units = 2 * counts[BC_ITEMS];   // (item, half)
    // per warp: REDUCE_STAGED_SLOTS slots x 32 lanes x 16 bytes of run-slot staging
    __shared__ __align__(16) float stage[(REDUCE_THREADS / 32) * REDUCE_STAGED_SLOTS * 32 * 4];
    // a second copy of the losses, to the caller's buffer (address read at run time)
    float* const loss_user = loss_user_pp ? *loss_user_pp : nullptr;
    // with n_obj: objects outside the batch report NaN (the batch's heads write the rest)
    if (n_obj) {
        const int K = *n_obj;
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
            if (obs[k].R == 0) {
                if (loss_out) loss_out[k] = __int_as_float(0x7fc00000);
                if (loss_user) loss_user[k] = __int_as_float(0x7fc00000);
            }
    }
    bool wrote_status = false;   // this lane froze its unit's object
    // one unit: half `half` of chunk `chunk` of object k; false: the step is void
    auto reduce_unit = [&](const int k, const int chunk, const int half) -> bool {
        const bool head = chunk == 0 && half == 0;   // the warp that reports per-object results
        const ObjDev& ob = objs[k];
        const ObjBatch& bt = obs[k];
        const int H = ob.hidden;
        const int P = (int)param_count(H);
        const long long stride = P + NEXTRA;
        const int nr = bt.n_runs;
        const float* e = part + bt.part_off + P;   // run t's loss sums at e[t * stride + 0..2]
        const int t1 = mode == RED_ADAM ? steps[k] + 1 : 1;
        const bool frozen = status[k] != 0;
        const int p = chunk * REDUCE_CHUNK + half * (REDUCE_CHUNK / 2) + 4 * lane;
        const bool act = mode != RED_LOSS && p < P;
        const long long q = ob.param_off + p;
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f), th0 = g, m0 = g, v0 = g;
        float ibc1 = 1.f, ibc2 = 1.f;   // reciprocal Adam bias corrections
        long long ioff = -1;            // the object's BF16 image, if any
        if (act && mode == RED_ADAM) {
            th0 = ld4(params + q);
            m0 = ld4(mom + q);
            v0 = ld4(vel + q);
            ibc1 = 1.f / (1.f - powf(sp.beta1, (float)t1));
            ibc2 = 1.f / (1.f - powf(sp.beta2, (float)t1));
            if (img) ioff = img_off[k];
        }
        // Launched behind the step's last tile kernel (programmatic dependent
        // launch), everything above (tables, step counts, weights, moments, Adam
        // bias corrections: none depend on the tile kernels) overlapped its end;
        // the run slots are the tile kernels' output. The wait names the values
        // computed above, so they are formed before it; `part` is not
        // __restrict__, as loads through a restrict-qualified read-only pointer
        // may be hoisted above the wait.
        asm volatile("griddepcontrol.wait;" : "+f"(ibc1), "+f"(ibc2), "+l"(ioff)::"memory");
        // a tensor-core kernel of this step gave up a wait: its run slots are
        // incomplete, so no object is updated (losses NaN, steps not advanced)
        // until the host has read and cleared the flag
        if (gave_up && *(volatile const int*)gave_up) {
            if (head && lane == 0) {
                if (loss_out) loss_out[k] = __int_as_float(0x7fc00000);
                if (loss_user) loss_user[k] = __int_as_float(0x7fc00000);
            }
            return false;
        }
        // loss terms of the first 32 runs, in flight with the gradient loads below
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        if (lane < nr) {
            const float* el = e + (long long)lane * stride;
            s0 = el[0]; s1 = el[1]; s2 = el[2];
        }
        if (act && nr > REDUCE_STAGED_SLOTS) {
            // many slots: REDUCE_STAGED_SLOTS per pass in flight as asynchronous 16-byte
            // copies into this lane's own shared-memory staging (no registers held while
            // they fly; the lane reads back only what it copied), added in slot order
            const float* src = part + bt.part_off + p;
            float* stg = stage + ((threadIdx.x >> 5) * REDUCE_STAGED_SLOTS * 32 + lane) * 4;
            const unsigned s0a = (unsigned)__cvta_generic_to_shared(stg);
            for (int t = 0; t < nr; t += REDUCE_STAGED_SLOTS) {
#pragma unroll
                for (int w = 0; w < REDUCE_STAGED_SLOTS; ++w)
                    if (t + w < nr)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s0a + 512u * w),
                                     "l"(src + (long long)(t + w) * stride)
                                     : "memory");
                asm volatile("cp.async.commit_group;\n" ::: "memory");
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
#pragma unroll
                for (int w = 0; w < REDUCE_STAGED_SLOTS; ++w)
                    if (t + w < nr) {
                        const float4 v = *reinterpret_cast<const float4*>(stg + 128 * w);
                        g.x += v.x; g.y += v.y; g.z += v.z; g.w += v.w;
                    }
            }
        } else if (act) {
            // few slots: (predicated) register loads in flight, added in slot order
            const float* src = part + bt.part_off + p;
            for (int t = 0; t < nr; t += REDUCE_SLOT_LOADS) {
                float4 v[REDUCE_SLOT_LOADS];
#pragma unroll
                for (int w = 0; w < REDUCE_SLOT_LOADS; ++w) v[w] = t + w < nr ? ld4(src + (long long)(t + w) * stride) : g;
#pragma unroll
                for (int w = 0; w < REDUCE_SLOT_LOADS; ++w)
                    if (t + w < nr) {
                        g.x += v[w].x; g.y += v[w].y; g.z += v[w].z; g.w += v[w].w;
                    }
            }
        }
        for (int t = 32 + lane; t < nr; t += 32) {
            const float* el = e + (long long)t * stride;
            s0 += el[0]; s1 += el[1]; s2 += el[2];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        const float R = (float)bt.R;
        const float L = s0 / R + sp.lam_c * (s1 / (3.f * R)) + sp.lam_o * (s2 / R);
        const float gl = grad_loss ? grad_loss[k] : 1.f;
        if (head && lane == 0) {
            const float lv = frozen ? __int_as_float(0x7fc00000) : L;
            if (loss_out) loss_out[k] = lv;
            if (loss_user) loss_user[k] = lv;
            if (dcenter_out) {
                float d[3] = {0.f, 0.f, 0.f};
                for (int t = 0; t < nr; ++t) {
                    const float* x = e + (long long)t * stride;
                    d[0] += x[3]; d[1] += x[4]; d[2] += x[5];
                }
                for (int c = 0; c < 3; ++c) dcenter_out[3 * k + c] = gl * d[c];
            }
        }
        if (mode == RED_LOSS) return true;
        if (mode == RED_ADAM && (frozen || !isfinite(L))) {
            if (!frozen && head && lane == 0) {
                status[k] = 1;
                wrote_status = true;
            }
            return true;
        }
        if (!act) return true;
        if (mode == RED_GRAD) {
#pragma unroll
            for (int i = 0; i < 4; ++i) grad_out[q + i] = gl * at4(g, i);
            return true;
        }
        float4 m = m0, v = v0, th = th0;
        bool bad = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float gi = at4(g, i);
            if (!isfinite(gi)) {       // leave the element, flag the object
                bad = true;
                continue;
            }
            const float mi = sp.beta1 * at4(m0, i) + (1.f - sp.beta1) * gi;
            const float vi = sp.beta2 * at4(v0, i) + (1.f - sp.beta2) * gi * gi;
            at4(m, i) = mi;
            at4(v, i) = vi;
            at4(th, i) = at4(th0, i) - sp.lr * (mi * ibc1) / (sqrtf(vi * ibc2) + sp.eps);
        }
        if (bad) {
            atomicOr(status + k, 2);
            wrote_status = true;
        }
        st4(mom + q, m);
        st4(vel + q, v);
        st4(params + q, th);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int wn, wk;
            const int l = weight_of(H, p + i, wn, wk);
            if (l < 0) continue;
            const float x = at4(th, i);
            const int N = l == 4 ? NOUT : H;
            if (wt) wt[ob.wt_off + wt_layer_off(H, l) + (long long)wk * N + wn] = x;   // transposed shadow
            if (ioff >= 0) {                                                     // BF16 operand image
                const long long base = l == 0 ? 0 : (long long)H * DINP + (long long)(l - 1) * H * H;
                img[ioff + base + cm_off(wn, wk, l == 0 ? DINP : H) / 2] = __float2bfloat16(x);
            }
        }
        return true;
    };
#pragma unroll 1
    for (int u = blockIdx.x * wpb + (threadIdx.x >> 5); u < n_units; u += gridDim.x * wpb) {
        const int2 item = items[u >> 1];
        const int k = item.x;
        wrote_status = false;
        const bool valid = reduce_unit(k, item.y, u & 1);
        if (mode == RED_ADAM && done) {
            // a status write must be visible before the arrival that may let the
            // last warp read the status; nothing else this warp wrote is read here
            __syncwarp();
            const bool fence = __any_sync(0xffffffffu, wrote_status);
            if (lane == 0) {
                if (fence) __threadfence();
                const int units = 2 * (int)((param_count(objs[k].hidden) + REDUCE_CHUNK - 1) / REDUCE_CHUNK);
                if (atomicAdd(done + k, 1) == units - 1) {
                    done[k] = 0;
                    if (valid && atomicAdd(status + k, 0) == 0) steps[k] += 1;
                }
            }
        }
    }
}

// seeded default init: parameter p draws word p % 4 of Philox block p / 4 with
// counter (block, 0, 0xFFFFFFFF, stream); value (2u - 1) / sqrt(fan_in)
__global__ void k_init_params(float* params, int H, unsigned stream, uint32_t key0, uint32_t key1) {
    const long long P = param_count(H);
    const long long nb = (P + 3) / 4;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)b, 0u, 0xFFFFFFFFu, stream), key0, key1);
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
        for (int l = 0; l < 4; ++l) {
            const long long p = 4 * b + l;
            if (p >= P) break;
            int fan_in = H;
            if (p < w_off(H, 1)) fan_in = DIN;
            params[p] = (2.f * word_to_unit(ww[l]) - 1.f) / sqrtf((float)fan_in);
        }
    }
}

// rebuild the transposed shadows of objects 0..n-1 (blockIdx.y = object)
__global__ void k_shadow_all(const ObjDev* __restrict__ objs, const float* __restrict__ params, float* wt) {
    const ObjDev& ob = objs[blockIdx.y];
    const int H = ob.hidden;
    const long long P = param_count(H);
    const float* p = params + ob.param_off;
    float* w = wt + ob.wt_off;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
        int n, k;
        const int l = weight_of(H, (int)i, n, k);
        if (l >= 0) w[wt_layer_off(H, l) + (long long)k * (l == 4 ? NOUT : H) + n] = p[i];
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * H; i += gridDim.x * blockDim.x) w[DIN * H + i] = 0.f;
}

// rebuild the transposed shadow of one object from its canonical parameters
__global__ void k_shadow(const float* __restrict__ params, float* wt, int H) {
    const long long P = param_count(H);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        const long long w = wt_index(H, p);
        if (w >= 0) wt[w] = params[p];
    }
    // padding rows 93..95 of W1^T
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * H; i += gridDim.x * blockDim.x)
        wt[DIN * H + i] = 0.f;
}

}  // namespace vmapk
