// Device-side batch builder: from the object table and the requested ray
// counts, lay out this step's batch (ray and sample offsets), cut every
// object's rays into tiles per width class, assign tiles to the persistent
// CTAs, number the gradient runs and their partial slots, and list the
// reduce work. A class whose tiles fit its dynamic slot capacity is
// scheduled dynamically: its CTAs take tiles from a counter, and every tile
// is a run with its own slot (the slot depends on the tile, not on the CTA
// that processes it, so the sums stay reproducible). Everything the step's other kernels need is read back from
// device memory, so the launch sequence never changes when objects are
// admitted, stopped or resized (the step can be captured in a CUDA graph
// once and replayed).
#pragma once
#include "vmap_common.cuh"

namespace vmapk {

constexpr int NCLASS = 4;                  // hidden widths 16, 32, 64, 128
constexpr int BUILD_THREADS = 1024;
constexpr int REDUCE_CHUNK = 256;          // parameters per reduce work item (half an item per warp)

__host__ __device__ inline int class_of(int H) { return H == 16 ? 0 : H == 32 ? 1 : H == 64 ? 2 : 3; }
__host__ __device__ inline int hidden_of(int c) { return 16 << c; }

// counts written by k_build (device int array)
enum BuildCount { BC_TILES = 0 /* + class */, BC_NB = 4, BC_RAYS = 5, BC_SAMPLES_LO = 6, BC_SAMPLES_HI = 7,
                  BC_ITEMS = 8, BC_DYN = 9 /* + class: scheduled dynamically */, BC_N = 16 };

struct BuildArgs {
    const ObjDev* objs;
    ObjBatch* ob;
    const int* n_obj;          // device: objects in the table
    const int* req;            // device [max_objects]: requested rays per object
    const int* status;         // device [max_objects]: non-zero = frozen
    int given;                 // 1: the batch's rays come from the caller, object-major
    int rt[NCLASS];            // rays per tile per class
    int mmax[NCLASS];          // samples per tile, at most, per class
    int rtmax;                 // rays per tile, at most
    int grid[NCLASS];          // persistent grid per class
    int dyn_cap[NCLASS];       // most tiles a class may have to be scheduled dynamically; 0: never
    TileDev* tiles;            // [NCLASS][tile_cap]
    int* flags;                // [NCLASS][tile_cap] scratch
    int tile_cap;
    long long part_base[NCLASS];
    int* bobj;                 // [max_objects] batch object ids
    int* bray;                 // [max_objects] their first batch ray
    int* ray_bj;               // [max_rays_total] object of each batch ray, or NULL
    int2* items;               // reduce work (batch index, chunk)
    int* counts;               // [BC_N]
    int* sig;                  // [2 + max_objects] inputs of the last build (n_obj, given, rays
                               // per object as built), or NULL: always build
};

__device__ __forceinline__ int rays_per_tile(const BuildArgs& a, int c, int S) {
    return max(1, min(min(a.rt[c], a.rtmax), a.mmax[c] / S));
}

// Block-wide exclusive scan of one long long per thread (BUILD_THREADS
// threads); returns the exclusive prefix and writes the block total.
__device__ long long block_scan(long long v, long long* total, long long* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        long long s = lane < (BUILD_THREADS >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        if (lane < (BUILD_THREADS >> 5)) sh[32 + lane] = s;
    }
    __syncthreads();
    const long long before = (w ? sh[32 + w - 1] : 0) + x - v;
    *total = sh[32 + (BUILD_THREADS >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(BUILD_THREADS) k_build(BuildArgs a) {
    __shared__ long long sh[64];
    __shared__ long long carry[8];
    __shared__ int changed;
    const int K = *a.n_obj;

    // ---- the layout depends only on (objects, rays per object as built, given):
    // when none changed since the last build, every output is still valid -----
    if (a.sig) {
        if (threadIdx.x == 0) changed = a.sig[0] != K || a.sig[1] != a.given;
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += BUILD_THREADS) {
            const int R = (a.objs[k].active && a.status[k] == 0 && a.req[k] > 0) ? a.req[k] : 0;
            if (R != a.sig[2 + k]) changed = 1;
        }
        __syncthreads();
        if (!changed) return;
        for (int k = threadIdx.x; k < K; k += BUILD_THREADS)
            a.sig[2 + k] = (a.objs[k].active && a.status[k] == 0 && a.req[k] > 0) ? a.req[k] : 0;
        if (threadIdx.x == 0) {
            a.sig[0] = K;
            a.sig[1] = a.given;
        }
    }
    if (threadIdx.x < 8) carry[threadIdx.x] = 0;
    __syncthreads();

    // ---- per object: rays, samples, tiles; offsets by block scans ----------
    for (int base = 0; base < K; base += BUILD_THREADS) {
        const int k = base + threadIdx.x;
        int R = 0, S = 1, c = 0, nt = 0;
        if (k < K) {
            const ObjDev& o = a.objs[k];
            R = (o.active && a.status[k] == 0 && a.req[k] > 0) ? a.req[k] : 0;
            S = o.S;
            c = class_of(o.hidden);
            const int rt = rays_per_tile(a, c, S);
            nt = R ? (R + rt - 1) / rt : 0;
        }
        long long tot;
        const long long ray0 = carry[0] + block_scan(R, &tot, sh);
        const long long nray = tot;
        const long long smp0 = carry[1] + block_scan((long long)R * S, &tot, sh);
        const long long nsmp = tot;
        const long long j0 = carry[2] + block_scan(R > 0 ? 1 : 0, &tot, sh);
        const long long njb = tot;
        long long tb[NCLASS], ntc[NCLASS];
#pragma unroll
        for (int q = 0; q < NCLASS; ++q) {
            tb[q] = carry[3 + q] + block_scan(c == q ? nt : 0, &tot, sh);
            ntc[q] = tot;
        }
        if (k < K) {
            ObjBatch& b = a.ob[k];
            b.R = R;
            b.ray_off = (int)ray0;
            b.sample_off = smp0;
            b.src_off = a.given ? ray0 : a.objs[k].pool_off;
            b.tile_begin = (int)tb[c];
            b.n_runs = 0;
            b.part_off = 0;
            if (R > 0) {
                a.bobj[j0] = k;
                a.bray[j0] = (int)ray0;
                if (a.ray_bj)
                    for (int i = 0; i < R; ++i) a.ray_bj[ray0 + i] = k;
                const int rt = rays_per_tile(a, c, S);
                TileDev* tl = a.tiles + (long long)c * a.tile_cap + tb[c];
                for (int i = 0; i < nt; ++i) {
                    TileDev td;
                    td.obj = k;
                    td.ray0 = (int)ray0 + i * rt;
                    td.nr = min(rt, R - i * rt);
                    td.pad = 0;
                    td.part = 0;
                    tl[i] = td;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry[0] += nray;
            carry[1] += nsmp;
            carry[2] += njb;
            for (int q = 0; q < NCLASS; ++q) carry[3 + q] += ntc[q];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < NCLASS; ++q) a.counts[BC_TILES + q] = (int)carry[3 + q];
        a.counts[BC_NB] = (int)carry[2];
        a.counts[BC_RAYS] = (int)carry[0];
        a.counts[BC_SAMPLES_LO] = (int)(carry[1] & 0x7FFFFFFF);
        a.counts[BC_SAMPLES_HI] = (int)(carry[1] >> 31);
    }
    __syncthreads();

    // ---- runs: tiles of one object inside one CTA's range share a slot ------
    for (int q = 0; q < NCLASS; ++q) {
        const int n = a.counts[BC_TILES + q];
        const int G = a.grid[q];
        TileDev* tl = a.tiles + (long long)q * a.tile_cap;
        int* fl = a.flags + (long long)q * a.tile_cap;
        const long long stride = param_count(hidden_of(q)) + NEXTRA;
        const bool dyn = a.dyn_cap[q] > 0 && n <= a.dyn_cap[q];
        if (threadIdx.x == 0) a.counts[BC_DYN + q] = dyn ? 1 : 0;
        for (int t = threadIdx.x; t < n; t += BUILD_THREADS)
            fl[t] = (dyn || t == 0 || tl[t].obj != tl[t - 1].obj) ? 1 : 0;
        __syncthreads();
        for (int cta = threadIdx.x; !dyn && cta < G; cta += BUILD_THREADS) {
            const long long s = (long long)cta * n / G;
            if (s < n) fl[s] = 1;
        }
        __syncthreads();
        long long run_carry = 0;
        for (int base = 0; base < n; base += BUILD_THREADS) {
            const int t = base + threadIdx.x;
            const int f = t < n ? fl[t] : 0;
            long long tot;
            const long long incl = run_carry + block_scan(f, &tot, sh) + f;
            if (t < n) tl[t].part = a.part_base[q] + (incl - 1) * stride;
            run_carry += tot;
        }
        __syncthreads();
    }
    // per object: first slot and slot count
    for (int k = threadIdx.x; k < K; k += BUILD_THREADS) {
        ObjBatch& b = a.ob[k];
        if (b.R == 0) continue;
        const int q = class_of(a.objs[k].hidden);
        const TileDev* tl = a.tiles + (long long)q * a.tile_cap;
        const int rt = rays_per_tile(a, q, a.objs[k].S);
        const int nt = (b.R + rt - 1) / rt;
        const long long stride = param_count(hidden_of(q)) + NEXTRA;
        const long long p0 = tl[b.tile_begin].part, p1 = tl[b.tile_begin + nt - 1].part;
        b.part_off = p0;
        b.n_runs = (int)((p1 - p0) / stride) + 1;
    }
    __syncthreads();

    // ---- reduce work items: (object, chunk of REDUCE_CHUNK parameters) -------
    const int nb = a.counts[BC_NB];
    long long icarry = 0;
    for (int base = 0; base < nb; base += BUILD_THREADS) {
        const int j = base + threadIdx.x;
        int nch = 0;
        if (j < nb) nch = (int)((param_count(a.objs[a.bobj[j]].hidden) + REDUCE_CHUNK - 1) / REDUCE_CHUNK);
        long long tot;
        const long long i0 = icarry + block_scan(nch, &tot, sh);
        for (int c = 0; c < nch; ++c) a.items[i0 + c] = make_int2(a.bobj[j], c);   // (object, chunk)
        icarry += tot;
    }
    if (threadIdx.x == 0) a.counts[BC_ITEMS] = (int)icarry;
}

}  // namespace vmapk
