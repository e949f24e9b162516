// Persistent fused FP32 training kernel: encoding, MLP forward, occupancy
// rendering, losses, and the backward through rendering, MLP and encoding.
//
// Work unit: a tile of whole rays of one object (so the per-ray scans of
// Eq. 3 stay inside one CTA). A class launch (one hidden width H) runs a
// fixed grid; CTA c processes the contiguous tile range
// [c n / G, (c + 1) n / G) of the class's n tiles, which the device-side batch
// builder wrote. Consecutive tiles of the same object form a run; the CTA adds
// each tile's weight gradient into the run's slot of the partial buffer (the
// first tile stores, the next ones add), so an object has at most
// (CTAs covering it + 1) slots and the reduce/Adam kernel adds them in a
// fixed order: results are bitwise reproducible. When the builder schedules
// the class dynamically, the CTAs take tiles from a counter instead, and each
// tile stores into its own slot: the CTAs that start early (on SMs another
// width class's kernel has left) take more tiles, and the sums stay the same.
//
// Activations live in shared memory, feature-major [feature][sample], row
// stride LD = Mpad + 4 (LD = 4 mod 8: eight consecutive rows read at one
// sample column hit distinct banks). Each layer is a shared-memory SIMT GEMM
// with 4x4 register tiles. For H >= 32 the 96-row encoding shares the rows of
// hidden layers 2-4 (it is recomputed for the layer-1 weight gradient), which
// lets two CTAs share an SM at H = 32.
#pragma once
#include <cuda_bf16.h>
#include "vmap_common.cuh"

namespace vmapk {

enum TileMode { MODE_TRAIN = 0, MODE_FORWARD = 1, MODE_GRAD_CENTER = 2, MODE_EVAL = 3, MODE_QUERY = 4 };

// MMAX: samples per tile; CTAS: CTAs per SM (shared memory); THREADS: CTA
// size. Width 64 (one CTA per SM, 112-sample tiles) runs 16 warps, which
// hide more shared-memory latency (0.666 vs 0.743 ms per step, 50 objects);
// width 128 runs 12: a 48-sample tile has 12 x 32 = 384 4x4 register tiles
// per hidden layer, one per thread (0.433 vs 0.461 ms per launch with 8).
template <int H> struct TileCfg;
template <> struct TileCfg<16>  { static constexpr int MMAX = 120; static constexpr bool GSEP = true;  static constexpr int CTAS = 2; static constexpr int THREADS = 256; };
template <> struct TileCfg<32>  { static constexpr int MMAX = 136; static constexpr bool GSEP = false; static constexpr int CTAS = 2; static constexpr int THREADS = 256; };
template <> struct TileCfg<64>  { static constexpr int MMAX = 112; static constexpr bool GSEP = false; static constexpr int CTAS = 1; static constexpr int THREADS = 512; };
template <> struct TileCfg<128> { static constexpr int MMAX = 48;  static constexpr bool GSEP = false; static constexpr int CTAS = 1; static constexpr int THREADS = 384; };

constexpr int RED_FLOATS = 4096;   // split-reduction scratch
constexpr int RAYF = 16;           // floats of per-ray scratch
constexpr int RTMAX = 32;          // rays per tile, at most (training / eval modes)

template <int H> struct TileSmem {
    static constexpr int MMAX = TileCfg<H>::MMAX;
    static constexpr bool GSEP = TileCfg<H>::GSEP;
    static_assert(GSEP || 3 * H >= DINP, "the encoding must fit in hidden rows 2-4");
    static constexpr int LD = MMAX + 4;
    static constexpr int WS = (DINP * H > H * H ? DINP * H : H * H);
    static constexpr int ACT = 0;                                      // [4][H][LD] hidden activations
    static constexpr int G = GSEP ? 4 * H * LD : H * LD;               // [96][LD] encoding
    static constexpr int Y = GSEP ? (4 * H + DINP) * LD : 4 * H * LD;  // [4][LD] outputs / grads
    static constexpr int W = Y + 4 * LD;                               // weight staging
    // a second weight buffer (widths up to 64, where it fits beside the
    // activations): each forward layer's weights are copied during the GEMM before it
    static constexpr bool WDB = H <= 64;
    static constexpr int W2 = W + WS;                                  // [H][H] second buffer
    static constexpr int RED = W2 + (WDB ? H * H : 0);
    static constexpr int PS = RED + RED_FLOATS;                        // [LD] per-sample scratch
    static constexpr int TS = PS + LD;                                 // [LD] sample depths t
    static constexpr int RAYS = TS + LD;                               // [RTMAX][RAYF]
    static constexpr int TOTAL = RAYS + RTMAX * RAYF;
    static constexpr size_t BYTES = (size_t)TOTAL * sizeof(float);
};

// ---------------------------------------------------------------------------
// out[n][m] = epi( sum_k A[k][m] * Bm[k][n] ),  m < Mpad, n < N.
// A: [K][lda] in smem, Bm: [K][N] dense in smem.
// EPI 0: + bias, ReLU;  EPI 1: + bias;  EPI 2: * (out[n][m] > 0), in place.
// A warp covers 4 sample quads x 8 output quads: its A loads touch 64
// consecutive bytes and its B loads 128. A warp's 16-byte shared load takes
// as many wavefronts as the most distinct vectors any group of four
// consecutive lanes reads, and two at least (measured with ncu's wavefront
// counters); so each four-lane group takes 2 sample quads x 2 output quads:
// two wavefronts per load for A and B (lanes along the sample quads would
// cost four for A). Sample quads are grouped by four, so a tile wastes at
// most three quads of padding per group.
// ---------------------------------------------------------------------------
template <int N, int K, int EPI>
__device__ __forceinline__ void gemm_fwd(const float* __restrict__ A, int lda,
                                         const float* __restrict__ Bm,
                                         const float* __restrict__ bias, float* out, int ldo,
                                         int Mpad) {
    constexpr int NQ = N / 4;
    const int MQ = Mpad >> 2;
    const int items = ((MQ + 3) >> 2) * 4 * NQ;
    for (int f = threadIdx.x; f < items; f += blockDim.x) {
        int mq, nq;
        if constexpr (NQ % 2 == 0) {
            // each group of four lanes takes 2 sample quads x 2 output quads (a
            // 16-byte shared load costs as many wavefronts as the most distinct
            // vectors any four-lane group reads, two at least)
            const int e = f % (4 * NQ), g = e >> 2, t = e & 3;
            mq = (f / (4 * NQ)) * 4 + 2 * (g & 1) + (t & 1);
            nq = 2 * (g >> 1) + (t >> 1);
        } else {
            mq = (f / (4 * NQ)) * 4 + (f & 3);
            nq = (f >> 2) % NQ;
        }
        if (mq >= MQ) continue;
        float acc[4][4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        if (EPI != 2) {
            // the bias, loaded before the k loop (its latency hides there)
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = bias[nq * 4 + j];
        }
        const float* a = A + mq * 4;
        const float* b = Bm + nq * 4;
#pragma unroll 16
        for (int k = 0; k < K; ++k) {
            const float4 av = *reinterpret_cast<const float4*>(a + k * lda);
            const float4 bv = *reinterpret_cast<const float4*>(b + k * N);
            const float am[4] = {av.x, av.y, av.z, av.w};
            const float bn[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(am[i], bn[j], acc[i][j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = nq * 4 + j;
            float* o = out + n * ldo + mq * 4;
            float4 v;
            if (EPI == 2) {
                const float4 prev = *reinterpret_cast<const float4*>(o);
                v.x = prev.x > 0.f ? acc[0][j] : 0.f;
                v.y = prev.y > 0.f ? acc[1][j] : 0.f;
                v.z = prev.z > 0.f ? acc[2][j] : 0.f;
                v.w = prev.w > 0.f ? acc[3][j] : 0.f;
            } else {
                v.x = acc[0][j] + bb[j]; v.y = acc[1][j] + bb[j]; v.z = acc[2][j] + bb[j]; v.w = acc[3][j] + bb[j];
                if (EPI == 0) {
                    v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f);
                }
            }
            *reinterpret_cast<float4*>(o) = v;
        }
    }
}

__device__ __forceinline__ void acc_store(float* p, float v, bool first) { *p = first ? v : *p + v; }

// ---------------------------------------------------------------------------
// dW[n][k] (+)= sum_m Z[n][m] * A[k][m]   (reduction over the tile's samples)
// and db[n] (+)= sum_m Z[n][m], into global g (canonical [n][Kreal]) and gb;
// `first` stores, otherwise the tile's sums are added to what the run holds.
// A thread owns rows n = nq + NQ i and k = kq + KQ j (i, j < 4). A warp covers
// 8 k-groups x 4 n-groups, each group of four lanes 2 x 2 (two wavefronts per
// 16-byte load, as in gemm_fwd; eight consecutive A rows fall on distinct
// banks), and the run slot's rows are read and written as 32-byte pieces.
// The sample range is split SPLIT ways (interleaved quads) to fill the CTA;
// split partials are combined in a fixed order through smem. Without a split
// the accumulators start from the run's old values (loaded before the sample
// loop, which hides their latency). NT is the CTA size.
// ---------------------------------------------------------------------------
template <int N, int KP, int NT = NTHREADS>
__device__ __forceinline__ void gemm_dw(const float* __restrict__ Z, const float* __restrict__ A,
                                        int ld, int Mpad, float* red, float* __restrict__ g,
                                        int Kreal, float* __restrict__ gb, bool first) {
    constexpr int NQ = N / 4, KQ = KP / 4, T = NQ * KQ;
    constexpr int S0 = NT / T > 0 ? NT / T : 1;
    constexpr int S1 = RED_FLOATS / (N * KP) > 0 ? RED_FLOATS / (N * KP) : 1;
    constexpr int SPLIT0 = S0 < S1 ? S0 : S1;
    // the output layer (N = 4, few items) combines its partials by a chain of
    // SPLIT loads per element: at most 64 threads' worth of partials (measured
    // best at hidden 16 and 32: 16 and 8 parts instead of 64 and 32)
    constexpr int SPLIT = (N < 8 && T * SPLIT0 > 64) ? (64 / T > 0 ? 64 / T : 1) : SPLIT0;   // SPLIT == 1 never touches red
    static_assert(SPLIT >= 1 && (SPLIT == 1 || SPLIT * N * KP <= RED_FLOATS), "split scratch");
    constexpr int NB = (N * 8 + NT - 1) / NT;   // bias-gradient items per thread
    const int MQ = Mpad >> 2;
    // the bias slot's old values, loaded first (in flight during the GEMM)
    float bold[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int f = threadIdx.x + u * NT;
        bold[u] = (!first && f < N * 8 && (f & 7) == 0) ? gb[f >> 3] : 0.f;
    }
    for (int f = threadIdx.x; f < T * SPLIT; f += blockDim.x) {
        const int s = f / T, r = f % T;
        int kq, nq;
        if constexpr (KQ % 8 == 0 && NQ % 4 == 0) {
            // a warp: 8 k-groups x 4 n-groups, each group of four lanes 2 k x 2 n
            // (two wavefronts per 16-byte load; see gemm_fwd), the warp's eight
            // A rows on distinct banks
            const int rw = r >> 5, lane = r & 31, g = lane >> 2, t = lane & 3;
            kq = (rw % (KQ / 8)) * 8 + 2 * (g & 3) + (t & 1);
            nq = (rw / (KQ / 8)) * 4 + 2 * (g >> 2) + (t >> 1);
        } else {
            kq = r % KQ;
            nq = r / KQ;
        }
        float acc[4][4];
        if (SPLIT == 1 && !first) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = kq + KQ * j;
                    acc[i][j] = k < Kreal ? g[(nq + NQ * i) * Kreal + k] : 0.f;
                }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        }
#pragma unroll 2
        for (int q = s; q < MQ; q += SPLIT) {
            float4 z[4], a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) z[i] = *reinterpret_cast<const float4*>(Z + (nq + NQ * i) * ld + q * 4);
#pragma unroll
            for (int j = 0; j < 4; ++j) a[j] = *reinterpret_cast<const float4*>(A + (kq + KQ * j) * ld + q * 4);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float v = acc[i][j];
                    v = fmaf(z[i].x, a[j].x, v);
                    v = fmaf(z[i].y, a[j].y, v);
                    v = fmaf(z[i].z, a[j].z, v);
                    v = fmaf(z[i].w, a[j].w, v);
                    acc[i][j] = v;
                }
        }
        if (SPLIT == 1) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = kq + KQ * j;
                    if (k < Kreal) g[(nq + NQ * i) * Kreal + k] = acc[i][j];
                }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) red[(s * N + nq + NQ * i) * KP + kq + KQ * j] = acc[i][j];
        }
    }
    // bias gradient: 8 lanes per output row, combined by a fixed xor tree
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int f = threadIdx.x + u * NT;
        if (f >= N * 8) break;   // uniform per warp: N * 8 is a multiple of 32
        const int n = f >> 3, l = f & 7;
        float v = 0.f;
        for (int q = l; q < MQ; q += 8) {
            const float4 z = *reinterpret_cast<const float4*>(Z + n * ld + q * 4);
            v += (z.x + z.y) + (z.z + z.w);
        }
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if (l == 0) gb[n] = first ? v : bold[u] + v;
    }
    if (SPLIT > 1) {
        __syncthreads();
        // four elements per thread per pass: their old values load together
        constexpr int NE = N * KP;
        for (int e0 = threadIdx.x; e0 < NE; e0 += 4 * blockDim.x) {
            float v[4], old[4];
            int idx[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * blockDim.x;
                const int n = e / KP, k = e % KP;
                idx[u] = (e < NE && k < Kreal) ? n * Kreal + k : -1;
                old[u] = (!first && idx[u] >= 0) ? g[idx[u]] : 0.f;
                float s_ = 0.f;
                if (idx[u] >= 0) {
                    s_ = red[n * KP + k];
                    for (int s = 1; s < SPLIT; ++s) s_ += red[(s * N + n) * KP + k];
                }
                v[u] = s_;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (idx[u] >= 0) g[idx[u]] = v[u] + old[u];
        }
    }
}

// copy n floats global -> smem (both 16-byte aligned, n multiple of 4) with
// asynchronous 16-byte copies: every copy of the thread is in flight at once
// and no register holds the data. stage_issue only starts them (work that
// does not touch dst may run meanwhile); stage_wait waits for this thread's
// copies, and the barrier after it publishes them to the CTA.
__device__ __forceinline__ void stage_issue(float* dst, const float* __restrict__ src, int n) {
    const unsigned base = (unsigned)__cvta_generic_to_shared(dst);
    for (int i = threadIdx.x * 4; i < n; i += blockDim.x * 4)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + 4u * i), "l"(src + i) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void stage(float* dst, const float* __restrict__ src, int n) {
    stage_issue(dst, src, n);
    stage_wait();
}

// W1 [H][93] (canonical) -> smem [H][96] zero padded, for the encoding backward
template <int H>
__device__ __forceinline__ void stage_w1_rows(float* dst, const float* __restrict__ w1) {
    for (int i = threadIdx.x; i < H * DINP; i += blockDim.x) {
        const int n = i / DINP, k = i % DINP;
        dst[i] = k < DIN ? w1[n * DIN + k] : 0.f;
    }
}

// sin p and cos p. For |p| <= 2^17 (the encoding's arguments stay far below:
// |B x~| is a few thousand at most): Cody & Waite's additive range reduction,
// p = k pi/2 + r with pi/2 split in two floats (c1 = pi/2 rounded, c2 the
// rest; the fused multiply-adds take k c1 exactly, and the dropped tail
// |k| 1.8e-15 stays below 3e-10), |r| <= pi/4 (+1 ulp); then the Taylor
// series of sin to r^9 and cos to r^10 (truncation below 2e-9), and the
// quadrant k mod 4 picks and signs them. Its result agrees with sincosf to a
// few ulp; a dependent chain of about 20 operations instead of the library
// routine's longer one. sincos_fast holds for |p| <= SINCOS_FAST_MAX only;
// sincos_enc sends larger |p| to sincosf.
constexpr float SINCOS_FAST_MAX = 131072.f;
__device__ __forceinline__ void sincos_fast(float p, float* sp_, float* cp_) {
    const float k = rintf(p * 0.636619746685028076171875f);        // 2/pi
    float r = fmaf(-k, 1.57079637050628662109375f, p);            // c1
    r = fmaf(-k, -4.37113882867379300296306610107421875e-8f, r);  // c2
    const float r2 = r * r;
    float ps = fmaf(r2, 2.7557319223985893e-6f, -1.9841269841269841e-4f);   // 1/9!, -1/7!
    ps = fmaf(r2, ps, 8.3333333333333333e-3f);                               // 1/5!
    ps = fmaf(r2, ps, -1.6666666666666667e-1f);                              // -1/3!
    const float sn = fmaf(r * r2, ps, r);
    float pc = fmaf(r2, -2.7557319223985891e-7f, 2.4801587301587302e-5f);    // -1/10!, 1/8!
    pc = fmaf(r2, pc, -1.3888888888888889e-3f);                              // -1/6!
    pc = fmaf(r2, pc, 4.1666666666666667e-2f);                               // 1/4!
    pc = fmaf(r2, pc, -0.5f);                                                // -1/2!
    const float cs = fmaf(r2, pc, 1.f);
    const int q = (int)k & 3;
    const float s0 = (q & 1) ? cs : sn, c0 = (q & 1) ? sn : cs;
    *sp_ = (q & 2) ? -s0 : s0;
    *cp_ = ((q + 1) & 2) ? -c0 : c0;
}
__device__ __forceinline__ void sincos_enc(float p, float* sp_, float* cp_) {
    if (fabsf(p) > SINCOS_FAST_MAX) sincosf(p, sp_, cp_);
    else sincos_fast(p, sp_, cp_);
}

// Gaussian encoding of the tile's points: rows 0..2 of g hold x~ on entry;
// rows 3..47 get sin(B x~), rows 48..92 cos(B x~), rows 93..95 zero.
// Item f = j Mpad + m is stepped by the CTA size without a division per item.
// A thread takes ENC_ITEMS items per pass: their loads first, then their
// sincos chains side by side, then their stores (the stores may alias the
// next pass's loads as far as the compiler knows, so within a pass is where
// the chains can overlap). Items past the last one compute a dummy and store
// nothing.
constexpr int ENC_ITEMS = 4;
template <int LD>
__device__ __forceinline__ void encode(const StepParams& sp, float* g, int Mpad) {
    if (Mpad <= 0) return;
    const int dq = blockDim.x / Mpad, dr = blockDim.x - dq * Mpad;
    int j = threadIdx.x / Mpad, m = threadIdx.x - j * Mpad;
    while (j < NF) {
        int jj[ENC_ITEMS], mm[ENC_ITEMS];
#pragma unroll
        for (int u = 0; u < ENC_ITEMS; ++u) {
            jj[u] = j;
            mm[u] = m;
            j += dq;
            m += dr;
            if (m >= Mpad) {
                m -= Mpad;
                ++j;
            }
        }
        float p[ENC_ITEMS], sn[ENC_ITEMS], cs[ENC_ITEMS];
#pragma unroll
        for (int u = 0; u < ENC_ITEMS; ++u) {
            const int jc = min(jj[u], NF - 1);
            p[u] = fmaf(sp.B[3 * jc + 2], g[2 * LD + mm[u]],
                        fmaf(sp.B[3 * jc + 1], g[1 * LD + mm[u]], sp.B[3 * jc] * g[0 * LD + mm[u]]));
        }
#pragma unroll
        for (int u = 0; u < ENC_ITEMS; ++u) sincos_fast(p[u], &sn[u], &cs[u]);
#pragma unroll
        for (int u = 0; u < ENC_ITEMS; ++u)
            if (fabsf(p[u]) > SINCOS_FAST_MAX) sincosf(p[u], &sn[u], &cs[u]);
#pragma unroll
        for (int u = 0; u < ENC_ITEMS; ++u)
            if (jj[u] < NF) {
                g[(3 + jj[u]) * LD + mm[u]] = sn[u];
                g[(3 + NF + jj[u]) * LD + mm[u]] = cs[u];
            }
    }
    for (int i = threadIdx.x; i < 3 * Mpad; i += blockDim.x) g[(DIN + i / Mpad) * LD + (i % Mpad)] = 0.f;
}

struct TileArgs {
    const ObjDev* objs;
    const ObjBatch* obs;
    const TileDev* tiles;     // this class's tiles
    const int* n_tiles;       // device count of this class's tiles
    const float* pool;        // ray source: pool arena, the batch staging buffer, or
                              // (MODE_EVAL) the caller's rays
    const int* pick;          // batch ray -> source index
    const float* tbuf;        // batch sample depths
    const float* params;      // canonical parameter arena
    const float* wt;          // transposed-weight arena
    float* part;              // run partial slots
    float* eval_out;          // MODE_EVAL: rendered depth per ray, or NULL
    float* eval_rec;          // MODE_EVAL: [n][5] (O^, D^, C^) per ray, or NULL
    float* ray_grad;          // MODE_GRAD_CENTER: [batch rays][6] dL/do, dL/dd per ray, or NULL
    float eval_half[3];       // MODE_EVAL: box half extents
    int eval_obj;             // MODE_EVAL / MODE_QUERY: the object
    long long eval_n;         // MODE_EVAL: rays; MODE_QUERY: points
    int eval_S;               // MODE_EVAL: samples per ray
    const float* qpts;        // MODE_QUERY: points [n][3]
    float* qocc;              // MODE_QUERY: occupancy [n]
    float* qrgb;              // MODE_QUERY: colour [n][3] or NULL
    int* dyn;                 // [2]: next tile, CTAs done (dynamic scheduling), or NULL
    const int* dyn_on;        // builder: non-zero when this step schedules the class dynamically
    float* enc_scratch;       // [grid][DINP * LD] (widths whose encoding shares the hidden rows): the
                              // encoding is saved there for the layer-1 weight gradient, or NULL
                              // (recomputed)
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Render one ray per warp (lane i = sample i, S <= 32): forward Eq. 3, the
// ray's loss terms, and (GRAD) dL/dy for its samples. The exclusive product
// P_i = prod_{j<i}(1 - o_j) is a multiplicative scan; the reverse recursion
// S_i = o_i g_i + (1 - o_i) S_{i+1} is a suffix scan of affine maps
// x -> (1 - o_i) x + o_i g_i (no division by 1 - o_i anywhere). With ACT the
// four outputs in yb already went through the sigmoid.
// With dyt (GRAD only), dL/dy of sample m goes, as 8 BF16 values (the 4
// outputs' gradients, then 4 zeros), to row m at column dc0 of that
// core-matrix tile with dcc columns, instead of back into yb.
template <bool GRAD, int LD, bool ACT = false>
__device__ __forceinline__ void render_ray_warp(const StepParams& sp, float* yb, const float* tsm,
                                                float* d, int r, int S, float invR,
                                                unsigned char* dyt = nullptr, int dcc = 0, int dc0 = 0) {
    const int i = threadIdx.x & 31;
    const bool v = i < S;
    const int m = r * S + i;
    float o = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, t = 0.f;
    if (v) {
        o = yb[m];
        c0 = yb[LD + m];
        c1 = yb[2 * LD + m];
        c2 = yb[3 * LD + m];
        if (!ACT) {
            o = sigmoidf_(o);
            c0 = sigmoidf_(c0);
            c1 = sigmoidf_(c1);
            c2 = sigmoidf_(c2);
        }
        t = tsm[m];
    }
    float incl = v ? 1.f - o : 1.f;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const float u = __shfl_up_sync(0xffffffffu, incl, s);
        if (i >= s) incl *= u;
    }
    float P = __shfl_up_sync(0xffffffffu, incl, 1);
    if (i == 0) P = 1.f;
    const float T = o * P;
    const float Oh = warp_sum(T), Dh = warp_sum(T * t);
    const float C0 = warp_sum(T * c0), C1 = warp_sum(T * c1), C2 = warp_sum(T * c2);
    const float D = d[6], Msk = d[10];
    const float wD = D > 0.f ? Msk : 0.f;
    const float eD = Dh - D, e0 = C0 - d[7], e1 = C1 - d[8], e2 = C2 - d[9], eO = Oh - Msk;
    if (i == 0) {
        d[13] = wD * fabsf(eD);
        d[14] = Msk * ((fabsf(e0) + fabsf(e1)) + fabsf(e2));
        d[15] = fabsf(eO);
    }
    if (!GRAD) return;
    const float a = wD * signf_(eD) * invR;
    const float bsc = sp.lam_c * Msk * invR / 3.f;
    const float b0 = bsc * signf_(e0), b1 = bsc * signf_(e1), b2 = bsc * signf_(e2);
    const float e = sp.lam_o * signf_(eO) * invR;
    const float gi = fmaf(a, t, fmaf(b0, c0, fmaf(b1, c1, b2 * c2))) + e;
    float al = v ? 1.f - o : 1.f, be = v ? o * gi : 0.f;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const float a2 = __shfl_down_sync(0xffffffffu, al, s);
        const float b2_ = __shfl_down_sync(0xffffffffu, be, s);
        if (i + s < 32) {
            be = fmaf(al, b2_, be);
            al = al * a2;
        }
    }
    float Sn = __shfl_down_sync(0xffffffffu, be, 1);
    if (i == 31) Sn = 0.f;
    if (v) {
        const float dLdo = P * (gi - Sn);
        const float g0 = dLdo * o * (1.f - o);
        const float g1 = T * b0 * c0 * (1.f - c0);
        const float g2 = T * b1 * c1 * (1.f - c1);
        const float g3 = T * b2 * c2 * (1.f - c2);
        if (dyt) {
            const __nv_bfloat162 p01 = __floats2bfloat162_rn(g0, g1), p23 = __floats2bfloat162_rn(g2, g3);
            uint4 u;
            u.x = *reinterpret_cast<const uint32_t*>(&p01);
            u.y = *reinterpret_cast<const uint32_t*>(&p23);
            u.z = 0u;
            u.w = 0u;
            *reinterpret_cast<uint4*>(dyt + (((m >> 3) * (dcc >> 3) + (dc0 >> 3)) * 128 + (m & 7) * 16)) = u;
        } else {
            yb[m] = g0;
            yb[LD + m] = g1;
            yb[2 * LD + m] = g2;
            yb[3 * LD + m] = g3;
        }
    }
}

template <int H, int MODE>
__global__ void __launch_bounds__(TileCfg<H>::THREADS, TileCfg<H>::CTAS) k_tile_fp32(StepParams sp, TileArgs ta) {
    using SM = TileSmem<H>;
    constexpr int LD = SM::LD;
    constexpr bool TRAINISH = MODE == MODE_TRAIN || MODE == MODE_FORWARD || MODE == MODE_GRAD_CENTER;
    constexpr bool GRAD = MODE == MODE_TRAIN || MODE == MODE_GRAD_CENTER;
    extern __shared__ __align__(16) float smem[];
    float* act = smem + SM::ACT;
    float* g = smem + SM::G;
    float* yb = smem + SM::Y;
    float* ws = smem + SM::W;
    float* ws2 = smem + SM::W2;
    float* red = smem + SM::RED;
    float* tsm = smem + SM::TS;
    float* rays = smem + SM::RAYS;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    __shared__ long long s_tile;
    long long t0, t1;
    bool dyn = false;
    if (TRAINISH) {
        const long long n = *ta.n_tiles;
        dyn = ta.dyn != nullptr && *ta.dyn_on != 0;
        t0 = dyn ? 0 : (long long)blockIdx.x * n / gridDim.x;
        t1 = dyn ? n : (long long)(blockIdx.x + 1) * n / gridDim.x;
    } else {
        t0 = blockIdx.x;
        t1 = t0 + 1;
    }
    // a width class launched behind this one may start on the SMs it leaves
    pdl_launch_dependents();
#pragma unroll 1
    for (long long it = t0;; ++it) {
        long long tl = it;
        if (dyn) {
            // every thread read the previous tile index before the barrier that
            // ended the previous tile
            if (threadIdx.x == 0) s_tile = atomicAdd(ta.dyn, 1);
            __syncthreads();
            tl = s_tile;
        }
        if (tl >= t1) break;
        // ---- the tile -----------------------------------------------------
        int k, nr, S;
        long long sbase = 0, part = 0, ray_first;
        bool first = true;
        if (MODE == MODE_EVAL || MODE == MODE_QUERY) {
            k = ta.eval_obj;
            S = MODE == MODE_EVAL ? ta.eval_S : 1;
            const int rt = MODE == MODE_EVAL ? min(RTMAX, SM::MMAX / S) : SM::MMAX;
            ray_first = tl * rt;
            nr = (int)min((long long)rt, ta.eval_n - ray_first);
        } else {
            const TileDev td = ta.tiles[tl];
            k = td.obj;
            nr = td.nr;
            ray_first = td.ray0;
            part = td.part;
            S = ta.objs[k].S;
            sbase = ta.obs[k].sample_off + (long long)(td.ray0 - ta.obs[k].ray_off) * S;
            first = dyn || tl == t0 || ta.tiles[tl - 1].obj != k;
        }
        const ObjDev& ob = ta.objs[k];
        const int M = nr * S;
        const int Mpad = (M + 7) & ~7;
        const float* P = ta.params + ob.param_off;
        const float* WT = ta.wt + ob.wt_off;
        const float cx = ob.c[0], cy = ob.c[1], cz = ob.c[2], sc = ob.scale;

        // ---- rays into smem -----------------------------------------------
        if (MODE != MODE_QUERY) {
            for (int r = threadIdx.x; r < nr; r += blockDim.x) {
                const float* rec;
                if (MODE == MODE_EVAL) rec = ta.pool + (ray_first + r) * REC;
                else rec = ta.pool + (ta.obs[k].src_off + ta.pick[ray_first + r]) * REC;
                float* d = rays + r * RAYF;
#pragma unroll
                for (int q = 0; q < 11; ++q) d[q] = rec[q];
                if (MODE == MODE_EVAL) {
                    // ray-box entry / exit (slab method) against c_k +- half
                    float tn = 0.f, tf = 3.0e38f;
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        const float o = d[ax], dir = d[3 + ax];
                        const float lo = ob.c[ax] - ta.eval_half[ax], hi = ob.c[ax] + ta.eval_half[ax];
                        if (dir != 0.f) {
                            const float u1 = (lo - o) / dir, u2 = (hi - o) / dir;
                            tn = fmaxf(tn, fminf(u1, u2));
                            tf = fminf(tf, fmaxf(u1, u2));
                        } else if (o < lo || o > hi) {
                            tf = -1.f;
                        }
                    }
                    d[11] = tn;
                    d[12] = tf;
                }
            }
            if (MODE == MODE_EVAL) {
                // a tile whose rays all miss the box renders zeros without the MLP
                // (ray r's entry/exit were written by thread r itself)
                const int r = threadIdx.x;
                const bool any =
                    __syncthreads_or(r < nr && rays[r * RAYF + 12] > rays[r * RAYF + 11] && rays[r * RAYF + 12] > 0.f);
                if (!any) {
                    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
                        if (ta.eval_out) ta.eval_out[ray_first + r] = 0.f;
                        if (ta.eval_rec)
                            for (int q = 0; q < 5; ++q) ta.eval_rec[(ray_first + r) * 5 + q] = 0.f;
                    }
                    continue;
                }
            } else {
                __syncthreads();
            }
        }

        // ---- points x~ = (o + t d - c) / s ----------------------------------
        for (int m = threadIdx.x; m < Mpad; m += blockDim.x) {
            float x0 = 0.f, x1 = 0.f, x2 = 0.f, t = 0.f;
            if (m < M) {
                if (MODE == MODE_QUERY) {
                    const float* q = ta.qpts + (ray_first + m) * 3;
                    x0 = (q[0] - cx) / sc;
                    x1 = (q[1] - cy) / sc;
                    x2 = (q[2] - cz) / sc;
                } else {
                    const int r = m / S, i = m - r * S;
                    const float* d = rays + r * RAYF;
                    if (MODE == MODE_EVAL) t = d[11] + ((float)i + 0.5f) / (float)S * (d[12] - d[11]);
                    else t = ta.tbuf[sbase + m];
                    x0 = (fmaf(t, d[3], d[0]) - cx) / sc;
                    x1 = (fmaf(t, d[4], d[1]) - cy) / sc;
                    x2 = (fmaf(t, d[5], d[2]) - cz) / sc;
                }
            }
            tsm[m] = t;
            g[0 * LD + m] = x0;
            g[1 * LD + m] = x1;
            g[2 * LD + m] = x2;
        }
        stage_issue(ws, WT + wt_layer_off(H, 0), DINP * H);   // W1^T [96][H], during the encoding
        if (SM::WDB) stage_issue(ws2, WT + wt_layer_off(H, 1), H * H);   // W2^T
        __syncthreads();
        encode<LD>(sp, g, Mpad);
        stage_wait();
        __syncthreads();
        // hidden layers 2-4 overwrite the encoding: keep a copy for the layer-1 weight gradient
        float* const enc_save = (!SM::GSEP && GRAD && ta.enc_scratch)
                                    ? ta.enc_scratch + (long long)blockIdx.x * (DINP * LD) : nullptr;
        if (enc_save)
            for (int i = threadIdx.x * 4; i < DINP * LD; i += blockDim.x * 4)
                *reinterpret_cast<float4*>(enc_save + i) = *reinterpret_cast<const float4*>(g + i);

        // ---- forward --------------------------------------------------------
        gemm_fwd<H, DINP, 0>(g, LD, ws, P + b_off(H, 0), act, LD, Mpad);
        __syncthreads();
        if (SM::WDB) {
            // layer l reads W_{l+1}^T from ws2 (l odd) or ws (l even); the layer
            // after it's weights go to the other buffer, which the previous GEMM
            // read (free since the barrier after it), and arrive during this GEMM
#pragma unroll 1
            for (int l = 1; l < 4; ++l) {
                float* const wcur = (l & 1) ? ws2 : ws;
                float* const wnext = (l & 1) ? ws : ws2;
                if (l < 3) stage_issue(wnext, WT + wt_layer_off(H, l + 1), H * H);
                else stage_issue(wnext, WT + wt_layer_off(H, 4), H * NOUT);
                gemm_fwd<H, H, 0>(act + (l - 1) * H * LD, LD, wcur, P + b_off(H, l), act + l * H * LD, LD, Mpad);
                stage_wait();
                __syncthreads();
            }
        } else {
#pragma unroll 1
            for (int l = 1; l < 4; ++l) {
                stage(ws, WT + wt_layer_off(H, l), H * H);
                __syncthreads();
                gemm_fwd<H, H, 0>(act + (l - 1) * H * LD, LD, ws, P + b_off(H, l), act + l * H * LD, LD, Mpad);
                __syncthreads();
            }
            stage(ws, WT + wt_layer_off(H, 4), H * NOUT);
            __syncthreads();
        }
        // W5^T [H][4] is in ws either way
        gemm_fwd<NOUT, H, 1>(act + 3 * H * LD, LD, ws, P + b_off(H, 4), yb, LD, Mpad);
        __syncthreads();
        if (MODE == MODE_QUERY) {
            for (int m = threadIdx.x; m < M; m += blockDim.x) {
                const long long q = ray_first + m;
                ta.qocc[q] = sigmoidf_(yb[m]);
                if (ta.qrgb) {
                    ta.qrgb[3 * q + 0] = sigmoidf_(yb[LD + m]);
                    ta.qrgb[3 * q + 1] = sigmoidf_(yb[2 * LD + m]);
                    ta.qrgb[3 * q + 2] = sigmoidf_(yb[3 * LD + m]);
                }
            }
            continue;
        }

        // ---- rendering (Eq. 3), losses (Eq. 4-5) and their gradient -----------
        if (MODE == MODE_EVAL) {
            // S may exceed 32 here: one thread per ray, sequential
            if (threadIdx.x < nr) {
                const int r = threadIdx.x;
                const float* d = rays + r * RAYF;
                float Pr = 1.f, Dh = 0.f, Oh = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
                for (int i = 0; i < S; ++i) {
                    const int m = r * S + i;
                    const float o = sigmoidf_(yb[m]);
                    const float T = o * Pr;
                    Dh = fmaf(T, tsm[m], Dh);
                    Oh += T;
                    if (ta.eval_rec) {
                        C0 = fmaf(T, sigmoidf_(yb[LD + m]), C0);
                        C1 = fmaf(T, sigmoidf_(yb[2 * LD + m]), C1);
                        C2 = fmaf(T, sigmoidf_(yb[3 * LD + m]), C2);
                    }
                    Pr = Pr * (1.f - o);
                }
                const bool hit = d[12] > d[11] && d[12] > 0.f;
                if (ta.eval_out) ta.eval_out[ray_first + r] = hit ? Dh : 0.f;
                if (ta.eval_rec) {
                    float* e = ta.eval_rec + (ray_first + r) * 5;
                    e[0] = hit ? Oh : 0.f;
                    e[1] = hit ? Dh : 0.f;
                    e[2] = hit ? C0 : 0.f;
                    e[3] = hit ? C1 : 0.f;
                    e[4] = hit ? C2 : 0.f;
                }
            }
            continue;
        }
        const float invR = 1.f / (float)ta.obs[k].R;
        for (int r = warp; r < nr; r += nwarps)
            render_ray_warp<GRAD, LD>(sp, yb, tsm, rays + r * RAYF, r, S, invR);
        // padded samples carry no gradient
        for (int m = M + threadIdx.x; m < Mpad; m += blockDim.x) {
            yb[m] = 0.f; yb[LD + m] = 0.f; yb[2 * LD + m] = 0.f; yb[3 * LD + m] = 0.f;
        }
        __syncthreads();
        float* gp = ta.part + part;   // this run's slot
        constexpr long long PC = param_count(H);
        if (threadIdx.x == 0) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            for (int r = 0; r < nr; ++r) {
                s0 += rays[r * RAYF + 13]; s1 += rays[r * RAYF + 14]; s2 += rays[r * RAYF + 15];
            }
            acc_store(gp + PC + 0, s0, first);
            acc_store(gp + PC + 1, s1, first);
            acc_store(gp + PC + 2, s2, first);
            if (first) { gp[PC + 3] = 0.f; gp[PC + 4] = 0.f; gp[PC + 5] = 0.f; }
        }
        if (MODE == MODE_FORWARD) {
            __syncthreads();
            continue;
        }

        // ---- backward -------------------------------------------------------
        // layer 5: dW5 = dY^T h4, dZ4 = (dY W5) * [h4 > 0]
        stage_issue(ws, P + w_off(H, 4), NOUT * H);     // W5 [4][H] == B[k=out][n=in]
        gemm_dw<NOUT, H, TileCfg<H>::THREADS>(yb, act + 3 * H * LD, LD, Mpad, red, gp + w_off(H, 4), H,
                                             gp + b_off(H, 4), first);
        stage_wait();
        __syncthreads();
        gemm_fwd<H, NOUT, 2>(yb, LD, ws, nullptr, act + 3 * H * LD, LD, Mpad);
        __syncthreads();
#pragma unroll 1
        for (int l = 3; l >= 1; --l) {
            // dW_{l+1} = dZ_{l+1}^T h_l ; dZ_l = (dZ_{l+1} W_{l+1}) * [h_l > 0]
            float* hz = act + l * H * LD;
            float* ha = act + (l - 1) * H * LD;
            stage_issue(ws, P + w_off(H, l), H * H);
            gemm_dw<H, H, TileCfg<H>::THREADS>(hz, ha, LD, Mpad, red, gp + w_off(H, l), H, gp + b_off(H, l), first);
            stage_wait();
            __syncthreads();
            gemm_fwd<H, H, 2>(hz, LD, ws, nullptr, ha, LD, Mpad);
            __syncthreads();
        }
        if (enc_save) {
            // the encoding was overwritten by hidden layers 2-4: copy it back (this
            // CTA's own stores, ordered before by the barriers since)
            stage(g, enc_save, DINP * LD);
            __syncthreads();
        } else if (!SM::GSEP) {
            // the encoding was overwritten by hidden layers 2-4: recompute it
            for (int m = threadIdx.x; m < Mpad; m += blockDim.x) {
                float x0 = 0.f, x1 = 0.f, x2 = 0.f;
                if (m < M) {
                    const int r = m / S;
                    const float* d = rays + r * RAYF;
                    const float t = tsm[m];
                    x0 = (fmaf(t, d[3], d[0]) - cx) / sc;
                    x1 = (fmaf(t, d[4], d[1]) - cy) / sc;
                    x2 = (fmaf(t, d[5], d[2]) - cz) / sc;
                }
                g[0 * LD + m] = x0;
                g[1 * LD + m] = x1;
                g[2 * LD + m] = x2;
            }
            __syncthreads();
            encode<LD>(sp, g, Mpad);
            __syncthreads();
        }
        // layer 1: dW1 = dZ1^T gamma
        gemm_dw<H, DINP, TileCfg<H>::THREADS>(act, g, LD, Mpad, red, gp + w_off(H, 0), DIN, gp + b_off(H, 0), first);
        if (MODE == MODE_GRAD_CENTER) {
            // encoding backward, one thread per sample:
            //   dgamma_j = sum_n dZ1[n] W1[n][j]
            //   dx~ = dgamma_xyz + sum_j B_j (cos_j dgamma_sin_j - sin_j dgamma_cos_j)
            //   dL/dc = -sum_samples dx~ / s
            __syncthreads();
            stage_w1_rows<H>(ws, P + w_off(H, 0));
            __syncthreads();
            float* acc3 = yb;  // [3][LD], free after the layer-5 backward
            for (int m = threadIdx.x; m < Mpad; m += blockDim.x) {
                float d0 = 0.f, d1 = 0.f, d2 = 0.f;
                if (m < M) {
                    for (int n = 0; n < H; ++n) {
                        const float z = act[n * LD + m];
                        d0 = fmaf(z, ws[n * DINP + 0], d0);
                        d1 = fmaf(z, ws[n * DINP + 1], d1);
                        d2 = fmaf(z, ws[n * DINP + 2], d2);
                    }
                    for (int j = 0; j < NF; ++j) {
                        float ds = 0.f, dc = 0.f;
                        for (int n = 0; n < H; ++n) {
                            const float z = act[n * LD + m];
                            ds = fmaf(z, ws[n * DINP + 3 + j], ds);
                            dc = fmaf(z, ws[n * DINP + 3 + NF + j], dc);
                        }
                        const float w = ds * g[(3 + NF + j) * LD + m] - dc * g[(3 + j) * LD + m];
                        d0 = fmaf(w, sp.B[3 * j], d0);
                        d1 = fmaf(w, sp.B[3 * j + 1], d1);
                        d2 = fmaf(w, sp.B[3 * j + 2], d2);
                    }
                }
                acc3[m] = d0; acc3[LD + m] = d1; acc3[2 * LD + m] = d2;
            }
            __syncthreads();
            if (threadIdx.x < 3) {
                float s = 0.f;
                for (int m = 0; m < M; ++m) s += acc3[threadIdx.x * LD + m];
                gp[PC + 3 + threadIdx.x] += -s / sc;
            }
            // per ray through x = o + t d (depths fixed): dL/do = sum dL/dx, dL/dd = sum t dL/dx
            if (ta.ray_grad) {
                for (int r = threadIdx.x; r < nr; r += blockDim.x) {
                    float go[3] = {0.f, 0.f, 0.f}, gd[3] = {0.f, 0.f, 0.f};
                    for (int i = 0; i < S; ++i) {
                        const int m = r * S + i;
                        const float t = tsm[m];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const float v = acc3[a * LD + m] / sc;
                            go[a] += v;
                            gd[a] = fmaf(t, v, gd[a]);
                        }
                    }
                    float* out = ta.ray_grad + (long long)(ray_first + r) * 6;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        out[a] = go[a];
                        out[3 + a] = gd[a];
                    }
                }
            }
        }
        __syncthreads();
    }
    if (dyn && threadIdx.x == 0 && atomicAdd(ta.dyn + 1, 1) == (int)gridDim.x - 1) {
        // every CTA has taken its last tile: reset the counter for the next launch
        ta.dyn[0] = 0;
        ta.dyn[1] = 0;
    }
    // launched behind another width class's tile kernel (programmatic stream
    // serialization, no wait at the start): complete only after it
    pdl_wait();
}

}  // namespace vmapk
