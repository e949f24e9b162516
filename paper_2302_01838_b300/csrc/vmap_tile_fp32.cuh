// Fused per-tile FP32 training kernel: encoding, MLP forward, occupancy
// rendering, losses, backward through rendering / MLP / encoding.
//
// One CTA processes a tile of whole rays of one object (so the per-ray scans
// of Eq. 3 stay inside the CTA). Activations live in shared memory in
// feature-major layout [feature][sample] with a row stride LD = Mpad + 4
// (LD = 4 mod 8, so eight rows read at the same sample column hit distinct
// banks). Each layer is a shared-memory SIMT GEMM with 4x4 register tiles.
// The CTA writes the tile's weight gradient and loss sums to its own slot of
// the partial buffer; the reduce/Adam kernel adds the slots of an object in a
// fixed order (bitwise reproducible).
#pragma once
#include "vmap_common.cuh"

namespace vmapk {

enum TileMode { MODE_TRAIN = 0, MODE_FORWARD = 1, MODE_GRAD_CENTER = 2, MODE_EVAL = 3, MODE_QUERY = 4 };

template <int H> struct TileCfg;
template <> struct TileCfg<16>  { static constexpr int MMAX = 240; };
template <> struct TileCfg<32>  { static constexpr int MMAX = 176; };
template <> struct TileCfg<64>  { static constexpr int MMAX = 112; };
template <> struct TileCfg<128> { static constexpr int MMAX = 48; };

constexpr int RED_FLOATS = 4096;   // split-reduction scratch
constexpr int RAYF = 16;           // floats of per-ray scratch

template <int H> struct TileSmem {
    static constexpr int MMAX = TileCfg<H>::MMAX;
    static constexpr int LD = MMAX + 4;
    static constexpr int RTMAX = MMAX;      // at most one sample per ray
    static constexpr int WS = (DINP * H > H * H ? DINP * H : H * H);
    static constexpr int G = 0;                                  // [96][LD] encoding
    static constexpr int ACT = G + DINP * LD;                    // [4][H][LD] hidden activations
    static constexpr int Y = ACT + 4 * H * LD;                   // [4][LD] outputs / their grads
    static constexpr int W = Y + 4 * LD;                         // weight staging
    static constexpr int RED = W + WS;                           // split reduction scratch
    static constexpr int PS = RED + RED_FLOATS;                  // [LD] prod_{j<i}(1-o_j)
    static constexpr int TS = PS + LD;                           // [LD] sample depths t
    static constexpr int RAYS = TS + LD;                         // [RTMAX][RAYF]
    static constexpr int TOTAL = RAYS + RTMAX * RAYF;
    static constexpr size_t BYTES = (size_t)TOTAL * sizeof(float);
};

// ---------------------------------------------------------------------------
// out[n][m] = epi( sum_k A[k][m] * Bm[k][n] ),  m < Mpad, n < N.
// A: [K][lda] in smem, Bm: [K][N] dense in smem.
// EPI 0: + bias, ReLU;  EPI 1: + bias;  EPI 2: * (out[n][m] > 0), in place;
// EPI 3: plain store.
// A warp covers 8 sample quads x 4 output quads: its A loads touch 128
// consecutive bytes and its B loads 64, one wavefront each.
// ---------------------------------------------------------------------------
template <int N, int K, int EPI>
__device__ __forceinline__ void gemm_fwd(const float* __restrict__ A, int lda,
                                         const float* __restrict__ Bm,
                                         const float* __restrict__ bias, float* out, int ldo,
                                         int Mpad) {
    constexpr int NQ = N / 4;
    const int MQ = Mpad >> 2;
    const int items = ((MQ + 7) >> 3) * 8 * NQ;
    for (int f = threadIdx.x; f < items; f += blockDim.x) {
        const int mq = (f / (8 * NQ)) * 8 + (f & 7);
        const int nq = (f >> 3) % NQ;
        if (mq >= MQ) continue;
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        const float* a = A + mq * 4;
        const float* b = Bm + nq * 4;
#pragma unroll 8
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
            } else if (EPI == 3) {
                v.x = acc[0][j]; v.y = acc[1][j]; v.z = acc[2][j]; v.w = acc[3][j];
            } else {
                const float bb = bias[n];
                v.x = acc[0][j] + bb; v.y = acc[1][j] + bb; v.z = acc[2][j] + bb; v.w = acc[3][j] + bb;
                if (EPI == 0) {
                    v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f);
                }
            }
            *reinterpret_cast<float4*>(o) = v;
        }
    }
}

// ---------------------------------------------------------------------------
// dW[n][k] = sum_m Z[n][m] * A[k][m]   (reduction over the tile's samples)
// and db[n] = sum_m Z[n][m]. Written to global g (canonical [n][Kreal]) and gb.
// The sample range is split SPLIT ways (interleaved quads) to fill the CTA;
// split partials are combined in a fixed order through smem.
// ---------------------------------------------------------------------------
template <int N, int KP>
__device__ __forceinline__ void gemm_dw(const float* __restrict__ Z, const float* __restrict__ A,
                                        int ld, int Mpad, float* red, float* __restrict__ g,
                                        int Kreal, float* __restrict__ gb) {
    constexpr int NQ = N / 4, KQ = KP / 4, T = NQ * KQ;
    constexpr int S0 = NTHREADS / T > 0 ? NTHREADS / T : 1;
    constexpr int S1 = RED_FLOATS / (N * KP) > 0 ? RED_FLOATS / (N * KP) : 1;
    constexpr int SPLIT = S0 < S1 ? S0 : S1;   // SPLIT == 1 never touches red
    static_assert(SPLIT >= 1 && (SPLIT == 1 || SPLIT * N * KP <= RED_FLOATS), "split scratch");
    const int MQ = Mpad >> 2;
    for (int f = threadIdx.x; f < T * SPLIT; f += blockDim.x) {
        const int s = f / T, r = f % T;
        const int nq = r % NQ, kq = r / NQ;
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int q = s; q < MQ; q += SPLIT) {
            float4 z[4], a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) z[i] = *reinterpret_cast<const float4*>(Z + (nq * 4 + i) * ld + q * 4);
#pragma unroll
            for (int j = 0; j < 4; ++j) a[j] = *reinterpret_cast<const float4*>(A + (kq * 4 + j) * ld + q * 4);
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
                    const int k = kq * 4 + j;
                    if (k < Kreal) g[(nq * 4 + i) * Kreal + k] = acc[i][j];
                }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) red[(s * N + nq * 4 + i) * KP + kq * 4 + j] = acc[i][j];
        }
    }
    // bias gradient: 8 lanes per output row, combined by a fixed xor tree
    for (int f = threadIdx.x; f < N * 8; f += blockDim.x) {
        const int n = f >> 3, l = f & 7;
        float v = 0.f;
        for (int q = l; q < MQ; q += 8) {
            const float4 z = *reinterpret_cast<const float4*>(Z + n * ld + q * 4);
            v += (z.x + z.y) + (z.z + z.w);
        }
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if (l == 0) gb[n] = v;
    }
    if (SPLIT > 1) {
        __syncthreads();
        for (int e = threadIdx.x; e < N * KP; e += blockDim.x) {
            const int n = e / KP, k = e % KP;
            if (k >= Kreal) continue;
            float v = red[n * KP + k];
            for (int s = 1; s < SPLIT; ++s) v += red[(s * N + n) * KP + k];
            g[n * Kreal + k] = v;
        }
    }
}

// copy n floats global -> smem (both 16-byte aligned, n multiple of 4)
__device__ __forceinline__ void stage(float* dst, const float* __restrict__ src, int n) {
    for (int i = threadIdx.x * 4; i < n; i += blockDim.x * 4)
        *reinterpret_cast<float4*>(dst + i) = *reinterpret_cast<const float4*>(src + i);
}

// W1 [H][93] (canonical) -> smem [H][96] zero padded, for the encoding backward
template <int H>
__device__ __forceinline__ void stage_w1_rows(float* dst, const float* __restrict__ w1) {
    for (int i = threadIdx.x; i < H * DINP; i += blockDim.x) {
        const int n = i / DINP, k = i % DINP;
        dst[i] = k < DIN ? w1[n * DIN + k] : 0.f;
    }
}

struct TileArgs {
    const ObjDev* objs;
    const TileDev* tiles;
    int tile_begin;
    const float* pool;        // ray source: pool arena, the batch staging buffer, or
                              // (MODE_EVAL) the caller's rays
    const int* pick;          // batch ray -> pool index (NULL in MODE_EVAL)
    const float* tbuf;        // batch sample depths
    const float* params;      // canonical parameter arena
    const float* wt;          // transposed-weight arena
    float* part;              // per-tile partials
    float* eval_out;          // MODE_EVAL: rendered depth per ray
    float eval_half[3];       // MODE_EVAL: box half extents
    int eval_obj;             // MODE_EVAL / MODE_QUERY: the object
    long long eval_n;         // MODE_EVAL: rays; MODE_QUERY: points
    int eval_S;               // MODE_EVAL: samples per ray
    const float* qpts;        // MODE_QUERY: points [n][3]
    float* qocc;              // MODE_QUERY: occupancy [n]
    float* qrgb;              // MODE_QUERY: colour [n][3] or NULL
};

template <int H, int MODE>
__global__ void __launch_bounds__(NTHREADS, 1) k_tile_fp32(StepParams sp, TileArgs ta) {
    using SM = TileSmem<H>;
    constexpr int LD = SM::LD;
    extern __shared__ __align__(16) float smem[];
    float* g = smem + SM::G;
    float* act = smem + SM::ACT;
    float* yb = smem + SM::Y;
    float* ws = smem + SM::W;
    float* red = smem + SM::RED;
    float* ps = smem + SM::PS;
    float* tsm = smem + SM::TS;
    float* rays = smem + SM::RAYS;

    // ---- the tile ---------------------------------------------------------
    int k, nr, S;
    long long sbase = 0, part = 0;
    long long ray_first;
    if (MODE == MODE_EVAL || MODE == MODE_QUERY) {
        k = ta.eval_obj;
        S = MODE == MODE_EVAL ? ta.eval_S : 1;
        const int rt = SM::MMAX / S;
        ray_first = (long long)blockIdx.x * rt;
        nr = (int)min((long long)rt, ta.eval_n - ray_first);
    } else {
        const TileDev td = ta.tiles[ta.tile_begin + blockIdx.x];
        k = td.obj;
        nr = td.nr;
        ray_first = td.ray0;
        part = td.part;
        S = ta.objs[k].S;
        sbase = ta.objs[k].sample_off + (long long)(td.ray0 - ta.objs[k].ray_off) * S;
    }
    const ObjDev& ob = ta.objs[k];
    const int M = nr * S;
    const int Mpad = (M + 7) & ~7;
    const float* P = ta.params + ob.param_off;
    const float* WT = ta.wt + ob.wt_off;
    const float cx = ob.c[0], cy = ob.c[1], cz = ob.c[2], sc = ob.scale;

    // ---- rays into smem ---------------------------------------------------
    for (int r = threadIdx.x; r < nr && MODE != MODE_QUERY; r += blockDim.x) {
        const float* rec;
        if (MODE == MODE_EVAL) rec = ta.pool + (ray_first + r) * REC;
        else rec = ta.pool + (ob.src_off + ta.pick[ray_first + r]) * REC;
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
                    float t1 = (lo - o) / dir, t2 = (hi - o) / dir;
                    tn = fmaxf(tn, fminf(t1, t2));
                    tf = fminf(tf, fmaxf(t1, t2));
                } else if (o < lo || o > hi) {
                    tf = -1.f;
                }
            }
            d[11] = tn;
            d[12] = tf;
        }
    }
    __syncthreads();

    // ---- points x~ = (o + t d - c) / s ------------------------------------
    for (int m = threadIdx.x; m < Mpad; m += blockDim.x) {
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        if (m < M) {
            const int r = m / S, i = m - r * S;
            const float* d = rays + r * RAYF;
            if (MODE == MODE_QUERY) {
                const float* q = ta.qpts + (ray_first + m) * 3;
                x0 = (q[0] - cx) / sc;
                x1 = (q[1] - cy) / sc;
                x2 = (q[2] - cz) / sc;
            } else {
                float t;
                if (MODE == MODE_EVAL) t = d[11] + ((float)i + 0.5f) / (float)S * (d[12] - d[11]);
                else t = ta.tbuf[sbase + m];
                tsm[m] = t;
                x0 = (fmaf(t, d[3], d[0]) - cx) / sc;
                x1 = (fmaf(t, d[4], d[1]) - cy) / sc;
                x2 = (fmaf(t, d[5], d[2]) - cz) / sc;
            }
        }
        if (m >= M) tsm[m] = 0.f;
        g[0 * LD + m] = x0;
        g[1 * LD + m] = x1;
        g[2 * LD + m] = x2;
    }
    for (int i = threadIdx.x; i < 3 * LD; i += blockDim.x) g[(DIN + i / LD) * LD + (i % LD)] = 0.f;
    __syncthreads();
    // ---- Gaussian encoding: sin / cos of B x~ --------------------------------
    for (int f = threadIdx.x; f < NF * Mpad; f += blockDim.x) {
        const int j = f / Mpad, m = f - j * Mpad;
        const float p = fmaf(sp.B[3 * j + 2], g[2 * LD + m],
                             fmaf(sp.B[3 * j + 1], g[1 * LD + m], sp.B[3 * j] * g[0 * LD + m]));
        float s, c;
        sincosf(p, &s, &c);
        g[(3 + j) * LD + m] = s;
        g[(3 + NF + j) * LD + m] = c;
    }
    // layer-1 weights (transposed [96][H])
    stage(ws, WT + wt_layer_off(H, 0), DINP * H);
    __syncthreads();

    // ---- forward ----------------------------------------------------------
    float* h[4] = {act, act + H * LD, act + 2 * H * LD, act + 3 * H * LD};
    gemm_fwd<H, DINP, 0>(g, LD, ws, P + b_off(H, 0), h[0], LD, Mpad);
    __syncthreads();
#pragma unroll 1
    for (int l = 1; l < 4; ++l) {
        stage(ws, WT + wt_layer_off(H, l), H * H);
        __syncthreads();
        gemm_fwd<H, H, 0>(h[l - 1], LD, ws, P + b_off(H, l), h[l], LD, Mpad);
        __syncthreads();
    }
    stage(ws, WT + wt_layer_off(H, 4), H * NOUT);
    __syncthreads();
    gemm_fwd<NOUT, H, 1>(h[3], LD, ws, P + b_off(H, 4), yb, LD, Mpad);
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
        return;
    }

    // ---- rendering (Eq. 3), losses (Eq. 4-5) and their gradient ---------------
    // one thread per ray; padded samples get zero gradient
    float* rsum = rays;   // per ray results reuse the ray scratch: [r*RAYF + 13..15]
    if (threadIdx.x < nr) {
        const int r = threadIdx.x;
        float* d = rays + r * RAYF;
        float Pr = 1.f, Oh = 0.f, Dh = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        for (int i = 0; i < S; ++i) {
            const int m = r * S + i;
            const float o = sigmoidf_(yb[m]);
            const float c0 = sigmoidf_(yb[LD + m]), c1 = sigmoidf_(yb[2 * LD + m]), c2 = sigmoidf_(yb[3 * LD + m]);
            const float T = o * Pr;
            Oh += T;
            Dh = fmaf(T, tsm[m], Dh);
            C0 = fmaf(T, c0, C0); C1 = fmaf(T, c1, C1); C2 = fmaf(T, c2, C2);
            ps[m] = Pr;
            yb[m] = o; yb[LD + m] = c0; yb[2 * LD + m] = c1; yb[3 * LD + m] = c2;
            Pr = Pr * (1.f - o);
        }
        if (MODE == MODE_EVAL) {
            const bool hit = d[12] > d[11] && d[12] > 0.f;
            ta.eval_out[ray_first + r] = hit ? Dh : 0.f;
        } else {
            const float D = d[6], Msk = d[10];
            const float valid = D > 0.f ? 1.f : 0.f;
            const float wD = Msk * valid;
            const float eD = Dh - D, e0 = C0 - d[7], e1 = C1 - d[8], e2 = C2 - d[9], eO = Oh - Msk;
            d[13] = wD * fabsf(eD);
            d[14] = Msk * ((fabsf(e0) + fabsf(e1)) + fabsf(e2));
            d[15] = fabsf(eO);
            if (MODE != MODE_FORWARD) {
                const float invR = 1.f / (float)ob.R;
                const float a = wD * signf_(eD) * invR;
                const float bsc = sp.lam_c * Msk * invR / 3.f;
                const float b0 = bsc * signf_(e0), b1 = bsc * signf_(e1), b2 = bsc * signf_(e2);
                const float e = sp.lam_o * signf_(eO) * invR;
                float Sn = 0.f;
                for (int i = S - 1; i >= 0; --i) {
                    const int m = r * S + i;
                    const float o = yb[m], c0 = yb[LD + m], c1 = yb[2 * LD + m], c2 = yb[3 * LD + m];
                    const float gi = fmaf(a, tsm[m], fmaf(b0, c0, fmaf(b1, c1, b2 * c2))) + e;
                    const float Pi = ps[m];
                    const float dLdo = Pi * (gi - Sn);
                    Sn = fmaf(o, gi, (1.f - o) * Sn);
                    const float T = o * Pi;
                    yb[m] = dLdo * o * (1.f - o);
                    yb[LD + m] = T * b0 * c0 * (1.f - c0);
                    yb[2 * LD + m] = T * b1 * c1 * (1.f - c1);
                    yb[3 * LD + m] = T * b2 * c2 * (1.f - c2);
                }
            }
        }
    }
    if (MODE == MODE_EVAL) return;
    // zero the gradient of padded samples
    for (int m = M + threadIdx.x; m < Mpad; m += blockDim.x) {
        yb[m] = 0.f; yb[LD + m] = 0.f; yb[2 * LD + m] = 0.f; yb[3 * LD + m] = 0.f;
    }
    __syncthreads();
    float* gp = ta.part + part;   // this tile's partial slot
    if (threadIdx.x == 0) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int r = 0; r < nr; ++r) { s0 += rsum[r * RAYF + 13]; s1 += rsum[r * RAYF + 14]; s2 += rsum[r * RAYF + 15]; }
        const long long P_ = param_count(H);
        gp[P_ + 0] = s0; gp[P_ + 1] = s1; gp[P_ + 2] = s2;
        gp[P_ + 3] = 0.f; gp[P_ + 4] = 0.f; gp[P_ + 5] = 0.f;
    }
    if (MODE == MODE_FORWARD) return;

    // ---- backward ----------------------------------------------------------
    // layer 5: dW5 = dY^T h4, dZ4 = (dY W5) * [h4 > 0]
    gemm_dw<NOUT, H>(yb, h[3], LD, Mpad, red, gp + w_off(H, 4), H, gp + b_off(H, 4));
    stage(ws, P + w_off(H, 4), NOUT * H);     // W5 [4][H] == B[k=out][n=in]
    __syncthreads();
    gemm_fwd<H, NOUT, 2>(yb, LD, ws, nullptr, h[3], LD, Mpad);
    __syncthreads();
#pragma unroll 1
    for (int l = 3; l >= 1; --l) {
        // dW_{l+1} = dZ_{l+1}^T h_l ; dZ_l = (dZ_{l+1} W_{l+1}) * [h_l > 0]
        gemm_dw<H, H>(h[l], h[l - 1], LD, Mpad, red, gp + w_off(H, l), H, gp + b_off(H, l));
        stage(ws, P + w_off(H, l), H * H);
        __syncthreads();
        gemm_fwd<H, H, 2>(h[l], LD, ws, nullptr, h[l - 1], LD, Mpad);
        __syncthreads();
    }
    // layer 1: dW1 = dZ1^T gamma
    gemm_dw<H, DINP>(h[0], g, LD, Mpad, red, gp + w_off(H, 0), DIN, gp + b_off(H, 0));
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
                    const float z = h[0][n * LD + m];
                    d0 = fmaf(z, ws[n * DINP + 0], d0);
                    d1 = fmaf(z, ws[n * DINP + 1], d1);
                    d2 = fmaf(z, ws[n * DINP + 2], d2);
                }
                for (int j = 0; j < NF; ++j) {
                    float ds = 0.f, dc = 0.f;
                    for (int n = 0; n < H; ++n) {
                        const float z = h[0][n * LD + m];
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
            gp[param_count(H) + 3 + threadIdx.x] = -s / sc;
        }
    }
}

}  // namespace vmapk
