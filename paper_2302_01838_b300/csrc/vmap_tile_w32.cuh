// FP32 training path for hidden width 128 (the background model of a room,
// section 3.2 / 4.1), in two kernels on FP32 SIMT arithmetic.
//
// The fused FP32 tile kernel holds a tile's four hidden activations in shared
// memory, which leaves room for 48 samples at width 128: its GEMMs then run
// on 4x4 register tiles, 32 bytes read from shared memory per 16 FMAs, at
// about 30% of the FFMA peak. Here the step is split so that every GEMM runs
// on 128-sample tiles with 8x8 register tiles per thread (64 bytes per 64
// FMAs, the shape an isolated 128x128x128 block runs at about 70% of peak):
//
//   k_w32_fb  per tile of <= 128 samples (whole rays of one object): encoding,
//             the five forward GEMMs, rendering and losses (Eq. 3-5), and the
//             input-gradient GEMMs dZ_l = (dZ_{l+1} W_{l+1}) * [h_l > 0]. Only
//             two activation buffers live in shared memory; the GEMM operands
//             the weight gradients of layers 1-4 need (encoding, h1..h3,
//             dZ1..dZ4) are written to a record buffer, FP32, sample-major
//             ([128 samples][features]) from the registers that formed them;
//             the output layer's weight and bias gradients and the bias
//             gradients of layers 1-4 are summed over the tile on chip. The
//             ReLU masks of h1..h4 stay in registers (a thread's backward block
//             is the same 8x8 block of samples and features as its forward
//             one). Tiles come from a counter.
//   k_w32_dw  weight gradients dW_l = sum over samples of dZ_l^T h_{l-1},
//             l = 1..4: CTA (range r, job j) streams job j's two operands of
//             every tile in range r through three stages of asynchronous
//             copies, in 64-sample chunks (contiguous in the sample-major
//             records), and accumulates 8x8 blocks of dW_l in registers, the
//             samples being the GEMM's reduction axis as in k_w32_fb's own
//             GEMMs. At the end of each object run the CTA stores its layer's
//             part of the run slot (adding the run's per-tile sums in tile
//             order), which the reduce kernel sums in slot order.
#pragma once
#include "vmap_common.cuh"
#include "vmap_tile_fp32.cuh"

namespace vmapk {

constexpr int W32H = 128;          // hidden width of this path
constexpr int W32M = 128;          // samples per tile
constexpr int W32_THREADS = 256;   // 16 x 16 threads, an 8x8 block each
constexpr int W32JOBS = 4;         // weight-gradient jobs: W1, W2, W3, W4
constexpr int W32LD = W32M + 4;    // activation row stride in shared memory (floats)

// per-tile record (floats): sample-major operand blocks [W32M samples][width],
// then the tile's sums that k_w32_fb forms on chip (bias gradients of layers
// 1..4, the output layer's weight and bias gradients)
struct W32Act {
    static constexpr int BLK = W32M * W32H;
    static constexpr int G0 = 0;                        // encoding [128][128] (features 96..127 zero)
    static constexpr int HL = G0 + BLK;                 // h1..h3 [128][128] each
    static constexpr int DZ = HL + 3 * BLK;             // dZ1..dZ4 [128][128] each
    static constexpr int DB = DZ + 4 * BLK;             // sum over samples of dZ1..dZ4 [4][128]
    static constexpr int DW5 = DB + 4 * W32H;           // sum over samples of dY[o] h4[k] [4][128]
    static constexpr int DB5 = DW5 + NOUT * W32H;       // sum over samples of dY [4] (+ 4 unused)
    static constexpr long long FLOATS = DB5 + 8;        // 132,104 (528,416 bytes)
    __host__ __device__ static constexpr int h(int l) { return HL + l * BLK; }    // h_{l+1}
    __host__ __device__ static constexpr int dz(int l) { return DZ + l * BLK; }   // dZ_{l+1}
};

// shared memory of k_w32_fb (floats)
struct W32FbCfg {
    static constexpr int XA = 0;                        // [128][W32LD] activations
    static constexpr int XB = XA + W32H * W32LD;        // [128][W32LD]
    static constexpr int W = XB + W32H * W32LD;         // [128][128] weights as B[k][n]
    static constexpr int YB = W + W32H * W32H;          // [4][W32LD] outputs, then dL/dy
    static constexpr int TS = YB + 4 * W32LD;           // [128] sample depths
    static constexpr int RAYS = TS + W32M;              // [RTMAX][RAYF]
    static constexpr int CS = RAYS + RTMAX * RAYF;      // [16][128] column sums of each thread row tm
    static constexpr int TOTAL = CS + 16 * W32H;
    static constexpr size_t BYTES = (size_t)TOTAL * sizeof(float);
    static_assert(BYTES <= 232448, "shared memory of one CTA");
};

// A thread's 8x8 block: samples tm*4 + i (i < 4) and 64 + tm*4 + i - 4 (i >= 4),
// features tn*4 + j (j < 4) and 64 + tn*4 + j - 4 (j >= 4).
__device__ __forceinline__ int w32_m(int tm, int i) { return (i < 4 ? 0 : 60) + tm * 4 + i; }
__device__ __forceinline__ int w32_n(int tn, int j) { return (j < 4 ? 0 : 60) + tn * 4 + j; }

// A thread's register-tile coordinates (16 x 16 over the CTA's 256 threads).
// A warp's 16-byte shared load costs as many wavefronts as the most distinct
// vectors any group of four consecutive lanes reads (two at least), so each
// four-lane group takes 2 tm x 2 tn (two wavefronts for every operand load;
// lanes along tn would cost four for B); a warp covers 4 tm x 8 tn.
static_assert(W32_THREADS == 256, "w32_lane_map covers 16 x 16 threads");
__device__ __forceinline__ void w32_lane_map(int tid, int& tm, int& tn) {
    const int w = tid >> 5, g = (tid >> 2) & 7, t = tid & 3;
    tm = (w >> 1) * 4 + 2 * (g & 1) + (t & 1);
    tn = (w & 1) * 8 + 2 * (g >> 1) + (t >> 1);
}

// acc[i][j] (+)= sum_k A[k][m_i] B[k][n_j] (m_i = w32_m(tm, i), n_j =
// w32_n(tn, j)); A: [K][LA], B: [K][LB]. The next k's operands load while
// this k's 64 FMAs run. ZERO: start from zero, else add to acc. kc < K
// stops after the first kc rows of k (RUNTIME_K only; rows of A and B up to
// kc are read).
template <int K, int LA = W32LD, int LB = W32H, bool ZERO = true, bool RUNTIME_K = false>
__device__ __forceinline__ void w32_mm(const float* __restrict__ A, const float* __restrict__ B, int tm, int tn,
                                       float (&acc)[8][8], int kc = K) {
    if (!RUNTIME_K) kc = K;
    if (ZERO) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    }
    const float* a = A + tm * 4;
    const float* b = B + tn * 4;
    float4 a0 = *reinterpret_cast<const float4*>(a), a1 = *reinterpret_cast<const float4*>(a + 64);
    float4 b0 = *reinterpret_cast<const float4*>(b), b1 = *reinterpret_cast<const float4*>(b + 64);
#pragma unroll 4
    for (int k = 0; k < kc; ++k) {
        const int kn = k + 1 < kc ? k + 1 : k;
        const float4 na0 = *reinterpret_cast<const float4*>(a + kn * LA);
        const float4 na1 = *reinterpret_cast<const float4*>(a + kn * LA + 64);
        const float4 nb0 = *reinterpret_cast<const float4*>(b + kn * LB);
        const float4 nb1 = *reinterpret_cast<const float4*>(b + kn * LB + 64);
        const float am[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bn[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(am[i], bn[j], acc[i][j]);
        a0 = na0; a1 = na1; b0 = nb0; b1 = nb1;
    }
}

// store a thread's block to out[n][m] (feature-major) and, when rec is not
// NULL, to the sample-major record rec[m][n] (a warp writes 128 consecutive
// bytes of each of four samples' rows): with bias, ReLU and the mask bits of
// the result (bit 8 i + j: h[n_j][m_i] > 0); or, with `mask`, the block
// times those bits
template <bool FWD>
__device__ __forceinline__ unsigned long long w32_store(float (&acc)[8][8], float* out, int tm, int tn,
                                                        const float* __restrict__ bias, unsigned long long mask,
                                                        float* __restrict__ rec, float* __restrict__ colsum = nullptr) {
    unsigned long long bits = 0ull;
    float* r0 = rec ? rec + tm * 4 * W32H + tn * 4 : nullptr;   // sample w32_m(tm, 0), feature w32_n(tn, 0)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float v;
            if (FWD) {
                v = fmaxf(acc[i][j] + bias[w32_n(tn, j)], 0.f);
                bits |= (v > 0.f ? 1ull : 0ull) << (8 * i + j);
            } else {
                v = (mask >> (8 * i + j)) & 1ull ? acc[i][j] : 0.f;
            }
            acc[i][j] = v;
        }
        if (rec) {
            float* r = r0 + (i < 4 ? i : 60 + i) * W32H;
            // streaming stores: the records (more than L2 holds per step) are read
            // once, and evicting them first keeps the run slots in L2 for the reduce
            __stcs(reinterpret_cast<float4*>(r), make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]));
            __stcs(reinterpret_cast<float4*>(r + 64), make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]));
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int n = w32_n(tn, j);
#pragma unroll
        for (int h = 0; h < 2; ++h)
            *reinterpret_cast<float4*>(out + n * W32LD + h * 64 + tm * 4) =
                make_float4(acc[4 * h][j], acc[4 * h + 1][j], acc[4 * h + 2][j], acc[4 * h + 3][j]);
    }
    if (colsum) {
        // column sums over the thread's 8 samples, to colsum[tm][n] (the 16
        // rows tm are added in order once every thread has stored)
#pragma unroll
        for (int j = 0; j < 8; ++j)
            colsum[tm * W32H + w32_n(tn, j)] =
                ((acc[0][j] + acc[1][j]) + (acc[2][j] + acc[3][j])) + ((acc[4][j] + acc[5][j]) + (acc[6][j] + acc[7][j]));
    }
    return bits;
}

// the encoding (rows 0..95 of a [row][W32LD] block) to its sample-major
// record [128][128], features 96..127 zero; a thread writes 32 bytes
__device__ __forceinline__ void w32_record_enc(float* __restrict__ dst, const float* __restrict__ src) {
    for (int e = threadIdx.x; e < W32M * (W32H / 8); e += blockDim.x) {
        const int m = e % W32M, k8 = e / W32M;
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = 8 * k8 + u < DINP ? src[(8 * k8 + u) * W32LD + m] : 0.f;
        __stcs(reinterpret_cast<float4*>(dst + m * W32H + 8 * k8), make_float4(v[0], v[1], v[2], v[3]));   // streaming (see w32_store)
        __stcs(reinterpret_cast<float4*>(dst + m * W32H + 8 * k8 + 4), make_float4(v[4], v[5], v[6], v[7]));
    }
}

struct W32Args {
    TileArgs t;
    float* const* act;    // device cell holding the record buffer (tile-indexed)
    float* tile_loss;     // [tiles][8]: depth, colour, occupancy sums, 0, centre gradient[3], 0
    int loss_only;        // k_w32_dw: only fold the tile losses into the run slots
};

template <int MODE>
__global__ void __launch_bounds__(W32_THREADS, 1) k_w32_fb(StepParams sp, W32Args wa) {
    using C = W32FbCfg;
    constexpr bool GRAD = MODE == MODE_TRAIN || MODE == MODE_GRAD_CENTER;
    const TileArgs& ta = wa.t;
    extern __shared__ __align__(16) float smem[];
    float* xa = smem + C::XA;
    float* xb = smem + C::XB;
    float* ws = smem + C::W;
    float* yb = smem + C::YB;
    float* tsm = smem + C::TS;
    float* rays = smem + C::RAYS;
    __shared__ long long s_tile;
    const int tid = threadIdx.x, warp = tid >> 5, nwarps = W32_THREADS / 32;
    // a warp writes 128-byte pieces of four samples' record rows
    int tm, tn;
    w32_lane_map(tid, tm, tn);
    float* cs = smem + C::CS;
    constexpr long long PC = param_count(W32H);
    const long long n = *ta.n_tiles;
    float* const act = *wa.act;
    // the weight-gradient kernel launched behind this one may start its set-up
    pdl_launch_dependents();
#pragma unroll 1
    for (;;) {
        // the next tile of the class's counter (every thread read the previous
        // tile index before the barrier that ended the previous tile)
        if (tid == 0) s_tile = atomicAdd(ta.dyn, 1);
        __syncthreads();
        const long long tl = s_tile;
        if (tl >= n) break;
        const TileDev td = ta.tiles[tl];
        const int k = td.obj;
        const int nr = td.nr;
        const ObjDev& ob = ta.objs[k];
        const int S = ob.S;
        const int M = nr * S;
        const long long sbase = ta.obs[k].sample_off + (long long)(td.ray0 - ta.obs[k].ray_off) * S;
        const float* P = ta.params + ob.param_off;
        const float* WT = ta.wt + ob.wt_off;
        const float cx = ob.c[0], cy = ob.c[1], cz = ob.c[2], sc = ob.scale;
        float* rec = act + tl * W32Act::FLOATS;

        // ---- rays, sample points, encoding ------------------------------------
        for (int r = tid; r < nr; r += W32_THREADS) {
            const float* src = ta.pool + (ta.obs[k].src_off + ta.pick[td.ray0 + r]) * REC;
            float* d = rays + r * RAYF;
#pragma unroll
            for (int q = 0; q < 11; ++q) d[q] = src[q];
        }
        stage_issue(ws, WT + wt_layer_off(W32H, 0), DINP * W32H);   // W1^T [96][128], during the encoding
        __syncthreads();
        for (int m = tid; m < W32M; m += W32_THREADS) {
            float x0 = 0.f, x1 = 0.f, x2 = 0.f, t = 0.f;
            if (m < M) {
                const float* d = rays + (m / S) * RAYF;
                t = ta.tbuf[sbase + m];
                x0 = (fmaf(t, d[3], d[0]) - cx) / sc;
                x1 = (fmaf(t, d[4], d[1]) - cy) / sc;
                x2 = (fmaf(t, d[5], d[2]) - cz) / sc;
            }
            tsm[m] = t;
            xa[0 * W32LD + m] = x0;
            xa[1 * W32LD + m] = x1;
            xa[2 * W32LD + m] = x2;
        }
        __syncthreads();
        encode<W32LD>(sp, xa, W32M);
        stage_wait();
        __syncthreads();
        if (GRAD) w32_record_enc(rec + W32Act::G0, xa);

        // ---- forward: h1 .. h4 (ping-pong xa -> xb -> xa ...), masks in registers;
        // the next layer's weights load while a layer's epilogue runs
        unsigned long long mk[4];
        float acc[8][8];
#pragma unroll
        for (int l = 0; l < 4; ++l) {   // unrolled: mk stays in registers
            float* in = (l & 1) ? xb : xa;
            float* out = (l & 1) ? xa : xb;
            if (l == 0) w32_mm<DINP>(in, ws, tm, tn, acc);
            else w32_mm<W32H>(in, ws, tm, tn, acc);
            __syncthreads();   // every thread is done with ws
            if (l < 3) stage_issue(ws, WT + wt_layer_off(W32H, l + 1), W32H * W32H);   // W_{l+2}^T
            else stage_issue(ws, WT + wt_layer_off(W32H, 4), W32H * NOUT);               // W5^T [128][4]
            // h_{l+1}; h4 has no record (the output layer's gradients are formed here)
            mk[l] = w32_store<true>(acc, out, tm, tn, P + b_off(W32H, l), 0ull,
                                    GRAD && l < 3 ? rec + W32Act::h(l) : nullptr);
            stage_wait();
            __syncthreads();
        }
        // h4 is in xa, W5^T in ws
        // output layer: y[o][m] = sum_k h4[k][m] W5^T[k][o] + b5[o], two outputs per thread
        {
            const int m = tid & 127, o0 = (tid >> 7) * 2;
            float y0 = 0.f, y1 = 0.f;
#pragma unroll 8
            for (int kk = 0; kk < W32H; ++kk) {
                const float h = xa[kk * W32LD + m];
                const float2 w = *reinterpret_cast<const float2*>(ws + kk * NOUT + o0);
                y0 = fmaf(h, w.x, y0);
                y1 = fmaf(h, w.y, y1);
            }
            yb[o0 * W32LD + m] = y0 + P[b_off(W32H, 4) + o0];
            yb[(o0 + 1) * W32LD + m] = y1 + P[b_off(W32H, 4) + o0 + 1];
        }
        __syncthreads();

        // ---- rendering (Eq. 3), losses (Eq. 4-5) and dL/dy ---------------------
        const float invR = 1.f / (float)ta.obs[k].R;
        for (int r = warp; r < nr; r += nwarps) render_ray_warp<GRAD, W32LD>(sp, yb, tsm, rays + r * RAYF, r, S, invR);
        for (int m = M + tid; m < W32M; m += W32_THREADS) {   // padded samples carry no gradient
            yb[m] = 0.f; yb[W32LD + m] = 0.f; yb[2 * W32LD + m] = 0.f; yb[3 * W32LD + m] = 0.f;
        }
        __syncthreads();
        if (tid == 0) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            for (int r = 0; r < nr; ++r) {
                s0 += rays[r * RAYF + 13]; s1 += rays[r * RAYF + 14]; s2 += rays[r * RAYF + 15];
            }
            float* tlo = wa.tile_loss + 8 * tl;
            tlo[0] = s0; tlo[1] = s1; tlo[2] = s2; tlo[3] = 0.f;
            tlo[4] = 0.f; tlo[5] = 0.f; tlo[6] = 0.f; tlo[7] = 0.f;
        }
        if (!GRAD) continue;   // (the loop's next barrier follows)

        // ---- the output layer's gradients over the tile: dW5[o][k] = sum_m dY[o][m] h4[k][m],
        // db5[o] = sum_m dY[o][m] (h4 is in xa, dY in yb)
        if (tid < W32H) {
            float a5[NOUT] = {0.f, 0.f, 0.f, 0.f};
            const float* hk = xa + tid * W32LD;
#pragma unroll 4
            for (int m = 0; m < W32M; m += 4) {
                const float4 h = *reinterpret_cast<const float4*>(hk + m);
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    const float4 y = *reinterpret_cast<const float4*>(yb + o * W32LD + m);
                    a5[o] = fmaf(y.x, h.x, fmaf(y.y, h.y, fmaf(y.z, h.z, fmaf(y.w, h.w, a5[o]))));
                }
            }
#pragma unroll
            for (int o = 0; o < NOUT; ++o) rec[W32Act::DW5 + o * W32H + tid] = a5[o];
        } else if (tid < W32H + NOUT) {
            const float* yo = yb + (tid - W32H) * W32LD;
            float sb = 0.f;
            for (int m = 0; m < W32M; m += 4) {
                const float4 y = *reinterpret_cast<const float4*>(yo + m);
                sb += (y.x + y.y) + (y.z + y.w);
            }
            rec[W32Act::DB5 + tid - W32H] = sb;
        }
        // ---- backward: dZ4 = (dY W5) * [h4 > 0], dZ_l = (dZ_{l+1} W_{l+1}) * [h_l > 0];
        // each layer's weights load while the epilogue before their GEMM runs
        __syncthreads();   // every thread is done with W5^T (output layer)
        stage_issue(ws, P + w_off(W32H, 4), NOUT * W32H);   // W5 [4][128] == B[k=o][n]
        stage_wait();
        __syncthreads();
#pragma unroll
        for (int l = 4; l >= 1; --l) {
            float* in = (l & 1) ? xa : xb;    // dZ_{l+1} (dY for l = 4)
            float* out = (l & 1) ? xb : xa;   // dZ_l
            if (l == 4) w32_mm<NOUT>(yb, ws, tm, tn, acc);
            else w32_mm<W32H>(in, ws, tm, tn, acc);
            __syncthreads();   // every thread is done with ws
            if (l > 1) stage_issue(ws, P + w_off(W32H, l - 1), W32H * W32H);   // W_l [n_out][n_in] == B[k][n]
            w32_store<false>(acc, out, tm, tn, nullptr, mk[l - 1], rec + W32Act::dz(l - 1), cs);
            if (l > 1) stage_wait();
            __syncthreads();
            if (tid < W32H) {   // the bias gradient of layer l over the tile, rows tm in order
                float c = 0.f;
#pragma unroll
                for (int r = 0; r < 16; ++r) c += cs[r * W32H + tid];
                rec[W32Act::DB + (l - 1) * W32H + tid] = c;
            }
        }
        // dZ1 is in xb
        if (MODE == MODE_GRAD_CENTER) {
            // encoding backward, one thread per sample:
            //   dgamma_j = sum_n dZ1[n] W1[n][j]
            //   dx~ = dgamma_xyz + sum_j B_j (cos_j dgamma_sin_j - sin_j dgamma_cos_j)
            //   dL/dc = -sum_samples dx~ / s
            stage_w1_rows<W32H>(ws, P + w_off(W32H, 0));   // W1 [128][96]
            // the encoding again (xa): x~ from the depths, then sin / cos
            for (int m = tid; m < W32M; m += W32_THREADS) {
                float x0 = 0.f, x1 = 0.f, x2 = 0.f;
                if (m < M) {
                    const float* d = rays + (m / S) * RAYF;
                    const float t = tsm[m];
                    x0 = (fmaf(t, d[3], d[0]) - cx) / sc;
                    x1 = (fmaf(t, d[4], d[1]) - cy) / sc;
                    x2 = (fmaf(t, d[5], d[2]) - cz) / sc;
                }
                xa[0 * W32LD + m] = x0;
                xa[1 * W32LD + m] = x1;
                xa[2 * W32LD + m] = x2;
            }
            __syncthreads();
            encode<W32LD>(sp, xa, W32M);
            __syncthreads();
            float* acc3 = yb;   // [3][W32LD]
            for (int m = tid; m < W32M; m += W32_THREADS) {
                float d0 = 0.f, d1 = 0.f, d2 = 0.f;
                if (m < M) {
                    for (int nn = 0; nn < W32H; ++nn) {
                        const float z = xb[nn * W32LD + m];
                        d0 = fmaf(z, ws[nn * DINP + 0], d0);
                        d1 = fmaf(z, ws[nn * DINP + 1], d1);
                        d2 = fmaf(z, ws[nn * DINP + 2], d2);
                    }
                    for (int j = 0; j < NF; ++j) {
                        float ds = 0.f, dc = 0.f;
                        for (int nn = 0; nn < W32H; ++nn) {
                            const float z = xb[nn * W32LD + m];
                            ds = fmaf(z, ws[nn * DINP + 3 + j], ds);
                            dc = fmaf(z, ws[nn * DINP + 3 + NF + j], dc);
                        }
                        const float w = ds * xa[(3 + NF + j) * W32LD + m] - dc * xa[(3 + j) * W32LD + m];
                        d0 = fmaf(w, sp.B[3 * j], d0);
                        d1 = fmaf(w, sp.B[3 * j + 1], d1);
                        d2 = fmaf(w, sp.B[3 * j + 2], d2);
                    }
                }
                acc3[m] = d0; acc3[W32LD + m] = d1; acc3[2 * W32LD + m] = d2;
            }
            __syncthreads();
            if (tid < 3) {
                float s = 0.f;
                for (int m = 0; m < M; ++m) s += acc3[tid * W32LD + m];
                wa.tile_loss[8 * tl + 4 + tid] = -s / sc;
            }
            // per ray through x = o + t d (depths fixed): dL/do = sum dL/dx, dL/dd = sum t dL/dx
            if (ta.ray_grad) {
                for (int r = tid; r < nr; r += W32_THREADS) {
                    float go[3] = {0.f, 0.f, 0.f}, gd[3] = {0.f, 0.f, 0.f};
                    for (int i = 0; i < S; ++i) {
                        const int m = r * S + i;
                        const float t = tsm[m];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const float v = acc3[a * W32LD + m] / sc;
                            go[a] += v;
                            gd[a] = fmaf(t, v, gd[a]);
                        }
                    }
                    float* out = ta.ray_grad + (long long)(td.ray0 + r) * 6;
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
    if (tid == 0 && atomicAdd(ta.dyn + 1, 1) == (int)gridDim.x - 1) {
        // every CTA has taken its last tile: reset the counter for the next launch
        ta.dyn[0] = 0;
        ta.dyn[1] = 0;
    }
}

// shared memory of k_w32_dw (floats): NST stages of 64-sample chunks, a
// chunk being two contiguous sample-major blocks (dZ_l and the layer's input)
constexpr int W32CH = 64;
constexpr int W32DW_ROWS = 1024;   // tiles of a range whose valid rows are tabled
struct W32DwCfg {
    static constexpr int BLK = W32CH * W32H;
    static constexpr int STAGE = 2 * BLK;          // A = dZ_l [64][128], B = input [64][128]
    static constexpr int NST = 3;                  // stages in flight
    static constexpr int TOTAL = NST * STAGE;
    static constexpr size_t BYTES = (size_t)TOTAL * sizeof(float);
    static_assert(BYTES <= 232448, "shared memory of one CTA");
};

__global__ void __launch_bounds__(W32_THREADS, 1) k_w32_dw(W32Args wa) {
    using C = W32DwCfg;
    const TileArgs& ta = wa.t;
    extern __shared__ __align__(16) float smem[];
    const int tid = threadIdx.x;
    // a thread's 8x8 block of dW_l: rows n = w32_m(ta_, i), columns k = w32_n(tb, j)
    int ta_, tb;
    w32_lane_map(tid, ta_, tb);
    const int ranges = gridDim.x / W32JOBS;
    const int rg = blockIdx.x / W32JOBS, j = blockIdx.x % W32JOBS;
    if (wa.loss_only && j != 0) return;
    constexpr long long PC = param_count(W32H);
    const long long n_tiles = *ta.n_tiles;
    const long long t0 = (long long)rg * n_tiles / ranges;
    const long long t1 = (long long)(rg + 1) * n_tiles / ranges;
    const int n = (int)(t1 - t0);
    // the reduce launched behind this kernel may start its table loads
    pdl_launch_dependents();
    // launched behind the step's other FP32 tile kernels (programmatic stream
    // serialization): the records and tile losses are k_w32_fb's
    pdl_wait();
    if (wa.loss_only) {
        // fold the tile losses of every run into its slot, in tile order
        if (tid == 0) {
            float l0 = 0.f, l1 = 0.f, l2 = 0.f;
            for (long long tl = t0; tl < t1; ++tl) {
                const int k = ta.tiles[tl].obj;
                if (tl == t0 || ta.tiles[tl - 1].obj != k) l0 = l1 = l2 = 0.f;
                const float* lo = wa.tile_loss + 8 * tl;
                l0 += lo[0]; l1 += lo[1]; l2 += lo[2];
                if (tl + 1 == t1 || ta.tiles[tl + 1].obj != k) {
                    float* gp = ta.part + ta.tiles[tl].part;
                    gp[PC + 0] = l0; gp[PC + 1] = l1; gp[PC + 2] = l2;
                    gp[PC + 3] = 0.f; gp[PC + 4] = 0.f; gp[PC + 5] = 0.f;
                }
            }
        }
        return;
    }
    if (n <= 0) return;
    const float* act = *wa.act;
    // valid samples of the range's first W32DW_ROWS tiles (later tiles count as
    // full): chunks copy and contract only those rows (the padded rows' dZ is
    // zero, so leaving them out changes no sum)
    __shared__ int s_rows[W32DW_ROWS];
    for (int i = tid; i < n && i < W32DW_ROWS; i += W32_THREADS) {
        const TileDev td = ta.tiles[t0 + i];
        s_rows[i] = min(W32M, td.nr * ta.objs[td.obj].S);
    }
    __syncthreads();
    auto chunk_rows = [&](int c) {
        const int i = c / (W32M / W32CH);
        const int r = (i < W32DW_ROWS ? s_rows[i] : W32M) - (c % (W32M / W32CH)) * W32CH;
        return r < 0 ? 0 : (r > W32CH ? W32CH : r);
    };
    // job j: dW_{j+1} from dZ_{j+1} and the layer's input (job 0: the encoding);
    // job 0 also gathers the output layer's per-tile sums
    const int L = j;
    const int a_off = W32Act::dz(L), b_off_rec = L == 0 ? W32Act::G0 : W32Act::h(L - 1);
    constexpr int CPT = W32M / W32CH;   // chunks per tile
    constexpr int PIECES = C::STAGE / 4 / W32_THREADS;   // 16-byte copies per thread and chunk
    const int nch = n * CPT;
    auto issue = [&](int c) {
        const float* rec = act + (t0 + c / CPT) * W32Act::FLOATS;
        const int m0 = (c % CPT) * W32CH;
        const int rows = chunk_rows(c);
        const float* srca = rec + a_off + m0 * W32H;
        const float* srcb = rec + b_off_rec + m0 * W32H;
        const unsigned base = (unsigned)__cvta_generic_to_shared(smem + (c % C::NST) * C::STAGE);
#pragma unroll
        for (int it = 0; it < PIECES; ++it) {
            const int p = tid + it * W32_THREADS;            // 16-byte piece of the stage
            const int q = p & (C::BLK / 4 - 1);              // ... within its block
            if (q / (W32H / 4) >= rows) continue;            // its row is padding
            const float* src = (p < C::BLK / 4 ? srca : srcb) + 4 * q;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + 16u * p), "l"(src) : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[i][u] = 0.f;
    // chunk c is loaded into stage c % NST, NST - 1 chunks ahead of the one in use
    issue(0);
    if (nch > 1) issue(1);
#pragma unroll 1
    for (int c = 0; c < nch; ++c) {
        if (c + 1 < nch) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        // stage (c + 2) % NST was last read for chunk c - 1 (before that chunk's barrier)
        if (c + 2 < nch) issue(c + 2);
        const float* st = smem + (c % C::NST) * C::STAGE;
        // dW[n][k] += sum over the chunk's samples m of dZ[m][n] x[m][k]
        w32_mm<W32CH, W32H, W32H, false, true>(st, st + C::BLK, ta_, tb, acc, chunk_rows(c));
        __syncthreads();   // every thread is done with stage c % NST before it is refilled
        // ---- run end: store this job's part of the run slot ------------------
        if (c % CPT != CPT - 1) continue;
        const long long tl = t0 + c / CPT;
        const int k = ta.tiles[tl].obj;
        if (tl + 1 < t1 && ta.tiles[tl + 1].obj == k) continue;
        float* gp = ta.part + ta.tiles[tl].part;
        const int Kreal = L == 0 ? DIN : W32H;
        float* gw = gp + w_off(W32H, L);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int nn = w32_m(ta_, i);
            if (L == 0) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int kk = w32_n(tb, u);
                    if (kk < Kreal) gw[nn * Kreal + kk] = acc[i][u];
                }
            } else {   // rows of 128 floats, 16-byte aligned in the slot
                *reinterpret_cast<float4*>(gw + nn * W32H + tb * 4) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                *reinterpret_cast<float4*>(gw + nn * W32H + 64 + tb * 4) =
                    make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[i][u] = 0.f;
        }
        // the run's per-tile sums, in tile order: bias of layer L + 1; (job 0)
        // the output layer's weights and bias, the loss terms and centre gradient
        long long tf = tl;
        while (tf > t0 && ta.tiles[tf - 1].obj == k) --tf;
        if (tid < W32H) {
            float sb = 0.f;
            for (long long u = tf; u <= tl; ++u) sb += act[u * W32Act::FLOATS + W32Act::DB + L * W32H + tid];
            gp[b_off(W32H, L) + tid] = sb;
        }
        if (j == 0) {
            for (int e = tid; e < NOUT * W32H; e += W32_THREADS) {
                float sw = 0.f;
                for (long long u = tf; u <= tl; ++u) sw += act[u * W32Act::FLOATS + W32Act::DW5 + e];
                gp[w_off(W32H, 4) + e] = sw;
            }
            if (tid < NOUT) {
                float sb = 0.f;
                for (long long u = tf; u <= tl; ++u) sb += act[u * W32Act::FLOATS + W32Act::DB5 + tid];
                gp[b_off(W32H, 4) + tid] = sb;
            }
            if (tid == 0) {
                float sl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (long long u = tf; u <= tl; ++u) {
                    const float* lo = wa.tile_loss + 8 * u;
                    sl[0] += lo[0]; sl[1] += lo[1]; sl[2] += lo[2];
                    sl[3] += lo[4]; sl[4] += lo[5]; sl[5] += lo[6];
                }
                for (int e = 0; e < 6; ++e) gp[PC + e] = sl[e];
            }
        }
    }
}

}  // namespace vmapk
