// Tensor-core training path for hidden width 128 (the background model of a
// room, section 3.2 / 4.1), in two kernels.
//
// One CTA cannot hold a width-128 object's BF16 weights (124 KB), the four
// hidden activation tiles the weight gradients need, and the gradient
// accumulators (496 of the 512 TMEM columns) at once. The step is split:
//
//   k_wide_fb  per tile of <= 128 samples: encoding, forward MMAs (weights
//              resident in shared memory), FP32 rendering and losses, and the
//              backward input-gradient MMAs dZ_l = (dZ_{l+1} W_{l+1}) * [h_l > 0].
//              Every GEMM operand it forms (encoding, h1..h4, dY, dZ1..dZ4;
//              BF16, core-matrix layout) is streamed to an activation buffer,
//              284 KB per tile, with the tile's loss sums.
//   k_wide_dw  weight gradients dW_l = sum over samples of dZ_l^T h_{l-1} as
//              split-K MMAs: CTA (range r, layer job j) streams job j's two
//              operands of every tile in range r through a three-stage ring
//              filled by bulk async copies (cp.async.bulk, mbarrier transaction
//              counts) and accumulates in TMEM; bias gradients are column sums
//              of the same BF16 operand tiles, in FP32, in a fixed order. At
//              the end of each object run the CTA writes its layer's slice of
//              the run slot, which the reduce kernel sums in slot order.
//
// The MMA shapes and descriptor conventions are those of vmap_tc.cuh.
#pragma once
#include <cuda_bf16.h>

#include "vmap_common.cuh"
#include "vmap_tc.cuh"
#include "vmap_tile_bf16.cuh"
#include "vmap_tile_fp32.cuh"

namespace vmapk {

constexpr int WH = 128;       // hidden width of this path
constexpr int WJOBS = 5;      // weight-gradient jobs: W1, W2, W3, W4, W5
constexpr int WIDE_THREADS = 512;   // k_wide_fb: 16 warps, 32 accumulator columns per thread

// per-tile activation record (bytes), every operand a core-matrix tile of 128 rows
struct WideAct {
    static constexpr int G0 = 0;                                  // encoding [128][96]
    static constexpr int HL = G0 + TM * DINP * 2;                 // h1..h4 [128][128]
    static constexpr int DY = HL + 4 * TM * WH * 2;               // dL/dy [128][16]
    static constexpr int DZ = DY + TM * 16 * 2;                   // dZ1..dZ4 [128][128]
    static constexpr long long BYTES = DZ + 4 * TM * WH * 2;      // 290,816
    __host__ __device__ static constexpr int h(int l) { return HL + l * TM * WH * 2; }
    __host__ __device__ static constexpr int dz(int l) { return DZ + l * TM * WH * 2; }
};

struct WideFbCfg {
    static constexpr int W1B = WH * DINP * 2, WHB = WH * WH * 2, W5B = 16 * WH * 2;
    static constexpr int WIMG = 0;                                // weight image (as in global memory)
    static constexpr int WIMG_BYTES = W1B + 3 * WHB + W5B;        // 126,976
    static constexpr int G0 = WIMG + WIMG_BYTES;                  // [128][96]; dY [128][16] after layer 1
    static constexpr int HA = G0 + TM * DINP * 2;                 // current h [128][128]
    static constexpr int DZ = HA + TM * WH * 2;                   // current dZ [128][128]
    static constexpr int MASK = DZ + TM * WH * 2;                 // [4][128][4] u32: bits of h_l > 0 (word = 32 columns)
    static constexpr int TSO = MASK + 4 * TM * 16;               // [128] sample depths
    static constexpr int YB = TSO + TM * 4;                       // [4][128]
    static constexpr int RAYS = YB + 4 * TM * 4;                  // [RTMAX][RAYF]
    static constexpr int BIAS = RAYS + RTMAX * RAYF * 4;          // [4][128] + [16] f32 biases of the run's object
    static constexpr int MBAR = BIAS + (4 * WH + 16) * 4;
    static constexpr int WBAR = MBAR + 8;                         // weight image loaded
    static constexpr int TSLOT = WBAR + 8;
    static constexpr int BYTES = TSLOT + 8;
    static constexpr int NCOLS = 128;
    static_assert(BYTES <= 232448, "shared memory of one CTA");
};

struct WideDwCfg {
    static constexpr int STAGE = 65536;                           // operand A at +0, operand B at +32 KB
    static constexpr int NST = 3;
    static constexpr int BSUM = NST * STAGE;                      // [16][128] f32 bias partials
    static constexpr int FULL = BSUM + 16 * 128 * 4;              // [NST] mbarriers: stage loaded
    static constexpr int EMPTY = FULL + 8 * NST;                  // [NST] mbarriers: stage's MMAs done
    static constexpr int TSLOT = EMPTY + 8 * NST;
    static constexpr int BYTES = TSLOT + 16;
    static constexpr int NCOLS = 128;
    static_assert(BYTES <= 232448, "shared memory of one CTA");
};

struct WideArgs {
    TileArgs t;
    const __nv_bfloat16* img;     // tensor-core weight images (arena)
    const long long* img_off;     // per object: element offset of its image
    int* err;                     // set to 1 when a bounded wait gives up
    unsigned char* const* act;    // device cell holding the activation buffer (tile-indexed)
    float* tile_loss;             // [tiles][4]: depth, colour, occupancy sums of each tile
    int loss_only;                // k_wide_dw: only fold the tile losses into the run slots
    long long polls;              // polls before an MMA or copy wait gives up
};

// bits (v[j] > 0) of 8 values, placed at bit offset `at` of a 64-bit word
__device__ __forceinline__ unsigned long long pos_bits(const float (&v)[8], int at) {
    unsigned b = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) b |= (v[j] > 0.f ? 1u : 0u) << j;
    return (unsigned long long)b << at;
}

template <int MODE>
__global__ void __launch_bounds__(WIDE_THREADS, 1) k_wide_fb(StepParams sp, WideArgs wa) {
    using C = WideFbCfg;
    constexpr bool GRAD = MODE == MODE_TRAIN;
    const TileArgs& ta = wa.t;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* W1 = sm + C::WIMG;
    auto Whp = [&](int l) { return W1 + C::W1B + l * C::WHB; };   // computed, not a local-memory array
    unsigned char* W5 = W1 + C::W1B + 3 * C::WHB;
    unsigned char* G0 = sm + C::G0;
    unsigned char* DYt = sm + C::G0;
    unsigned char* HA = sm + C::HA;
    unsigned char* DZ = sm + C::DZ;
    uint32_t* mask = reinterpret_cast<uint32_t*>(sm + C::MASK);
    float* bsm = reinterpret_cast<float*>(sm + C::BIAS);
    float* tsm = reinterpret_cast<float*>(sm + C::TSO);
    float* yb = reinterpret_cast<float*>(sm + C::YB);
    float* rays = reinterpret_cast<float*>(sm + C::RAYS);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + C::MBAR);
    uint64_t* wbar = reinterpret_cast<uint64_t*>(sm + C::WBAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + C::TSLOT);
    // 16 warps: warp w reads TMEM lane quadrant w % 4 (the hardware rule) and
    // accumulator columns (w / 4) * 32 .. + 31
    const int tid = threadIdx.x, warp = tid >> 5;
    const int q = warp & 3, qc = warp >> 2;
    const int row = q * 32 + (tid & 31);
    const int col0 = qc * 32;
    unsigned char* act = GRAD ? *wa.act : nullptr;
    // every CTA of this grid is resident once each has passed this point: the
    // weight-gradient kernel launched behind it may then take freed SMs
    pdl_launch_dependents();

    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_init(wbar, 1);
    }
    if (warp == 0) tmem_alloc(tslot, C::NCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tl_lane = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t phase = 0, wphase = 0;
    bool abort = false, wpend = false;
    bool pre = false;                    // this tile's rays and depths were prefetched
    int npick = 0;                       // pick of the next tile's ray `tid`

    // Every thread waits for an MMA commit by itself (no CTA barrier); a wait
    // that gave up is agreed on at the next CTA barrier, before any further MMA
    // is issued, so a give-up leaves at most one commit outstanding: its parity
    // is kept and drained before tensor memory is freed.
    bool wfail = false, lost = false;
    uint32_t lpar = 0;
    auto wait_mma = [&]() {
        if (!mbar_wait(mbar, phase, wa.polls)) {
            wfail = true;
            lost = true;
            lpar = phase;
        }
        phase ^= 1;
        tc_fence_after();
    };
    // operand writes and TMEM reads done -> MMA may start. The record copy of the
    // previous round (the other of the two ping-pong tiles) has finished reading
    // before the barrier, so that tile may be rewritten in the next round.
    auto sync_for_mma = [&]() {
        tmem_ld_wait();
        fence_async_smem();
        tc_fence_before();
        if (tid == 0) bulk_wait_read();
        if (__syncthreads_or(wfail)) {
            abort = true;
            if (tid == 0) atomicExch(wa.err, 1);
        }
        tc_fence_after();
    };
    // h_{l+1} (forward round l) and dZ_{l+1} (backward round l) alternate between
    // the two 32 KB tiles: h1, h3, dZ4, dZ2 -> HA; h2, h4, dZ3, dZ1 -> DZ
    auto hbuf = [&](int l) { return (l & 1) ? DZ : HA; };
    auto zbuf = [&](int l) { return (l & 1) ? HA : DZ; };
    // the activation record receives an operand tile by one bulk copy (after sync_for_mma)
    auto record = [&](unsigned char* dst, const unsigned char* tile, int bytes) {
        if (tid == 0) {
            bulk_store(dst, tile, (uint32_t)bytes);
            bulk_commit();
        }
    };
    // this thread's 32 accumulator columns
    auto load_acc = [&](float (&v)[32]) {
        float a[16];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            tmem_ld16(tl_lane + col0 + 16 * c, a);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[16 * c + i] = a[i];
        }
        tmem_ld_wait();
    };

    // Tile ranges front-loaded: the first n % G CTAs take one tile more. CTAs
    // start in block order, so when this kernel starts on the SMs that a
    // preceding tile kernel frees, the CTAs that start last have the least to do.
    const long long n_tiles = *ta.n_tiles;
    const long long nG = gridDim.x, per = n_tiles / nG, rem = n_tiles % nG, cb = blockIdx.x;
    const long long t0 = cb < rem ? cb * (per + 1) : rem * (per + 1) + (cb - rem) * per;
    const long long t1 = t0 + (cb < rem ? per + 1 : per);

#pragma unroll 1
    for (long long tl = t0; tl < t1 && !abort; ++tl) {
        const TileDev td = ta.tiles[tl];
        const int k = td.obj, nr = td.nr;
        const bool first = tl == t0 || ta.tiles[tl - 1].obj != k;
        const ObjDev& ob = ta.objs[k];
        const int S = ob.S, M = nr * S;
        const long long sbase = ta.obs[k].sample_off + (long long)(td.ray0 - ta.obs[k].ray_off) * S;
        const float* P = ta.params + ob.param_off;
        const float cx = ob.c[0], cy = ob.c[1], cz = ob.c[2], sc = ob.scale;
        const float isc = 1.f / sc;   // points are normalised by one multiply (within 1 ulp of dividing)
        unsigned char* at = GRAD ? act + (long long)tl * WideAct::BYTES : nullptr;
        if (tid == 0) bulk_wait_read();   // the previous tile's last records have left shared memory

        if (first && tid == 0) {
            // the weight image arrives by bulk copy while the tile is encoded
            mbar_expect_tx(wbar, (uint32_t)C::WIMG_BYTES);
            bulk_load(W1, wa.img + wa.img_off[k], (uint32_t)C::WIMG_BYTES, wbar);
            wpend = true;
        }
        // (after the first tile of a training range, the previous tile's backward
        // already brought this tile's rays and depths in by cp.async)
        if (!pre) {
            for (int r = tid; r < nr; r += blockDim.x) {
                const float* rec = ta.pool + (ta.obs[k].src_off + ta.pick[td.ray0 + r]) * REC;
                float* d = rays + r * RAYF;
#pragma unroll
                for (int u = 0; u < 11; ++u) d[u] = rec[u];
            }
        } else {
            cp_async_wait_all();
        }
        if (first)   // the object's biases, read by the epilogues from shared memory
            for (int i = tid; i < 4 * WH + NOUT; i += blockDim.x) bsm[i] = P[b_off(WH, i / WH) + i % WH];
        __syncthreads();
        // ---- points and encoding -> G0 (and the activation record); two threads
        // per sample, each forming the sample's normalised point itself ------------
        for (int f = tid; f < 2 * TM; f += blockDim.x) {
            const int m = f % TM, half = f / TM;
            float x0 = 0.f, x1 = 0.f, x2 = 0.f;
            if (m < M) {
                const float* d = rays + (m / S) * RAYF;
                const float t = pre ? tsm[m] : ta.tbuf[sbase + m];
                if (!pre && half == 0) tsm[m] = t;
                x0 = (fmaf(t, d[3], d[0]) - cx) * isc;
                x1 = (fmaf(t, d[4], d[1]) - cy) * isc;
                x2 = (fmaf(t, d[5], d[2]) - cz) * isc;
            }
            encode_row_half(sp, x0, x1, x2, m, half, G0, nullptr);
        }
        sync_for_mma();
        if (abort) break;
        if (GRAD) record(at + WideAct::G0, G0, TM * DINP * 2);
        if (first) {
            const bool ok = mbar_wait(wbar, wphase, wa.polls);
            if (__syncthreads_or(!ok)) {
                abort = true;
                if (tid == 0) atomicExch(wa.err, 1);
                break;
            }
            wphase ^= 1;
            wpend = false;
        }

        // ---- forward -----------------------------------------------------------
        if (warp == 0) {
#pragma unroll
            for (int kc = 0; kc < DINP / 16; ++kc)
                mma_bf16_w(tmem, desc_kmajor(G0, DINP, 16 * kc), desc_kmajor(W1, DINP, 16 * kc),
                         idesc_bf16(TM, WH, 0, 0), kc > 0);
            mma_commit_w(mbar);
        }
        // the next tile of this range: its picks now, its rays and depths during the backward
        const bool has_next = GRAD && tl + 1 < t1;
        TileDev tdn{};
        if (has_next) {
            tdn = ta.tiles[tl + 1];
            if (tid < tdn.nr) npick = ta.pick[tdn.ray0 + tid];
        }
        wait_mma();
        if (abort) break;
#pragma unroll 1
        for (int l = 0; l < 4; ++l) {
            unsigned char* hb = hbuf(l);
            float v[32];
            load_acc(v);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float u[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) u[j] = fmaxf(v[8 * c + j] + bsm[l * WH + col0 + 8 * c + j], 0.f);
                st_bf16x8(hb, cm_off(row, col0 + 8 * c, WH), u);
            }
            sync_for_mma();
            if (abort) break;
            if (GRAD) record(at + WideAct::h(l), hb, TM * WH * 2);
            if (warp == 0) {
                if (l < 3) {
#pragma unroll
                    for (int kc = 0; kc < WH / 16; ++kc)
                        mma_bf16_w(tmem, desc_kmajor(hb, WH, 16 * kc), desc_kmajor(Whp(l), WH, 16 * kc),
                                 idesc_bf16(TM, WH, 0, 0), kc > 0);
                } else {
#pragma unroll
                    for (int kc = 0; kc < WH / 16; ++kc)
                        mma_bf16_w(tmem, desc_kmajor(hb, WH, 16 * kc), desc_kmajor(W5, WH, 16 * kc),
                                 idesc_bf16(TM, 16, 0, 0), kc > 0);
                }
                mma_commit_w(mbar);
            }
            if (GRAD) {
                // the ReLU mask of h_{l+1} (needed by the backward), from the BF16
                // tile the MMA is reading, while the MMA runs
                unsigned bits = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float a[8];
                    ld_bf16x8(hb, cm_off(row, col0 + 8 * c, WH), a);
                    bits |= (unsigned)pos_bits(a, 8 * c);
                }
                mask[(l * TM + row) * 4 + qc] = bits;
            }
            wait_mma();
        }
        if (abort) break;
        {
            float v[8];
            tmem_ld8(tl_lane, v);
            tmem_ld_wait();
            if (qc == 0) {
                const float* b5 = bsm + 4 * WH;
#pragma unroll
                for (int j = 0; j < NOUT; ++j) yb[j * TM + row] = sigmoidf_(v[j] + b5[j]);   // o, c (Eq. 1 heads)
            }
        }
        if (__syncthreads_or(wfail)) {
            abort = true;
            if (tid == 0) atomicExch(wa.err, 1);
        }
        if (abort) break;

        // ---- rendering, loss, dL/dy (FP32) ---------------------------------------
        const float invR = 1.f / (float)ta.obs[k].R;
        for (int r = warp; r < nr; r += blockDim.x / 32)
            render_ray_warp<GRAD, TM, true>(sp, yb, tsm, rays + r * RAYF, r, S, invR);
        for (int m = M + tid; m < TM; m += blockDim.x) {
            yb[m] = 0.f; yb[TM + m] = 0.f; yb[2 * TM + m] = 0.f; yb[3 * TM + m] = 0.f;
        }
        __syncthreads();
        if (warp == 0) {   // the tile's loss sums, rays in order (lane r holds ray r's terms)
            const int ln = tid & 31;
            float e0 = 0.f, e1 = 0.f, e2 = 0.f;
            if (ln < nr) {
                e0 = rays[ln * RAYF + 13]; e1 = rays[ln * RAYF + 14]; e2 = rays[ln * RAYF + 15];
            }
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            for (int r = 0; r < nr; ++r) {
                s0 += __shfl_sync(0xffffffffu, e0, r);
                s1 += __shfl_sync(0xffffffffu, e1, r);
                s2 += __shfl_sync(0xffffffffu, e2, r);
            }
            if (ln == 0) *reinterpret_cast<float4*>(wa.tile_loss + 4 * tl) = make_float4(s0, s1, s2, 0.f);
        }
        if (!GRAD) {
            __syncthreads();
            continue;
        }
        // dY -> BF16 [128][16] (columns 4..15 zero), over the dead encoding tile
        for (int m = tid; m < TM * 2; m += blockDim.x) {
            const int r = m % TM, half = m / TM;
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = (half == 0 && j < NOUT) ? yb[j * TM + r] : 0.f;
            st_bf16x8(DYt, cm_off(r, half * 8, 16), v);
        }
        sync_for_mma();
        if (abort) break;
        record(at + WideAct::DY, DYt, TM * 16 * 2);
        // rays, depths and the loss terms of this tile are consumed: prefetch the next tile's
        pre = false;
        if (has_next) {
            const ObjBatch& obn = ta.obs[tdn.obj];
            const int Sn = ta.objs[tdn.obj].S;
            if (tid < tdn.nr) {
                const float* rec = ta.pool + (obn.src_off + npick) * REC;
                float* d = rays + tid * RAYF;
                cp_async16(d, rec);
                cp_async16(d + 4, rec + 4);
                cp_async16(d + 8, rec + 8);
            }
            const long long sb = obn.sample_off + (long long)(tdn.ray0 - obn.ray_off) * Sn;
            for (int i = tid; i < tdn.nr * Sn; i += blockDim.x) cp_async4(tsm + i, ta.tbuf + sb + i);
            cp_async_commit();
            pre = true;
        }

        // ---- backward: input gradients ------------------------------------------
        if (warp == 0) {
            mma_bf16_w(tmem, desc_kmajor(DYt, 16, 0), desc_mnmajor(W5, WH, 0), idesc_bf16(TM, WH, 0, 1), false);
            mma_commit_w(mbar);
        }
#pragma unroll 1
        for (int l = 3; l >= 0; --l) {
            // accumulator = dZ_{l+2} W_{l+2} (dY W5 for l = 3); dZ_{l+1} = acc * [h_{l+1} > 0]
            unsigned char* zb = zbuf(l);
            wait_mma();
            float v[32];
            load_acc(v);
            const unsigned bits = mask[(l * TM + row) * 4 + qc];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float u[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) u[j] = (bits >> (8 * c + j)) & 1u ? v[8 * c + j] : 0.f;
                st_bf16x8(zb, cm_off(row, col0 + 8 * c, WH), u);
            }
            sync_for_mma();
            if (abort) break;
            record(at + WideAct::dz(l), zb, TM * WH * 2);
            if (l == 0) break;
            if (warp == 0) {
#pragma unroll
                for (int kc = 0; kc < WH / 16; ++kc)
                    mma_bf16_w(tmem, desc_kmajor(zb, WH, 16 * kc), desc_mnmajor(Whp(l - 1), WH, 16 * kc),
                             idesc_bf16(TM, WH, 0, 1), kc > 0);
                mma_commit_w(mbar);
            }
        }
        if (abort) break;
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    // drain (bounded) what a give-up left in flight: the MMA commit given up on
    // and a weight copy; then prefetches and activation-record stores
    if (lost) mbar_wait(mbar, lpar, DRAIN_POLLS);
    if (wpend) mbar_wait(wbar, wphase, DRAIN_POLLS);
    cp_async_wait_all();   // prefetches issued before an abort land before the CTA exits
    if (tid == 0) bulk_wait_all();   // every activation record is written before the CTA exits
    // when launched behind a tile kernel (programmatic stream serialization),
    // this grid completes only after that kernel has: what follows in the
    // stream sees both
    pdl_wait();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, C::NCOLS);
}

// Weight-gradient jobs: operand A (M side, 128 TMEM lanes = input index) and
// B (N side = output index) of job j inside a tile's activation record, their
// column counts, and N. Every job computes a transposed gradient
// dW_{j+1}^T [in][out] = a_j^T dZ_{j+1} (a_0 = encoding, a_j = h_j, dZ_5 = dY),
// so a warp's flush writes 32 consecutive inputs of one output row.
struct WideJob {
    int a_off, a_cc, a_bytes, b_off, b_cc, b_bytes, n;
};
__device__ __forceinline__ WideJob wide_job(int j) {
    if (j == 0) return {WideAct::G0, DINP, TM * DINP * 2, WideAct::dz(0), WH, TM * WH * 2, WH};
    if (j < 4) return {WideAct::h(j - 1), WH, TM * WH * 2, WideAct::dz(j), WH, TM * WH * 2, WH};
    return {WideAct::h(3), WH, TM * WH * 2, WideAct::DY, 16, TM * 16 * 2, 16};
}

__global__ void __launch_bounds__(NTHREADS, 1) k_wide_dw(WideArgs wa) {
    using C = WideDwCfg;
    const TileArgs& ta = wa.t;
    extern __shared__ __align__(1024) unsigned char sm[];
    float* bsum = reinterpret_cast<float*>(sm + C::BSUM);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + C::FULL);
    uint64_t* empty = reinterpret_cast<uint64_t*>(sm + C::EMPTY);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + C::TSLOT);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int q = warp & 3, hf = warp >> 2;
    const int row = q * 32 + (tid & 31);
    const int ranges = gridDim.x / WJOBS;
    const int rg = blockIdx.x / WJOBS, j = blockIdx.x % WJOBS;
    if (wa.loss_only && j != 0) return;
    const WideJob jb = wide_job(j);
    constexpr long long PC = param_count(WH);
    const long long n_tiles = *ta.n_tiles;
    const long long t0 = (long long)rg * n_tiles / ranges;
    const long long t1 = (long long)(rg + 1) * n_tiles / ranges;
    const int n = (int)(t1 - t0);
    // every CTA is resident once each has passed this point: the reduce
    // launched behind this kernel may start its table loads on free SMs
    pdl_launch_dependents();

    if (wa.loss_only) {
        pdl_wait();   // the tile losses come from k_wide_fb
        // fold the tile losses of every run into its slot, in tile order
        if (tid == 0) {
            float l0 = 0.f, l1 = 0.f, l2 = 0.f;
            for (long long tl = t0; tl < t1; ++tl) {
                const int k = ta.tiles[tl].obj;
                if (tl == t0 || ta.tiles[tl - 1].obj != k) l0 = l1 = l2 = 0.f;
                const float4 l4 = *reinterpret_cast<const float4*>(wa.tile_loss + 4 * tl);
                l0 += l4.x; l1 += l4.y; l2 += l4.z;
                if (tl + 1 == t1 || ta.tiles[tl + 1].obj != k) {
                    float* gp = ta.part + ta.tiles[tl].part;
                    gp[PC + 0] = l0; gp[PC + 1] = l1; gp[PC + 2] = l2;
                    gp[PC + 3] = 0.f; gp[PC + 4] = 0.f; gp[PC + 5] = 0.f;
                }
            }
        }
        return;
    }

    const unsigned char* act = *wa.act;
    if (tid == 0) {
        for (int s = 0; s < C::NST; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
    }
    if (warp == 0) tmem_alloc(tslot, C::NCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // launched behind k_wide_fb (programmatic stream serialization): the set-up
    // above overlapped its end; the operand records and tile losses are its
    pdl_wait();
    const uint32_t tmem = *tslot;
    bool abort = false;
    // thread 0 fills stage i % NST with tile t0 + i
    auto issue_load = [&](int i) {
        unsigned char* st = sm + (i % C::NST) * C::STAGE;
        const unsigned char* src = act + (t0 + i) * WideAct::BYTES;
        uint64_t* fb = full + i % C::NST;
        mbar_expect_tx(fb, (uint32_t)(jb.a_bytes + jb.b_bytes));
        bulk_load(st, src + jb.a_off, (uint32_t)jb.a_bytes, fb);
        bulk_load(st + 32768, src + jb.b_off, (uint32_t)jb.b_bytes, fb);
    };
    int issued = 0;   // tiles whose loads were issued (thread 0's count; uniform by construction)
    if (tid == 0)
        for (; issued < min(C::NST, n); ++issued) issue_load(issued);
    issued = min(C::NST, n);
    int consumed = 0;   // tiles whose stage was seen loaded

    // bias partial sums: thread = (column chunk c8, row r8 within a core matrix, strip parity sp2);
    // a warp reads 512 contiguous bytes of the core-matrix tile (no bank conflicts)
    const int c8 = (tid >> 3) & 15, r8 = tid & 7, sp2 = tid >> 7;
    const int b_cc = jb.b_cc;
    const int b_src = 32768;               // operand B holds dZ (or dY for job 4)
    const bool b_active = c8 * 8 < b_cc;
    float bs[8];
    float lacc[3] = {0.f, 0.f, 0.f};

#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        const long long tl = t0 + i;
        const int s = i % C::NST;
        const uint32_t par = (uint32_t)((i / C::NST) & 1);
        const int k = ta.tiles[tl].obj;
        const bool first = i == 0 || ta.tiles[tl - 1].obj != k;
        const bool last = i + 1 == n || ta.tiles[tl + 1].obj != k;
        if (first) {
#pragma unroll
            for (int u = 0; u < 8; ++u) bs[u] = 0.f;
            lacc[0] = lacc[1] = lacc[2] = 0.f;
        }
        if (j == 0 && tid == 0) {
            const float4 l4 = *reinterpret_cast<const float4*>(wa.tile_loss + 4 * tl);
            lacc[0] += l4.x; lacc[1] += l4.y; lacc[2] += l4.z;
        }
        // stage s holds tile i
        const bool ok = mbar_wait(full + s, par, wa.polls);
        if (__syncthreads_or(!ok)) {
            abort = true;
            if (tid == 0) atomicExch(wa.err, 1);
            break;
        }
        consumed = i + 1;
        unsigned char* st = sm + s * C::STAGE;
        if (warp == 0) {
            tc_fence_after();
#pragma unroll
            for (int kc = 0; kc < TM / 16; ++kc)
                mma_bf16_w(tmem, desc_mnmajor(st, jb.a_cc, 16 * kc), desc_mnmajor(st + 32768, jb.b_cc, 16 * kc),
                         idesc_bf16(TM, jb.n, 1, 1), !(first && kc == 0));
            mma_commit_w(empty + s);
        }
        if (b_active) {
#pragma unroll
            for (int strip = sp2; strip < TM / 8; strip += 2) {
                float v[8];
                ld_bf16x8(st + b_src, cm_off(strip * 8 + r8, c8 * 8, b_cc), v);
#pragma unroll
                for (int u = 0; u < 8; ++u) bs[u] += v[u];
            }
        }
        __syncthreads();   // every thread is done reading stage s
        // refill the stage of tile i - 1 (its MMAs had this iteration to finish)
        // with tile i - 1 + NST; tile i's own stage is refilled one iteration later
        if (i >= 1 && i - 1 + C::NST < n) {
            const int sp_ = (i - 1) % C::NST;
            const uint32_t pp = (uint32_t)(((i - 1) / C::NST) & 1);
            bool okr = true;
            if (tid == 0) {
                okr = mbar_wait(empty + sp_, pp, wa.polls);
                if (okr) issue_load(i - 1 + C::NST);
            }
            if (__syncthreads_or(!okr)) {
                abort = true;
                if (tid == 0) atomicExch(wa.err, 1);
                break;
            }
            ++issued;
        }
        if (!last) continue;
        // ---- run end: write this job's slice of the run slot --------------------
        float* gp = ta.part + ta.tiles[tl].part;
        if (j == 0 && tid == 0) {
            gp[PC + 0] = lacc[0]; gp[PC + 1] = lacc[1]; gp[PC + 2] = lacc[2];
            gp[PC + 3] = 0.f; gp[PC + 4] = 0.f; gp[PC + 5] = 0.f;
        }
        // tile i's MMAs were the run's last (commit order = issue order)
        const bool okf = mbar_wait(empty + s, par, wa.polls);
        if (__syncthreads_or(!okf)) {
            abort = true;
            if (tid == 0) atomicExch(wa.err, 1);
            break;
        }
        tc_fence_after();
        if (j < 4) {
            // lane = input index, column = output index: W_{j+1}[out][in]
            const int fan = j == 0 ? DIN : WH;
            float* w = gp + w_off(WH, j) + row;
#pragma unroll 1
            for (int c0 = 0; c0 < WH / 2; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + hf * (WH / 2) + c0, v);
                tmem_ld_wait();
                if (row < fan) {
#pragma unroll
                    for (int u = 0; u < 16; ++u) w[(long long)(hf * (WH / 2) + c0 + u) * fan] = v[u];
                }
            }
        } else {
            float v[8];
            tmem_ld8(tmem + ((uint32_t)(q * 32) << 16), v);
            tmem_ld_wait();
            if (hf == 0) {
#pragma unroll
                for (int o = 0; o < NOUT; ++o) gp[w_off(WH, 4) + o * WH + row] = v[o];
            }
        }
        if (b_active) {
#pragma unroll
            for (int u = 0; u < 8; ++u) bsum[(sp2 * 8 + r8) * 128 + c8 * 8 + u] = bs[u];
        }
        __syncthreads();
        const int nb = j < 4 ? WH : NOUT;
        if (tid < nb) {
            float sum = 0.f;
            for (int r = 0; r < 16; ++r) sum += bsum[r * 128 + tid];
            gp[b_off(WH, j) + tid] = sum;
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (abort && tid == 0) {
        // drain (bounded) before tensor memory is freed: the bulk copies still in
        // flight, and the MMAs of the last tile whose MMAs were issued (its
        // commit is that stage's latest phase and covers every earlier MMA)
        for (int u = consumed; u < issued; ++u)
            mbar_wait(full + u % C::NST, (uint32_t)((u / C::NST) & 1), DRAIN_POLLS);
        if (consumed > 0) {
            const int u = consumed - 1;
            mbar_wait(empty + u % C::NST, (uint32_t)((u / C::NST) & 1), DRAIN_POLLS);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, C::NCOLS);
}

}  // namespace vmapk
