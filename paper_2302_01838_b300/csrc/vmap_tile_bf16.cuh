// Persistent fused training kernel with the MLP GEMMs on the 5th-generation
// tensor cores (tcgen05, BF16 operands, FP32 accumulation in tensor memory).
// Hidden widths 16, 32 and 64.
//
// Per tile of whole rays (<= 128 samples, one MMA M = 128):
//   encoding (FP32 math, BF16 operand tile)  -> 5 forward MMA layers, each
//   epilogue (bias, ReLU) reading the FP32 accumulator from TMEM and writing
//   the next BF16 operand tile -> FP32 rendering / loss / dL/dy (warp scans)
//   -> backward: the input-gradient chain dZ_prev = (dZ W) * [a > 0] as MMAs,
//   and the weight gradients dW^T = A^T dZ as MMAs with M = fan-in (the
//   activation tile read MN-major), accumulated in TMEM over all tiles of a
//   run (consecutive tiles of one object in the CTA's range).
// Weight-gradient layouts:
//   hidden 16 / 32 ("fused"): an MMA costs about the same to issue for any N
//   up to 128, so layers share MMAs. Operand tiles are laid side by side:
//     X  = [encoding (96) | h4 (H)]      Hs = [h1 | h2 | h3 | 1 | 0...]
//     Z  = [dZ2 | dZ3 | dZ4]             ZY = [dZ1 | dY (16)]
//   S2 = Hs^T Z (N = 3H) holds dW2^T, dW3^T, dW4^T as its diagonal blocks and
//   their bias gradients in the ones lane (3H); S1 = X^T ZY (N = H + 16) holds
//   dW1^T (lanes 0..92 x dZ1 columns), dW5^T (h4 lanes x dY columns) and b1, b5
//   in the encoding's ones lane (93). 16 weight-gradient MMAs per tile
//   instead of 40; the off-diagonal blocks are not used.
//   hidden 64 ("split"): one weight-gradient MMA sequence per layer; each
//   activation tile carries a ones column that yields its layer's bias
//   gradient.
// A run's gradient leaves TMEM once, when the CTA moves to another object or
// ends. FP32 is kept for rendering (the transmittance product), losses, master
// weights and Adam moments; only GEMM operands are BF16.
#pragma once
#include <cuda_bf16.h>

#include "vmap_common.cuh"
#include "vmap_optim.cuh"
#include "vmap_tc.cuh"
#include "vmap_tile_fp32.cuh"

namespace vmapk {

constexpr int TM = 128;                       // samples per tile (MMA M)
// Polls of an mbarrier before a wait gives up: the default of the runtime limit
// (Bf16Args::polls / WideArgs::polls, set per context) and the fixed bound of
// the waits that drain a CTA's own MMAs and copies before it frees tensor
// memory and exits (the work drained was issued, so those waits end).
constexpr long long MMA_WAIT_LIMIT = 1LL << 26;
constexpr long long DRAIN_POLLS = 1LL << 26;

template <int H> struct Bf16Cfg {
    static_assert(H == 16 || H == 32 || H == 64, "tensor-core path: hidden 16, 32 or 64");
    static constexpr bool FUSED = H <= 32;    // fused weight-gradient MMAs (see the file comment)
    static constexpr int NFWD = H;            // forward accumulator columns
    // fused layout: operand tiles (columns) and tensor-memory columns
    static constexpr int XC = DINP + H;       // X: encoding | h4
    static constexpr int HSC = 3 * H + 8;     // Hs: h1 | h2 | h3 | ones | zeros
    static constexpr int ONES_HS = 3 * H;     // the ones column of Hs (bias lane of S2)
    static constexpr int ZC = 3 * H;          // Z: dZ2 | dZ3 | dZ4
    static constexpr int ZYC = H + 16;        // ZY: dZ1 | dY (4 used, 12 zero)
    static constexpr int C_S1 = NFWD;         // X^T ZY
    static constexpr int C_S2 = NFWD + ZYC;   // Hs^T Z
    // split layout (hidden 64)
    static constexpr int CH = H + 8;          // activation tile columns: H values, ones, zeros
    static constexpr int C_FWD = 0;
    static constexpr int C_DX = FUSED ? 0 : NFWD;   // fused: shares the forward accumulator
    static constexpr int C_DW5 = 2 * NFWD;
    static constexpr int C_DW1 = C_DW5 + 16;  // dW1..dW4 at C_DW1 + l * H
    static constexpr int NCOLS_USED = FUSED ? C_S2 + ZC : C_DW1 + 4 * H;
    static constexpr int NCOLS = NCOLS_USED <= 128 ? 128 : NCOLS_USED <= 256 ? 256 : 512;
    static constexpr int CTAS = FUSED ? 2 : 1;
    // shared memory (bytes). Fused: X | Hs | Z | ZY (an MN-major read of Hs or X
    // with M = 128 lanes runs past its last strip into the next tile: unused lanes)
    static constexpr int X = 0;
    static constexpr int HS = X + TM * XC * 2;
    static constexpr int Z = HS + TM * HSC * 2;
    static constexpr int ZY = Z + TM * ZC * 2;
    static constexpr int FUSED_END = ZY + TM * ZYC * 2;
    // split: G0 | HA[4] | DZ[2] | DY | tail room for MN-major over-reads
    static constexpr int G0 = 0;                                  // [128][96] bf16 encoding
    static constexpr int HA = G0 + TM * DINP * 2;                 // 4 x [128][CH]
    static constexpr int HA_BYTES = TM * CH * 2;
    static constexpr int DZ = HA + 4 * HA_BYTES;                  // 2 x [128][H]
    static constexpr int DZ_BYTES = TM * H * 2;
    static constexpr int DY = DZ + 2 * DZ_BYTES;                  // [128][16]
    static constexpr int SPLIT_END = DY + TM * 16 * 2;
    static constexpr int WIMG = FUSED ? FUSED_END : SPLIT_END;    // weight image
    static constexpr int W1B = H * DINP * 2, WHB = H * H * 2, W5B = 16 * H * 2;
    static constexpr int WIMG_BYTES = W1B + 3 * WHB + W5B;
    static constexpr int F32 = WIMG + WIMG_BYTES + (FUSED ? 0 : 4096);
    static constexpr int TSO = F32;                               // [2][128] sample depths (this tile, next tile)
    // [4][128] outputs / dL/dy; fused: in Z, which is dead from the previous
    // tile's last weight-gradient MMA until this tile's dZ4
    static constexpr int YB = FUSED ? Z : TSO + 2 * TM * 4;
    static constexpr int RAYS = FUSED ? TSO + 2 * TM * 4 : YB + 4 * TM * 4;   // [2][32][16] ray records
    static constexpr int LOSS = RAYS + 2 * RTMAX * RAYF * 4;      // [RTMAX][3] run loss sums per ray slot
    static constexpr int BIAS = LOSS + RTMAX * 3 * 4;             // [4][H] + [NOUT] f32 biases of the run's object
    static constexpr int MBAR = BIAS + (4 * H + 16) * 4;
    static constexpr int WBAR = MBAR + 8;                         // weight image loaded
    static constexpr int MBAR2 = WBAR + 8;                        // weight-gradient MMAs done
    static constexpr int TSLOT = MBAR2 + 8;
    static constexpr int BYTES = TSLOT + 8;
    static_assert(WIMG_BYTES % 16 == 0 && WIMG % 16 == 0, "bulk copy size and alignment");
    static_assert(!FUSED || ZC * 2 * TM >= 4 * TM * 4, "outputs fit in Z");
    // two CTAs per SM: 228 KB per SM, 1 KB reserved per CTA
    static_assert(CTAS * (BYTES + 1024) <= 233472, "shared memory of the CTAs of one SM");
};

__device__ __forceinline__ void st_bf16x8(unsigned char* tile, int off, const float (&v)[8]) {
    __nv_bfloat162 p[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4*>(tile + off) = *reinterpret_cast<uint4*>(p);
}
__device__ __forceinline__ void ld_bf16x8(const unsigned char* tile, int off, float (&v)[8]) {
    const uint4 u = *reinterpret_cast<const uint4*>(tile + off);
    const __nv_bfloat162* p = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(p[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

// sin / cos after reduction to [-pi, pi] (the hardware approximations are
// accurate there; the result is rounded to BF16 anyway)
__device__ __forceinline__ float red2pi(float p) {
    // nearest integer of t by adding and removing 1.5 * 2^23 (exact for |t| < 2^22,
    // ties to even like rintf), kept on the FMA pipe
    const float t = __fmul_rn(p, 0.15915494309189533577f);
    const float k = __fsub_rn(__fadd_rn(t, 12582912.f), 12582912.f);
    return fmaf(-6.28318530717958647692f, k, p);
}

// Encoding of one sample into row m of a [128][96] BF16 core-matrix tile:
// columns 0..2 x~, 3..47 sin(B x~), 48..92 cos(B x~), 93 one, 94..95 zero.
// The two threads of a sample split the 45 projections so that each owns
// whole 8-column core-matrix rows: half 0 takes angles 0..23 and writes
// columns 0..23 (x~, sin 0..20) and 48..71 (cos 0..23); half 1 takes angles
// 21..44 and writes columns 24..47 (sin 21..44) and 72..95 (cos 24..44, the
// one, padding). Each thread computes 24 projections and 45 sines/cosines;
// every feature index is a compile-time constant, so B is read as immediate
// constant-bank operands. gcopy (may be NULL) receives the same bytes.
__device__ __forceinline__ float enc_proj(const StepParams& sp, int j, float x0, float x1, float x2) {
    return red2pi(fmaf(sp.B[3 * j + 2], x2, fmaf(sp.B[3 * j + 1], x1, sp.B[3 * j] * x0)));
}
template <int CC>
__device__ __forceinline__ void enc_store(unsigned char* tile, unsigned char* gcopy, int m, int ch, const float (&v)[8]) {
    const int off = cm_off(m, ch * 8, CC);
    st_bf16x8(tile, off, v);
    if (gcopy) *reinterpret_cast<uint4*>(gcopy + off) = *reinterpret_cast<const uint4*>(tile + off);
}
// one half of a sample's row: angles J0 .. J0 + 23, sine columns of groups
// SG .. SG + 2 and cosine columns of groups CG .. CG + 2
template <int J0, int SG, int CG, int CC>
__device__ __forceinline__ void encode_half(const StepParams& sp, float x0, float x1, float x2, int m,
                                            unsigned char* tile, unsigned char* gcopy) {
    float pr[24];
#pragma unroll
    for (int j = 0; j < 24; ++j) pr[j] = enc_proj(sp, J0 + j, x0, x1, x2);
#pragma unroll
    for (int ch = SG; ch < SG + 3; ++ch) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = ch * 8 + u;   // column c < 3: x~; else the sine of angle c - 3
            v[u] = c == 0 ? x0 : c == 1 ? x1 : c == 2 ? x2 : __sinf(pr[c - 3 - J0]);
        }
        enc_store<CC>(tile, gcopy, m, ch, v);
    }
#pragma unroll
    for (int ch = CG; ch < CG + 3; ++ch) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = ch * 8 + u;   // cosine of angle c - 3 - NF, then the one and padding
            v[u] = c < DIN ? __cosf(pr[c - 3 - NF - J0]) : (c == DIN ? 1.f : 0.f);
        }
        enc_store<CC>(tile, gcopy, m, ch, v);
    }
}
// CC: column count of the tile the encoding occupies the first 96 columns of
template <int CC = DINP>
__device__ __forceinline__ void encode_row_half(const StepParams& sp, float x0, float x1, float x2, int m, int half,
                                                unsigned char* tile, unsigned char* gcopy) {
    static_assert(NF == 45 && DIN == 93 && DINP == 96, "feature split below assumes 45 Gaussian features");
    if (half == 0) encode_half<0, 0, 6, CC>(sp, x0, x1, x2, m, tile, gcopy);
    else encode_half<21, 3, 9, CC>(sp, x0, x1, x2, m, tile, gcopy);
}

struct Bf16Args {
    TileArgs t;
    const __nv_bfloat16* img;   // tensor-core weight images (arena)
    const long long* img_off;   // per object: element offset of its image
    int* err;                   // set to 1 when a bounded wait gives up
    long long polls;            // polls before an MMA or weight-copy wait gives up
    // 1: wait for the preceding grid at the start (launched behind the sampler,
    // or without programmatic serialization); 0: launched behind another tile
    // kernel, whose start already waited for the sampler: no wait at the start,
    // the wait comes before the CTA exits (so completions stay in stream order)
    int wait_first;
};

template <int H, int MODE>
__global__ void __launch_bounds__(NTHREADS, Bf16Cfg<H>::CTAS) k_tile_bf16(StepParams sp, Bf16Args ba) {
    using C = Bf16Cfg<H>;
    constexpr bool FUSED = C::FUSED;
    constexpr int CH = C::CH;
    constexpr bool GRAD = MODE == MODE_TRAIN;
    const TileArgs& ta = ba.t;
    extern __shared__ __align__(1024) unsigned char sm[];
    // fused layout
    unsigned char* Xt = sm + C::X;
    unsigned char* Hst = sm + C::HS;
    unsigned char* Zt = sm + C::Z;
    unsigned char* ZYt = sm + C::ZY;
    // split layout; tiles by index, computed (a pointer array indexed in a
    // loop would live in local memory)
    unsigned char* G0 = sm + C::G0;
    auto HAp = [&](int l) { return sm + C::HA + l * C::HA_BYTES; };
    auto DZp = [&](int i) { return sm + C::DZ + i * C::DZ_BYTES; };
    unsigned char* DYt = sm + C::DY;
    unsigned char* W1 = sm + C::WIMG;
    auto Whp = [&](int l) { return W1 + C::W1B + l * C::WHB; };
    unsigned char* W5 = W1 + C::W1B + 3 * C::WHB;
    float* yb = reinterpret_cast<float*>(sm + C::YB);
    float* lossacc = reinterpret_cast<float*>(sm + C::LOSS);
    float* bsm = reinterpret_cast<float*>(sm + C::BIAS);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + C::MBAR);
    uint64_t* wbar = reinterpret_cast<uint64_t*>(sm + C::WBAR);
    uint64_t* mbar2 = reinterpret_cast<uint64_t*>(sm + C::MBAR2);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + C::TSLOT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hf = warp >> 2;   // TMEM lane quadrant, column half
    const int row = q * 32 + lane;            // the sample (or fan-in lane) this thread reads

    // operand tile of the forward MMA of layer l (0: encoding, 1..4: h1..h4):
    // tile, its column count, first column
    auto fwd_a = [&](int l, int& cc, int& c0) -> unsigned char* {
        if constexpr (FUSED) {
            if (l == 0) { cc = C::XC; c0 = 0; return Xt; }
            if (l < 4) { cc = C::HSC; c0 = (l - 1) * H; return Hst; }
            cc = C::XC; c0 = DINP; return Xt;
        } else {
            if (l == 0) { cc = DINP; c0 = 0; return G0; }
            cc = CH; c0 = 0; return HAp(l - 1);
        }
    };

    // ---- set-up: barrier, tensor memory, constant columns ---------------------
    if (tid == 0) {
        mbar_init(mbar, 1);
        mbar_init(wbar, 1);
        mbar_init(mbar2, 1);
    }
    if (warp == 0) tmem_alloc(tslot, C::NCOLS);
    if constexpr (FUSED) {
        // the ones column of Hs (the bias lane of S2) and the zero columns after
        // it; the dY columns of ZY (the render rewrites the first 8 of each row)
        for (int r = tid; r < TM; r += blockDim.x) {
            float v[8] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            st_bf16x8(Hst, cm_off(r, C::ONES_HS, C::HSC), v);
            *reinterpret_cast<uint4*>(ZYt + cm_off(r, H, C::ZYC)) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(ZYt + cm_off(r, H + 8, C::ZYC)) = make_uint4(0u, 0u, 0u, 0u);
        }
    } else {
        for (int i = tid; i < 4 * TM; i += blockDim.x) {
            const int l = i / TM, r = i % TM;
            float v[8] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            st_bf16x8(HAp(l), cm_off(r, H, CH), v);   // column H = 1 (bias gradient lane)
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tl_lane = tmem + ((uint32_t)(q * 32) << 16);   // this warp's lane quadrant
    uint32_t phase = 0, wphase = 0, phase2 = 0;
    bool abort = false, wpend = false;   // wpend: a weight copy was issued and not yet seen complete
    // the ray records and depths of consecutive tiles alternate between two
    // buffers, so the next tile's are prefetched (cp.async) during this tile's forward
    bool pre_next = false;               // the next tile's rays and depths were prefetched
    int bufi = 1;
    bool dwpend = false;                 // the last tile's final weight-gradient MMAs were issued and not yet waited for
    int npick = 0;                       // pick of the next tile's ray `tid`

    // Every thread waits for an MMA commit by itself (no CTA barrier, so a
    // thread that has no epilogue share in a round is not waited for); a
    // wait that gave up is agreed on at the next CTA barrier, before any
    // further MMA is issued, so at most one commit per mbarrier is left
    // outstanding by a give-up: its parity is kept and drained before exit.
    bool wfail = false;
    bool lost1 = false, lost2 = false;   // this thread gave up on a commit of mbar / mbar2
    uint32_t lpar1 = 0, lpar2 = 0;
    auto wait_mma = [&]() {
        if (!mbar_wait(mbar, phase, ba.polls)) {
            wfail = true;
            lost1 = true;
            lpar1 = phase;
        }
        phase ^= 1;
        tc_fence_after();
    };
    auto wait_mma2 = [&]() {
        if (!mbar_wait(mbar2, phase2, ba.polls)) {
            wfail = true;
            lost2 = true;
            lpar2 = phase2;
        }
        phase2 ^= 1;
        tc_fence_after();
    };
    auto agree = [&]() {   // CTA barrier; every thread learns whether any wait gave up
        if (__syncthreads_or(wfail)) {
            abort = true;
            if (tid == 0) atomicExch(ba.err, 1);
        }
    };
    auto sync_for_mma = [&]() {   // smem operand writes and TMEM reads done -> MMA may start
        tmem_ld_wait();
        fence_async_smem();
        tc_fence_before();
        agree();
        tc_fence_after();
    };

    const long long n_tiles = *ta.n_tiles;
    const long long t0 = (long long)blockIdx.x * n_tiles / gridDim.x;
    const long long t1 = (long long)(blockIdx.x + 1) * n_tiles / gridDim.x;
    constexpr long long PC = param_count(H);

    auto flush_loss = [&](float* gp) {
        if (tid == 0) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;   // ray slots in order
            for (int r = 0; r < RTMAX; ++r) {
                s0 += lossacc[3 * r]; s1 += lossacc[3 * r + 1]; s2 += lossacc[3 * r + 2];
            }
            gp[PC + 0] = s0;
            gp[PC + 1] = s1;
            gp[PC + 2] = s2;
            gp[PC + 3] = 0.f;
            gp[PC + 4] = 0.f;
            gp[PC + 5] = 0.f;
        }
    };
    // flush a finished run: TMEM gradient accumulators and loss sums -> its slot
    auto flush_run = [&](long long part) {
        float* gp = ta.part + part;
        tc_fence_after();
        if constexpr (FUSED) {
            if (GRAD) {
                // Each warp loads (8 columns at a time, alternating with the other
                // warp of its lane quadrant, one wait) only the columns its lanes own.
                // S1 = X^T ZY: lane = X column (encoding 0..95 with the ones lane 93,
                // h4 from 96), column = ZY column (dZ1 0..H-1, dY H..H+15).
                {
                    float v[3][8];
                    const int ndz = q < 3 ? H / 16 : 0;          // dZ1 chunks of this thread
                    const bool dyc = q >= 2 && hf == 0;          // the dY chunk (lane 93, h4 lanes)
#pragma unroll
                    for (int j = 0; j < 2; ++j)
                        if (j < ndz) tmem_ld8(tl_lane + C::C_S1 + 8 * (hf + 2 * j), v[j]);
                    if (dyc) tmem_ld8(tl_lane + C::C_S1 + H, v[2]);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 2; ++j)
                        if (j < ndz) {
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const int col = 8 * (hf + 2 * j) + u;
                                if (row < DIN) gp[w_off(H, 0) + col * DIN + row] = v[j][u];    // dW1[n][in]
                                else if (row == DIN) gp[b_off(H, 0) + col] = v[j][u];          // b1
                            }
                        }
                    if (dyc) {
#pragma unroll
                        for (int o = 0; o < NOUT; ++o) {
                            if (row == DIN) gp[b_off(H, 4) + o] = v[2][o];                   // b5
                            else if (row >= DINP && row < DINP + H)
                                gp[w_off(H, 4) + o * H + (row - DINP)] = v[2][o];          // dW5[o][in]
                        }
                    }
                }
                // S2 = Hs^T Z: lane = Hs column (h1 | h2 | h3 | ones lane 3H), column = Z
                // column (dZ2 | dZ3 | dZ4); layer l's block is lanes and columns
                // l*H .. l*H + H - 1, the ones lane holds b2 | b3 | b4
                {
                    const int r0 = 32 * q, r1 = r0 + 32;
                    const bool bias_q = C::ONES_HS >= r0 && C::ONES_HS < r1;
                    const int wr1 = min(r1, C::ONES_HS);
                    const int lo = bias_q ? 0 : (r0 < C::ONES_HS ? (r0 / H) * H : 0);
                    const int hi = bias_q ? C::ONES_HS : (r0 < C::ONES_HS ? ((wr1 - 1) / H + 1) * H : 0);
#pragma unroll 1
                    for (int g = 0; g < 2; ++g) {   // up to 6 chunks per thread, 3 per wait
                        float v[3][8];
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            const int c8 = lo / 8 + hf + 2 * (3 * g + j);
                            if (8 * c8 < hi) tmem_ld8(tl_lane + C::C_S2 + 8 * c8, v[j]);
                        }
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            const int c8 = lo / 8 + hf + 2 * (3 * g + j);
                            if (8 * c8 < hi) {
#pragma unroll
                                for (int u = 0; u < 8; ++u) {
                                    const int col = 8 * c8 + u, lc = col / H;
                                    if (row == C::ONES_HS) gp[b_off(H, lc + 1) + col % H] = v[j][u];   // b2..b4
                                    else if (row / H == lc && row < C::ONES_HS)
                                        gp[w_off(H, lc + 1) + (col % H) * H + (row % H)] = v[j][u];    // dW2..4[n][in]
                                }
                            }
                        }
                    }
                }
            }
        } else {
            // dW1 (lanes = fan-in 0..95, lane 93 = bias)
#pragma unroll
            for (int c0 = 0; c0 < H / 2; c0 += 8) {
                float v[8];
                tmem_ld8(tl_lane + C::C_DW1 + hf * (H / 2) + c0, v);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = hf * (H / 2) + c0 + j;
                    if (row < DIN) gp[w_off(H, 0) + n * DIN + row] = v[j];
                    else if (row == DIN) gp[b_off(H, 0) + n] = v[j];
                }
            }
#pragma unroll
            for (int l = 1; l < 4; ++l) {
#pragma unroll
                for (int c0 = 0; c0 < H / 2; c0 += 8) {
                    float v[8];
                    tmem_ld8(tl_lane + C::C_DW1 + l * H + hf * (H / 2) + c0, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int n = hf * (H / 2) + c0 + j;
                        if (row < H) gp[w_off(H, l) + n * H + row] = v[j];
                        else if (row == H) gp[b_off(H, l) + n] = v[j];
                    }
                }
            }
            {
                float v[8];
                tmem_ld8(tl_lane + C::C_DW5 + hf * 8, v);
                tmem_ld_wait();
                if (hf == 0) {
#pragma unroll
                    for (int j = 0; j < NOUT; ++j) {
                        if (row < H) gp[w_off(H, 4) + j * H + row] = v[j];
                        else if (row == H) gp[b_off(H, 4) + j] = v[j];
                    }
                }
            }
        }
        flush_loss(gp);
    };

    // what a tile needs from the tile list and its object's records (two
    // dependent global loads): read for the next tile during this tile's forward
    struct TileHead {
        long long sbase, part, src_off, img_off;
        const float* P;
        float cx, cy, cz, sc, invR;
        int k, nr, ray0, S;
        bool first, last;
    };
    auto load_head = [&](long long tl) {
        TileHead h;
        const TileDev td = ta.tiles[tl];
        h.k = td.obj;
        h.nr = td.nr;
        h.ray0 = td.ray0;
        h.part = td.part;
        h.first = tl == t0 || ta.tiles[tl - 1].obj != h.k;
        h.last = tl + 1 == t1 || ta.tiles[tl + 1].obj != h.k;
        const ObjDev& o = ta.objs[h.k];
        const ObjBatch& b = ta.obs[h.k];
        h.S = o.S;
        h.sbase = b.sample_off + (long long)(td.ray0 - b.ray_off) * o.S;
        h.src_off = b.src_off;
        h.P = ta.params + o.param_off;
        h.cx = o.c[0];
        h.cy = o.c[1];
        h.cz = o.c[2];
        h.sc = o.scale;
        h.invR = 1.f / (float)b.R;
        h.img_off = ba.img_off[h.k];
        return h;
    };
    TileHead nxt{};
    bool have_nxt = false;
    if (t0 < t1) {   // the first tile's head reads only the batch layout
        nxt = load_head(t0);
        have_nxt = true;
    }
    // Launched behind the sampler (programmatic dependent launch), the kernel
    // has done its set-up so far; the sampler's picks and depths are complete
    // past this wait. Dependents are released only after it, so a kernel
    // launched behind this one (the next width class's, or the width-128
    // kernel, which read the sampler's output too) starts after the sampler's
    // completion; every CTA of this grid is resident once each has passed this
    // point. Launched behind another width class's tile kernel, whose CTAs all
    // passed that wait before this grid could start, the sampler is complete
    // already.
    if (ba.wait_first) pdl_wait();
    pdl_launch_dependents();

#pragma unroll 1
    for (long long tl = t0; tl < t1 && !abort; ++tl) {
        bufi ^= 1;
        const bool pre = pre_next;   // this tile's rays and depths were prefetched
        pre_next = false;
        float* tsm = reinterpret_cast<float*>(sm + C::TSO) + bufi * TM;
        float* rays = reinterpret_cast<float*>(sm + C::RAYS) + bufi * (RTMAX * RAYF);
        const TileHead th = have_nxt ? nxt : load_head(tl);
        have_nxt = false;
        const int k = th.k, nr = th.nr;
        const bool first = th.first, last = th.last;
        const int S = th.S, M = nr * S;
        const long long sbase = th.sbase;
        const float* P = th.P;
        const float cx = th.cx, cy = th.cy, cz = th.cz, sc = th.sc;
        const float isc = 1.f / sc;   // points are normalised by one multiply (within 1 ulp of dividing)

        // ---- rays, depths, points; weights at the start of a run ---------------
        // (after the first tile of a training range, the previous tile's
        // forward already started this tile's rays and depths by cp.async)
        if (!pre) {
            // depths in flight with the picks and records
            for (int i = tid; i < M; i += blockDim.x) tsm[i] = ta.tbuf[sbase + i];
            for (int r = tid; r < nr; r += blockDim.x) {
                const float* rec = ta.pool + (th.src_off + ta.pick[th.ray0 + r]) * REC;
                float* d = rays + r * RAYF;
#pragma unroll
                for (int u = 0; u < 11; ++u) d[u] = rec[u];
            }
        } else {
            cp_async_wait_all();
        }
        if (first) {
            // the weight image arrives by bulk copy while the tile is encoded
            if (tid == 0) {
                mbar_expect_tx(wbar, (uint32_t)C::WIMG_BYTES);
                bulk_load(W1, ba.img + th.img_off, (uint32_t)C::WIMG_BYTES, wbar);
                wpend = true;
            }
            for (int i = tid; i < 3 * RTMAX; i += blockDim.x) lossacc[i] = 0.f;
            // the object's biases, read by the epilogues from shared memory
            for (int i = tid; i < 4 * H + NOUT; i += blockDim.x) bsm[i] = P[b_off(H, i / H) + i % H];
        }
        __syncthreads();
        // the previous tile's last weight-gradient MMAs read the tiles rewritten
        // below: they ran during this tile's set-up above and must be done now
        auto wait_dw = [&]() {
            if constexpr (FUSED) {
                wait_mma2();
            } else {
                wait_mma();
                wait_mma2();
            }
            dwpend = false;
        };
        // ---- points and encoding (BF16; two threads per sample, each forms the
        // sample's normalised point itself) ----------------------------------------
        if (dwpend) wait_dw();
        for (int f = tid; f < 2 * TM; f += blockDim.x) {
            const int m = f % TM, half = f / TM;
            float x0 = 0.f, x1 = 0.f, x2 = 0.f;
            if (m < M) {
                const float* d = rays + (m / S) * RAYF;
                const float t = tsm[m];
                x0 = (fmaf(t, d[3], d[0]) - cx) * isc;
                x1 = (fmaf(t, d[4], d[1]) - cy) * isc;
                x2 = (fmaf(t, d[5], d[2]) - cz) * isc;
            }
            if constexpr (FUSED) encode_row_half<C::XC>(sp, x0, x1, x2, m, half, Xt, nullptr);
            else encode_row_half<DINP>(sp, x0, x1, x2, m, half, G0, nullptr);
        }
        sync_for_mma();
        if (abort) break;

        // ---- forward ------------------------------------------------------------
        if (first) {
            const bool ok = mbar_wait(wbar, wphase, ba.polls);
            if (__syncthreads_or(!ok)) {
                abort = true;
                if (tid == 0) atomicExch(ba.err, 1);
                break;
            }
            wphase ^= 1;
            wpend = false;
        }
        // layer 1: [128 x 96] x W1^T -> C_FWD
        if (warp == 0) {
            int cc, c0;
            unsigned char* a = fwd_a(0, cc, c0);
#pragma unroll
            for (int kc = 0; kc < DINP / 16; ++kc)
                mma_bf16_w(tmem + C::C_FWD, desc_kmajor(a, cc, c0 + 16 * kc), desc_kmajor(W1, DINP, 16 * kc),
                         idesc_bf16(TM, H, 0, 0), kc > 0);
            mma_commit_w(mbar);
        }
        constexpr int NC = H / 2;
        // the next tile of this range: its picks now, its rays and depths (into the
        // other buffers) once the picks have arrived
        const bool has_next = GRAD && tl + 1 < t1;
        if (has_next) {
            nxt = load_head(tl + 1);
            have_nxt = true;
            if (tid < nxt.nr) npick = ta.pick[nxt.ray0 + tid];
        }
        wait_mma();
        if (abort) break;
        if (has_next) {
            float* rays_n = reinterpret_cast<float*>(sm + C::RAYS) + (bufi ^ 1) * (RTMAX * RAYF);
            float* tsm_n = reinterpret_cast<float*>(sm + C::TSO) + (bufi ^ 1) * TM;
            if (tid < nxt.nr) {
                const float* rec = ta.pool + (nxt.src_off + npick) * REC;
                float* d = rays_n + tid * RAYF;
                cp_async16(d, rec);
                cp_async16(d + 4, rec + 4);
                cp_async16(d + 8, rec + 8);
            }
            if (tid < nxt.nr * nxt.S) cp_async4(tsm_n + tid, ta.tbuf + nxt.sbase + tid);
            cp_async_commit();
            pre_next = true;
        }
#pragma unroll 1
        for (int l = 0; l < 4; ++l) {
            // epilogue of layer l + 1: bias, ReLU, BF16 -> the operand tile of h_{l+1}
            {
                int cc, cb;
                unsigned char* ht = fwd_a(l + 1, cc, cb);
                float v[NC];
                tmem_ld_cols<NC>(tl_lane + C::C_FWD + hf * NC, v);
#pragma unroll
                for (int c0 = 0; c0 < NC; c0 += 8) {
                    float u[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) u[j] = fmaxf(v[c0 + j] + bsm[l * H + hf * NC + c0 + j], 0.f);
                    st_bf16x8(ht, cm_off(row, cb + hf * NC + c0, cc), u);
                }
            }
            sync_for_mma();
            if (abort) break;
            if (warp == 0) {
                int cc, cb;
                unsigned char* a = fwd_a(l + 1, cc, cb);
                if (l < 3) {
#pragma unroll
                    for (int kc = 0; kc < H / 16; ++kc)
                        mma_bf16_w(tmem + C::C_FWD, desc_kmajor(a, cc, cb + 16 * kc), desc_kmajor(Whp(l), H, 16 * kc),
                                 idesc_bf16(TM, H, 0, 0), kc > 0);
                } else {
#pragma unroll
                    for (int kc = 0; kc < H / 16; ++kc)
                        mma_bf16_w(tmem + C::C_FWD, desc_kmajor(a, cc, cb + 16 * kc), desc_kmajor(W5, H, 16 * kc),
                                 idesc_bf16(TM, 16, 0, 0), kc > 0);
                }
                mma_commit_w(mbar);
            }
            wait_mma();
            if (abort) break;
        }
        if (abort) break;
        // layer-5 epilogue: y = acc + b5 -> yb (FP32, feature-major)
        {
            float v[8];
            tmem_ld8(tl_lane + C::C_FWD + hf * 8, v);
            tmem_ld_wait();
            if (hf == 0) {
                const float* b5 = bsm + 4 * H;
#pragma unroll
                for (int j = 0; j < NOUT; ++j) yb[j * TM + row] = sigmoidf_(v[j] + b5[j]);   // o, c (Eq. 1 heads)
            }
        }
        agree();
        if (abort) break;

        // ---- rendering, loss, dL/dy (FP32) ----------------------------------------
        const float invR = th.invR;
        for (int r = warp; r < nr; r += NTHREADS / 32) {
            float* d = rays + r * RAYF;
            // fused: each sample's dL/dy goes straight to its row of the dY columns of ZY
            if constexpr (FUSED) render_ray_warp<GRAD, TM, true>(sp, yb, tsm, d, r, S, invR, GRAD ? ZYt : nullptr,
                                                                 C::ZYC, H);
            else render_ray_warp<GRAD, TM, true>(sp, yb, tsm, d, r, S, invR);
            // the ray's loss terms join its slot's run sums (lane 0 wrote them)
            if (lane == 0) {
                lossacc[3 * r] += d[13]; lossacc[3 * r + 1] += d[14]; lossacc[3 * r + 2] += d[15];
            }
        }
        if constexpr (FUSED) {
            if (GRAD)   // rows past the tile's samples: zero dL/dy
                for (int m = M + tid; m < TM; m += blockDim.x)
                    *reinterpret_cast<uint4*>(ZYt + cm_off(m, H, C::ZYC)) = make_uint4(0u, 0u, 0u, 0u);
        } else {
            for (int m = M + tid; m < TM; m += blockDim.x) {
                yb[m] = 0.f; yb[TM + m] = 0.f; yb[2 * TM + m] = 0.f; yb[3 * TM + m] = 0.f;
            }
        }
        if (!GRAD) __syncthreads();
        if (!GRAD) {
            __syncthreads();
            if (last) {
                if constexpr (FUSED) flush_loss(ta.part + th.part);
                else flush_run(th.part);
            }
            __syncthreads();
            continue;
        }
        // split: dY -> BF16 [128][16] (columns 4..15 zero)
        if constexpr (!FUSED) {
            __syncthreads();
            for (int m = tid; m < TM * 2; m += blockDim.x) {
                const int r = m % TM, half = m / TM;
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = (half == 0 && j < NOUT) ? yb[j * TM + r] : 0.f;
                st_bf16x8(DYt, cm_off(r, half * 8, 16), v);
            }
        }
        sync_for_mma();
        if (abort) break;

        // ---- backward -------------------------------------------------------------
        // The input-gradient chain dZ4 -> dZ3 -> dZ2 -> dZ1 is the critical path:
        // each round commits its input-gradient MMA alone. Issuing eight MMAs
        // holds thread 0 for hundreds of cycles, so in a round that follows such
        // an issue warp 0 has no epilogue share: warp 4 (the same TMEM lane
        // quadrant) takes both column halves.
        // dZ = acc * [a > 0] (a: BF16 activations at column ac0 of tile `at`,
        // acc columns 0..H-1 of C_DX) -> column zc0 of tile `zt`
        auto dx_epi = [&](const unsigned char* at, int acc_, int ac0, unsigned char* zt, int zcc, int zc0,
                          bool shift) {
            if (shift && warp == 0) return;
            const int nh = shift && warp == 4 ? 2 : 1;
#pragma unroll 1
            for (int hh = 0; hh < nh; ++hh) {
                const int h2 = nh == 2 ? hh : hf;
                float v[NC];
                tmem_ld_cols<NC>(tl_lane + C::C_DX + h2 * NC, v);
#pragma unroll
                for (int c0 = 0; c0 < NC; c0 += 8) {
                    float a[8], u[8];
                    ld_bf16x8(at, cm_off(row, ac0 + h2 * NC + c0, acc_), a);
#pragma unroll
                    for (int j = 0; j < 8; ++j) u[j] = a[j] > 0.f ? v[c0 + j] : 0.f;
                    st_bf16x8(zt, cm_off(row, zc0 + h2 * NC + c0, zcc), u);
                }
            }
        };
        // C_DX = dZ W (dZ at column z0 of tile z with zcc columns; W MN-major)
        auto issue_dx = [&](const unsigned char* z, int zcc, int z0, const unsigned char* w) {
#pragma unroll
            for (int kc = 0; kc < H / 16; ++kc)
                mma_bf16_w(tmem + C::C_DX, desc_kmajor(z, zcc, z0 + 16 * kc), desc_mnmajor(w, H, 16 * kc),
                         idesc_bf16(TM, H, 0, 1), kc > 0);
            mma_commit_w(mbar);
        };
        // dW^T [fan-in lanes][n] += a^T z over the tile's samples
        auto issue_dw = [&](int col, const unsigned char* a, int acc_, const unsigned char* z, int zcc, int n) {
#pragma unroll
            for (int kc = 0; kc < TM / 16; ++kc)
                mma_bf16_w(tmem + col, desc_mnmajor(a, acc_, 16 * kc), desc_mnmajor(z, zcc, 16 * kc),
                         idesc_bf16(TM, n, 1, 1), !first || kc > 0);
        };
        if constexpr (FUSED) {
            // layer 5: dY W5
            if (warp == 0) {
                mma_bf16_w(tmem + C::C_DX, desc_kmajor(ZYt, C::ZYC, H), desc_mnmajor(W5, H, 0), idesc_bf16(TM, H, 0, 1),
                         false);
                mma_commit_w(mbar);
            }
            wait_mma();
            dx_epi(Xt, C::XC, DINP, Zt, C::ZC, 2 * H, false);           // dZ4 = . * [h4 > 0]
            sync_for_mma();
            if (abort) break;
            if (warp == 0) issue_dx(Zt, C::ZC, 2 * H, Whp(2));           // dZ4 W4
            wait_mma();
            dx_epi(Hst, C::HSC, 2 * H, Zt, C::ZC, H, false);            // dZ3 = . * [h3 > 0]
            sync_for_mma();
            if (abort) break;
            if (warp == 0) issue_dx(Zt, C::ZC, H, Whp(1));               // dZ3 W3
            wait_mma();
            dx_epi(Hst, C::HSC, H, Zt, C::ZC, 0, false);                // dZ2 = . * [h2 > 0]
            sync_for_mma();
            if (abort) break;
            if (warp == 0) {
                issue_dx(Zt, C::ZC, 0, Whp(0));                         // dZ2 W2
                issue_dw(C::C_S2, Hst, C::HSC, Zt, C::ZC, C::ZC);       // S2 += Hs^T [dZ2 | dZ3 | dZ4]
            }
            wait_mma();
            dx_epi(Hst, C::HSC, 0, ZYt, C::ZYC, 0, true);               // dZ1 = . * [h1 > 0]
            sync_for_mma();
            if (abort) break;
            if (warp == 0) {
                issue_dw(C::C_S1, Xt, C::XC, ZYt, C::ZYC, C::ZYC);      // S1 += [enc | h4]^T [dZ1 | dY]
                mma_commit_w(mbar2);                                      // (also covers S2's MMAs)
            }
        } else {
            // dZ_l = acc * [h_l > 0] (h_l in HA[l - 1]) -> dst with zcc columns
            // Buffers: dZ4 -> DZ[0], dZ3 -> DZ[1], dZ2 -> HA[3] (h4 is dead once dW5
            // has run), dZ1 -> DZ[0] (dZ4 is dead once dW4 has run); a commit tracks
            // every earlier MMA of its thread, so each rewritten buffer's last reader
            // has finished. Each round commits its input-gradient MMA alone and then
            // issues the previous layer's weight-gradient MMAs behind it; in the last
            // round thread 0 feeds dW2 and thread 128 feeds dW1 (each accumulator
            // always from the same thread, in order).
            if (warp == 0) {
                mma_bf16_w(tmem + C::C_DX, desc_kmajor(DYt, 16, 0), desc_mnmajor(W5, H, 0), idesc_bf16(TM, H, 0, 1),
                         false);
                mma_commit_w(mbar);
            }
            wait_mma();
            dx_epi(HAp(3), CH, 0, DZp(0), H, 0, false);                  // dZ4
            sync_for_mma();
            if (abort) break;
            if (warp == 0) {
                issue_dx(DZp(0), H, 0, Whp(2));                          // dZ4 W4
                issue_dw(C::C_DW5, HAp(3), CH, DYt, 16, 16);             // dW5^T += h4^T dY
            }
            wait_mma();
            dx_epi(HAp(2), CH, 0, DZp(1), H, 0, true);                   // dZ3
            sync_for_mma();
            if (abort) break;
            if (warp == 0) {
                issue_dx(DZp(1), H, 0, Whp(1));                          // dZ3 W3
                issue_dw(C::C_DW1 + 3 * H, HAp(2), CH, DZp(0), H, H);     // dW4^T += h3^T dZ4
            }
            wait_mma();
            dx_epi(HAp(1), CH, 0, HAp(3), CH, 0, true);                  // dZ2
            sync_for_mma();
            if (abort) break;
            if (warp == 0) {
                issue_dx(HAp(3), CH, 0, Whp(0));                         // dZ2 W2
                issue_dw(C::C_DW1 + 2 * H, HAp(1), CH, DZp(1), H, H);     // dW3^T += h2^T dZ3
            }
            wait_mma();
            dx_epi(HAp(0), CH, 0, DZp(0), H, 0, true);                   // dZ1
            sync_for_mma();
            if (abort) break;
            if (warp == 0) {
                issue_dw(C::C_DW1 + H, HAp(0), CH, HAp(3), CH, H);        // dW2^T += h1^T dZ2
                mma_commit_w(mbar);
            } else if (warp == 4) {
                issue_dw(C::C_DW1, G0, DINP, DZp(0), H, H);              // dW1^T += enc^T dZ1
                mma_commit_w(mbar2);
            }
        }
        dwpend = true;
        if (last) {   // the run's gradient leaves TMEM: wait for its last MMAs now
            wait_dw();
            agree();
            if (abort) break;
            flush_run(th.part);
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    // Drain before tensor memory is freed: the range's last tile ends a run, so
    // nothing is pending unless a wait gave up; then the commit given up on,
    // weight-gradient MMAs issued before the give-up was agreed on, and a weight
    // copy still in flight are waited for (bounded; they were issued, so they end).
    if (lost1) mbar_wait(mbar, lpar1, DRAIN_POLLS);
    if (lost2) mbar_wait(mbar2, lpar2, DRAIN_POLLS);
    if (dwpend) {
        if (!FUSED) mbar_wait(mbar, phase, DRAIN_POLLS);
        mbar_wait(mbar2, phase2, DRAIN_POLLS);
    }
    if (wpend) mbar_wait(wbar, wphase, DRAIN_POLLS);
    cp_async_wait_all();   // prefetches issued before an abort land before the CTA exits
    // behind another tile kernel: complete only after it (what follows in the
    // stream waits for this grid alone and must see both)
    if (!ba.wait_first) pdl_wait();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, C::NCOLS);
}

// rebuild an object's tensor-core weight image from its canonical parameters
__global__ void k_image(const float* __restrict__ params, __nv_bfloat16* img, int H) {
    const long long n = img_count(H);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        img[i] = __float2bfloat16(0.f);
    __syncthreads();   // single-block launch: zero fill, then scatter
    const long long P = param_count(H);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const long long w = img_index(H, p);
        if (w >= 0) img[w] = __float2bfloat16(params[p]);
    }
}

}  // namespace vmapk
