// Warm-start set-encoder hypernetwork: forward, backward and Adam on the GPU.
//
// From N points (x~, occupancy, rgb) of a newly seen object's first keyframe,
// predict the object MLP's initial weights:
//   per point  h1 = ReLU(W1 x + b1), h2 = ReLU(W2 h1 + b2), h3 = ReLU(W3 h2 + b3)
//   per set    z = channel-wise max of h3 over the points (ties: lowest index)
//   head       u = Wa z + ba (rank r), theta = Wb u + bb (P outputs)
//   loss       L = sum (theta - target)^2 / (B P)
// In FP32 mode every GEMM is a tiled FP32 SIMT kernel (64 x 64 tiles, 4 x 4
// per thread, split over K where the reduction is long). In BF16 mode the six
// GEMMs of the 128-wide shared layers (two forward layers, their input and
// weight gradients) run on the tensor cores (vmap_hgemm.cuh: BF16 operands,
// FP32 accumulation); the 7-input first layer and the rank-16 head stay FP32.
// Column sums and split partials are added in a fixed order, so results are
// bitwise reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/vmap.h"
#include "vmap_hgemm.cuh"

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias, ReLU); A(m,k) = TA ? A[k lda + m] : A[m lda + k],
// B(k,n) = TB ? B[n ldb + k] : B[k ldb + n]. gridDim.z splits K into chunks of kchunk; split z
// writes C + z * M * ldc (no epilogue then).
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                               const float* __restrict__ bias, int kchunk) {
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += BK) {
        for (int i = tid; i < BK * BM; i += 256) {
            const int kk = i / BM, mm = i % BM;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < ke) ? (TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : 0.f;
        }
        for (int i = tid; i < BK * BN; i += 256) {
            const int kk = i / BN, nn = i % BN;
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < N && k < ke) ? (TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* Cz = C + (long long)blockIdx.z * M * ldc;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                float v = acc[i][j];
                if (EPI >= 1) v += bias[n];
                if (EPI == 2) v = fmaxf(v, 0.f);
                Cz[(long long)m * ldc + n] = v;
            }
        }
}

// out[m][n] = sum_z part[z][m][n] (z in order) (+ bias)
__global__ void k_sum_splits(int M, int N, int Z, const float* __restrict__ part, float* __restrict__ out,
                             const float* __restrict__ bias) {
    const long long total = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int z = 0; z < Z; ++z) v += part[z * total + i];
        if (bias) v += bias[i % N];
        out[i] = v;
    }
}

// column sums in two fixed-order passes: part[c][n] = sum of rows in chunk c; out[n] = sum_c part[c][n]
constexpr int COL_CHUNKS = 64;
__global__ void k_colsum_part(int M, int N, const float* __restrict__ A, float* __restrict__ part) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
    if (n >= N) return;
    const int r0 = (int)((long long)c * M / COL_CHUNKS), r1 = (int)((long long)(c + 1) * M / COL_CHUNKS);
    float v = 0.f;
    for (int r = r0; r < r1; ++r) v += A[(long long)r * N + n];
    part[c * N + n] = v;
}
__global__ void k_colsum_fin(int N, const float* __restrict__ part, float* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float v = 0.f;
    for (int c = 0; c < COL_CHUNKS; ++c) v += part[c * N + n];
    out[n] = v;
}

// z[b][c] = max_i h[b N + i][c], arg = first index reaching it
__global__ void k_maxpool(int B, int N, int W, const float* __restrict__ h, float* __restrict__ z, int* __restrict__ arg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * W) return;
    const int b = i / W, c = i % W;
    float best = h[(long long)b * N * W + c];
    int bi = 0;
    for (int p = 1; p < N; ++p) {
        const float v = h[((long long)b * N + p) * W + c];
        if (v > best) { best = v; bi = p; }
    }
    z[i] = best;
    arg[i] = bi;
}

// dz3 = scatter(dz by arg) * [h3 > 0]
__global__ void k_unpool(int B, int N, int W, const float* __restrict__ dz, const int* __restrict__ arg,
                         const float* __restrict__ h3, float* __restrict__ d) {
    const long long total = (long long)B * N * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % W);
        const long long row = i / W;
        const int b = (int)(row / N), p = (int)(row % N);
        d[i] = (arg[b * W + c] == p && h3[i] > 0.f) ? dz[b * W + c] : 0.f;
    }
}

__global__ void k_relu_mask(long long n, float* __restrict__ d, const float* __restrict__ a) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(a[i] > 0.f)) d[i] = 0.f;
}

// dth = 2 (theta - target) / n, per-block partial sums of the squared error
__global__ void __launch_bounds__(256) k_mse(long long n, const float* __restrict__ th, const float* __restrict__ tg,
                                             float* __restrict__ dth, float* __restrict__ part) {
    __shared__ float sh[256];
    float s = 0.f;
    const float sc = 2.f / (float)n;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
        const float d = th[i] - tg[i];
        s = fmaf(d, d, s);
        dth[i] = sc * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void k_mse_fin(int nb, long long n, const float* __restrict__ part, float* __restrict__ loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < nb; ++i) s += part[i];
        *loss = s / (float)n;
    }
}

__global__ void k_adam_flat(long long n, float* p, const float* __restrict__ g, float* m, float* v, float lr,
                            float b1, float b2, float eps, float bc1, float bc2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// seeded init: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a 64-bit mixing hash of (seed, index)
__global__ void k_hyper_init(long long n, float* p, const long long* __restrict__ bounds, const int* __restrict__ fan,
                             int nseg, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int s = 0;
        while (s + 1 < nseg && i >= bounds[s + 1]) ++s;
        unsigned long long x = seed ^ (0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1));
        x ^= x >> 30; x *= 0xBF58476D1CE4E5B9ull; x ^= x >> 27; x *= 0x94D049BB133111EBull; x ^= x >> 31;
        const float u = (float)((x >> 40) + 0.5) * (1.0f / 16777216.0f);
        p[i] = (2.f * u - 1.f) / sqrtf((float)fan[s]);
    }
}

}  // namespace

struct vmap_hyper {
    int N = 256, W = 128, R = 16, P = 6308, D = 7, max_batch = 0;
    cudaStream_t stream = nullptr;
    long long n_params = 0;
    long long off[10] = {0};
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    int step = 0;
    float *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *da = nullptr, *db = nullptr;
    int* arg = nullptr;
    float *z = nullptr, *u = nullptr, *th = nullptr, *dth = nullptr, *du = nullptr, *dz = nullptr;
    float *split = nullptr, *colpart = nullptr, *mse_part = nullptr, *loss_tmp = nullptr;
    long long *seg_bounds = nullptr;
    int* seg_fan = nullptr;
    int bf16 = 0;                      // tensor-core GEMMs for the 128-wide layers
    float* tc_part = nullptr;          // [n_sm][128][128] split-K partials of the tensor-core weight gradients
    int* err_d = nullptr;              // set when a bounded MMA wait gives up
    int n_sm = 148;
    std::string err;
};

namespace {

constexpr int SPLIT_MAX = 32;
constexpr int MSE_BLOCKS = 256;

vmap_status hfail(vmap_hyper* h, vmap_status s, const char* fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    return s;
}

#define HCU(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return hfail(h, VMAP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <bool B_MN, int EPI>
cudaError_t launch_hgemm_rows(vmap_hyper* h, long long M, const float* A, const float* B, const float* bias, float* C) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(vmapk::k_hgemm_rows<B_MN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)vmapk::HgemmSmem::BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    vmapk::k_hgemm_rows<B_MN, EPI><<<(unsigned)((M + 127) / 128), 128, vmapk::HgemmSmem::BYTES, h->stream>>>(
        M, A, B, bias, C, h->err_d);
    return cudaGetLastError();
}

// tensor-core forms: C[M][128] = A[M][128] W^T (TB) or A W (!TB), and dW[128][128] = A^T B over K rows
template <bool TA, bool TB>
bool tc_shape(vmap_hyper* h, int M, int N, int K, int lda, int ldb) {
    if (!h->bf16) return false;
    if (!TA) return N == vmapk::HG && K == vmapk::HG && lda == vmapk::HG && ldb == vmapk::HG;
    return !TB && M == vmapk::HG && N == vmapk::HG && lda == vmapk::HG && ldb == vmapk::HG;
}

template <bool TA, bool TB>
vmap_status gemm_tc(vmap_hyper* h, int M, int N, int K, const float* A, const float* B, float* C, const float* bias,
                    bool relu) {
    cudaError_t e;
    if (!TA) {
        if (TB) e = relu ? launch_hgemm_rows<false, 2>(h, M, A, B, bias, C)
                        : bias ? launch_hgemm_rows<false, 1>(h, M, A, B, bias, C)
                               : launch_hgemm_rows<false, 0>(h, M, A, B, nullptr, C);
        else e = launch_hgemm_rows<true, 0>(h, M, A, B, nullptr, C);
    } else {
        static bool attr = false;
        if (!attr) {
            e = cudaFuncSetAttribute(vmapk::k_hgemm_tn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)vmapk::HgemmSmem::BYTES);
            if (e != cudaSuccess) return hfail(h, VMAP_ERR_CUDA, "hgemm attribute: %s", cudaGetErrorString(e));
            attr = true;
        }
        const long long per = ((long long)K + h->n_sm - 1) / h->n_sm;
        const long long chunk = std::max<long long>(vmapk::HG, (per + vmapk::HG - 1) / vmapk::HG * vmapk::HG);
        const int splits = (int)((K + chunk - 1) / chunk);
        vmapk::k_hgemm_tn<<<splits, 128, vmapk::HgemmSmem::BYTES, h->stream>>>(K, chunk, A, B, h->tc_part, h->err_d);
        k_sum_splits<<<256, 256, 0, h->stream>>>(vmapk::HG, vmapk::HG, splits, h->tc_part, C, bias);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return hfail(h, VMAP_ERR_CUDA, "tensor-core GEMM: %s", cudaGetErrorString(e));
    return VMAP_OK;
}

// C = op(A) op(B) (+bias, ReLU); long reductions are split over K and summed in order
template <bool TA, bool TB>
vmap_status gemm(vmap_hyper* h, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                 const float* bias, bool relu) {
    if (tc_shape<TA, TB>(h, M, N, K, lda, ldb)) return gemm_tc<TA, TB>(h, M, N, K, A, B, C, bias, relu);
    const dim3 blk(256);
    const int gm = (M + BM - 1) / BM, gn = (N + BN - 1) / BN;
    int splits = 1;
    if ((long long)gm * gn < 148 && K > 256) splits = std::min(SPLIT_MAX, std::max(1, K / 256));
    if (splits == 1) {
        const dim3 grid(gn, gm, 1);
        if (relu) k_sgemm<TA, TB, 2><<<grid, blk, 0, h->stream>>>(M, N, K, A, lda, B, ldb, C, N, bias, K);
        else if (bias) k_sgemm<TA, TB, 1><<<grid, blk, 0, h->stream>>>(M, N, K, A, lda, B, ldb, C, N, bias, K);
        else k_sgemm<TA, TB, 0><<<grid, blk, 0, h->stream>>>(M, N, K, A, lda, B, ldb, C, N, nullptr, K);
    } else {
        const int kchunk = ((K + splits - 1) / splits + BK - 1) / BK * BK;
        splits = (K + kchunk - 1) / kchunk;
        const dim3 grid(gn, gm, splits);
        k_sgemm<TA, TB, 0><<<grid, blk, 0, h->stream>>>(M, N, K, A, lda, B, ldb, h->split, N, nullptr, kchunk);
        k_sum_splits<<<256, 256, 0, h->stream>>>(M, N, splits, h->split, C, bias);
        if (relu) k_relu_mask<<<256, 256, 0, h->stream>>>((long long)M * N, C, C);
    }
    HCU(cudaGetLastError());
    return VMAP_OK;
}

vmap_status colsum(vmap_hyper* h, int M, int N, const float* A, float* out) {
    k_colsum_part<<<dim3((N + 255) / 256, COL_CHUNKS), 256, 0, h->stream>>>(M, N, A, h->colpart);
    k_colsum_fin<<<(N + 255) / 256, 256, 0, h->stream>>>(N, h->colpart, out);
    HCU(cudaGetLastError());
    return VMAP_OK;
}

vmap_status check_batch(vmap_hyper* h, int batch, const void* X) {
    if (!h || !X) return VMAP_ERR_ARG;
    if (batch < 1) return hfail(h, VMAP_ERR_ARG, "batch must be >= 1");
    if (batch > h->max_batch) return hfail(h, VMAP_ERR_CAPACITY, "batch %d exceeds max_batch %d", batch, h->max_batch);
    return VMAP_OK;
}

vmap_status forward(vmap_hyper* h, int B, const float* X) {
    const float* p = h->params;
    const int rows = B * h->N;
    if (vmap_status s = gemm<false, true>(h, rows, h->W, h->D, X, h->D, p + h->off[0], h->D, h->h1, p + h->off[1], true)) return s;
    if (vmap_status s = gemm<false, true>(h, rows, h->W, h->W, h->h1, h->W, p + h->off[2], h->W, h->h2, p + h->off[3], true)) return s;
    if (vmap_status s = gemm<false, true>(h, rows, h->W, h->W, h->h2, h->W, p + h->off[4], h->W, h->h3, p + h->off[5], true)) return s;
    k_maxpool<<<(B * h->W + 255) / 256, 256, 0, h->stream>>>(B, h->N, h->W, h->h3, h->z, h->arg);
    if (vmap_status s = gemm<false, true>(h, B, h->R, h->W, h->z, h->W, p + h->off[6], h->W, h->u, p + h->off[7], false)) return s;
    return gemm<false, true>(h, B, h->P, h->R, h->u, h->R, p + h->off[8], h->R, h->th, p + h->off[9], false);
}

vmap_status backward(vmap_hyper* h, int B, const float* X, const float* T, float* loss) {
    const float* p = h->params;
    float* g = h->grad;
    const long long nth = (long long)B * h->P;
    const int rows = B * h->N;
    k_mse<<<MSE_BLOCKS, 256, 0, h->stream>>>(nth, h->th, T, h->dth, h->mse_part);
    k_mse_fin<<<1, 32, 0, h->stream>>>(MSE_BLOCKS, nth, h->mse_part, loss ? loss : h->loss_tmp);
    // head
    if (vmap_status s = gemm<true, false>(h, h->P, h->R, B, h->dth, h->P, h->u, h->R, g + h->off[8], nullptr, false)) return s;
    if (vmap_status s = colsum(h, B, h->P, h->dth, g + h->off[9])) return s;
    if (vmap_status s = gemm<false, false>(h, B, h->R, h->P, h->dth, h->P, p + h->off[8], h->R, h->du, nullptr, false)) return s;
    if (vmap_status s = gemm<true, false>(h, h->R, h->W, B, h->du, h->R, h->z, h->W, g + h->off[6], nullptr, false)) return s;
    if (vmap_status s = colsum(h, B, h->R, h->du, g + h->off[7])) return s;
    if (vmap_status s = gemm<false, false>(h, B, h->W, h->R, h->du, h->R, p + h->off[6], h->W, h->dz, nullptr, false)) return s;
    // max-pool, then the shared per-point layers
    k_unpool<<<512, 256, 0, h->stream>>>(B, h->N, h->W, h->dz, h->arg, h->h3, h->da);
    // layer 3
    if (vmap_status s = gemm<true, false>(h, h->W, h->W, rows, h->da, h->W, h->h2, h->W, g + h->off[4], nullptr, false)) return s;
    if (vmap_status s = colsum(h, rows, h->W, h->da, g + h->off[5])) return s;
    if (vmap_status s = gemm<false, false>(h, rows, h->W, h->W, h->da, h->W, p + h->off[4], h->W, h->db, nullptr, false)) return s;
    k_relu_mask<<<512, 256, 0, h->stream>>>((long long)rows * h->W, h->db, h->h2);
    // layer 2
    if (vmap_status s = gemm<true, false>(h, h->W, h->W, rows, h->db, h->W, h->h1, h->W, g + h->off[2], nullptr, false)) return s;
    if (vmap_status s = colsum(h, rows, h->W, h->db, g + h->off[3])) return s;
    if (vmap_status s = gemm<false, false>(h, rows, h->W, h->W, h->db, h->W, p + h->off[2], h->W, h->da, nullptr, false)) return s;
    k_relu_mask<<<512, 256, 0, h->stream>>>((long long)rows * h->W, h->da, h->h1);
    // layer 1
    if (vmap_status s = gemm<true, false>(h, h->W, h->D, rows, h->da, h->W, X, h->D, g + h->off[0], nullptr, false)) return s;
    if (vmap_status s = colsum(h, rows, h->W, h->da, g + h->off[1])) return s;
    HCU(cudaGetLastError());
    return VMAP_OK;
}

}  // namespace

extern "C" {

vmap_status vmap_hyper_create(vmap_hyper** out, int n_points, int width, int rank, int hidden, int max_batch,
                              unsigned long long seed, void* cuda_stream) {
    if (!out) return VMAP_ERR_ARG;
    *out = nullptr;
    if (n_points < 1 || width < 1 || rank < 1 || max_batch < 1) return VMAP_ERR_ARG;
    if (hidden != 16 && hidden != 32 && hidden != 64 && hidden != 128) return VMAP_ERR_ARG;
    vmap_hyper* h = new vmap_hyper();
    h->N = n_points;
    h->W = width;
    h->R = rank;
    h->P = (int)(93LL * hidden + hidden + 3LL * (hidden * hidden + hidden) + 4LL * hidden + 4);
    h->max_batch = max_batch;
    h->stream = (cudaStream_t)cuda_stream;
    const long long sizes[10] = {(long long)h->W * h->D, h->W, (long long)h->W * h->W, h->W, (long long)h->W * h->W,
                                 h->W, (long long)h->R * h->W, h->R, (long long)h->P * h->R, h->P};
    const int fans[10] = {h->D, h->D, h->W, h->W, h->W, h->W, h->W, h->W, h->R, h->R};
    long long o = 0;
    for (int i = 0; i < 10; ++i) {
        h->off[i] = o;
        o += sizes[i];
    }
    h->n_params = o;
    const long long rows = (long long)max_batch * n_points;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** pp, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(pp, bytes);
    };
    alloc((void**)&h->params, sizeof(float) * o);
    alloc((void**)&h->grad, sizeof(float) * o);
    alloc((void**)&h->m, sizeof(float) * o);
    alloc((void**)&h->v, sizeof(float) * o);
    alloc((void**)&h->h1, sizeof(float) * rows * width);
    alloc((void**)&h->h2, sizeof(float) * rows * width);
    alloc((void**)&h->h3, sizeof(float) * rows * width);
    alloc((void**)&h->da, sizeof(float) * rows * width);
    alloc((void**)&h->db, sizeof(float) * rows * width);
    alloc((void**)&h->arg, sizeof(int) * max_batch * width);
    alloc((void**)&h->z, sizeof(float) * max_batch * width);
    alloc((void**)&h->u, sizeof(float) * max_batch * rank);
    alloc((void**)&h->th, sizeof(float) * (long long)max_batch * h->P);
    alloc((void**)&h->dth, sizeof(float) * (long long)max_batch * h->P);
    alloc((void**)&h->du, sizeof(float) * max_batch * rank);
    alloc((void**)&h->dz, sizeof(float) * max_batch * width);
    const long long split_elems = SPLIT_MAX * std::max<long long>({(long long)width * width, (long long)h->P * rank,
                                                                   (long long)max_batch * width, (long long)width * 8});
    alloc((void**)&h->split, sizeof(float) * split_elems);
    alloc((void**)&h->colpart, sizeof(float) * COL_CHUNKS * std::max(h->P, width));
    alloc((void**)&h->mse_part, sizeof(float) * MSE_BLOCKS);
    alloc((void**)&h->loss_tmp, sizeof(float));
    alloc((void**)&h->seg_bounds, sizeof(long long) * 10);
    alloc((void**)&h->seg_fan, sizeof(int) * 10);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->seg_bounds, h->off, sizeof h->off, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->seg_fan, fans, sizeof fans, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        k_hyper_init<<<256, 256, 0, h->stream>>>(o, h->params, h->seg_bounds, h->seg_fan, 10, seed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->m, 0, sizeof(float) * o, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->v, 0, sizeof(float) * o, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        vmap_hyper_destroy(h);
        return VMAP_ERR_CUDA;
    }
    *out = h;
    return VMAP_OK;
}

vmap_status vmap_hyper_destroy(vmap_hyper* h) {
    if (!h) return VMAP_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    void* ptrs[] = {h->params, h->grad, h->m, h->v, h->h1, h->h2, h->h3, h->da, h->db, h->arg, h->z, h->u,
                    h->th, h->dth, h->du, h->dz, h->split, h->colpart, h->mse_part, h->loss_tmp, h->seg_bounds,
                    h->seg_fan, h->tc_part, h->err_d};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete h;
    return VMAP_OK;
}

const char* vmap_hyper_last_error(const vmap_hyper* h) { return h ? h->err.c_str() : "null hypernetwork"; }

vmap_status vmap_hyper_set_precision(vmap_hyper* h, int precision) {
    if (!h) return VMAP_ERR_ARG;
    if (precision != VMAP_FP32 && precision != VMAP_BF16) return hfail(h, VMAP_ERR_ARG, "unknown precision %d", precision);
    if (precision == VMAP_BF16) {
        if (h->W != vmapk::HG) return hfail(h, VMAP_ERR_ARG, "BF16 GEMMs need width %d", vmapk::HG);
        HCU(cudaStreamSynchronize(h->stream));
        if (!h->tc_part) {
            int dev = 0;
            HCU(cudaGetDevice(&dev));
            HCU(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));
            HCU(cudaMalloc((void**)&h->tc_part, sizeof(float) * (size_t)h->n_sm * vmapk::HG * vmapk::HG));
            HCU(cudaMalloc((void**)&h->err_d, sizeof(int)));
            HCU(cudaMemset(h->err_d, 0, sizeof(int)));
        }
    }
    h->bf16 = precision == VMAP_BF16;
    return VMAP_OK;
}

vmap_status vmap_hyper_param_count(vmap_hyper* h, long long* n, int* out_params) {
    if (!h) return VMAP_ERR_ARG;
    if (n) *n = h->n_params;
    if (out_params) *out_params = h->P;
    return VMAP_OK;
}

vmap_status vmap_hyper_get_params(vmap_hyper* h, float* flat) {
    if (!h || !flat) return VMAP_ERR_ARG;
    HCU(cudaMemcpyAsync(flat, h->params, sizeof(float) * h->n_params, cudaMemcpyDeviceToDevice, h->stream));
    return VMAP_OK;
}

vmap_status vmap_hyper_set_params(vmap_hyper* h, const float* flat) {
    if (!h || !flat) return VMAP_ERR_ARG;
    HCU(cudaMemcpyAsync(h->params, flat, sizeof(float) * h->n_params, cudaMemcpyDeviceToDevice, h->stream));
    HCU(cudaMemsetAsync(h->m, 0, sizeof(float) * h->n_params, h->stream));
    HCU(cudaMemsetAsync(h->v, 0, sizeof(float) * h->n_params, h->stream));
    h->step = 0;
    return VMAP_OK;
}

vmap_status vmap_hyper_predict(vmap_hyper* h, int batch, const float* X, float* out) {
    if (vmap_status s = check_batch(h, batch, X)) return s;
    if (!out) return VMAP_ERR_ARG;
    if (vmap_status s = forward(h, batch, X)) return s;
    HCU(cudaMemcpyAsync(out, h->th, sizeof(float) * (long long)batch * h->P, cudaMemcpyDeviceToDevice, h->stream));
    return VMAP_OK;
}

vmap_status vmap_hyper_grad(vmap_hyper* h, int batch, const float* X, const float* T, float* grad, float* loss) {
    if (vmap_status s = check_batch(h, batch, X)) return s;
    if (!T) return VMAP_ERR_ARG;
    if (vmap_status s = forward(h, batch, X)) return s;
    if (vmap_status s = backward(h, batch, X, T, loss)) return s;
    if (grad) HCU(cudaMemcpyAsync(grad, h->grad, sizeof(float) * h->n_params, cudaMemcpyDeviceToDevice, h->stream));
    return VMAP_OK;
}

vmap_status vmap_hyper_train_step(vmap_hyper* h, int batch, const float* X, const float* T, float lr, float* loss) {
    if (vmap_status s = vmap_hyper_grad(h, batch, X, T, nullptr, loss)) return s;
    h->step += 1;
    const float bc1 = 1.f - powf(0.9f, (float)h->step), bc2 = 1.f - powf(0.999f, (float)h->step);
    k_adam_flat<<<512, 256, 0, h->stream>>>(h->n_params, h->params, h->grad, h->m, h->v, lr, 0.9f, 0.999f, 1e-8f, bc1,
                                            bc2);
    HCU(cudaGetLastError());
    return VMAP_OK;
}

}  // extern "C"
