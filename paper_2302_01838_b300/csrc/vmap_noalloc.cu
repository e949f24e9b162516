// Allocation-free gradient of one object: the training step's forward,
// rendering, loss and backward for a single object on caller-chosen rays,
// with every scratch buffer (batch tables, sample depths, the transposed
// weights and the gradient run slots) carved out of one file-scope device
// array instead of cudaMalloc'd memory. It launches the same kernels as the
// context-based path (batch builder, sampler, fused tile kernel, reduce).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/vmap.h"

// This translation unit keeps its own copy of the kernels, with internal
// linkage (the shared headers define them outside any template).
namespace {
#include "vmap_build.cuh"
#include "vmap_common.cuh"
#include "vmap_optim.cuh"
#include "vmap_sample.cuh"
#include "vmap_tile_fp32.cuh"
}  // namespace

namespace {
using namespace vmapk;

constexpr int NA_MAX_RAYS = 1024;     // rays per call, at most
constexpr int NA_GRID = 16;           // CTAs of the tile kernel: at most NA_GRID + 1 gradient runs
constexpr int NA_TILE_CAP = NA_MAX_RAYS + 16;
constexpr int NA_MAX_DEVICES = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets inside the scratch array
constexpr size_t OFF_OBJ = 0;
constexpr size_t OFF_OB = align256(OFF_OBJ + sizeof(ObjDev));
constexpr size_t OFF_INTS = align256(OFF_OB + sizeof(ObjBatch));   // n_obj, req, status, step
constexpr size_t OFF_COUNTS = align256(OFF_INTS + 4 * sizeof(int));
constexpr size_t OFF_BOBJ = align256(OFF_COUNTS + BC_N * sizeof(int));
constexpr size_t OFF_BRAY = align256(OFF_BOBJ + sizeof(int));
constexpr size_t OFF_ITEMS = align256(OFF_BRAY + sizeof(int));
constexpr size_t OFF_TILES =
    align256(OFF_ITEMS + sizeof(int2) * ((param_count(128) + REDUCE_CHUNK - 1) / REDUCE_CHUNK));
constexpr size_t OFF_FLAGS = align256(OFF_TILES + sizeof(TileDev) * (size_t)NA_TILE_CAP * NCLASS);
constexpr size_t OFF_PICK = align256(OFF_FLAGS + sizeof(int) * (size_t)NA_TILE_CAP * NCLASS);
constexpr size_t OFF_T = align256(OFF_PICK + sizeof(int) * NA_MAX_RAYS);
constexpr size_t OFF_WT = align256(OFF_T + sizeof(float) * (size_t)NA_MAX_RAYS * SMAX);
constexpr size_t OFF_PART = align256(OFF_WT + sizeof(float) * wt_count(128));
constexpr size_t SCRATCH_BYTES = align256(OFF_PART + sizeof(float) * (NA_GRID + 1) * (param_count(128) + NEXTRA));

// Shared by every call on a device (about 4.8 MB); see vmap_object_grad_static.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Per device: the array's device address, looked up once (under na_mutex).
std::atomic<unsigned char*> g_scratch_dev[NA_MAX_DEVICES];
std::mutex na_mutex;

// The call's object record and header ints reach the scratch array through
// this kernel's by-value arguments, so no host-to-device copy is queued.
__global__ void k_na_init(ObjDev o, int4 head, ObjDev* objs, int* ints) {
    if (threadIdx.x == 0) {
        *objs = o;
        ints[0] = head.x;
        ints[1] = head.y;
        ints[2] = head.z;
        ints[3] = head.w;
    }
}

template <int H>
cudaError_t prepare_tile() {
    return cudaFuncSetAttribute(k_tile_fp32<H, MODE_TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TileSmem<H>::BYTES);
}

template <int H>
cudaError_t run_tile(cudaStream_t st, const StepParams& sp, const TileArgs& ta) {
    k_tile_fp32<H, MODE_TRAIN><<<NA_GRID, TileCfg<H>::THREADS, TileSmem<H>::BYTES, st>>>(sp, ta);
    return cudaGetLastError();
}

int mmax_class(int c) {
    return c == 0 ? TileCfg<16>::MMAX : c == 1 ? TileCfg<32>::MMAX : c == 2 ? TileCfg<64>::MMAX : TileCfg<128>::MMAX;
}

}  // namespace

extern "C" vmap_status vmap_object_grad_static(const vmap_config* cfg, const vmap_object_desc* desc,
                                               const float* params, int step, float* grad, float* loss,
                                               void* cuda_stream) {
    if (!cfg || !desc || !params || !grad || !loss || !desc->rays || !cfg->B) return VMAP_ERR_ARG;
    const int H = desc->hidden;
    if (H != 16 && H != 32 && H != 64 && H != 128) return VMAP_ERR_ARG;
    const int S = desc->n_surface + desc->n_strat;
    if (desc->n_surface < 0 || desc->n_strat < 0 || S < 1 || S > SMAX) return VMAP_ERR_ARG;
    const int c = class_of(H);
    if (S > mmax_class(c)) return VMAP_ERR_ARG;
    if (!(desc->scale > 0.f) || !std::isfinite(desc->scale) || step < 0) return VMAP_ERR_ARG;
    if (desc->n_rays < 1) return VMAP_ERR_ARG;
    if (desc->n_rays > NA_MAX_RAYS) return VMAP_ERR_CAPACITY;   // beyond the static scratch

    // one-time set-up per device, with that device current
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return VMAP_ERR_CUDA;
    unsigned char* base = g_scratch_dev[dev].load(std::memory_order_acquire);
    if (!base) {
        std::lock_guard<std::mutex> lock(na_mutex);
        base = g_scratch_dev[dev].load(std::memory_order_relaxed);
        if (!base) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return VMAP_ERR_CUDA;
            if (prepare_tile<16>() != cudaSuccess || prepare_tile<32>() != cudaSuccess ||
                prepare_tile<64>() != cudaSuccess || prepare_tile<128>() != cudaSuccess)
                return VMAP_ERR_CUDA;
            base = (unsigned char*)p;
            g_scratch_dev[dev].store(base, std::memory_order_release);
        }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;

    ObjDev* objs = (ObjDev*)(base + OFF_OBJ);
    ObjBatch* ob = (ObjBatch*)(base + OFF_OB);
    int* ints = (int*)(base + OFF_INTS);   // [0] n_obj, [1] req, [2] status, [3] step
    int* counts = (int*)(base + OFF_COUNTS);
    int* bobj = (int*)(base + OFF_BOBJ);
    int* bray = (int*)(base + OFF_BRAY);
    int2* items = (int2*)(base + OFF_ITEMS);
    TileDev* tiles = (TileDev*)(base + OFF_TILES);
    int* flags = (int*)(base + OFF_FLAGS);
    int* pick = (int*)(base + OFF_PICK);
    float* tbuf = (float*)(base + OFF_T);
    float* wt = (float*)(base + OFF_WT);
    float* part = (float*)(base + OFF_PART);

    StepParams sp{};
    std::memcpy(sp.B, cfg->B, sizeof(float) * NF * 3);
    sp.t_near = cfg->t_near;
    sp.depth_pad = cfg->depth_pad;
    sp.d_sigma = cfg->d_sigma;
    sp.t_far = cfg->t_far;
    sp.lam_c = cfg->lambda_colour;
    sp.lam_o = cfg->lambda_occ;
    sp.lr = cfg->lr;
    sp.beta1 = cfg->beta1;
    sp.beta2 = cfg->beta2;
    sp.eps = cfg->eps;
    sp.key0 = (uint32_t)(cfg->seed & 0xFFFFFFFFull);
    sp.key1 = (uint32_t)(cfg->seed >> 32);

    ObjDev o{};
    o.hidden = H;
    o.S = S;
    o.n_surface = desc->n_surface;
    o.n_strat = desc->n_strat;
    for (int a = 0; a < 3; ++a) o.c[a] = desc->center[a];
    o.scale = desc->scale;
    o.pool_n = desc->n_rays;
    o.stream = desc->stream;
    o.active = 1;
    // n_obj, requested rays, status (0: the reduce writes gradient and loss), step count
    k_na_init<<<1, 32, 0, st>>>(o, make_int4(1, (int)desc->n_rays, 0, step), objs, ints);

    k_shadow<<<16, 256, 0, st>>>(params, wt, H);

    BuildArgs a{};
    a.objs = objs;
    a.ob = ob;
    a.n_obj = ints + 0;
    a.req = ints + 1;
    a.status = ints + 2;
    a.given = 1;
    for (int q = 0; q < NCLASS; ++q) {
        a.rt[q] = RTMAX;
        a.mmax[q] = mmax_class(q);
        a.grid[q] = NA_GRID;
        a.part_base[q] = 0;   // one object, one width class: all runs start at slot 0
    }
    a.rtmax = RTMAX;
    a.tiles = tiles;
    a.flags = flags;
    a.tile_cap = NA_TILE_CAP;
    a.bobj = bobj;
    a.bray = bray;
    a.items = items;
    a.counts = counts;
    k_build<<<1, BUILD_THREADS, 0, st>>>(a);
    k_sample<<<(desc->n_rays + SAMPLE_RAYS_PER_BLOCK - 1) / SAMPLE_RAYS_PER_BLOCK, 32 * SAMPLE_RAYS_PER_BLOCK, 0,
               st>>>(sp, objs, ob, bobj, bray, nullptr, counts, desc->rays, 1, ints + 3, pick, tbuf);
    TileArgs ta{};
    ta.objs = objs;
    ta.obs = ob;
    ta.tiles = tiles + (long long)c * NA_TILE_CAP;
    ta.n_tiles = counts + BC_TILES + c;
    ta.pool = desc->rays;
    ta.pick = pick;
    ta.tbuf = tbuf;
    ta.params = params;
    ta.wt = wt;
    ta.part = part;
    cudaError_t e = c == 0 ? run_tile<16>(st, sp, ta)
                  : c == 1 ? run_tile<32>(st, sp, ta)
                  : c == 2 ? run_tile<64>(st, sp, ta)
                           : run_tile<128>(st, sp, ta);
    if (e != cudaSuccess) return VMAP_ERR_CUDA;
    // the step slot holds `step`, the status slot 0: the reduce writes the gradient and the loss
    k_reduce<<<8, REDUCE_THREADS, 0, st>>>(sp, objs, ob, items, counts, part, nullptr, nullptr, nullptr, nullptr,
                                ints + 3, ints + 2, RED_GRAD, nullptr, grad, loss, nullptr, nullptr, nullptr,
                                nullptr, nullptr, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? VMAP_OK : VMAP_ERR_CUDA;
}
