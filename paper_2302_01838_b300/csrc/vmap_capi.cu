// C ABI of the vMAP training library: context, object table, launches,
// CUDA-graph replay, profiling and the launch autotuner. The batch layout is
// built on the device (vmap_build.cuh), so one step is a fixed sequence of
// launches that a CUDA graph can replay while objects come and go.
// See include/vmap.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vmap.h"
#include "vmap_build.cuh"
#include "vmap_mesh.cuh"
#include "vmap_common.cuh"
#include "vmap_optim.cuh"
#include "vmap_pose.cuh"
#include "vmap_sample.cuh"
#include "vmap_scene.cuh"
#include "vmap_tile_bf16.cuh"
#include "vmap_tile_fp32.cuh"
#include "vmap_tile_w32.cuh"
#include "vmap_tile_wide.cuh"

using namespace vmapk;

namespace {

enum ProfSlot { PS_BUILD = 0, PS_SAMPLE = 1, PS_TILE = 2 /* + class */, PS_REDUCE = 6, PS_FINISH = 7,
                PS_GRAPH_SAMPLE = 8, PS_GRAPH_TRAIN = 9, PS_WIDE_DW = 10, PS_N = 11 };
const char* kProfNames[PS_N] = {"k_build",         "k_sample",         "k_tile_fp32<16>", "k_tile_fp32<32>",
                                "k_tile_fp32<64>", "k_tile_fp32<128>", "k_reduce",        "k_finish",
                                "graph:sample",    "graph:train",      "k_wide_dw<128>"};
const char* kProfNamesBf16[NCLASS] = {"k_tile_bf16<16>", "k_tile_bf16<32>", "k_tile_bf16<64>", "k_wide_fb<128>"};

int mmax_of(int c) {
    switch (c) {
        case 0: return TileCfg<16>::MMAX;
        case 1: return TileCfg<32>::MMAX;
        case 2: return TileCfg<64>::MMAX;
        default: return TileCfg<128>::MMAX;
    }
}
int ctas_of(int c) {
    switch (c) {
        case 0: return TileCfg<16>::CTAS;
        case 1: return TileCfg<32>::CTAS;
        case 2: return TileCfg<64>::CTAS;
        default: return TileCfg<128>::CTAS;
    }
}
bool valid_hidden(int H) { return H == 16 || H == 32 || H == 64 || H == 128; }
constexpr int GMULT_MAX = 2;   // persistent grid: n_sm * CTAS * gmult CTAs per class
constexpr long long DYN_SLOT_BYTES = 256LL << 20;   // per class, for dynamically scheduled FP32 classes

struct ProfPair {
    int slot;
    cudaEvent_t a, b;
};

}  // namespace

struct vmap_ctx {
    vmap_config cfg{};
    cudaStream_t stream = nullptr;
    std::string err;
    StepParams sp{};
    int device = 0, n_sm = 148;

    // objects: static table (host + device mirror), per-batch table (device)
    std::vector<ObjDev> objs;
    ObjDev* objs_d = nullptr;
    ObjBatch* ob_d = nullptr;
    int* n_obj_d = nullptr;
    int* steps_d = nullptr;
    int* status_d = nullptr;
    int* req_d = nullptr;
    std::vector<int> req_h;

    // arenas
    float *params_d = nullptr, *wt_d = nullptr, *m_d = nullptr, *v_d = nullptr;
    long long param_used = 0, param_cap = 0, wt_used = 0, wt_cap = 0;
    float* pool_d = nullptr;
    long long pool_used = 0, pool_cap = 0;

    // batch
    int* pick_d = nullptr;
    float* t_d = nullptr;
    int *bobj_d = nullptr, *bray_d = nullptr;
    int* ray_bj_d = nullptr;        // object of each batch ray (written by the builder)
    TileDev* tiles_d = nullptr;
    int* flags_d = nullptr;
    int tile_cap = 0;
    float* part_d = nullptr;
    long long part_base[NCLASS] = {0, 0, 0, 0};
    int2* items_d = nullptr;
    int* counts_d = nullptr;
    int* sig_d = nullptr;           // inputs of the last batch build ([0] = -1: rebuild)
    int* dyn_d = nullptr;           // [NCLASS][2] tile counters of dynamically scheduled classes
    float* enc_d[NCLASS] = {nullptr, nullptr, nullptr, nullptr};   // FP32 per-CTA encoding copies
    int dyn_cap[NCLASS] = {0, 0, 0, 0};   // tiles a class may have to be scheduled dynamically
    int* done_d = nullptr;          // per object: reduce warps that have finished (reset by the last)
    long long build_key = -1;       // launch shape the last build ran with
    // host-side inputs of the last batch build: when none changed, the builder
    // is not launched (objects frozen on the device since then stay in the
    // layout; the reduce already leaves them untouched)
    long long layout_gen = 0;       // bumped by every change of an object's layout fields or status
    bool built = false;
    int built_K = -1, built_given = -1;
    long long built_gen = -1, built_key = -1;
    std::vector<int> built_req;
    float* given_d = nullptr;
    float* loss_d = nullptr;
    bool batch_ready = false;
    bool batch_given = false;
    int total_rays = 0;
    long long total_samples = 0;

    // launch configuration (autotuned)
    int rt[NCLASS] = {RTMAX, RTMAX, RTMAX, RTMAX};
    int gmult[NCLASS] = {1, 1, 1, 1};

    // BF16 tensor-core path: per-object operand images of the weights
    bool bf16 = false;
    __nv_bfloat16* img_d = nullptr;
    long long* img_off_d = nullptr;
    long long img_used = 0, img_cap = 0;
    std::vector<long long> img_off;
    int* err_d = nullptr;   // set by a kernel whose bounded wait gave up
    long long wait_polls = MMA_WAIT_LIMIT;   // polls before a tensor-core wait gives up
    // the training step's second loss destination (the caller's out_loss): its
    // address lives on the device, so a captured step writes wherever it points
    float** loss_pp_d = nullptr;
    float* loss_user_h = nullptr;   // the address loss_pp_d holds
    // width-128 tensor-core path: per-tile activation records, grown on demand;
    // kernels read the buffer's address from act_pp_d, so captured graphs survive a regrowth
    unsigned char* act_d = nullptr;
    unsigned char** act_pp_d = nullptr;
    long long act_cap = 0;          // tiles
    float* tile_loss_d = nullptr;   // [tile_cap][8] per-tile loss sums (the BF16 pair uses 4 of them)
    // scene rendering: per (object, ray) records, grown on demand
    float* scene_d = nullptr;
    long long scene_cap = 0;        // floats
    float* ray_grad_out = nullptr;  // set only while vmap_ray_gradients launches
    // BF16 training does not keep the FP32 transposed shadow current (only the
    // FP32 eval/query kernels read it there); it is rebuilt before they run
    bool shadow_stale = false;

    // CUDA graphs (captured on a private stream, replayed on the context stream)
    bool graph_on = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t g_sample[2] = {nullptr, nullptr};   // [given]: builder + sampler
    cudaGraphExec_t g_sample_only[2] = {nullptr, nullptr};   // [given]: sampler alone
    cudaGraphExec_t g_train = nullptr;
    cudaGraphExec_t g_step[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [given][build]: sampler + step
    int g_step_classes[2][2] = {{-1, -1}, {-1, -1}};
    int g_classes = -1;                 // class mask the train graph was captured for

    // profiling
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<ProfPair> pending;
    bool capturing = false;
    // the sampler was the stream's last launch (one step's sequence, no profiling
    // event between): the step's first BF16 tile kernel starts behind it
    bool after_sample = false;
    double prof_ms[PS_N] = {0};
    long long prof_n[PS_N] = {0};
};

namespace {

vmap_status fail(vmap_ctx* c, vmap_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CU(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ctx, VMAP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

#define CHECK_LAUNCH(name)                                                                     \
    do {                                                                                       \
        cudaError_t e_ = cudaGetLastError();                                                   \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ctx, VMAP_ERR_CUDA, "launch of %s failed: %s", name,                   \
                        cudaGetErrorString(e_));                                               \
    } while (0)

// ---- profiling: event pairs around launches ---------------------------------
cudaEvent_t take_event(vmap_ctx* ctx) {
    cudaEvent_t e = nullptr;
    if (ctx->ev_free.empty()) {
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    } else {
        e = ctx->ev_free.back();
        ctx->ev_free.pop_back();
    }
    return e;
}

int prof_begin(vmap_ctx* ctx, int slot) {
    if (!ctx->prof_on || ctx->capturing) return -1;
    ProfPair p{slot, take_event(ctx), take_event(ctx)};
    if (!p.a || !p.b) return -1;
    cudaEventRecord(p.a, ctx->stream);
    ctx->pending.push_back(p);
    return (int)ctx->pending.size() - 1;
}

void prof_end(vmap_ctx* ctx, int idx) {
    if (idx < 0) return;
    cudaEventRecord(ctx->pending[idx].b, ctx->stream);
}

// synchronise and accumulate every pending pair
void prof_flush(vmap_ctx* ctx) {
    if (ctx->pending.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ctx->prof_ms[p.slot] += ms;
            ctx->prof_n[p.slot] += 1;
        }
        ctx->ev_free.push_back(p.a);
        ctx->ev_free.push_back(p.b);
    }
    ctx->pending.clear();
}

void drop_graphs(vmap_ctx* ctx) {
    prof_flush(ctx);
    for (auto& g : ctx->g_sample_only)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (auto& g : ctx->g_sample)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (ctx->g_train) {
        cudaGraphExecDestroy(ctx->g_train);
        ctx->g_train = nullptr;
    }
    ctx->g_classes = -1;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            if (ctx->g_step[i][j]) cudaGraphExecDestroy(ctx->g_step[i][j]);
            ctx->g_step[i][j] = nullptr;
            ctx->g_step_classes[i][j] = -1;
        }
}

vmap_status check_obj(vmap_ctx* ctx, int obj) {
    if (!ctx) return VMAP_ERR_ARG;
    if (obj < 0 || obj >= (int)ctx->objs.size())
        return fail(ctx, VMAP_ERR_ARG, "object index %d out of range [0, %d)", obj, (int)ctx->objs.size());
    return VMAP_OK;
}

vmap_status upload_obj(vmap_ctx* ctx, int k, bool layout = true) {
    if (layout) ++ctx->layout_gen;
    // pageable source: the bytes are staged before the call returns
    CU(cudaMemcpyAsync(ctx->objs_d + k, &ctx->objs[k], sizeof(ObjDev), cudaMemcpyHostToDevice, ctx->stream));
    return VMAP_OK;
}

int class_mask(vmap_ctx* ctx) {
    int m = 0;
    for (const ObjDev& o : ctx->objs) m |= 1 << class_of(o.hidden);
    return m;
}

bool uses_tc(vmap_ctx* ctx, int c) { return ctx->bf16 && c < 3; }
bool uses_wide(vmap_ctx* ctx, int c) { return ctx->bf16 && c == 3; }
// the FP32 width-128 pair (k_w32_fb, k_w32_dw)
bool uses_w32(vmap_ctx* ctx, int c) { return !ctx->bf16 && c == 3; }

// tile ranges of the width-128 weight-gradient kernel (WJOBS or W32JOBS CTAs
// each; one wave of CTAs at gmult 1)
int wide_ranges(vmap_ctx* ctx) { return std::max(1, ctx->n_sm / (ctx->bf16 ? WJOBS : W32JOBS)) * ctx->gmult[3]; }

// CTA ranges that own a run slot (the builder's partition of the class's tiles)
int grid_of(vmap_ctx* ctx, int c) {
    return uses_wide(ctx, c) || uses_w32(ctx, c) ? wide_ranges(ctx) : ctx->n_sm * ctas_of(c) * ctx->gmult[c];
}

TileArgs base_args(vmap_ctx* ctx) {
    TileArgs ta{};
    ta.objs = ctx->objs_d;
    ta.obs = ctx->ob_d;
    ta.pool = ctx->batch_given ? ctx->given_d : ctx->pool_d;
    ta.pick = ctx->pick_d;
    ta.tbuf = ctx->t_d;
    ta.params = ctx->params_d;
    ta.wt = ctx->wt_d;
    ta.part = ctx->part_d;
    ta.ray_grad = ctx->ray_grad_out;
    return ta;
}

enum { PDL_NONE = 0, PDL_AFTER_SAMPLE = 1, PDL_AFTER_TILE = 2 };

// FP32 tile kernel. With PDL_AFTER_TILE it is launched with programmatic
// stream serialization behind another width class's FP32 tile kernel: its CTAs
// start on the SMs that kernel leaves (the classes touch disjoint objects and
// slots) and it completes only after that kernel.
template <int H, int MODE>
cudaError_t launch_tile(int grid, cudaStream_t st, const StepParams& sp, const TileArgs& ta, int pdl = PDL_NONE) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_fp32<H, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)TileSmem<H>::BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (grid <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(TileCfg<H>::THREADS);
    cfg.dynamicSmemBytes = TileSmem<H>::BYTES;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl == PDL_AFTER_TILE ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_tile_fp32<H, MODE>, sp, ta);
}

template <int MODE>
cudaError_t launch_tile_c(int c, int grid, cudaStream_t st, const StepParams& sp, const TileArgs& ta,
                          int pdl = PDL_NONE) {
    switch (c) {
        case 0: return launch_tile<16, MODE>(grid, st, sp, ta, pdl);
        case 1: return launch_tile<32, MODE>(grid, st, sp, ta, pdl);
        case 2: return launch_tile<64, MODE>(grid, st, sp, ta, pdl);
        default: return launch_tile<128, MODE>(grid, st, sp, ta, pdl);
    }
}

// With `pdl` the tile kernel is launched with programmatic stream
// serialization behind the previous kernel in the stream: the sampler
// (PDL_AFTER_SAMPLE: set-up and first tile records run on SMs the sampler's
// last blocks free, then it waits for the sampler before reading the picks and
// depths) or another width class's tile kernel (PDL_AFTER_TILE: its CTAs start
// on SMs that kernel frees, with no wait at the start, and wait for it before
// they exit).
template <int H, int MODE>
cudaError_t launch_tile_bf16(int grid, cudaStream_t st, const StepParams& sp, Bf16Args ba, int pdl = PDL_NONE) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_bf16<H, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Bf16Cfg<H>::BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (grid <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = Bf16Cfg<H>::BYTES;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl != PDL_NONE ? 1 : 0;
    ba.wait_first = pdl != PDL_AFTER_TILE;
    return cudaLaunchKernelEx(&cfg, k_tile_bf16<H, MODE>, sp, ba);
}

WideArgs wide_args(vmap_ctx* ctx) {
    TileArgs ta = base_args(ctx);
    ta.tiles = ctx->tiles_d + 3LL * ctx->tile_cap;
    ta.n_tiles = ctx->counts_d + BC_TILES + 3;
    return WideArgs{ta, ctx->img_d, ctx->img_off_d, ctx->err_d, ctx->act_pp_d, ctx->tile_loss_d, 0, ctx->wait_polls};
}

// overlap: with `after_tile` (the previous kernel in the stream is a BF16 tile
// kernel, which signals its dependents once all its CTAs are resident and past
// their wait for the sampler), the width-128 kernel is launched with
// programmatic stream serialization, so its CTAs start on SMs as the tile
// kernel's CTAs finish; it waits for the tile kernel's completion before it
// exits (the two touch disjoint objects)
template <int MODE>
cudaError_t launch_wide_fb(vmap_ctx* ctx, bool after_tile = false) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_wide_fb<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)WideFbCfg::BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ctx->n_sm * ctx->gmult[3]));
    cfg.blockDim = dim3(WIDE_THREADS);
    cfg.dynamicSmemBytes = WideFbCfg::BYTES;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = after_tile ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_wide_fb<MODE>, ctx->sp, wide_args(ctx));
}

// with `after_fb` (the previous kernel in the stream is k_wide_fb, which
// signals its dependents once all its CTAs are resident) the weight-gradient
// kernel is launched with programmatic stream serialization: its set-up runs on
// SMs k_wide_fb frees, and it waits for k_wide_fb before reading the records
cudaError_t launch_wide_dw(vmap_ctx* ctx, int loss_only, bool after_fb = false) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_wide_dw, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)WideDwCfg::BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    WideArgs wa = wide_args(ctx);
    wa.loss_only = loss_only;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(WJOBS * wide_ranges(ctx)));
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = WideDwCfg::BYTES;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = after_fb ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_wide_dw, wa);
}

W32Args w32_args(vmap_ctx* ctx) {
    TileArgs ta = base_args(ctx);
    ta.tiles = ctx->tiles_d + 3LL * ctx->tile_cap;
    ta.n_tiles = ctx->counts_d + BC_TILES + 3;
    ta.dyn = ctx->dyn_d + 2 * 3;
    return W32Args{ta, reinterpret_cast<float* const*>(ctx->act_pp_d), ctx->tile_loss_d, 0};
}

// FP32 width-128 forward/input-gradient kernel: one CTA per SM taking tiles
// from the class's counter; launched in stream order (it starts the step's
// FP32 tile kernels), the narrower classes chained behind it
template <int MODE>
cudaError_t launch_w32_fb(vmap_ctx* ctx) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_w32_fb<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)W32FbCfg::BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_w32_fb<MODE><<<ctx->n_sm, W32_THREADS, W32FbCfg::BYTES, ctx->stream>>>(ctx->sp, w32_args(ctx));
    return cudaGetLastError();
}

// FP32 width-128 weight-gradient kernel, after the step's other FP32 tile
// kernels; with `pdl` launched with programmatic stream serialization (its
// CTAs wait for the previous kernel, and through it for k_w32_fb, before
// reading the records)
cudaError_t launch_w32_dw(vmap_ctx* ctx, int loss_only, bool pdl) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_w32_dw, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)W32DwCfg::BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    W32Args wa = w32_args(ctx);
    wa.loss_only = loss_only;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(W32JOBS * wide_ranges(ctx)));
    cfg.blockDim = dim3(W32_THREADS);
    cfg.dynamicSmemBytes = W32DwCfg::BYTES;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_w32_dw, wa);
}

// one width class of the step's tile kernel (FP32 SIMT, or BF16 tensor cores)
template <int MODE>
cudaError_t launch_class(vmap_ctx* ctx, int c, int pdl = PDL_NONE) {
    TileArgs ta = base_args(ctx);
    ta.tiles = ctx->tiles_d + (long long)c * ctx->tile_cap;
    ta.n_tiles = ctx->counts_d + BC_TILES + c;
    const int grid = grid_of(ctx, c);
    if (uses_wide(ctx, c)) {
        constexpr int BM = MODE == MODE_FORWARD ? MODE_FORWARD : MODE_TRAIN;
        cudaError_t e = launch_wide_fb<BM>(ctx);
        return e != cudaSuccess ? e : launch_wide_dw(ctx, BM == MODE_FORWARD);
    }
    if (uses_tc(ctx, c)) {
        constexpr int BM = MODE == MODE_FORWARD ? MODE_FORWARD : MODE_TRAIN;
        Bf16Args ba{ta, ctx->img_d, ctx->img_off_d, ctx->err_d, ctx->wait_polls, 1};
        switch (c) {
            case 0: return launch_tile_bf16<16, BM>(grid, ctx->stream, ctx->sp, ba, pdl);
            case 1: return launch_tile_bf16<32, BM>(grid, ctx->stream, ctx->sp, ba, pdl);
            default: return launch_tile_bf16<64, BM>(grid, ctx->stream, ctx->sp, ba, pdl);
        }
    }
    if (ctx->dyn_cap[c] > 0) {
        ta.dyn = ctx->dyn_d + 2 * c;
        ta.dyn_on = ctx->counts_d + BC_DYN + c;
    }
    ta.enc_scratch = ctx->enc_d[c];
    return launch_tile_c<MODE>(c, grid, ctx->stream, ctx->sp, ta, pdl);
}

int class_mmax(vmap_ctx* ctx, int c) {
    return uses_tc(ctx, c) || uses_wide(ctx, c) ? TM : uses_w32(ctx, c) ? W32M : mmax_of(c);
}

// ---- the step's launches ------------------------------------------------------
vmap_status launch_build_sample(vmap_ctx* ctx, int given, bool build = true) {
    BuildArgs a{};
    a.objs = ctx->objs_d;
    a.ob = ctx->ob_d;
    a.n_obj = ctx->n_obj_d;
    a.req = ctx->req_d;
    a.status = ctx->status_d;
    a.given = given;
    for (int c = 0; c < NCLASS; ++c) {
        a.rt[c] = ctx->rt[c];
        a.mmax[c] = class_mmax(ctx, c);
        a.grid[c] = grid_of(ctx, c);
        a.dyn_cap[c] = ctx->dyn_cap[c];
        a.part_base[c] = ctx->part_base[c];
    }
    a.rtmax = RTMAX;
    a.tiles = ctx->tiles_d;
    a.flags = ctx->flags_d;
    a.tile_cap = ctx->tile_cap;
    a.bobj = ctx->bobj_d;
    a.bray = ctx->bray_d;
    a.ray_bj = ctx->ray_bj_d;
    a.items = ctx->items_d;
    a.counts = ctx->counts_d;
    a.sig = ctx->sig_d;
    int pi = -1;
    if (build) {
        pi = prof_begin(ctx, PS_BUILD);
        k_build<<<1, BUILD_THREADS, 0, ctx->stream>>>(a);
        prof_end(ctx, pi);
        CHECK_LAUNCH("k_build");
    }
    // one wave of blocks whose warps stride over the batch (at most one warp per ray)
    const int blocks = std::min((ctx->cfg.max_rays_total + SAMPLE_RAYS_PER_BLOCK - 1) / SAMPLE_RAYS_PER_BLOCK,
                                ctx->n_sm * SAMPLE_BLOCKS_PER_SM);
    pi = prof_begin(ctx, PS_SAMPLE);
    k_sample<<<blocks, 32 * SAMPLE_RAYS_PER_BLOCK, 0, ctx->stream>>>(ctx->sp, ctx->objs_d, ctx->ob_d, ctx->bobj_d, ctx->bray_d,
                                             ctx->ray_bj_d, ctx->counts_d, given ? ctx->given_d : ctx->pool_d, given,
                                             ctx->steps_d, ctx->pick_d, ctx->t_d);
    prof_end(ctx, pi);
    CHECK_LAUNCH("k_sample");
    return VMAP_OK;
}

// FP32 classes run widest first: the hidden-128 kernel's long tiles start at
// once, and the narrower classes (scheduled dynamically when their slots
// allow) start on the SMs it leaves and fill them as they free up.
template <int MODE>
vmap_status launch_tiles(vmap_ctx* ctx, int mask) {
    bool after_tile = false;   // the last launch in the stream is a BF16 tile kernel
    bool after_fp32 = false;   // ... an FP32 tile kernel
    bool after_sample = ctx->after_sample;   // ... the sampler
    ctx->after_sample = false;
    bool w32_dw = false;       // the FP32 width-128 weight-gradient kernel is due
    static const int order_tc[NCLASS] = {0, 1, 2, 3}, order_fp32[NCLASS] = {3, 0, 1, 2};
    for (int ci = 0; ci < NCLASS; ++ci) {
        const int c = ctx->bf16 ? order_tc[ci] : order_fp32[ci];
        if (!(mask & (1 << c))) continue;
        cudaError_t e;
        const bool after_sample_c = after_sample;   // only the first launch follows the sampler
        after_sample = false;
        if (uses_w32(ctx, c)) {
            // forward and input gradients first; the weight gradients after the
            // narrower classes, which fill the SMs its CTAs leave
            const int pi = MODE == MODE_TRAIN ? prof_begin(ctx, PS_TILE + c) : -1;
            e = launch_w32_fb<MODE>(ctx);
            prof_end(ctx, pi);
            w32_dw = true;
            after_fp32 = pi < 0;
        } else if (uses_wide(ctx, c)) {
            constexpr int BM = MODE == MODE_FORWARD ? MODE_FORWARD : MODE_TRAIN;
            int pi = MODE == MODE_TRAIN ? prof_begin(ctx, PS_TILE + c) : -1;
            e = launch_wide_fb<BM>(ctx, after_tile && pi < 0);
            prof_end(ctx, pi);
            if (e == cudaSuccess) {
                const bool fb_plain = pi < 0;   // no profiling event between the two launches
                pi = MODE == MODE_TRAIN ? prof_begin(ctx, PS_WIDE_DW) : -1;
                e = launch_wide_dw(ctx, BM == MODE_FORWARD, fb_plain && pi < 0);
                prof_end(ctx, pi);
            }
        } else {
            const int pi = MODE == MODE_TRAIN ? prof_begin(ctx, PS_TILE + c) : -1;
            // the first class starts behind the sampler, each further one behind
            // the previous class's tile kernel (no profiling event between)
            int pdl = PDL_NONE;
            if (pi < 0 && uses_tc(ctx, c)) pdl = after_sample_c ? PDL_AFTER_SAMPLE : after_tile ? PDL_AFTER_TILE : PDL_NONE;
            if (pi < 0 && !uses_tc(ctx, c) && after_fp32) pdl = PDL_AFTER_TILE;
            e = launch_class<MODE>(ctx, c, pdl);
            prof_end(ctx, pi);
            after_tile = uses_tc(ctx, c) && pi < 0;
            after_fp32 = !uses_tc(ctx, c) && pi < 0;
        }
        if (e != cudaSuccess)
            return fail(ctx, VMAP_ERR_CUDA, "tile kernel (H=%d) failed: %s", hidden_of(c), cudaGetErrorString(e));
    }
    if (w32_dw) {
        const int pi = MODE == MODE_TRAIN ? prof_begin(ctx, PS_WIDE_DW) : -1;
        const cudaError_t e = launch_w32_dw(ctx, MODE == MODE_FORWARD, after_fp32 && pi < 0);
        prof_end(ctx, pi);
        if (e != cudaSuccess) return fail(ctx, VMAP_ERR_CUDA, "k_w32_dw failed: %s", cudaGetErrorString(e));
    }
    return VMAP_OK;
}

// In a training step with no profiling event before it, the reduce is
// launched with programmatic stream serialization behind the step's last tile
// kernel: its blocks load the tables, step counts, weights and moments on SMs
// that kernel frees, then wait for it before reading the run slots.
vmap_status launch_reduce(vmap_ctx* ctx, int mode, const float* grad_loss, float* grad_out, float* loss_out,
                          float* dcenter_out, bool train = false) {
    const int pi = prof_begin(ctx, PS_REDUCE);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ctx->n_sm * REDUCE_BLOCKS_PER_SM));
    cfg.blockDim = dim3(REDUCE_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = train && pi < 0 && (!ctx->prof_on || ctx->capturing) ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(
        &cfg, k_reduce, ctx->sp, (const ObjDev*)ctx->objs_d, (const ObjBatch*)ctx->ob_d, (const int2*)ctx->items_d,
        (const int*)ctx->counts_d, (const float*)ctx->part_d, ctx->params_d, ctx->bf16 ? nullptr : ctx->wt_d, ctx->m_d,
        ctx->v_d, ctx->steps_d, ctx->status_d, mode, grad_loss, grad_out, loss_out, dcenter_out,
        ctx->bf16 ? ctx->img_d : nullptr, (const long long*)ctx->img_off_d, ctx->done_d,
        (const int*)(train ? ctx->n_obj_d : nullptr), (float* const*)(train ? ctx->loss_pp_d : nullptr),
        (const int*)(ctx->bf16 ? ctx->err_d : nullptr));
    prof_end(ctx, pi);
    if (e != cudaSuccess) return fail(ctx, VMAP_ERR_CUDA, "k_reduce launch failed: %s", cudaGetErrorString(e));
    return VMAP_OK;
}

// point the training step's second loss destination at `out` (NULL: none)
vmap_status set_loss_dest(vmap_ctx* ctx, float* out) {
    if (out != ctx->loss_user_h) {   // pageable source: staged before the call returns
        ctx->loss_user_h = out;
        CU(cudaMemcpyAsync(ctx->loss_pp_d, &ctx->loss_user_h, sizeof(float*), cudaMemcpyHostToDevice, ctx->stream));
    }
    return VMAP_OK;
}

// The reduce writes every object's loss (NaN outside the batch) to loss_d and
// to the caller's buffer whose address loss_pp_d holds: no fill before the
// step and no copy after it.
vmap_status launch_train(vmap_ctx* ctx, int mask) {
    if (vmap_status s = launch_tiles<MODE_TRAIN>(ctx, mask)) return s;
    // the last warp of each object advances its step count
    return launch_reduce(ctx, RED_ADAM, nullptr, nullptr, ctx->loss_d, nullptr, true);
}

// capture fn() into an executable graph on the context stream
template <typename F>
vmap_status capture(vmap_ctx* ctx, cudaGraphExec_t* out, F fn) {
    cudaGraph_t g = nullptr;
    if (!ctx->cap_stream) CU(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    // the context stream may be the legacy default stream, which cannot be captured
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->cap_stream;
    ctx->capturing = true;
    vmap_status s = fn();
    ctx->capturing = false;
    ctx->stream = user;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (s) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return fail(ctx, VMAP_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, VMAP_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    return VMAP_OK;
}

// with profiling on, a replay is timed as a whole (slot graph:sample / graph:train)
vmap_status replay(vmap_ctx* ctx, cudaGraphExec_t g, int slot) {
    const int pi = prof_begin(ctx, slot);
    CU(cudaGraphLaunch(g, ctx->stream));
    prof_end(ctx, pi);
    return VMAP_OK;
}

// Build the batch: rays_per_object[k] rays of every active object. With
// given == NULL the rays are picked from the objects' pools; otherwise given
// holds sum_k R_k records (object-major, active objects with R_k > 0, in
// index order) in memory of the kind `kind`, which are staged on the device.
// Activation records of the width-128 path for `need` tiles. The buffer
// only grows (by at least a quarter); its address is published through
// act_pp_d, which captured graphs read at replay.
vmap_status grow_act(vmap_ctx* ctx, long long need) {
    const long long cap = std::max(need, ctx->act_cap + ctx->act_cap / 4) + 8;
    CU(cudaStreamSynchronize(ctx->stream));   // no kernel still uses the old buffer
    if (ctx->act_d) CU(cudaFree(ctx->act_d));
    ctx->act_d = nullptr;
    ctx->act_cap = 0;
    const size_t per_tile = ctx->bf16 ? (size_t)WideAct::BYTES : (size_t)W32Act::FLOATS * sizeof(float);
    CU(cudaMalloc((void**)&ctx->act_d, (size_t)cap * per_tile));
    ctx->act_cap = cap;
    // pageable source: staged before the call returns
    CU(cudaMemcpyAsync(ctx->act_pp_d, &ctx->act_d, sizeof(unsigned char*), cudaMemcpyHostToDevice, ctx->stream));
    return VMAP_OK;
}

// what sample_plan settles on the host before a batch's launches
struct SamplePlan {
    int K = 0, gi = 0;
    bool build = false;
    long long key = 0, rays = 0, samples = 0;
};

vmap_status sample_plan(vmap_ctx* ctx, const int* rays_per_object, const float* given, cudaMemcpyKind kind,
                        SamplePlan& sp) {
    if (!ctx || !rays_per_object) return fail(ctx, VMAP_ERR_ARG, "null argument");
    const int K = (int)ctx->objs.size();
    long long rays = 0, samples = 0;
    long long tiles[NCLASS] = {0, 0, 0, 0};
    for (int k = 0; k < K; ++k) {
        if (rays_per_object[k] < 0) return fail(ctx, VMAP_ERR_ARG, "negative ray count for object %d", k);
        const ObjDev& ob = ctx->objs[k];
        const int R = ob.active ? rays_per_object[k] : 0;
        if (R == 0) continue;
        const int c = class_of(ob.hidden);
        const int rt = std::max(1, std::min(std::min(ctx->rt[c], RTMAX), class_mmax(ctx, c) / ob.S));
        rays += R;
        samples += (long long)R * ob.S;
        tiles[c] += (R + rt - 1) / rt;
    }
    if (rays > ctx->cfg.max_rays_total)
        return fail(ctx, VMAP_ERR_CAPACITY, "%lld rays exceed max_rays_total %d", rays, ctx->cfg.max_rays_total);
    for (int c = 0; c < NCLASS; ++c)
        if (tiles[c] > ctx->tile_cap) return fail(ctx, VMAP_ERR_CAPACITY, "too many tiles");
    if ((uses_wide(ctx, 3) || uses_w32(ctx, 3)) && tiles[3] > ctx->act_cap)
        if (vmap_status s = grow_act(ctx, tiles[3])) return s;
    // the builder skips unchanged layouts; a new launch shape invalidates its record
    long long key = 0;
    for (int c = 0; c < NCLASS; ++c) key = key * 64 + ctx->rt[c] * 4 + ctx->gmult[c];
    if (key != ctx->build_key) {
        CU(cudaMemsetAsync(ctx->sig_d, 0xFF, sizeof(int), ctx->stream));
        ctx->build_key = key;
    }
    const int gi = given ? 1 : 0;
    // the layout depends on (objects, their layout fields and status, rays per
    // object, given or pool rays, launch shape): skip the builder when the host
    // changed none of them since the last build
    const bool same = ctx->built && ctx->built_K == K && ctx->built_given == gi && ctx->built_gen == ctx->layout_gen &&
                      ctx->built_key == key && std::equal(rays_per_object, rays_per_object + K, ctx->built_req.begin());
    if (!same) {
        ctx->req_h.assign(rays_per_object, rays_per_object + K);
        if (K) CU(cudaMemcpyAsync(ctx->req_d, ctx->req_h.data(), sizeof(int) * K, cudaMemcpyHostToDevice, ctx->stream));
    }
    ctx->batch_given = given != nullptr;
    if (given && rays) CU(cudaMemcpyAsync(ctx->given_d, given, sizeof(float) * REC * rays, kind, ctx->stream));
    sp.K = K;
    sp.gi = gi;
    sp.build = !same;
    sp.key = key;
    sp.rays = rays;
    sp.samples = samples;
    return VMAP_OK;
}

// the host's record of the batch whose launches were just issued
void sample_done(vmap_ctx* ctx, const int* rays_per_object, const SamplePlan& sp) {
    ctx->built = true;
    ctx->built_K = sp.K;
    ctx->built_given = sp.gi;
    ctx->built_gen = ctx->layout_gen;
    ctx->built_key = sp.key;
    ctx->built_req.assign(rays_per_object, rays_per_object + sp.K);
    ctx->total_rays = (int)sp.rays;          // upper bounds until read back (frozen objects drop out)
    ctx->total_samples = sp.samples;
    ctx->batch_ready = true;
}

vmap_status sample_impl(vmap_ctx* ctx, const int* rays_per_object, const float* given, cudaMemcpyKind kind) {
    SamplePlan sp;
    if (vmap_status s = sample_plan(ctx, rays_per_object, given, kind, sp)) return s;
    if (ctx->graph_on) {
        cudaGraphExec_t* g = sp.build ? &ctx->g_sample[sp.gi] : &ctx->g_sample_only[sp.gi];
        if (!*g) {
            vmap_status s = capture(ctx, g, [&] { return launch_build_sample(ctx, sp.gi, sp.build); });
            if (s) return s;
        }
        if (vmap_status s = replay(ctx, *g, PS_GRAPH_SAMPLE)) return s;
    } else {
        if (vmap_status s = launch_build_sample(ctx, sp.gi, sp.build)) return s;
    }
    sample_done(ctx, rays_per_object, sp);
    return VMAP_OK;
}

// the FP32 kernels (eval, query) read the transposed shadow: refresh it after BF16 training
vmap_status fresh_shadow(vmap_ctx* ctx) {
    if (!ctx->shadow_stale || ctx->objs.empty()) return VMAP_OK;
    k_shadow_all<<<dim3(16, (unsigned)ctx->objs.size()), 256, 0, ctx->stream>>>(ctx->objs_d, ctx->params_d, ctx->wt_d);
    CHECK_LAUNCH("k_shadow_all");
    ctx->shadow_stale = false;
    return VMAP_OK;
}

vmap_status fill_nan(vmap_ctx* ctx, float* p, size_t n) {
    if (p && n) CU(cudaMemsetAsync(p, 0xFF, n * sizeof(float), ctx->stream));
    return VMAP_OK;
}

}  // namespace

extern "C" {

void vmap_default_config(vmap_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->t_near = 0.05f;
    cfg->depth_pad = 0.10f;
    cfg->d_sigma = 0.03f;
    cfg->t_far = 8.0f;
    cfg->lambda_colour = 5.0f;
    cfg->lambda_occ = 0.0f;
    cfg->lr = 1e-3f;
    cfg->beta1 = 0.9f;
    cfg->beta2 = 0.999f;
    cfg->eps = 1e-8f;
    cfg->precision = VMAP_FP32;
}

const char* vmap_last_error(const vmap_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

vmap_status vmap_init_objects(vmap_ctx** out, const vmap_config* cfg, void* cuda_stream) {
    if (!out || !cfg) return VMAP_ERR_ARG;
    *out = nullptr;
    if (cfg->max_objects <= 0 || cfg->max_rays_total <= 0 || cfg->max_pool_rays <= 0 || !cfg->B)
        return VMAP_ERR_ARG;
    if (cfg->precision != VMAP_FP32 && cfg->precision != VMAP_BF16) return VMAP_ERR_ARG;
    vmap_ctx* ctx = new vmap_ctx();
    ctx->cfg = *cfg;
    ctx->cfg.B = nullptr;
    ctx->stream = (cudaStream_t)cuda_stream;
    std::memcpy(ctx->sp.B, cfg->B, sizeof(float) * NF * 3);
    ctx->sp.t_near = cfg->t_near;
    ctx->sp.depth_pad = cfg->depth_pad;
    ctx->sp.d_sigma = cfg->d_sigma;
    ctx->sp.t_far = cfg->t_far;
    ctx->sp.lam_c = cfg->lambda_colour;
    ctx->sp.lam_o = cfg->lambda_occ;
    ctx->sp.lr = cfg->lr;
    ctx->sp.beta1 = cfg->beta1;
    ctx->sp.beta2 = cfg->beta2;
    ctx->sp.eps = cfg->eps;
    ctx->sp.key0 = (uint32_t)(cfg->seed & 0xFFFFFFFFull);
    ctx->sp.key1 = (uint32_t)(cfg->seed >> 32);
    ctx->bf16 = cfg->precision == VMAP_BF16;

    auto bail = [&](vmap_status s) {
        vmap_destroy(ctx);
        return s;
    };
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) return bail(VMAP_ERR_CUDA);
    // the step's small kernels run between kernels that take most of an SM's
    // shared memory: with the same carveout no SM reconfigures its L1/shared
    // split (an idle gap of microseconds) at each of their boundaries
    for (const void* f : {(const void*)k_sample, (const void*)k_reduce, (const void*)k_build}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return bail(VMAP_ERR_CUDA);
    }
#define ALLOC(ptr, bytes)                                                                      \
    do {                                                                                       \
        e = cudaMalloc((void**)&(ptr), (bytes));                                               \
        if (e != cudaSuccess) return bail(VMAP_ERR_CUDA);                                      \
    } while (0)
    const int K = cfg->max_objects;
    ctx->param_cap = cfg->max_param_floats > 0 ? cfg->max_param_floats : (long long)K * param_count(128);
    ctx->param_cap = (ctx->param_cap + 63) & ~63LL;
    ctx->wt_cap = ctx->param_cap + 64LL * K;   // wt_count(H) <= param_count(H) per object + alignment
    ctx->pool_cap = cfg->max_pool_rays;
    ALLOC(ctx->objs_d, sizeof(ObjDev) * K);
    ALLOC(ctx->ob_d, sizeof(ObjBatch) * K);
    ALLOC(ctx->n_obj_d, sizeof(int));
    ALLOC(ctx->steps_d, sizeof(int) * K);
    ALLOC(ctx->status_d, sizeof(int) * K);
    ALLOC(ctx->req_d, sizeof(int) * K);
    ALLOC(ctx->params_d, sizeof(float) * ctx->param_cap);
    ALLOC(ctx->wt_d, sizeof(float) * ctx->wt_cap);
    ALLOC(ctx->m_d, sizeof(float) * ctx->param_cap);
    ALLOC(ctx->v_d, sizeof(float) * ctx->param_cap);
    ALLOC(ctx->pool_d, sizeof(float) * REC * ctx->pool_cap);
    ALLOC(ctx->pick_d, sizeof(int) * cfg->max_rays_total);
    ALLOC(ctx->t_d, sizeof(float) * (size_t)cfg->max_rays_total * SMAX);
    ALLOC(ctx->bobj_d, sizeof(int) * K);
    ALLOC(ctx->bray_d, sizeof(int) * K);
    ALLOC(ctx->ray_bj_d, sizeof(int) * (size_t)cfg->max_rays_total);
    ctx->tile_cap = cfg->max_rays_total + 16;
    ALLOC(ctx->tiles_d, sizeof(TileDev) * (size_t)ctx->tile_cap * NCLASS);
    ALLOC(ctx->flags_d, sizeof(int) * (size_t)ctx->tile_cap * NCLASS);
    // run slots per class: at most one per CTA plus one per object; the FP32
    // hidden 16-64 classes may also take one per tile (dynamic scheduling) up
    // to DYN_SLOT_BYTES of slots, and are scheduled statically when a step has
    // more tiles than that
    long long part = 0;
    for (int c = 0; c < NCLASS; ++c) {
        ctx->part_base[c] = part;
        const long long stride = param_count(hidden_of(c)) + NEXTRA;
        ctx->dyn_cap[c] = 0;
        if (!ctx->bf16 && c < 3)
            ctx->dyn_cap[c] = (int)std::min<long long>(ctx->tile_cap, DYN_SLOT_BYTES / (stride * (long long)sizeof(float)));
        const long long slots = std::max<long long>((long long)ctx->n_sm * ctas_of(c) * GMULT_MAX + K, ctx->dyn_cap[c]);
        part += slots * stride;
    }
    ALLOC(ctx->part_d, sizeof(float) * part);
    ALLOC(ctx->items_d, sizeof(int2) * (size_t)K * ((param_count(128) + REDUCE_CHUNK - 1) / REDUCE_CHUNK));
    ALLOC(ctx->counts_d, sizeof(int) * BC_N);
    ALLOC(ctx->sig_d, sizeof(int) * (2 + (size_t)K));
    ALLOC(ctx->dyn_d, sizeof(int) * 2 * NCLASS);
    if (!ctx->bf16) {
        // the FP32 tile kernel's encoding copies (hidden 32 and 64: the encoding shares the
        // hidden rows), one block per CTA of the largest grid
        const long long enc_floats[NCLASS] = {0, (long long)DINP * TileSmem<32>::LD, (long long)DINP * TileSmem<64>::LD, 0};
        for (int c = 1; c < 3; ++c)
            ALLOC(ctx->enc_d[c], sizeof(float) * (size_t)enc_floats[c] * ctx->n_sm * ctas_of(c) * GMULT_MAX);
    }
    ALLOC(ctx->done_d, sizeof(int) * K);
    ALLOC(ctx->given_d, sizeof(float) * REC * (size_t)cfg->max_rays_total);
    ALLOC(ctx->loss_d, sizeof(float) * K);
    ALLOC(ctx->loss_pp_d, sizeof(float*));
    ALLOC(ctx->err_d, sizeof(int));
    ALLOC(ctx->img_off_d, sizeof(long long) * K);
    if (ctx->bf16) {
        // img_count(H) - param_count(H) = 11 H - 4 <= 1408, plus 64-element alignment per object
        ctx->img_cap = ctx->param_cap + 1536LL * K;
        ALLOC(ctx->img_d, sizeof(__nv_bfloat16) * ctx->img_cap);
    }
    // width-128 records (grown on demand) and per-tile loss sums, both paths
    ALLOC(ctx->act_pp_d, sizeof(unsigned char*));
    ALLOC(ctx->tile_loss_d, sizeof(float) * 8 * (size_t)ctx->tile_cap);
#undef ALLOC
    e = cudaMemsetAsync(ctx->steps_d, 0, sizeof(int) * K, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status_d, 0, sizeof(int) * K, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->req_d, 0, sizeof(int) * K, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->n_obj_d, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->counts_d, 0, sizeof(int) * BC_N, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->sig_d, 0xFF, sizeof(int) * (2 + (size_t)K), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dyn_d, 0, sizeof(int) * 2 * NCLASS, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->done_d, 0, sizeof(int) * K, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->err_d, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->img_off_d, 0xFF, sizeof(long long) * K, ctx->stream);
    if (e == cudaSuccess && ctx->act_pp_d) e = cudaMemsetAsync(ctx->act_pp_d, 0, sizeof(unsigned char*), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->loss_pp_d, 0, sizeof(float*), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(VMAP_ERR_CUDA);
    *out = ctx;
    return VMAP_OK;
}

vmap_status vmap_destroy(vmap_ctx* ctx) {
    if (!ctx) return VMAP_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    drop_graphs(ctx);
    void* ptrs[] = {ctx->objs_d,   ctx->ob_d,     ctx->n_obj_d,  ctx->steps_d, ctx->status_d, ctx->req_d,
                    ctx->params_d, ctx->wt_d,     ctx->m_d,      ctx->v_d,     ctx->pool_d,   ctx->pick_d,
                    ctx->t_d,      ctx->bobj_d,   ctx->bray_d,   ctx->tiles_d, ctx->flags_d,  ctx->part_d,
                    ctx->items_d,  ctx->counts_d, ctx->given_d,  ctx->loss_d,  ctx->err_d,  ctx->img_off_d,
                    ctx->img_d,    ctx->act_d,    ctx->act_pp_d, ctx->tile_loss_d, ctx->sig_d,  ctx->done_d, ctx->dyn_d,
                    ctx->scene_d,  ctx->ray_bj_d, ctx->loss_pp_d};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (float* p : ctx->enc_d)
        if (p) cudaFree(p);
    for (auto& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
    return VMAP_OK;
}

vmap_status vmap_add_object(vmap_ctx* ctx, const vmap_object_desc* d, const float* init_params, int* out_id) {
    if (!ctx || !d || !out_id) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (!valid_hidden(d->hidden)) return fail(ctx, VMAP_ERR_ARG, "hidden %d not in {16,32,64,128}", d->hidden);
    const int S = d->n_surface + d->n_strat;
    if (d->n_surface < 0 || d->n_strat < 0 || S < 1 || S > SMAX)
        return fail(ctx, VMAP_ERR_ARG, "samples per ray %d+%d not in [1, %d]", d->n_surface, d->n_strat, SMAX);
    if (S > mmax_of(class_of(d->hidden)))
        return fail(ctx, VMAP_ERR_ARG, "samples per ray %d exceed the tile of hidden %d", S, d->hidden);
    if (!(d->scale > 0.f) || !std::isfinite(d->scale)) return fail(ctx, VMAP_ERR_ARG, "scale must be > 0");
    if (!d->rays || d->n_rays < 1) return fail(ctx, VMAP_ERR_ARG, "empty ray pool");
    if ((int)ctx->objs.size() >= ctx->cfg.max_objects)
        return fail(ctx, VMAP_ERR_CAPACITY, "max_objects %d reached", ctx->cfg.max_objects);
    const long long P = param_count(d->hidden);
    const long long poff = (ctx->param_used + 63) & ~63LL;
    const long long woff = (ctx->wt_used + 63) & ~63LL;
    if (poff + P > ctx->param_cap || woff + wt_count(d->hidden) > ctx->wt_cap)
        return fail(ctx, VMAP_ERR_CAPACITY, "parameter arena full");
    if (ctx->pool_used + d->n_rays > ctx->pool_cap)
        return fail(ctx, VMAP_ERR_CAPACITY, "ray pool arena full (%lld + %lld > %lld)", ctx->pool_used, d->n_rays,
                    ctx->pool_cap);
    const int id = (int)ctx->objs.size();
    ObjDev ob{};
    ob.hidden = d->hidden;
    ob.S = S;
    ob.n_surface = d->n_surface;
    ob.n_strat = d->n_strat;
    for (int a = 0; a < 3; ++a) ob.c[a] = d->center[a];
    ob.scale = d->scale;
    ob.param_off = poff;
    ob.wt_off = woff;
    ob.pool_off = ctx->pool_used;
    ob.pool_n = d->n_rays;
    ob.stream = d->stream;
    ob.active = 1;
    CU(cudaMemcpyAsync(ctx->pool_d + ob.pool_off * REC, d->rays, sizeof(float) * REC * d->n_rays,
                       cudaMemcpyDeviceToDevice, ctx->stream));
    if (init_params) {
        CU(cudaMemcpyAsync(ctx->params_d + poff, init_params, sizeof(float) * P, cudaMemcpyDeviceToDevice,
                           ctx->stream));
    } else {
        k_init_params<<<8, 256, 0, ctx->stream>>>(ctx->params_d + poff, d->hidden, d->stream, ctx->sp.key0,
                                                  ctx->sp.key1);
        CHECK_LAUNCH("k_init_params");
    }
    k_shadow<<<16, 256, 0, ctx->stream>>>(ctx->params_d + poff, ctx->wt_d + woff, d->hidden);
    CHECK_LAUNCH("k_shadow");
    long long ioff = -1;
    if (ctx->bf16) {
        ioff = ctx->img_used;
        if (ioff + img_count(d->hidden) > ctx->img_cap) return fail(ctx, VMAP_ERR_CAPACITY, "weight image arena full");
        k_image<<<1, 256, 0, ctx->stream>>>(ctx->params_d + poff, ctx->img_d + ioff, d->hidden);
        CHECK_LAUNCH("k_image");
        ctx->img_used = (ioff + img_count(d->hidden) + 63) & ~63LL;
    }
    CU(cudaMemcpyAsync(ctx->img_off_d + id, &ioff, sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
    ctx->img_off.push_back(ioff);
    CU(cudaMemsetAsync(ctx->m_d + poff, 0, sizeof(float) * P, ctx->stream));
    CU(cudaMemsetAsync(ctx->v_d + poff, 0, sizeof(float) * P, ctx->stream));
    CU(cudaMemsetAsync(ctx->steps_d + id, 0, sizeof(int), ctx->stream));
    CU(cudaMemsetAsync(ctx->status_d + id, 0, sizeof(int), ctx->stream));
    ++ctx->layout_gen;
    CU(cudaMemsetAsync(ctx->req_d + id, 0, sizeof(int), ctx->stream));
    ctx->param_used = poff + P;
    ctx->wt_used = woff + wt_count(d->hidden);
    ctx->pool_used += d->n_rays;
    ctx->objs.push_back(ob);
    if (vmap_status s = upload_obj(ctx, id)) return s;
    const int n = (int)ctx->objs.size();
    CU(cudaMemcpyAsync(ctx->n_obj_d, &n, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    ctx->batch_ready = false;
    *out_id = id;
    return VMAP_OK;
}

vmap_status vmap_sample_rays(vmap_ctx* ctx, const int* rays_per_object) {
    return sample_impl(ctx, rays_per_object, nullptr, cudaMemcpyDeviceToDevice);
}

vmap_status vmap_sample_rays_given(vmap_ctx* ctx, const float* rays, const int* rays_per_object) {
    if (!rays) return fail(ctx, VMAP_ERR_ARG, "null rays");
    return sample_impl(ctx, rays_per_object, rays, cudaMemcpyDeviceToDevice);
}

}  // extern "C"

namespace {
// a batch and its training step as one launch sequence (one graph replay)
vmap_status step_impl(vmap_ctx* ctx, const int* rays_per_object, const float* given, cudaMemcpyKind kind,
                      float* out_loss) {
    SamplePlan sp;
    if (vmap_status s = sample_plan(ctx, rays_per_object, given, kind, sp)) return s;
    const int mask = class_mask(ctx);
    if (vmap_status s = set_loss_dest(ctx, out_loss)) return s;
    auto seq = [&]() -> vmap_status {
        if (vmap_status s = launch_build_sample(ctx, sp.gi, sp.build)) return s;
        ctx->after_sample = !ctx->prof_on || ctx->capturing;   // no profiling event after the sampler
        vmap_status s = launch_train(ctx, mask);
        ctx->after_sample = false;
        return s;
    };
    if (ctx->graph_on) {
        cudaGraphExec_t& g = ctx->g_step[sp.gi][sp.build ? 1 : 0];
        int& gc = ctx->g_step_classes[sp.gi][sp.build ? 1 : 0];
        if (g && gc != mask) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
        if (!g) {
            if (vmap_status s = capture(ctx, &g, seq)) return s;
            gc = mask;
        }
        if (vmap_status s = replay(ctx, g, PS_GRAPH_TRAIN)) return s;
    } else {
        if (vmap_status s = seq()) return s;
    }
    sample_done(ctx, rays_per_object, sp);
    if (ctx->bf16) ctx->shadow_stale = true;
    ctx->batch_ready = false;
    return VMAP_OK;
}
}  // namespace

extern "C" {

vmap_status vmap_step(vmap_ctx* ctx, const int* rays_per_object, float* out_loss) {
    return step_impl(ctx, rays_per_object, nullptr, cudaMemcpyDeviceToDevice, out_loss);
}

vmap_status vmap_train_step(vmap_ctx* ctx, float* out_loss) {
    if (!ctx) return VMAP_ERR_ARG;
    if (!ctx->batch_ready) return fail(ctx, VMAP_ERR_STATE, "train_step needs a fresh vmap_sample_rays");
    const int mask = class_mask(ctx);
    if (vmap_status s = set_loss_dest(ctx, out_loss)) return s;
    if (ctx->graph_on) {
        if (ctx->g_train && ctx->g_classes != mask) {
            cudaGraphExecDestroy(ctx->g_train);
            ctx->g_train = nullptr;
        }
        if (!ctx->g_train) {
            vmap_status s = capture(ctx, &ctx->g_train, [&] { return launch_train(ctx, mask); });
            if (s) return s;
            ctx->g_classes = mask;
        }
        if (vmap_status s = replay(ctx, ctx->g_train, PS_GRAPH_TRAIN)) return s;
    } else {
        if (vmap_status s = launch_train(ctx, mask)) return s;
    }
    // BF16 steps (eager or replayed) leave the FP32 shadow behind the weights
    if (ctx->bf16) ctx->shadow_stale = true;
    ctx->batch_ready = false;
    return VMAP_OK;
}

vmap_status vmap_train_step_host(vmap_ctx* ctx, const float* rays, const int* rays_per_object, float* loss) {
    if (!ctx || !rays || !loss) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (vmap_status s = step_impl(ctx, rays_per_object, rays, cudaMemcpyHostToDevice, nullptr)) return s;
    CU(cudaMemcpyAsync(loss, ctx->loss_d, sizeof(float) * ctx->objs.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return VMAP_OK;
}

vmap_status vmap_forward(vmap_ctx* ctx, float* out_loss) {
    if (!ctx || !out_loss) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (!ctx->batch_ready) return fail(ctx, VMAP_ERR_STATE, "forward needs a drawn batch");
    if (vmap_status s = fill_nan(ctx, out_loss, ctx->objs.size())) return s;
    if (vmap_status s = launch_tiles<MODE_FORWARD>(ctx, class_mask(ctx))) return s;
    return launch_reduce(ctx, RED_LOSS, nullptr, nullptr, out_loss, nullptr);
}

vmap_status vmap_backward(vmap_ctx* ctx, const float* grad_loss, float* grad_params, float* grad_center) {
    if (!ctx || !grad_params) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (!ctx->batch_ready) return fail(ctx, VMAP_ERR_STATE, "backward needs a drawn batch");
    if (grad_center && ctx->bf16)
        return fail(ctx, VMAP_ERR_ARG, "the centre gradient needs an FP32 context");
    const int mask = class_mask(ctx);
    vmap_status s = grad_center ? launch_tiles<MODE_GRAD_CENTER>(ctx, mask) : launch_tiles<MODE_TRAIN>(ctx, mask);
    if (s) return s;
    return launch_reduce(ctx, RED_GRAD, grad_loss, grad_params, nullptr, grad_center);
}

vmap_status vmap_ray_gradients(vmap_ctx* ctx, float* grad_rays) {
    if (!ctx || !grad_rays) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (!ctx->batch_ready) return fail(ctx, VMAP_ERR_STATE, "ray gradients need a drawn batch");
    if (ctx->bf16) return fail(ctx, VMAP_ERR_ARG, "ray gradients need an FP32 context");
    ctx->ray_grad_out = grad_rays;
    vmap_status s = launch_tiles<MODE_GRAD_CENTER>(ctx, class_mask(ctx));
    ctx->ray_grad_out = nullptr;
    return s;
}

vmap_status vmap_pose_step(vmap_ctx* ctx, int obj, const float* dc, const float* meas, int n, float* pose,
                           float* adam, float lr_t, float lr_r, float* rays_work, float* grad_work, float* loss) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (!dc || !meas || !pose || !adam || !rays_work || !grad_work || !loss || n < 1)
        return fail(ctx, VMAP_ERR_ARG, "bad argument");
    if (ctx->bf16) return fail(ctx, VMAP_ERR_ARG, "pose refinement needs an FP32 context");
    if (n > ctx->cfg.max_rays_total) return fail(ctx, VMAP_ERR_CAPACITY, "%d rays exceed max_rays_total", n);
    // the camera's rays from the current pose, their samples
    k_pose_rays<<<(n + 255) / 256, 256, 0, ctx->stream>>>(pose, dc, meas, n, rays_work);
    CHECK_LAUNCH("k_pose_rays");
    std::vector<int> req(ctx->objs.size(), 0);
    req[obj] = n;
    if (vmap_status s = sample_impl(ctx, req.data(), rays_work, cudaMemcpyDeviceToDevice)) return s;
    // one pass: per-ray gradients and the loss sums of the same samples
    if (vmap_status s = fill_nan(ctx, loss, ctx->objs.size())) return s;
    ctx->ray_grad_out = grad_work;
    vmap_status s = launch_tiles<MODE_GRAD_CENTER>(ctx, class_mask(ctx));
    ctx->ray_grad_out = nullptr;
    if (s) return s;
    if (vmap_status s2 = launch_reduce(ctx, RED_LOSS, nullptr, nullptr, loss, nullptr)) return s2;
    // pose gradient and one Adam step on the device
    k_pose_update<<<1, POSE_THREADS, 0, ctx->stream>>>(pose, adam, grad_work, rays_work, n, lr_t, lr_r,
                                                        ctx->cfg.beta1, ctx->cfg.beta2, 1e-12f);
    CHECK_LAUNCH("k_pose_update");
    return VMAP_OK;
}

vmap_status vmap_query_occupancy(vmap_ctx* ctx, int obj, const float* pts, long long n, float* occ, float* rgb) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (vmap_status s = fresh_shadow(ctx)) return s;
    if (n < 0) return fail(ctx, VMAP_ERR_ARG, "negative point count");
    if (n == 0) return VMAP_OK;
    if (!pts || !occ) return fail(ctx, VMAP_ERR_ARG, "null argument");
    const int c = class_of(ctx->objs[obj].hidden);
    TileArgs ta = base_args(ctx);
    ta.eval_obj = obj;
    ta.eval_n = n;
    ta.qpts = pts;
    ta.qocc = occ;
    ta.qrgb = rgb;
    const int rt = mmax_of(c);
    const long long blocks = (n + rt - 1) / rt;
    cudaError_t e = launch_tile_c<MODE_QUERY>(c, (int)blocks, ctx->stream, ctx->sp, ta);
    if (e != cudaSuccess) return fail(ctx, VMAP_ERR_CUDA, "query kernel failed: %s", cudaGetErrorString(e));
    return VMAP_OK;
}

vmap_status vmap_render_depth(vmap_ctx* ctx, int obj, const float* rays, long long n, const float* box_half,
                              int n_samples, float* depth) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (vmap_status s = fresh_shadow(ctx)) return s;
    if (!rays || !box_half || !depth) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (n < 0) return fail(ctx, VMAP_ERR_ARG, "negative ray count");
    const int c = class_of(ctx->objs[obj].hidden);
    if (n_samples < 1 || n_samples > mmax_of(c))
        return fail(ctx, VMAP_ERR_ARG, "n_samples must be in [1, %d] for hidden %d", mmax_of(c), hidden_of(c));
    if (n == 0) return VMAP_OK;
    TileArgs ta = base_args(ctx);
    ta.pool = rays;
    ta.eval_out = depth;
    for (int a = 0; a < 3; ++a) ta.eval_half[a] = box_half[a];
    ta.eval_obj = obj;
    ta.eval_n = n;
    ta.eval_S = n_samples;
    const int rt = std::min(RTMAX, mmax_of(c) / n_samples);
    const long long blocks = (n + rt - 1) / rt;
    cudaError_t e = launch_tile_c<MODE_EVAL>(c, (int)blocks, ctx->stream, ctx->sp, ta);
    if (e != cudaSuccess) return fail(ctx, VMAP_ERR_CUDA, "eval kernel failed: %s", cudaGetErrorString(e));
    return VMAP_OK;
}

vmap_status vmap_render_scene(vmap_ctx* ctx, const float* rays, long long n, const int* objs, int m,
                              const float* box_half, int n_samples, float* depth, float* rgb, float* occ) {
    if (!ctx) return VMAP_ERR_ARG;
    if (!rays || !box_half || !depth) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (n < 0 || m < 1) return fail(ctx, VMAP_ERR_ARG, "need n >= 0 rays and m >= 1 objects");
    for (int j = 0; j < m; ++j) {
        const int k = objs ? objs[j] : j;
        if (vmap_status s = check_obj(ctx, k)) return s;
        const int c = class_of(ctx->objs[k].hidden);
        if (n_samples < 1 || n_samples > mmax_of(c))
            return fail(ctx, VMAP_ERR_ARG, "n_samples must be in [1, %d] for hidden %d", mmax_of(c), hidden_of(c));
    }
    if (n == 0) return VMAP_OK;
    if (vmap_status s = fresh_shadow(ctx)) return s;
    const long long need = (long long)m * n * 5;
    if (need > ctx->scene_cap) {
        CU(cudaStreamSynchronize(ctx->stream));
        if (ctx->scene_d) CU(cudaFree(ctx->scene_d));
        ctx->scene_d = nullptr;
        ctx->scene_cap = 0;
        CU(cudaMalloc((void**)&ctx->scene_d, sizeof(float) * need));
        ctx->scene_cap = need;
    }
    for (int j = 0; j < m; ++j) {
        const int k = objs ? objs[j] : j;
        const int c = class_of(ctx->objs[k].hidden);
        TileArgs ta = base_args(ctx);
        ta.pool = rays;
        ta.eval_out = nullptr;
        ta.eval_rec = ctx->scene_d + (long long)j * n * 5;
        for (int a = 0; a < 3; ++a) ta.eval_half[a] = box_half[3 * j + a];
        ta.eval_obj = k;
        ta.eval_n = n;
        ta.eval_S = n_samples;
        const int rt = std::min(RTMAX, mmax_of(c) / n_samples);
        const long long blocks = (n + rt - 1) / rt;
        cudaError_t e = launch_tile_c<MODE_EVAL>(c, (int)blocks, ctx->stream, ctx->sp, ta);
        if (e != cudaSuccess) return fail(ctx, VMAP_ERR_CUDA, "eval kernel failed: %s", cudaGetErrorString(e));
    }
    const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)ctx->n_sm * 16);
    k_compose<<<blocks, 256, 0, ctx->stream>>>(ctx->scene_d, m, n, depth, rgb, occ);
    CHECK_LAUNCH("k_compose");
    return VMAP_OK;
}

vmap_status vmap_extract_mesh(vmap_ctx* ctx, int obj, const float* box_half, int res, float level, float* tris,
                              long long max_tris, long long* n_tris) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (!box_half || !n_tris) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (res < 1 || res > 512) return fail(ctx, VMAP_ERR_ARG, "res must be in [1, 512]");
    if (max_tris < 0 || (max_tris > 0 && !tris)) return fail(ctx, VMAP_ERR_ARG, "bad triangle buffer");
    if (vmap_status s = fresh_shadow(ctx)) return s;
    const ObjDev& ob = ctx->objs[obj];
    const long long n1 = res + 1, nv = n1 * n1 * n1, nc = (long long)res * res * res;
    // scratch: lattice points, occupancy, per-cube counts, offsets
    const size_t b_pts = sizeof(float) * 3 * nv, b_occ = sizeof(float) * nv, b_cnt = sizeof(int) * nc;
    const size_t o_occ = (b_pts + 255) & ~(size_t)255, o_cnt = (o_occ + b_occ + 255) & ~(size_t)255;
    const size_t o_off = (o_cnt + b_cnt + 255) & ~(size_t)255, total = o_off + sizeof(long long) * (nc + 1);
    unsigned char* scratch = nullptr;
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaMalloc((void**)&scratch, total));
    float* pts = (float*)scratch;
    float* occ = (float*)(scratch + o_occ);
    int* counts = (int*)(scratch + o_cnt);
    long long* offs = (long long*)(scratch + o_off);
    MtGrid g{};
    g.occ = occ;
    g.res = res;
    g.level = level;
    for (int a = 0; a < 3; ++a) {
        g.o[a] = ob.c[a] - box_half[a];
        g.s[a] = 2.f * box_half[a] / (float)res;
    }
    const int blocks = (int)std::min<long long>((nv + 255) / 256, (long long)ctx->n_sm * 32);
    k_lattice_points<<<blocks, 256, 0, ctx->stream>>>(pts, res, g.o[0], g.o[1], g.o[2], g.s[0], g.s[1], g.s[2]);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        const int c = class_of(ob.hidden);
        TileArgs ta = base_args(ctx);
        ta.eval_obj = obj;
        ta.eval_n = nv;
        ta.qpts = pts;
        ta.qocc = occ;
        ta.qrgb = nullptr;
        e = launch_tile_c<MODE_QUERY>(c, (int)((nv + mmax_of(c) - 1) / mmax_of(c)), ctx->stream, ctx->sp, ta);
    }
    const int cblocks = (int)std::min<long long>((nc + 255) / 256, (long long)ctx->n_sm * 32);
    if (e == cudaSuccess) {
        k_mt_count<<<cblocks, 256, 0, ctx->stream>>>(g, counts);
        k_scan_counts<<<1, BUILD_THREADS, 0, ctx->stream>>>(counts, nc, offs);
        if (max_tris > 0) k_mt_emit<<<cblocks, 256, 0, ctx->stream>>>(g, offs, tris, max_tris);
        e = cudaGetLastError();
    }
    long long n = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n, offs + nc, sizeof n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(scratch);
    if (e != cudaSuccess) return fail(ctx, VMAP_ERR_CUDA, "mesh extraction failed: %s", cudaGetErrorString(e));
    *n_tris = n;
    return VMAP_OK;
}

vmap_status vmap_get_object_state(vmap_ctx* ctx, int obj, float* params, float* m, float* v, int* step) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    const ObjDev& ob = ctx->objs[obj];
    const size_t bytes = sizeof(float) * param_count(ob.hidden);
    if (params)
        CU(cudaMemcpyAsync(params, ctx->params_d + ob.param_off, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (m) CU(cudaMemcpyAsync(m, ctx->m_d + ob.param_off, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (v) CU(cudaMemcpyAsync(v, ctx->v_d + ob.param_off, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (step) {
        CU(cudaMemcpyAsync(step, ctx->steps_d + obj, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    return VMAP_OK;
}

vmap_status vmap_set_object_state(vmap_ctx* ctx, int obj, const float* params, const float* m, const float* v,
                                  int step) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (step < 0) return fail(ctx, VMAP_ERR_ARG, "negative step");
    const ObjDev& ob = ctx->objs[obj];
    const size_t bytes = sizeof(float) * param_count(ob.hidden);
    if (params) {
        CU(cudaMemcpyAsync(ctx->params_d + ob.param_off, params, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        k_shadow<<<16, 256, 0, ctx->stream>>>(ctx->params_d + ob.param_off, ctx->wt_d + ob.wt_off, ob.hidden);
        CHECK_LAUNCH("k_shadow");
        if (ctx->img_off[obj] >= 0) {
            k_image<<<1, 256, 0, ctx->stream>>>(ctx->params_d + ob.param_off, ctx->img_d + ctx->img_off[obj], ob.hidden);
            CHECK_LAUNCH("k_image");
        }
    }
    if (m) CU(cudaMemcpyAsync(ctx->m_d + ob.param_off, m, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (v) CU(cudaMemcpyAsync(ctx->v_d + ob.param_off, v, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->steps_d + obj, &step, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->batch_ready = false;
    return VMAP_OK;
}

vmap_status vmap_param_arena_size(vmap_ctx* ctx, long long* n) {
    if (!ctx || !n) return VMAP_ERR_ARG;
    *n = ctx->param_used;
    return VMAP_OK;
}

vmap_status vmap_get_params(vmap_ctx* ctx, float* arena) {
    if (!ctx || !arena) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (ctx->param_used)
        CU(cudaMemcpyAsync(arena, ctx->params_d, sizeof(float) * ctx->param_used, cudaMemcpyDeviceToDevice,
                           ctx->stream));
    return VMAP_OK;
}

vmap_status vmap_set_params(vmap_ctx* ctx, const float* arena) {
    if (!ctx || !arena) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (!ctx->param_used) return VMAP_OK;
    CU(cudaMemcpyAsync(ctx->params_d, arena, sizeof(float) * ctx->param_used, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    for (size_t k = 0; k < ctx->objs.size(); ++k) {
        const ObjDev& ob = ctx->objs[k];
        k_shadow<<<16, 256, 0, ctx->stream>>>(ctx->params_d + ob.param_off, ctx->wt_d + ob.wt_off, ob.hidden);
        CHECK_LAUNCH("k_shadow");
        if (ctx->img_off[k] >= 0) {
            k_image<<<1, 256, 0, ctx->stream>>>(ctx->params_d + ob.param_off, ctx->img_d + ctx->img_off[k], ob.hidden);
            CHECK_LAUNCH("k_image");
        }
    }
    return VMAP_OK;
}

vmap_status vmap_set_object_active(vmap_ctx* ctx, int obj, int active) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    ctx->objs[obj].active = active ? 1 : 0;
    if (active) CU(cudaMemsetAsync(ctx->status_d + obj, 0, sizeof(int), ctx->stream));
    ctx->batch_ready = false;
    return upload_obj(ctx, obj);
}

vmap_status vmap_set_object_center(vmap_ctx* ctx, int obj, const float* center) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (!center) return fail(ctx, VMAP_ERR_ARG, "null center");
    for (int a = 0; a < 3; ++a) ctx->objs[obj].c[a] = center[a];
    return upload_obj(ctx, obj, false);   // the centre is not a layout input
}

vmap_status vmap_object_info(vmap_ctx* ctx, int obj, int* hidden, int* param_count_out, long long* param_offset,
                             int* spr) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    const ObjDev& ob = ctx->objs[obj];
    if (hidden) *hidden = ob.hidden;
    if (param_count_out) *param_count_out = (int)param_count(ob.hidden);
    if (param_offset) *param_offset = ob.param_off;
    if (spr) *spr = ob.S;
    return VMAP_OK;
}

vmap_status vmap_num_objects(vmap_ctx* ctx, int* n) {
    if (!ctx || !n) return VMAP_ERR_ARG;
    *n = (int)ctx->objs.size();
    return VMAP_OK;
}

vmap_status vmap_batch_info(vmap_ctx* ctx, int* n_rays, long long* n_samples) {
    if (!ctx) return VMAP_ERR_ARG;
    int c[BC_N];
    CU(cudaMemcpyAsync(c, ctx->counts_d, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->total_rays = c[BC_RAYS];
    ctx->total_samples = ((long long)c[BC_SAMPLES_HI] << 31) | (long long)c[BC_SAMPLES_LO];
    if (n_rays) *n_rays = ctx->total_rays;
    if (n_samples) *n_samples = ctx->total_samples;
    return VMAP_OK;
}

vmap_status vmap_get_samples(vmap_ctx* ctx, int* pick, float* t) {
    if (!ctx) return VMAP_ERR_ARG;
    if (vmap_status s = vmap_batch_info(ctx, nullptr, nullptr)) return s;
    if (pick && ctx->total_rays)
        CU(cudaMemcpyAsync(pick, ctx->pick_d, sizeof(int) * ctx->total_rays, cudaMemcpyDeviceToDevice, ctx->stream));
    if (t && ctx->total_samples)
        CU(cudaMemcpyAsync(t, ctx->t_d, sizeof(float) * ctx->total_samples, cudaMemcpyDeviceToDevice, ctx->stream));
    return VMAP_OK;
}

vmap_status vmap_sync_status(vmap_ctx* ctx, int* n_faulted, int* ids, int max_ids) {
    if (!ctx) return VMAP_ERR_ARG;
    const int K = (int)ctx->objs.size();
    std::vector<int> st(K);
    if (K) CU(cudaMemcpyAsync(st.data(), ctx->status_d, sizeof(int) * K, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    int timed_out = 0;
    CU(cudaMemcpy(&timed_out, ctx->err_d, sizeof(int), cudaMemcpyDeviceToHost));
    if (timed_out) {   // reported once: the flag is cleared, the next steps update objects again
        CU(cudaMemset(ctx->err_d, 0, sizeof(int)));
        return fail(ctx, VMAP_ERR_TIMEOUT, "a tensor-core wait gave up (MMA or copy not complete within the poll limit)");
    }
    int nf = 0;
    for (int k = 0; k < K; ++k)
        if (st[k]) {
            if (ids && nf < max_ids) ids[nf] = k;
            ++nf;
        }
    if (n_faulted) *n_faulted = nf;
    return nf ? VMAP_ERR_NAN : VMAP_OK;
}

vmap_status vmap_profile_enable(vmap_ctx* ctx, int on) {
    if (!ctx) return VMAP_ERR_ARG;
    prof_flush(ctx);
    ctx->prof_on = on != 0;
    return VMAP_OK;
}

vmap_status vmap_profile_reset(vmap_ctx* ctx) {
    if (!ctx) return VMAP_ERR_ARG;
    prof_flush(ctx);
    for (int i = 0; i < PS_N; ++i) {
        ctx->prof_ms[i] = 0.0;
        ctx->prof_n[i] = 0;
    }
    return VMAP_OK;
}

vmap_status vmap_profile_read(vmap_ctx* ctx, int slot, const char** name, long long* launches, double* total_ms) {
    if (!ctx) return VMAP_ERR_ARG;
    if (slot < 0 || slot >= PS_N) return VMAP_ERR_ARG;
    prof_flush(ctx);
    if (name) {
        *name = (slot >= PS_TILE && slot < PS_TILE + NCLASS && ctx->bf16) ? kProfNamesBf16[slot - PS_TILE]
                                                                         : kProfNames[slot];
        if (!ctx->bf16 && slot == PS_TILE + 3) *name = "k_w32_fb<128>";
        if (!ctx->bf16 && slot == PS_WIDE_DW) *name = "k_w32_dw<128>";
    }
    if (launches) *launches = ctx->prof_n[slot];
    if (total_ms) *total_ms = ctx->prof_ms[slot];
    return VMAP_OK;
}

vmap_status vmap_warmstart(vmap_ctx* ctx, int obj, vmap_hyper* h, const float* X) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (!h || !X) return fail(ctx, VMAP_ERR_ARG, "null argument");
    const ObjDev& ob = ctx->objs[obj];
    int P = 0;
    vmap_hyper_param_count(h, nullptr, &P);
    if (P != (int)param_count(ob.hidden))
        return fail(ctx, VMAP_ERR_ARG, "hypernetwork emits %d parameters, object %d has %lld", P, obj,
                    param_count(ob.hidden));
    CU(cudaStreamSynchronize(ctx->stream));
    if (vmap_status s = vmap_hyper_predict(h, 1, X, ctx->params_d + ob.param_off))
        return fail(ctx, s, "hypernetwork predict failed: %s", vmap_hyper_last_error(h));
    CU(cudaDeviceSynchronize());
    const size_t bytes = sizeof(float) * param_count(ob.hidden);
    k_shadow<<<16, 256, 0, ctx->stream>>>(ctx->params_d + ob.param_off, ctx->wt_d + ob.wt_off, ob.hidden);
    CHECK_LAUNCH("k_shadow");
    if (ctx->img_off[obj] >= 0) {
        k_image<<<1, 256, 0, ctx->stream>>>(ctx->params_d + ob.param_off, ctx->img_d + ctx->img_off[obj], ob.hidden);
        CHECK_LAUNCH("k_image");
    }
    CU(cudaMemsetAsync(ctx->m_d + ob.param_off, 0, bytes, ctx->stream));
    CU(cudaMemsetAsync(ctx->v_d + ob.param_off, 0, bytes, ctx->stream));
    CU(cudaMemsetAsync(ctx->steps_d + obj, 0, sizeof(int), ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->batch_ready = false;
    return VMAP_OK;
}

vmap_status vmap_set_wait_limit(vmap_ctx* ctx, long long polls) {
    if (!ctx) return VMAP_ERR_ARG;
    if (polls < 0) return fail(ctx, VMAP_ERR_ARG, "negative poll limit");
    if (polls != ctx->wait_polls) {
        drop_graphs(ctx);   // captured launches carry the limit as an argument
        ctx->wait_polls = polls;
    }
    return VMAP_OK;
}

vmap_status vmap_set_graph(vmap_ctx* ctx, int on) {
    if (!ctx) return VMAP_ERR_ARG;
    drop_graphs(ctx);
    ctx->graph_on = on != 0;
    return VMAP_OK;
}

vmap_status vmap_get_launch(vmap_ctx* ctx, int* rays_per_tile, int* grid_mult) {
    if (!ctx) return VMAP_ERR_ARG;
    for (int c = 0; c < NCLASS; ++c) {
        if (rays_per_tile) rays_per_tile[c] = ctx->rt[c];
        if (grid_mult) grid_mult[c] = ctx->gmult[c];
    }
    return VMAP_OK;
}

vmap_status vmap_set_launch(vmap_ctx* ctx, const int* rays_per_tile, const int* grid_mult) {
    if (!ctx) return VMAP_ERR_ARG;
    for (int c = 0; c < NCLASS; ++c) {
        if (rays_per_tile && (rays_per_tile[c] < 1 || rays_per_tile[c] > RTMAX))
            return fail(ctx, VMAP_ERR_ARG, "rays per tile must be in [1, %d]", RTMAX);
        if (grid_mult && (grid_mult[c] < 1 || grid_mult[c] > GMULT_MAX))
            return fail(ctx, VMAP_ERR_ARG, "grid multiplier must be in [1, %d]", GMULT_MAX);
    }
    drop_graphs(ctx);
    for (int c = 0; c < NCLASS; ++c) {
        if (rays_per_tile) ctx->rt[c] = rays_per_tile[c];
        if (grid_mult) ctx->gmult[c] = grid_mult[c];
    }
    ctx->batch_ready = false;
    return VMAP_OK;
}

vmap_status vmap_autotune(vmap_ctx* ctx, const int* rays_per_object, int reps, float* best_ms) {
    if (!ctx || !rays_per_object || reps < 1) return fail(ctx, VMAP_ERR_ARG, "bad argument");
    const int mask = class_mask(ctx);
    // The candidates are timed on real steps (sampling, tile kernels, reduce,
    // Adam; graph-replayed when graph mode is on, with the overlapped
    // launches), so the training state is saved first and put back at the end.
    const int K = (int)ctx->objs.size();
    const size_t np = (size_t)ctx->param_used, nw = ctx->bf16 ? 0 : (size_t)ctx->wt_used;
    const size_t ni = ctx->bf16 ? (size_t)ctx->img_used : 0;
    const size_t bytes = 3 * np * sizeof(float) + nw * sizeof(float) + ni * sizeof(__nv_bfloat16) + 2 * (size_t)K * sizeof(int);
    unsigned char* snap = nullptr;
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaMalloc((void**)&snap, std::max<size_t>(bytes, 16)));
    const bool prof = ctx->prof_on;
    prof_flush(ctx);
    ctx->prof_on = false;
    struct Part { void* p; size_t n; };
    const Part parts[] = {{ctx->params_d, np * sizeof(float)}, {ctx->m_d, np * sizeof(float)},
                          {ctx->v_d, np * sizeof(float)},      {ctx->wt_d, nw * sizeof(float)},
                          {ctx->img_d, ni * sizeof(__nv_bfloat16)}, {ctx->steps_d, K * sizeof(int)},
                          {ctx->status_d, K * sizeof(int)}};
    auto copy_state = [&](bool save) -> cudaError_t {
        size_t off = 0;
        for (const Part& q : parts) {
            if (q.n) {
                cudaError_t e = save ? cudaMemcpyAsync(snap + off, q.p, q.n, cudaMemcpyDeviceToDevice, ctx->stream)
                                     : cudaMemcpyAsync(q.p, snap + off, q.n, cudaMemcpyDeviceToDevice, ctx->stream);
                if (e != cudaSuccess) return e;
            }
            off += q.n;
        }
        return cudaStreamSynchronize(ctx->stream);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = copy_state(true);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    vmap_status status = ce == cudaSuccess ? VMAP_OK : fail(ctx, VMAP_ERR_CUDA, "autotune set-up: %s", cudaGetErrorString(ce));
    // one candidate: two untimed steps (graph capture, layout build), then `reps` timed
    auto time_steps = [&](float& ms) -> vmap_status {
        drop_graphs(ctx);
        for (int i = 0; i < 2; ++i)
            if (vmap_status s = step_impl(ctx, rays_per_object, nullptr, cudaMemcpyDeviceToDevice, nullptr)) return s;
        CU(cudaEventRecord(e0, ctx->stream));
        for (int r = 0; r < reps; ++r)
            if (vmap_status s = step_impl(ctx, rays_per_object, nullptr, cudaMemcpyDeviceToDevice, nullptr)) return s;
        CU(cudaEventRecord(e1, ctx->stream));
        CU(cudaEventSynchronize(e1));
        CU(cudaEventElapsedTime(&ms, e0, e1));
        ms /= reps;
        return VMAP_OK;
    };
    float best = 1e30f;
    if (status == VMAP_OK) status = time_steps(best);
    // coordinate descent over the width classes present: each class's
    // (rays per tile, grid multiplier) swept with the others held; a second
    // pass if the first changed anything
    for (int pass = 0; pass < 2 && status == VMAP_OK; ++pass) {
        bool changed = false;
        for (int c = NCLASS - 1; c >= 0 && status == VMAP_OK; --c) {
            if (!(mask & (1 << c))) continue;
            int Smin = SMAX;
            for (const ObjDev& o : ctx->objs)
                if (class_of(o.hidden) == c) Smin = std::min(Smin, o.S);
            const int rt_hi = std::max(1, std::min(RTMAX, class_mmax(ctx, c) / Smin));
            int best_rt = ctx->rt[c], best_g = ctx->gmult[c];
            for (int g = 1; g <= GMULT_MAX && status == VMAP_OK; ++g) {
                for (int rt = rt_hi; rt >= 1 && status == VMAP_OK; rt = rt > 4 ? rt - 1 : rt / 2) {
                    if (rt == best_rt && g == best_g) {
                        if (rt == 1) break;
                        continue;   // the current shape: already timed
                    }
                    ctx->rt[c] = rt;
                    ctx->gmult[c] = g;
                    float ms = 0.f;
                    status = time_steps(ms);
                    if (status) break;
                    if (ms < best) {
                        best = ms;
                        best_rt = rt;
                        best_g = g;
                        changed = true;
                    }
                    if (rt == 1) break;
                }
            }
            ctx->rt[c] = best_rt;
            ctx->gmult[c] = best_g;
        }
        if (!changed) break;
    }
    if (best_ms)
        for (int c = 0; c < NCLASS; ++c) best_ms[c] = (mask & (1 << c)) ? best : 0.f;
    drop_graphs(ctx);
    ce = copy_state(false);
    if (status == VMAP_OK && ce != cudaSuccess)
        status = fail(ctx, VMAP_ERR_CUDA, "autotune restore: %s", cudaGetErrorString(ce));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(snap);
    if (ctx->bf16) ctx->shadow_stale = true;
    ctx->prof_on = prof;
    ctx->batch_ready = false;
    return status;
}

}  // extern "C"
