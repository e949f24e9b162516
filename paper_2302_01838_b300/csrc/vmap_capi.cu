// C ABI of the vMAP training library: context, object table, batch
// construction and kernel launches. See include/vmap.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vmap.h"
#include "vmap_common.cuh"
#include "vmap_optim.cuh"
#include "vmap_sample.cuh"
#include "vmap_tile_fp32.cuh"

using namespace vmapk;

struct vmap_ctx {
    vmap_config cfg{};
    cudaStream_t stream = nullptr;
    std::string err;
    StepParams sp{};
    int device = 0;

    // object table
    std::vector<ObjDev> objs;
    ObjDev* objs_d = nullptr;
    int* steps_d = nullptr;
    int* status_d = nullptr;

    // arenas
    float* params_d = nullptr;
    float* wt_d = nullptr;
    float* m_d = nullptr;
    float* v_d = nullptr;
    long long param_used = 0, param_cap = 0, wt_used = 0, wt_cap = 0;
    float* pool_d = nullptr;
    long long pool_used = 0, pool_cap = 0;

    // batch
    int* pick_d = nullptr;
    float* t_d = nullptr;
    int* bobj_d = nullptr;
    int* bray_d = nullptr;
    TileDev* tiles_d = nullptr;
    float* part_d = nullptr;
    long long part_cap = 0;
    int tile_cap = 0;
    bool batch_ready = false;
    int nb = 0;
    int total_rays = 0;
    long long total_samples = 0;
    std::vector<int> bobj;
    int cls_begin[4] = {0, 0, 0, 0}, cls_count[4] = {0, 0, 0, 0};
    int n_tiles = 0;
    int max_chunks = 1;
    bool batch_given = false;      // the batch's rays came from the caller (staging buffer)
    float* given_d = nullptr;      // [max_rays_total][12] staging for caller-given rays
    float* loss_d = nullptr;       // [max_objects] loss scratch of vmap_train_step_host

    // profiling: CUDA events around every kernel launch, on the context stream
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_free;
    struct Pending { int slot; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    double prof_ms[16] = {0};
    long long prof_n[16] = {0};
};

namespace {

const int kHidden[4] = {16, 32, 64, 128};

enum ProfSlot { PS_SAMPLE = 0, PS_TILE = 1 /* + hidden class */, PS_REDUCE = 5, PS_FINISH = 6, PS_N = 7 };
const char* kProfNames[PS_N] = {"k_sample", "k_tile_fp32<16>", "k_tile_fp32<32>", "k_tile_fp32<64>",
                                "k_tile_fp32<128>", "k_reduce", "k_finish"};

// returns a pending index (or -1) after recording the start event
int prof_begin(vmap_ctx* ctx, int slot) {
    if (!ctx->prof_on) return -1;
    cudaEvent_t ev[2];
    for (int i = 0; i < 2; ++i) {
        if (ctx->ev_free.empty()) {
            if (cudaEventCreate(&ev[i]) != cudaSuccess) return -1;
        } else {
            ev[i] = ctx->ev_free.back();
            ctx->ev_free.pop_back();
        }
    }
    cudaEventRecord(ev[0], ctx->stream);
    ctx->pending.push_back({slot, ev[0], ev[1]});
    return (int)ctx->pending.size() - 1;
}

void prof_end(vmap_ctx* ctx, int idx) {
    if (idx >= 0) cudaEventRecord(ctx->pending[idx].b, ctx->stream);
}

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

int hidden_class(int H) {
    for (int c = 0; c < 4; ++c)
        if (kHidden[c] == H) return c;
    return -1;
}

int mmax_of(int H) {
    switch (H) {
        case 16: return TileCfg<16>::MMAX;
        case 32: return TileCfg<32>::MMAX;
        case 64: return TileCfg<64>::MMAX;
        default: return TileCfg<128>::MMAX;
    }
}

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

template <int H>
size_t tile_smem() { return TileSmem<H>::BYTES; }

size_t tile_smem_of(int H) {
    switch (H) {
        case 16: return tile_smem<16>();
        case 32: return tile_smem<32>();
        case 64: return tile_smem<64>();
        default: return tile_smem<128>();
    }
}

template <int H, int MODE>
cudaError_t launch_tile(int n_tiles, cudaStream_t st, const StepParams& sp, const TileArgs& ta) {
    static bool attr_set = false;
    const size_t smem = TileSmem<H>::BYTES;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_fp32<H, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (n_tiles <= 0) return cudaSuccess;
    k_tile_fp32<H, MODE><<<n_tiles, NTHREADS, smem, st>>>(sp, ta);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_tile_h(int H, int n_tiles, cudaStream_t st, const StepParams& sp,
                          const TileArgs& ta) {
    switch (H) {
        case 16: return launch_tile<16, MODE>(n_tiles, st, sp, ta);
        case 32: return launch_tile<32, MODE>(n_tiles, st, sp, ta);
        case 64: return launch_tile<64, MODE>(n_tiles, st, sp, ta);
        default: return launch_tile<128, MODE>(n_tiles, st, sp, ta);
    }
}

vmap_status check_obj(vmap_ctx* ctx, int obj) {
    if (!ctx) return VMAP_ERR_ARG;
    if (obj < 0 || obj >= (int)ctx->objs.size())
        return fail(ctx, VMAP_ERR_ARG, "object index %d out of range [0, %d)", obj,
                    (int)ctx->objs.size());
    return VMAP_OK;
}

vmap_status upload_objs(vmap_ctx* ctx) {
    if (ctx->objs.empty()) return VMAP_OK;
    CU(cudaMemcpyAsync(ctx->objs_d, ctx->objs.data(), sizeof(ObjDev) * ctx->objs.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    // the host vector may change before the copy runs: make the copy complete
    CU(cudaStreamSynchronize(ctx->stream));
    return VMAP_OK;
}

TileArgs base_args(vmap_ctx* ctx) {
    TileArgs ta{};
    ta.objs = ctx->objs_d;
    ta.tiles = ctx->tiles_d;
    ta.pool = ctx->batch_given ? ctx->given_d : ctx->pool_d;
    ta.pick = ctx->pick_d;
    ta.tbuf = ctx->t_d;
    ta.params = ctx->params_d;
    ta.wt = ctx->wt_d;
    ta.part = ctx->part_d;
    return ta;
}

template <int MODE>
vmap_status run_tiles(vmap_ctx* ctx) {
    TileArgs ta = base_args(ctx);
    for (int c = 0; c < 4; ++c) {
        if (ctx->cls_count[c] == 0) continue;
        ta.tile_begin = ctx->cls_begin[c];
        const int pi = MODE == MODE_TRAIN ? prof_begin(ctx, PS_TILE + c) : -1;
        cudaError_t e = launch_tile_h<MODE>(kHidden[c], ctx->cls_count[c], ctx->stream, ctx->sp, ta);
        prof_end(ctx, pi);
        if (e != cudaSuccess)
            return fail(ctx, VMAP_ERR_CUDA, "tile kernel (H=%d) failed: %s", kHidden[c],
                        cudaGetErrorString(e));
    }
    return VMAP_OK;
}

vmap_status run_reduce(vmap_ctx* ctx, int mode, const float* grad_loss, float* grad_out,
                       float* loss_out, float* dcenter_out) {
    if (ctx->nb == 0) return VMAP_OK;
    dim3 grid(ctx->max_chunks, ctx->nb);
    const int pi = prof_begin(ctx, PS_REDUCE);
    k_reduce<<<grid, 256, 0, ctx->stream>>>(ctx->sp, ctx->objs_d, ctx->bobj_d, ctx->part_d,
                                            ctx->params_d, ctx->wt_d, ctx->m_d, ctx->v_d,
                                            ctx->steps_d, ctx->status_d, mode, grad_loss, grad_out,
                                            loss_out, dcenter_out);
    prof_end(ctx, pi);
    CHECK_LAUNCH("k_reduce");
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
    if (cfg->precision != VMAP_FP32) return VMAP_ERR_ARG;
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

    auto bail = [&](vmap_status s) { vmap_destroy(ctx); return s; };
    cudaError_t e;
#define ALLOC(ptr, bytes)                                                                      \
    do {                                                                                       \
        e = cudaMalloc((void**)&(ptr), (bytes));                                               \
        if (e != cudaSuccess) return bail(VMAP_ERR_CUDA);                                      \
    } while (0)
    cudaGetDevice(&ctx->device);
    const int K = cfg->max_objects;
    ctx->param_cap = cfg->max_param_floats > 0 ? cfg->max_param_floats : (long long)K * param_count(128);
    ctx->param_cap = (ctx->param_cap + 63) & ~63LL;
    ctx->wt_cap = ctx->param_cap + 64LL * K;   // wt_count(H) <= param_count(H) per object + alignment
    ctx->pool_cap = cfg->max_pool_rays;
    ALLOC(ctx->objs_d, sizeof(ObjDev) * K);
    ALLOC(ctx->steps_d, sizeof(int) * K);
    ALLOC(ctx->status_d, sizeof(int) * K);
    ALLOC(ctx->params_d, sizeof(float) * ctx->param_cap);
    ALLOC(ctx->wt_d, sizeof(float) * ctx->wt_cap);
    ALLOC(ctx->m_d, sizeof(float) * ctx->param_cap);
    ALLOC(ctx->v_d, sizeof(float) * ctx->param_cap);
    ALLOC(ctx->pool_d, sizeof(float) * REC * ctx->pool_cap);
    ALLOC(ctx->pick_d, sizeof(int) * cfg->max_rays_total);
    ALLOC(ctx->t_d, sizeof(float) * (size_t)cfg->max_rays_total * SMAX);
    ALLOC(ctx->bobj_d, sizeof(int) * K);
    ALLOC(ctx->bray_d, sizeof(int) * (K + 1));
    // tiles: every object contributes at most ceil(R_k / rt_k) <= R_k tiles
    ctx->tile_cap = cfg->max_rays_total + K;
    ALLOC(ctx->tiles_d, sizeof(TileDev) * ctx->tile_cap);
    ALLOC(ctx->given_d, sizeof(float) * REC * (size_t)cfg->max_rays_total);
    ALLOC(ctx->loss_d, sizeof(float) * K);
#undef ALLOC
    e = cudaMemsetAsync(ctx->steps_d, 0, sizeof(int) * K, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status_d, 0, sizeof(int) * K, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(VMAP_ERR_CUDA);
    *out = ctx;
    return VMAP_OK;
}

vmap_status vmap_destroy(vmap_ctx* ctx) {
    if (!ctx) return VMAP_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    void* ptrs[] = {ctx->objs_d, ctx->steps_d, ctx->status_d, ctx->params_d, ctx->wt_d, ctx->m_d,
                    ctx->v_d, ctx->pool_d, ctx->pick_d, ctx->t_d, ctx->bobj_d, ctx->bray_d,
                    ctx->tiles_d, ctx->part_d, ctx->given_d, ctx->loss_d};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
    delete ctx;
    return VMAP_OK;
}

vmap_status vmap_add_object(vmap_ctx* ctx, const vmap_object_desc* d, const float* init_params,
                            int* out_id) {
    if (!ctx || !d || !out_id) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (hidden_class(d->hidden) < 0) return fail(ctx, VMAP_ERR_ARG, "hidden %d not in {16,32,64,128}", d->hidden);
    const int S = d->n_surface + d->n_strat;
    if (d->n_surface < 0 || d->n_strat < 0 || S < 1 || S > SMAX)
        return fail(ctx, VMAP_ERR_ARG, "samples per ray %d+%d not in [1, %d]", d->n_surface, d->n_strat, SMAX);
    if (S > mmax_of(d->hidden))
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
        return fail(ctx, VMAP_ERR_CAPACITY, "ray pool arena full (%lld + %lld > %lld)",
                    ctx->pool_used, d->n_rays, ctx->pool_cap);
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
        CU(cudaMemcpyAsync(ctx->params_d + poff, init_params, sizeof(float) * P,
                           cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        k_init_params<<<8, 256, 0, ctx->stream>>>(ctx->params_d + poff, d->hidden, d->stream,
                                                  ctx->sp.key0, ctx->sp.key1);
        CHECK_LAUNCH("k_init_params");
    }
    k_shadow<<<16, 256, 0, ctx->stream>>>(ctx->params_d + poff, ctx->wt_d + woff, d->hidden);
    CHECK_LAUNCH("k_shadow");
    CU(cudaMemsetAsync(ctx->m_d + poff, 0, sizeof(float) * P, ctx->stream));
    CU(cudaMemsetAsync(ctx->v_d + poff, 0, sizeof(float) * P, ctx->stream));
    CU(cudaMemsetAsync(ctx->steps_d + id, 0, sizeof(int), ctx->stream));
    CU(cudaMemsetAsync(ctx->status_d + id, 0, sizeof(int), ctx->stream));
    ctx->param_used = poff + P;
    ctx->wt_used = woff + wt_count(d->hidden);
    ctx->pool_used += d->n_rays;
    ctx->objs.push_back(ob);
    ctx->max_chunks = std::max(ctx->max_chunks, (int)((P + 1023) / 1024));
    ctx->batch_ready = false;
    *out_id = id;
    return upload_objs(ctx);
}

}  // extern "C"

namespace {
// Build the batch: rays_per_object[k] rays of every active object. With
// given == NULL the rays are picked from the objects' pools; otherwise given
// holds sum_k R_k records (object-major, active objects with R_k > 0, in
// index order) in memory of the kind `kind`, which are staged on the device.
vmap_status sample_impl(vmap_ctx* ctx, const int* rays_per_object, const float* given, cudaMemcpyKind kind) {
    if (!ctx || !rays_per_object) return fail(ctx, VMAP_ERR_ARG, "null argument");
    const int K = (int)ctx->objs.size();
    long long rays = 0, samples = 0, part = 0;
    int tiles = 0;
    for (int k = 0; k < K; ++k) {
        if (rays_per_object[k] < 0) return fail(ctx, VMAP_ERR_ARG, "negative ray count for object %d", k);
        const ObjDev& ob = ctx->objs[k];
        const int R = ob.active ? rays_per_object[k] : 0;
        if (R == 0) continue;
        const int rt = mmax_of(ob.hidden) / ob.S;
        const int nt = (R + rt - 1) / rt;
        rays += R;
        samples += (long long)R * ob.S;
        tiles += nt;
        part += (long long)nt * (param_count(ob.hidden) + NEXTRA);
    }
    if (rays > ctx->cfg.max_rays_total)
        return fail(ctx, VMAP_ERR_CAPACITY, "%lld rays exceed max_rays_total %d", rays, ctx->cfg.max_rays_total);
    if (tiles > ctx->tile_cap) return fail(ctx, VMAP_ERR_CAPACITY, "too many tiles");
    if (part > ctx->part_cap) {
        // grow the partial buffer (synchronises; never inside a captured region)
        CU(cudaStreamSynchronize(ctx->stream));
        if (ctx->part_d) CU(cudaFree(ctx->part_d));
        ctx->part_d = nullptr;
        ctx->part_cap = 0;
        const long long cap = part + part / 4 + 4096;
        CU(cudaMalloc((void**)&ctx->part_d, sizeof(float) * cap));
        ctx->part_cap = cap;
    }
    // batch objects in index order; tiles grouped by hidden class, object order within
    ctx->bobj.clear();
    std::vector<int> bray;
    int ray_off = 0;
    long long s_off = 0;
    for (int k = 0; k < K; ++k) {
        ObjDev& ob = ctx->objs[k];
        const int R = ob.active ? rays_per_object[k] : 0;
        ob.R = R;
        ob.n_tiles = 0;
        if (R == 0) continue;
        ob.ray_off = ray_off;
        ob.sample_off = s_off;
        ob.src_off = given ? (long long)ray_off : ob.pool_off;
        ctx->bobj.push_back(k);
        bray.push_back(ray_off);
        ray_off += R;
        s_off += (long long)R * ob.S;
    }
    std::vector<TileDev> tl;
    tl.reserve(tiles);
    long long poff = 0;
    for (int c = 0; c < 4; ++c) {
        ctx->cls_begin[c] = (int)tl.size();
        for (int k : ctx->bobj) {
            ObjDev& ob = ctx->objs[k];
            if (ob.hidden != kHidden[c]) continue;
            const int rt = mmax_of(ob.hidden) / ob.S;
            const long long stride = param_count(ob.hidden) + NEXTRA;
            ob.tile_begin = (int)tl.size();
            ob.part_off = poff;
            int idx = 0;
            for (int r0 = 0; r0 < ob.R; r0 += rt, ++idx) {
                TileDev td{};
                td.obj = k;
                td.ray0 = ob.ray_off + r0;
                td.nr = std::min(rt, ob.R - r0);
                td.idx = idx;
                td.part = poff;
                poff += stride;
                tl.push_back(td);
            }
            ob.n_tiles = idx;
        }
        ctx->cls_count[c] = (int)tl.size() - ctx->cls_begin[c];
    }
    ctx->nb = (int)ctx->bobj.size();
    ctx->total_rays = (int)rays;
    ctx->total_samples = samples;
    ctx->n_tiles = (int)tl.size();
    ctx->batch_given = given != nullptr;
    if (given && rays)
        CU(cudaMemcpyAsync(ctx->given_d, given, sizeof(float) * REC * rays, kind, ctx->stream));
    if (vmap_status s = upload_objs(ctx)) return s;
    if (ctx->nb) {
        CU(cudaMemcpyAsync(ctx->bobj_d, ctx->bobj.data(), sizeof(int) * ctx->nb, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(ctx->bray_d, bray.data(), sizeof(int) * ctx->nb, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(ctx->tiles_d, tl.data(), sizeof(TileDev) * tl.size(), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));   // host vectors go out of scope
        const int blocks = (int)((rays + 127) / 128);
        const int pi = prof_begin(ctx, PS_SAMPLE);
        k_sample<<<blocks, 128, 0, ctx->stream>>>(ctx->sp, ctx->objs_d, ctx->bobj_d, ctx->bray_d, ctx->nb,
                                                 (int)rays, given ? ctx->given_d : ctx->pool_d, given ? 1 : 0,
                                                 ctx->steps_d, ctx->pick_d, ctx->t_d);
        prof_end(ctx, pi);
        CHECK_LAUNCH("k_sample");
    }
    ctx->batch_ready = true;
    return VMAP_OK;
}

}  // namespace

extern "C" {

vmap_status vmap_sample_rays(vmap_ctx* ctx, const int* rays_per_object) {
    return sample_impl(ctx, rays_per_object, nullptr, cudaMemcpyDeviceToDevice);
}

vmap_status vmap_sample_rays_given(vmap_ctx* ctx, const float* rays, const int* rays_per_object) {
    if (!rays) return fail(ctx, VMAP_ERR_ARG, "null rays");
    return sample_impl(ctx, rays_per_object, rays, cudaMemcpyDeviceToDevice);
}

vmap_status vmap_train_step_host(vmap_ctx* ctx, const float* rays, const int* rays_per_object,
                                 float* loss) {
    if (!ctx || !rays || !loss) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (vmap_status s = sample_impl(ctx, rays_per_object, rays, cudaMemcpyHostToDevice)) return s;
    if (vmap_status s = vmap_train_step(ctx, ctx->loss_d)) return s;
    CU(cudaMemcpyAsync(loss, ctx->loss_d, sizeof(float) * ctx->objs.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return VMAP_OK;
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
    if (name) *name = kProfNames[slot];
    if (launches) *launches = ctx->prof_n[slot];
    if (total_ms) *total_ms = ctx->prof_ms[slot];
    return VMAP_OK;
}

vmap_status vmap_train_step(vmap_ctx* ctx, float* out_loss) {
    if (!ctx) return VMAP_ERR_ARG;
    if (!ctx->batch_ready) return fail(ctx, VMAP_ERR_STATE, "train_step needs a fresh vmap_sample_rays");
    if (vmap_status s = fill_nan(ctx, out_loss, ctx->objs.size())) return s;
    if (vmap_status s = run_tiles<MODE_TRAIN>(ctx)) return s;
    if (vmap_status s = run_reduce(ctx, RED_ADAM, nullptr, nullptr, out_loss, nullptr)) return s;
    if (ctx->nb) {
        const int pi = prof_begin(ctx, PS_FINISH);
        k_finish<<<1, 256, 0, ctx->stream>>>(ctx->bobj_d, ctx->nb, ctx->steps_d, ctx->status_d);
        prof_end(ctx, pi);
        CHECK_LAUNCH("k_finish");
    }
    ctx->batch_ready = false;
    return VMAP_OK;
}

vmap_status vmap_forward(vmap_ctx* ctx, float* out_loss) {
    if (!ctx || !out_loss) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (!ctx->batch_ready) return fail(ctx, VMAP_ERR_STATE, "forward needs a drawn batch");
    if (vmap_status s = fill_nan(ctx, out_loss, ctx->objs.size())) return s;
    if (vmap_status s = run_tiles<MODE_FORWARD>(ctx)) return s;
    return run_reduce(ctx, RED_LOSS, nullptr, nullptr, out_loss, nullptr);
}

vmap_status vmap_backward(vmap_ctx* ctx, const float* grad_loss, float* grad_params, float* grad_center) {
    if (!ctx || !grad_params) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (!ctx->batch_ready) return fail(ctx, VMAP_ERR_STATE, "backward needs a drawn batch");
    vmap_status s = grad_center ? run_tiles<MODE_GRAD_CENTER>(ctx) : run_tiles<MODE_TRAIN>(ctx);
    if (s) return s;
    return run_reduce(ctx, RED_GRAD, grad_loss, grad_params, nullptr, grad_center);
}

vmap_status vmap_query_occupancy(vmap_ctx* ctx, int obj, const float* pts, long long n, float* occ, float* rgb) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (n < 0) return fail(ctx, VMAP_ERR_ARG, "negative point count");
    if (n == 0) return VMAP_OK;
    if (!pts || !occ) return fail(ctx, VMAP_ERR_ARG, "null argument");
    const int H = ctx->objs[obj].hidden;
    TileArgs ta = base_args(ctx);
    ta.eval_obj = obj;
    ta.eval_n = n;
    ta.qpts = pts;
    ta.qocc = occ;
    ta.qrgb = rgb;
    const int rt = mmax_of(H);
    const long long blocks = (n + rt - 1) / rt;
    cudaError_t e = launch_tile_h<MODE_QUERY>(H, (int)blocks, ctx->stream, ctx->sp, ta);
    if (e != cudaSuccess) return fail(ctx, VMAP_ERR_CUDA, "query kernel failed: %s", cudaGetErrorString(e));
    return VMAP_OK;
}

vmap_status vmap_render_depth(vmap_ctx* ctx, int obj, const float* rays, long long n,
                              const float* box_half, int n_samples, float* depth) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (!rays || !box_half || !depth) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (n < 0) return fail(ctx, VMAP_ERR_ARG, "negative ray count");
    const int H = ctx->objs[obj].hidden;
    if (n_samples < 1 || n_samples > mmax_of(H))
        return fail(ctx, VMAP_ERR_ARG, "n_samples must be in [1, %d] for hidden %d", mmax_of(H), H);
    if (n == 0) return VMAP_OK;
    TileArgs ta = base_args(ctx);
    ta.pool = rays;
    ta.pick = nullptr;
    ta.eval_out = depth;
    for (int a = 0; a < 3; ++a) ta.eval_half[a] = box_half[a];
    ta.eval_obj = obj;
    ta.eval_n = n;
    ta.eval_S = n_samples;
    const int rt = mmax_of(H) / n_samples;
    const long long blocks = (n + rt - 1) / rt;
    cudaError_t e = launch_tile_h<MODE_EVAL>(H, (int)blocks, ctx->stream, ctx->sp, ta);
    if (e != cudaSuccess) return fail(ctx, VMAP_ERR_CUDA, "eval kernel failed: %s", cudaGetErrorString(e));
    return VMAP_OK;
}

vmap_status vmap_get_object_state(vmap_ctx* ctx, int obj, float* params, float* m, float* v, int* step) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    const ObjDev& ob = ctx->objs[obj];
    const size_t bytes = sizeof(float) * param_count(ob.hidden);
    if (params) CU(cudaMemcpyAsync(params, ctx->params_d + ob.param_off, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (m) CU(cudaMemcpyAsync(m, ctx->m_d + ob.param_off, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (v) CU(cudaMemcpyAsync(v, ctx->v_d + ob.param_off, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (step) {
        CU(cudaMemcpyAsync(step, ctx->steps_d + obj, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    return VMAP_OK;
}

vmap_status vmap_set_object_state(vmap_ctx* ctx, int obj, const float* params, const float* m, const float* v, int step) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (step < 0) return fail(ctx, VMAP_ERR_ARG, "negative step");
    const ObjDev& ob = ctx->objs[obj];
    const size_t bytes = sizeof(float) * param_count(ob.hidden);
    if (params) {
        CU(cudaMemcpyAsync(ctx->params_d + ob.param_off, params, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        k_shadow<<<16, 256, 0, ctx->stream>>>(ctx->params_d + ob.param_off, ctx->wt_d + ob.wt_off, ob.hidden);
        CHECK_LAUNCH("k_shadow");
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
        CU(cudaMemcpyAsync(arena, ctx->params_d, sizeof(float) * ctx->param_used, cudaMemcpyDeviceToDevice, ctx->stream));
    return VMAP_OK;
}

vmap_status vmap_set_params(vmap_ctx* ctx, const float* arena) {
    if (!ctx || !arena) return fail(ctx, VMAP_ERR_ARG, "null argument");
    if (!ctx->param_used) return VMAP_OK;
    CU(cudaMemcpyAsync(ctx->params_d, arena, sizeof(float) * ctx->param_used, cudaMemcpyDeviceToDevice, ctx->stream));
    for (const ObjDev& ob : ctx->objs) {
        k_shadow<<<16, 256, 0, ctx->stream>>>(ctx->params_d + ob.param_off, ctx->wt_d + ob.wt_off, ob.hidden);
        CHECK_LAUNCH("k_shadow");
    }
    return VMAP_OK;
}

vmap_status vmap_set_object_active(vmap_ctx* ctx, int obj, int active) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    ctx->objs[obj].active = active ? 1 : 0;
    if (active) CU(cudaMemsetAsync(ctx->status_d + obj, 0, sizeof(int), ctx->stream));
    ctx->batch_ready = false;
    return VMAP_OK;
}

vmap_status vmap_set_object_center(vmap_ctx* ctx, int obj, const float* center) {
    if (vmap_status s = check_obj(ctx, obj)) return s;
    if (!center) return fail(ctx, VMAP_ERR_ARG, "null center");
    for (int a = 0; a < 3; ++a) ctx->objs[obj].c[a] = center[a];
    return upload_objs(ctx);
}

vmap_status vmap_object_info(vmap_ctx* ctx, int obj, int* hidden, int* param_count_out, long long* param_offset, int* spr) {
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
    if (n_rays) *n_rays = ctx->total_rays;
    if (n_samples) *n_samples = ctx->total_samples;
    return VMAP_OK;
}

vmap_status vmap_get_samples(vmap_ctx* ctx, int* pick, float* t) {
    if (!ctx) return VMAP_ERR_ARG;
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
    if (K) {
        CU(cudaMemcpyAsync(st.data(), ctx->status_d, sizeof(int) * K, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    int nf = 0;
    for (int k = 0; k < K; ++k)
        if (st[k]) {
            if (ids && nf < max_ids) ids[nf] = k;
            ++nf;
        }
    if (n_faulted) *n_faulted = nf;
    return nf ? VMAP_ERR_NAN : VMAP_OK;
}

}  // extern "C"
