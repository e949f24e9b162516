/*
 * vmap.h - C ABI of the B300 (sm_103a) vectorised object-MLP training library.
 *
 * The library trains many independent per-object MLP occupancy/colour fields
 * in one pass, as vMAP does (Kong, Liu, Taher, Davison, "vMAP: Vectorised
 * Object Mapping for Neural Field SLAM", CVPR 2023, section 3.2 "Vectorised
 * Training"). One training step, for every object k in the batch:
 *   - picks R_k rays, uniformly with replacement, from the object's own ray
 *     pool (section 3.2 "Object Supervision": each object samples its own
 *     keyframes);
 *   - draws N_c stratified depths in [t_near, t_s + depth_pad] (Eq. 1) and
 *     N_s depths ~ N(t_s, d_sigma^2) (Eq. 2), t_s = the ray's depth, or t_far
 *     when the depth is invalid (<= 0), sorted ascending; a ray off the
 *     object's mask (M = 0) ends at the surface it hits (supplementary
 *     material, depth-guided sampling): range [t_near, t_s], Gaussian
 *     samples clamped above at t_s;
 *   - encodes x~ = (o + t d - c_k) / s_k (supplementary B, object-level
 *     scale) as [x~, sin(B x~), cos(B x~)] (93 features, B is 45 x 3);
 *   - runs the object's MLP 93 -> H -> H -> H -> H -> 4 (ReLU hidden units,
 *     sigmoid occupancy and colour; section 4.1 "Implementation Details");
 *   - renders T_i = o_i prod_{j<i}(1 - o_j), O^ = sum T_i, D^ = sum T_i t_i,
 *     C^ = sum T_i c_i (Eq. 3);
 *   - takes the loss L_k = mean_r M|D^ - D| + lambda_colour mean_{r,c} M|C^ - C|
 *     + lambda_occ mean_r |O^ - M| (Eq. 4-5 read as means over the batch;
 *     M is the ray's mask value, and the depth term is dropped for invalid
 *     depths);
 *   - back-propagates through rendering, MLP and encoding, and
 *   - applies Adam with the object's own step count.
 *
 * Conventions
 *   - Every call is stream-ordered and asynchronous on the stream given to
 *     vmap_init_objects, unless its comment says it synchronises.
 *   - Pointers documented as DEVICE must point to memory of the current
 *     CUDA device; HOST pointers to host memory. Sizes are element counts.
 *   - The library owns weights, Adam moments, ray pools and scratch; the
 *     caller owns every buffer it passes in, and may reuse it as soon as the
 *     stream has passed the call.
 *   - No C++ exception crosses this boundary. Every function returns a
 *     vmap_status; on failure vmap_last_error(ctx) gives a message. A failed
 *     call leaves the context usable unless it returns VMAP_ERR_CUDA.
 *   - Floating-point work is FP32 (VMAP_FP32) or BF16 tensor-core GEMMs with
 *     FP32 accumulation, FP32 master weights, moments, rendering and losses
 *     (VMAP_BF16).
 *
 * Ray record: 12 floats per ray, 48 bytes, row-major [n][12]:
 *   [0..2] origin (world, metres)   [3..5] direction (world, unnormalised:
 *   the ray parameter t is the camera z-depth)   [6] depth (<= 0: invalid)
 *   [7..9] rgb in [0, 1]   [10] mask M (1 inside the object mask, 0 inside
 *   its 2D box only)   [11] reserved, 0.
 *
 * Parameters of one object, canonical packed layout (P(H) floats):
 *   W1 [H][93], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H], W4 [H][H],
 *   b4 [H], W5 [4][H], b5 [4]; W row-major [out][in].
 *   P(16) = 2388, P(32) = 6308, P(64) = 18756, P(128) = 62084.
 */
#ifndef VMAP_H
#define VMAP_H

#ifdef __cplusplus
extern "C" {
#endif

#define VMAP_REC_FLOATS 12
#define VMAP_N_FREQ 45
#define VMAP_D_IN 93
#define VMAP_MAX_SAMPLES 32

typedef struct vmap_ctx vmap_ctx;
typedef struct vmap_hyper vmap_hyper;

typedef enum {
    VMAP_OK = 0,
    VMAP_ERR_ARG = -1,       /* invalid argument (NULL, out of range, bad handle) */
    VMAP_ERR_CAPACITY = -2,  /* a capacity fixed at vmap_init_objects is exceeded */
    VMAP_ERR_CUDA = -3,      /* a CUDA call failed; the message names it */
    VMAP_ERR_NAN = -4,       /* an object's loss or gradient was not finite: it is frozen */
    VMAP_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up */
    VMAP_ERR_STATE = -6      /* call out of order (e.g. train_step without sample_rays) */
} vmap_status;

enum { VMAP_FP32 = 0, VMAP_BF16 = 1 };

typedef struct {
    int max_objects;              /* objects the context can hold */
    int max_rays_total;           /* rays per step over all objects */
    long long max_pool_rays;      /* ray records over all object pools */
    long long max_param_floats;   /* parameters over all objects; 0 = max_objects * P(128) */
    float t_near;                 /* near bound t_n (0.05 m) */
    float depth_pad;              /* stratified samples reach depth + pad (0.1 m) */
    float d_sigma;                /* std of the surface samples (0.03 m, section 3.3) */
    float t_far;                  /* far bound used for invalid depths */
    float lambda_colour;          /* lambda_1 (5) */
    float lambda_occ;             /* lambda_2 (0 on the plain path; 10 in the full objective) */
    float lr, beta1, beta2, eps;  /* Adam (1e-3, 0.9, 0.999, 1e-8) */
    int precision;                /* VMAP_FP32 or VMAP_BF16 */
    unsigned long long seed;      /* Philox4x32-10 key of every random draw */
    const float* B;               /* HOST [45][3] row-major encoding matrix; copied */
} vmap_config;

typedef struct {
    int hidden;                   /* H: 16, 32, 64 or 128 */
    int n_surface;                /* N_s Gaussian samples per ray */
    int n_strat;                  /* N_c stratified samples per ray; 1 <= N_s + N_c <= 32 */
    float center[3];              /* c_k: centre of the object's bound (world) */
    float scale;                  /* s_k > 0: maps the bound into about [-1, 1]^3 */
    const float* rays;            /* DEVICE [n_rays][12] ray records; copied into the pool */
    long long n_rays;             /* >= 1 */
    unsigned int stream;          /* Philox stream id of the object (its draws depend only
                                     on seed, stream, its own step count and the ray index) */
} vmap_object_desc;

/* Fill *cfg with the defaults listed above (capacities 0 must be set). */
void vmap_default_config(vmap_config* cfg);

/* Create a context on the current device. cuda_stream is a cudaStream_t
 * (NULL = legacy default stream). Allocates every arena up front from the
 * capacities in *cfg. Synchronises. */
vmap_status vmap_init_objects(vmap_ctx** out, const vmap_config* cfg, void* cuda_stream);

/* Free the context and all device memory it owns. Synchronises. NULL is a no-op. */
vmap_status vmap_destroy(vmap_ctx* ctx);

/* Message of the last failed call on ctx ("" if none). Valid until the next call. */
const char* vmap_last_error(const vmap_ctx* ctx);

/* Add an object (section 3.2: a new object model appended to the stack).
 * init_params: DEVICE [P(H)] canonical layout, or NULL for the seeded default
 * U(-1/sqrt(fan_in), 1/sqrt(fan_in)) draw. Adam moments start at zero and the
 * object's step count at 0. *out_id (HOST) receives the object index. Objects
 * can be added between any two steps; nothing already recorded must change. */
vmap_status vmap_add_object(vmap_ctx* ctx, const vmap_object_desc* desc,
                            const float* init_params, int* out_id);

/* Draw this step's batch: rays_per_object HOST [n_objects], R_k >= 0 rays of
 * object k (0 = object k sits this step out; inactive objects are skipped).
 * Picks rays and draws sorted sample depths (Eq. 1-2) on the device. */
vmap_status vmap_sample_rays(vmap_ctx* ctx, const int* rays_per_object);

/* Like vmap_sample_rays, but the caller gives this step's rays instead of
 * the library picking them from the pools (e.g. a caller with its own
 * keyframe buffers). rays: DEVICE [sum_k R_k][12], object-major: the R_k
 * rays of every active object with R_k > 0, in object-index order. The
 * records are copied; sample depths are drawn on the device as above. */
vmap_status vmap_sample_rays_given(vmap_ctx* ctx, const float* rays, const int* rays_per_object);

/* One whole step for a caller whose data lives in host memory: copies the
 * given rays (HOST [sum_k R_k][12], layout as vmap_sample_rays_given; pinned
 * memory makes the copy asynchronous), draws depths, trains, and copies the
 * per-object losses to loss (HOST [n_objects], NaN for objects not trained).
 * Synchronises. */
vmap_status vmap_train_step_host(vmap_ctx* ctx, const float* rays, const int* rays_per_object,
                                 float* loss);

/* One training step over the batch drawn by the last vmap_sample_rays:
 * forward, rendering, loss, backward and Adam for every object in it, then
 * each trained object's step count advances. out_loss: DEVICE [n_objects]
 * or NULL; receives L_k before the update (NaN for objects not trained).
 * An object whose loss or gradient is not finite is frozen and flagged (see
 * vmap_sync_status); the others are unaffected. */
vmap_status vmap_train_step(vmap_ctx* ctx, float* out_loss);

/* vmap_sample_rays(ctx, rays_per_object) followed by vmap_train_step(ctx,
 * out_loss), with the same results, issued as one launch sequence (in graph
 * mode one replay): the step's first tile kernel is launched behind the
 * sampler (programmatic dependent launch) and waits for it before reading
 * the batch. Arguments, ownership and errors as for the two calls. */
vmap_status vmap_step(vmap_ctx* ctx, const int* rays_per_object, float* out_loss);

/* Loss of the current batch without changing any state.
 * out_loss: DEVICE [n_objects] (NaN for objects not in the batch). */
vmap_status vmap_forward(vmap_ctx* ctx, float* out_loss);

/* Gradients of sum_k grad_loss[k] * L_k over the current batch, no update.
 * grad_loss: DEVICE [n_objects] or NULL (all ones). grad_params: DEVICE,
 * parameter-arena layout (vmap_param_arena_size floats, object k's block at
 * its vmap_object_info offset); entries of objects outside the batch are
 * left untouched. grad_center: DEVICE [n_objects][3] or NULL: dL/dc_k through
 * the encoding (the encoding backward). */
vmap_status vmap_backward(vmap_ctx* ctx, const float* grad_loss, float* grad_params,
                          float* grad_center);

/* Per-ray gradients of the current batch, the primitive of camera-pose
 * refinement (section 4, tracking with the map fixed): for batch ray i of
 * object k, grad_rays[i] = (dL_k/do_i, dL_k/dd_i) through x = o + t d with
 * the drawn sample depths held fixed (the encoding backward, summed over the
 * ray's samples). A camera at (p, R) with d = R d_c gets dL/dp = sum dL/do
 * and, for a rotation exp([w]x) R, dL/dw = sum d x dL/dd. grad_rays: DEVICE
 * [n_rays][6], batch order (object-major, as vmap_get_samples). No state
 * changes. FP32 contexts only. */
vmap_status vmap_ray_gradients(vmap_ctx* ctx, float* grad_rays);

/* One iteration of camera-pose refinement against object `obj` with the
 * map held fixed, entirely on the device (the paper refines camera poses
 * through the map, section 4 "Tracking"; the gradients are those of
 * vmap_ray_gradients): the camera at position p with rotation R
 * (world from camera) casts rays o = p, d = R d_c; their samples are drawn
 * as vmap_sample_rays_given draws them; one tile pass gives the object's
 * loss on them and the per-ray (dL/do, dL/dd); one kernel forms
 * dL/dp = sum_rays dL/do and dL/dw = sum_rays d x dL/dd (for the rotation
 * update R <- exp([w]x) R; fixed summation order) and takes one Adam step
 * (the context's beta1, beta2; epsilon 1e-12) with learning rates lr_t for
 * p and lr_r for w. Nothing synchronises.
 *   dc:        DEVICE [n][3] camera-frame ray directions ((u + 1/2 - cx)/f, (v + 1/2 - cy)/f, 1).
 *   meas:      DEVICE [n][5] measured depth, rgb and mask per ray.
 *   pose:      DEVICE [12] p[3], R[9] row-major; updated in place.
 *   adam:      DEVICE [13] first moments [6], second moments [6], step count; zero it
 *              before the first iteration.
 *   rays_work: DEVICE [n][12], grad_work: DEVICE [n][6]: scratch the caller owns.
 *   loss:      DEVICE [n_objects]: this iteration's loss of `obj` (before the update);
 *              NaN for the other objects.
 * FP32 contexts only (VMAP_ERR_ARG otherwise); n <= max_rays_total
 * (VMAP_ERR_CAPACITY). The context's current batch becomes these rays. */
vmap_status vmap_pose_step(vmap_ctx* ctx, int obj, const float* dc, const float* meas, int n,
                           float* pose, float* adam, float lr_t, float lr_r,
                           float* rays_work, float* grad_work, float* loss);

/* Occupancy (and colour) of n arbitrary world points of one object (section
 * 3.4: an object is queried inside its bound). pts DEVICE [n][3];
 * occ DEVICE [n]; rgb DEVICE [n][3] or NULL. n = 0 is a no-op. */
vmap_status vmap_query_occupancy(vmap_ctx* ctx, int obj, const float* pts, long long n,
                                 float* occ, float* rgb);

/* Rendered depth of n rays of one object with n_samples stratified
 * midpoints between the ray's entry and exit of the box c_k +- box_half
 * (world, metres). rays DEVICE [n][12] (only origin and direction are read);
 * depth DEVICE [n]; a ray that misses the box renders 0. */
vmap_status vmap_render_depth(vmap_ctx* ctx, int obj, const float* rays, long long n,
                              const float* box_half, int n_samples, float* depth);

/* Compositional scene render (section 3.4): each listed object renders the
 * rays inside its box c_k +- box_half[j] with n_samples midpoints (as
 * vmap_render_depth), giving (O^, D^, C^) per ray; the objects a ray meets
 * are ranked by their expected hit depth D^/O^ (ties: earlier list entry
 * first; O^ = 0 skipped) and composed front to back as Eq. 3 composes
 * samples: D = sum A_k D^_k, C = sum A_k C^_k, O = sum A_k O^_k with
 * A_k = prod over earlier-ranked objects of (1 - O^_j).
 *   rays: DEVICE [n][12] (origin and direction read); objs: HOST [m] object
 *   indices, or NULL for objects 0..m-1; box_half: HOST [m][3];
 *   depth: DEVICE [n]; rgb: DEVICE [n][3] or NULL; occ: DEVICE [n] or NULL.
 * Keeps m * n * 5 floats of scratch in the context (grown on demand, which
 * synchronises). n = 0 is a no-op. */
vmap_status vmap_render_scene(vmap_ctx* ctx, const float* rays, long long n, const int* objs, int m,
                              const float* box_half, int n_samples, float* depth, float* rgb, float* occ);

/* Mesh of one object (section 4 evaluates object meshes obtained by querying
 * each object inside its 3D bound): occupancy on a (res+1)^3 lattice over
 * c_k +- box_half, then marching tetrahedra (six Kuhn tetrahedra per cube,
 * a lattice vertex inside when its occupancy > level; the surface is closed
 * inside the box and each triangle faces from inside to outside).
 *   box_half: HOST [3]; 1 <= res <= 512.
 *   tris: DEVICE [max_tris][3][3] world-space vertices, in a deterministic
 *   order (cube index with x fastest, then tetrahedron, then triangle), or
 *   NULL with max_tris = 0 to count only. *n_tris (HOST) receives the total,
 *   which may exceed max_tris (then only max_tris are written).
 * Allocates and frees its scratch; synchronises. */
vmap_status vmap_extract_mesh(vmap_ctx* ctx, int obj, const float* box_half, int res, float level, float* tris,
                              long long max_tris, long long* n_tris);

/* Object state in canonical layout. Any DEVICE pointer may be NULL.
 * step: HOST, may be NULL (reading it synchronises). */
vmap_status vmap_get_object_state(vmap_ctx* ctx, int obj, float* params, float* m, float* v,
                                  int* step);
vmap_status vmap_set_object_state(vmap_ctx* ctx, int obj, const float* params, const float* m,
                                  const float* v, int step);

/* Whole parameter arena (all objects, vmap_param_arena_size floats), DEVICE. */
vmap_status vmap_get_params(vmap_ctx* ctx, float* arena);
vmap_status vmap_set_params(vmap_ctx* ctx, const float* arena);
vmap_status vmap_param_arena_size(vmap_ctx* ctx, long long* n_floats);

/* Stop (0) or resume (1) training of one object (section 3.2: training of any
 * object can stop and resume with no interference). Takes effect at the
 * next vmap_sample_rays. Resuming clears a NaN freeze. */
vmap_status vmap_set_object_active(vmap_ctx* ctx, int obj, int active);

/* Move an object's centre c_k (HOST [3]). Takes effect at the next call. */
vmap_status vmap_set_object_center(vmap_ctx* ctx, int obj, const float* center);

/* HOST outputs, any may be NULL. */
vmap_status vmap_object_info(vmap_ctx* ctx, int obj, int* hidden, int* param_count,
                             long long* param_offset, int* samples_per_ray);
vmap_status vmap_num_objects(vmap_ctx* ctx, int* n);

/* The current batch, for inspection: total rays and samples (HOST), and
 * DEVICE copies of the picked pool indices [rays] and sample depths
 * [samples] (object-major, ray-major, sorted per ray). Either array may be NULL. */
vmap_status vmap_batch_info(vmap_ctx* ctx, int* n_rays, long long* n_samples);
vmap_status vmap_get_samples(vmap_ctx* ctx, int* pick, float* t);

/* Synchronise and report frozen objects: *n_faulted (HOST) and, if ids is
 * not NULL, up to max_ids of their indices. Returns VMAP_ERR_NAN if any.
 * Returns VMAP_ERR_TIMEOUT (and leaves *n_faulted unset) if a tensor-core
 * kernel gave up one of its bounded waits since the last report; the flag is
 * cleared by this report. While the flag is set, training steps update no
 * object (every loss is NaN, no step count advances) and vmap_forward /
 * vmap_backward write NaN losses and no gradient: a step whose wait gave up
 * has incomplete gradient sums, so it is void rather than applied. */
vmap_status vmap_sync_status(vmap_ctx* ctx, int* n_faulted, int* ids, int max_ids);

/* Failure detection of the BF16 tensor-core kernels: every wait for an MMA
 * commit or a bulk copy polls its mbarrier at most `polls` times (default
 * 2^26, far longer than any MMA takes) before it gives up; the CTA then
 * stops its work, waits (with the fixed default bound) for the MMAs and
 * copies it has already issued, frees its tensor memory and exits, and the
 * context's error flag is set (see vmap_sync_status). polls = 0 gives up at
 * once: a way to exercise this path without making any MMA fail. Captured
 * graphs are dropped when the limit changes. polls < 0: VMAP_ERR_ARG. The
 * paper has no counterpart (it runs no custom kernels). */
vmap_status vmap_set_wait_limit(vmap_ctx* ctx, long long polls);

/* Tracing: with profiling enabled, every kernel launch is bracketed by CUDA
 * events on the context stream (in graph mode, every graph replay, as the
 * slots "graph:sample" and "graph:train"). vmap_profile_read synchronises and
 * returns, for slot `slot` (0 .. until VMAP_ERR_ARG), its name (static
 * string), launch count and summed device milliseconds since the last reset. */
vmap_status vmap_profile_enable(vmap_ctx* ctx, int on);
vmap_status vmap_profile_reset(vmap_ctx* ctx);
vmap_status vmap_profile_read(vmap_ctx* ctx, int slot, const char** name, long long* launches,
                              double* total_ms);

/* Replay the step as CUDA graphs (on = 1) or launch kernel by kernel (0, the
 * default). The batch layout lives in device memory, so a captured step stays
 * valid while objects are admitted, stopped or resized; adding the first
 * object of a new hidden width recaptures once. Graphs are captured lazily at
 * the next vmap_sample_rays / vmap_train_step. */
vmap_status vmap_set_graph(vmap_ctx* ctx, int on);

/* Launch shape per hidden-width class (index 0..3 = H 16, 32, 64, 128):
 * rays per tile (1..32, further capped so a tile holds at most the class's
 * sample budget) and the persistent grid multiplier (1..2; the grid is
 * SMs x CTAs per SM x multiplier). HOST arrays [4], either may be NULL. */
vmap_status vmap_get_launch(vmap_ctx* ctx, int* rays_per_tile, int* grid_mult);
vmap_status vmap_set_launch(vmap_ctx* ctx, const int* rays_per_tile, const int* grid_mult);

/* Autotuner: choose the launch shape of every width class present by timing
 * whole training steps (vmap_step: sampling, tile kernels, reduce and Adam,
 * replayed as a graph when graph mode is on, so the overlapped launches are
 * what is timed) on the batch rays_per_object (HOST [n_objects]). Candidates
 * per class: rays per tile (samples per tile = rays x the class's samples per
 * ray, from the class's tile budget down to one ray) x grid multiplier
 * (1..2), swept one class at a time with the others held (coordinate
 * descent, a second pass if the first changed a shape); each candidate is
 * timed over `reps` steps after two untimed ones. Every object's weights,
 * moments, step count and status are saved on the device first and restored
 * at the end, so no object state changes; the next step draws a fresh batch.
 * best_ms: HOST [4] or NULL, the best step time found (the same value for
 * every present class, 0 for absent classes). Allocates a temporary copy of
 * the training state. Synchronises. */
vmap_status vmap_autotune(vmap_ctx* ctx, const int* rays_per_object, int reps, float* best_ms);

/* ---------------------------------------------------------------------------
 * Warm-start set-encoder hypernetwork (not in the paper: this library's
 * learned extension). From n_points samples (x~ = (x - c_k)/s_k, occupancy,
 * rgb: 7 floats each) of a newly seen object's first keyframe it predicts
 * initial weights for the object's MLP (canonical layout, P(hidden) floats):
 *   per point  h1 = ReLU(W1 x + b1), h2 = ReLU(W2 h1 + b2), h3 = ReLU(W3 h2 + b3)
 *   per set    z = channel-wise max of h3 over the points (ties: lowest index)
 *   head       u = Wa z + ba (rank `rank`), theta = Wb u + bb
 * Trained on (samples, converged weights) pairs with the mean squared error
 * L = sum (theta - target)^2 / (batch P). Parameters (flat, in this order):
 * W1 [width][7], b1, W2 [width][width], b2, W3, b3, Wa [rank][width], ba,
 * Wb [P][rank], bb [P]. All calls are asynchronous on the stream given to
 * vmap_hyper_create. Inputs X: DEVICE [batch][n_points][7]; targets T and
 * outputs: DEVICE [batch][P]; grad: DEVICE [n_params]; loss: DEVICE [1]
 * or NULL. batch > max_batch gives VMAP_ERR_CAPACITY. */
vmap_status vmap_hyper_create(vmap_hyper** out, int n_points, int width, int rank, int hidden,
                              int max_batch, unsigned long long seed, void* cuda_stream);
vmap_status vmap_hyper_destroy(vmap_hyper* h);
const char* vmap_hyper_last_error(const vmap_hyper* h);
/* GEMM precision (default VMAP_FP32). VMAP_BF16 (width 128 only): the GEMMs
 * of the three 128-wide shared layers (forward, input and weight gradients)
 * run on the tensor cores with BF16 operands and FP32 accumulation; the
 * 7-input first layer, the rank-r head, biases, losses and Adam stay FP32.
 * Synchronises when switching to VMAP_BF16 the first time. */
vmap_status vmap_hyper_set_precision(vmap_hyper* h, int precision);
/* HOST outputs: number of hypernetwork parameters, and P (outputs per object). */
vmap_status vmap_hyper_param_count(vmap_hyper* h, long long* n_params, int* out_params);
vmap_status vmap_hyper_get_params(vmap_hyper* h, float* flat);
/* Setting the parameters also resets the Adam moments and step count. */
vmap_status vmap_hyper_set_params(vmap_hyper* h, const float* flat);
vmap_status vmap_hyper_predict(vmap_hyper* h, int batch, const float* X, float* out);
/* Loss and gradient without an update. */
vmap_status vmap_hyper_grad(vmap_hyper* h, int batch, const float* X, const float* T, float* grad,
                            float* loss);
/* One Adam step (betas 0.9, 0.999, eps 1e-8) on one batch. */
vmap_status vmap_hyper_train_step(vmap_hyper* h, int batch, const float* X, const float* T, float lr,
                                  float* loss);
/* Warm start: predict object obj's weights from X (DEVICE [n_points][7]) and
 * install them with zero Adam moments and step count 0. The hypernetwork's
 * output count must equal the object's P(H). Synchronises the device. */
vmap_status vmap_warmstart(vmap_ctx* ctx, int obj, vmap_hyper* h, const float* X);

/* Gradient and loss of ONE object on caller-chosen rays, for callers that
 * cannot allocate device memory: code running inside a memory pool or
 * allocator it must not re-enter, real-time loops where a cudaMalloc could
 * stall or fail, or hosts that pre-plan every device allocation. The paper
 * has no counterpart; it is a convenience of this library.
 *
 * No context is needed and nothing is allocated: the scratch (batch tables,
 * sample depths, transposed weights and gradient slots) lives in one
 * file-scope device array of about 4.8 MB that every GPU loading the
 * library keeps until the process exits. The computation equals
 * vmap_sample_rays_given + vmap_forward + vmap_backward on a context holding
 * the same object whose step count is `step` (same Philox draws), up to
 * FP32 summation order.
 *   cfg:    HOST; hyper-parameters, B and seed (capacities are ignored).
 *   desc:   HOST; hidden, n_surface, n_strat, center, scale and stream as in
 *           vmap_add_object; rays = DEVICE [n_rays][12] rays of this batch,
 *           each used once; 1 <= n_rays <= 1024.
 *   params: DEVICE [P(H)] canonical layout.
 *   step:   the object's step count (the counter of its random draws).
 *   grad:   DEVICE [P(H)] receives dL/dparams; loss: DEVICE [1] receives L.
 *   cuda_stream: cudaStream_t the work is queued on (asynchronous).
 * Returns VMAP_ERR_CAPACITY if n_rays exceeds 1024, VMAP_ERR_ARG for other
 * invalid arguments (nothing is queued then), VMAP_ERR_CUDA if a launch fails.
 * The first call on a device (with that device current) looks up the
 * array's device address and sets kernel attributes; make that first call
 * before any stream capture. Each call hands its per-call values (the
 * object record, ray count and step count) to the device as kernel
 * arguments, so no host-to-device copy is queued. All calls share the one
 * array, which keeps the last call's contents (every call rewrites what it
 * reads): calls whose work overlaps on the GPU (other streams, other
 * threads) race; serialise them on one stream. */
vmap_status vmap_object_grad_static(const vmap_config* cfg, const vmap_object_desc* desc,
                                    const float* params, int step, float* grad, float* loss,
                                    void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* VMAP_H */
