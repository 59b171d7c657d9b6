/*
 * mvp.h -- C ABI of the GB300 ray-march library for Mixture of Volumetric
 * Primitives (Lombardi et al., "Mixture of Volumetric Primitives for Efficient
 * Neural Rendering", ACM TOG 40(4), 2021).
 *
 * The library implements the paper's rendering hot path (Sec. 3.2): a per-frame
 * bounding volume hierarchy over moving, oriented primitives (Sec. 3.2.1, built
 * with the data-parallel LBVH construction the paper cites), per-ray lists of the
 * primitives each ray intersects (Sec. 3.2.1), the fixed-step ray march with
 * trilinear payload sampling and clamped additive opacity accumulation
 * (Sec. 3.2.2), its adjoint, payload precision conversion, and a serving loop.
 *
 * Conventions for every call:
 *   - Pointers documented as "device" are CUDA device pointers owned by the
 *     caller; the library never frees them. "host" pointers are ordinary memory.
 *   - Opaque handles (mvp_ctx, mvp_bvh, mvp_server) are created and freed by the
 *     library's *_create / *_destroy calls.
 *   - Calls that take an mvp_stream are asynchronous on that stream unless their
 *     comment says they synchronise. A NULL stream is the legacy default stream.
 *   - Every call returns an mvp_status; nothing throws or aborts across the ABI.
 *     Host-side argument checks return MVP_ERR_INVALID_ARG before any launch.
 *     Errors found by a kernel (a traversal stack overflow) are recorded in the
 *     context's device status word and reported by the next mvp_ctx_sync on that
 *     context.
 *     mvp_last_error() returns a thread-local message for the last failure.
 *   - All floating-point arithmetic on the device is FP32. Payloads may be stored
 *     as FP32, BF16 or FP16; interpolation and compositing are FP32.
 *
 * Geometry (Sec. 3.1.2). Primitive k has centre t_k, rotation R_k = R(q_k/|q_k|)
 * from the quaternion q_k = (w, x, y, z), and half extents s_k > 0: a local point
 * y in [-1,1]^3 lies at t_k + R_k diag(s_k) y in the world. Its payload is an
 * M x M x M grid of RGBA voxels (colour and opacity density), indexed
 * [k][z][y][x][c] with x fastest; voxel centres sit on the box corners and faces
 * (the voxel coordinate of a local coordinate y is (y + 1)/2 * (M - 1)).
 *
 * Quadrature (Sec. 3.2.2). A ray o + t d (d unit) is sampled at
 * t_i = t_near + i*dt for i in [0, n_steps), n_steps = mvp_num_steps(...). Every
 * primitive whose box contains t_i contributes alpha_k and rgb_k (trilinear);
 * a = dt * sum alpha_k, c = dt * sum alpha_k rgb_k, w = min(a, 1 - T),
 * I += c * w / a, T += w. The march stops once T >= 1 - eps_early. The output is
 * (I + (1 - A) * bg, A) with A the final T (Sec. 3.1.4 composite, with I already
 * weighted by the accumulated opacity).
 * Box membership of a sample is decided in FP32 with a fixed operation order
 * (the slab interval of the ray against the box, compared with the FP32 sample
 * time), which makes hit lists reproducible bit for bit.
 */
#ifndef MVP_H
#define MVP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MVP_API __attribute__((visibility("default")))
#else
#define MVP_API
#endif

#define MVP_ABI_VERSION 1
#define MVP_MAX_M 128          /* largest payload edge */
#define MVP_MAX_STEPS 65535    /* largest n_steps per ray */
#define MVP_MAX_PRIMS (1 << 24)

typedef struct CUstream_st *mvp_stream; /* same type as cudaStream_t */

typedef enum mvp_status {
  MVP_OK = 0,
  MVP_NOT_READY = 1,         /* a polled request has not finished yet */
  MVP_ERR_INVALID_ARG = -1,  /* rejected on the host before any launch */
  MVP_ERR_CUDA = -2,         /* a CUDA runtime call failed */
  MVP_ERR_OOM = -3,          /* a library allocation failed */
  MVP_ERR_CAPACITY = -4,     /* a fixed capacity was exceeded (see the call) */
  MVP_ERR_TIMEOUT = -5,      /* a bounded wait ran out */
  MVP_ERR_DEVICE = -6        /* a kernel reported an inconsistent state */
} mvp_status;

typedef enum mvp_dtype { MVP_F32 = 0, MVP_BF16 = 1, MVP_F16 = 2 } mvp_dtype;

/* Primitive set (Sec. 3.1.2). All pointers are device pointers. */
typedef struct mvp_prims {
  int32_t n;            /* number of primitives, 0 <= n <= MVP_MAX_PRIMS */
  int32_t M;            /* payload edge, 2 <= M <= MVP_MAX_M */
  int32_t dtype;        /* mvp_dtype of payload */
  int32_t reserved;     /* must be 0 */
  const float *t;       /* [n][3] centres */
  const float *q;       /* [n][4] quaternions (w, x, y, z), nonzero */
  const float *s;       /* [n][3] half extents, > 0 */
  const void *payload;  /* [n][M][M][M][4] RGBA, x fastest; 16-byte aligned */
} mvp_prims;

/* Rays and quadrature parameters (Sec. 3.2.2). o, d are device pointers. */
typedef struct mvp_rays {
  int64_t n;            /* number of rays, >= 0 */
  const float *o;       /* [n][3] origins */
  const float *d;       /* [n][3] unit directions */
  float t_near, t_far;  /* integration range, t_near < t_far */
  float dt;             /* step, > 0 */
  float eps_early;      /* stop once T >= 1 - eps_early, 0 <= eps_early < 1 */
  float bg[3];          /* constant background colour */
  int32_t width;        /* if width * height == n: rays form a row-major image  */
  int32_t height;       /* and are marched in 2-D pixel tiles; else 1-D groups  */
  int32_t flags;        /* 0, or MVP_BLEND_SEQUENTIAL | MVP_COMPOSITE_LITERAL */
} mvp_rays;

/* mvp_rays.flags: blend the primitives that share a ray's saturating sample one by
 * one in BVH order (the order of their leaves: ascending (morton << 32 | k)), as the
 * paper describes for overlapping primitives (Sec. 3.2.2), instead of summing them and
 * clamping once. Every other sample is unaffected (the two rules agree wherever T
 * stays below 1). mvp_raymarch_bwd differentiates the rule the forward applied (pass
 * the same flags to both). */
#define MVP_BLEND_SEQUENTIAL 1
/* mvp_rays.flags: the background composite read literally as I~ = A I + (1 - A) B
 * (Sec. 3.1.4) instead of I~ = I + (1 - A) B, which treats the marched I as already
 * weighted by the accumulated opacity (its integrand carries dT). Forward only:
 * mvp_raymarch_bwd rejects it. */
#define MVP_COMPOSITE_LITERAL 2

typedef struct mvp_ctx mvp_ctx;
typedef struct mvp_bvh mvp_bvh;

/* ---------------------------------------------------------------- basics */
MVP_API const char *mvp_version(void);
MVP_API const char *mvp_status_string(int status);
/* Message of the last failed call on this thread ("" if none). */
MVP_API const char *mvp_last_error(void);
/* n_steps = ceil((t_far - t_near)/dt - 1e-4) computed in double from the FP32
 * values (a sample within 1e-4*dt of t_far is not taken); 0 if t_far <= t_near. */
MVP_API int64_t mvp_num_steps(float t_near, float t_far, float dt);

/* Context: binds a device and owns the device status word. */
MVP_API mvp_status mvp_ctx_create(int device, mvp_ctx **out);
MVP_API void mvp_ctx_destroy(mvp_ctx *ctx);
/* Synchronises `stream`, then reads and clears the device status word:
 * MVP_ERR_CAPACITY if a kernel hit a capacity limit since the last sync
 * (MVP_STATUS_CAPACITY), MVP_ERR_INVALID_ARG if a BVH build met a primitive whose
 * pose defines no box (MVP_STATUS_POSE: t, q or s not finite, q = 0 or s <= 0;
 * renders that used it are finite and read nothing out of bounds, but that
 * primitive's contribution is unspecified), else MVP_OK (or MVP_ERR_CUDA if the
 * stream reported an error). */
#define MVP_STATUS_CAPACITY 1
#define MVP_STATUS_POSE 4
/* Checked builds only (compiled with -DMVP_CHECK_BOUNDS, the library's stand-in for a
 * memory checker): an index fell outside its array; the access was skipped.
 * mvp_ctx_sync reports it as MVP_ERR_DEVICE. */
#define MVP_STATUS_BOUNDS 8
/* 1 if this library is a checked build, else 0. */
MVP_API int32_t mvp_bounds_checked(void);
MVP_API mvp_status mvp_ctx_sync(mvp_ctx *ctx, mvp_stream stream);

/* ------------------------------------------------------ BVH (Sec. 3.2.1) */
/* A BVH handle owns its device buffers and grows them as needed; reuse one
 * handle across frames to avoid reallocation. */
MVP_API mvp_status mvp_bvh_create(mvp_ctx *ctx, mvp_bvh **out);
MVP_API void mvp_bvh_destroy(mvp_bvh *bvh);
/* Rebuild the hierarchy over `prims` (the per-frame rebuild of Sec. 3.2.1):
 * per-primitive rotation, oriented-box world bounds and 30-bit Morton code of the
 * centre within the centres' bounds; the keys (morton << 32 | k) sorted; the binary
 * radix tree of the sorted keys; each node's box = the union of its leaves' boxes.
 * Four launches up to 8192 primitives, seventeen above. Reallocation (first use or
 * larger n) synchronises the stream; a rebuild at the same or smaller n allocates
 * nothing and only enqueues kernels. */
MVP_API mvp_status mvp_build_bvh(mvp_ctx *ctx, const mvp_prims *prims, mvp_bvh *bvh, mvp_stream stream);
/* Number of primitives of the last build. */
MVP_API int32_t mvp_bvh_size(const mvp_bvh *bvh);
/* Copy the last build to caller device buffers (any may be NULL), asynchronously:
 * keys [n] uint64 sorted (morton << 32 | k); children [n-1][2] int32 (internal
 * nodes 0..n-2, leaf j = node n-1+j holding primitive keys[j] & 0xffffffff);
 * bounds [2n-1][6] float32 node boxes (lo xyz, hi xyz), slightly inflated;
 * scene [6] float32 centre bounds used for the Morton codes. */
MVP_API mvp_status mvp_bvh_export(mvp_ctx *ctx, const mvp_bvh *bvh, uint64_t *keys, int32_t *children,
                          float *bounds, float *scene, mvp_stream stream);

/* Per-ray hit lists (Sec. 3.2.1: "compute and store the primitives each ray
 * intersects"). Fills CSR arrays (device): offs [n_rays + 1] int64, and for each
 * hit the primitive id and the FP32 slab interval [tin, tout] clipped to
 * [t_near, t_far], in traversal order within a ray. Writes at most `cap` hits;
 * *n_hits (host) receives the total. Returns MVP_ERR_CAPACITY (with offs valid)
 * if the total exceeds cap. Synchronises the stream. */
MVP_API mvp_status mvp_hitlists(mvp_ctx *ctx, const mvp_prims *prims, const mvp_bvh *bvh, const mvp_rays *rays,
                        int64_t *offs, int32_t *ids, float *tin, float *tout, int64_t cap,
                        int64_t *n_hits, mvp_stream stream);

/* ------------------------------------------ forward march (Sec. 3.2.2) */
/* Bytes of per-ray state the forward saves for the adjoint (32 per ray). */
MVP_API size_t mvp_saved_bytes(int64_t n_rays);
/* The tile schedule of the frame kernel and of the adjoint (on by default): each
 * mvp_raymarch_fwd (and, separately, each mvp_raymarch_bwd) records how long each
 * warp tile took and the next call with the same number of tiles starts the
 * heaviest tiles first, so that no expensive tile (rays grazing many primitives)
 * starts late and outlasts the frame. It changes no image (the adjoint's gradients
 * only by the order of their float reductions). The first call at a new, larger
 * tile count allocates its buffers (cudaMalloc). Calls on other streams that overlap
 * the last scheduled one use the plain order. enable = 0 always uses the plain
 * order; a frame (mvp_build_bvh at an unchanged or smaller primitive count, then
 * mvp_raymarch_fwd) then only enqueues kernels and can be captured into a CUDA graph. */
MVP_API mvp_status mvp_ctx_set_tile_schedule(mvp_ctx *ctx, int32_t enable);
/* How mvp_raymarch_bwd walks the primitives (no counterpart in the paper: a memory
 * schedule of the Sec. 3.2.2 replay). When the payload and its gradient together
 * exceed twice `bytes`, the adjoint cuts the primitives into groups of consecutive BVH
 * positions of about `bytes` each (at most 64 groups) and replays every warp tile once
 * per group its rays meet, group after group, so that a group's payload and
 * g_payload stay in L2 while all rays that touch them are replayed. bytes = 0 picks
 * the size from the device's L2 (a third of it; the default); bytes < 0 never
 * groups. The grouped replay takes stream-ordered scratch (cudaMallocAsync, about
 * 8 + 4 x groups bytes per warp tile); where that allocation fails the call replays in
 * one pass. Results equal the ungrouped replay up to the order of the float
 * reductions. */
MVP_API mvp_status mvp_ctx_set_bwd_group_bytes(mvp_ctx *ctx, int64_t bytes);
/* Render: out_rgba [n][4] float32 device = (I + (1 - A) bg, A). `saved`
 * (device, mvp_saved_bytes(n) bytes, nullable) receives the per-ray state the
 * adjoint needs. `bvh` must have been built from the same prims. Rays are marched
 * by warps over 8x4 pixel tiles; each tile gathers at most 48 primitives at once
 * and splits its sample range when more overlap it; a single sample met by more
 * than 48 primitives across one tile is evaluated against all of them by an extra
 * traversal. A traversal stack overflow (256 entries per tile) records
 * MVP_ERR_CAPACITY. */
MVP_API mvp_status mvp_raymarch_fwd(mvp_ctx *ctx, const mvp_prims *prims, const mvp_bvh *bvh,
                            const mvp_rays *rays, float *out_rgba, void *saved, mvp_stream stream);
/* Same march, writing only the number of (sample, primitive) evaluations of each
 * ray to n_eval [n] int32 device (the work count used for roofline figures). */
MVP_API mvp_status mvp_raymarch_count(mvp_ctx *ctx, const mvp_prims *prims, const mvp_bvh *bvh,
                              const mvp_rays *rays, int32_t *n_eval, mvp_stream stream);

/* --------------------------------------------------------- adjoint */
/* Gradients of a loss L given grad_rgba = dL/d(out_rgba) [n][4] (device),
 * replaying the march from `saved` (written by mvp_raymarch_fwd with the same
 * inputs). Accumulates (+=) into device FP32 buffers: g_payload [n][M][M][M][4],
 * g_t [n][3], g_q [n][4], g_s [n][3] (any may be NULL to skip it; g_t, g_q and g_s
 * are produced together). Pose gradients pass through an internal per-primitive
 * FP32 buffer owned by the bvh handle. Gradient accumulation uses atomics, so the
 * summation order (and the last bits) may vary between runs. */
MVP_API mvp_status mvp_raymarch_bwd(mvp_ctx *ctx, const mvp_prims *prims, mvp_bvh *bvh, const mvp_rays *rays,
                            const void *saved, const float *grad_rgba, float *g_payload, float *g_t,
                            float *g_q, float *g_s, mvp_stream stream);

/* ------------------------------------------------ precision and cameras */
/* Convert n_values FP32 values (device) to dtype (device dst, round to nearest
 * even); MVP_F32 copies. */
MVP_API mvp_status mvp_pack_payload(mvp_ctx *ctx, const float *src, void *dst, int64_t n_values, int32_t dtype,
                            mvp_stream stream);
/* Pinhole rays of a W x H image, row-major: c2w (host, row-major 3x4 =
 * [right down forward | eye]), focal in pixels, pixel centres at (col + 0.5,
 * row + 0.5), principal point at the image centre. o, d: [W*H][3] device. */
MVP_API mvp_status mvp_camera_rays(mvp_ctx *ctx, const float *c2w, float focal, int32_t width, int32_t height,
                           float *o, float *d, mvp_stream stream);

/* ------------------------------------------------------------ serving */
/* Continuous batching of render requests (avatar = resident primitive set,
 * camera, resolution). Each admitted request is launched at once, on the least
 * loaded of 8 streams, as a grid with one warp per 8x4-pixel tile that generates
 * its pinhole rays and marches them with the code of mvp_raymarch_fwd, so a
 * request's image equals mvp_camera_rays + mvp_raymarch_fwd on the same avatar,
 * alone or in any mix. Requests in flight overlap on the device (a request's
 * blocks start as SMs free up from the ones before it); each completes as soon as
 * its own tiles are done, seen by the host through mapped memory. No device code
 * waits for anything. Admission: a request needs a free slot, and its image
 * (width*height*16 bytes) must fit the HBM budget (resident avatars + images in
 * flight) and the server's image arena; otherwise it queues (FIFO) and is admitted
 * by a later submit or poll. All calls are thread-safe. */
typedef struct mvp_server mvp_server;

typedef struct mvp_request {
  int32_t avatar;        /* id from mvp_serve_register_avatar */
  int32_t width, height; /* image size in pixels (>= 1), per view */
  float focal;           /* pixels */
  float c2w[12];         /* row-major 3x4 [right down forward | eye], as mvp_camera_rays */
  float t_near, t_far, dt, eps_early;
  float bg[3];
  int32_t views;         /* 1 (0 counts as 1), or 2: a stereo pair (the paper's binocular
                          * viewer, Sec. 4) rendered from one BVH in one launch; the image
                          * is then [2][height][width][4], view 0 from c2w, view 1 from
                          * c2w_right */
  float c2w_right[12];   /* second view's camera (views = 2) */
  const void *payload;   /* NULL: the avatar's payload. Else this request's own payload
                          * (device, caller-owned; the avatar's n, M and dtype and its
                          * alignment), e.g. the view-dependent payload assembled for
                          * this camera by mvp_assemble_payload; both views of a stereo
                          * request use it. Its writes must be complete before the call
                          * (synchronise the producing stream), and it must stay valid
                          * until the request completes. It does not count against the
                          * server's HBM budget. */
} mvp_request;

typedef struct mvp_serve_info {
  int64_t pending, in_flight, max_in_flight, completed;
  int64_t resident_bytes, in_flight_bytes;
  int32_t grid_blocks;    /* blocks of the serving kernel resident on the GPU at once */
  int32_t avatars;
  int32_t device_status;  /* status bits set by the serving kernel (0: none) */
  int32_t reserved;
  int64_t batches;        /* request launches so far */
  int64_t cancelled;      /* requests cancelled so far */
} mvp_serve_info;

/* hbm_budget: bytes for resident avatars (payload + BVH) plus images in flight;
 * max_slots: requests in flight at once (1..65536); arena_bytes: device memory
 * allocated up front for images in flight (0: the budget; capped by it). */
MVP_API mvp_status mvp_serve_create(mvp_ctx *ctx, size_t hbm_budget, int32_t max_slots, size_t arena_bytes,
                                    mvp_server **out);
/* Waits for the server's device work, then frees it (avatars' payloads stay the
 * caller's). */
MVP_API void mvp_serve_destroy(mvp_server *server);
/* Keeps `prims` (device pointers, caller-owned, must stay valid) resident and builds
 * its BVH once (avatars do not move between requests). Synchronises.
 * MVP_ERR_CAPACITY if it does not fit the budget; MVP_ERR_INVALID_ARG if a
 * primitive's pose defines no box (see MVP_STATUS_POSE). */
MVP_API mvp_status mvp_serve_register_avatar(mvp_server *server, const mvp_prims *prims, int32_t *avatar_id);
/* Queues a request and admits what fits; *ticket identifies it. MVP_ERR_CAPACITY
 * if the image alone exceeds the budget or the arena; MVP_ERR_INVALID_ARG for a
 * bad avatar or parameters. */
MVP_API mvp_status mvp_serve_submit(mvp_server *server, const mvp_request *req, uint64_t *ticket);
/* Non-blocking: MVP_NOT_READY while the request is queued or running; MVP_OK once
 * done, after copying the image ([h][w][4] float32) to out_rgba (device or host
 * pointer, or NULL to drop it) and releasing its slot and memory. latency_ms
 * (nullable) = host time from submit until this poll saw it done. */
MVP_API mvp_status mvp_serve_poll(mvp_server *server, uint64_t ticket, float *out_rgba, double *latency_ms);
/* Withdraws a request: a queued one is dropped before anything runs; a running one
 * finishes on the device (its launch cannot be stopped) and the server frees its
 * slot and image memory once it is done. Either way the ticket is unknown from now
 * on. MVP_ERR_INVALID_ARG for an unknown (or already collected) ticket. */
MVP_API mvp_status mvp_serve_cancel(mvp_server *server, uint64_t ticket);
/* Polls until done or timeout_ms passes (MVP_ERR_TIMEOUT, request still queued or
 * running). */
MVP_API mvp_status mvp_serve_wait(mvp_server *server, uint64_t ticket, double timeout_ms, float *out_rgba,
                                  double *latency_ms);
/* Counters, and the kernel status bits (reads the device status word). */
MVP_API mvp_status mvp_serve_stats(mvp_server *server, mvp_serve_info *info);

/* ------------------------------------------------ decode-side epilogues */
/* The steps just upstream of the march that turn a decoder's outputs into march
 * inputs, and their gradients. All asynchronous on `stream`.
 *
 * Opacity fade (Sec. 3.1.3): dst = src with the opacity (channel 3) of every voxel
 * multiplied by W(x,y,z) = exp(-alpha (x^beta + y^beta + z^beta)), (x,y,z) in [-1,1]^3
 * the voxel's corner-aligned coordinates 2 (i, j, l)/(M - 1) - 1 (the paper uses
 * alpha = beta = 8; beta in [0, 64] is an integer). src: [n_prims][M][M][M][4] FP32
 * device; dst: the same layout in `dtype` (FP32, BF16 or FP16, round to nearest even),
 * so the fade is fused into the precision conversion. dst may equal src only for
 * FP32 output; other overlaps are rejected. Applied to a payload gradient (FP32, in
 * place) it gives the gradient with respect to the unfaded opacity. */
MVP_API mvp_status mvp_fade_payload(mvp_ctx *ctx, const float *src, void *dst, int64_t n_prims, int32_t M,
                                    int32_t dtype, float alpha, int32_t beta, mvp_stream stream);
/* A view's payload (Sec. 3.1.3: the colour decoder takes a view vector, the opacity
 * decoder does not): dst voxel = (rgb, opacity x W) with W the opacity fade above
 * (alpha = 0 gives W = 1). rgb [n_prims][M][M][M][3] FP32 (the view-dependent colour
 * decoded for this view), opacity [n_prims][M][M][M] FP32 (shared by every view), both
 * device, 4-byte aligned; dst [n_prims][M][M][M][4] in `dtype` (FP32, BF16 or FP16,
 * round to nearest even), 16-byte (FP32) or 8-byte aligned, overlapping neither input.
 * The result feeds mvp_prims.payload, or mvp_request.payload for one serving request. */
MVP_API mvp_status mvp_assemble_payload(mvp_ctx *ctx, const float *rgb, const float *opacity, void *dst,
                                        int64_t n_prims, int32_t M, int32_t dtype, float alpha, int32_t beta,
                                        mvp_stream stream);
/* Rotation from an axis-angle (Rodrigues) vector (Sec. 3.1.2: the paper's rotation
 * parameterisation): q = (cos(th/2), sin(th/2) r/th), th = |r| (q = (1, 0, 0, 0) at
 * r = 0). r [n][3], q [n][4] FP32 device; q feeds mvp_prims.q. */
MVP_API mvp_status mvp_axis_angle_to_quat(mvp_ctx *ctx, const float *r, int32_t n, float *q, mvp_stream stream);
/* Its vector-Jacobian product: g_r [n][3] += (dq/dr)^T g_q [n][4] (FP32 device), to
 * chain a g_q from mvp_raymarch_bwd to the axis-angle parameters. */
MVP_API mvp_status mvp_axis_angle_backward(mvp_ctx *ctx, const float *r, const float *g_q, int32_t n, float *g_r,
                                           mvp_stream stream);
/* Volume minimisation prior (Sec. 3.3): L_vol = lambda sum_k prod_j (2 s_kj), the
 * summed volumes with side lengths twice the half extents s [n][3] (FP32 device);
 * the paper uses lambda = 0.01. loss (device float, nullable) += L_vol; g_s (device
 * [n][3], nullable) += dL_vol/ds. */
MVP_API mvp_status mvp_volume_prior(mvp_ctx *ctx, const float *s, int32_t n, float lambda, float *loss, float *g_s,
                                    mvp_stream stream);

/* ------------------------------------------------ roofline probe */
/* No counterpart in the paper: a measurement of the GPU, the ceiling that the march's
 * and the adjoint's roofline fractions are taken against. Issues the voxel accesses of
 * the march (mode 0: per lane and sample, loads of the 8 corner voxels of one cell of
 * `payload` [n][M][M][M][4] in `dtype`) or of the adjoint (mode 1: a float4 reduction
 * into each of the 8 corners of `grad`, FP32 [n][M][M][M][4]) in the march's coherence
 * pattern (8x4-pixel warp tiles, neighbouring lanes a quarter voxel apart, consecutive
 * samples two thirds of a voxel apart), with no other work, one wave of full blocks on
 * every SM, `steps` samples per lane. Modes 2 and 3 gather the same 8 corners from
 * duplicated layouts: 2 = each voxel stored with its +x neighbour (`payload`
 * [n][M][M][M][2][4], 4 loads per cell), 3 = each voxel with its +x, +y and +x+y
 * neighbours ([n][M][M][M][2][2][4], 2 loads per cell). Mode 4 stages the plain
 * layout through shared memory: per chunk of 4 samples a warp copies the box of
 * voxels its lanes' cells span (up to 256 voxels; larger boxes are read directly)
 * and reads the corners from there. footprint 0: each SM works inside one primitive
 * (L1-resident after first touch); 1: warps move between all n primitives every 16
 * samples (L2-resident when the array fits L2). sink (device float[1], mode 0) receives
 * the sum of the loaded values; grad (mode 1) receives the reductions (contents are
 * meaningless). *accesses (host, nullable) = voxel accesses of the launch (each 16 B
 * FP32 or 8 B BF16/FP16). Arrays are device memory owned by the caller: payload 16-byte
 * (FP32) or 8-byte aligned (times 2 in mode 2 and 4 in mode 3), grad 16-byte aligned.
 * mode | (B << 8), B in 1..16, for modes 0 and 1: the same accesses at a fixed residency
 * of B 4-warp blocks per SM, each holding the march kernels' shared memory, under a
 * carveout that fits exactly B of them (the march runs 5 such blocks per SM, the adjoint
 * 3): the ceiling at the warps and L1 those kernels actually get; MVP_ERR_INVALID_ARG if
 * the device does not give that residency.
 * MVP_ERR_INVALID_ARG for bad sizes, modes or alignment. Asynchronous on `stream`; time it with events on that stream. */
MVP_API mvp_status mvp_gather_probe(const void *payload, int32_t dtype, int32_t n, int32_t M, int32_t mode,
                                    int32_t footprint, int32_t steps, float *grad, float *sink, int64_t *accesses,
                                    mvp_stream stream);

/* ------------------------------------------------ allocation-free render */
/* No counterpart in the paper. For callers that cannot allocate device memory:
 * a plug-in inside a host application that owns every device allocation, a
 * real-time frame loop that must not stall on the implicit synchronisation of
 * cudaMalloc/cudaFree, or a component whose memory budget is fixed at start-up.
 * Rebuilds the BVH of `prims` and renders `rays` into out_rgba (device, [n][4])
 * exactly as mvp_build_bvh + mvp_raymarch_fwd would, on the current CUDA device,
 * without a context or handle and without allocating: the BVH and the status word
 * live in a file-scope device array sized for MVP_STATIC_MAX_PRIMS primitives
 * (about 4 MB, held by every GPU that loads the library until the process exits).
 * Returns MVP_ERR_INVALID_ARG for more primitives than that (or any other bad
 * argument), before launching anything. The first call on a device looks up the
 * array's device address, and so does the first call after that device's context
 * was re-created (cudaDeviceReset, or the primary context released and retained
 * again): make those calls before any stream capture. Every call reuses
 * the same array and it keeps the last call's contents; calls whose GPU work
 * overlaps (other streams or threads) race on it and must be serialised by the
 * caller. status_out (device int32, nullable) receives the kernels' status bits
 * (MVP_STATUS_CAPACITY: a tile's BVH traversal stack overflowed; MVP_STATUS_POSE: a
 * primitive's pose defines no box).
 * Asynchronous on `stream`; no adjoint state is saved. */
#define MVP_STATIC_MAX_PRIMS 16384
MVP_API mvp_status mvp_raymarch_fwd_static(const mvp_prims *prims, const mvp_rays *rays, float *out_rgba,
                                           int32_t *status_out, mvp_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* MVP_H */
