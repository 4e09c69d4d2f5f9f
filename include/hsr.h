/*
 * hsr — batched triangle-mesh sensor rendering (colour, depth, semantic ids).
 *
 * C-ABI of the rendering hot path described in "Habitat: A Platform for
 * Embodied AI Research" (arXiv:1904.01201):
 *   - a scene is loaded once and its resources are shared by every agent that
 *     renders it (Appendix A, "Memory-efficient management of 3D environment
 *     resources ... cached and reused");
 *   - agents carry sensors at a pose and render observations of the scene
 *     (Appendix A, key abstractions "Agent", "Sensor"; Sec. 4 "Sensory input":
 *     colour camera and idealised depth sensor at the same pose, 90 degree FOV);
 *   - colour, depth and semantic outputs come from one pass (Sec. 3 "Rendering
 *     engine", multi-attachment "uber-shader").
 *
 * Conventions used by every call:
 *   - world is Y-up, metres; a pose is the camera position and a unit
 *     quaternion (w, x, y, z) rotating camera axes into world axes; the camera
 *     looks down its -Z axis with +Y up; depth is planar (d = -z_eye).
 *   - front faces are counter-clockwise seen from their visible side; back
 *     faces are culled.
 *   - outputs: RGB uint8 [n][H][W][3], depth float32 [n][H][W] (0 where
 *     nothing is hit), ids uint32 [n][H][W] (semantic[tri] when the scene has
 *     a semantic table, else the triangle index; 0xFFFFFFFF where nothing is
 *     hit). Row 0 is the top of the image.
 *   - render calls are asynchronous on the caller's CUDA stream (a
 *     cudaStream_t passed as void*, NULL = legacy default stream). Host input
 *     arrays (poses) may be reused as soon as the call returns. Output buffers
 *     are caller-owned device memory and must stay valid until the stream
 *     reaches the render.
 *   - every call returns an hsr_status; an error affects only that call.
 *     Calls are thread-safe for distinct scenes; a scene may be rendered from
 *     several threads and streams at once, but must not be freed while a
 *     render that uses it is in flight.
 */
#ifndef HSR_H
#define HSR_H

#include <stdint.h>

#if defined(__GNUC__)
#define HSR_API __attribute__((visibility("default")))
#else
#define HSR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HSR_OK = 0,
    HSR_ERR_INVALID_ARG = 1,  /* null pointer, zero count, index >= n_verts,
                                 non-finite input, non-unit quaternion
                                 (| |q| - 1 | > 1e-3), width/height outside
                                 1..4096, or intrinsics outside their limits
                                 (see hsr_intrinsics)                          */
    HSR_ERR_OOM = 2,          /* device or host allocation failed             */
    HSR_ERR_CUDA = 3,         /* a CUDA runtime call failed                    */
    HSR_ERR_TIMEOUT = 4,      /* a bounded device wait expired                 */
    HSR_ERR_OVERFLOW = 5,     /* a fixed-capacity buffer would overflow        */
    HSR_ERR_NO_DEVICE = 6     /* no CUDA device is visible                     */
} hsr_status;

typedef struct hsr_scene hsr_scene;          /* opaque, library-owned */
typedef struct hsr_agents hsr_agents;        /* opaque, library-owned (device-resident agents) */

typedef struct {
    float pos[3];      /* camera position in world metres                  */
    float quat[4];     /* w, x, y, z: world-from-camera rotation            */
} hsr_pose;

/*
 * Pinhole intrinsics. Limits (else HSR_ERR_INVALID_ARG): all finite, fx > 0,
 * fy > 0, |cx| <= 65536, |cy| <= 65536, 2^-20 <= znear < zfar.
 * Projected vertices are snapped to 1/256 pixel in 32-bit integers; a
 * triangle whose snapped coordinates would reach +-2^30 sub-pixels (very
 * near the camera, at large focal lengths or tiny near planes) is first
 * clipped to a guard band 2^21 pixels either side of the principal point,
 * which leaves the pixels it covers unchanged, so any pose is rendered.
 */
typedef struct {
    float fx, fy;      /* focal lengths in pixels (90 deg HFOV: fx = W/2)   */
    float cx, cy;      /* principal point in pixels (image centre: W/2,H/2) */
    float znear;       /* near clip distance, metres                        */
    float zfar;        /* fragments with depth > zfar are discarded         */
} hsr_intrinsics;

typedef struct {
    uint32_t n_tris, n_verts, n_meshlets, n_groups;
    uint64_t device_bytes;     /* device memory held by the scene           */
    float aabb_min[3], aabb_max[3];
} hsr_scene_info;

/*
 * Load a static triangle mesh into device memory (Appendix A: resources are
 * loaded once and shared by all agents rendering the scene).
 *   xyz          host, [n_verts][3] float32 world positions (finite, |v| <= 2^20)
 *   idx          host, [n_tris][3] uint32 vertex indices (< n_verts)
 *   uv           host, [n_verts][2] float32 texture coordinates, or NULL
 *   vert_rgb     host, [n_verts][3] uint8 vertex colours, or NULL
 *   atlas_rgba8  host, [atlas_h][atlas_w][4] uint8 texture (row 0 is v = 0), or NULL
 *   tri_semantic host, [n_tris] uint32 semantic ids (!= 0xFFFFFFFF), or NULL
 * Colour source: atlas+uv if both are given, else vertex colours, else white.
 * All inputs are copied; the caller may free them on return. On success *out
 * receives a scene handle owned by the library until hsr_scene_free.
 * The current CUDA device at load time owns the scene; render on that device.
 */
HSR_API int hsr_scene_load(const float *xyz, uint32_t n_verts, const uint32_t *idx, uint32_t n_tris,
                   const float *uv, const uint8_t *vert_rgb, const uint8_t *atlas_rgba8,
                   uint32_t atlas_w, uint32_t atlas_h, const uint32_t *tri_semantic,
                   hsr_scene **out);

/* Release a scene (synchronises the device first). NULL is accepted. */
HSR_API int hsr_scene_free(hsr_scene *scene);

/* Sizes and device footprint of a loaded scene. */
HSR_API int hsr_scene_get_info(const hsr_scene *scene, hsr_scene_info *info);

/*
 * Render n agents of one scene, one observation each (Sec. 4 "Sensory input":
 * colour + depth at the same pose and intrinsics; Sec. 3: one pass for all
 * outputs). poses: host [n]. intr: host, shared by all n views.
 * rgb: device [n][height][width][3]; depth: device [n][height][width], or
 * NULL for a colour-only sensor set; ids: device [n][height][width] or NULL.
 */
HSR_API int hsr_render(const hsr_scene *scene, const hsr_pose *poses, uint32_t n,
               const hsr_intrinsics *intr, uint32_t width, uint32_t height,
               uint8_t *rgb, float *depth, uint32_t *ids, void *cuda_stream);

/*
 * Render n agents spread over several resident scenes in one launch (the
 * batched replacement of the paper's multi-process GPU sharing, Table 1 and
 * Table 2 "processes"). scenes: host [n_scenes]; scene_of_agent: host [n],
 * each < n_scenes; outputs as for hsr_render, agent i at frame i.
 */
HSR_API int hsr_render_batch(const hsr_scene *const *scenes, uint32_t n_scenes,
                     const uint32_t *scene_of_agent, const hsr_pose *poses, uint32_t n,
                     const hsr_intrinsics *intr, uint32_t width, uint32_t height,
                     uint8_t *rgb, float *depth, uint32_t *ids, void *cuda_stream);

/*
 * Depth-sensor noise (Appendix C, noisy-depth evaluation): iid Gaussian noise
 * of standard deviation depth_sigma (1/m) added to the inverse depth of every
 * covered pixel; the paper's experiment uses 0.4. Pixel p of an agent with
 * key a draws two words of Philox-4x32-10 (Salmon et al., SC'11) at counter
 * (p, a, 0x6e6f6973, 0) under key (seed low word, seed high word), maps each
 * word x to u = ((x >> 9) + 0.5) * 2^-23 in (0, 1) and takes the Box-Muller
 * variate z = sqrt(-2 ln u1) cos(2 pi u2); q' = 1/depth + depth_sigma * z.
 * The pixel reports depth 1/q', or 0 (no return) when q' <= 1/zfar.
 * Background pixels stay 0; colour and ids are unchanged. agent_ids: host [n]
 * stream keys, or NULL to key each agent by its output frame. depth_sigma
 * must be finite and >= 0 (0 = noise-free) and reserved 0, else
 * HSR_ERR_INVALID_ARG. The struct and agent_ids are read before the call
 * returns.
 */
typedef struct {
    float depth_sigma;
    uint32_t reserved;
    uint64_t seed;
    const uint32_t *agent_ids;
} hsr_depth_noise;

/* hsr_render_batch with depth noise (noise may be NULL; scene_of_agent may be
 * NULL when n_scenes == 1). */
HSR_API int hsr_render_noisy(const hsr_scene *const *scenes, uint32_t n_scenes,
                     const uint32_t *scene_of_agent, const hsr_pose *poses, uint32_t n,
                     const hsr_intrinsics *intr, uint32_t width, uint32_t height,
                     uint8_t *rgb, float *depth, uint32_t *ids, const hsr_depth_noise *noise,
                     void *cuda_stream);

/*
 * Texture sampling of a textured scene (the paper does not state its
 * filtering): HSR_SAMPLE_BILINEAR (default) samples the atlas bilinearly;
 * HSR_SAMPLE_TRILINEAR samples minified textures through a mip chain built
 * from the atlas on the first call: level l+1 is max(1, W_l >> 1) x
 * max(1, H_l >> 1) texels, each the rounded mean (a + b + c + d + 2) >> 2 of
 * its 2x2 block of level l (reads past the last row or column repeat it).
 * Per pixel, lambda = log2(rho), rho the larger texel-space length of the
 * perspective-correct uv derivative along x and along y at the pixel centre;
 * lambda <= 0 samples level 0 bilinearly (as HSR_SAMPLE_BILINEAR); otherwise
 * the bilinear samples of levels floor(lambda) and floor(lambda) + 1 (the
 * last level beyond it) are blended with weight frac(lambda), each level
 * sampled at (u W_l - 0.5, v H_l - 0.5), and rounded. Applies to renders
 * issued after the call returns; HSR_ERR_INVALID_ARG for an untextured scene
 * or an unknown mode.
 */
enum { HSR_SAMPLE_BILINEAR = 0, HSR_SAMPLE_TRILINEAR = 1 };
HSR_API int hsr_scene_set_sampling(hsr_scene *scene, int mode);

/*
 * General view lists: each view names its scene, pose, output frame and the
 * outputs it writes, so one call can render several sensors per agent, such
 * as the semantic sensor of Table 2 (footnote), whose ids come from a
 * separate, denser semantic mesh: view (colour mesh, pose, frame f,
 * HSR_OUT_RGB | HSR_OUT_DEPTH) plus view (semantic mesh, pose, frame f,
 * HSR_OUT_IDS). views: host [n]; outputs 0 means every present buffer;
 * frame < n_frames (the frames the output buffers hold); no output of a frame
 * may be written by two views (HSR_ERR_INVALID_ARG). A buffer may be NULL
 * when no view writes it (at least one buffer must be given). Noise streams
 * are keyed by noise->agent_ids[i], else by the view's frame.
 */
enum { HSR_OUT_RGB = 1, HSR_OUT_DEPTH = 2, HSR_OUT_IDS = 4 };
typedef struct {
    hsr_pose pose;
    uint32_t scene;            /* index into scenes */
    uint32_t frame;            /* output frame */
    uint32_t outputs;          /* HSR_OUT_* bits, or 0 for all */
} hsr_view;
HSR_API int hsr_render_views(const hsr_scene *const *scenes, uint32_t n_scenes, const hsr_view *views, uint32_t n,
                             uint32_t n_frames, const hsr_intrinsics *intr, uint32_t width, uint32_t height,
                             uint8_t *rgb, float *depth, uint32_t *ids, const hsr_depth_noise *noise,
                             void *cuda_stream);

/*
 * Serving (continuous batching of render requests as rollout workers step).
 * A server keeps the scenes resident, owns a pool of output framebuffers per
 * served square resolution (its admission budget, fb_bytes, split by
 * res_weight), and runs a scheduler thread: submitted requests queue per
 * resolution; a request is admitted when a framebuffer slot of its
 * resolution is free; admitted requests of one resolution are packed into a
 * micro-batch (<= max_batch views, waiting at most max_wait_us for more) and
 * rendered by replaying that resolution's captured graph on one of n_streams
 * streams, so micro-batches overlap on the device. A completion thread polls
 * each stream's event while a micro-batch is in flight (it keeps one host
 * core busy then, and sleeps otherwise). Each request yields one result
 * (polled), which points at its device frame until released.
 * Results are identical to a one-shot hsr_render of the same view.
 *
 * Action requests (agent >= 0; needs hsr_server_attach_agents) carry an
 * action instead of a pose: the agent's device-resident pose is moved by the
 * actuation rules of hsr_batch_step and the new view is rendered; scene and
 * pose fields are ignored. Per agent, actions apply in submission order and
 * one at a time: an agent's next action is launched after its previous one
 * completed. A micro-batch holds either pose or action requests.
 */
typedef struct hsr_server hsr_server;
typedef struct {
    uint32_t n_res;            /* served square resolutions (1..8) */
    uint32_t res[8];           /* side lengths in pixels */
    float res_weight[8];       /* share of fb_bytes per resolution */
    uint64_t fb_bytes;         /* framebuffer pool: the admission budget */
    uint32_t max_batch;        /* views per micro-batch */
    uint32_t n_streams;        /* micro-batches in flight */
    uint32_t max_queue;        /* queued requests beyond this are rejected */
    uint32_t max_wait_us;      /* a partial micro-batch waits at most this long */
    float znear, zfar;         /* every resolution: 90 degree HFOV pinhole */
    int with_ids;              /* also produce the id buffer */
} hsr_server_config;
typedef struct {
    uint64_t tag;              /* caller's identifier, returned in the result */
    uint32_t scene;            /* pose requests: index into the server's scenes */
    uint32_t res;              /* one of the served resolutions */
    hsr_pose pose;             /* pose requests: the camera pose to render */
    int32_t agent;             /* < 0: pose request; else an action request of this agent of the attached set */
    uint32_t action;           /* action requests: hsr_action applied on the device before rendering */
} hsr_request;
typedef struct {
    uint64_t tag;
    int status;                /* HSR_OK, HSR_ERR_OVERFLOW (queue full), HSR_ERR_INVALID_ARG, ... */
    uint32_t res, slot;
    uint8_t *rgb;              /* device [res][res][3] */
    float *depth;              /* device [res][res] */
    uint32_t *ids;             /* device [res][res] or NULL */
    double t_submit, t_launch, t_done;   /* seconds on hsr_server_now's clock */
} hsr_result;
typedef struct {
    uint64_t submitted, completed, rejected, batches;
    uint32_t queued, in_flight;
    uint64_t fb_bytes_used, fb_bytes_total;
} hsr_server_stats;
HSR_API int hsr_server_create(const hsr_scene *const *scenes, uint32_t n_scenes, const hsr_server_config *cfg,
                              hsr_server **out);
/* Bind the agent set that action requests step (its scenes: the server's, in
 * the same order; same device). Only while no request is queued or in
 * flight; agents must outlive the server or a later attach. NULL detaches. */
HSR_API int hsr_server_attach_agents(hsr_server *server, hsr_agents *agents);
HSR_API int hsr_server_submit(hsr_server *server, const hsr_request *requests, uint32_t n);
/* Completed results (up to max); waits up to wait_us for the first one. */
HSR_API int hsr_server_poll(hsr_server *server, hsr_result *out, uint32_t max, uint32_t *n_out, uint32_t wait_us);
/* Return the framebuffers of consumed results to the pool. */
HSR_API int hsr_server_release(hsr_server *server, const hsr_result *results, uint32_t n);
HSR_API int hsr_server_get_stats(hsr_server *server, hsr_server_stats *stats);
HSR_API double hsr_server_now(void);
HSR_API int hsr_server_destroy(hsr_server *server);

/*
 * Launch configuration of the render kernels (performance only: every valid
 * configuration produces identical outputs).
 */
typedef struct {
    uint32_t small_px;     /* triangles with at most this many candidate pixels: one thread each (1..32) */
    uint32_t bin_px;       /* more than this: binned to 8x8 screen tiles; in between: per-warp queue */
    uint32_t chunk;        /* visible (view, meshlet) pairs a raster warp fetches at a time (1..32) */
    uint32_t ctas_per_sm;  /* raster CTAs per SM (1..3) */
    uint32_t n_phases;     /* occlusion phases (1..3); 1 disables occlusion culling */
    float phase_r[2];      /* distance bands of the phases, metres */
} hsr_config;

/*
 * Persistent batch (the batched form of the scope: many agents of several
 * resident scenes per launch, captured once in a CUDA graph and replayed).
 * hsr_batch_create sizes all scratch for up to n_cap views at width x height
 * of the given scenes, binds the output buffers (rgb [n_cap][H][W][3], depth
 * [n_cap][H][W], ids [n_cap][H][W] or NULL, device), and captures the whole
 * render (descriptor upload, culling, raster phases, shading) into CUDA
 * graphs; cfg == NULL uses the tuned configuration of this signature, if
 * any, else the default. hsr_batch_render sets up n <= n_cap views from host
 * poses (scene_of_agent: host [n] indices into the create-time scenes, or
 * NULL for scene 0; frames: host [n] output frames < n_cap, or NULL for
 * 0..n-1) and replays the graph on `cuda_stream`. Replays of one batch must
 * be ordered on the GPU (same stream or explicit waits): they share scratch.
 * Host arrays may be reused when the call returns; it may wait for the
 * replay before last to finish its descriptor upload.
 */
typedef struct hsr_batch hsr_batch;
HSR_API int hsr_batch_create(const hsr_scene *const *scenes, uint32_t n_scenes, uint32_t n_cap,
                             const hsr_intrinsics *intr, uint32_t width, uint32_t height, uint8_t *rgb,
                             float *depth, uint32_t *ids, const hsr_config *cfg, hsr_batch **out);
HSR_API int hsr_batch_render(hsr_batch *batch, const uint32_t *scene_of_agent, const hsr_pose *poses, uint32_t n,
                             const uint32_t *frames, void *cuda_stream);
/* hsr_batch_render with depth noise (noise may be NULL); agents without
 * agent_ids are keyed by their output frame. The noise settings are per
 * replay: one captured graph serves noisy and noise-free batches. */
HSR_API int hsr_batch_render_noisy(hsr_batch *batch, const uint32_t *scene_of_agent, const hsr_pose *poses,
                                   uint32_t n, const uint32_t *frames, const hsr_depth_noise *noise,
                                   void *cuda_stream);
/* View-list render on a batch (views as for hsr_render_views, n <= n_cap,
 * frame < the batch's frame count). */
HSR_API int hsr_batch_render_views(hsr_batch *batch, const hsr_view *views, uint32_t n,
                                   const hsr_depth_noise *noise, void *cuda_stream);
/*
 * Render to host memory (the GPU->CPU transfer of Table 2): hsr_batch_render
 * of n views into frames 0..n-1, then device->host copies of those frames'
 * outputs on the same stream: host_rgb [n][H][W][3], host_depth [n][H][W],
 * host_ids [n][H][W] (host memory, page-locked for the copies to run
 * asynchronously; each may be NULL to skip that output, and a non-NULL one
 * needs the batch's device buffer of that output, else HSR_ERR_INVALID_ARG).
 * Asynchronous like cudaMemcpyAsync: the host buffers hold the frames once
 * the stream has passed the copies. Copies of one call overlap the render of
 * another only on another stream: alternate two batches (each with its own
 * device outputs) on two streams to keep both the copy engine and the SMs
 * busy. *h2d_bytes (may be NULL) receives the bytes the call uploads (the
 * view descriptor block).
 */
HSR_API int hsr_batch_render_host(hsr_batch *batch, const uint32_t *scene_of_agent, const hsr_pose *poses,
                                  uint32_t n, uint8_t *host_rgb, float *host_depth, uint32_t *host_ids,
                                  void *cuda_stream, uint64_t *h2d_bytes);
HSR_API int hsr_batch_destroy(hsr_batch *batch);

/*
 * Agents with device-resident state (Sec. 4 "Agent embodiment and action
 * space": the agent acts with stop, move_forward, turn_left, turn_right,
 * mapped to idealised actuations of 0.25 m and 10 degrees). A step batch
 * takes one action per agent instead of a pose: a pass on the device moves
 * each agent's pose and builds its camera, then the render runs; the host
 * sends only action ids.
 *
 * Actuation rules (double arithmetic from the float pose, each stored
 * component rounded once to float):
 *   stop         : pose unchanged (the observation is rendered again).
 *   move_forward : heading = R (0, 0, -1) of the normalised quaternion with its
 *                  vertical part dropped, h = (-2(xz + wy), -(1 - 2(x^2 + y^2)));
 *                  p' = p + forward_m * h / |h| on x and z, rounded to float.
 *                  Refused (pose unchanged; no sliding) when |h| = 0 or the
 *                  grid cell (floor((x - x0)/cell), floor((z - z0)/cell)) of
 *                  p' is outside the grid or not navigable.
 *   turn_left / turn_right : q' = r q with r = (cos(t/2), 0, sin(t/2), 0),
 *                  t = +turn_deg / -turn_deg (about world +Y), then q' / |q'|.
 *
 * hsr_agents_create: scenes [n_scenes] (the same array, in the same order, as
 * the batches that step these agents), navmaps [n_scenes] (grid: host
 * [nz][nx] bytes, nonzero = navigable, copied; the grid's x/z extent must lie
 * inside the scene's bounding box), scene_of_agent [n_agents] (NULL: scene 0),
 * poses [n_agents]: valid camera poses (unit quaternion within 1e-3) on
 * navigable cells with y inside the scene's bounding box; act NULL means
 * 0.25 m and 10 degrees. Errors: HSR_ERR_INVALID_ARG for any violation,
 * HSR_ERR_OOM, HSR_ERR_CUDA. The state lives on the device current at create.
 * hsr_agents_get_poses copies all poses to host [n_agents] after the work
 * queued on cuda_stream (it waits for that stream).
 * hsr_agents_set_poses overwrites agents idx [n] (host) with poses [n] under
 * the create-time rules, ordered on cuda_stream.
 * hsr_batch_step: agent_idx [n] distinct agents (< n_agents), actions [n]
 * (hsr_action), frames [n] output frames or NULL for 0..n-1, noise as for
 * hsr_batch_render_noisy (streams keyed by the output frame unless
 * agent_ids are given). The batch and the agents must have the same scenes
 * and device. Steps that touch the same agent must be ordered on the GPU.
 */
enum { HSR_ACTION_STOP = 0, HSR_ACTION_MOVE_FORWARD = 1, HSR_ACTION_TURN_LEFT = 2, HSR_ACTION_TURN_RIGHT = 3 };
typedef struct {
    float x0, z0;          /* world x, z of the grid's corner: cell (0, 0) covers [x0, x0 + cell) x [z0, z0 + cell) */
    float cell;            /* cell edge, metres (> 0) */
    uint32_t nx, nz;       /* grid size (>= 1 each) */
    const uint8_t *grid;   /* host [nz][nx] */
} hsr_navmap;
typedef struct {
    float forward_m;       /* move_forward displacement, metres (finite, >= 0) */
    float turn_deg;        /* turn angle, degrees (finite) */
} hsr_actuation;
HSR_API int hsr_agents_create(const hsr_scene *const *scenes, uint32_t n_scenes, const hsr_navmap *navmaps,
                              uint32_t n_agents, const uint32_t *scene_of_agent, const hsr_pose *poses,
                              const hsr_actuation *act, hsr_agents **out);
HSR_API int hsr_agents_get_poses(hsr_agents *agents, hsr_pose *poses, void *cuda_stream);
HSR_API int hsr_agents_set_poses(hsr_agents *agents, const uint32_t *idx, const hsr_pose *poses, uint32_t n,
                                 void *cuda_stream);
HSR_API int hsr_agents_destroy(hsr_agents *agents);
HSR_API int hsr_batch_step(hsr_batch *batch, hsr_agents *agents, const uint32_t *agent_idx, const uint8_t *actions,
                           uint32_t n, const uint32_t *frames, const hsr_depth_noise *noise, void *cuda_stream);

/* Fill *cfg with the built-in default configuration. */
HSR_API int hsr_config_default(hsr_config *cfg);

/*
 * Autotuner (the batching row of the scope: bin and tile sizes chosen per
 * workload). Renders the given batch repeatedly (into the given outputs)
 * under candidate configurations, each captured as a batch graph (as
 * hsr_batch_create does) and timed with CUDA events on the caller's stream
 * around its launch, after a 256 MiB device write that evicts L2 (median of
 * `reps` timed launches after one warm-up; the 256 MiB is allocated for the
 * call), by two sweeps of coordinate descent (small-triangle bound, bin
 * threshold, chunk, occlusion phases together with their band radii, CTAs per
 * SM) from the default for this call's size (one occlusion phase below 16,384
 * culling items, two above; bins above 32 candidates up to 2^24 pixels over
 * all views, above 256 beyond); stores the fastest configuration for
 * this workload signature (scene set, n, width, height, ids present) so that
 * later hsr_render / hsr_render_batch calls with the same signature use it,
 * and returns it in *best (and its time in *best_ms). Synchronises the stream.
 * Arguments as for hsr_render_batch (scene_of_agent may be NULL when
 * n_scenes == 1).
 */
HSR_API int hsr_autotune(const hsr_scene *const *scenes, uint32_t n_scenes, const uint32_t *scene_of_agent,
                         const hsr_pose *poses, uint32_t n, const hsr_intrinsics *intr, uint32_t width,
                         uint32_t height, uint8_t *rgb, float *depth, uint32_t *ids, void *cuda_stream,
                         uint32_t reps, hsr_config *best, float *best_ms);

/* Register a configuration for a workload signature (e.g. one loaded from a
 * tuning cache); cfg == NULL removes it. */
HSR_API int hsr_set_tuned_config(const hsr_scene *const *scenes, uint32_t n_scenes, uint32_t n, uint32_t width,
                                 uint32_t height, int with_ids, const hsr_config *cfg);

/*
 * Diagnostic stage timing (measurement support, not part of the method).
 * While enabled, every render call records CUDA events on its stream around
 * its three stages; hsr_get_stage_timing waits for the last call's events and
 * writes ms[0] = cull, ms[1] = raster, ms[2] = shade, ms[3] = all three
 * (milliseconds). It returns HSR_ERR_INVALID_ARG if no call was timed since
 * timing was enabled. The event set is global: use from one thread at a time.
 */
HSR_API int hsr_set_stage_timing(int enable);
HSR_API int hsr_get_stage_timing(float *ms);

/*
 * Diagnostic work counters (measurement support, not part of the method).
 * While enabled, render calls count, per occlusion phase, the visible
 * (view, meshlet) pairs rasterised and the meshlets skipped as hidden;
 * hsr_get_stage_stats synchronises the device and writes counts[0..2] = pairs
 * per phase, counts[3..5] = skipped per phase, counts[6] = (view, meshlet)
 * pairs inside the frustum, counts[7] = of those, planar meshlets facing away
 * but kept (the margin did not prove every triangle culled), counts[8] =
 * planar meshlets skipped as facing away, for the last call (counts: 9
 * words). Enabling allocates 64 bytes of device memory once. Use from one
 * thread at a time.
 */
HSR_API int hsr_set_stage_stats(int enable);
HSR_API int hsr_get_stage_stats(uint32_t *counts);

/*
 * Allocation-free variant of hsr_render (the paper has no counterpart; this is
 * a library-integration feature). Same arguments, outputs and results as
 * hsr_render (any non-empty subset of rgb, depth, ids), but no memory is
 * allocated on the call path: its scratch (view descriptors, z-buffer,
 * visible-meshlet list) is one fixed 32 MiB array in device memory, present
 * on every GPU that loads the library until the process exits. For callers
 * that cannot let a library allocate: processes whose framework already
 * holds the device memory in its own pool, loops that cannot afford an
 * allocator call, and hosts that route every allocation through their own
 * allocator.
 *   - A call needing more than 32 MiB of scratch (about 8 B per output pixel
 *     per view + 48 B per meshlet per view + 192 B per view) returns
 *     HSR_ERR_OVERFLOW; split such batches or use hsr_render.
 *   - The view descriptors are staged in a fixed 1 MiB host buffer (192 B per
 *     view: at most 5,457 views per call, more return HSR_ERR_OVERFLOW). It is
 *     ordinary pageable memory, copied with cudaMemcpyAsync under a
 *     process-wide lock: the copy has read it when the call returns, and the
 *     call may wait for work queued earlier on the stream.
 *   - Large triangles are rasterised by the warp that set them up (the
 *     separate large-triangle pass of hsr_render needs scratch this array
 *     does not hold): the images are the same, the speed can differ.
 *   - All calls share the array and it keeps the last call's contents (each
 *     call re-initialises what it needs). Calls whose work overlaps on the
 *     GPU race and corrupt each other's images: order them on one stream.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it for the process.
 */
HSR_API int hsr_render_noalloc(const hsr_scene *scene, const hsr_pose *poses, uint32_t n,
                       const hsr_intrinsics *intr, uint32_t width, uint32_t height,
                       uint8_t *rgb, float *depth, uint32_t *ids, void *cuda_stream);

/* Static description of a status code. */
/*
 * Device status: the raster kernels stage geometry with asynchronous bulk
 * copies and wait for them with a time limit (one second); a wait that
 * expires makes the kernel stop, record the failure and return, leaving the
 * context usable (the frame is then incomplete). hsr_device_status waits for
 * the current device and returns HSR_ERR_TIMEOUT if any kernel recorded such
 * a failure since the last clear (clear != 0 resets the record),
 * HSR_ERR_OVERFLOW if a triangle was dropped because its guard-band-clipped
 * vertices still left the fixed-point range (not reachable within the
 * documented input limits), HSR_OK otherwise, HSR_ERR_CUDA if the device
 * cannot be queried.
 */
HSR_API int hsr_device_status(int clear);
/* Test hook for the failure path above: renders launched while extra_bytes
 * is non-zero arm every geometry staging for extra_bytes more than their
 * copies deliver, so each wait expires (about one second per raster warp).
 * 0 restores normal operation. Not for production use. */
HSR_API int hsr_debug_inject_wait_fault(uint32_t extra_bytes);

HSR_API const char *hsr_status_string(int status);

/* Library version, "major.minor.patch". */
HSR_API const char *hsr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HSR_H */
