// Internal layout shared by the host library (api.cpp) and the kernels (render.cu).
#pragma once
#include <algorithm>

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hsr.h"

namespace hsr {

// Meshlets: up to 32 triangles and 64 distinct vertices, spatially coherent
// (Morton order of triangle centroids). Groups: 32 consecutive meshlets,
// group g holding meshlets [32 g, 32 g + 32) (the last one fewer).
constexpr int kMeshletTris = 32;
constexpr int kMeshletVerts = 64;
constexpr int kGroupMeshlets = 32;

// Meshlet m owns vertices [vbase, meshlets[m+1].vbase) and triangles
// [tbase, meshlets[m+1].tbase); a sentinel entry follows the last meshlet.
struct alignas(16) Meshlet {
    float bmin[3];
    uint32_t vbase;
    float bmax[3];
    uint32_t tbase;
};

struct alignas(16) Group {
    float bmin[3];
    uint32_t m0;
    float bmax[3];
    uint32_t m1;     // meshlets [m0, m1)
};

enum ColorMode : int { kColorWhite = 0, kColorTexture = 1, kColorVertex = 2 };

// Device-side view of a loaded scene (all pointers are device memory).
struct SceneDev {
    const Meshlet *meshlets;   // n_meshlets + 1
    const Group *groups;       // n_groups
    const float4 *mvert;       // meshlet vertices: x, y, z, bits(caller vertex index)
    const uint2 *mtri;         // x: local indices (8 bits each, canonical order), y: triangle index
    const uint4 *tri;          // canonical (i0, i1, i2) + output id, per triangle index
    const float4 *vert;        // x, y, z, 0 per caller vertex
    // per triangle, one 64-byte shading record (4 float4), vertices in canonical
    // order: p0.xyz p1.x | p1.yz p2.xy | p2.z a0 a1 a2 | a3 a4 a5 bits(id), where
    // a = uv0.uv uv1.uv uv2.uv (textured), or bits(rgb0, rgb1, rgb2), 0, 0, 0
    const float4 *srec;
    // per meshlet, two records: (unit normal n, plane offset w) of its triangles'
    // common plane, and (minimum triangle area, longest edge, max |n.x - w| over
    // its vertices, max |n_t - n| over its triangles); longest edge < 0 when the
    // triangles are not one plane (never back-face culled as a whole)
    const float4 *mplane;
    float coord_max;           // largest |coordinate| of any vertex
    const float2 *uv;          // per vertex, or null
    const uint32_t *vrgb;      // r | g << 8 | b << 16 per vertex, or null
    const uint32_t *atlas;     // RGBA8 texels, row-major, or null
    unsigned long long atlas_tex;  // the atlas as a texture object (uchar4, clamp, unnormalised), or 0
    uint32_t atlas_w, atlas_h;
    uint32_t n_groups, n_meshlets, n_tris, n_verts;
    int color_mode;
    uint32_t sample_mode;      // HSR_SAMPLE_BILINEAR or HSR_SAMPLE_TRILINEAR
    const uint32_t *mips;      // mip levels 1.. of the atlas, RGBA8 texels (trilinear sampling)
    uint32_t n_levels;         // levels including the atlas itself (level 0)
    uint32_t mip_off[16];      // texel offset of level l in `mips` (l >= 1); level l is max(1, W >> l) x max(1, H >> l)
};

// One rendered view: world-to-eye matrix (rows of a 3x4), the six world-space
// frustum planes used for culling (n . p + off >= 0 inside), its scene, and
// the output frame it writes.
struct alignas(16) View {
    float M[12];
    float planes[24];
    float pos[3];              // camera position (distance bands of the occlusion phases)
    uint32_t scene;
    uint32_t frame;
    uint32_t agent;            // key of the depth-noise stream
    uint32_t state;            // agent-state slot moved by the actuation pass (step batches)
    uint32_t action;           // action applied to that slot first (hsr_action)
    uint32_t outputs;          // HSR_OUT_* bits this view writes (with its buffer present), | kViewGuard
    uint32_t pad_[3];
};

static_assert(sizeof(View) == 192, "View is 12 x 16 bytes");

// Navigability grid of one scene on the device.
struct NavDev {
    float x0, z0, cell;
    uint32_t nx, nz, pad_;
    const uint8_t *grid;       // [nz][nx], nonzero = navigable
};

// Device-resident agents: poses, per-scene grids, actuation amounts. Its
// device address sits in the descriptor header (dyn[6], dyn[7]) of a step
// batch, so one captured graph serves any agent set.
struct AgentsDev {
    float *pose;               // [n_agents][7]: x, y, z, qw, qx, qy, qz
    const NavDev *nav;         // [n_scenes]
    uint32_t n_agents, n_scenes;
    double step;               // forward displacement, metres
    double c_turn[2], s_turn[2];   // cos, sin of half the left [0] / right [1] turn angle
};

// Texels of the tile-z pyramid over a w x h tile grid (levels halve, rounding
// up, down to 1 x 1); *levels receives the level count.
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t hiz_pyramid_texels(uint32_t w, uint32_t h, uint32_t *levels)
{
    uint32_t total = 0, n = 0;
    for (;;) {
        total += w * h;
        n++;
        if (w <= 1 && h <= 1) break;
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    if (levels) *levels = n;
    return total;
}

// A visible (view, meshlet) pair as the raster consumes it, self-contained so
// that no meshlet record is read on the raster path:
//   x = view | (n_verts - 1) << 21 | (n_tris - 1) << 27, y = meshlet,
//   z = first vertex, w = first triangle of the meshlet's ranges.
constexpr uint32_t kMaxViews = 1u << 21;
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint4 pair_entry(uint32_t view, uint32_t meshlet, uint32_t vbase, uint32_t nv, uint32_t tbase, uint32_t nt)
{
    return uint4{view | (nv - 1u) << 21 | (nt - 1u) << 27, meshlet, vbase, tbase};
}
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t pair_view(const uint4 &e) { return e.x & (kMaxViews - 1u); }
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t pair_nv(const uint4 &e) { return ((e.x >> 21) & 63u) + 1u; }
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t pair_nt(const uint4 &e) { return (e.x >> 27) + 1u; }

// Set in View::outputs by the rasteriser when it emitted a guard-band-clipped
// triangle for the view; the host writes every view record afresh for each
// render.
constexpr uint32_t kViewGuard = 1u << 31;

constexpr uint32_t kErrWaitTimeout = 1u;    // a bounded wait for a bulk copy gave up
constexpr uint32_t kErrRange = 2u;          // a guard-clipped vertex still left the fixed-point range

struct Params {
    const SceneDev *scenes;    // device array
    const View *views;         // device array, n_views (sorted by scene)
    unsigned long long *zbuf;  // [n_views][H][W] 64-bit keys, preset to ~0
    uint8_t *rgb;
    float *depth;
    uint32_t *ids;             // may be null
    // Visible (view, meshlet) pairs written by the cull kernel (pair_entry
    // layout), one list per occlusion phase in a buffer of 2 * vis_cap
    // entries: phase 0 grows up from vis[0], phase 2 grows down from
    // vis[vis_cap - 1], phase 1 grows up from vis[vis_cap] (vis_cap = worst
    // case, every meshlet in every view).
    uint4 *vis;
    uint32_t *vis_count;       // [3] pairs per phase (preset to 0)
    uint32_t *work_counter;    // [3] raster work cursor per phase (preset to 0)
    uint32_t vis_cap;
    // Views are sorted by scene; slot k covers views [slot_view_base[k], ...)
    // of scene slot_scene[k] and work items [slot_item_base[k], slot_item_base[k+1]),
    // item = slot_item_base[k] + (view - slot_view_base[k]) * n_groups + group.
    const uint32_t *slot_item_base;   // n_slots + 1
    const uint32_t *slot_view_base;   // n_slots
    const uint32_t *slot_scene;       // n_slots
    uint32_t n_slots;          // capacity of the slot arrays
    uint32_t n_views, width, height;   // n_views: capacity (frames of scratch); the active count is dyn[0]
    uint32_t total_items;      // upper bound of the work items (grid sizing); the exact count is dyn[1]
    // dyn[0] = active views, dyn[1] = (view, group) work items, dyn[2] = slots in use,
    // dyn[3] = depth-noise sigma (float bits; 0 = noise-free), dyn[4..5] = noise seed (low, high),
    // dyn[6..7] = device address of the AgentsDev of a step batch (low, high):
    // read by the kernels from device memory, so one captured graph can replay
    // batches of different sizes and scene mixes
    const uint32_t *dyn;
    float inv_far;             // 1/far: a noisy inverse depth at or below it reports depth 0
    float fx, fy, cx, cy, znear, zfar;
    float q_far;               // smallest float q with 1/q <= zfar
    float gx, gy;              // guard planes |x_e| <= gx d, |y_e| <= gy d (2^21 / fx, 2^21 / fy)
    uint32_t small_px;         // per-thread raster when a triangle has at most this many candidate pixels
    uint32_t bin_px;           // bins for triangles with more candidate pixels than this; per-warp queue between
    uint32_t chunk;            // consecutive visible pairs a raster warp takes per step (<= 32)
    // occlusion phases: a visible meshlet at distance r from the camera goes
    // to phase (r > phase_r[0]) + (r > phase_r[1]), limited to n_phases - 1;
    // phases after the first skip meshlets the hierarchical z-buffer proves hidden
    uint32_t n_phases;         // 1 (no occlusion culling) .. 3
    float phase_r2[2];         // squared band radii, metres^2
    // Tile-z pyramid per view (hiz_total texels): level 0 is the hiz_w x
    // hiz_h grid of 8x8-pixel tiles, each the largest stored key >> 32 (the
    // farthest fragment, or 0xFFFFFFFF for background); level l+1 halves
    // level l (rounding up), each texel the max of its up to 2x2 children,
    // down to 1 x 1.
    uint32_t *hiz;
    uint32_t hiz_total;
    // Pairs of phases 1 and 2 that the pyramid does not prove hidden,
    // compacted by occl_kernel for the raster of that phase.
    uint4 *surv;
    uint32_t *surv_count;      // [2] survivors of phase 1, phase 2 (preset to 0)
    uint32_t fault_tx;         // test hook: extra bytes each meshlet staging waits for (0 in normal operation)
    uint32_t cull_views;       // views a culling warp item covers (1..16, from the amount of work)
    uint32_t *stats;           // diagnostic counters or null: [0..2] pairs per phase, [3..5] skipped per phase
    // Bins of large triangles: a triangle with more than bin_px candidate
    // pixels is stored once in `big_rec` and binned as runs of up to 32 rows
    // of its candidate rectangle (`big_inst`, one list of big_inst_cap
    // entries per phase); big_raster_kernel rasterises the bins after each
    // phase. Null / full bins fall back to the per-warp queue.
    struct BigTri *big_rec;
    uint32_t *big_rec_count;   // [1]
    uint32_t big_rec_cap;
    uint2 *big_inst;           // (record, first row of a run from the top of its candidate rectangle | run length << 16)
    uint32_t *big_inst_count;  // [3]
    uint32_t big_inst_cap;
    uint32_t hiz_w, hiz_h;
};

constexpr int kHizTile = 8;
constexpr uint32_t kMaxMeshlets = 0x0FFFFFFFu;

// Launch configuration chosen by the host (autotuned).
constexpr uint32_t kBigRecCap = 1u << 18;
// storage size of one binned large triangle (kernels/raster.cuh BigTri)
struct alignas(16) BigTriStorage {
    unsigned char bytes[64];
};
constexpr uint32_t kBigInstCap = 1u << 20;

struct LaunchCfg {
    uint32_t small_px = 32;
    uint32_t bin_px = 64;
    uint32_t chunk = 4;
    uint32_t raster_ctas_per_sm = 3;
    uint32_t n_phases = 2;
    float phase_r[2] = {4.0f, 10.0f};
};


// Sets kernel attributes for the current device (call before stream capture).
cudaError_t prepare_kernels();

// Launches the cull, raster and shade kernels on `stream`; `guard`: some view
// may snap a vertex beyond +-2^30 sub-pixels (guard_free failed for it), so
// shading compiles in the guard-band path; `noise`: the call adds depth noise
// (the shading variant with the noise model); `pdl`: kernels after the cull
// use programmatic dependent launch (direct calls; graph-captured batches,
// whose launch gaps are already small and which serve concurrent streams,
// launch them plainly: early-scheduled waiting CTAs would hold SM slots the
// other streams' work could use).
cudaError_t launch_render(const Params &p, const LaunchCfg &cfg, cudaStream_t stream, bool guard, bool noise,
                          bool pdl);
// Device error flags (kErrWaitTimeout, ...) raised by kernels on the current
// device since the last clear; waits for the device.
cudaError_t read_device_errors(uint32_t *flags, bool clear);
// Test hook for the bounded waits (see hsr_debug_inject_wait_fault).
uint32_t debug_fault_tx();
void set_debug_fault_tx(uint32_t bytes);
// What a step batch needs to know about an agent set (agents.cpp).
struct AgentsView {
    int device;
    const hsr_scene *const *scenes;
    uint32_t n_scenes;
    const uint32_t *scene_of_agent;    // [n_agents]
    uint32_t n_agents;
    const AgentsDev *dev;              // device address
    const hsr_scene_info *info;        // [n_scenes]
};
bool agents_view(const hsr_agents *a, AgentsView &out);

// Mip level l+1 (w2 x h2) of level l (w x h): per channel the rounded mean
// (a + b + c + d + 2) >> 2 of each 2x2 block, block reads clamped to level l.
cudaError_t launch_mip_down(const uint32_t *src, uint32_t w, uint32_t h, uint32_t *dst, uint32_t w2, uint32_t h2,
                            cudaStream_t stream);

// Actuation pass of a step batch: applies each view's action to its agent
// state and writes the view's camera (n_cap: capacity, the grid size).
cudaError_t launch_actuate(const Params &p, uint32_t n_cap, cudaStream_t stream);

// Stage timing (diagnostic): events around cull / raster / shade.
cudaError_t stage_timing_enable(bool on);
cudaError_t stage_timing_read(float ms[4]);

// Diagnostic counters of the last render call (null when disabled).
uint32_t *stage_stats_buffer();
cudaError_t stage_stats_enable(bool on);
cudaError_t stage_stats_read(uint32_t out[6]);

}  // namespace hsr
