// Internal layout shared by the host library (api.cpp) and the kernels (render.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hsr {

// Meshlets: up to 32 triangles and 64 distinct vertices, spatially coherent
// (Morton order of triangle centroids). Groups: 32 consecutive meshlets.
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
    const float2 *uv;          // per vertex, or null
    const uint32_t *vrgb;      // r | g << 8 | b << 16 per vertex, or null
    const uint32_t *atlas;     // RGBA8 texels, row-major, or null
    uint32_t atlas_w, atlas_h;
    uint32_t n_groups, n_meshlets, n_tris, n_verts;
    int color_mode;
    int pad_;
};

// One rendered view: world-to-eye matrix (rows of a 3x4), its scene and the
// output frame it writes.
struct alignas(16) View {
    float M[12];
    uint32_t scene;
    uint32_t frame;
    uint32_t pad_[2];
};

struct Params {
    const SceneDev *scenes;    // device array
    const View *views;         // device array, n_views
    uint8_t *rgb;
    float *depth;
    uint32_t *ids;             // may be null
    uint32_t *work_counter;    // persistent mode: items past gridDim.x; null: one item per CTA
    uint32_t n_views, width, height;
    float fx, fy, cx, cy, znear, zfar;
    float q_far;               // smallest float q with 1/q <= zfar
    uint32_t region_w, region_h, regions_x, regions_y;
    uint32_t n_items;          // n_views * regions_x * regions_y
    uint32_t small_px;         // per-thread raster when a triangle has at most this many candidate pixels
};

// Launch configuration chosen by the host (autotuned).
struct LaunchCfg {
    uint32_t region_w = 64, region_h = 64;
    uint32_t small_px = 16;
    uint32_t ctas_per_sm = 2;
    bool persistent = true;
};

// Launches the fused render kernel; returns a cudaError_t.
cudaError_t launch_render(const Params &p, const LaunchCfg &cfg, cudaStream_t stream);
size_t render_smem_bytes(const LaunchCfg &cfg);

}  // namespace hsr
