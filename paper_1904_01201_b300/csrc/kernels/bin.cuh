// K3 — binning of scene geometry to screen regions.
//
// A CTA owns one (view, screen region). Geometry reaches it through a two-level
// hierarchy (groups of 32 meshlets, meshlets of <= 32 triangles) tested against
// the region's frustum: six world-space planes through the region's pixel
// rectangle expanded by kRegionMarginPx pixels, the near plane and the far
// plane. The test is conservative (expanded planes, inflated bounding boxes),
// so a triangle that could put a sample in the region is never dropped; the
// per-triangle pixel range then bins what survives to the region's pixels
// exactly. Visible meshlets of a chunk of groups are appended to a
// shared-memory queue that the CTA's warps drain.
#pragma once
#include "../hsr_internal.h"

namespace hsr {

constexpr float kRegionMarginPx = 2.0f;
constexpr float kDepthMargin = 1e-4f;     // metres

struct Plane {
    float nx, ny, nz, off;      // inside: n . p + off >= 0 (world space)
};

// Plane k of the region frustum in world space. Eye-space inequalities
// (d = -z_e > 0):  sx >= rx0 - m, sx <= rx1 + m, sy >= ry0 - m, sy <= ry1 + m,
// d >= near, d <= far; each written as n_e . p_e + o_e >= 0 and moved to the
// world through p_e = M [p; 1].
__device__ __forceinline__ Plane region_plane(int k, const float *M, const Params &p, int rx0, int ry0,
                                              int rx1, int ry1)
{
    const float m = kRegionMarginPx;
    float ne[3] = {0.f, 0.f, 0.f}, oe = 0.f;
    switch (k) {
        case 0: ne[0] = p.fx; ne[2] = -(p.cx - ((float)rx0 - m)); break;            // left
        case 1: ne[0] = -p.fx; ne[2] = -(((float)rx1 + m) - p.cx); break;           // right
        case 2: ne[1] = -p.fy; ne[2] = -(p.cy - ((float)ry0 - m)); break;           // top
        case 3: ne[1] = p.fy; ne[2] = -(((float)ry1 + m) - p.cy); break;            // bottom
        case 4: ne[2] = -1.f; oe = -(p.znear - kDepthMargin); break;               // near
        default: ne[2] = 1.f; oe = p.zfar + kDepthMargin; break;                   // far
    }
    Plane w;
    w.nx = M[0] * ne[0] + M[4] * ne[1] + M[8] * ne[2];
    w.ny = M[1] * ne[0] + M[5] * ne[1] + M[9] * ne[2];
    w.nz = M[2] * ne[0] + M[6] * ne[1] + M[10] * ne[2];
    w.off = M[3] * ne[0] + M[7] * ne[1] + M[11] * ne[2] + oe;
    return w;
}

// False when the box lies entirely on the outer side of one plane.
__device__ __forceinline__ bool aabb_visible(const Plane *pl, const float *bmin, const float *bmax)
{
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const Plane P = pl[k];
        const float x = P.nx >= 0.f ? bmax[0] : bmin[0];
        const float y = P.ny >= 0.f ? bmax[1] : bmin[1];
        const float z = P.nz >= 0.f ? bmax[2] : bmin[2];
        if (P.nx * x + P.ny * y + P.nz * z + P.off < 0.f) return false;
    }
    return true;
}

}  // namespace hsr
