// K3 — binning of scene geometry to views (hierarchical frustum culling).
//
// Work is (view, meshlet group) items. A group (32 meshlets) and then each of
// its meshlets (<= 32 triangles) is tested against the view's six frustum
// planes: the four image borders pushed out by two pixels, the near and the
// far plane. Planes are built on the host in double precision and boxes are
// inflated at load, so the test is conservative: geometry that could put a
// sample on screen is never dropped. Surviving (view, meshlet) pairs form a
// compact list; the per-triangle pixel range then bins each triangle to its
// pixels exactly.
#pragma once
#include "../hsr_internal.h"

namespace hsr {

// False when the box lies entirely on the outer side of one plane
// (plane k: n . p + off >= 0 inside; stored as planes[4k .. 4k+3]).
__device__ __forceinline__ bool aabb_visible(const float *pl, const float *bmin, const float *bmax)
{
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const float nx = pl[4 * k], ny = pl[4 * k + 1], nz = pl[4 * k + 2], off = pl[4 * k + 3];
        const float x = nx >= 0.f ? bmax[0] : bmin[0];
        const float y = ny >= 0.f ? bmax[1] : bmin[1];
        const float z = nz >= 0.f ? bmax[2] : bmin[2];
        if (__fmaf_rn(nx, x, __fmaf_rn(ny, y, __fmaf_rn(nz, z, off))) < 0.f) return false;
    }
    return true;
}

}  // namespace hsr
