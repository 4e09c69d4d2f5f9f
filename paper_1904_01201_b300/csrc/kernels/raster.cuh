// K4 — fixed-point edge-function rasteriser with an order-independent
// 64-bit z-buffer per view.
//
// Coverage (reading; the paper's OpenGL rasteriser is not specified): sample
// at pixel centres (256x+128, 256y+128) in 24.8 fixed point; E_k for the edge
// opposite vertex k is exact in integers; a sample is inside when every
// E_k > 0, or E_k == 0 on a top or left edge. The depth test keeps, per pixel,
// the minimum key (~bits(q) << 32 | triangle index): largest inverse depth q
// first, lower triangle index on ties. The key is a total order, so the
// result does not depend on the order fragments arrive in; each fragment is
// merged with one 64-bit atomic minimum (a fire-and-forget reduction in L2).
//
// Two paths:
//  * small triangles (<= small_px <= 32 candidate pixels, bounding box under 2^15
//    sub-pixels per axis so every edge value fits in int32): one thread walks
//    its own triangle's pixels;
//  * other triangles are queued per warp in shared memory and rasterised by
//    the whole warp, lanes spread over an 8x4 pixel footprint, int64 edges.
#pragma once
#include "setup.cuh"

namespace hsr {

// A large triangle for the warp-cooperative and tile-bin paths (64 bytes).
struct alignas(16) BigTri {
    int X0, Y0, X1, Y1, X2, Y2;
    float pa, pb, q0, qlo, qhi;
    uint32_t id;
    unsigned short x0, y0, x1, y1;      // candidate pixel range, clipped to the image
    uint32_t view;                       // z-buffer the triangle belongs to (tile-bin path)
    uint32_t pad_;
};

__device__ __forceinline__ unsigned long long depth_key(float q, uint32_t id)
{
    return ((unsigned long long)(~__float_as_uint(q)) << 32) | id;
}

__device__ __forceinline__ void zmin(unsigned long long *z, unsigned long long key)
{
    atomicMin(z, key);
}

// One thread, one small triangle (at most 32 candidate pixels). Coverage is
// found first; the depth plane (two divisions) is only built when at least
// one sample is covered. Exactness: |X_j - X_i| and |P - X_i| are below 2^15
// inside the bounding box, so every product is below 2^30 and every edge
// value below 2^31.
__device__ __forceinline__ void raster_small(const Tri2D &t, uint32_t id, int x0, int x1, int y0, int y1,
                                             float q_far, unsigned long long *zbuf, int W)
{
    const int b0 = edge_bias(t.X1, t.Y1, t.X2, t.Y2);
    const int b1 = edge_bias(t.X2, t.Y2, t.X0, t.Y0);
    const int b2 = edge_bias(t.X0, t.Y0, t.X1, t.Y1);
    const int dx0 = t.X2 - t.X1, dy0 = t.Y2 - t.Y1;
    const int dx1 = t.X0 - t.X2, dy1 = t.Y0 - t.Y2;
    const int dx2 = t.X1 - t.X0, dy2 = t.Y1 - t.Y0;
    const int w = x1 - x0 + 1;
    uint32_t mask = 0;
    int k = 0;
    for (int py = y0; py <= y1; ++py) {
        const int Py = 256 * py + 128;
        for (int px = x0; px <= x1; ++px, ++k) {
            const int Px = 256 * px + 128;
            const int e0 = dx0 * (Py - t.Y1) - dy0 * (Px - t.X1);
            const int e1 = dx1 * (Py - t.Y2) - dy1 * (Px - t.X2);
            const int e2 = dx2 * (Py - t.Y0) - dy2 * (Px - t.X0);
            if (((e0 - b0) | (e1 - b1) | (e2 - b2)) >= 0) mask |= 1u << k;
        }
    }
    if (!mask) return;
    float pa, pb;
    depth_plane(t, pa, pb);
    const float qlo = tri_qlo(t), qhi = tri_qhi(t);
    while (mask) {
        const int b = __ffs(mask) - 1;
        mask &= mask - 1;
        const int px = x0 + b % w, py = y0 + b / w;
        const int Px = 256 * px + 128, Py = 256 * py + 128;
        const float q = plane_q(pa, pb, t.q0, Px - t.X0, Py - t.Y0, qlo, qhi);
        if (!(q >= q_far)) continue;
        zmin(zbuf + (size_t)py * W + px, depth_key(q, id));
    }
}

// The whole warp, one 8x8 tile of a binned triangle: lane (lx, ly) covers
// pixels (lx, ly) and (lx, ly + 4) of the tile, int64 edges.
__device__ __forceinline__ void raster_tile_warp(const BigTri &t, int tx, int ty, int lane, float q_far,
                                                 unsigned long long *zbuf, int W)
{
    const int b0 = edge_bias(t.X1, t.Y1, t.X2, t.Y2);
    const int b1 = edge_bias(t.X2, t.Y2, t.X0, t.Y0);
    const int b2 = edge_bias(t.X0, t.Y0, t.X1, t.Y1);
    const int dx0 = t.X2 - t.X1, dy0 = t.Y2 - t.Y1;
    const int dx1 = t.X0 - t.X2, dy1 = t.Y0 - t.Y2;
    const int dx2 = t.X1 - t.X0, dy2 = t.Y1 - t.Y0;
    const int px = tx * 8 + (lane & 7);
    if (px < (int)t.x0 || px > (int)t.x1) return;
    const int Px = 256 * px + 128;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int py = ty * 8 + (lane >> 3) + 4 * h;
        if (py < (int)t.y0 || py > (int)t.y1) continue;
        const int Py = 256 * py + 128;
        const long long e0 = (long long)dx0 * (Py - t.Y1) - (long long)dy0 * (Px - t.X1);
        const long long e1 = (long long)dx1 * (Py - t.Y2) - (long long)dy1 * (Px - t.X2);
        const long long e2 = (long long)dx2 * (Py - t.Y0) - (long long)dy2 * (Px - t.X0);
        if (((e0 - b0) | (e1 - b1) | (e2 - b2)) < 0) continue;
        const float q = plane_q(t.pa, t.pb, t.q0, Px - t.X0, Py - t.Y0, t.qlo, t.qhi);
        if (!(q >= q_far)) continue;
        zmin(zbuf + (size_t)py * W + px, depth_key(q, t.id));
    }
}

// The whole warp, one queued triangle.
__device__ __forceinline__ void raster_big_warp(const BigTri &t, int lane, float q_far, unsigned long long *zbuf,
                                                int W)
{
    const int b0 = edge_bias(t.X1, t.Y1, t.X2, t.Y2);
    const int b1 = edge_bias(t.X2, t.Y2, t.X0, t.Y0);
    const int b2 = edge_bias(t.X0, t.Y0, t.X1, t.Y1);
    const int dx0 = t.X2 - t.X1, dy0 = t.Y2 - t.Y1;
    const int dx1 = t.X0 - t.X2, dy1 = t.Y0 - t.Y2;
    const int dx2 = t.X1 - t.X0, dy2 = t.Y1 - t.Y0;
    const int lx = lane & 7, ly = lane >> 3;
    for (int py = (int)t.y0 + ly; py <= (int)t.y1; py += 4) {
        const int Py = 256 * py + 128;
        for (int px = (int)t.x0 + lx; px <= (int)t.x1; px += 8) {
            const int Px = 256 * px + 128;
            const long long e0 = (long long)dx0 * (Py - t.Y1) - (long long)dy0 * (Px - t.X1);
            const long long e1 = (long long)dx1 * (Py - t.Y2) - (long long)dy1 * (Px - t.X2);
            const long long e2 = (long long)dx2 * (Py - t.Y0) - (long long)dy2 * (Px - t.X0);
            if (((e0 - b0) | (e1 - b1) | (e2 - b2)) < 0) continue;
            const float q = plane_q(t.pa, t.pb, t.q0, Px - t.X0, Py - t.Y0, t.qlo, t.qhi);
            if (!(q >= q_far)) continue;
            zmin(zbuf + (size_t)py * W + px, depth_key(q, t.id));
        }
    }
}

}  // namespace hsr
