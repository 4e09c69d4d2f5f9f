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
//  * other triangles are rasterised by a whole warp, row by row over the
//    candidate samples of conservative per-row spans, int64 edges: queued per
//    warp in shared memory (up to bin_px candidates) or binned in global
//    memory as work items of up to 32 rows for a later pass.
#pragma once
#include "setup.cuh"

namespace hsr {

// A large triangle for the warp queue and the binned pass (64 bytes).
struct alignas(16) BigTri {
    int X0, Y0, X1, Y1, X2, Y2;
    float pa, pb, q0, qlo, qhi;
    uint32_t id;
    unsigned short x0, y0, x1, y1;      // candidate pixel range, clipped to the image
    uint32_t view;                       // z-buffer the triangle belongs to (binned pass)
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

// Coverage of a small triangle (at most 32 candidate pixels, bounding box
// under 2^15 sub-pixels per axis): bit k of the result is candidate k, row
// k / w, column k % w of [x0, x1] x [y0, y1]. Exactness: |X_j - X_i| and
// |P - X_i| are below 2^15 inside the bounding box, so every edge value at a
// candidate sample is below 2^31 in magnitude. The values are evaluated once
// at the first candidate and then stepped (one pixel right: -256 dy, one row
// down: +256 dx) in wrap-around unsigned arithmetic, which is exact wherever
// the true value fits in 32 bits, as it does at every evaluated sample.
__device__ __forceinline__ uint32_t small_coverage(const Tri2D &t, int x0, int x1, int y0, int y1)
{
    const int b0 = edge_bias(t.X1, t.Y1, t.X2, t.Y2);
    const int b1 = edge_bias(t.X2, t.Y2, t.X0, t.Y0);
    const int b2 = edge_bias(t.X0, t.Y0, t.X1, t.Y1);
    const int dx0 = t.X2 - t.X1, dy0 = t.Y2 - t.Y1;
    const int dx1 = t.X0 - t.X2, dy1 = t.Y0 - t.Y2;
    const int dx2 = t.X1 - t.X0, dy2 = t.Y1 - t.Y0;
    const int Px = 256 * x0 + 128, Py = 256 * y0 + 128;
    // biased edge values at the first candidate: inside iff all three >= 0
    uint32_t r0 = (uint32_t)(dx0 * (Py - t.Y1) - dy0 * (Px - t.X1) - b0);
    uint32_t r1 = (uint32_t)(dx1 * (Py - t.Y2) - dy1 * (Px - t.X2) - b1);
    uint32_t r2 = (uint32_t)(dx2 * (Py - t.Y0) - dy2 * (Px - t.X0) - b2);
    const uint32_t sx0 = 256u * (uint32_t)dy0, sx1 = 256u * (uint32_t)dy1, sx2 = 256u * (uint32_t)dy2;
    const uint32_t sy0 = 256u * (uint32_t)dx0, sy1 = 256u * (uint32_t)dx1, sy2 = 256u * (uint32_t)dx2;
    const int w = x1 - x0 + 1;
    uint32_t mask = 0;
    int k = 0;
    for (int py = y0; py <= y1; ++py) {
        uint32_t e0 = r0, e1 = r1, e2 = r2;
        for (int i = 0; i < w; ++i, ++k) {
            if ((int)(e0 | e1 | e2) >= 0) mask |= 1u << k;
            e0 -= sx0;
            e1 -= sx1;
            e2 -= sx2;
        }
        r0 += sy0;
        r1 += sy1;
        r2 += sy2;
    }
    return mask;
}

// Position of the k-th (from 0) set bit of m, k < popcount(m): binary search
// on the popcounts of the low halves.
__device__ __forceinline__ int select_bit(uint32_t m, uint32_t k)
{
    int pos = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t c = (uint32_t)__popc(m & ((1u << s) - 1u));
        if (k >= c) {
            k -= c;
            m >>= s;
            pos += s;
        }
    }
    return pos;
}

// A small triangle's covered samples and depth plane, held by the lane that
// set it up until the warp rasterises the fragments of all its lanes.
struct SmallFrag {
    uint32_t mask;            // covered candidates (0: nothing to raster)
    int X0, Y0;               // vertex 0 (sub-pixels): origin of the depth plane
    int x0, y0, w;            // candidate rectangle origin and width (pixels)
    float pa, pb, q0, qlo, qhi;
    float rw;                 // 1 / w
    uint32_t id;
};

__device__ __forceinline__ void small_setup(const Tri2D &t, uint32_t id, int x0, int x1, int y0, int y1,
                                            SmallFrag &f)
{
    f.mask = small_coverage(t, x0, x1, y0, y1);
    if (!f.mask) return;
    depth_plane_narrow(t, f.pa, f.pb);
    f.q0 = t.q0;
    f.qlo = tri_qlo(t);
    f.qhi = tri_qhi(t);
    f.X0 = t.X0;
    f.Y0 = t.Y0;
    f.x0 = x0;
    f.y0 = y0;
    f.w = x1 - x0 + 1;
    f.rw = __fdividef(1.0f, (float)f.w);       // within 2 ulp: enough for the row (see below)
    f.id = id;
}

// Covered samples of a lane's own small triangle, merged by that lane: the
// same candidate numbering, plane evaluation, far test and key as the warp
// pass below (used for triangles with at most kDirectFrags covered samples,
// the common case, which the warp pass would otherwise spread one by one).
constexpr int kDirectFrags = 4;
__device__ __forceinline__ void raster_fragments_lane(const SmallFrag &f, float q_far, unsigned long long *zbuf,
                                                      int W)
{
    uint32_t m = f.mask;
#pragma unroll
    for (int i = 0; i < kDirectFrags; i++) {
        if (!m) break;
        const int b = __ffs(m) - 1;
        m &= m - 1u;
        const int row = (int)(((float)b + 0.5f) * f.rw);
        const int px = f.x0 + (b - row * f.w), py = f.y0 + row;
        const float q = plane_q(f.pa, f.pb, f.q0, 256 * px + 128 - f.X0, 256 * py + 128 - f.Y0, f.qlo, f.qhi);
        if (!(q >= q_far)) continue;
        zmin(zbuf + (size_t)py * W + px, depth_key(q, f.id));
    }
}

// Fragments of the small triangles of all lanes, spread over the warp (every
// lane calls it): covered samples are numbered consecutively across lanes
// (warp prefix sum of the mask popcounts), lane i takes fragment base + i,
// finds the lane owning it (binary search of the prefix) and the candidate
// bit (its k-th covered bit), and merges the fragment exactly as a per-lane
// loop would: same plane evaluation, same far test, same key. Row and column
// of candidate bit b < 32 of a rectangle w <= 32 wide: row = floor((b + 1/2)
// / w) computed as (b + 0.5) * rw in fp32 with rw within 2 ulp of 1/w: the
// product is within 2^-17 of (b + 1/2) / w, which is at least 1/(2w) >= 1/64
// away from an integer, so the floor is exact.
__device__ __forceinline__ void raster_fragments_warp(const SmallFrag &f, int lane, float q_far,
                                                      unsigned long long *zbuf, int W)
{
    const uint32_t cnt = (uint32_t)__popc(f.mask);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const uint32_t excl = incl - cnt;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t g = base + (uint32_t)lane;
        int j = 0;                                   // last lane whose range starts at or before g
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            const int c = j + s;
            const uint32_t e = __shfl_sync(0xFFFFFFFFu, excl, c & 31);
            if (c < 32 && e <= g) j = c;
        }
        const uint32_t ej = __shfl_sync(0xFFFFFFFFu, excl, j);
        const uint32_t mj = __shfl_sync(0xFFFFFFFFu, f.mask, j);
        const int X0 = __shfl_sync(0xFFFFFFFFu, f.X0, j), Y0 = __shfl_sync(0xFFFFFFFFu, f.Y0, j);
        const int x0 = __shfl_sync(0xFFFFFFFFu, f.x0, j), y0 = __shfl_sync(0xFFFFFFFFu, f.y0, j);
        const int w = __shfl_sync(0xFFFFFFFFu, f.w, j);
        const float rw = __shfl_sync(0xFFFFFFFFu, f.rw, j);
        const float pa = __shfl_sync(0xFFFFFFFFu, f.pa, j), pb = __shfl_sync(0xFFFFFFFFu, f.pb, j);
        const float q0 = __shfl_sync(0xFFFFFFFFu, f.q0, j);
        const float qlo = __shfl_sync(0xFFFFFFFFu, f.qlo, j), qhi = __shfl_sync(0xFFFFFFFFu, f.qhi, j);
        const uint32_t id = __shfl_sync(0xFFFFFFFFu, f.id, j);
        if (g >= total) continue;
        const int b = select_bit(mj, g - ej);
        if (!((mj >> b) & 1u)) continue;            // never: g lies in lane j's range
        const int row = (int)(((float)b + 0.5f) * rw);
        const int px = x0 + (b - row * w), py = y0 + row;
        const float q = plane_q(pa, pb, q0, 256 * px + 128 - X0, 256 * py + 128 - Y0, qlo, qhi);
        if (!(q >= q_far)) continue;
        zmin(zbuf + (size_t)py * W + px, depth_key(q, id));
    }
}

// One thread, one small triangle (the per-lane form of the two functions
// above, for triangles set up outside the warp's common path).
__device__ __forceinline__ void raster_small(const Tri2D &t, uint32_t id, int x0, int x1, int y0, int y1,
                                             float q_far, unsigned long long *zbuf, int W)
{
    uint32_t mask = small_coverage(t, x0, x1, y0, y1);
    if (!mask) return;
    float pa, pb;
    depth_plane_narrow(t, pa, pb);
    const float qlo = tri_qlo(t), qhi = tri_qhi(t);
    const int w = x1 - x0 + 1;
    // covered samples row by row (bit k of the mask is row k / w, column k % w)
    const uint32_t rowbits = w >= 32 ? 0xFFFFFFFFu : ((1u << w) - 1u);
    for (int py = y0; mask; ++py) {
        uint32_t row = mask & rowbits;
        mask = w >= 32 ? 0u : mask >> w;
        const int Pyr = 256 * py + 128;
        while (row) {
            const int b = __ffs(row) - 1;
            row &= row - 1;
            const int px = x0 + b;
            const float q = plane_q(pa, pb, t.q0, 256 * px + 128 - t.X0, Pyr - t.Y0, qlo, qhi);
            if (!(q >= q_far)) continue;
            zmin(zbuf + (size_t)py * W + px, depth_key(q, id));
        }
    }
}

// int64 -> float with relative error below 2^-22 (magnitude split into two
// 32-bit halves, both converted without cancellation): for conservative
// bounds only.
__device__ __forceinline__ float i64_to_float_rel(long long v)
{
    const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const float f = __fmaf_rn(__uint2float_rn((uint32_t)(a >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)a));
    return v < 0 ? -f : f;
}

// Rows of a large triangle per work item of the binned pass: about 1024
// candidate pixels, at most one row per lane.
__device__ __forceinline__ int big_rows_per_item(int x0, int x1)
{
    return max(1, min(32, 1024 / (x1 - x0 + 1)));
}

// The whole warp, rows [r0, r1] of a large triangle (within its candidate
// rectangle). Lane k bounds the inside columns of row r0 + k; the candidates
// of the 32 rows are then numbered consecutively (warp prefix sum of the row
// lengths) and spread over the lanes 32 at a time, each lane finding its row
// by a binary search of the prefix. Every candidate takes the exact edge test
// and the same fp32 plane and key as the other paths: the row bounds only
// skip columns that cannot be inside, so they never change a result.
//
// Row bounds: with E(j) the biased edge value at column x0 + j, a sample is
// inside an edge iff E(j) = E(0) - 256 dy j >= 0, so the inside columns lie at
// or below E(0) / (256 dy) (dy > 0) or at or above it (dy < 0); dy == 0
// decides the whole row.
//  * narrow triangles (bounding box under 2^15 sub-pixels per axis): every
//    edge value at a candidate fits in int32 (as for small triangles); the
//    quotient is taken in fp32 with relative error below 2^-21 (a correctly
//    rounded conversion and product, and a reciprocal within 2 ulp), under
//    2^-6 of a column where it can fall inside the rectangle (under 2^15
//    columns from its start), and the bound is rounded with a 1/32-column
//    allowance;
//  * others: int64 edge values, the quotient from a conversion with relative
//    error below 2^-19 (under 32 sub-pixels wherever it falls inside the
//    image), widened by a whole column on each side.
__device__ __forceinline__ void raster_rows_warp(const BigTri &t, int r0, int r1, int lane, float q_far,
                                                 unsigned long long *zbuf, int W)
{
    const int Xb[3] = {t.X1, t.X2, t.X0}, Yb[3] = {t.Y1, t.Y2, t.Y0};
    const int dx[3] = {t.X2 - t.X1, t.X0 - t.X2, t.X1 - t.X0};
    const int dy[3] = {t.Y2 - t.Y1, t.Y0 - t.Y2, t.Y1 - t.Y0};
    const int bias[3] = {edge_bias(t.X1, t.Y1, t.X2, t.Y2), edge_bias(t.X2, t.Y2, t.X0, t.Y0),
                         edge_bias(t.X0, t.Y0, t.X1, t.Y1)};
    const int mnx = min(t.X0, min(t.X1, t.X2)), mxx = max(t.X0, max(t.X1, t.X2));
    const int mny = min(t.Y0, min(t.Y1, t.Y2)), mxy = max(t.Y0, max(t.Y1, t.Y2));
    const bool narrow = mxx - mnx < 32768 && mxy - mny < 32768;
    const int Px0 = 256 * (int)t.x0 + 128;
    const float jmax = (float)((int)t.x1 - (int)t.x0);
    float rdy[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        rdy[k] = dy[k] != 0 ? __fdividef(1.0f, __int2float_rn(narrow ? 256 * dy[k] : dy[k])) : 0.f;
    for (int rb = r0; rb <= r1; rb += 32) {
        const int py = rb + lane;
        int xa = 0, len = 0;
        if (py <= r1) {
            const int Py = 256 * py + 128;
            float lo = 0.f, hi = jmax;          // columns, from t.x0
            bool empty = false;
            if (narrow) {
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const int E = dx[k] * (Py - Yb[k]) - dy[k] * (Px0 - Xb[k]) - bias[k];
                    if (dy[k] == 0) {
                        empty |= E < 0;
                    } else {
                        const float lim = __fmul_rn(__int2float_rn(E), rdy[k]);
                        if (dy[k] > 0)
                            hi = fminf(hi, floorf(lim + 0.03125f));
                        else
                            lo = fmaxf(lo, ceilf(lim - 0.03125f));
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const long long c = (long long)dx[k] * (Py - Yb[k]) + (long long)dy[k] * Xb[k] - bias[k];
                    if (dy[k] == 0) {
                        empty |= c < 0;
                    } else {
                        // sample column bound c / dy, as a column index from t.x0
                        const float lim = (__fmul_rn(i64_to_float_rel(c), rdy[k]) - (float)Px0) * (1.0f / 256.0f);
                        if (dy[k] > 0)
                            hi = fminf(hi, floorf(lim) + 1.0f);
                        else
                            lo = fmaxf(lo, ceilf(lim) - 1.0f);
                    }
                }
            }
            if (!empty && lo <= hi) {
                xa = (int)t.x0 + (int)lo;
                len = (int)hi - (int)lo + 1;
            }
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        const int excl = incl - len;
        for (int base = 0; base < total; base += 32) {
            const int g = base + lane;
            int j = 0;                                   // last row whose run starts at or before g
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const int c = j + s;
                const int e = __shfl_sync(0xFFFFFFFFu, excl, c & 31);
                if (c < 32 && e <= g) j = c;
            }
            const int ej = __shfl_sync(0xFFFFFFFFu, excl, j);
            const int xj = __shfl_sync(0xFFFFFFFFu, xa, j);
            if (g >= total) continue;
            const int px = xj + (g - ej), pyj = rb + j;
            const int Px = 256 * px + 128, Py = 256 * pyj + 128;
            bool inside;
            if (narrow) {
                const int e0 = dx[0] * (Py - t.Y1) - dy[0] * (Px - t.X1);
                const int e1 = dx[1] * (Py - t.Y2) - dy[1] * (Px - t.X2);
                const int e2 = dx[2] * (Py - t.Y0) - dy[2] * (Px - t.X0);
                inside = ((e0 - bias[0]) | (e1 - bias[1]) | (e2 - bias[2])) >= 0;
            } else {
                const long long e0 = (long long)dx[0] * (Py - t.Y1) - (long long)dy[0] * (Px - t.X1);
                const long long e1 = (long long)dx[1] * (Py - t.Y2) - (long long)dy[1] * (Px - t.X2);
                const long long e2 = (long long)dx[2] * (Py - t.Y0) - (long long)dy[2] * (Px - t.X0);
                inside = ((e0 - bias[0]) | (e1 - bias[1]) | (e2 - bias[2])) >= 0;
            }
            if (!inside) continue;
            const float q = plane_q(t.pa, t.pb, t.q0, Px - t.X0, Py - t.Y0, t.qlo, t.qhi);
            if (!(q >= q_far)) continue;
            zmin(zbuf + (size_t)pyj * W + px, depth_key(q, t.id));
        }
    }
}

// The whole warp, one queued triangle.
__device__ __forceinline__ void raster_big_warp(const BigTri &t, int lane, float q_far, unsigned long long *zbuf,
                                                int W)
{
    raster_rows_warp(t, (int)t.y0, (int)t.y1, lane, q_far, zbuf, W);
}

}  // namespace hsr
