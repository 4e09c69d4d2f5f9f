// K2 — triangle setup: trivial reject, near-plane clip, back-face / degenerate
// cull, orientation, depth plane, and the candidate pixel range.
//
// Rules (readings; the paper renders through OpenGL and states none):
//  * reject when all three d < near or all three d > far;
//  * Sutherland-Hodgman clip against d >= near; an edge's endpoints are taken
//    in ascending caller vertex index so shared edges clip to identical points;
//    t = (near - d_a)/(d_b - d_a), p = fma(t, p_b - p_a, p_a), d := near;
//    fan triangulation from the first emitted vertex;
//  * A = (X1-X0)(Y2-Y0) - (Y1-Y0)(X2-X0) in int64; keep A < 0 (front faces are
//    counter-clockwise in the world; screen y points down), then swap 1 and 2;
//  * depth plane of q = 1/d relative to vertex 0 (fixed fp32 op order),
//    clamped to the vertices' range of q;
//  * candidate pixels: centres (256x+128, 256y+128) inside the bounding box.
#pragma once
#include "transform.cuh"

namespace hsr {

// Vertex entering the near clip. NA attributes travel with it (0 in raster,
// 2 (u,v) or 3 (r,g,b) when shading).
template <int NA>
struct CVert {
    float xe, ye, d;
    uint32_t gid;
    float a[NA > 0 ? NA : 1];
};

template <int NA>
__device__ __forceinline__ CVert<NA> clip_edge(const CVert<NA> &p, const CVert<NA> &r, float znear)
{
    const bool swap = r.gid < p.gid;
    const CVert<NA> &a = swap ? r : p;
    const CVert<NA> &b = swap ? p : r;
    const float t = __fdiv_rn(__fsub_rn(znear, a.d), __fsub_rn(b.d, a.d));
    CVert<NA> o;
    o.xe = __fmaf_rn(t, __fsub_rn(b.xe, a.xe), a.xe);
    o.ye = __fmaf_rn(t, __fsub_rn(b.ye, a.ye), a.ye);
    o.d = znear;
    o.gid = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < NA; k++) o.a[k] = __fmaf_rn(t, __fsub_rn(b.a[k], a.a[k]), a.a[k]);
    return o;
}

// Clip a (canonically ordered) triangle with at least one vertex in front of
// the near plane; returns the polygon size (3 or 4).
template <int NA>
__device__ __forceinline__ int clip_near(const CVert<NA> (&v)[3], float znear, CVert<NA> (&out)[4])
{
    int n = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const CVert<NA> &a = v[k];
        const CVert<NA> &b = v[k == 2 ? 0 : k + 1];
        const bool ain = a.d >= znear, bin = b.d >= znear;
        if (ain) out[n++] = a;
        if (ain != bin) out[n++] = clip_edge<NA>(a, b, znear);
    }
    return n;
}

// Fan sub-triangles of a clipped polygon (near plane or guard band) take the
// vertex of smallest q as the origin of their depth plane (the first such on
// ties, in oriented order): the cyclic rotation that puts it first. Their
// other vertices can sit at q = 1/near or far outside the image, where a
// plane referenced at them loses the on-screen depth to cancellation.
__device__ __forceinline__ int min_q_rotation(float q0, float q1, float q2)
{
    return (q1 < q0 && q1 <= q2) ? 1 : ((q2 < q0 && q2 < q1) ? 2 : 0);
}

// A front-facing triangle in oriented (positive-area) order.
struct Tri2D {
    int X0, Y0, X1, Y1, X2, Y2;
    float q0, q1, q2;
    long long A;           // oriented doubled area, > 0
};

// Back-face / degenerate cull and orientation. Returns false when culled.
// Vertex order in: as produced by the clip / fan; out: vertices 1 and 2 swapped.
__device__ __forceinline__ bool orient_cull(int X0, int Y0, float q0, int X1, int Y1, float q1, int X2,
                                            int Y2, float q2, Tri2D &t)
{
    const long long A = (long long)(X1 - X0) * (long long)(Y2 - Y0) - (long long)(Y1 - Y0) * (long long)(X2 - X0);
    if (A >= 0) return false;
    t.X0 = X0; t.Y0 = Y0; t.q0 = q0;
    t.X1 = X2; t.Y1 = Y2; t.q1 = q2;
    t.X2 = X1; t.Y2 = Y1; t.q2 = q1;
    t.A = -A;
    return true;
}

// Orientation of fan sub-triangle (0, f+1, f+2) of a clipped polygon: false
// when culled; else its vertex indices in oriented order, rotated to the
// min-q origin, and the triangle.
__device__ __forceinline__ bool clipped_fan_tri(const int *X, const int *Y, const float *q, int f, int (&ix)[3],
                                                Tri2D &t)
{
    const int i1 = f + 1, i2 = f + 2;
    const long long A = (long long)(X[i1] - X[0]) * (long long)(Y[i2] - Y[0]) -
                        (long long)(Y[i1] - Y[0]) * (long long)(X[i2] - X[0]);
    if (A >= 0) return false;
    const int o[3] = {0, i2, i1};
    const int r = min_q_rotation(q[o[0]], q[o[1]], q[o[2]]);
    ix[0] = o[r];
    ix[1] = o[r == 2 ? 0 : r + 1];
    ix[2] = o[r == 0 ? 2 : r - 1];
    t.X0 = X[ix[0]]; t.Y0 = Y[ix[0]]; t.q0 = q[ix[0]];
    t.X1 = X[ix[1]]; t.Y1 = Y[ix[1]]; t.q1 = q[ix[1]];
    t.X2 = X[ix[2]]; t.Y2 = Y[ix[2]]; t.q2 = q[ix[2]];
    t.A = -A;
    return true;
}

// Guard band (reading; the paper states no rasterisation rule): a
// (near-clipped) polygon with a snapped coordinate at or beyond +-2^30
// sub-pixels is clipped, Sutherland-Hodgman, against the eye-space planes
// x_e >= -gx d, x_e <= gx d, y_e >= -gy d, y_e <= gy d in that order
// (gx = 2^21 / fx, gy = 2^21 / fy: 2^29 sub-pixels either side of the
// principal point). Plane distances are fma(g, d, +-x); a crossing edge is
// cut from its endpoint b nearer the cut (the inside one when
// s_in <= -s_out, else the outside one): t = s_b / (s_b - s_r),
// p = fma(t, p_r - p_b, p_b) for x, y, d and the attributes. The choice
// depends only on the edge's two endpoints, so the two triangles sharing an
// edge cut it at the same point, and no cut is computed against a far
// endpoint's rounding. Out of line: few triangles ever take it.
constexpr int kMaxClipVerts = 8;

// A near-clipped polygon passed by value to the out-of-line guard-band
// functions (their callers keep no hot state in memory for them).
template <int NA>
struct ClipPoly {
    CVert<NA> v[4];
    int n;
};

// The camera constants the guard band needs, by value (a kernel's parameter
// block passed by reference to an out-of-line function would be copied to
// local memory in every thread).
struct GuardCam {
    float gx, gy, fx, fy, cx, cy;
};

template <int NA>
__device__ __forceinline__ int clip_guard(const ClipPoly<NA> &in, float gx, float gy, CVert<NA> (&out)[kMaxClipVerts])
{
    CVert<NA> a[kMaxClipVerts], b[kMaxClipVerts];
    int na = in.n;
    for (int k = 0; k < in.n; k++) a[k] = in.v[k];
    for (int pl = 0; pl < 4; pl++) {
        const float g = pl < 2 ? gx : gy;
        float dist[kMaxClipVerts];
        for (int k = 0; k < na; k++) {
            const float c = pl < 2 ? a[k].xe : a[k].ye;
            dist[k] = __fmaf_rn(g, a[k].d, (pl & 1) ? -c : c);
        }
        int nb = 0;
        for (int k = 0; k < na; k++) {
            const int k1 = k + 1 == na ? 0 : k + 1;
            const bool ain = dist[k] >= 0.f, bin = dist[k1] >= 0.f;
            if (ain) b[nb++] = a[k];
            if (ain != bin) {
                const int ii = ain ? k : k1, io = ain ? k1 : k;
                const bool from_in = dist[ii] <= -dist[io];
                const CVert<NA> &pb = a[from_in ? ii : io];
                const CVert<NA> &pr = a[from_in ? io : ii];
                const float sb = dist[from_in ? ii : io], sr = dist[from_in ? io : ii];
                const float t = __fdiv_rn(sb, __fsub_rn(sb, sr));
                CVert<NA> o;
                o.xe = __fmaf_rn(t, __fsub_rn(pr.xe, pb.xe), pb.xe);
                o.ye = __fmaf_rn(t, __fsub_rn(pr.ye, pb.ye), pb.ye);
                o.d = __fmaf_rn(t, __fsub_rn(pr.d, pb.d), pb.d);
                o.gid = 0xFFFFFFFFu;
#pragma unroll
                for (int c = 0; c < NA; c++) o.a[c] = __fmaf_rn(t, __fsub_rn(pr.a[c], pb.a[c]), pb.a[c]);
                b[nb++] = o;
            }
        }
        na = nb;
        for (int k = 0; k < na; k++) a[k] = b[k];
        if (na == 0) break;
    }
    for (int k = 0; k < na; k++) out[k] = a[k];
    return na;
}

// Guard clip, projection and the oriented, min-q-rotated fan of a clipped
// polygon: writes up to 6 sub-triangles to out (their vertex indices into
// the clipped polygon to ix when non-null) and returns their count, or -1
// if a clipped vertex still leaves the fixed-point range (not reachable
// within the documented input limits). Out of line: few triangles take it.
template <int NA>
__device__ __noinline__ int guard_fan(const ClipPoly<NA> poly, const GuardCam cam, Tri2D *out,
                                      CVert<NA> *gout)
{
    CVert<NA> g[kMaxClipVerts];
    const int ng = clip_guard<NA>(poly, cam.gx, cam.gy, g);
    int X[kMaxClipVerts], Y[kMaxClipVerts];
    float q[kMaxClipVerts];
    bool in_range = true;
    for (int k = 0; k < ng; k++)
        in_range &= project_snap(g[k].xe, g[k].ye, g[k].d, cam.fx, cam.fy, cam.cx, cam.cy, q[k], X[k], Y[k]);
    if (!in_range) return -1;
    int m = 0;
    for (int f = 0; f + 2 < ng; f++) {
        int ix[3];
        Tri2D t;
        if (!clipped_fan_tri(X, Y, q, f, ix, t)) continue;
        out[m] = t;
        if (gout) {
            gout[3 * m] = g[ix[0]];
            gout[3 * m + 1] = g[ix[1]];
            gout[3 * m + 2] = g[ix[2]];
        }
        m++;
    }
    return m;
}

// Plane of q over the snapped vertices, relative to vertex 0:
//   a = fma(dq1, Y2-Y0, -(dq2*(Y1-Y0))) / A,  b = fma(dq2, X1-X0, -(dq1*(X2-X0))) / A.
// int64 -> float rounded to nearest, ties to even (the result of
// __ll2float_rn) in integer arithmetic: the leading 24 significant bits, the
// discarded bits decide the rounding, and the scale by 2^shift is exact. The
// 64-bit conversion instruction runs on a slow unit of this part.
__device__ __forceinline__ float i64_to_float_rn(long long v)
{
    const bool neg = v < 0;
    const unsigned long long a = neg ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int top = 63 - __clzll((long long)(a | 1ull));          // index of the leading bit
    const int sh = max(top - 23, 0);                                // bits that do not fit a float
    unsigned long long m = a >> sh;
    const unsigned long long rem = a & ((1ull << sh) - 1ull);
    const unsigned long long half = sh > 0 ? 1ull << (sh - 1) : 0ull;
    if (sh > 0 && (rem > half || (rem == half && (m & 1ull)))) m++;
    const float f = __fmul_rn(__uint2float_rn((uint32_t)m), __int_as_float((sh + 127) << 23));
    return neg ? -f : f;
}

// int64 -> float within 3 units in the last place (two 32-bit conversions):
// for shading weights, which tolerate it.
__device__ __forceinline__ float i64_to_float_approx(long long v)
{
    return __fmaf_rn(__int2float_rn((int)(v >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)v));
}

__device__ __forceinline__ void depth_plane(const Tri2D &t, float &pa, float &pb)
{
    const float fA = i64_to_float_rn(t.A);
    const float dq1 = __fsub_rn(t.q1, t.q0), dq2 = __fsub_rn(t.q2, t.q0);
    pa = __fdiv_rn(__fmaf_rn(dq1, __int2float_rn(t.Y2 - t.Y0), -__fmul_rn(dq2, __int2float_rn(t.Y1 - t.Y0))), fA);
    pb = __fdiv_rn(__fmaf_rn(dq2, __int2float_rn(t.X1 - t.X0), -__fmul_rn(dq1, __int2float_rn(t.X2 - t.X0))), fA);
}

// depth_plane for a triangle whose bounding box is under 2^15 sub-pixels per
// axis: each product of A is below 2^30 in magnitude, so 0 < A < 2^31 and the
// int32 conversion gives the same rounded float as i64_to_float_rn.
__device__ __forceinline__ void depth_plane_narrow(const Tri2D &t, float &pa, float &pb)
{
    const float fA = __int2float_rn((int)t.A);
    const float dq1 = __fsub_rn(t.q1, t.q0), dq2 = __fsub_rn(t.q2, t.q0);
    pa = __fdiv_rn(__fmaf_rn(dq1, __int2float_rn(t.Y2 - t.Y0), -__fmul_rn(dq2, __int2float_rn(t.Y1 - t.Y0))), fA);
    pb = __fdiv_rn(__fmaf_rn(dq2, __int2float_rn(t.X1 - t.X0), -__fmul_rn(dq1, __int2float_rn(t.X2 - t.X0))), fA);
}

// q at a sample, from its offset (exact integers) to vertex 0, clamped to the
// range [qlo, qhi] of the triangle's vertex values (interior points lie
// between the vertices' depths; the clamp keeps that true under rounding).
__device__ __forceinline__ float plane_q(float pa, float pb, float q0, int dx, int dy, float qlo, float qhi)
{
    const float q = __fmaf_rn(pa, __int2float_rn(dx), __fmaf_rn(pb, __int2float_rn(dy), q0));
    return fminf(fmaxf(q, qlo), qhi);
}

__device__ __forceinline__ float tri_qlo(const Tri2D &t) { return fminf(t.q0, fminf(t.q1, t.q2)); }
__device__ __forceinline__ float tri_qhi(const Tri2D &t) { return fmaxf(t.q0, fmaxf(t.q1, t.q2)); }

// Top-left bias of edge i->j: 0 if the edge is top (dy == 0, dx > 0) or left
// (dy < 0), else 1 (a sample exactly on it is outside).
__device__ __forceinline__ int edge_bias(int Xi, int Yi, int Xj, int Yj)
{
    const int dy = Yj - Yi, dx = Xj - Xi;
    return (dy < 0 || (dy == 0 && dx > 0)) ? 0 : 1;
}

// Candidate pixel range of the bounding box: centres 256x+128 in [min, max].
__device__ __forceinline__ void pixel_range(const Tri2D &t, int &x0, int &x1, int &y0, int &y1, int &spanx,
                                            int &spany)
{
    const int mnx = min(t.X0, min(t.X1, t.X2)), mxx = max(t.X0, max(t.X1, t.X2));
    const int mny = min(t.Y0, min(t.Y1, t.Y2)), mxy = max(t.Y0, max(t.Y1, t.Y2));
    x0 = (mnx + 127) >> 8;     // ceil((mnx - 128) / 256)
    x1 = (mxx - 128) >> 8;     // floor((mxx - 128) / 256)
    y0 = (mny + 127) >> 8;
    y1 = (mxy - 128) >> 8;
    spanx = mxx - mnx;
    spany = mxy - mny;
}

}  // namespace hsr
