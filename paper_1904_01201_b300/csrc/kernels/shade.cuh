// K5 — resolve and shade (deferred): each pixel's winning key names the
// triangle and its inverse depth; the triangle's setup is rebuilt exactly as
// the rasteriser built it, and the three sensor outputs of the single pass are
// produced (Sec. 3 "Rendering engine": colour, depth and semantic outputs
// together).
//
// Readings: perspective-correct weights w_k = E_k(P) * q_k normalised;
// texture lookups are bilinear, clamp-to-edge, at (u*Wt - 0.5, v*Ht - 0.5)
// with atlas row 0 at v = 0; channels round half up and saturate at 255;
// depth = 1/q; background is RGB 0, depth 0, id 0xFFFFFFFF.
#pragma once
#include "raster.cuh"

namespace hsr {

constexpr uint32_t kBackgroundId = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t round_channel(float c)
{
    const float r = floorf(__fadd_rn(c, 0.5f));
    return (uint32_t)fminf(fmaxf(r, 0.0f), 255.0f);
}

// Channel c (0..2) of a packed texel as a float, exactly: the byte placed in
// the low mantissa bits of 2^23 (one byte permute), minus 2^23.
__device__ __forceinline__ float texel_channel(uint32_t t, int c)
{
    return __fsub_rn(__uint_as_float(__byte_perm(t, 0x4B000000u, 0x7440u | (uint32_t)c)), 8388608.0f);
}

__device__ __forceinline__ uint32_t sample_bilinear(const SceneDev &S, float u, float v)
{
    const float aw = (float)S.atlas_w, ah = (float)S.atlas_h;
    float s = __fmaf_rn(u, aw, -0.5f), t = __fmaf_rn(v, ah, -0.5f);
    s = fminf(fmaxf(s, -1.0f), aw);
    t = fminf(fmaxf(t, -1.0f), ah);
    const float fs = floorf(s), ft = floorf(t);
    const float ax = __fsub_rn(s, fs), ay = __fsub_rn(t, ft);
    const int ix = (int)fs, iy = (int)ft;
    const float gx = __fsub_rn(1.0f, ax), gy = __fsub_rn(1.0f, ay);
    uint32_t out = 0;
    if (S.atlas_tex) {
        // one gather returns the footprint (ix, iy) .. (ix + 1, iy + 1),
        // clamped to the edge, as four packed texels (the texture has one
        // 32-bit channel): at unnormalised (ix + 1, iy + 1) the footprint's
        // corner is floor(ix + 1/2) = ix, half a texel from any rounding
        // boundary; the texels come as x (ix, iy + 1), y (ix + 1, iy + 1),
        // z (ix + 1, iy), w (ix, iy)
        const uint4 g = tex2Dgather<uint4>((cudaTextureObject_t)S.atlas_tex, (float)(ix + 1), (float)(iy + 1), 0);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float v00 = texel_channel(g.w, c), v10 = texel_channel(g.z, c);
            const float v01 = texel_channel(g.x, c), v11 = texel_channel(g.y, c);
            const float top = __fmaf_rn(ax, v10, __fmul_rn(gx, v00));
            const float bot = __fmaf_rn(ax, v11, __fmul_rn(gx, v01));
            out |= round_channel(__fmaf_rn(ay, bot, __fmul_rn(gy, top))) << (8 * c);
        }
        return out;
    }
    const int W = (int)S.atlas_w, H = (int)S.atlas_h;
    const int x0 = min(max(ix, 0), W - 1), x1 = min(max(ix + 1, 0), W - 1);
    const int y0 = min(max(iy, 0), H - 1), y1 = min(max(iy + 1, 0), H - 1);
    const uint32_t c00 = __ldg(S.atlas + (size_t)y0 * W + x0), c10 = __ldg(S.atlas + (size_t)y0 * W + x1);
    const uint32_t c01 = __ldg(S.atlas + (size_t)y1 * W + x0), c11 = __ldg(S.atlas + (size_t)y1 * W + x1);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float top = __fmaf_rn(ax, texel_channel(c10, c), __fmul_rn(gx, texel_channel(c00, c)));
        const float bot = __fmaf_rn(ax, texel_channel(c11, c), __fmul_rn(gx, texel_channel(c01, c)));
        out |= round_channel(__fmaf_rn(ay, bot, __fmul_rn(gy, top))) << (8 * c);
    }
    return out;
}

// Unrounded bilinear sample (channels 0..2) of mip level l: level 0 is the
// atlas, level l is max(1, W >> l) x max(1, H >> l), same addressing rules.
__device__ __forceinline__ void sample_level(const SceneDev &S, uint32_t l, float u, float v, float (&c)[3])
{
    const uint32_t Wl = max(1u, S.atlas_w >> l), Hl = max(1u, S.atlas_h >> l);
    const uint32_t *img = l == 0 ? S.atlas : S.mips + S.mip_off[l];
    const float aw = (float)Wl, ah = (float)Hl;
    float s = __fmaf_rn(u, aw, -0.5f), t = __fmaf_rn(v, ah, -0.5f);
    s = fminf(fmaxf(s, -1.0f), aw);
    t = fminf(fmaxf(t, -1.0f), ah);
    const float fs = floorf(s), ft = floorf(t);
    const float ax = __fsub_rn(s, fs), ay = __fsub_rn(t, ft);
    const int ix = (int)fs, iy = (int)ft;
    const int W = (int)Wl, H = (int)Hl;
    const int x0 = min(max(ix, 0), W - 1), x1 = min(max(ix + 1, 0), W - 1);
    const int y0 = min(max(iy, 0), H - 1), y1 = min(max(iy + 1, 0), H - 1);
    const uint32_t c00 = __ldg(img + (size_t)y0 * W + x0), c10 = __ldg(img + (size_t)y0 * W + x1);
    const uint32_t c01 = __ldg(img + (size_t)y1 * W + x0), c11 = __ldg(img + (size_t)y1 * W + x1);
    const float gx = __fsub_rn(1.0f, ax), gy = __fsub_rn(1.0f, ay);
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        const float v00 = texel_channel(c00, ch), v10 = texel_channel(c10, ch);
        const float v01 = texel_channel(c01, ch), v11 = texel_channel(c11, ch);
        const float top = __fmaf_rn(ax, v10, __fmul_rn(gx, v00));
        const float bot = __fmaf_rn(ax, v11, __fmul_rn(gx, v01));
        c[ch] = __fmaf_rn(ay, bot, __fmul_rn(gy, top));
    }
}

// Trilinear sample at level of detail lambda: lambda <= 0 is the plain
// bilinear rule; beyond the last level, that level; otherwise the two
// neighbouring levels blended by frac(lambda), then rounded.
__device__ __forceinline__ uint32_t sample_trilinear(const SceneDev &S, float u, float v, float lambda)
{
    if (!(lambda > 0.0f)) return sample_bilinear(S, u, v);
    const uint32_t last = S.n_levels - 1;
    float c[3];
    if (lambda >= (float)last) {
        sample_level(S, last, u, v, c);
    } else {
        const float fl = floorf(lambda);
        const uint32_t l0 = (uint32_t)fl;
        const float f = __fsub_rn(lambda, fl), g = __fsub_rn(1.0f, f);
        float a[3], b[3];
        sample_level(S, l0, u, v, a);
        sample_level(S, l0 + 1, u, v, b);
#pragma unroll
        for (int ch = 0; ch < 3; ch++) c[ch] = __fmaf_rn(f, b[ch], __fmul_rn(g, a[ch]));
    }
    return round_channel(c[0]) | (round_channel(c[1]) << 8) | (round_channel(c[2]) << 16);
}

// Vertices of a triangle with NA attributes, in eye space.
template <int NA>
__device__ __forceinline__ void load_tri(const SceneDev &S, const float *M, const uint4 &T, CVert<NA> (&v)[3])
{
    const uint32_t gi[3] = {T.x, T.y, T.z};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float4 P = __ldg(S.vert + gi[k]);
        eye_transform(M, P.x, P.y, P.z, v[k].xe, v[k].ye, v[k].d);
        v[k].gid = gi[k];
        if (NA == 2) {
            const float2 t = __ldg(S.uv + gi[k]);
            v[k].a[0] = t.x;
            v[k].a[NA > 1 ? 1 : 0] = t.y;
        } else if (NA == 3) {
            const uint32_t c = __ldg(S.vrgb + gi[k]);
            v[k].a[0] = (float)(c & 255u);
            v[k].a[NA > 1 ? 1 : 0] = (float)((c >> 8) & 255u);
            v[k].a[NA > 2 ? 2 : 0] = (float)((c >> 16) & 255u);
        }
    }
}

// Perspective-correct attribute interpolation at P over an oriented triangle
// whose attributes are a0 (vertex 0), a1 (vertex 1), a2 (vertex 2).
// `narrow`: the triangle's bounding box is under 2^15 sub-pixels per axis and
// P lies in it, so every edge value fits in int32 and converts in one step.
template <int NA>
__device__ __forceinline__ void interp(const Tri2D &t, bool narrow, int Px, int Py, const float *a0,
                                       const float *a1, const float *a2, float (&attr)[3])
{
    float f0, f1, f2;
    if (narrow) {
        f0 = __int2float_rn((t.X2 - t.X1) * (Py - t.Y1) - (t.Y2 - t.Y1) * (Px - t.X1));
        f1 = __int2float_rn((t.X0 - t.X2) * (Py - t.Y2) - (t.Y0 - t.Y2) * (Px - t.X2));
        f2 = __int2float_rn((t.X1 - t.X0) * (Py - t.Y0) - (t.Y1 - t.Y0) * (Px - t.X0));
    } else {
        f0 = i64_to_float_approx((long long)(t.X2 - t.X1) * (Py - t.Y1) - (long long)(t.Y2 - t.Y1) * (Px - t.X1));
        f1 = i64_to_float_approx((long long)(t.X0 - t.X2) * (Py - t.Y2) - (long long)(t.Y0 - t.Y2) * (Px - t.X2));
        f2 = i64_to_float_approx((long long)(t.X1 - t.X0) * (Py - t.Y0) - (long long)(t.Y1 - t.Y0) * (Px - t.X0));
    }
    const float w0 = __fmul_rn(f0, t.q0);
    const float w1 = __fmul_rn(f1, t.q1);
    const float w2 = __fmul_rn(f2, t.q2);
    const float r = __fdividef(1.0f, __fadd_rn(__fadd_rn(w0, w1), w2));     // shading tolerates 2 ulp
    const float l0 = __fmul_rn(w0, r), l1 = __fmul_rn(w1, r), l2 = __fmul_rn(w2, r);
#pragma unroll
    for (int c = 0; c < NA; c++) attr[c] = __fmaf_rn(l0, a0[c], __fmaf_rn(l1, a1[c], __fmul_rn(l2, a2[c])));
}

// Level of detail at P of an oriented triangle with uv a0, a1, a2: lambda =
// log2 of the larger texel-space length of the uv derivative along x and
// along y, from the exact derivatives of the perspective-correct weights
// w_k = E_k q_k (one pixel is 256 sub-pixel steps of each edge function).
__device__ __forceinline__ float lod_lambda(uint32_t atlas_w, uint32_t atlas_h, const Tri2D &t, int Px, int Py,
                                            const float *a0, const float *a1, const float *a2)
{
    const long long e0 = (long long)(t.X2 - t.X1) * (Py - t.Y1) - (long long)(t.Y2 - t.Y1) * (Px - t.X1);
    const long long e1 = (long long)(t.X0 - t.X2) * (Py - t.Y2) - (long long)(t.Y0 - t.Y2) * (Px - t.X2);
    const long long e2 = (long long)(t.X1 - t.X0) * (Py - t.Y0) - (long long)(t.Y1 - t.Y0) * (Px - t.X0);
    const float w0 = __fmul_rn(i64_to_float_approx(e0), t.q0);
    const float w1 = __fmul_rn(i64_to_float_approx(e1), t.q1);
    const float w2 = __fmul_rn(i64_to_float_approx(e2), t.q2);
    const float r = __fdividef(1.0f, __fadd_rn(__fadd_rn(w0, w1), w2));
    const float l0 = __fmul_rn(w0, r), l1 = __fmul_rn(w1, r), l2 = __fmul_rn(w2, r);
    const float x0 = __fmul_rn(-256.0f * __int2float_rn(t.Y2 - t.Y1), t.q0);
    const float x1 = __fmul_rn(-256.0f * __int2float_rn(t.Y0 - t.Y2), t.q1);
    const float x2 = __fmul_rn(-256.0f * __int2float_rn(t.Y1 - t.Y0), t.q2);
    const float y0 = __fmul_rn(256.0f * __int2float_rn(t.X2 - t.X1), t.q0);
    const float y1 = __fmul_rn(256.0f * __int2float_rn(t.X0 - t.X2), t.q1);
    const float y2 = __fmul_rn(256.0f * __int2float_rn(t.X1 - t.X0), t.q2);
    const float sx = __fadd_rn(__fadd_rn(x0, x1), x2), sy = __fadd_rn(__fadd_rn(y0, y1), y2);
    const float gx0 = __fmul_rn(__fmaf_rn(-l0, sx, x0), r), gy0 = __fmul_rn(__fmaf_rn(-l0, sy, y0), r);
    const float gx1 = __fmul_rn(__fmaf_rn(-l1, sx, x1), r), gy1 = __fmul_rn(__fmaf_rn(-l1, sy, y1), r);
    const float gx2 = __fmul_rn(__fmaf_rn(-l2, sx, x2), r), gy2 = __fmul_rn(__fmaf_rn(-l2, sy, y2), r);
    const float aw = (float)atlas_w, ah = (float)atlas_h;
    const float ux = __fmul_rn(__fmaf_rn(gx0, a0[0], __fmaf_rn(gx1, a1[0], __fmul_rn(gx2, a2[0]))), aw);
    const float vx = __fmul_rn(__fmaf_rn(gx0, a0[1], __fmaf_rn(gx1, a1[1], __fmul_rn(gx2, a2[1]))), ah);
    const float uy = __fmul_rn(__fmaf_rn(gy0, a0[0], __fmaf_rn(gy1, a1[0], __fmul_rn(gy2, a2[0]))), aw);
    const float vy = __fmul_rn(__fmaf_rn(gy0, a0[1], __fmaf_rn(gy1, a1[1], __fmul_rn(gy2, a2[1]))), ah);
    const float rx = sqrtf(__fmaf_rn(ux, ux, __fmul_rn(vx, vx)));
    const float ry = sqrtf(__fmaf_rn(uy, uy, __fmul_rn(vy, vy)));
    return log2f(fmaxf(rx, ry));
}

// Setup of the last triangle a thread shaded (neighbouring pixels often share it).
template <int NA>
struct ShadeTri {
    uint32_t tri = 0xFFFFFFFFu;
    bool clipped = false;
    bool narrow = false;                // bounding box under 2^15 sub-pixels per axis
    Tri2D t;                            // oriented (unclipped case; t.A is not set)
    float a[3][NA > 0 ? NA : 1];        // attributes in oriented order
    uint32_t id;                        // output id
};

// G: the view may hold winners that need the guard band (a snapped vertex
// at or beyond +-2^30 sub-pixels sends the triangle to the clipping path);
// views without any (flagged by the rasteriser) skip the range test.
template <int NA, bool G>
__device__ __forceinline__ void build_shade_tri(ShadeTri<NA> &st, const SceneDev &S, const float *M,
                                                const Params &p, uint32_t tri)
{
    st.tri = tri;
    // the triangle's shading record: one 64-byte line
    const float4 *rec = S.srec + 4 * (size_t)tri;
    const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r2 = __ldg(rec + 2), r3 = __ldg(rec + 3);
    st.id = __float_as_uint(r3.w);
    const float px[3] = {r0.x, r0.w, r1.z}, py[3] = {r0.y, r1.x, r1.w}, pz[3] = {r0.z, r1.y, r2.x};
    CVert<NA> v[3];
#pragma unroll
    for (int k = 0; k < 3; k++) eye_transform(M, px[k], py[k], pz[k], v[k].xe, v[k].ye, v[k].d);
    if (NA == 2) {
        const float u[3] = {r2.y, r2.w, r3.y}, w[3] = {r2.z, r3.x, r3.z};
#pragma unroll
        for (int k = 0; k < 3; k++) {
            v[k].a[0] = u[k];
            v[k].a[NA > 1 ? 1 : 0] = w[k];
        }
    } else if (NA == 3) {
        const uint32_t c[3] = {__float_as_uint(r2.y), __float_as_uint(r2.z), __float_as_uint(r2.w)};
#pragma unroll
        for (int k = 0; k < 3; k++) {
            v[k].a[0] = (float)(c[k] & 255u);
            v[k].a[NA > 1 ? 1 : 0] = (float)((c[k] >> 8) & 255u);
            v[k].a[NA > 2 ? 2 : 0] = (float)((c[k] >> 16) & 255u);
        }
    }
    st.clipped = !(v[0].d >= p.znear && v[1].d >= p.znear && v[2].d >= p.znear);
    if (st.clipped) return;
    int X[3], Y[3];
    float q[3];
    bool in_range = true;
#pragma unroll
    for (int k = 0; k < 3; k++)
        in_range &= project_snap(v[k].xe, v[k].ye, v[k].d, p.fx, p.fy, p.cx, p.cy, q[k], X[k], Y[k]);
    if (G && !in_range) {      // guard band: the clipping path
        st.clipped = true;
        return;
    }
    // a winning fragment exists, so the triangle is front facing (its area
    // is negative): orient_cull's order, vertices 1 and 2 swapped
    st.t.X0 = X[0]; st.t.Y0 = Y[0]; st.t.q0 = q[0];
    st.t.X1 = X[2]; st.t.Y1 = Y[2]; st.t.q1 = q[2];
    st.t.X2 = X[1]; st.t.Y2 = Y[1]; st.t.q2 = q[1];
    st.narrow = max(X[0], max(X[1], X[2])) - min(X[0], min(X[1], X[2])) < 32768 &&
                max(Y[0], max(Y[1], Y[2])) - min(Y[0], min(Y[1], Y[2])) < 32768;
#pragma unroll
    for (int c = 0; c < NA; c++) {
        st.a[0][c] = v[0].a[c];
        st.a[1][c] = v[2].a[c];
        st.a[2][c] = v[1].a[c];
    }
}

// The fan sub-triangle (0, f+1, f+2) of a near-clipped polygon (at most 4
// vertices: f = 0, 1) that covers P, by the rasteriser's orientation and
// coverage rule: its perspective-correct attributes and level of detail. At
// most one covers P: two front-facing sub-triangles (0, 1, 2) and (0, 2, 3)
// lie on opposite sides of their shared edge 0-2, which the top-left rule
// gives to one of them, so coverage alone names the sub-triangle that
// produced the pixel's fragment.
template <int NA>
__device__ __forceinline__ bool shade_fan(const SceneDev &S, const CVert<NA> (&poly)[4], const int (&X)[4],
                                          const int (&Y)[4], const float (&q)[4], int np, int Px, int Py,
                                          float (&attr)[3], float &lambda)
{
#pragma unroll
    for (int f = 0; f < 2; f++) {
        if (f + 2 >= np) break;
        Tri2D t;
        if (!orient_cull(X[0], Y[0], q[0], X[f + 1], Y[f + 1], q[f + 1], X[f + 2], Y[f + 2], q[f + 2], t)) continue;
        const long long e0 = (long long)(t.X2 - t.X1) * (Py - t.Y1) - (long long)(t.Y2 - t.Y1) * (Px - t.X1);
        const long long e1 = (long long)(t.X0 - t.X2) * (Py - t.Y2) - (long long)(t.Y0 - t.Y2) * (Px - t.X2);
        const long long e2 = (long long)(t.X1 - t.X0) * (Py - t.Y0) - (long long)(t.Y1 - t.Y0) * (Px - t.X0);
        const int b0 = edge_bias(t.X1, t.Y1, t.X2, t.Y2);
        const int b1 = edge_bias(t.X2, t.Y2, t.X0, t.Y0);
        const int b2 = edge_bias(t.X0, t.Y0, t.X1, t.Y1);
        if (((e0 - b0) | (e1 - b1) | (e2 - b2)) < 0) continue;
        // oriented order is (poly 0, poly f+2, poly f+1)
        interp<NA>(t, false, Px, Py, poly[0].a, poly[f + 2].a, poly[f + 1].a, attr);
        if constexpr (NA == 2)
            if (S.sample_mode == HSR_SAMPLE_TRILINEAR)
                lambda = lod_lambda(S.atlas_w, S.atlas_h, t, Px, Py, poly[0].a, poly[f + 2].a, poly[f + 1].a);
        return true;
    }
    return false;
}

// The guard-band search: the fan sub-triangle of the guard-clipped polygon
// (up to six) whose fragment at P has inverse depth qk (the rasteriser's
// coverage and min-q plane), its attributes and level of detail.
template <int NA>
__device__ __forceinline__ bool shade_guard_fan(const SceneDev &S, const ClipPoly<NA> &poly, const GuardCam &cam,
                                                int Px, int Py, float qk, float (&attr)[3], float &lambda)
{
    Tri2D t[kMaxClipVerts - 2];
    CVert<NA> v[3 * (kMaxClipVerts - 2)];
    const int m = guard_fan<NA>(poly, cam, t, v);
    for (int k = 0; k < m; k++) {
        const Tri2D &s = t[k];
        const long long e0 = (long long)(s.X2 - s.X1) * (Py - s.Y1) - (long long)(s.Y2 - s.Y1) * (Px - s.X1);
        const long long e1 = (long long)(s.X0 - s.X2) * (Py - s.Y2) - (long long)(s.Y0 - s.Y2) * (Px - s.X2);
        const long long e2 = (long long)(s.X1 - s.X0) * (Py - s.Y0) - (long long)(s.Y1 - s.Y0) * (Px - s.X0);
        const int b0 = edge_bias(s.X1, s.Y1, s.X2, s.Y2);
        const int b1 = edge_bias(s.X2, s.Y2, s.X0, s.Y0);
        const int b2 = edge_bias(s.X0, s.Y0, s.X1, s.Y1);
        if (((e0 - b0) | (e1 - b1) | (e2 - b2)) < 0) continue;
        float pa, pb;
        depth_plane(s, pa, pb);
        const float qq = plane_q(pa, pb, s.q0, Px - s.X0, Py - s.Y0, tri_qlo(s), tri_qhi(s));
        if (__float_as_uint(qq) != __float_as_uint(qk)) continue;
        interp<NA>(s, false, Px, Py, v[3 * k].a, v[3 * k + 1].a, v[3 * k + 2].a, attr);
        if constexpr (NA == 2)
            if (S.sample_mode == HSR_SAMPLE_TRILINEAR)
                lambda = lod_lambda(S.atlas_w, S.atlas_h, s, Px, Py, v[3 * k].a, v[3 * k + 1].a, v[3 * k + 2].a);
        return true;
    }
    return false;
}

// Clipped triangle: rebuild the near-clipped polygon and find the fan
// sub-triangle that produced P's fragment (inverse depth qk); with G, a
// polygon beyond the fixed-point range is clipped to the guard band first.
template <int NA, bool G>
__device__ __forceinline__ bool shade_clipped(const SceneDev &S, const float *M, const Params &p, const uint4 &T,
                                              int Px, int Py, float qk, float (&attr)[3], float &lambda)
{
    CVert<NA> v[3];
    load_tri<NA>(S, M, T, v);
    CVert<NA> poly[4];
    const int np = clip_near<NA>(v, p.znear, poly);
    int X[4], Y[4];
    float q[4];
    bool in_range = true;
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (k < np)
            in_range &= project_snap(poly[k].xe, poly[k].ye, poly[k].d, p.fx, p.fy, p.cx, p.cy, q[k], X[k], Y[k]);
    if constexpr (G) {
        if (!in_range) {
            ClipPoly<NA> cp;
#pragma unroll
            for (int k = 0; k < 4; k++) cp.v[k] = poly[k];
            cp.n = np;
            return shade_guard_fan<NA>(S, cp, GuardCam{p.gx, p.gy, p.fx, p.fy, p.cx, p.cy}, Px, Py, qk, attr, lambda);
        }
    }
    return shade_fan<NA>(S, poly, X, Y, q, np, Px, Py, attr, lambda);
}

template <int NA>
__device__ __forceinline__ uint32_t shade_colour(const SceneDev &S, const float (&a)[3], float lambda = 0.0f)
{
    if (NA == 2)
        return S.sample_mode == HSR_SAMPLE_TRILINEAR ? sample_trilinear(S, a[0], a[1], lambda)
                                                     : sample_bilinear(S, a[0], a[1]);
    if (NA == 3) return round_channel(a[0]) | (round_channel(a[1]) << 8) | (round_channel(a[2]) << 16);
    return 0xFFFFFFu;
}

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 products mixed with the other counter words and a key bumped by
// Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Appendix C noise model: inverse depth plus iid Gaussian noise of std sigma
// (Box-Muller on two Philox words at counter (pixel, agent, 'nois', 0));
// a noisy inverse depth at or below 1/far reports no return (depth 0).
// PRECISE (the shading variant every noisy call launches): the cosine as
// cospi(2 u2), whose argument is exact in fp32 (u2 has 23 bits); the rounded
// argument of cos(2 pi u2) would dominate the error of z. The other form is
// compiled into the noise-free variant only because its register allocation
// measured fastest with it (that variant never runs it).
template <bool PRECISE>
__device__ __forceinline__ float noisy_depth(float sigma, uint32_t k0, uint32_t k1, float inv_far, float q,
                                             uint32_t pixel, uint32_t agent)
{
    const uint4 r = philox4x32_10(make_uint4(pixel, agent, 0x6e6f6973u, 0u), k0, k1);
    const float u1 = ((float)(r.x >> 9) + 0.5f) * 1.1920928955078125e-07f;   // 2^-23
    const float u2 = ((float)(r.y >> 9) + 0.5f) * 1.1920928955078125e-07f;
    const float c = PRECISE ? cospif(2.0f * u2) : cosf(6.283185307179586f * u2);
    const float z = sqrtf(-2.0f * logf(u1)) * c;
    const float qn = __fmaf_rn(sigma, z, q);
    return qn > inv_far ? __frcp_rn(qn) : 0.0f;
}

// Shade one pixel given its key; `st` caches the last triangle's setup (G:
// the view may hold winners that need the guard band).
template <int NA, bool G>
__device__ __forceinline__ void shade_pixel(ShadeTri<NA> &st, const SceneDev &S, const float *M, const Params &p,
                                            int px, int py, unsigned long long key, uint32_t &rgb, float &depth,
                                            uint32_t &id, bool colour)
{
    if (key == ~0ull) {
        rgb = 0;
        depth = 0.0f;
        id = kBackgroundId;
        return;
    }
    const uint32_t tri = (uint32_t)key;
    const float qk = __uint_as_float(~(uint32_t)(key >> 32));
    depth = __frcp_rn(qk);
    if (!colour) {             // depth / id views: no attribute work
        rgb = 0;
        id = S.tri[tri].w;
        return;
    }
    if (tri != st.tri) build_shade_tri<NA, G>(st, S, M, p, tri);
    id = st.id;
    const int Px = 256 * px + 128, Py = 256 * py + 128;
    float a[3] = {0.f, 0.f, 0.f};
    float lambda = 0.0f;
    if (!st.clipped) {
        interp<NA>(st.t, st.narrow, Px, Py, st.a[0], st.a[1], st.a[2], a);
        if constexpr (NA == 2)
            if (S.sample_mode == HSR_SAMPLE_TRILINEAR)
                lambda = lod_lambda(S.atlas_w, S.atlas_h, st.t, Px, Py, st.a[0], st.a[1], st.a[2]);
        rgb = shade_colour<NA>(S, a, lambda);
    } else {
        rgb = shade_clipped<NA, G>(S, M, p, __ldg(S.tri + tri), Px, Py, qk, a, lambda) ? shade_colour<NA>(S, a, lambda)
                                                                                      : 0u;
    }
}

}  // namespace hsr
