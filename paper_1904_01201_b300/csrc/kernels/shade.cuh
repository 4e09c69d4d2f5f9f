// K5 — resolve and shade (deferred): for each pixel of the region, decode the
// winning key, rebuild that triangle's setup exactly as the rasteriser did,
// find the (sub-)triangle that produced the fragment, and write the three
// sensor outputs of the single pass (Sec. 3 "Rendering engine": colour, depth
// and semantic outputs together).
//
// Readings: perspective-correct weights w_k = E_k(P) * q_k normalised;
// texture lookups are bilinear, clamp-to-edge, at (u*Wt - 0.5, v*Ht - 0.5)
// with atlas row 0 at v = 0; channels round half up and saturate at 255;
// depth = 1/q; background is RGB 0, depth 0, id 0xFFFFFFFF.
#pragma once
#include "raster.cuh"

namespace hsr {

constexpr uint32_t kBackgroundId = 0xFFFFFFFFu;

struct ShadeOut {
    uint32_t rgb;      // r | g << 8 | b << 16
    float depth;
    uint32_t id;
};

__device__ __forceinline__ uint32_t round_channel(float c)
{
    const float r = floorf(__fadd_rn(c, 0.5f));
    return (uint32_t)fminf(fmaxf(r, 0.0f), 255.0f);
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
    const int W = (int)S.atlas_w, H = (int)S.atlas_h;
    const int x0 = min(max(ix, 0), W - 1), x1 = min(max(ix + 1, 0), W - 1);
    const int y0 = min(max(iy, 0), H - 1), y1 = min(max(iy + 1, 0), H - 1);
    const uint32_t c00 = __ldg(S.atlas + (size_t)y0 * W + x0), c10 = __ldg(S.atlas + (size_t)y0 * W + x1);
    const uint32_t c01 = __ldg(S.atlas + (size_t)y1 * W + x0), c11 = __ldg(S.atlas + (size_t)y1 * W + x1);
    const float gx = 1.0f - ax, gy = 1.0f - ay;
    uint32_t out = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float v00 = (float)((c00 >> (8 * c)) & 255u), v10 = (float)((c10 >> (8 * c)) & 255u);
        const float v01 = (float)((c01 >> (8 * c)) & 255u), v11 = (float)((c11 >> (8 * c)) & 255u);
        const float top = __fmaf_rn(ax, v10, __fmul_rn(gx, v00));
        const float bot = __fmaf_rn(ax, v11, __fmul_rn(gx, v01));
        out |= round_channel(__fmaf_rn(ay, bot, __fmul_rn(gy, top))) << (8 * c);
    }
    return out;
}

// Rebuild triangle `tri` with NA attributes, find the sub-triangle whose
// fragment at (Px, Py) has inverse depth qk, and interpolate its attributes.
template <int NA>
__device__ __forceinline__ bool refind_fragment(const SceneDev &S, const float *M, const Params &p,
                                                const uint4 &T, int Px, int Py, float qk, float (&attr)[3])
{
    CVert<NA> v[3];
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
    CVert<NA> poly[4];
    int np;
    if (v[0].d >= p.znear && v[1].d >= p.znear && v[2].d >= p.znear) {
        poly[0] = v[0]; poly[1] = v[1]; poly[2] = v[2];
        np = 3;
    } else {
        np = clip_near<NA>(v, p.znear, poly);
    }
    int X[4], Y[4];
    float q[4];
    for (int k = 0; k < np; k++) project_snap(poly[k].xe, poly[k].ye, poly[k].d, p.fx, p.fy, p.cx, p.cy, q[k], X[k], Y[k]);
    for (int f = 0; f + 2 < np; f++) {
        Tri2D t;
        if (!orient_cull(X[0], Y[0], q[0], X[f + 1], Y[f + 1], q[f + 1], X[f + 2], Y[f + 2], q[f + 2], t)) continue;
        const long long e0 = (long long)(t.X2 - t.X1) * (Py - t.Y1) - (long long)(t.Y2 - t.Y1) * (Px - t.X1);
        const long long e1 = (long long)(t.X0 - t.X2) * (Py - t.Y2) - (long long)(t.Y0 - t.Y2) * (Px - t.X2);
        const long long e2 = (long long)(t.X1 - t.X0) * (Py - t.Y0) - (long long)(t.Y1 - t.Y0) * (Px - t.X0);
        const int b0 = edge_bias(t.X1, t.Y1, t.X2, t.Y2);
        const int b1 = edge_bias(t.X2, t.Y2, t.X0, t.Y0);
        const int b2 = edge_bias(t.X0, t.Y0, t.X1, t.Y1);
        if (((e0 - b0) | (e1 - b1) | (e2 - b2)) < 0) continue;
        float pa, pb;
        depth_plane(t, pa, pb);
        const float qq = plane_q(pa, pb, t.q0, Px - t.X0, Py - t.Y0);
        if (__float_as_uint(qq) != __float_as_uint(qk)) continue;
        // oriented order is (poly 0, poly f+2, poly f+1)
        const float w0 = __fmul_rn(__ll2float_rn(e0), t.q0);
        const float w1 = __fmul_rn(__ll2float_rn(e1), t.q1);
        const float w2 = __fmul_rn(__ll2float_rn(e2), t.q2);
        const float r = __frcp_rn(__fadd_rn(__fadd_rn(w0, w1), w2));
        const float l0 = __fmul_rn(w0, r), l1 = __fmul_rn(w1, r), l2 = __fmul_rn(w2, r);
#pragma unroll
        for (int c = 0; c < NA; c++)
            attr[c] = __fmaf_rn(l0, poly[0].a[c], __fmaf_rn(l1, poly[f + 2].a[c], __fmul_rn(l2, poly[f + 1].a[c])));
        return true;
    }
    return false;
}

__device__ __forceinline__ ShadeOut shade_pixel(const SceneDev &S, const float *M, const Params &p, int px,
                                                int py, unsigned long long key)
{
    ShadeOut o;
    if (key == ~0ull) {
        o.rgb = 0;
        o.depth = 0.0f;
        o.id = kBackgroundId;
        return o;
    }
    const uint32_t tri = (uint32_t)key;
    const float qk = __uint_as_float(~(uint32_t)(key >> 32));
    o.depth = __frcp_rn(qk);
    const uint4 T = __ldg(S.tri + tri);
    o.id = T.w;
    const int Px = 256 * px + 128, Py = 256 * py + 128;
    float a[3] = {0.f, 0.f, 0.f};
    if (S.color_mode == kColorTexture) {
        o.rgb = refind_fragment<2>(S, M, p, T, Px, Py, qk, a) ? sample_bilinear(S, a[0], a[1]) : 0u;
    } else if (S.color_mode == kColorVertex) {
        if (refind_fragment<3>(S, M, p, T, Px, Py, qk, a))
            o.rgb = round_channel(a[0]) | (round_channel(a[1]) << 8) | (round_channel(a[2]) << 16);
        else
            o.rgb = 0;
    } else {
        o.rgb = 0xFFFFFFu;
    }
    return o;
}

}  // namespace hsr
