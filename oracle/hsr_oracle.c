/*
 * CPU oracle for the sensor-rendering hot path.  TEST INFRASTRUCTURE ONLY:
 * only the tests, the package smoke check and the benchmark's CPU-baseline leg
 * may load this file's library.  It shares no code with the CUDA path.
 *
 * What it computes is the plain definition of a rasterised observation
 * (Sec. 3 "Rendering engine": one pass yields colour, depth and semantic
 * outputs; Sec. 4 "Sensory input": pinhole colour + idealised depth sensor at
 * the same pose).  For every pixel centre it takes, over ALL triangles and
 * all pixels of each triangle's bounding box (no binning, no culling beyond
 * the rules below), the covering fragment with the largest interpolated
 * inverse depth, ties to the lower triangle index, and shades that fragment.
 *
 * The paper fixes none of the rasterisation rules (it uses an OpenGL
 * pipeline); every rule below is a stated reading:
 *   order    : each index triple is rotated cyclically so that its
 *              lexicographically smallest rotation comes first.
 *   camera   : unit quaternion (w,x,y,z) -> R (world-from-camera) in double,
 *              M = [R^T | -R^T pos] rounded once to float; camera looks down
 *              -Z, +Y up; eye depth d = -z_e (planar depth).
 *   transform: x_e = fma(M00,x, fma(M01,y, fma(M02,z, M03))) (same for y, z).
 *   reject   : all three d < near, or all three d > far.
 *   near clip: Sutherland-Hodgman against d >= near; an edge's endpoints are
 *              ordered by ascending vertex index; t = (near-d_a)/(d_b-d_a),
 *              p = fma(t, p_b - p_a, p_a), d := near; fan from first vertex.
 *   project  : q = 1/d, sx = fma(fx, x_e*q, cx), sy = fma(-fy, y_e*q, cy),
 *              X = rint(256 sx), Y = rint(256 sy)  (8 sub-pixel bits).
 *   guard    : a (near-clipped) polygon with a snapped coordinate at or
 *              beyond +-2^30 is clipped further, Sutherland-Hodgman, against
 *              the eye-space planes x_e >= -gx d, x_e <= gx d, y_e >= -gy d,
 *              y_e <= gy d in that order, gx = 2^21 / fx, gy = 2^21 / fy
 *              (float division): they project 2^21 pixels (2^29 sub-pixels)
 *              either side of the principal point.  Plane distances are
 *              fma(g, d, +-x_e); a crossing edge is cut from its endpoint
 *              b nearer the cut (the inside one when s_in <= -s_out, else the
 *              outside one), other endpoint r: t = s_b / (s_b - s_r),
 *              p = fma(t, p_r - p_b, p_b), attributes likewise.  The choice
 *              depends only on the two endpoints, so the two triangles sharing
 *              an edge cut it at the same point, and the cut is computed from
 *              the nearer endpoint, without cancellation against the far one.
 *              The polygon is then projected again and fanned from its first
 *              vertex.
 *   cull     : A = (X1-X0)(Y2-Y0) - (Y1-Y0)(X2-X0) in int64, keep A < 0
 *              (front faces are counter-clockwise in the world), then swap
 *              vertices 1 and 2 so that A > 0.
 *   coverage : sample (256x+128, 256y+128); edge k opposite vertex k;
 *              inside iff E_k > 0, or E_k == 0 and edge k is top or left
 *              (edge i->j is top iff dy == 0 and dx > 0, left iff dy < 0).
 *   depth    : plane of q over the snapped vertices, relative to vertex 0,
 *              fp32 op order below, clamped to [min q_i, max q_i] of the
 *              (sub-)triangle's vertices; fragment kept iff 1/q <= far.  The
 *              sub-triangles of a clipped polygon (near plane or guard band)
 *              are first rotated cyclically so that vertex 0 has the smallest
 *              q (the first such on ties): their other vertices can sit at
 *              q = 1/near or far outside the image, where an fp32 plane
 *              referenced at them loses the on-screen depth to cancellation.
 *   key      : ((~bits(q)) << 32) | triangle index; per-pixel minimum.
 *   shade    : perspective-correct weights E_k * q_k (fp64), bilinear
 *              clamp-to-edge texture lookup at (u*Wt - 0.5, v*Ht - 0.5), or
 *              vertex colours; channel = min(255, floor(c + 0.5)).
 *   outputs  : RGB u8, depth 1/q (float), id = semantic[tri] or tri;
 *              background RGB 0, depth 0, id 0xFFFFFFFF.
 *   mipmaps  : optional trilinear sampling of minified textures: level l+1
 *              is max(1, W_l >> 1) x max(1, H_l >> 1) texels, each the
 *              rounded mean (a + b + c + d + 2) >> 2 of its 2x2 block of level
 *              l (block coordinates clamped to level l); lambda = log2(rho),
 *              rho = max over x and y of the texel-space length of the
 *              perspective-correct uv derivative at the pixel centre (from the
 *              exact derivatives of the weights E_k q_k); lambda <= 0 samples
 *              level 0 bilinearly (the plain rule above); otherwise the
 *              bilinear samples of levels floor(lambda) and floor(lambda) + 1
 *              (the last level beyond it) blend with weight frac(lambda),
 *              each level sampled at (u W_l - 0.5, v H_l - 0.5), then round.
 *   noise    : optional noisy depth (Appendix C: iid Gaussian, mean 0,
 *              std sigma, added to inverse depth per pixel): for a hit pixel
 *              q' = q + sigma z, z = sqrt(-2 ln u1) cos(2 pi u2) (fp64), with
 *              u1, u2 from Philox-4x32-10 (Salmon et al. 2011) at counter
 *              (pixel index, agent, 0x6e6f6973, 0) and key (seed lo, seed hi),
 *              u = ((x >> 9) + 0.5) 2^-23; depth = 1/q', or 0 when
 *              q' <= 1/far (no valid return).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_OOM 2
#define OR_ERR_RANGE 3      /* a snapped coordinate beyond +-2^30 sub-pixels after the guard clip */

static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

/* Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
   multiplies two counter words by fixed odd constants, mixes the high and low
   halves with the other words and the key, and bumps the key by the Weyl
   increments. */
void oracle_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += W0;
        k1 += W1;
    }
    for (int i = 0; i < 4; i++) out[i] = c[i];
}

static double unit_open(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* camera matrix from a pose (x, y, z, qw, qx, qy, qz) */
int oracle_camera(const float *pose, float *M)
{
    double px = pose[0], py = pose[1], pz = pose[2];
    double w = pose[3], x = pose[4], y = pose[5], z = pose[6];
    double n2 = ((w * w + x * x) + y * y) + z * z;
    double n = sqrt(n2);
    if (!(fabs(n - 1.0) <= 1e-3)) return OR_ERR_ARG;
    w /= n; x /= n; y /= n; z /= n;
    double R[3][3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) M[i * 4 + j] = (float)R[j][i];
        M[i * 4 + 3] = (float)(-((R[0][i] * px + R[1][i] * py) + R[2][i] * pz));
    }
    return OR_OK;
}

/*
 * Agent actuation (Sec. 4 "Agent embodiment and action space": stop,
 * move_forward 0.25 m, turn_left / turn_right 10 degrees, idealised, no
 * actuation noise).  Readings, all arithmetic in double from the float state,
 * each pose component rounded once to float at the end:
 *   stop    : the pose is unchanged.
 *   forward : heading = R (0, 0, -1) of the normalised quaternion with its
 *             vertical component dropped: h = (-2(xz + wy), -(1 - 2(x^2 + y^2)));
 *             p' = p + step * h / |h| on x and z (y unchanged), rounded to
 *             float; refused (pose unchanged) when |h| = 0 or when the grid
 *             cell holding the rounded p' is not navigable: cell
 *             (floor((x - x0)/cell), floor((z - z0)/cell)), outside the grid
 *             counts as blocked (no sliding along obstacles).
 *   turn    : q' = r * q with r = (cos(t/2), 0, sin(t/2), 0) about world +Y,
 *             t = +turn for left, -turn for right (degrees * pi / 180), then
 *             q' / |q'|.  Products and sums in the order written below.
 * grid: [nz][nx] bytes, nonzero = navigable.  Returns 1 if the pose moved or
 * turned, 0 if unchanged, -1 for an unknown action.
 */
int oracle_actuate(const float *pose, int action, double step, double turn_deg, float x0, float z0, float cell,
                   uint32_t nx, uint32_t nz, const uint8_t *grid, float *out)
{
    memcpy(out, pose, 7 * sizeof(float));
    double w = pose[3], x = pose[4], y = pose[5], z = pose[6];
    const double n = sqrt(((w * w + x * x) + y * y) + z * z);
    w /= n; x /= n; y /= n; z /= n;
    if (action == 0) return 0;
    if (action == 1) {
        const double hx = -2.0 * (x * z + w * y);
        const double hz = -(1.0 - 2.0 * (x * x + y * y));
        const double len = sqrt(hx * hx + hz * hz);
        if (!(len > 0.0)) return 0;
        const float nxp = (float)((double)pose[0] + step * (hx / len));
        const float nzp = (float)((double)pose[2] + step * (hz / len));
        const double ci = floor(((double)nxp - (double)x0) / (double)cell);
        const double ck = floor(((double)nzp - (double)z0) / (double)cell);
        if (!(ci >= 0.0 && ci < (double)nx && ck >= 0.0 && ck < (double)nz)) return 0;
        if (!grid[(size_t)ck * nx + (size_t)ci]) return 0;
        out[0] = nxp;
        out[2] = nzp;
        return 1;
    }
    if (action == 2 || action == 3) {
        const double t = (action == 2 ? turn_deg : -turn_deg) * (3.14159265358979323846 / 180.0);
        const double c = cos(0.5 * t), s = sin(0.5 * t);
        const double w2 = c * w - s * y;
        const double x2 = c * x + s * z;
        const double y2 = c * y + s * w;
        const double z2 = c * z - s * x;
        const double n2 = sqrt(((w2 * w2 + x2 * x2) + y2 * y2) + z2 * z2);
        out[3] = (float)(w2 / n2);
        out[4] = (float)(x2 / n2);
        out[5] = (float)(y2 / n2);
        out[6] = (float)(z2 / n2);
        return 1;
    }
    return -1;
}

typedef struct {
    float xe, ye, d;        /* eye space, d = -z_e */
    uint32_t vid;           /* caller's vertex index (clip ordering) */
    double attr[3];         /* u, v (textured) or r, g, b (vertex colour) */
} overt;

typedef struct {
    /* scene */
    const float *xyz; uint32_t nv;
    const uint32_t *idx; uint32_t nt;
    const float *uv; const uint8_t *vrgb;
    const uint8_t *atlas; uint32_t aw, ah;
    /* mip chain (trilinear sampling): level 0 is the atlas */
    int nlev;
    const uint8_t *mip[16]; uint32_t mw[16], mh[16];
    float *lod;             /* optional per-pixel lambda of the shaded fragment */
    const uint32_t *sem;
    /* views */
    const float *poses; uint32_t n;
    float fx, fy, cx, cy, znear, zfar;
    float gx, gy;           /* guard planes |x_e| <= gx d, |y_e| <= gy d */
    uint32_t W, H;
    uint8_t *rgb; float *depth; uint32_t *ids; uint32_t *cover;
    /* depth noise */
    float noise_sigma;
    uint64_t noise_seed;
    const uint32_t *agent_ids;
    /* work split */
    uint32_t f0, f1;
    int status;
} ojob;

static int64_t floordiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
static int64_t ceildiv(int64_t a, int64_t b) { return -floordiv(-a, b); }

static double texel_of(const uint8_t *img, uint32_t w, uint32_t h, int64_t x, int64_t y, int c)
{
    if (x < 0) x = 0;
    if (x > (int64_t)w - 1) x = w - 1;
    if (y < 0) y = 0;
    if (y > (int64_t)h - 1) y = h - 1;
    return (double)img[((size_t)y * w + (size_t)x) * 4 + c];
}

/* bilinear sample (unrounded, channels 0..2) of an RGBA8 image at (u, v),
   clamp to edge, texel centres at half-integers */
static void bilinear(const uint8_t *img, uint32_t w, uint32_t h, double u, double vv, double out[3])
{
    double sx = u * w - 0.5, sy = vv * h - 0.5;
    if (!(sx >= -1.0)) sx = -1.0;
    if (sx > w) sx = w;
    if (!(sy >= -1.0)) sy = -1.0;
    if (sy > h) sy = h;
    double x0 = floor(sx), y0 = floor(sy);
    double ax = sx - x0, ay = sy - y0;
    int64_t ix = (int64_t)x0, iy = (int64_t)y0;
    for (int c = 0; c < 3; c++) {
        double c00 = texel_of(img, w, h, ix, iy, c), c10 = texel_of(img, w, h, ix + 1, iy, c);
        double c01 = texel_of(img, w, h, ix, iy + 1, c), c11 = texel_of(img, w, h, ix + 1, iy + 1, c);
        out[c] = (1 - ax) * (1 - ay) * c00 + ax * (1 - ay) * c10 + (1 - ax) * ay * c01 + ax * ay * c11;
    }
}

/* level l+1 of a mip chain from level l (w x h): rounded 2x2 means */
static void mip_down(const uint8_t *src, uint32_t w, uint32_t h, uint8_t *dst, uint32_t w2, uint32_t h2)
{
    for (uint32_t y = 0; y < h2; y++)
        for (uint32_t x = 0; x < w2; x++)
            for (int c = 0; c < 4; c++) {
                unsigned sum = 2;
                for (int dy = 0; dy < 2; dy++)
                    for (int dx = 0; dx < 2; dx++) {
                        uint32_t sx = 2 * x + dx, sy = 2 * y + dy;
                        if (sx > w - 1) sx = w - 1;
                        if (sy > h - 1) sy = h - 1;
                        sum += src[((size_t)sy * w + sx) * 4 + c];
                    }
                dst[((size_t)y * w2 + x) * 4 + c] = (uint8_t)(sum >> 2);
            }
}

static uint8_t round_channel(double c)
{
    double r = floor(c + 0.5);
    if (r < 0) r = 0;
    if (r > 255) r = 255;
    return (uint8_t)r;
}

/* shade one fragment in fp64: weights E_k * q_k (perspective-correct) */
/* shade one fragment in fp64: weights E_k * q_k (perspective-correct);
   dEx[k], dEy[k]: change of E_k per sub-pixel step in x and in y.  Returns
   lambda for trilinear sampling (NAN when not computed). */
static double shade(const ojob *J, int mode, const overt *v[3], const float q[3], const int64_t E[3],
                    const int64_t dEx[3], const int64_t dEy[3], uint8_t out[3])
{
    double w0 = (double)E[0] * (double)q[0];
    double w1 = (double)E[1] * (double)q[1];
    double w2 = (double)E[2] * (double)q[2];
    double s = w0 + w1 + w2;
    double l0 = w0 / s, l1 = w1 / s, l2 = w2 / s;
    double lambda = NAN;
    if (mode == 1) {
        double u = l0 * v[0]->attr[0] + l1 * v[1]->attr[0] + l2 * v[2]->attr[0];
        double vv = l0 * v[0]->attr[1] + l1 * v[1]->attr[1] + l2 * v[2]->attr[1];
        double val[3];
        if (J->nlev > 0) {
            /* d(l_k)/dx = (dw_k/dx - l_k dS/dx) / S, one pixel = 256 sub-pixels */
            const double l[3] = {l0, l1, l2};
            double dwx[3], dwy[3], dsx = 0, dsy = 0;
            for (int k = 0; k < 3; k++) {
                dwx[k] = 256.0 * (double)dEx[k] * (double)q[k];
                dwy[k] = 256.0 * (double)dEy[k] * (double)q[k];
                dsx += dwx[k];
                dsy += dwy[k];
            }
            double dudx = 0, dvdx = 0, dudy = 0, dvdy = 0;
            for (int k = 0; k < 3; k++) {
                const double gx = (dwx[k] - l[k] * dsx) / s, gy = (dwy[k] - l[k] * dsy) / s;
                dudx += gx * v[k]->attr[0];
                dvdx += gx * v[k]->attr[1];
                dudy += gy * v[k]->attr[0];
                dvdy += gy * v[k]->attr[1];
            }
            const double rx = sqrt((dudx * J->aw) * (dudx * J->aw) + (dvdx * J->ah) * (dvdx * J->ah));
            const double ry = sqrt((dudy * J->aw) * (dudy * J->aw) + (dvdy * J->ah) * (dvdy * J->ah));
            lambda = log2(rx > ry ? rx : ry);
            if (!(lambda > 0.0)) {
                bilinear(J->mip[0], J->mw[0], J->mh[0], u, vv, val);
            } else if (lambda >= (double)(J->nlev - 1)) {
                const int L = J->nlev - 1;
                bilinear(J->mip[L], J->mw[L], J->mh[L], u, vv, val);
            } else {
                const int l0i = (int)floor(lambda);
                const double f = lambda - (double)l0i;
                double a[3], b[3];
                bilinear(J->mip[l0i], J->mw[l0i], J->mh[l0i], u, vv, a);
                bilinear(J->mip[l0i + 1], J->mw[l0i + 1], J->mh[l0i + 1], u, vv, b);
                for (int c = 0; c < 3; c++) val[c] = (1.0 - f) * a[c] + f * b[c];
            }
        } else {
            bilinear(J->atlas, J->aw, J->ah, u, vv, val);
        }
        for (int c = 0; c < 3; c++) out[c] = round_channel(val[c]);
    } else if (mode == 2) {
        for (int c = 0; c < 3; c++)
            out[c] = round_channel(l0 * v[0]->attr[c] + l1 * v[1]->attr[c] + l2 * v[2]->attr[c]);
    } else {
        out[0] = out[1] = out[2] = 255;
    }
    return lambda;
}

static overt clip_point(const overt *p, const overt *r, float znear, int nattr)
{
    const overt *a = p, *b = r;
    if (b->vid < a->vid) { a = r; b = p; }
    float t = (znear - a->d) / (b->d - a->d);
    overt o;
    o.xe = fmaf(t, b->xe - a->xe, a->xe);
    o.ye = fmaf(t, b->ye - a->ye, a->ye);
    o.d = znear;
    o.vid = 0xFFFFFFFFu;
    for (int k = 0; k < nattr; k++) o.attr[k] = a->attr[k] + (double)t * (b->attr[k] - a->attr[k]);
    for (int k = nattr; k < 3; k++) o.attr[k] = 0;
    return o;
}

/* Guard-band clip of a polygon (n <= 4 vertices, all d >= near) against the
   four planes of the reading in the header; returns the new size (<= 8). */
static int guard_clip(const overt *in, int n, float gx, float gy, int nattr, overt *out)
{
    overt a[8], b[8];
    int na = n;
    for (int k = 0; k < n; k++) a[k] = in[k];
    for (int pl = 0; pl < 4; pl++) {
        const float g = pl < 2 ? gx : gy;
        const float sgn = (pl & 1) ? -1.0f : 1.0f;     /* L, R, B, T: fma(g, d, +x), fma(g, d, -x), ... */
        float dist[8];
        for (int k = 0; k < na; k++) dist[k] = fmaf(g, a[k].d, sgn * (pl < 2 ? a[k].xe : a[k].ye));
        int nb = 0;
        for (int k = 0; k < na; k++) {
            const int k1 = (k + 1) % na;
            const int ain = dist[k] >= 0.0f, bin = dist[k1] >= 0.0f;
            if (ain) b[nb++] = a[k];
            if (ain != bin) {
                /* cut from the endpoint nearer the cut: the inside one when
                   s_in <= -s_out, else the outside one */
                const overt *pi = ain ? &a[k] : &a[k1], *po = ain ? &a[k1] : &a[k];
                const float si = ain ? dist[k] : dist[k1], so = ain ? dist[k1] : dist[k];
                const int from_in = si <= -so;
                const overt *pb = from_in ? pi : po, *pr = from_in ? po : pi;
                const float sb = from_in ? si : so, sr = from_in ? so : si;
                const float t = sb / (sb - sr);
                overt o;
                o.xe = fmaf(t, pr->xe - pb->xe, pb->xe);
                o.ye = fmaf(t, pr->ye - pb->ye, pb->ye);
                o.d = fmaf(t, pr->d - pb->d, pb->d);
                o.vid = 0xFFFFFFFFu;
                for (int c = 0; c < nattr; c++) o.attr[c] = pb->attr[c] + (double)t * (pr->attr[c] - pb->attr[c]);
                for (int c = nattr; c < 3; c++) o.attr[c] = 0;
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

/* The guard clip on its own (for the pins): in, out [n][3] = (x_e, y_e, d)
   per vertex; returns the clipped size (out holds up to 8 vertices). */
int oracle_guard_clip(const float *in, int n, float gx, float gy, float *out)
{
    if (n < 0 || n > 4) return -1;
    overt v[4], r[8];
    for (int k = 0; k < n; k++) {
        v[k].xe = in[3 * k]; v[k].ye = in[3 * k + 1]; v[k].d = in[3 * k + 2];
        v[k].vid = (uint32_t)k;
        v[k].attr[0] = v[k].attr[1] = v[k].attr[2] = 0;
    }
    const int m = guard_clip(v, n, gx, gy, 0, r);
    for (int k = 0; k < m; k++) { out[3 * k] = r[k].xe; out[3 * k + 1] = r[k].ye; out[3 * k + 2] = r[k].d; }
    return m;
}

/* Project and snap the polygon's vertices; 0 if a coordinate is at or beyond
   +-2^30 sub-pixels (or not a number). */
static int project_poly(const ojob *J, const overt *poly, int np, int32_t *X, int32_t *Y, float *q)
{
    for (int k = 0; k < np; k++) {
        q[k] = 1.0f / poly[k].d;
        float sx = fmaf(J->fx, poly[k].xe * q[k], J->cx);
        float sy = fmaf(-J->fy, poly[k].ye * q[k], J->cy);
        float rx = rintf(sx * 256.0f), ry = rintf(sy * 256.0f);
        if (!(fabsf(rx) < 1073741824.0f) || !(fabsf(ry) < 1073741824.0f)) return 0;
        X[k] = (int32_t)rx;
        Y[k] = (int32_t)ry;
    }
    return 1;
}

static int render_frame(ojob *J, uint32_t f, uint64_t *best)
{
    const uint32_t W = J->W, H = J->H;
    const size_t npx = (size_t)W * H;
    float M[12];
    if (oracle_camera(J->poses + 7 * (size_t)f, M) != OR_OK) return OR_ERR_ARG;
    const int mode = (J->uv && J->atlas) ? 1 : (J->vrgb ? 2 : 0);
    const int nattr = mode == 1 ? 2 : (mode == 2 ? 3 : 0);
    uint8_t *rgb = J->rgb + (size_t)f * npx * 3;
    float *dep = J->depth + (size_t)f * npx;
    uint32_t *ids = J->ids ? J->ids + (size_t)f * npx : NULL;
    uint32_t *cov = J->cover ? J->cover + (size_t)f * npx : NULL;
    for (size_t i = 0; i < npx; i++) best[i] = ~(uint64_t)0;
    memset(rgb, 0, npx * 3);
    for (size_t i = 0; i < npx; i++) dep[i] = 0.0f;
    if (ids) for (size_t i = 0; i < npx; i++) ids[i] = 0xFFFFFFFFu;
    if (cov) memset(cov, 0, npx * 4);

    for (uint32_t t = 0; t < J->nt; t++) {
        overt v[3];
        /* canonical cyclic order: the lexicographically smallest rotation of
           the index triple comes first (orientation is unchanged) */
        uint32_t tri[3] = {J->idx[3 * (size_t)t], J->idx[3 * (size_t)t + 1], J->idx[3 * (size_t)t + 2]};
        int r = 0;
        for (int c = 1; c < 3; c++) {
            for (int k = 0; k < 3; k++) {
                uint32_t a = tri[(c + k) % 3], b = tri[(r + k) % 3];
                if (a != b) { if (a < b) r = c; break; }
            }
        }
        for (int k = 0; k < 3; k++) {
            uint32_t vi = tri[(r + k) % 3];
            float x = J->xyz[3 * (size_t)vi], y = J->xyz[3 * (size_t)vi + 1], z = J->xyz[3 * (size_t)vi + 2];
            v[k].xe = fmaf(M[0], x, fmaf(M[1], y, fmaf(M[2], z, M[3])));
            v[k].ye = fmaf(M[4], x, fmaf(M[5], y, fmaf(M[6], z, M[7])));
            float ze = fmaf(M[8], x, fmaf(M[9], y, fmaf(M[10], z, M[11])));
            v[k].d = -ze;
            v[k].vid = vi;
            for (int c = 0; c < 3; c++) v[k].attr[c] = 0;
            if (mode == 1) { v[k].attr[0] = J->uv[2 * (size_t)vi]; v[k].attr[1] = J->uv[2 * (size_t)vi + 1]; }
            if (mode == 2) for (int c = 0; c < 3; c++) v[k].attr[c] = J->vrgb[3 * (size_t)vi + c];
        }
        const float zn = J->znear, zf = J->zfar;
        if (v[0].d < zn && v[1].d < zn && v[2].d < zn) continue;
        if (v[0].d > zf && v[1].d > zf && v[2].d > zf) continue;
        overt poly[8];
        int np = 0;
        if (v[0].d >= zn && v[1].d >= zn && v[2].d >= zn) {
            poly[0] = v[0]; poly[1] = v[1]; poly[2] = v[2]; np = 3;
        } else {
            for (int k = 0; k < 3; k++) {
                const overt *a = &v[k], *b = &v[(k + 1) % 3];
                int ain = a->d >= zn, bin = b->d >= zn;
                if (ain) poly[np++] = *a;
                if (ain != bin) poly[np++] = clip_point(a, b, zn, nattr);
            }
        }
        /* project and snap; beyond the fixed-point range, clip to the guard band */
        int32_t X[8], Y[8];
        float q[8];
        int clipped = np != 3 || poly[0].vid != v[0].vid || poly[1].vid != v[1].vid || poly[2].vid != v[2].vid;
        if (!project_poly(J, poly, np, X, Y, q)) {
            clipped = 1;
            overt near_poly[4];
            for (int k = 0; k < np; k++) near_poly[k] = poly[k];
            np = guard_clip(near_poly, np, J->gx, J->gy, nattr, poly);
            if (!project_poly(J, poly, np, X, Y, q)) return OR_ERR_RANGE;
        }
        for (int fan = 0; fan + 2 < np; fan++) {
            int i0 = 0, i1 = fan + 1, i2 = fan + 2;
            int64_t A = (int64_t)(X[i1] - X[i0]) * (Y[i2] - Y[i0]) - (int64_t)(Y[i1] - Y[i0]) * (X[i2] - X[i0]);
            if (A >= 0) continue;
            int tmp = i1; i1 = i2; i2 = tmp;      /* orient to positive area */
            A = -A;
            if (clipped) {
                /* a clipped polygon's vertices can sit at q = 1/near or on the
                   guard planes: the plane is referenced at the sub-triangle's
                   vertex of smallest q (first in oriented order on ties), a
                   cyclic rotation that keeps the orientation */
                if (q[i1] < q[i0] && q[i1] <= q[i2]) { tmp = i0; i0 = i1; i1 = i2; i2 = tmp; }
                else if (q[i2] < q[i0] && q[i2] < q[i1]) { tmp = i0; i0 = i2; i2 = i1; i1 = tmp; }
            }
            const int32_t X0 = X[i0], Y0 = Y[i0], X1 = X[i1], Y1 = Y[i1], X2 = X[i2], Y2 = Y[i2];
            const float q0 = q[i0], q1 = q[i1], q2 = q[i2];
            /* plane of q, relative to vertex 0 */
            const float qlo = fminf(q0, fminf(q1, q2)), qhi = fmaxf(q0, fmaxf(q1, q2));
            const float fA = (float)A;
            const float dq1 = q1 - q0, dq2 = q2 - q0;
            const float pa = fmaf(dq1, (float)(Y2 - Y0), -(dq2 * (float)(Y1 - Y0))) / fA;
            const float pb = fmaf(dq2, (float)(X1 - X0), -(dq1 * (float)(X2 - X0))) / fA;
            /* top-left flags per edge k (opposite vertex k) */
            const int32_t ex[3][2] = {{X1, X2}, {X2, X0}, {X0, X1}};
            const int32_t ey[3][2] = {{Y1, Y2}, {Y2, Y0}, {Y0, Y1}};
            int tl[3];
            int64_t dEx[3], dEy[3];
            for (int k = 0; k < 3; k++) {
                int64_t dx = (int64_t)ex[k][1] - ex[k][0], dy = (int64_t)ey[k][1] - ey[k][0];
                tl[k] = (dy < 0) || (dy == 0 && dx > 0);
                dEx[k] = -dy;
                dEy[k] = dx;
            }
            int32_t mnx = X0, mxx = X0, mny = Y0, mxy = Y0;
            if (X1 < mnx) mnx = X1;
            if (X2 < mnx) mnx = X2;
            if (X1 > mxx) mxx = X1;
            if (X2 > mxx) mxx = X2;
            if (Y1 < mny) mny = Y1;
            if (Y2 < mny) mny = Y2;
            if (Y1 > mxy) mxy = Y1;
            if (Y2 > mxy) mxy = Y2;
            int64_t x0 = ceildiv((int64_t)mnx - 128, 256), x1 = floordiv((int64_t)mxx - 128, 256);
            int64_t y0 = ceildiv((int64_t)mny - 128, 256), y1 = floordiv((int64_t)mxy - 128, 256);
            if (x0 < 0) x0 = 0;
            if (y0 < 0) y0 = 0;
            if (x1 > (int64_t)W - 1) x1 = (int64_t)W - 1;
            if (y1 > (int64_t)H - 1) y1 = (int64_t)H - 1;
            const overt *sv[3] = {&poly[i0], &poly[i1], &poly[i2]};
            const float sq[3] = {q0, q1, q2};
            for (int64_t py = y0; py <= y1; py++) {
                for (int64_t px = x0; px <= x1; px++) {
                    const int64_t Px = 256 * px + 128, Py = 256 * py + 128;
                    int64_t E[3];
                    int in = 1;
                    for (int k = 0; k < 3; k++) {
                        E[k] = ((int64_t)ex[k][1] - ex[k][0]) * (Py - ey[k][0]) -
                               ((int64_t)ey[k][1] - ey[k][0]) * (Px - ex[k][0]);
                        if (!(E[k] > 0 || (E[k] == 0 && tl[k]))) in = 0;
                    }
                    if (!in) continue;
                    const size_t pix = (size_t)py * W + (size_t)px;
                    if (cov) cov[pix]++;
                    float qq = fmaf(pa, (float)(Px - X0), fmaf(pb, (float)(Py - Y0), q0));
                    /* interior points lie between the vertices' depths: clamp the
                       rounded plane value to the vertices' range of q */
                    qq = fminf(fmaxf(qq, qlo), qhi);
                    if (!(qq > 0.0f)) continue;
                    const float dd = 1.0f / qq;
                    if (dd > zf) continue;
                    const uint64_t key = ((uint64_t)(~f2u(qq)) << 32) | t;
                    if (key < best[pix]) {
                        best[pix] = key;
                        const double lam = shade(J, mode, sv, sq, E, dEx, dEy, rgb + 3 * pix);
                        if (J->lod) J->lod[(size_t)f * npx + pix] = (float)lam;
                        dep[pix] = dd;
                        if (ids) ids[pix] = J->sem ? J->sem[t] : t;
                    }
                }
            }
        }
    }
    if (J->noise_sigma > 0.0f) {
        const uint32_t agent = J->agent_ids ? J->agent_ids[f] : f;
        const uint32_t key[2] = {(uint32_t)J->noise_seed, (uint32_t)(J->noise_seed >> 32)};
        for (size_t pix = 0; pix < npx; pix++) {
            if (best[pix] == ~(uint64_t)0) continue;
            const uint32_t ctr[4] = {(uint32_t)pix, agent, 0x6e6f6973u, 0u};
            uint32_t r[4];
            oracle_philox4x32_10(ctr, key, r);
            const double z = sqrt(-2.0 * log(unit_open(r[0]))) * cos(2.0 * 3.14159265358979323846 * unit_open(r[1]));
            const double q = (double)u2f(~(uint32_t)(best[pix] >> 32));
            const double qn = q + (double)J->noise_sigma * z;
            dep[pix] = qn <= 1.0 / (double)J->zfar ? 0.0f : (float)(1.0 / qn);
        }
    }
    return OR_OK;
}

static void *worker(void *arg)
{
    ojob *J = (ojob *)arg;
    uint64_t *best = (uint64_t *)malloc((size_t)J->W * J->H * sizeof(uint64_t));
    if (!best) { J->status = OR_ERR_OOM; return NULL; }
    J->status = OR_OK;
    for (uint32_t f = J->f0; f < J->f1 && J->status == OR_OK; f++) J->status = render_frame(J, f, best);
    free(best);
    return NULL;
}

int oracle_render_noisy(const float *xyz, uint32_t nv, const uint32_t *idx, uint32_t nt,
                        const float *uv, const uint8_t *vrgb, const uint8_t *atlas, uint32_t aw, uint32_t ah,
                        const uint32_t *sem, const float *poses, uint32_t n, const float *intr,
                        uint32_t W, uint32_t H, uint8_t *rgb, float *depth, uint32_t *ids, uint32_t *cover,
                        int nthreads, float noise_sigma, uint64_t noise_seed, const uint32_t *agent_ids);

int oracle_render(const float *xyz, uint32_t nv, const uint32_t *idx, uint32_t nt,
                  const float *uv, const uint8_t *vrgb, const uint8_t *atlas, uint32_t aw, uint32_t ah,
                  const uint32_t *sem, const float *poses, uint32_t n, const float *intr,
                  uint32_t W, uint32_t H, uint8_t *rgb, float *depth, uint32_t *ids, uint32_t *cover,
                  int nthreads)
{
    return oracle_render_noisy(xyz, nv, idx, nt, uv, vrgb, atlas, aw, ah, sem, poses, n, intr, W, H, rgb, depth,
                               ids, cover, nthreads, 0.0f, 0, NULL);
}

/* The full entry: trilinear != 0 samples textures through a mip chain of the
   atlas; lod (optional, [n][H][W], caller-initialised) receives lambda of
   each shaded textured pixel. */
int oracle_render_full(const float *xyz, uint32_t nv, const uint32_t *idx, uint32_t nt,
                       const float *uv, const uint8_t *vrgb, const uint8_t *atlas, uint32_t aw, uint32_t ah,
                       const uint32_t *sem, const float *poses, uint32_t n, const float *intr,
                       uint32_t W, uint32_t H, uint8_t *rgb, float *depth, uint32_t *ids, uint32_t *cover,
                       int nthreads, float noise_sigma, uint64_t noise_seed, const uint32_t *agent_ids,
                       int trilinear, float *lod)
{
    if (!xyz || !idx || !poses || !intr || !rgb || !depth || n == 0 || W == 0 || H == 0) return OR_ERR_ARG;
    for (size_t i = 0; i < 3 * (size_t)nt; i++)
        if (idx[i] >= nv) return OR_ERR_ARG;
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if ((uint32_t)nthreads > n) nthreads = (int)n;
    /* mip chain: level 0 is the atlas, halving down to 1 x 1 */
    int nlev = 0;
    uint8_t *levels[16] = {0};
    uint32_t mw[16], mh[16];
    if (trilinear && atlas && aw && ah) {
        mw[0] = aw; mh[0] = ah;
        nlev = 1;
        while ((mw[nlev - 1] > 1 || mh[nlev - 1] > 1) && nlev < 16) {
            mw[nlev] = mw[nlev - 1] > 1 ? mw[nlev - 1] >> 1 : 1;
            mh[nlev] = mh[nlev - 1] > 1 ? mh[nlev - 1] >> 1 : 1;
            levels[nlev] = (uint8_t *)malloc((size_t)mw[nlev] * mh[nlev] * 4);
            if (!levels[nlev]) {
                for (int l = 1; l < nlev; l++) free(levels[l]);
                return OR_ERR_OOM;
            }
            mip_down(nlev == 1 ? atlas : levels[nlev - 1], mw[nlev - 1], mh[nlev - 1], levels[nlev], mw[nlev],
                     mh[nlev]);
            nlev++;
        }
    }
    ojob *jobs = (ojob *)calloc((size_t)nthreads, sizeof(ojob));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        for (int l = 1; l < nlev; l++) free(levels[l]);
        return OR_ERR_OOM;
    }
    for (int i = 0; i < nthreads; i++) {
        ojob *J = &jobs[i];
        J->xyz = xyz; J->nv = nv; J->idx = idx; J->nt = nt;
        J->uv = uv; J->vrgb = vrgb; J->atlas = atlas; J->aw = aw; J->ah = ah; J->sem = sem;
        J->poses = poses; J->n = n;
        J->fx = intr[0]; J->fy = intr[1]; J->cx = intr[2]; J->cy = intr[3];
        J->znear = intr[4]; J->zfar = intr[5];
        J->gx = 2097152.0f / J->fx;
        J->gy = 2097152.0f / J->fy;
        J->W = W; J->H = H; J->rgb = rgb; J->depth = depth; J->ids = ids; J->cover = cover;
        J->noise_sigma = noise_sigma; J->noise_seed = noise_seed; J->agent_ids = agent_ids;
        J->nlev = nlev;
        for (int l = 0; l < nlev; l++) {
            J->mip[l] = l == 0 ? atlas : levels[l];
            J->mw[l] = mw[l];
            J->mh[l] = mh[l];
        }
        J->lod = lod;
        J->f0 = (uint32_t)((uint64_t)n * i / nthreads);
        J->f1 = (uint32_t)((uint64_t)n * (i + 1) / nthreads);
    }
    int st = OR_OK;
    if (nthreads == 1) {
        worker(&jobs[0]);
        st = jobs[0].status;
    } else {
        for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, worker, &jobs[i]);
        for (int i = 0; i < nthreads; i++) {
            pthread_join(th[i], NULL);
            if (jobs[i].status != OR_OK && st == OR_OK) st = jobs[i].status;
        }
    }
    free(jobs);
    free(th);
    for (int l = 1; l < nlev; l++) free(levels[l]);
    return st;
}

int oracle_render_noisy(const float *xyz, uint32_t nv, const uint32_t *idx, uint32_t nt,
                        const float *uv, const uint8_t *vrgb, const uint8_t *atlas, uint32_t aw, uint32_t ah,
                        const uint32_t *sem, const float *poses, uint32_t n, const float *intr,
                        uint32_t W, uint32_t H, uint8_t *rgb, float *depth, uint32_t *ids, uint32_t *cover,
                        int nthreads, float noise_sigma, uint64_t noise_seed, const uint32_t *agent_ids)
{
    return oracle_render_full(xyz, nv, idx, nt, uv, vrgb, atlas, aw, ah, sem, poses, n, intr, W, H, rgb, depth,
                              ids, cover, nthreads, noise_sigma, noise_seed, agent_ids, 0, NULL);
}
