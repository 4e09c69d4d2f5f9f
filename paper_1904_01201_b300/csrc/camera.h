// Camera setup of one view (step a1): the world-to-eye matrix of a pose and
// the world-space culling planes of its frustum. Compiled for the host (descriptor fill) and
// for the device (the actuation pass, which moves agents and rebuilds their
// cameras without a host round trip); both builds run the same IEEE double
// operations in the same order (no contraction on either side), so a pose
// yields the same float matrix wherever it is set up.
#pragma once

#include <cfloat>
#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define HSR_HD __host__ __device__ __forceinline__
#else
#define HSR_HD inline
#endif

namespace hsr {

constexpr double kPlaneMarginPx = 2.0;          // culling planes pushed out by this many pixels
constexpr double kPlaneMarginDepth = 1e-4;      // and the near / far planes by this many metres

HSR_HD bool finite_f(float v) { return v == v && v <= FLT_MAX && v >= -FLT_MAX; }

// M = [R^T | -R^T pos] of the unit quaternion (w, x, y, z) (world-from-camera;
// the camera looks down -Z with +Y up), R in double, each entry rounded once
// to float. False for non-finite input or |q| off 1 by more than 1e-3.
HSR_HD bool camera_from_pose(const float pos[3], const float quat[4], float M[12])
{
    for (int i = 0; i < 3; i++)
        if (!finite_f(pos[i])) return false;
    for (int i = 0; i < 4; i++)
        if (!finite_f(quat[i])) return false;
    double w = quat[0], x = quat[1], y = quat[2], z = quat[3];
    const double n = sqrt(((w * w + x * x) + y * y) + z * z);
    if (!(fabs(n - 1.0) <= 1e-3)) return false;
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
    const double px = pos[0], py = pos[1], pz = pos[2];
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) M[i * 4 + j] = (float)R[j][i];
        M[i * 4 + 3] = (float)(-((R[0][i] * px + R[1][i] * py) + R[2][i] * pz));
    }
    return true;
}

// World-space culling planes of a view (n . p + off >= 0 inside), double
// precision from the float matrix: the image borders pushed out by
// kPlaneMarginPx pixels and the near / far planes by kPlaneMarginDepth
// metres, so culling only removes geometry that cannot produce a sample.
HSR_HD void frustum_planes(const float M[12], double fx, double fy, double cx, double cy, double znear,
                           double zfar, uint32_t W, uint32_t H, float planes[24])
{
    const double m = kPlaneMarginPx;
    const double ne[6][3] = {{fx, 0, -(cx + m)},
                             {-fx, 0, -((double)W + m - cx)},
                             {0, -fy, -(cy + m)},
                             {0, fy, -((double)H + m - cy)},
                             {0, 0, -1},
                             {0, 0, 1}};
    const double oe[6] = {0, 0, 0, 0, -(znear - kPlaneMarginDepth), zfar + kPlaneMarginDepth};
    for (int k = 0; k < 6; k++) {
        for (int j = 0; j < 3; j++) {
            double nn = 0;
            for (int i = 0; i < 3; i++) nn += (double)M[i * 4 + j] * ne[k][i];
            planes[4 * k + j] = (float)nn;
        }
        double off = oe[k];
        for (int i = 0; i < 3; i++) off += (double)M[i * 4 + 3] * ne[k][i];
        planes[4 * k + 3] = (float)off;
    }
}

// Whether a view from `pos` of a scene inside the box [amin, amax] keeps
// every snapped coordinate inside +-2^30 sub-pixels, so that no triangle can
// need the guard band: any vertex (or near-clipped point) has |x_e|, |y_e| <=
// the distance R to the farthest box corner and d >= near, hence
// |256 s| <= 256 (f R / near + |c| + 2). Conservative; a call whose views
// all pass it shades without the guard-band path.
HSR_HD bool guard_free(const float amin[3], const float amax[3], const float pos[3], double fx, double fy, double cx,
                       double cy, double znear)
{
    double r2 = 0.0;
    for (int c = 0; c < 8; c++) {
        double d2 = 0.0;
        for (int k = 0; k < 3; k++) {
            const double v = (c >> k) & 1 ? amax[k] : amin[k];
            const double dd = v - (double)pos[k];
            d2 += dd * dd;
        }
        r2 = r2 > d2 ? r2 : d2;
    }
    const double R = sqrt(r2) * (1.0 + 1e-6) + 1e-6;
    const double f = fx > fy ? fx : fy;
    const double c = fabs(cx) > fabs(cy) ? fabs(cx) : fabs(cy);
    return 256.0 * (f * R / znear + c + 2.0) < 1073741824.0;
}

}  // namespace hsr
