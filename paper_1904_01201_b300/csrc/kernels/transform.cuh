// K1 — per-(agent, vertex) transform to eye space and projection to 24.8 fixed point.
//
// Rule (reading of Sec. 4 "Sensory input": pinhole camera at the agent pose;
// the paper fixes no arithmetic): x_e = fma(M00,x, fma(M01,y, fma(M02,z, M03)))
// and likewise y_e, z_e; planar depth d = -z_e; q = 1/d;
// sx = fma(fx, x_e*q, cx), sy = fma(-fy, y_e*q, cy); X = rint(256 sx), Y = rint(256 sy).
// Every operation is a correctly rounded single IEEE op (explicit intrinsics,
// and the file is compiled with --fmad=false), so results are reproducible.
#pragma once
#include "../hsr_internal.h"

namespace hsr {

// Per meshlet vertex, cached in shared memory for the warp that owns the
// meshlet, split so that the common path reads one 16-byte record:
//   hot  — snapped X, Y and q, and d; q = 0 marks a vertex that is in front
//          of the near plane or whose snap leaves the fixed-point range (its
//          triangles take the clipping path);
//   cold — eye-space x, y and the caller vertex index (near-clip path only).
struct alignas(16) EyeHot {
    int X, Y;
    float q, d;
};
struct alignas(16) EyeCold {
    float xe, ye;
    uint32_t gid;
    uint32_t pad_;
};

__device__ __forceinline__ void eye_transform(const float *M, float x, float y, float z,
                                              float &xe, float &ye, float &d)
{
    xe = __fmaf_rn(M[0], x, __fmaf_rn(M[1], y, __fmaf_rn(M[2], z, M[3])));
    ye = __fmaf_rn(M[4], x, __fmaf_rn(M[5], y, __fmaf_rn(M[6], z, M[7])));
    const float ze = __fmaf_rn(M[8], x, __fmaf_rn(M[9], y, __fmaf_rn(M[10], z, M[11])));
    d = -ze;
}

// Projection and snap of a point with d >= near (> 0). Returns false when a
// snapped coordinate would lie at or beyond +-2^30 sub-pixels (or is not a
// number): such a triangle is clipped to the guard band first (setup.cuh).
// Near 2^30 floats are multiples of 64, so testing the product before
// rounding decides exactly as testing rint of it.
__device__ __forceinline__ bool project_snap(float xe, float ye, float d, float fx, float fy, float cx, float cy,
                                             float &q, int &X, int &Y)
{
    q = __frcp_rn(d);
    const float sx = __fmaf_rn(fx, __fmul_rn(xe, q), cx);
    const float sy = __fmaf_rn(-fy, __fmul_rn(ye, q), cy);
    const float fsx = __fmul_rn(sx, 256.0f), fsy = __fmul_rn(sy, 256.0f);
    X = __float2int_rn(fsx);
    Y = __float2int_rn(fsy);
    return fabsf(fsx) < 1073741824.0f && fabsf(fsy) < 1073741824.0f;
}

}  // namespace hsr
