// Actuation pass of a step batch (Sec. 4 "Agent embodiment and action space":
// stop, move_forward 0.25 m, turn_left / turn_right 10 degrees, idealised).
// One thread per view: it applies the view's action to its agent's
// device-resident pose, then sets up the view's camera from the new pose, so
// a step batch needs only action ids from the host.
//
// Rules (double arithmetic from the float pose, one rounding to float per
// stored component):
//  * forward: heading R (0, 0, -1) of the normalised quaternion with its
//    vertical component dropped, h = (-2(xz + wy), -(1 - 2(x^2 + y^2)));
//    p' = p + step h / |h| on x and z, rounded to float; refused when
//    |h| = 0, when the grid cell (floor((x - x0)/cell), floor((z - z0)/cell))
//    of p' lies outside the grid or is not navigable (no sliding), or when
//    p' would take the scene out of the fixed-point range of the raster.
//  * turn: q' = r q, r = (cos(t/2), 0, sin(t/2), 0) about world +Y
//    (t = +angle for left, -angle for right), then q' / |q'|.
//  * stop: unchanged.
#include <cuda_runtime.h>

#include "camera.h"
#include "hsr_internal.h"

namespace hsr {

namespace {

constexpr int kActuateThreads = 128;

__device__ bool navigable(const NavDev &nav, float x, float z)
{
    const double ci = floor(((double)x - (double)nav.x0) / (double)nav.cell);
    const double ck = floor(((double)z - (double)nav.z0) / (double)nav.cell);
    if (!(ci >= 0.0 && ci < (double)nav.nx && ck >= 0.0 && ck < (double)nav.nz)) return false;
    return nav.grid[(size_t)ck * nav.nx + (size_t)ci] != 0;
}

__global__ void __launch_bounds__(kActuateThreads) actuate_kernel(const Params p)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.dyn[0]) return;
    const AgentsDev *ag = reinterpret_cast<const AgentsDev *>((uint64_t)p.dyn[6] | ((uint64_t)p.dyn[7] << 32));
    if (!ag) return;
    // the descriptors live in this batch's own device buffer; the pass fills
    // in the camera part of each view before any render kernel reads it
    View &v = const_cast<View &>(p.views[i]);
    const uint32_t a = v.state;
    if (a >= ag->n_agents || v.scene >= ag->n_scenes) return;
    float *st = ag->pose + 7 * (size_t)a;
    float pose[7];
#pragma unroll
    for (int k = 0; k < 7; k++) pose[k] = st[k];
    double w = pose[3], x = pose[4], y = pose[5], z = pose[6];
    const double n = sqrt(((w * w + x * x) + y * y) + z * z);
    w /= n; x /= n; y /= n; z /= n;
    if (v.action == HSR_ACTION_MOVE_FORWARD) {
        const double hx = -2.0 * (x * z + w * y);
        const double hz = -(1.0 - 2.0 * (x * x + y * y));
        const double len = sqrt(hx * hx + hz * hz);
        if (len > 0.0) {
            const float nx = (float)((double)pose[0] + ag->step * (hx / len));
            const float nz = (float)((double)pose[2] + ag->step * (hz / len));
            const NavDev &nav = ag->nav[v.scene];
            if (navigable(nav, nx, nz)) {
                pose[0] = nx;
                pose[2] = nz;
            }
        }
    } else if (v.action == HSR_ACTION_TURN_LEFT || v.action == HSR_ACTION_TURN_RIGHT) {
        const int r = v.action == HSR_ACTION_TURN_LEFT ? 0 : 1;
        const double c = ag->c_turn[r], s = ag->s_turn[r];
        const double w2 = c * w - s * y;
        const double x2 = c * x + s * z;
        const double y2 = c * y + s * w;
        const double z2 = c * z - s * x;
        const double n2 = sqrt(((w2 * w2 + x2 * x2) + y2 * y2) + z2 * z2);
        pose[3] = (float)(w2 / n2);
        pose[4] = (float)(x2 / n2);
        pose[5] = (float)(y2 / n2);
        pose[6] = (float)(z2 / n2);
    }
#pragma unroll
    for (int k = 0; k < 7; k++) st[k] = pose[k];
    camera_from_pose(pose, pose + 3, v.M);
    frustum_planes(v.M, p.fx, p.fy, p.cx, p.cy, p.znear, p.zfar, p.width, p.height, v.planes);
    v.pos[0] = pose[0];
    v.pos[1] = pose[1];
    v.pos[2] = pose[2];
}

}  // namespace

cudaError_t launch_actuate(const Params &p, uint32_t n_cap, cudaStream_t stream)
{
    const uint32_t blocks = (n_cap + kActuateThreads - 1) / kActuateThreads;
    actuate_kernel<<<blocks, kActuateThreads, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace hsr
