// Host-side launch heuristics: the configuration a render call uses when no
// tuned one is registered for its signature.
#pragma once
#include <cstdint>

#include "hsr_internal.h"

namespace hsr {

// The configuration used when none was tuned for a call's signature: the
// defaults, with a single occlusion phase for small calls (under 16k
// (view, group) items, where the extra kernels of a phase cost more than the
// culling saves), and the large-triangle bins taking triangles above 32
// candidate pixels while the call's z-buffers stay within L2 (up to 2^24
// pixels over all views), above 256 beyond (the values the autotuner picks
// on the 64-view 256^2 and 256-view 512^2 workloads: with z-buffers far
// larger than L2 the separate pass loses the locality of the warps that set
// the triangles up).
inline LaunchCfg default_launch_cfg(uint64_t items, uint64_t pixels)
{
    LaunchCfg c;
    if (items < 16384) c.n_phases = 1;
    c.bin_px = pixels <= (1ull << 24) ? 32u : 256u;
    return c;
}

}  // namespace hsr
