// mppi_points.cu -- the static-cloud control cycle for small clouds without
// a d_min output: the sample kernel is capped at 64 registers and holds only
// the point-level pruning path (kPathPoints), which keeps the code each block
// fetches once per cycle small; see mppi_kernels.cuh.  Only the
// instantiation lives here, so it compiles in parallel with mppi.cu.
#include "mppi_kernels.cuh"

namespace exact {

int launch_cycle_points(const SceneView &V, const exact_footprint *fp, cudaStream_t st, bool pdl,
                        const float4 *circ, int sms) {
    return launch_cycle_t<false, 4, kPathPoints>(V, fp, st, pdl, circ, sms);
}

}  // namespace exact
