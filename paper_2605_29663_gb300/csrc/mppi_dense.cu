// mppi_dense.cu -- the static-cloud control cycle with the sample kernel
// capped at 64 registers (four resident blocks per SM), used when the sample
// grid spans several waves; see mppi_kernels.cuh.  Only the instantiation
// lives here, so it compiles in parallel with mppi.cu.
#include "mppi_kernels.cuh"

namespace exact {

int launch_cycle_dense(const SceneView &V, const exact_footprint *fp, cudaStream_t st, bool pdl,
                       const float4 *circ, int sms) {
    return launch_cycle_t<false, 4>(V, fp, st, pdl, circ, sms);
}

}  // namespace exact
