// mppi_predicted.cu -- mppi_step_predicted: the control cycle of mppi_step
// with time-indexed obstacle predictions (the extension named in Sec. V-F):
// every obstacle point carries a velocity and each horizon step's signed
// distances are taken against the constant-velocity prediction o + t_h v at
// the time t_h of the scored state, instead of the current observation only.
// The kernels are those of mppi.cu instantiated for (position, velocity)
// points; this file holds only their instantiation, so it compiles in
// parallel with mppi.cu.
#include "mppi_kernels.cuh"

namespace exact {

int launch_cycle_moving(const SceneView &V, const exact_footprint *fp, cudaStream_t st, bool pdl,
                        const float4 *circ, int sms) {
    return launch_cycle_t<true, 4>(V, fp, st, pdl, circ, sms);
}

}  // namespace exact

extern "C" int mppi_step_predicted(exact_ctx *ctx, const float *state, const float *cloud, const float *velocity,
                                   const uint8_t *mask, int n_points, const float *waypoints, int n_wp, float *U,
                                   const float *noise, const exact_footprint *fp, const exact_mppi_params *params,
                                   float *u_star, float *costs, float *weights, int *valid, float *U_upd,
                                   float *dmin, void *stream) {
    if (n_points > 0 && !velocity) return EXACT_EINVAL;
    return exact::mppi_step_impl(ctx, state, cloud, velocity, mask, n_points, waypoints, n_wp, U, noise, fp, params,
                                 u_star, costs, weights, valid, U_upd, dmin, stream);
}
