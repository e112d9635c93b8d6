// hybrid.cu -- hybrid-mode EXACT-MPPI (Sec. IV-F, Algorithm 2, steps 1-2).
//
// The modes of one robot are the scenes of one batch plan: a step runs
// Algorithm 1 for every mode in the batched launch set (persistent sample
// kernel, update, validation with the nominal's cost), then one single-thread
// selection kernel applies the switch penalty, the validation exclusion, the
// safe stop and the cooldown, and writes the chosen mode's first command.
// Everything stays on the device, so a whole hybrid cycle is capturable.
#include <new>

#include "mppi_cycle.cuh"

namespace exact {

struct HybridTable {
    const int *valid[EXACT_MAX_MODES];
    const float *nom[EXACT_MAX_MODES];
    const float *ustar[EXACT_MAX_MODES];
    int nu[EXACT_MAX_MODES];
    int M;
    float lambda_switch;
    int cool_max;
};

__global__ void hybrid_select_kernel(const HybridTable t, int *__restrict__ state, float *__restrict__ u_out,
                                     float *__restrict__ Jbar) {
    grid_dep_wait();   // launched behind the validation phase: its results are ready now
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int m_prev = state[0], tau = state[1];
    int best = -1;
    float best_j = finf();
    for (int m = 0; m < t.M; ++m) {
        const float jb = *t.valid[m] ? *t.nom[m] + (m != m_prev ? t.lambda_switch : 0.f) : finf();
        if (Jbar) Jbar[m] = jb;
        if (jb < best_j) { best_j = jb; best = m; }   // strict: the lowest index wins ties
    }
    if (best < 0) {   // every candidate failed validation: safe stop
        u_out[0] = u_out[1] = u_out[2] = 0.f;
        state[2] = 1;
        return;
    }
    int ms = best;
    if (tau > 0 && ms != m_prev && m_prev >= 0 && m_prev < t.M) ms = m_prev;   // cooldown
    state[1] = ms != m_prev ? t.cool_max : (tau > 0 ? tau - 1 : 0);
    state[0] = ms;
    state[2] = 0;
    for (int j = 0; j < 3; ++j) u_out[j] = j < t.nu[ms] ? t.ustar[ms][j] : 0.f;
}

}  // namespace exact

using namespace exact;

struct exact_hybrid {
    exact_batch *batch = nullptr;
    void *dev = nullptr;   // the object's own valid / nominal-cost words
    HybridTable tab;
};

extern "C" int exact_hybrid_create(int n_modes, const exact_scene *modes, const exact_hybrid_params *hp,
                                   exact_hybrid **out) {
    if (!out) return EXACT_EINVAL;
    *out = nullptr;
    if (!modes || !hp || n_modes < 1) return EXACT_EINVAL;
    if (n_modes > EXACT_MAX_MODES) return EXACT_ECAPACITY;
    if (!(hp->lambda_switch >= 0.f) || !(hp->lambda_switch < 3.0e38f) || hp->cool_max < 0) return EXACT_EINVAL;
    exact_hybrid *h = new (std::nothrow) exact_hybrid();
    if (!h) return EXACT_EINVAL;
    if (cudaMalloc(&h->dev, 2 * EXACT_MAX_MODES * sizeof(int)) != cudaSuccess) {
        delete h;
        return EXACT_ECUDA;
    }
    int *own_valid = static_cast<int *>(h->dev);
    float *own_nom = reinterpret_cast<float *>(own_valid + EXACT_MAX_MODES);
    exact_scene sc[EXACT_MAX_MODES];
    for (int m = 0; m < n_modes; ++m) {
        sc[m] = modes[m];
        if (!sc[m].valid) sc[m].valid = own_valid + m;
        if (!sc[m].nom_cost) sc[m].nom_cost = own_nom + m;
        h->tab.valid[m] = sc[m].valid;
        h->tab.nom[m] = sc[m].nom_cost;
        h->tab.ustar[m] = sc[m].u_star;
        h->tab.nu[m] = sc[m].params.n_u;
    }
    for (int m = n_modes; m < EXACT_MAX_MODES; ++m) {
        h->tab.valid[m] = nullptr;
        h->tab.nom[m] = nullptr;
        h->tab.ustar[m] = nullptr;
        h->tab.nu[m] = 0;
    }
    h->tab.M = n_modes;
    h->tab.lambda_switch = hp->lambda_switch;
    h->tab.cool_max = hp->cool_max;
    const int rc = exact_batch_create(n_modes, sc, &h->batch);
    if (rc != EXACT_OK) {
        cudaFree(h->dev);
        delete h;
        return rc;
    }
    *out = h;
    return EXACT_OK;
}

extern "C" void exact_hybrid_destroy(exact_hybrid *h) {
    if (!h) return;
    exact_batch_destroy(h->batch);   // synchronises the device
    cudaFree(h->dev);
    delete h;
}

extern "C" exact_batch *exact_hybrid_batch(exact_hybrid *h) { return h ? h->batch : nullptr; }

extern "C" int mppi_step_hybrid(exact_hybrid *h, int *mode_state, float *u_out, float *Jbar, void *stream) {
    if (!h || !mode_state || !u_out) return EXACT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int rc = mppi_step_batched(h->batch, stream);
    if (rc != EXACT_OK) return rc;
    return cuda_status(launch_dependent(hybrid_select_kernel, 1u, 32u, 0, st, (const HybridTable)h->tab, mode_state,
                                        u_out, Jbar));
}
