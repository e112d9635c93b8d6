// noalloc.cu -- mppi_step_noalloc: the control cycle of mppi_step with its
// scratch in a fixed, file-scope device array instead of a context arena.
//
// Some callers cannot allocate device memory: a controller that must not
// call cudaMalloc once its real-time loop has started, code running while a
// stream is being captured into a CUDA graph (allocation is not allowed
// there), or a host program whose device memory is owned by someone else's
// allocator.  This entry point serves them: the caller still passes every
// input and output, and the scratch lives in g_noalloc_arena, which every
// GPU that loads the library holds until the process exits.
#include <mutex>

#include "mppi_cycle.cuh"

namespace exact {
int check_params(const exact_mppi_params *p);
MppiP to_device_params(const exact_mppi_params *p);
int launch_cycle(const SceneView &V, const exact_footprint *fp, cudaStream_t st, bool pdl, const float4 *circ,
                 int sms);
}  // namespace exact

using namespace exact;

// Scratch of the allocation-free entry point.  Device code could name it
// directly; host code must not (there the name is a host-side stand-in, not
// a device address), so its address is looked up per device below.
static __device__ __align__(256) unsigned char g_noalloc_arena[EXACT_NOALLOC_ARENA_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Device address of g_noalloc_arena on the current device (looked up once per
// device, with that device current) and its SM count.
int arena_for_current_device(void **addr, int *sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EXACT_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return EXACT_ECAPACITY;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_arena) != cudaSuccess || !p) return EXACT_ECUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return EXACT_ECUDA;
        g_addr[dev] = p;
        g_sms[dev] = n;
    }
    *addr = g_addr[dev];
    *sms = g_sms[dev];
    return EXACT_OK;
}
}  // namespace

extern "C" int mppi_step_noalloc(const float *state, const float *cloud, const uint8_t *mask, int n_points,
                                 const float *waypoints, int n_wp, float *U, const float *noise,
                                 const exact_footprint *fp, const exact_mppi_params *params, float *u_star,
                                 float *costs, float *weights, int *valid, float *U_upd, float *dmin,
                                 void *stream) {
    if (!fp || !state || !U || !noise || !waypoints || n_wp < 1 || n_points < 0) return EXACT_EINVAL;
    if (n_points > 0 && (!cloud || ((uintptr_t)cloud & 7u) != 0)) return EXACT_EINVAL;
    int rc = check_params(params);
    if (rc != EXACT_OK) return rc;
    void *arena = nullptr;
    int sms = 0;
    if ((rc = arena_for_current_device(&arena, &sms)) != EXACT_OK) return rc;
    const MppiP P = to_device_params(params);
    const int parts = parts_for(P.K, P.T, sms);
    if (kArenaHeader + scene_scratch_bytes(P.K, P.T, parts) > (size_t)EXACT_NOALLOC_ARENA_BYTES)
        return EXACT_ECAPACITY;
    SceneView V;
    V.P = P;
    V.state = state;
    V.pts = reinterpret_cast<const float2 *>(cloud);
    V.mask = mask;
    V.N = n_points;
    V.wp = waypoints;
    V.W = n_wp;
    V.U = U;
    V.noise = noise;
    V.u_star = u_star; V.costs = costs; V.weights = weights; V.U_upd_out = U_upd; V.dmin = dmin; V.valid = valid;
    V.nom_cost = nullptr;
    V.err = nullptr;   // no context: device-side errors are not recorded
    V.vel = nullptr;
    V.hdr = reinterpret_cast<ArenaHeader *>(arena);
    carve_scene(V, static_cast<char *>(arena) + kArenaHeader, P.K, P.T, parts);
    V.upd_chunk = upd_chunk_for(P.K, P.T, P.nu);
    V.upd_blocks = upd_blocks_for(P.K, P.T, P.nu);
    V.val_chunks = val_chunks_for(n_points);
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: zero the control words
    // and counters that must start at zero (no allocation involved)
    if (cudaMemsetAsync(arena, 0, kArenaHeader, st) != cudaSuccess) return EXACT_ECUDA;
    if (parts > 1 && cudaMemsetAsync(V.tk, 0, (size_t)P.K * sizeof(unsigned), st) != cudaSuccess) return EXACT_ECUDA;
    return launch_cycle(V, fp, st, false, nullptr, sms);
}
