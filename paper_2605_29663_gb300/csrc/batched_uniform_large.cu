// batched_uniform_large.cu -- polygons of 24 to 64 edges; see batched_uniform.cuh.
#include "batched_uniform.cuh"

namespace exact {

int launch_uniform_large(exact_batch *b, const SceneDev *table, cudaStream_t st, bool validate) {
    const exact_footprint *fp = &b->fp;
    auto go = [&](auto fpc) -> int {
        return validate ? launch_uniform_validate_t(b, st, fpc) : launch_uniform_sample_t(b, table, st, fpc);
    };
    if (fp->kind == EXACT_FP_POLYGON) {
        switch (fp->n_pad) {
        case 24: return go(make_poly<24>(fp));
        case 32: return go(make_poly<32>(fp));
        case 40: return go(make_poly<40>(fp));
        case 48: return go(make_poly<48>(fp));
        case 56: return go(make_poly<56>(fp));
        case 64: return go(make_poly<64>(fp));
        default: return EXACT_EINVAL;
        }
    }
    return EXACT_EINVAL;
}

}  // namespace exact
