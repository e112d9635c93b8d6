// batched_uniform_small.cu -- rectangle covers and polygons of up to 16 edges; see batched_uniform.cuh.
#include "batched_uniform.cuh"

namespace exact {

int launch_uniform_small(exact_batch *b, const SceneDev *table, cudaStream_t st, bool validate) {
    const exact_footprint *fp = &b->fp;
    auto go = [&](auto fpc) -> int {
        return validate ? launch_uniform_validate_t(b, st, fpc) : launch_uniform_sample_t(b, table, st, fpc);
    };
    if (fp->kind == EXACT_FP_POLYGON) {
        switch (fp->n_pad) {
        case 4: return go(make_poly<4>(fp));
        case 6: return go(make_poly<6>(fp));
        case 8: return go(make_poly<8>(fp));
        case 10: return go(make_poly<10>(fp));
        case 12: return go(make_poly<12>(fp));
        case 14: return go(make_poly<14>(fp));
        case 16: return go(make_poly<16>(fp));
        default: return EXACT_EINVAL;
        }
    }
    switch (fp->n_pad) {
        case 1: return go(make_rect<1>(fp));
        case 2: return go(make_rect<2>(fp));
        case 3: return go(make_rect<3>(fp));
        case 4: return go(make_rect<4>(fp));
        case 5: return go(make_rect<5>(fp));
        case 6: return go(make_rect<6>(fp));
        case 7: return go(make_rect<7>(fp));
        case 8: return go(make_rect<8>(fp));
    default: return EXACT_EINVAL;
    }
}

}  // namespace exact
