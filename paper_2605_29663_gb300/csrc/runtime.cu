// runtime.cu -- footprint objects, contexts, scratch and status strings of
// the EXACT-MPPI C ABI.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "internal.h"

namespace {

// Orientation of (a, b, c): sign of the cross product (b - a) x (c - a).
int orient(double ax, double ay, double bx, double by, double cx, double cy) {
    const double v = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    return (v > 0.0) - (v < 0.0);
}

// c collinear with segment ab: does it lie within the segment's box?
bool on_segment(double ax, double ay, double bx, double by, double cx, double cy) {
    return fmin(ax, bx) <= cx && cx <= fmax(ax, bx) && fmin(ay, by) <= cy && cy <= fmax(ay, by);
}

bool segments_touch(const double *p, const double *q, const double *r, const double *s) {
    const int o1 = orient(p[0], p[1], q[0], q[1], r[0], r[1]);
    const int o2 = orient(p[0], p[1], q[0], q[1], s[0], s[1]);
    const int o3 = orient(r[0], r[1], s[0], s[1], p[0], p[1]);
    const int o4 = orient(r[0], r[1], s[0], s[1], q[0], q[1]);
    if (o1 != o2 && o3 != o4) return true;
    if (o1 == 0 && on_segment(p[0], p[1], q[0], q[1], r[0], r[1])) return true;
    if (o2 == 0 && on_segment(p[0], p[1], q[0], q[1], s[0], s[1])) return true;
    if (o3 == 0 && on_segment(r[0], r[1], s[0], s[1], p[0], p[1])) return true;
    if (o4 == 0 && on_segment(r[0], r[1], s[0], s[1], q[0], q[1])) return true;
    return false;
}

// Simple-polygon check (O(n^2)): no repeated vertex, non-adjacent edges do
// not meet, adjacent edges do not fold back onto each other, non-zero area.
int check_simple(const double *v, int n) {
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (v[2 * i] == v[2 * j] && v[2 * i + 1] == v[2 * j + 1]) return EXACT_ENOTSIMPLE;
    for (int i = 0; i < n; ++i) {
        const double *a = v + 2 * i, *b = v + 2 * ((i + 1) % n);
        for (int j = i + 1; j < n; ++j) {
            const double *c = v + 2 * j, *d = v + 2 * ((j + 1) % n);
            const bool adjacent = (j == i + 1) || (i == 0 && j == n - 1);
            if (adjacent) {
                // shared vertex: the far end of one edge must not lie on the other
                const double *far_i = (j == i + 1) ? a : b;
                const double *far_j = (j == i + 1) ? d : c;
                if (orient(a[0], a[1], b[0], b[1], far_j[0], far_j[1]) == 0 &&
                    on_segment(a[0], a[1], b[0], b[1], far_j[0], far_j[1]))
                    return EXACT_ENOTSIMPLE;
                if (orient(c[0], c[1], d[0], d[1], far_i[0], far_i[1]) == 0 &&
                    on_segment(c[0], c[1], d[0], d[1], far_i[0], far_i[1]))
                    return EXACT_ENOTSIMPLE;
            } else if (segments_touch(a, b, c, d)) {
                return EXACT_ENOTSIMPLE;
            }
        }
    }
    double area2 = 0.0;
    for (int i = 0; i < n; ++i) {
        const double *a = v + 2 * i, *b = v + 2 * ((i + 1) % n);
        area2 += a[0] * b[1] - a[1] * b[0];
    }
    if (!(fabs(area2) > 1e-12)) return EXACT_ENOTSIMPLE;
    return EXACT_OK;
}

int poly_bucket(int n) {
    static const int sizes[] = {4, 6, 8, 10, 12, 14, 16, 24, 32, 40, 48, 56, 64};
    for (int s : sizes)
        if (n <= s) return s;
    return -1;
}

int rect_bucket(int n) {
    static const int sizes[] = {1, 2, 3, 4, 5, 6, 7, 8};
    for (int s : sizes)
        if (n <= s) return s;
    return -1;
}

}  // namespace

extern "C" const char *exact_status_string(int status) {
    switch (status) {
    case EXACT_OK: return "ok";
    case EXACT_EINVAL: return "invalid argument";
    case EXACT_ENOTSIMPLE: return "polygon is not simple";
    case EXACT_ECAPACITY: return "size beyond the supported maximum";
    case EXACT_ECUDA: return "CUDA runtime error";
    case EXACT_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown status";
    }
}

extern "C" int exact_footprint_create(int kind, const float *host_data, int n, exact_footprint **out) {
    if (!out || !host_data) return EXACT_EINVAL;
    *out = nullptr;
    const int per = kind == EXACT_FP_POLYGON ? 2 : kind == EXACT_FP_RECTS ? 4 : 0;
    if (per == 0 || n <= 0) return EXACT_EINVAL;
    for (int i = 0; i < n * per; ++i)
        if (!isfinite(host_data[i])) return EXACT_EINVAL;
    exact_footprint *fp = new (std::nothrow) exact_footprint();
    if (!fp) return EXACT_EINVAL;
    memset(fp, 0, sizeof(*fp));
    fp->kind = kind;
    fp->n = n;
    if (kind == EXACT_FP_POLYGON) {
        if (n < 3) { delete fp; return EXACT_EINVAL; }
        if (n > EXACT_MAX_POLY_VERTICES) { delete fp; return EXACT_ECAPACITY; }
        double v[2 * EXACT_MAX_POLY_VERTICES];
        for (int i = 0; i < 2 * n; ++i) v[i] = (double)host_data[i] + 0.0;  // -0 -> +0
        const int rc = check_simple(v, n);
        if (rc != EXACT_OK) { delete fp; return rc; }
        const int E = poly_bucket(n);
        fp->n_pad = E;
        for (int b = 0; b < E; ++b) {
            const int ib = b < n ? b : 0;
            const int nb = (b + 1) < n ? b + 1 : 0;   // padded vertices repeat vertex 0
            const double vx = v[2 * ib], vy = v[2 * ib + 1];
            const double wx = v[2 * nb], wy = v[2 * nb + 1];
            const double ex = (b < n) ? wx - vx : 0.0, ey = (b < n) ? wy - vy : 0.0;
            const double len2 = ex * ex + ey * ey;
            fp->vx[b] = (float)vx;
            fp->vy[b] = (float)vy;
            fp->ex[b] = (float)ex;
            fp->ey[b] = (float)ey;
            fp->exn[b] = len2 > 0.0 ? (float)(ex / len2) : 0.f;
            fp->eyn[b] = len2 > 0.0 ? (float)(ey / len2) : 0.f;
            fp->kx[b] = ey != 0.0 ? (float)(ex / ey) : 0.f;
        }
    } else {
        if (n > EXACT_MAX_RECTS) { delete fp; return EXACT_ECAPACITY; }
        for (int j = 0; j < n; ++j)
            if (!(host_data[4 * j + 2] > 0.f) || !(host_data[4 * j + 3] > 0.f)) { delete fp; return EXACT_EINVAL; }
        const int R = rect_bucket(n);
        fp->n_pad = R;
        for (int j = 0; j < R; ++j) {
            const int s = j < n ? j : 0;   // padded boxes repeat box 0
            fp->cx[j] = host_data[4 * s] + 0.f;
            fp->cy[j] = host_data[4 * s + 1] + 0.f;
            fp->sx[j] = host_data[4 * s + 2];
            fp->sy[j] = host_data[4 * s + 3];
        }
    }
    // bounding circle of the footprint (centre of the bounding box, largest
    // vertex / box-corner distance) and the bounding box itself (half
    // extents about that centre), both rounded outwards so that the float
    // circle and box contain the footprint, for the bounds that let the
    // MPPI kernels skip far point chunks and far points
    double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
    auto corners = [&](auto &&visit) {
        if (kind == EXACT_FP_POLYGON) {
            for (int b = 0; b < n; ++b) visit((double)host_data[2 * b], (double)host_data[2 * b + 1]);
        } else {
            for (int j = 0; j < n; ++j)
                for (int sx = -1; sx <= 1; sx += 2)
                    for (int sy = -1; sy <= 1; sy += 2)
                        visit((double)host_data[4 * j] + sx * (double)host_data[4 * j + 2],
                              (double)host_data[4 * j + 1] + sy * (double)host_data[4 * j + 3]);
        }
    };
    corners([&](double x, double y) {
        lo[0] = fmin(lo[0], x); lo[1] = fmin(lo[1], y);
        hi[0] = fmax(hi[0], x); hi[1] = fmax(hi[1], y);
    });
    const double bcx = 0.5 * (lo[0] + hi[0]), bcy = 0.5 * (lo[1] + hi[1]);
    double r2 = 0.0;
    corners([&](double x, double y) { r2 = fmax(r2, (x - bcx) * (x - bcx) + (y - bcy) * (y - bcy)); });
    fp->bcx = (float)bcx;
    fp->bcy = (float)bcy;
    fp->brad = (float)(sqrt(r2) * (1.0 + 1e-6) + 1e-6 + fabs((double)fp->bcx - bcx) + fabs((double)fp->bcy - bcy));
    const double shift = fabs((double)fp->bcx - bcx) + fabs((double)fp->bcy - bcy);
    fp->bhx = (float)(0.5 * (hi[0] - lo[0]) * (1.0 + 1e-6) + 1e-6 + shift);
    fp->bhy = (float)(0.5 * (hi[1] - lo[1]) * (1.0 + 1e-6) + 1e-6 + shift);
    *out = fp;
    return EXACT_OK;
}

extern "C" void exact_footprint_destroy(exact_footprint *fp) { delete fp; }

extern "C" int exact_footprint_info(const exact_footprint *fp, int *kind, int *n) {
    if (!fp) return EXACT_EINVAL;
    if (kind) *kind = fp->kind;
    if (n) *n = fp->n;
    return EXACT_OK;
}

namespace exact {

int current_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

int ensure_scratch(exact_ctx *ctx, size_t bytes) {
    if (!ctx) return EXACT_EINVAL;
    if (bytes <= ctx->scratch_bytes) return EXACT_OK;
    bytes = align_up(bytes, (size_t)1 << 20);
    if (ctx->scratch) {
        if (cudaDeviceSynchronize() != cudaSuccess) return EXACT_ECUDA;
        cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
    }
    if (cudaMalloc(&ctx->scratch, bytes) != cudaSuccess) {
        ctx->scratch = nullptr;
        return EXACT_ECUDA;
    }
    // counters and flags in the arena must start at zero
    if (cudaMemset(ctx->scratch, 0, bytes) != cudaSuccess) return EXACT_ECUDA;
    ctx->scratch_bytes = bytes;
    ctx->mppi_layout = -1;
    return EXACT_OK;
}

}  // namespace exact

extern "C" int exact_ctx_create(exact_ctx **out) {
    if (!out) return EXACT_EINVAL;
    *out = nullptr;
    exact_ctx *ctx = new (std::nothrow) exact_ctx();
    if (!ctx) return EXACT_EINVAL;
    if (cudaGetDevice(&ctx->device) != cudaSuccess) { delete ctx; return EXACT_ECUDA; }
    ctx->sm_count = exact::current_sm_count();
    if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess) { delete ctx; return EXACT_ECUDA; }
    if (cudaMalloc(&ctx->d_stats, sizeof(exact_cycle_stats)) != cudaSuccess) {
        cudaFree(ctx->d_err);
        delete ctx;
        return EXACT_ECUDA;
    }
    if (cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_stats, 0, sizeof(exact_cycle_stats)) != cudaSuccess) {
        cudaFree(ctx->d_err);
        cudaFree(ctx->d_stats);
        delete ctx;
        return EXACT_ECUDA;
    }
    *out = ctx;
    return EXACT_OK;
}

extern "C" void exact_ctx_destroy(exact_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_stats) cudaFree(ctx->d_stats);
    delete ctx;
}

extern "C" int exact_ctx_enable_stats(exact_ctx *ctx, int enable) {
    if (!ctx) return EXACT_EINVAL;
    ctx->stats = enable != 0;
    return EXACT_OK;
}

extern "C" int exact_ctx_get_stats(exact_ctx *ctx, exact_cycle_stats *out, void *stream) {
    if (!ctx || !out) return EXACT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // read, then zero the two counters (the first 16 bytes), in stream order
    if (cudaMemcpyAsync(out, ctx->d_stats, sizeof(exact_cycle_stats), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(ctx->d_stats, 0, 2 * sizeof(long long), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return EXACT_ECUDA;
    return EXACT_OK;
}

extern "C" int exact_ctx_get_error(exact_ctx *ctx, void *stream) {
    if (!ctx) return EXACT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int err = 0;
    // read and clear in stream order, then wait for this stream only
    if (cudaMemcpyAsync(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return EXACT_ECUDA;
    return err;
}
