// slab.cu -- row slabs: one grid split across ranks, with halo rows exchanged
// between temporal blocks.
//
// The paper decomposes the grid into tiles, one per processing element, pads
// each tile with a halo (Sec. IV-A) and swaps halos between neighbours before
// every step (Sec. IV-B..IV-D).  On GPUs the counterpart is a 1-D row-slab
// decomposition: rank p owns rows [y0, y1) of the ny x nx grid and keeps G =
// radius * S ghost rows above and below them, where S is the number of steps
// between two exchanges.  Because full-width rows are exchanged, the corner
// values a box stencil needs come along, and the paper's two-stage corner
// forwarding is not needed.
//
// A slab step runs S (or fewer) Jacobi steps on the whole slab buffer, ghost
// rows included, treating the buffer as a grid of its own: the rows next to
// an exchanged edge of the buffer see wrong neighbours (zeros, or the far edge
// of the buffer for the periodic rule), and that error moves inward by at most
// `radius` rows per step, so after s <= S steps it is confined to the G ghost
// rows and every owned row is exact.  Edges of the global grid under the zero
// rule get no ghost rows: there the buffer edge is the grid edge, and the
// kernels' frozen zero halo is the right boundary at every sub-step.  The
// arithmetic per point is that of stencil_run, so the owned rows are
// bit-identical to the same rows of a single-domain run (FP32 storage; BF16
// and FP16 storage round once per launch, so they match when both runs use the
// same launch depths).
#include <cuda_runtime.h>

#include <new>
#include <string>

#include "../../include/stencil.h"

namespace {

thread_local std::string g_slab_error;

stencil_status_t sfail(stencil_status_t st, const std::string& msg) {
    g_slab_error = msg;
    return st;
}

}  // namespace

struct stencil_slab {
    stencil_plan_t* plan = nullptr;
    stencil_slab_info_t info{};
};

extern "C" {

const char* stencil_slab_last_error(void) { return g_slab_error.c_str(); }

stencil_status_t stencil_slab_geometry(int64_t ny, int64_t nx, int64_t y0, int64_t y1, int radius,
                                       int boundary, int64_t steps_per_exchange,
                                       stencil_slab_info_t* info) {
    if (!info) return sfail(STENCIL_ERR_INVALID_ARG, "info is NULL");
    if (ny < 1 || nx < 1) return sfail(STENCIL_ERR_INVALID_ARG, "ny and nx must be >= 1");
    if (y0 < 0 || y1 > ny || y0 >= y1) return sfail(STENCIL_ERR_INVALID_ARG, "need 0 <= y0 < y1 <= ny");
    if (radius < 1 || radius > 3) return sfail(STENCIL_ERR_INVALID_ARG, "radius must be in 1..3");
    if (boundary != STENCIL_BOUNDARY_ZERO && boundary != STENCIL_BOUNDARY_PERIODIC)
        return sfail(STENCIL_ERR_INVALID_ARG, "bad boundary");
    if (steps_per_exchange < 1 || steps_per_exchange > (1 << 20))
        return sfail(STENCIL_ERR_INVALID_ARG, "steps_per_exchange must be in 1..2^20");
    const int64_t G = (int64_t)radius * steps_per_exchange;
    const int64_t owned = y1 - y0;
    const bool periodic = boundary == STENCIL_BOUNDARY_PERIODIC;
    const int64_t ga = (periodic || y0 > 0) ? G : 0;
    const int64_t gb = (periodic || y1 < ny) ? G : 0;
    // Every ghost row must come from the one neighbour next to it: that
    // neighbour owns at least G rows when every slab does.
    if ((ga || gb) && owned < G)
        return sfail(STENCIL_ERR_UNSUPPORTED, "a slab must own at least radius * steps_per_exchange rows (" +
                                                  std::to_string(G) + ")");
    if (!periodic && ((ga && y0 < G) || (gb && ny - y1 < G)))
        return sfail(STENCIL_ERR_UNSUPPORTED, "the neighbouring slabs own fewer rows than the ghost depth");
    if (ga + owned + gb > (1LL << 30)) return sfail(STENCIL_ERR_UNSUPPORTED, "slab buffer too tall");
    stencil_slab_info_t i{};
    i.ny = ny;
    i.nx = nx;
    i.y0 = y0;
    i.y1 = y1;
    i.radius = radius;
    i.boundary = boundary;
    i.steps_per_exchange = steps_per_exchange;
    i.ghost_depth = G;
    i.ghost_above = ga;
    i.ghost_below = gb;
    i.buffer_rows = ga + owned + gb;
    i.send_above_row = ga;
    i.send_below_row = ga + owned - G;
    i.recv_above_row = 0;
    i.recv_below_row = ga + owned;
    *info = i;
    return STENCIL_OK;
}

stencil_status_t stencil_slab_create(stencil_slab_t** slab, int64_t ny, int64_t nx, int64_t y0, int64_t y1,
                                     int radius, const float* weights, int dtype, int boundary,
                                     int64_t steps_per_exchange, const stencil_options_t* opt) {
    if (!slab) return sfail(STENCIL_ERR_INVALID_ARG, "slab pointer is NULL");
    *slab = nullptr;
    stencil_slab_info_t info{};
    stencil_status_t st = stencil_slab_geometry(ny, nx, y0, y1, radius, boundary, steps_per_exchange, &info);
    if (st != STENCIL_OK) return st;
    stencil_options_t o{};
    if (opt) o = *opt;
    if (o.kernel == STENCIL_KERNEL_AUTO) o.kernel = STENCIL_KERNEL_STREAM;
    if (o.kernel != STENCIL_KERNEL_STREAM || (o.compute != STENCIL_COMPUTE_AUTO && o.compute != STENCIL_COMPUTE_FP32))
        return sfail(STENCIL_ERR_UNSUPPORTED, "slabs run the streaming kernel with FP32 arithmetic");
    stencil_slab* s = new (std::nothrow) stencil_slab();
    if (!s) return sfail(STENCIL_ERR_OOM, "host allocation failed");
    s->info = info;
    st = stencil_plan_create(&s->plan, info.buffer_rows, nx, radius, weights, dtype, boundary, &o);
    if (st != STENCIL_OK) {
        g_slab_error = std::string("stencil_plan_create: ") + stencil_last_error();
        delete s;
        return st;
    }
    *slab = s;
    return STENCIL_OK;
}

void stencil_slab_destroy(stencil_slab_t* slab) {
    if (!slab) return;
    stencil_plan_destroy(slab->plan);
    delete slab;
}

stencil_status_t stencil_slab_info(const stencil_slab_t* slab, stencil_slab_info_t* info) {
    if (!slab || !info) return sfail(STENCIL_ERR_INVALID_ARG, "slab or info is NULL");
    *info = slab->info;
    return STENCIL_OK;
}

stencil_plan_t* stencil_slab_plan(stencil_slab_t* slab) { return slab ? slab->plan : nullptr; }

stencil_status_t stencil_slab_step(stencil_slab_t* slab, void* buf, int64_t steps, stencil_stream_t stream) {
    if (!slab || !buf) return sfail(STENCIL_ERR_INVALID_ARG, "slab or buffer is NULL");
    if (steps < 0 || steps > slab->info.steps_per_exchange)
        return sfail(STENCIL_ERR_INVALID_ARG, "steps must be in 0..steps_per_exchange");
    stencil_status_t st = stencil_run(slab->plan, buf, buf, steps, stream);
    if (st != STENCIL_OK) g_slab_error = std::string("stencil_run: ") + stencil_last_error();
    return st;
}

}  // extern "C"
