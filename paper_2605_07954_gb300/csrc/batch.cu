// batch.cu -- many independent grids in one persistent launch (CUDA-graph replayed).
//
// Each grid of a batch runs the Jacobi update of Sec. II-C for its own T with
// its own weights (Star or Box, Sec. II-B).  Grids are split into the same
// (strip x row-tile) tiles as the single-grid streaming kernel and every
// tile advances K steps per work item, so a grid of B = T/K blocks gives
// B x tiles items.  One persistent launch (a CTA per resident slot) pops items
// from a device queue in block-major order:
//
//   item (grid g, tile i, block b) may start once every tile in the 3x3
//   neighbourhood of i has completed block b-1.
//
// That covers the reads of block b (the neighbours' block b-1 outputs, within
// the K*R halo) and the overwrite of block b's destination (the same
// neighbours read it, as their block b-1 source).  Tile completion is
// published with a per-tile epoch counter (release after a CTA barrier) and
// observed with acquire loads; input rows come through cp.async.cg (L2, never
// a stale L1 line).  Because items are popped in block-major order and every
// CTA is resident, an item only ever waits on items already held by running
// CTAs, so the queue cannot deadlock.  Every wait is bounded by a
// %globaltimer deadline; when one runs out the kernel records
// STENCIL_ERR_TIMEOUT in the batch's status word, raises an abort flag that
// stops every CTA, and returns.  Nothing traps.
//
// Grids live in plan-owned ping-pong buffers whose row pitch is rounded up to
// 4 elements, so every row is 16-byte aligned for the cp.async ring; the
// caller's dense grids are copied in and out with cudaMemcpy2DAsync.  The
// whole sequence (counter resets, copies, launches) is captured once into a
// CUDA graph and replayed by stencil_run_batched.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/stencil.h"
#include "common.cuh"
#include "stream_depths.h"
#include "sweep_stream.cuh"

namespace gbst {

struct BatchGrid {
    void* buf[2];  // padded ping-pong buffers
    int ny, nx, ld;
    int strips, tiles_y, bx, by, H;
    int tile_base;  // index of the grid's tile 0 in the epoch array
    int star, periodic;
    float2 w2[kMaxTaps];
};

struct BatchParams {
    const BatchGrid* grids;
    const int4* items;  // (grid, tile, global block index, unused)
    int item_begin, item_end;
    int* ticket;        // next item to pop (this launch's counter)
    int* epochs;        // per tile: blocks completed
    unsigned* status;   // STENCIL_ERR_TIMEOUT when a wait ran out
    int* abort_flag;
    long long timeout_ns;
    int deps;           // 1: wait on neighbour epochs (persistent); 0: no waits
    int withhold;       // item whose completion is never published (-1: none; test hook)
};

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int R, int K, typename TS>
__global__ void __launch_bounds__(kStreamMaxThreads)
    batch_stream_kernel(const __grid_constant__ BatchParams bp) {
    constexpr int D = 2 * R + 1;
    constexpr int CB = 4 * (int)sizeof(TS);
    extern __shared__ float4 smem_f4[];
    char* ring = reinterpret_cast<char*>(smem_f4);
    float* ebuf = reinterpret_cast<float*>(ring + stream_prefetch(K) * (int)blockDim.x * CB);
    __shared__ int s_item;
    const int NT = blockDim.x;
    const int tid = threadIdx.x;

    for (int i = tid; i < 2 * K * stream_buf_floats(R); i += NT) ebuf[i] = 0.f;

    for (;;) {
        __syncthreads();  // the previous item is finished by every thread
        if (tid == 0) {
            int it = -1;
            if (!*(volatile int*)bp.abort_flag) {
                const int t = atomicAdd(bp.ticket, 1) + bp.item_begin;
                if (t < bp.item_end) it = t;
            }
            if (it >= 0 && bp.deps) {
                const int4 item = bp.items[it];
                const BatchGrid& g = bp.grids[item.x];
                const int tx = item.y % g.strips, ty = item.y / g.strips;
                const long long t0 = global_ns();
                unsigned spins = 0;  // second bound, in case the timer were to stall
                for (int dy = -1; dy <= 1 && it >= 0; ++dy) {
                    for (int dx = -1; dx <= 1 && it >= 0; ++dx) {
                        const int ux = tx + dx, uy = ty + dy;
                        if (ux < 0 || ux >= g.strips || uy < 0 || uy >= g.tiles_y) continue;
                        const int* e = bp.epochs + g.tile_base + uy * g.strips + ux;
                        while (ld_acquire(e) < item.z) {
                            if (*(volatile int*)bp.abort_flag) {
                                it = -1;
                                break;
                            }
                            if (global_ns() - t0 > bp.timeout_ns || ++spins > (1u << 26)) {
                                atomicCAS(bp.status, 0u, (unsigned)STENCIL_ERR_TIMEOUT);
                                atomicExch(bp.abort_flag, 1);
                                it = -1;
                                break;
                            }
                            __nanosleep(64);
                        }
                    }
                }
            }
            s_item = it;
        }
        __syncthreads();
        const int it = s_item;
        if (it < 0) break;

        const int4 item = bp.items[it];
        const BatchGrid& g = bp.grids[item.x];
        const int tx = item.y % g.strips, ty = item.y / g.strips;
        StreamParams p;
        p.in = g.buf[item.z & 1];
        p.out = g.buf[(item.z + 1) & 1];
        p.ny = g.ny;
        p.nx = g.nx;
        p.ld = g.ld;
        p.nlev = K;
        p.H = g.H;
        p.bx = g.bx;
        p.by = g.by;
        p.strips = g.strips;
        p.periodic = g.periodic;
        p.vec = 1;
        RegWeights<D * D> ws;
#pragma unroll
        for (int i = 0; i < D * D; ++i) ws.w[i] = g.w2[i];
        const int x0 = tx * g.bx, y0 = ty * g.by;
        const int ylast = min(y0 + g.by, g.ny);
        // Interior: no masking needed, and the columns the idle threads of the
        // CTA read lie inside the neighbouring tiles' outputs.
        const bool interior = y0 - R * K >= 0 && ylast + stream_rows_after(R, K) <= g.ny && x0 - g.H >= 0 &&
                              x0 - g.H + 4 * NT <= g.nx && 4 * NT <= 2 * g.bx + g.H;
        if (g.star) {
            if (interior)
                stream_tile<R, true, K, TS, true, false>(p, ws, ring, ebuf, NT, tid, x0, y0);
            else
                stream_tile<R, true, K, TS, true, true>(p, ws, ring, ebuf, NT, tid, x0, y0);
        } else {
            if (interior)
                stream_tile<R, false, K, TS, true, false>(p, ws, ring, ebuf, NT, tid, x0, y0);
            else
                stream_tile<R, false, K, TS, true, true>(p, ws, ring, ebuf, NT, tid, x0, y0);
        }
        __syncthreads();  // every thread's stores of this tile are issued
        if (tid == 0 && it != bp.withhold) {
            __threadfence();
            red_release_add(bp.epochs + g.tile_base + item.y, 1);
        }
    }
}

struct BatchKernelRef {
    const void* fn;
};

template <int R, int K>
static const void* batch_kernel_dtype(int dtype) {
    switch (dtype) {
        case DT_F32: return (const void*)batch_stream_kernel<R, K, float>;
        case DT_BF16: return (const void*)batch_stream_kernel<R, K, __nv_bfloat16>;
        case DT_F16: return (const void*)batch_stream_kernel<R, K, __half>;
        default: return nullptr;
    }
}

// Batched kernels are instantiated for the depths {1, 2, 4, 8} (radius 1)
// and {1, 2} (radius 2, 3); other depths fall back to the largest below.
static const void* batch_kernel(int R, int K, int dtype) {
    if (R == 1) {
        switch (K) {
            case 1: return batch_kernel_dtype<1, 1>(dtype);
            case 2: return batch_kernel_dtype<1, 2>(dtype);
            case 4: return batch_kernel_dtype<1, 4>(dtype);
            case 8: return batch_kernel_dtype<1, 8>(dtype);
        }
    } else if (R == 2) {
        switch (K) {
            case 1: return batch_kernel_dtype<2, 1>(dtype);
            case 2: return batch_kernel_dtype<2, 2>(dtype);
        }
    } else if (R == 3) {
        switch (K) {
            case 1: return batch_kernel_dtype<3, 1>(dtype);
            case 2: return batch_kernel_dtype<3, 2>(dtype);
        }
    }
    return nullptr;
}

static int batch_depth_at_most(int R, int k) {
    static const int d1[] = {1, 2, 4, 8}, d23[] = {1, 2};
    const int* d = R == 1 ? d1 : d23;
    const int n = R == 1 ? 4 : 2;
    int m = 1;
    for (int i = 0; i < n; ++i)
        if (d[i] <= k) m = d[i];
    return m;
}

}  // namespace gbst

using namespace gbst;

namespace {

thread_local std::string g_batch_error;

stencil_status_t bfail(stencil_status_t st, const std::string& msg) {
    g_batch_error = msg;
    return st;
}

#define BCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail(STENCIL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

// One kernel launch of the batch: a radius group advancing `depth` steps for
// the items [begin, end).
struct Launch {
    int R, depth;
    int begin, end;  // item range
    int deps;        // 1: persistent launch with neighbour waits
    int ctas;
    int smem;
    const void* fn;
};

struct HostGrid {
    stencil_grid_desc_t d;  // d.weights points at w below
    std::vector<float> w;
    int R, star;
    int ld;
    int blocks;  // time blocks run in all launches (decides the final buffer)
    void* buf[2];
};

}  // namespace

struct stencil_batch {
    int n = 0;
    int dtype = 0;
    size_t elem = 4;
    stencil_batch_options_t opt{};
    int device = 0, sms = 0;
    int k = 8;                 // depth of the main launches
    int threads = 128;
    std::vector<HostGrid> grids;
    std::vector<BatchGrid> dgrids_h;
    std::vector<int4> items_h;
    std::vector<Launch> launches;
    int n_tiles = 0;
    BatchGrid* dgrids = nullptr;
    int4* items = nullptr;
    int* counters = nullptr;   // [0, nl): per-launch tickets; [nl]: abort flag; then epochs
    int n_counter_ints = 0;
    unsigned* status = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long timeout_ns = 2000000000LL;
    double last_points_steps = 0;
};

namespace {

void free_device_plan(stencil_batch* b) {
    if (b->dgrids) cudaFree(b->dgrids);
    if (b->items) cudaFree(b->items);
    if (b->counters) cudaFree(b->counters);
    b->dgrids = nullptr;
    b->items = nullptr;
    b->counters = nullptr;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// Tile every grid for depth k with CTAs of `threads`, and build the block-major
// item list and the launches.  Host-side only, then uploads.
stencil_status_t build_schedule(stencil_batch* b, int k, int threads, int tile_rows) {
    free_device_plan(b);
    b->k = k;
    b->threads = threads;
    b->dgrids_h.assign(b->n, BatchGrid{});
    b->items_h.clear();
    b->launches.clear();
    int tiles = 0;
    for (int gi = 0; gi < b->n; ++gi) {
        HostGrid& hg = b->grids[gi];
        BatchGrid& g = b->dgrids_h[gi];
        const int R = hg.R;
        const int kg = batch_depth_at_most(R, k);
        g.buf[0] = hg.buf[0];
        g.buf[1] = hg.buf[1];
        g.ny = (int)hg.d.ny;
        g.nx = (int)hg.d.nx;
        g.ld = hg.ld;
        g.H = (R * kg + 3) / 4 * 4;
        const int bx_max = 4 * threads - 2 * g.H;
        if (bx_max < 4) return bfail(STENCIL_ERR_UNSUPPORTED, "CTA too narrow for this depth");
        g.strips = (int)cdiv(g.nx, bx_max);
        g.bx = (int)(cdiv(cdiv(g.nx, g.strips), 4) * 4);
        // Tiles at least R*k + 2R + 1 rows high keep every dependency in the
        // 3x3 neighbourhood.
        const int want = tile_rows > 0 ? tile_rows : 256;
        const int min_rows = R * kg + 2 * R + 2;
        int ty = (int)std::max(1LL, cdiv(g.ny, std::max(want, min_rows)));
        while (ty > 1 && cdiv(g.ny, ty) < min_rows) --ty;
        g.by = (int)cdiv(g.ny, ty);
        g.tiles_y = (int)cdiv(g.ny, g.by);
        g.tile_base = tiles;
        tiles += g.strips * g.tiles_y;
        g.star = hg.star;
        g.periodic = hg.d.boundary == STENCIL_BOUNDARY_PERIODIC;
        const int D = 2 * R + 1;
        for (int i = 0; i < D * D; ++i) g.w2[i] = make_float2(hg.d.weights[i], hg.d.weights[i]);
        hg.blocks = 0;
    }
    b->n_tiles = tiles;

    // Launch groups: per radius, the main depth-k blocks (persistent), then
    // remainder depths (greedy), each a persistent launch of its own.
    for (int R = 1; R <= 3; ++R) {
        std::vector<int> members;
        for (int gi = 0; gi < b->n; ++gi)
            if (b->grids[gi].R == R && b->grids[gi].d.T > 0) members.push_back(gi);
        if (members.empty()) continue;
        const int kg = batch_depth_at_most(R, k);
        // Main launch: blocks of kg, block-major, larger tiles first within a block.
        std::sort(members.begin(), members.end(), [&](int a, int c) {
            const BatchGrid &ga = b->dgrids_h[a], &gc = b->dgrids_h[c];
            return (long long)ga.bx * ga.by > (long long)gc.bx * gc.by;
        });
        long long maxB = 0;
        for (int gi : members) maxB = std::max<long long>(maxB, b->grids[gi].d.T / kg);
        auto add_launch = [&](int depth, const std::vector<std::pair<int, long long>>& plan_blocks) {
            // plan_blocks: (grid, number of depth-`depth` blocks in this launch)
            Launch L{};
            L.R = R;
            L.depth = depth;
            L.begin = (int)b->items_h.size();
            long long nb = 0;
            for (auto& pb : plan_blocks) nb = std::max(nb, pb.second);
            for (long long blk = 0; blk < nb; ++blk)
                for (auto& pb : plan_blocks) {
                    if (blk >= pb.second) continue;
                    HostGrid& hg = b->grids[pb.first];
                    const BatchGrid& g = b->dgrids_h[pb.first];
                    for (int t = 0; t < g.strips * g.tiles_y; ++t)
                        b->items_h.push_back(make_int4(pb.first, t, (int)(hg.blocks + blk), 0));
                }
            for (auto& pb : plan_blocks) b->grids[pb.first].blocks += (int)pb.second;
            L.end = (int)b->items_h.size();
            L.deps = 1;
            b->launches.push_back(L);
        };
        std::vector<std::pair<int, long long>> main_blocks;
        for (int gi : members) main_blocks.push_back({gi, b->grids[gi].d.T / kg});
        if (maxB > 0) add_launch(kg, main_blocks);
        // Remainders T mod kg: one launch per instantiated depth below kg, each
        // giving one block to every grid that still has at least that many steps.
        std::vector<int> left(b->n, 0);
        for (int gi : members) left[gi] = (int)(b->grids[gi].d.T % kg);
        for (int d = kg - 1; d >= 1; --d) {
            if (batch_depth_at_most(R, d) != d) continue;
            std::vector<std::pair<int, long long>> blocks;
            for (int gi : members)
                if (left[gi] >= d) {
                    blocks.push_back({gi, 1});
                    left[gi] -= d;
                }
            if (!blocks.empty()) add_launch(d, blocks);
        }
    }
    for (auto& L : b->launches) {
        L.fn = batch_kernel(L.R, L.depth, b->dtype);
        if (!L.fn) return bfail(STENCIL_ERR_UNSUPPORTED, "no batched kernel for this depth");
        L.smem = stream_smem_bytes(L.R, L.depth, (int)b->elem, true, false, kStreamMaxThreads);
        BCK(cudaFuncSetAttribute(L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem));
        int per_sm = 0;
        BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, L.fn, threads, L.smem));
        if (per_sm < 1) return bfail(STENCIL_ERR_UNSUPPORTED, "batched kernel does not fit on an SM");
        L.ctas = (int)std::min<long long>((long long)per_sm * b->sms, L.end - L.begin);
    }

    // Upload descriptors, items and counters.
    BCK(cudaMalloc(&b->dgrids, sizeof(BatchGrid) * std::max(1, b->n)));
    BCK(cudaMemcpy(b->dgrids, b->dgrids_h.data(), sizeof(BatchGrid) * b->n, cudaMemcpyHostToDevice));
    BCK(cudaMalloc(&b->items, sizeof(int4) * std::max<size_t>(1, b->items_h.size())));
    if (!b->items_h.empty())
        BCK(cudaMemcpy(b->items, b->items_h.data(), sizeof(int4) * b->items_h.size(),
                       cudaMemcpyHostToDevice));
    b->n_counter_ints = (int)b->launches.size() + 1 + tiles;
    BCK(cudaMalloc(&b->counters, sizeof(int) * std::max(1, b->n_counter_ints)));
    return STENCIL_OK;
}

// Enqueue one full batch run on `st`.
stencil_status_t enqueue(stencil_batch* b, cudaStream_t st) {
    const int nl = (int)b->launches.size();
    BCK(cudaMemsetAsync(b->counters, 0, sizeof(int) * b->n_counter_ints, st));
    for (auto& hg : b->grids) {
        if (hg.d.T == 0) {
            BCK(cudaMemcpyAsync(hg.d.out, hg.d.in, (size_t)hg.d.ny * hg.d.nx * b->elem,
                                cudaMemcpyDeviceToDevice, st));
            continue;
        }
        BCK(cudaMemcpy2DAsync(hg.buf[0], (size_t)hg.ld * b->elem, hg.d.in, (size_t)hg.d.nx * b->elem,
                              (size_t)hg.d.nx * b->elem, (size_t)hg.d.ny, cudaMemcpyDeviceToDevice, st));
    }
    for (int li = 0; li < nl; ++li) {
        const Launch& L = b->launches[li];
        BatchParams bp{};
        bp.grids = b->dgrids;
        bp.items = b->items;
        bp.item_begin = L.begin;
        bp.item_end = L.end;
        bp.ticket = b->counters + li;
        bp.abort_flag = b->counters + nl;
        bp.epochs = b->counters + nl + 1;
        bp.status = b->status;
        bp.timeout_ns = b->timeout_ns;
        bp.deps = L.deps;
        bp.withhold = b->opt.debug_withhold_item > 0 && li == 0 ? b->opt.debug_withhold_item - 1 : -1;
        void* args[] = {&bp};
        BCK(cudaLaunchKernel(L.fn, dim3((unsigned)L.ctas), dim3((unsigned)b->threads), args,
                             (size_t)L.smem, st));
    }
    for (auto& hg : b->grids) {
        if (hg.d.T == 0) continue;
        BCK(cudaMemcpy2DAsync(hg.d.out, (size_t)hg.d.nx * b->elem, hg.buf[hg.blocks & 1],
                              (size_t)hg.ld * b->elem, (size_t)hg.d.nx * b->elem, (size_t)hg.d.ny,
                              cudaMemcpyDeviceToDevice, st));
    }
    return STENCIL_OK;
}

stencil_status_t time_batch(stencil_batch* b, cudaStream_t st, float* ms) {
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    stencil_status_t s = enqueue(b, st);  // warm-up
    if (s == STENCIL_OK) {
        cudaEventRecord(e0, st);
        s = enqueue(b, st);
        cudaEventRecord(e1, st);
    }
    cudaError_t e = cudaEventSynchronize(e1);
    if (s == STENCIL_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != STENCIL_OK) return s;
    if (e != cudaSuccess) return bfail(STENCIL_ERR_CUDA, std::string("batch timing: ") + cudaGetErrorString(e));
    return STENCIL_OK;
}

}  // namespace

extern "C" {

const char* stencil_batch_last_error(void) { return g_batch_error.c_str(); }

stencil_status_t stencil_batch_create(stencil_batch_t** out, int n, const stencil_grid_desc_t* descs,
                                      int dtype, const stencil_batch_options_t* opt) {
    if (!out) return bfail(STENCIL_ERR_INVALID_ARG, "batch pointer is NULL");
    *out = nullptr;
    if (n < 1 || !descs) return bfail(STENCIL_ERR_INVALID_ARG, "need n >= 1 grid descriptors");
    if (dtype < STENCIL_F32 || dtype > STENCIL_F16) return bfail(STENCIL_ERR_INVALID_ARG, "bad dtype");
    stencil_batch_options_t o{};
    if (opt) o = *opt;
    if (o.tb_depth < 0 || o.threads < 0 || o.tile_rows < 0 || o.timeout_ms < 0 || o.debug_withhold_item < 0)
        return bfail(STENCIL_ERR_INVALID_ARG, "bad option value");
    if (o.threads && (o.threads < 32 || o.threads > kStreamMaxThreads || o.threads % 32))
        return bfail(STENCIL_ERR_INVALID_ARG, "threads must be a multiple of 32 in 32..256");
    stencil_batch* b = new (std::nothrow) stencil_batch();
    if (!b) return bfail(STENCIL_ERR_OOM, "host allocation failed");
    b->n = n;
    b->dtype = dtype;
    b->elem = dtype == STENCIL_F32 ? 4 : 2;
    b->opt = o;
    if (o.timeout_ms > 0) b->timeout_ns = (long long)o.timeout_ms * 1000000LL;
    auto bail = [&](stencil_status_t st) {
        stencil_batch_destroy(b);
        return st;
    };
    b->grids.resize(n);
    for (int i = 0; i < n; ++i) {
        const stencil_grid_desc_t& d = descs[i];
        if (d.ny < 1 || d.nx < 1 || d.ny > (1LL << 30) || d.nx > (1LL << 30) || d.T < 0 || !d.weights ||
            !d.in || !d.out)
            return bail(bfail(STENCIL_ERR_INVALID_ARG, "bad descriptor " + std::to_string(i)));
        if (d.radius < 1 || d.radius > kMaxRadius)
            return bail(bfail(STENCIL_ERR_UNSUPPORTED, "radius must be 1..3 (grid " + std::to_string(i) + ")"));
        if (d.boundary != STENCIL_BOUNDARY_ZERO && d.boundary != STENCIL_BOUNDARY_PERIODIC)
            return bail(bfail(STENCIL_ERR_INVALID_ARG, "bad boundary (grid " + std::to_string(i) + ")"));
        if (d.boundary == STENCIL_BOUNDARY_PERIODIC && d.nx % 4)
            return bail(bfail(STENCIL_ERR_UNSUPPORTED,
                              "periodic grids in a batch need nx % 4 == 0 (grid " + std::to_string(i) + ")"));
        HostGrid& hg = b->grids[i];
        hg.d = d;
        hg.R = d.radius;
        const int D = 2 * d.radius + 1;
        hg.star = 1;
        for (int a = 0; a < D; ++a)
            for (int c = 0; c < D; ++c) {
                const float v = d.weights[a * D + c];
                if (!std::isfinite(v)) return bail(bfail(STENCIL_ERR_INVALID_ARG, "weights must be finite"));
                if (a != d.radius && c != d.radius && v != 0.f) hg.star = 0;
            }
        hg.ld = (int)(cdiv(d.nx, 4) * 4);
        hg.buf[0] = hg.buf[1] = nullptr;
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return bail(bfail(STENCIL_ERR_CUDA, cudaGetErrorString(e)));
    // The weights pointer of a descriptor is only valid during this call.
    for (auto& hg : b->grids) {
        const int D = 2 * hg.R + 1;
        hg.w.assign(hg.d.weights, hg.d.weights + D * D);
        hg.d.weights = hg.w.data();
    }
    for (auto& hg : b->grids) {
        if (hg.d.T == 0) continue;
        const size_t bytes = (size_t)hg.ld * hg.d.ny * b->elem;
        for (int j = 0; j < 2; ++j) {
            if (cudaMalloc(&hg.buf[j], bytes) != cudaSuccess) {
                cudaGetLastError();
                hg.buf[j] = nullptr;
                return bail(bfail(STENCIL_ERR_OOM, "cudaMalloc of a batch workspace failed"));
            }
            // Pad columns [nx, ld) stay finite (zero) for the whole-chunk loads.
            if (cudaMemset(hg.buf[j], 0, bytes) != cudaSuccess)
                return bail(bfail(STENCIL_ERR_CUDA, "cudaMemset of a batch workspace failed"));
        }
    }
    if (cudaMalloc(&b->status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(b->status, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(STENCIL_ERR_OOM, "cudaMalloc of the status word failed"));
    }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(bfail(STENCIL_ERR_CUDA, "cudaStreamCreate failed"));

    const int threads = o.threads ? o.threads : 128;
    if (o.autotune) {
        // Time every instantiated radius-1 depth (and CTA size unless fixed) on the
        // whole batch; keep the fastest.
        const int ks[4] = {1, 2, 4, 8};
        const int ths[3] = {64, 128, 256};
        float best = 1e30f;
        int bk = 8, bt = threads;
        for (int k : ks) {
            if (o.tb_depth && k != o.tb_depth) continue;
            for (int th : ths) {
                if (o.threads && th != o.threads) continue;
                if (build_schedule(b, k, th, o.tile_rows) != STENCIL_OK) continue;
                float ms = 0.f;
                stencil_status_t s = time_batch(b, b->cap, &ms);
                if (s != STENCIL_OK) return bail(s);
                if (ms < best) {
                    best = ms;
                    bk = k;
                    bt = th;
                }
            }
        }
        stencil_status_t s = build_schedule(b, bk, bt, o.tile_rows);
        if (s != STENCIL_OK) return bail(s);
    } else {
        // Default depth 4: the measured best for the 256-grid radius-1 batch on GB300
        // (deeper items cost more halo rows per tile at these tile heights).
        stencil_status_t s = build_schedule(b, o.tb_depth ? o.tb_depth : 4, threads, o.tile_rows);
        if (s != STENCIL_OK) return bail(s);
    }
    *out = b;
    return STENCIL_OK;
}

stencil_status_t stencil_run_batched(stencil_batch_t* b, stencil_stream_t stream) {
    if (!b) return bfail(STENCIL_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->exec) {
        // Capture the whole run once on the batch's own stream, then replay it.
        BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        stencil_status_t s = enqueue(b, b->cap);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
        if (s != STENCIL_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return bfail(STENCIL_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(STENCIL_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    BCK(cudaGraphLaunch(b->exec, st));
    return STENCIL_OK;
}

stencil_status_t stencil_batch_status(stencil_batch_t* b) {
    if (!b) return bfail(STENCIL_ERR_INVALID_ARG, "batch is NULL");
    BCK(cudaDeviceSynchronize());
    unsigned word = 0;
    BCK(cudaMemcpy(&word, b->status, sizeof(word), cudaMemcpyDeviceToHost));
    BCK(cudaMemset(b->status, 0, sizeof(word)));
    if (word == 0) return STENCIL_OK;
    return word == STENCIL_ERR_TIMEOUT ? STENCIL_ERR_TIMEOUT : STENCIL_ERR_DEVICE_CHECK;
}

stencil_status_t stencil_batch_info(const stencil_batch_t* b, stencil_batch_info_t* info) {
    if (!b || !info) return bfail(STENCIL_ERR_INVALID_ARG, "NULL argument");
    stencil_batch_info_t i{};
    i.n = b->n;
    i.tb_depth = b->k;
    i.threads = b->threads;
    i.tiles = b->n_tiles;
    i.items = (int64_t)b->items_h.size();
    i.launches = (int)b->launches.size();
    i.ctas = b->launches.empty() ? 0 : b->launches[0].ctas;
    int64_t pts = 0;
    for (auto& hg : b->grids) pts += hg.d.ny * hg.d.nx * hg.d.T;
    i.point_steps = pts;
    *info = i;
    return STENCIL_OK;
}

void stencil_batch_destroy(stencil_batch_t* b) {
    if (!b) return;
    free_device_plan(b);
    for (auto& hg : b->grids) {
        for (int j = 0; j < 2; ++j)
            if (hg.buf[j]) cudaFree(hg.buf[j]);
    }
    if (b->status) cudaFree(b->status);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // extern "C"
