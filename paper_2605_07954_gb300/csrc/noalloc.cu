// noalloc.cu -- stencil_run_noalloc: a T-step sweep that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need a sweep:
// a plugin inside an inference engine whose enqueue step must not allocate,
// code running while a framework's caching allocator already holds the free
// memory, or a latency-critical loop where cudaMalloc's implicit device-wide
// synchronisation is not acceptable.  stencil_plan_create() allocates a
// ping-pong workspace (and stencil_run() needs a plan), so such callers use
// this entry point instead.  Its ping-pong buffer is a fixed, file-scope
// device array of STENCIL_NOALLOC_MAX_BYTES; every GPU that loads it keeps it
// until the process exits.
//
// Only the host code of this file needs the array's device address: on the
// host, `g_noalloc_scratch` names a host-side stand-in, not device memory, so
// the address is fetched once per device with cudaGetSymbolAddress (with that
// device current) and cached.  That set-up happens inside the first call on
// each device, after its arguments are checked and before anything else (so a
// call with T = 0 serves as a warm-up).  Under CUDA's lazy module loading (the
// default) the set-up is also what loads this file's module, which reserves
// the array's device memory at that moment: the first call on a device may
// therefore take up to STENCIL_NOALLOC_MAX_BYTES of device memory (and fail
// with STENCIL_ERR_CUDA if there is none), so it belongs before any region
// that must not allocate and before any stream capture.  Later calls take
// nothing.
//
// The array is shared by every call in the process and keeps the contents of
// the last call.  Nothing in it has to start at zero: each launch writes every
// element of its destination before any launch reads it.  Calls whose work
// overlaps on the GPU (for example on two streams at once) race on the array.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/stencil.h"
#include "common.cuh"
#include "stream_depths.h"
#include "sweep_stream.cuh"

namespace gbst {
#define GBST_DECL_STREAM(R, DT) StreamKernelRef get_stream_kernel_r##R##_##DT(int star, int k, int vec);
GBST_DECL_STREAM(1, f32) GBST_DECL_STREAM(1, bf16) GBST_DECL_STREAM(1, f16)
GBST_DECL_STREAM(2, f32) GBST_DECL_STREAM(2, bf16) GBST_DECL_STREAM(2, f16)
GBST_DECL_STREAM(3, f32) GBST_DECL_STREAM(3, bf16) GBST_DECL_STREAM(3, f16)
#undef GBST_DECL_STREAM
}  // namespace gbst

using namespace gbst;

static __device__ __align__(256) unsigned char g_noalloc_scratch[STENCIL_NOALLOC_MAX_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device
std::mutex g_scratch_mu;
thread_local std::string g_noalloc_error;

stencil_status_t nfail(stencil_status_t st, const std::string& msg) {
    g_noalloc_error = msg;
    return st;
}

// A failed runtime call also clears the runtime's last-error state (for
// errors that are not sticky), so the caller's next error check does not
// report it a second time.
#define NCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            (void)cudaGetLastError();                                                       \
            return nfail(STENCIL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                   \
    } while (0)

// Device address of the scratch array on the current device (set up once).
stencil_status_t scratch_address(void** addr) {
    int dev = 0;
    NCK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return nfail(STENCIL_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        NCK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    return STENCIL_OK;
}

StreamKernelRef kernel_for(int R, int star, int k, int dtype, int vec) {
    typedef StreamKernelRef (*Getter)(int, int, int);
    static const Getter table[3][3] = {
        {get_stream_kernel_r1_f32, get_stream_kernel_r1_bf16, get_stream_kernel_r1_f16},
        {get_stream_kernel_r2_f32, get_stream_kernel_r2_bf16, get_stream_kernel_r2_f16},
        {get_stream_kernel_r3_f32, get_stream_kernel_r3_bf16, get_stream_kernel_r3_f16}};
    return table[R - 1][dtype](star, k, vec);
}

int depth_at_most(int R, int star, int k) {
    int m = 0;
    for (int i = 0; i < 8 && kStreamDepths[R - 1][star][i]; ++i)
        if (kStreamDepths[R - 1][star][i] <= k) m = kStreamDepths[R - 1][star][i];
    return m;
}

long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

// Tile geometry of the streaming kernel for depth k, CTAs of `threads`.
struct Geometry {
    int H, bx, nt, strips, by, tiles_y;
};

stencil_status_t launch_depth(const Geometry& g, const StreamParams& base, int R, int star,
                              int dtype, int elem, int depth, const void* src, void* dst,
                              cudaStream_t st) {
    StreamParams sp = base;
    sp.in = src;
    sp.out = dst;
    sp.nlev = depth;
    const size_t vb = 4 * (size_t)elem;
    sp.vec = (sp.nx % 4 == 0) && ((uintptr_t)src % vb == 0) && ((uintptr_t)dst % vb == 0);
    StreamKernelRef r = kernel_for(R, star, depth, dtype, sp.vec);
    if (!r.fn) return nfail(STENCIL_ERR_UNSUPPORTED, "no streaming kernel for this depth");
    const int smem = stream_smem_bytes(R, depth, elem, sp.vec != 0, false, g.nt);
    NCK(cudaFuncSetAttribute(r.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    void* args[] = {&sp};
    NCK(cudaLaunchKernel(r.fn, dim3((unsigned)(g.strips * g.tiles_y)), dim3((unsigned)g.nt), args,
                         (size_t)smem, st));
    return STENCIL_OK;
}

}  // namespace

extern "C" {

const char* stencil_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

stencil_status_t stencil_run_noalloc(int64_t ny, int64_t nx, int radius, const float* weights,
                                     int dtype, int boundary, const void* in, void* out, int64_t T,
                                     stencil_stream_t stream) {
    if (ny < 1 || nx < 1) return nfail(STENCIL_ERR_INVALID_ARG, "ny and nx must be >= 1");
    if (radius < 1) return nfail(STENCIL_ERR_INVALID_ARG, "radius must be >= 1");
    if (radius > kMaxRadius) return nfail(STENCIL_ERR_UNSUPPORTED, "radius > 3 is not supported");
    if (!weights || !in || !out) return nfail(STENCIL_ERR_INVALID_ARG, "NULL pointer argument");
    if (dtype < STENCIL_F32 || dtype > STENCIL_F16) return nfail(STENCIL_ERR_INVALID_ARG, "bad dtype");
    if (boundary != STENCIL_BOUNDARY_ZERO && boundary != STENCIL_BOUNDARY_PERIODIC)
        return nfail(STENCIL_ERR_INVALID_ARG, "bad boundary");
    if (T < 0) return nfail(STENCIL_ERR_INVALID_ARG, "T must be >= 0");
    const int elem = dtype == STENCIL_F32 ? 4 : 2;
    if (ny > (1LL << 30) || nx > (1LL << 30) ||
        (unsigned long long)ny * (unsigned long long)nx * elem > STENCIL_NOALLOC_MAX_BYTES)
        return nfail(STENCIL_ERR_UNSUPPORTED,
                     "grid of " + std::to_string(ny) + "x" + std::to_string(nx) +
                         " exceeds the allocation-free scratch of " +
                         std::to_string((long long)STENCIL_NOALLOC_MAX_BYTES) + " bytes");
    const int D = 2 * radius + 1;
    StreamParams base{};
    base.ny = ny;
    base.nx = nx;
    base.ld = nx;
    base.periodic = boundary == STENCIL_BOUNDARY_PERIODIC;
    int star = 1;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            const float v = weights[a * D + b];
            if (!(v == v) || v - v != 0.f) return nfail(STENCIL_ERR_INVALID_ARG, "weights must be finite");
            base.w.w[a * D + b] = v;
            base.w2.w2[a * D + b] = make_float2(v, v);
            if (a != radius && b != radius && v != 0.f) star = 0;
        }

    // Per-device set-up first, so that any call (T = 0 included) does it.
    void* scratch = nullptr;
    stencil_status_t s = scratch_address(&scratch);
    if (s != STENCIL_OK) return s;

    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)ny * (size_t)nx * elem;
    if (T == 0) {
        if (in != out) NCK(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st));
        return STENCIL_OK;
    }

    // Fixed configuration: the library's default depth and CTA size (64 threads
    // for the radius-1 box, 256 for the radius-3 box, else 128).
    const int kdef = radius == 1 ? 8 : (radius == 2 ? 4 : (star ? 3 : 2));
    const int k = depth_at_most(radius, star, kdef);
    Geometry g{};
    g.H = (radius * k + 3) / 4 * 4;
    const int threads = (radius == 1 && !star) ? 64 : ((radius == 3 && !star) ? 256 : 128);
    g.strips = (int)cdiv(nx, 4 * threads - 2 * g.H);
    g.bx = (int)(cdiv(cdiv(nx, g.strips), 4) * 4);
    g.nt = (int)(cdiv(cdiv(g.bx + 2 * g.H, 4), 32) * 32);
    int dev = 0, sms = 0, per_sm = 0;
    NCK(cudaGetDevice(&dev));
    NCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    {
        const int vec = nx % 4 == 0;
        StreamKernelRef r = kernel_for(radius, star, k, dtype, vec);
        if (!r.fn) return nfail(STENCIL_ERR_UNSUPPORTED, "no streaming kernel for this shape");
        const int smem = stream_smem_bytes(radius, k, elem, vec != 0, false, g.nt);
        NCK(cudaFuncSetAttribute(r.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        NCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, r.fn, g.nt, smem));
    }
    if (per_sm < 1) return nfail(STENCIL_ERR_UNSUPPORTED, "streaming kernel does not fit on an SM");
    const long long resident = (long long)per_sm * sms;
    const long long by_min = std::max(8LL, 4LL * radius * k);
    const long long tiles = std::max(1LL, std::min(std::max(1LL, resident / g.strips), cdiv(ny, by_min)));
    g.by = (int)cdiv(ny, tiles);
    g.tiles_y = (int)cdiv(ny, g.by);
    base.H = g.H;
    base.bx = g.bx;
    base.by = g.by;
    base.strips = g.strips;

    // Launches: T/k of depth k, then the remainder split into instantiated
    // depths.  Launch i writes `out` when L-1-i is even, else the scratch, so
    // the last one writes `out` and `in` is never written.
    const long long full = T / k;
    const int rem = (int)(T % k);
    long long L = full;
    for (int r = rem; r > 0; r -= depth_at_most(radius, star, r)) ++L;
    const void* src = in;
    // in == out with an odd launch count would make launch 0 write what it
    // reads: split the first depth-k launch in two, or stage the input.
    int ka = 0, kb = 0;
    if (in == out && L % 2 == 1) {
        ka = depth_at_most(radius, star, k / 2);
        kb = depth_at_most(radius, star, k - ka);
        if (full > 0 && ka > 0 && ka + kb == k) {
            ++L;
        } else {
            ka = kb = 0;
            NCK(cudaMemcpyAsync(scratch, in, bytes, cudaMemcpyDeviceToDevice, st));
            src = scratch;
        }
    }
    long long i = 0;
    auto run = [&](int d) -> stencil_status_t {
        void* dst = ((L - 1 - i) % 2 == 0) ? out : scratch;
        stencil_status_t r = launch_depth(g, base, radius, star, dtype, elem, d, src, dst, st);
        src = dst;
        ++i;
        return r;
    };
    long long f = 0;
    if (ka) {
        if ((s = run(ka)) != STENCIL_OK) return s;
        if ((s = run(kb)) != STENCIL_OK) return s;
        f = 1;
    }
    for (; f < full; ++f)
        if ((s = run(k)) != STENCIL_OK) return s;
    for (int r = rem; r > 0;) {
        const int d = depth_at_most(radius, star, r);
        if ((s = run(d)) != STENCIL_OK) return s;
        r -= d;
    }
    return STENCIL_OK;
}

}  // extern "C"
