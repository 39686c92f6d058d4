// residual.cu -- T steps with a convergence check every m steps.
//
// The paper's host drives the wafer through long uninterrupted runs "save for
// periodic convergence checks" (Sec. IV).  stencil_run_residual runs T Jacobi
// steps (Sec. II-C) and, after every m-th step t, records
//     residual[j] = || u_t - u_{t-1} ||_2   (j = t/m - 1),
// the change made by that step, accumulated in FP64 over the whole grid.
//
// To have u_{t-1} and u_t both in memory, each checked interval runs its
// first m-1 steps with the plan's temporally blocked kernels (stencil_run)
// and its m-th step as one launch into a second buffer; residual_kernel then
// reads both (8 B per point for FP32 storage, once per interval).  The
// per-point arithmetic of every step is the one stencil_run uses, so the
// final state is bit-identical to stencil_run's.  The reduction is
// deterministic: a fixed grid of CTAs each sums a fixed index range in FP64,
// then one block adds the CTA sums in a fixed tree.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <string>

#include "../../include/stencil.h"
#include "common.cuh"

namespace gbst {

void** plan_aux_slot(stencil_plan_t* p, int id);
void plan_set_aux_free(stencil_plan_t* p, int id, void (*freer)(void*));

constexpr int kResBlocks = 1024;

template <typename TS>
__global__ void __launch_bounds__(256)
    residual_partials_kernel(const TS* __restrict__ a, const TS* __restrict__ b, long long n,
                             double* __restrict__ partials) {
    __shared__ double sh[256];
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    double s = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += 256) {
        const double d = (double)Storage<TS>::load1(a + i) - (double)Storage<TS>::load1(b + i);
        s += d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256)
    residual_finish_kernel(const double* __restrict__ partials, int n, double* __restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += partials[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sqrt(sh[0]);
}

}  // namespace gbst

using namespace gbst;

namespace {

thread_local std::string g_res_error;

stencil_status_t rfail(stencil_status_t st, const std::string& msg) {
    g_res_error = msg;
    return st;
}

#define RCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return rfail(STENCIL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct ResScratch {
    char* grids = nullptr;  // two grids
    size_t bytes = 0;       // per grid
    double* partials = nullptr;
};

void res_scratch_free(void* v) {
    ResScratch* sc = static_cast<ResScratch*>(v);
    if (sc->grids) cudaFree(sc->grids);
    if (sc->partials) cudaFree(sc->partials);
    delete sc;
}

}  // namespace

extern "C" {

const char* stencil_residual_last_error(void) { return g_res_error.c_str(); }

stencil_status_t stencil_run_residual(stencil_plan_t* plan, const void* in, void* out, int64_t T,
                                      int64_t m, double* residuals, stencil_stream_t stream) {
    if (!plan || !in || !out || !residuals) return rfail(STENCIL_ERR_INVALID_ARG, "NULL argument");
    if (T < 0 || m < 1) return rfail(STENCIL_ERR_INVALID_ARG, "need T >= 0 and m >= 1");
    stencil_plan_info_t info{};
    stencil_status_t s = stencil_plan_info(plan, &info);
    if (s != STENCIL_OK) return rfail(s, "stencil_plan_info failed");
    const size_t elem = info.dtype == STENCIL_F32 ? 4 : 2;
    const long long n = info.ny * info.nx;
    const size_t bytes = (size_t)n * elem;
    cudaStream_t st = (cudaStream_t)stream;

    void** slot = plan_aux_slot(plan, 1);
    ResScratch* sc = static_cast<ResScratch*>(*slot);
    if (!sc) {
        sc = new (std::nothrow) ResScratch();
        if (!sc) return rfail(STENCIL_ERR_OOM, "host allocation failed");
        *slot = sc;
        plan_set_aux_free(plan, 1, res_scratch_free);
    }
    if (!sc->grids) {
        if (cudaMalloc((void**)&sc->grids, 2 * bytes) != cudaSuccess ||
            cudaMalloc((void**)&sc->partials, sizeof(double) * kResBlocks) != cudaSuccess) {
            cudaGetLastError();
            return rfail(STENCIL_ERR_OOM, "cudaMalloc of the residual scratch failed");
        }
        sc->bytes = bytes;
    }
    void* A = sc->grids;          // u_{t-1} of a check
    void* B = sc->grids + bytes;  // u_t of a check
    const void* cur = in;
    int64_t t = 0, j = 0;
    while (t + m <= T) {
        // m-1 steps (temporally blocked) to u_{t+m-1}, then one step to u_{t+m}
        const void* prev = cur;
        if (m > 1) {
            s = stencil_run(plan, cur, A, m - 1, stream);
            if (s != STENCIL_OK) return rfail(s, std::string("run: ") + stencil_last_error());
            prev = A;
        }
        void* next = (prev == B) ? A : B;
        s = stencil_run(plan, prev, next, 1, stream);
        if (s != STENCIL_OK) return rfail(s, std::string("run: ") + stencil_last_error());
        if (info.dtype == STENCIL_F32)
            residual_partials_kernel<float><<<kResBlocks, 256, 0, st>>>(
                static_cast<const float*>(prev), static_cast<const float*>(next), n, sc->partials);
        else if (info.dtype == STENCIL_BF16)
            residual_partials_kernel<__nv_bfloat16><<<kResBlocks, 256, 0, st>>>(
                static_cast<const __nv_bfloat16*>(prev), static_cast<const __nv_bfloat16*>(next), n,
                sc->partials);
        else
            residual_partials_kernel<__half><<<kResBlocks, 256, 0, st>>>(
                static_cast<const __half*>(prev), static_cast<const __half*>(next), n, sc->partials);
        residual_finish_kernel<<<1, 256, 0, st>>>(sc->partials, kResBlocks, residuals + j);
        RCK(cudaGetLastError());
        cur = next;
        t += m;
        ++j;
    }
    // the remaining T mod m steps, straight into `out`
    s = stencil_run(plan, cur, out, T - t, stream);
    if (s != STENCIL_OK) return rfail(s, std::string("run: ") + stencil_last_error());
    return STENCIL_OK;
}

}  // extern "C"
