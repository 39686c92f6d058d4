// sweep_naive.cu -- one Jacobi step per launch, one thread per grid point.
//
// The direct form of Sec. II-C: each thread gathers its (2R+1)^2 neighbours
// from global memory (zero outside the grid, or wrapped) and sums
// W[dy+R][dx+R] * u[i+dy][j+dx] dy-major, dx-minor with FMAs.  It is the
// correctness baseline for the streaming kernel and the fallback for shapes
// the streaming kernel does not take.
#include "common.cuh"

namespace gbst {

template <int R, typename TS>
__global__ void __launch_bounds__(256) sweep_naive_kernel(const TS* __restrict__ in,
                                                          TS* __restrict__ out, long long ny,
                                                          long long nx, int periodic, Weights w) {
    constexpr int D = 2 * R + 1;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = (long long)blockIdx.y * blockDim.y + threadIdx.y; i < ny;
         i += (long long)gridDim.y * blockDim.y) {
        if (j >= nx) return;
        float acc = 0.f;
#pragma unroll
        for (int dy = -R; dy <= R; ++dy) {
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                const float wv = w.w[(dy + R) * D + (dx + R)];
                long long y = i + dy, x = j + dx;
                float v = 0.f;
                if (periodic) {
                    v = Storage<TS>::load1(in + wrap_index(y, ny) * nx + wrap_index(x, nx));
                } else if (y >= 0 && y < ny && x >= 0 && x < nx) {
                    v = Storage<TS>::load1(in + y * nx + x);
                }
                acc = fmaf(wv, v, acc);
            }
        }
        Storage<TS>::store1(out + i * nx + j, acc);
    }
}

template <int R>
static const void* naive_for_dtype(int dtype) {
    switch (dtype) {
        case DT_F32: return (const void*)sweep_naive_kernel<R, float>;
        case DT_BF16: return (const void*)sweep_naive_kernel<R, __nv_bfloat16>;
        case DT_F16: return (const void*)sweep_naive_kernel<R, __half>;
        default: return nullptr;
    }
}

const void* get_naive_kernel(int radius, int dtype) {
    switch (radius) {
        case 1: return naive_for_dtype<1>(dtype);
        case 2: return naive_for_dtype<2>(dtype);
        case 3: return naive_for_dtype<3>(dtype);
        default: return nullptr;
    }
}

}  // namespace gbst
