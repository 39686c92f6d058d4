// sweep_resident.cu -- small grids held entirely in the shared memory of one
// thread-block cluster, all T steps of a run in one launch.
//
// The Jacobi update of Sec. II-C, as the streaming kernel computes it, for
// grids whose two ping-pong copies fit in the distributed shared memory of a
// cluster of C <= 16 CTAs.  CTA k of the cluster owns the row slab
// [k*rp, min(ny, (k+1)*rp)) and stages it with R halo rows above and below
// and R halo columns on each side, in two buffers.  One step:
//   1. every CTA computes its slab from the source buffer into the other one
//      (each thread a column of up to 8 output rows, sliding a register
//      window over the input rows: (8 + 2R)(2R+1) shared loads for 8 outputs);
//   2. periodic grids refresh the halo columns of the new rows (wrap copies);
//   3. every CTA writes its top R rows into the bottom halo of the CTA above
//      and its bottom R rows into the top halo of the CTA below, through
//      distributed shared memory (periodic grids wrap around the cluster);
//   4. cluster barrier (release / acquire), then the buffers swap.
// The zero boundary of Sec. IV-A is the staged halo that nothing writes: it
// stays 0 at every step.  Global memory is read once (the initial state) and
// written once (the final state), so in == out is safe: every read precedes
// the first cluster barrier and every write follows the last one.
//
// This removes the launch-per-temporal-block cost that bounds small grids
// (a few microseconds per launch against a fraction of a microsecond of work
// per step), at the price of using only C SMs.
//
// Summation order: each output adds its taps with dy ascending and, within a
// row, dx ascending (FMA), the order of the oracle's loops.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace gbst {

constexpr int kResThreads = 1024;
constexpr int kResRB = 8;          // output rows per thread item
constexpr int kResMaxCluster = 16;

// Staged floats of one buffer: (rp + 2R) rows x pitch.  The dynamic shared
// memory holds two buffers and kResRB zero rows after them: the register
// window of a slab's last item reads up to kResRB - 1 rows past its buffer
// (for outputs that are never stored), and those reads must stay inside the
// allocation.
__host__ __device__ inline int resident_buf_floats(int rp, int pitch, int R) { return (rp + 2 * R) * pitch; }
__host__ __device__ inline int resident_smem_floats(int rp, int pitch, int R) {
    return 2 * resident_buf_floats(rp, pitch, R) + kResRB * pitch;
}

template <int R>
__device__ __forceinline__ void resident_wrap_columns(float* buf, int r_begin, int r_end, int nx, int pitch) {
    const int n = (r_end - r_begin) * 2 * R;
    for (int i = threadIdx.x; i < n; i += kResThreads) {
        const int r = r_begin + i / (2 * R), c = i % (2 * R);
        float* row = buf + r * pitch;
        if (c < R)
            row[c] = row[nx + c];  // left halo column c <- grid column nx - R + c
        else
            row[nx + c] = row[c];  // right halo column nx + c - R <- grid column c - R
    }
}

template <int R, bool STAR>
__device__ __forceinline__ void resident_step(const ResidentParams& p, const float* __restrict__ src,
                                              float* __restrict__ dst, int rows) {
    constexpr int D = 2 * R + 1;
    const int nx = p.nx, pitch = p.pitch;
    const int nb = (rows + kResRB - 1) / kResRB;
    for (int it = threadIdx.x; it < nb * nx; it += kResThreads) {
        const int b = it / nx, x = it - b * nx;
        const int r0 = b * kResRB;  // first output row of the item (slab-local)
        float acc[kResRB];
#pragma unroll
        for (int o = 0; o < kResRB; ++o) acc[o] = 0.f;
        // staged row r0 + i holds slab row r0 + i - R
#pragma unroll
        for (int i = 0; i < kResRB + 2 * R; ++i) {
            const float* row = src + (r0 + i) * pitch + x;  // row[d] is column x + d - R
            float v[D];
#pragma unroll
            for (int d = 0; d < D; ++d) v[d] = (STAR && (i < R || i >= kResRB + R) && d != R) ? 0.f : row[d];
#pragma unroll
            for (int dy = -R; dy <= R; ++dy) {
                const int o = i - R - dy;  // output row fed by this input row through weight row dy
                if (o < 0 || o >= kResRB) continue;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    if (STAR && dy != 0 && d != R) continue;
                    acc[o] = fmaf(p.w.w[(dy + R) * D + d], v[d], acc[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < kResRB; ++o)
            if (r0 + o < rows) dst[(R + r0 + o) * pitch + R + x] = acc[o];
    }
}

template <int R, bool STAR, typename TS>
__global__ void __launch_bounds__(kResThreads, 1) sweep_resident_kernel(const __grid_constant__ ResidentParams p) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int k = (int)cluster.block_rank();
    extern __shared__ float res_smem[];
    const int bufsz = resident_buf_floats(p.rp, p.pitch, R);
    float* const buf0 = res_smem;
    float* const buf1 = res_smem + bufsz;
    const int ny = p.ny, nx = p.nx, pitch = p.pitch;
    auto rows_of = [&](int r) { return max(0, min(p.rp, ny - r * p.rp)); };
    const int y0 = k * p.rp, rows = rows_of(k);
    int up = k - 1, dn = k + 1;  // neighbouring slabs; -1: none (zero rule)
    if (p.periodic) {
        up = (k + C - 1) % C;
        dn = (k + 1) % C;
    } else if (dn >= C) {
        dn = -1;
    }
    const int rows_up = up >= 0 ? rows_of(up) : 0;

    // Zero both buffers and the padding: what no step writes is the frozen zero halo.
    const int total = resident_smem_floats(p.rp, pitch, R);
    for (int i = threadIdx.x; i < total; i += kResThreads) res_smem[i] = 0.f;
    __syncthreads();
    // Stage the slab and its R halo rows from the initial state.
    const TS* gin = static_cast<const TS*>(p.in);
    for (int i = threadIdx.x; i < (rows + 2 * R) * nx; i += kResThreads) {
        const int r = i / nx, x = i - r * nx;
        int y = y0 - R + r;
        bool ok = true;
        if (p.periodic)
            y = (y % ny + ny) % ny;
        else
            ok = y >= 0 && y < ny;
        if (ok) buf0[r * pitch + R + x] = Storage<TS>::load1(gin + (size_t)y * p.ld + x);
    }
    if (p.periodic) {
        __syncthreads();
        resident_wrap_columns<R>(buf0, 0, rows + 2 * R, nx, pitch);
    }
    cluster.sync();  // every CTA's second buffer is zeroed before anyone writes into it

    for (int t = 0; t < p.T; ++t) {
        const float* src = (t & 1) ? buf1 : buf0;
        float* dst = (t & 1) ? buf0 : buf1;
        resident_step<R, STAR>(p, src, dst, rows);
        __syncthreads();
        if (p.periodic) {
            resident_wrap_columns<R>(dst, R, R + rows, nx, pitch);
            __syncthreads();
        }
        // Halo rows of the neighbours (full pitch, so box corners come along).
        if (up >= 0) {
            float* rem = cluster.map_shared_rank(dst, up) + (R + rows_up) * pitch;
            const float* mine = dst + R * pitch;
            for (int i = threadIdx.x; i < R * pitch; i += kResThreads) rem[i] = mine[i];
        }
        if (dn >= 0) {
            float* rem = cluster.map_shared_rank(dst, dn);
            const float* mine = dst + rows * pitch;
            for (int i = threadIdx.x; i < R * pitch; i += kResThreads) rem[i] = mine[i];
        }
        cluster.sync();
    }

    const float* fin = (p.T & 1) ? buf1 : buf0;
    TS* gout = static_cast<TS*>(p.out);
    for (int i = threadIdx.x; i < rows * nx; i += kResThreads) {
        const int r = i / nx, x = i - r * nx;
        Storage<TS>::store1(gout + (size_t)(y0 + r) * p.ld + x, fin[(R + r) * pitch + R + x]);
    }
}

template <int R, bool STAR>
static const void* resident_for_dtype(int dtype) {
    if (dtype == DT_F32) return (const void*)sweep_resident_kernel<R, STAR, float>;
    if (dtype == DT_BF16) return (const void*)sweep_resident_kernel<R, STAR, __nv_bfloat16>;
    if (dtype == DT_F16) return (const void*)sweep_resident_kernel<R, STAR, __half>;
    return nullptr;
}

const void* get_resident_kernel(int radius, int star, int dtype) {
    switch (radius * 2 + (star ? 1 : 0)) {
        case 2: return resident_for_dtype<1, false>(dtype);
        case 3: return resident_for_dtype<1, true>(dtype);
        case 4: return resident_for_dtype<2, false>(dtype);
        case 5: return resident_for_dtype<2, true>(dtype);
        case 6: return resident_for_dtype<3, false>(dtype);
        case 7: return resident_for_dtype<3, true>(dtype);
        default: return nullptr;
    }
}

int resident_threads() { return kResThreads; }
int resident_max_cluster() { return kResMaxCluster; }

// Shared memory of a launch with slab height rp, or -1 if a slab of the last
// rank would be shorter than the halo it must provide.
int resident_smem_bytes(int ny, int nx, int radius, int periodic, int C, int* rp_out) {
    const int rp = (ny + C - 1) / C;
    const int last = ny - (C - 1) * rp;
    if (last < 1) return -1;
    if ((C > 1 || periodic) && last < radius) return -1;
    if (rp_out) *rp_out = rp;
    return resident_smem_floats(rp, nx + 2 * radius, radius) * (int)sizeof(float);
}

// Launch one cluster of C CTAs for T steps.
cudaError_t launch_resident(const void* fn, int C, int smem, const ResidentParams& prm, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kResThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {const_cast<ResidentParams*>(&prm)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// Whether a cluster of C CTAs with `smem` bytes each can be scheduled.
bool resident_cluster_fits(const void* fn, int C, int smem) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kResThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n >= 1;
}

}  // namespace gbst
