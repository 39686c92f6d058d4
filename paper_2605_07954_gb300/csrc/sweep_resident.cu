// sweep_resident.cu -- small grids held entirely in the shared memory of one
// thread-block cluster, all T steps of a run in one launch.
//
// The Jacobi update of Sec. II-C, as the streaming kernel computes it, for
// grids whose ping-pong copies fit in the distributed shared memory of a
// cluster of C <= 16 CTAs.  CTA k of the cluster owns the row slab
// [k*rp, min(ny, (k+1)*rp)) and stages it with H = kb*R halo rows above and
// below and R halo columns on each side, in two buffers.  The steps run in
// groups of kb (temporal blocking inside the cluster):
//   1. sub-step s of a group computes the slab plus (kb-1-s)*R rows on each
//      side (the rows the next sub-steps need), each thread a column of up to
//      8 output rows with a register window over the input rows; periodic
//      grids then refresh the halo columns (wrap copies);
//   2. after the group every CTA writes its top H rows and its bottom H rows
//      into mailboxes of the CTAs above and below, through distributed shared
//      memory (periodic grids wrap around the cluster), and the cluster meets
//      at one barrier;
//   3. the next group starts by copying its mailboxes into its halo rows.
// The mailboxes alternate between two copies by group parity, so a neighbour
// that finishes its next group early never overwrites halo rows that are
// still being read: one cluster barrier per kb steps suffices.
// The zero boundary of Sec. IV-A is the staged halo that nothing writes (rows
// outside the grid are never computed): it stays 0 at every step.  Global
// memory is read once (the initial state) and written once (the final
// state), so in == out is safe: every read precedes the first cluster barrier
// and every write follows the last one.
//
// This removes the launch-per-temporal-block cost that bounds small grids
// (a few microseconds per launch against a fraction of a microsecond of work
// per step), at the price of using only C SMs.
//
// Summation order: each output adds its taps with dy ascending and, within a
// row, dx ascending (FMA), the order of the oracle's loops; the result does
// not depend on kb or C.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace gbst {

constexpr int kResThreads = 1024;
constexpr int kResRB = 8;          // output rows per thread item
constexpr int kResMaxCluster = 16;

// Shared memory of a CTA, in floats: two staged buffers of (rp + 2H) rows x
// pitch, kResRB zero rows after them (the register window of a slab's last
// item reads up to kResRB - 1 rows past its buffer, for outputs that are
// never stored, and those reads must stay inside the allocation), and the
// mailboxes: 2 parities x 2 sides x H rows.
__host__ __device__ inline int resident_buf_floats(int rp, int pitch, int H) { return (rp + 2 * H) * pitch; }
__host__ __device__ inline int resident_smem_floats(int rp, int pitch, int H, int kb) {
    return 2 * resident_buf_floats(rp, pitch, H) + kResRB * pitch + (kb > 1 ? 4 * H * pitch : 0);
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

// Staged rows [rb, re) of dst from src: each item is a column and up to
// kResRB rows; staged row i of dst reads staged rows i-R .. i+R of src.
template <int R, bool STAR>
__device__ __forceinline__ void resident_step(const ResidentParams& p, const float* __restrict__ src,
                                              float* __restrict__ dst, int rb, int re) {
    constexpr int D = 2 * R + 1;
    const int nx = p.nx, pitch = p.pitch;
    const int rows = re - rb;
    const int nb = (rows + kResRB - 1) / kResRB;
    for (int it = threadIdx.x; it < nb * nx; it += kResThreads) {
        const int b = it / nx, x = it - b * nx;
        const int r0 = rb + b * kResRB;  // first output row of the item (staged index)
        float acc[kResRB];
#pragma unroll
        for (int o = 0; o < kResRB; ++o) acc[o] = 0.f;
        // input row i of the window is staged row r0 - R + i
#pragma unroll
        for (int i = 0; i < kResRB + 2 * R; ++i) {
            const float* row = src + (r0 - R + i) * pitch + x;  // row[d] is column x + d - R
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
            if (r0 + o < re) dst[(r0 + o) * pitch + R + x] = acc[o];
    }
}

template <int R, bool STAR, typename TS>
__global__ void __launch_bounds__(kResThreads, 1) sweep_resident_kernel(const __grid_constant__ ResidentParams p) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int k = (int)cluster.block_rank();
    extern __shared__ float res_smem[];
    const int ny = p.ny, nx = p.nx, pitch = p.pitch, H = p.H;
    const int bufsz = resident_buf_floats(p.rp, pitch, H);
    float* const buf0 = res_smem;
    float* const buf1 = res_smem + bufsz;
    // mail + (parity * 2 + side) * H * pitch; side 0: top halo, side 1: bottom halo
    float* const mail = res_smem + 2 * bufsz + kResRB * pitch;
    auto rows_of = [&](int r) { return max(0, min(p.rp, ny - r * p.rp)); };
    const int y0 = k * p.rp, rows = rows_of(k);
    int up = k - 1, dn = k + 1;  // neighbouring slabs; -1: none (zero rule)
    if (p.periodic) {
        up = (k + C - 1) % C;
        dn = (k + 1) % C;
    } else if (dn >= C) {
        dn = -1;
    }

    // Zero everything: what no step writes is the frozen zero halo.
    const int total = resident_smem_floats(p.rp, pitch, H, p.kb);
    for (int i = threadIdx.x; i < total; i += kResThreads) res_smem[i] = 0.f;
    __syncthreads();
    // Stage the slab and its H halo rows from the initial state.
    const TS* gin = static_cast<const TS*>(p.in);
    for (int i = threadIdx.x; i < (rows + 2 * H) * nx; i += kResThreads) {
        const int r = i / nx, x = i - r * nx;
        int y = y0 - H + r;
        bool ok = true;
        if (p.periodic)
            y = (y % ny + ny) % ny;
        else
            ok = y >= 0 && y < ny;
        if (ok) buf0[r * pitch + R + x] = Storage<TS>::load1(gin + (size_t)y * p.ld + x);
    }
    if (p.periodic) {
        __syncthreads();
        resident_wrap_columns<R>(buf0, 0, rows + 2 * H, nx, pitch);
    }
    cluster.sync();  // every CTA is initialised before anyone writes into its mailboxes

    // Staged rows that exist in the grid (zero rule): [H - y0, H + ny - y0).
    const int lo = p.periodic ? 0 : H - y0, hi = p.periodic ? rows + 2 * H : H + ny - y0;
    float* cur = buf0;
    float* nxt = buf1;
    if (p.kb == 1) {
        // One step per exchange: the edge rows go straight into the neighbours'
        // next buffer, which no CTA reads during this step.
        const int rows_up = up >= 0 ? rows_of(up) : 0;
        for (int t = 0; t < p.T; ++t) {
            resident_step<R, STAR>(p, cur, nxt, H, H + rows);
            __syncthreads();
            if (p.periodic) {
                resident_wrap_columns<R>(nxt, H, H + rows, nx, pitch);
                __syncthreads();
            }
            if (t + 1 < p.T) {
                if (up >= 0) {
                    float* rem = cluster.map_shared_rank(nxt, up) + (H + rows_up) * pitch;
                    const float* mine = nxt + H * pitch;
                    for (int i = threadIdx.x; i < H * pitch; i += kResThreads) rem[i] = mine[i];
                }
                if (dn >= 0) {
                    float* rem = cluster.map_shared_rank(nxt, dn);
                    const float* mine = nxt + rows * pitch;
                    for (int i = threadIdx.x; i < H * pitch; i += kResThreads) rem[i] = mine[i];
                }
                cluster.sync();
            }
            float* tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
    }
    int g = 0;
    for (int t = (p.kb == 1 ? p.T : 0); t < p.T; ++g) {
        const int kk = min(p.kb, p.T - t);
        if (g > 0) {  // the halo rows the neighbours sent after the previous group
            const float* mb = mail + ((g - 1) & 1) * 2 * H * pitch;
            if (up >= 0)
                for (int i = threadIdx.x; i < H * pitch; i += kResThreads) cur[i] = mb[i];
            if (dn >= 0)
                for (int i = threadIdx.x; i < H * pitch; i += kResThreads)
                    cur[(H + rows) * pitch + i] = mb[H * pitch + i];
            __syncthreads();
        }
        for (int s = 0; s < kk; ++s) {
            const int ext = (kk - 1 - s) * R;
            const int rb = max(H - ext, lo), re = min(H + rows + ext, hi);
            resident_step<R, STAR>(p, cur, nxt, rb, re);
            __syncthreads();
            if (p.periodic) {
                resident_wrap_columns<R>(nxt, rb, re, nx, pitch);
                __syncthreads();
            }
            float* tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        t += kk;
        if (t < p.T) {  // edge rows into the neighbours' mailboxes of this group's parity
            const int par = g & 1;
            if (up >= 0) {  // my top H rows become the bottom halo of the slab above
                float* rem = cluster.map_shared_rank(mail, up) + (par * 2 + 1) * H * pitch;
                const float* mine = cur + H * pitch;
                for (int i = threadIdx.x; i < H * pitch; i += kResThreads) rem[i] = mine[i];
            }
            if (dn >= 0) {  // my bottom H rows become the top halo of the slab below
                float* rem = cluster.map_shared_rank(mail, dn) + (par * 2) * H * pitch;
                const float* mine = cur + rows * pitch;
                for (int i = threadIdx.x; i < H * pitch; i += kResThreads) rem[i] = mine[i];
            }
            cluster.sync();
        }
    }

    TS* gout = static_cast<TS*>(p.out);
    for (int i = threadIdx.x; i < rows * nx; i += kResThreads) {
        const int r = i / nx, x = i - r * nx;
        Storage<TS>::store1(gout + (size_t)(y0 + r) * p.ld + x, cur[(H + r) * pitch + R + x]);
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

// Shared memory (bytes) of a cluster of C CTAs running kb steps per halo
// exchange, or -1 where that does not work: every slab must be at least
// H = kb*R rows high where halos are exchanged, H at most half a slab for
// kb > 1 (the redundant halo rows stay under ~50 %), and the CTA's shared
// memory must fit `max_smem`.  *rp_out: the slab height.
int resident_config(int ny, int nx, int radius, int periodic, int C, int kb, int max_smem, int* rp_out) {
    const int rp = (ny + C - 1) / C;
    const int last = ny - (C - 1) * rp;
    if (last < 1 || kb < 1) return -1;
    const int H = kb * radius;
    if ((C > 1 || periodic) && last < H) return -1;
    if (kb > 1 && 2 * H > rp) return -1;
    const long long bytes = (long long)resident_smem_floats(rp, nx + 2 * radius, H, kb) * (long long)sizeof(float);
    if (bytes > max_smem) return -1;
    if (rp_out) *rp_out = rp;
    return (int)bytes;
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
