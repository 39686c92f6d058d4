// sweep_stream.cuh -- row-streaming, temporally blocked Jacobi sweep (sm_103a).
//
// Computes nlev steps of the Jacobi update of Sec. II-C per launch:
//     u^{t+1}[i][j] = sum_{dy,dx} W[dy+R][dx+R] * u~^t[i+dy][j+dx]
// with u~ zero outside the grid (the fixed zero padding of Sec. IV-A) or
// wrapped (periodic).
//
// Decomposition.  A CTA owns an output tile of `by` rows x `bx` columns.  It
// loads a strip of bx + 2H columns (H >= R*nlev halo columns per side, the GPU
// counterpart of the paper's per-tile halo padding, Sec. IV-A step 3, made
// nlev times deeper so that nlev steps need no exchange with other CTAs) and
// streams down the rows from y0 - R*nlev to y0 + by - 1 + R*nlev.
//
// Each thread owns 4 adjacent columns.  Time level l+1 is produced from level
// l as a pipeline along y: when row y of level l arrives, it is the last
// contribution to output row y-R of level l+1 and the first to row y+R.  A
// thread therefore keeps 2R+1 partial sums per column and level in registers
// (a register window sliding down the rows); a completed level-(l+1) row is
// immediately fed to level l+2 in the same row step.  Only the R columns on
// each side of a thread's 4 columns cross threads: each level's newest row
// is written once to a double-buffered shared-memory row and the halo values
// are read back after one barrier.  The input row comes from HBM with one
// 16-byte (FP32) or 8-byte (BF16/FP16) vector load per thread; only the level
// nlev row goes back to HBM.  So HBM traffic is ~(4+4)/nlev bytes per
// point-step for FP32, plus the halo overlap.
//
// Boundary: with the zero rule, every level's values outside the grid are
// forced to 0 after they are computed, so the halo stays a frozen zero at
// every sub-step, exactly as the padding in the paper.  With the periodic
// rule, loads wrap and nothing is masked.
//
// Summation order: each output accumulates dy = -R .. R (row by row as rows
// arrive) and, within a row, dx = -R .. R, with one FMA per weight: the
// dy-major, dx-minor order of the plain loop.  Star footprints skip the
// off-axis (zero) weights.
#pragma once

#include "common.cuh"

namespace gbst {

template <typename TS>
__device__ __forceinline__ void load_chunk(const StreamParams& p, long long y, long long c0,
                                           bool active, float (&v)[4]) {
    const TS* in = static_cast<const TS*>(p.in);
    v[0] = v[1] = v[2] = v[3] = 0.f;
    if (!active) return;
    if (p.periodic) {
        const long long yy = wrap_index(y, p.ny);
        const TS* row = in + yy * p.nx;
        if (p.vec) {
            const long long cc = wrap_index(c0, p.nx);
            float4 q = Storage<TS>::load4(row + cc);
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = Storage<TS>::load1(row + wrap_index(c0 + e, p.nx));
        }
        return;
    }
    if (y < 0 || y >= p.ny) return;
    const TS* row = in + y * p.nx;
    if (p.vec && c0 >= 0 && c0 + 4 <= p.nx) {
        float4 q = Storage<TS>::load4(row + c0);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const long long c = c0 + e;
            if (c >= 0 && c < p.nx) v[e] = Storage<TS>::load1(row + c);
        }
    }
}

template <int R, bool STAR, int KMAX, typename TS>
__global__ void __launch_bounds__(256) sweep_stream_kernel(const __grid_constant__ StreamParams p) {
    constexpr int D = 2 * R + 1;
    extern __shared__ float4 smem_f4[];
    float* smem = reinterpret_cast<float*>(smem_f4);

    const int NT = blockDim.x;
    const int rowlen = 4 * NT + 8;  // 4 padding floats on each side keep 16-byte alignment
    const int tid = threadIdx.x;
    const int strip = blockIdx.x % p.strips;
    const int tile = blockIdx.x / p.strips;
    const long long x0 = (long long)strip * p.bx;  // first output column of the tile
    const long long y0 = (long long)tile * p.by;   // first output row of the tile
    const long long c0 = x0 - p.H + 4LL * tid;     // this thread's first column
    const int nlev = p.nlev;
    const long long ybeg = y0 - (long long)R * nlev;
    const long long ylast = min(y0 + p.by, p.ny);  // one past the last output row
    const bool active = 4 * tid < p.bx + 2 * p.H;

    for (int i = tid; i < 2 * KMAX * rowlen; i += NT) smem[i] = 0.f;

    // Columns outside the grid (zero rule) are forced to zero at every level.
    bool col_in[4];
    bool any_out = false;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        col_in[e] = p.periodic || (c0 + e >= 0 && c0 + e < p.nx);
        any_out |= !col_in[e];
    }
    const bool store_chunk = active && c0 >= x0 && c0 + 4 <= x0 + p.bx && c0 < p.nx;

    float acc[KMAX][D][4];
#pragma unroll
    for (int l = 0; l < KMAX; ++l)
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[l][m][e] = 0.f;

    const int nreal = (int)(ylast - y0) + 2 * R * nlev;  // row steps that matter
    const int nsteps = (nreal + D - 1) / D * D;          // rounded up to the unroll

    float nxt[4];
    load_chunk<TS>(p, ybeg, c0, active, nxt);
    __syncthreads();

    for (int s0 = 0; s0 < nsteps; s0 += D) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const int s = s0 + j;
            float cur[4] = {nxt[0], nxt[1], nxt[2], nxt[3]};
            if (s + 1 < nsteps) load_chunk<TS>(p, ybeg + s + 1, c0, active, nxt);
            const int par = s & 1;
#pragma unroll
            for (int l = 0; l < KMAX; ++l) {
                // Level l's row ybeg - l*R + s arrives; it feeds level l+1.
                if (l < nlev && s >= 2 * l * R) {
                    float* row = smem + (2 * l + par) * rowlen + 4;
                    *reinterpret_cast<float4*>(row + 4 * tid) =
                        make_float4(cur[0], cur[1], cur[2], cur[3]);
                    __syncthreads();
                    float h[4 + 2 * R];
#pragma unroll
                    for (int e = 0; e < 4; ++e) h[R + e] = cur[e];
                    if constexpr (R == 1) {
                        h[0] = row[4 * tid - 1];
                        h[5] = row[4 * tid + 4];
                    } else if constexpr (R == 2) {
                        float2 a = *reinterpret_cast<const float2*>(row + 4 * tid - 2);
                        float2 b = *reinterpret_cast<const float2*>(row + 4 * tid + 4);
                        h[0] = a.x; h[1] = a.y; h[2 * R + 4 - 2] = b.x; h[2 * R + 4 - 1] = b.y;
                    } else {
                        float4 a = *reinterpret_cast<const float4*>(row + 4 * tid - 4);
                        float4 b = *reinterpret_cast<const float4*>(row + 4 * tid + 4);
                        h[0] = a.y; h[1] = a.z; h[2] = a.w;
                        h[R + 4 + 0] = b.x; h[R + 4 + 1] = b.y; h[R + 4 + 2] = b.z;
                    }
                    // m = dy + R: this row is the (m+1)-th contribution to output row
                    // (arriving row) - dy, held in slot (j - m + R) mod D.
#pragma unroll
                    for (int m = 0; m < D; ++m) {
                        const int slot = (j - m + R + 2 * D) % D;
                        if (STAR && m != R) {
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float wv = p.w.w[m * D + R];
                                acc[l][slot][e] = (m == 0) ? wv * h[R + e]
                                                           : fmaf(wv, h[R + e], acc[l][slot][e]);
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                float a = (m == 0) ? p.w.w[m * D] * h[e]
                                                   : fmaf(p.w.w[m * D], h[e], acc[l][slot][e]);
#pragma unroll
                                for (int dx = 1; dx < D; ++dx) a = fmaf(p.w.w[m * D + dx], h[e + dx], a);
                                acc[l][slot][e] = a;
                            }
                        }
                    }
                    // Output row (arriving row) - R of level l+1 is complete.
                    const int cs = (j + R + 1) % D;
                    const long long yo = ybeg - (long long)(l + 1) * R + s;
                    const bool row_out = !p.periodic && (yo < 0 || yo >= p.ny);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float v = acc[l][cs][e];
                        if (row_out || (any_out && !col_in[e])) v = 0.f;
                        cur[e] = v;
                    }
                }
            }
            // cur holds level nlev's row ybeg - nlev*R + s.
            const long long yo = ybeg - (long long)R * nlev + s;
            if (store_chunk && yo >= y0 && yo < ylast) {
                TS* orow = static_cast<TS*>(p.out) + yo * p.nx;
                if (p.vec && c0 + 4 <= p.nx) {
                    Storage<TS>::store4(orow + c0, make_float4(cur[0], cur[1], cur[2], cur[3]));
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (c0 + e < p.nx) Storage<TS>::store1(orow + c0 + e, cur[e]);
                }
            }
        }
    }
}

// Host-side handle of one instantiation.
struct StreamKernelRef {
    const void* fn;
    int kmax;
};

}  // namespace gbst
