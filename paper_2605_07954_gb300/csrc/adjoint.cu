// adjoint.cu -- reverse-mode gradient of T Jacobi steps (stencil_adjoint).
//
// Forward (Sec. II-C): u_{t+1} = A u_t, (A u)[i][j] = sum_{dy,dx} W[dy+R][dx+R] u~[i+dy][j+dx].
// For a loss L(u_T) with lambda_T = dL/du_T:
//     lambda_t = A^T lambda_{t+1},  (A^T l)[p][q] = sum_{dy,dx} W[dy+R][dx+R] l~[p-dy][q-dx]
//              (a correlation with the flipped weights, same boundary rule),
//     dL/dW[dy+R][dx+R] = sum_{t<T} sum_{i,j} lambda_{t+1}[i][j] u~_t[i+dy][j+dx],
//     dL/du_0 = lambda_0.
//
// Memory: the states u_t are recomputed, not stored: a checkpoint every s
// steps (s = ceil(sqrt(T)) by default) is written by a temporally blocked
// forward pass; walking the segments backwards, each segment's s states are
// recomputed from its checkpoint (temporally blocked launches that store every
// time level), then the adjoint steps of the segment run from its last state
// down to its first.  Both forward paths use the same per-point arithmetic, so
// the result does not depend on s.
//
// adjoint_step_kernel fuses, for one step, the lambda update and the
// weight-gradient products: a CTA stages a 32x64 tile of lambda_{t+1} and of
// u_t with an R-wide halo in shared memory, writes lambda_t for the tile, and
// adds the tile's (2R+1)^2 products lambda_{t+1} * shifted(u_t) to a per-tile
// FP64 partial.  Tile t of a launch is always CTA t and launches are ordered,
// so each partial sums its steps in a fixed order; a last kernel sums the
// partials over tiles in a fixed order.  The gradient is deterministic.
// adjoint_stream_kernel does the same step with rows streamed through
// registers instead of a staged tile (radius 1, widths a multiple of 4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "../../include/stencil.h"
#include "common.cuh"

namespace gbst {

// Internal accessors of a plan (plan.cu).
void plan_weights(const stencil_plan_t* p, float* w);
void** plan_aux_slot(stencil_plan_t* p, int id);
void plan_set_aux_free(stencil_plan_t* p, int id, void (*freer)(void*));
stencil_status_t plan_run_states(stencil_plan_t* p, const void* in, float* const* outs, int64_t n,
                                 cudaStream_t st);

constexpr int kAdjTX = 32;          // output tile columns (one per lane)
constexpr int kAdjTY = 64;          // output tile rows
constexpr int kAdjRowsPerThread = 8;  // 8 warps x 8 rows

// One reverse step on a 32 x 64 tile.  Lane tx owns column x0 + tx and warp ty
// rows y0 + 8 ty .. + 7; it walks its rows keeping the last 2R+1 staged rows
// of lambda_{t+1} and u_t (its column +- R) in registers, so each row costs
// 2 (2R+1) shared-memory loads for (2R+1)^2 lambda FMAs and (2R+1)^2 gradient FMAs.
template <int R>
__global__ void __launch_bounds__(256)
    adjoint_step_kernel(const float* __restrict__ lam_in, const float* __restrict__ u,
                        float* __restrict__ lam_out, double* __restrict__ partials, int ny, int nx,
                        int periodic, Weights w, int tiles_x) {
    constexpr int D = 2 * R + 1;
    constexpr int SY = kAdjTY + 2 * R, SX = kAdjTX + 2 * R;
    __shared__ float sl[SY][SX + 1];
    __shared__ float su[SY][SX + 1];
    __shared__ float red[8][D * D];
    const int tx = threadIdx.x, ty = threadIdx.y;  // (32, 8)
    const int x0 = (blockIdx.x % tiles_x) * kAdjTX;
    const int y0 = (blockIdx.x / tiles_x) * kAdjTY;

    // Stage both tiles with their halo (zero outside, or wrapped).  Every
    // thread issues all of its loads before its first shared-memory store, so
    // the DRAM latencies overlap.  Item i = tid + 256 it is staged row i / SX,
    // column i % SX, advanced without division.
    {
        constexpr int ITEMS = SY * SX, ITERS = (ITEMS + 255) / 256;
        const int tid0 = ty * 32 + tx;
        int r = tid0 / SX, c = tid0 % SX;
        float va[ITERS], vb[ITERS];
        int ra[ITERS], ca[ITERS];
#pragma unroll
        for (int it = 0; it < ITERS; ++it) {
            ra[it] = r;
            ca[it] = c;
            va[it] = vb[it] = 0.f;
            if (r < SY) {
                int y = y0 - R + r, x = x0 - R + c;
                bool ok = y >= 0 && y < ny && x >= 0 && x < nx;
                if (periodic) {
                    y = (y % ny + ny) % ny;
                    x = (x % nx + nx) % nx;
                    ok = true;
                }
                if (ok) {
                    const size_t i = (size_t)y * nx + x;
                    va[it] = __ldg(lam_in + i);
                    vb[it] = __ldg(u + i);
                }
            }
            c += 256 % SX;
            r += 256 / SX;
            if (c >= SX) {
                c -= SX;
                ++r;
            }
        }
#pragma unroll
        for (int it = 0; it < ITERS; ++it) {
            if (ra[it] < SY) {
                sl[ra[it]][ca[it]] = va[it];
                su[ra[it]][ca[it]] = vb[it];
            }
        }
    }
    __syncthreads();

    float g[D * D];
#pragma unroll
    for (int k = 0; k < D * D; ++k) g[k] = 0.f;
    // Register windows: wl[i][e] = lambda staged row (row0 + i), column tx + e;
    // wu likewise for u.  The output row o = r0 + k needs lambda rows o-R..o+R
    // (flipped correlation) and u rows o-R..o+R.
    const int r0 = ty * kAdjRowsPerThread;  // first output row (tile-local)
    float wl[D][D], wu[D][D];
#pragma unroll
    for (int i = 0; i < D - 1; ++i)
#pragma unroll
        for (int e = 0; e < D; ++e) {
            wl[i + 1][e] = sl[r0 + i][tx + e];
            wu[i + 1][e] = su[r0 + i][tx + e];
        }
#pragma unroll
    for (int k = 0; k < kAdjRowsPerThread; ++k) {
        // slide: drop the oldest staged row, append staged row r0 + k + 2R
#pragma unroll
        for (int i = 0; i < D - 1; ++i)
#pragma unroll
            for (int e = 0; e < D; ++e) {
                wl[i][e] = wl[i + 1][e];
                wu[i][e] = wu[i + 1][e];
            }
#pragma unroll
        for (int e = 0; e < D; ++e) {
            wl[D - 1][e] = sl[r0 + k + 2 * R][tx + e];
            wu[D - 1][e] = su[r0 + k + 2 * R][tx + e];
        }
        // window row i holds staged row r0 + k + i, i.e. grid row o - R + i for o = y0 + r0 + k
        const int y = y0 + r0 + k, x = x0 + tx;
        if (y >= ny || x >= nx) continue;
        // lambda_t[o] = sum_d W[d] lambda_{t+1}[o - d], dy-major then dx
        float acc = 0.f;
#pragma unroll
        for (int dy = -R; dy <= R; ++dy)
#pragma unroll
            for (int dx = -R; dx <= R; ++dx)
                acc = fmaf(w.w[(dy + R) * D + (dx + R)], wl[R - dy][R - dx], acc);
        lam_out[(size_t)y * nx + x] = acc;
        // dL/dW[d] += lambda_{t+1}[o] * u_t[o + d]
        const float lp = wl[R][R];
#pragma unroll
        for (int dy = -R; dy <= R; ++dy)
#pragma unroll
            for (int dx = -R; dx <= R; ++dx)
                g[(dy + R) * D + (dx + R)] = fmaf(lp, wu[R + dy][R + dx], g[(dy + R) * D + (dx + R)]);
    }
    // Fixed-order reduction: butterfly within each warp, then warps in order.
#pragma unroll
    for (int k = 0; k < D * D; ++k) {
        float v = g[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (tx == 0) red[ty][k] = v;
    }
    __syncthreads();
    const int tid = ty * 32 + tx;
    if (tid < D * D) {
        double s = 0.0;
        for (int wv = 0; wv < 8; ++wv) s += (double)red[wv][tid];
        partials[(size_t)blockIdx.x * D * D + tid] += s;
    }
}

// grad_w[k] = sum over tiles of partials[tile][k] in a fixed order: thread i of
// the block sums tiles i, i + 256, ... in increasing order, then the 256
// thread sums are added pairwise in a fixed tree.  One block per tap.
__global__ void __launch_bounds__(256)
    reduce_partials_kernel(const double* __restrict__ partials, int tiles, int taps,
                           double* __restrict__ grad_w) {
    __shared__ double sh[256];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int t = threadIdx.x; t < tiles; t += 256) s += partials[(size_t)t * taps + k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad_w[k] = sh[0];
}

// Row-streaming variant of the reverse step (radius 1, widths a multiple of
// 4).  A warp owns a 128-column strip of kAdsRows output rows, 4 adjacent
// columns per lane, and walks down the rows of lambda_{t+1} holding the last
// 2R+1 of them in registers, each extended by R columns on either side (the
// neighbouring lanes' columns by shuffles, the strip's outer columns loaded by
// lanes 0 and 31).  Rows arrive as 16-byte chunks kAdsAhead rows before their
// use; nothing goes through shared memory on the way.
//
// The arithmetic runs as packed FP32x2 FMAs on column pairs: own pairs
// (c0, c1), (c2, c3) and the three pairs that straddle them, (c-1, c0),
// (c1, c2), (c3, c4), built once per row.  Every tap (dy, dx) reads the same
// pair of the extended lambda_{t+1} row for both products of an output pair:
//   lambda_t[o][x]   += W[dy][dx] * lambda_{t+1}[o - dy][x - dx]
//   dL/dW[dy][dx]    += u_t[o][x] * lambda_{t+1}[o - dy][x - dx]
// The second line is the weight gradient sum_o lambda_{t+1}[o] u_t[o + d]
// with its terms grouped by the u_t point (o + d -> o): every (point, tap)
// term is counted once, by the warp that owns the u_t row, and lambda_{t+1}
// outside the grid is zero (or wrapped) as in the lambda update, so u_t is
// read only at the warp's own points, without halo.  Per output the lambda
// update is adjoint_step_kernel's, in the same order (bit-identical lambda);
// each thread adds its gradient products row by row, the CTA reduces them in
// a fixed order into its FP64 partial.
//
// A warp whose rows and halo columns all lie inside the grid walks without any
// bounds or wrap logic (pointer increments, unconditional loads); warps at the
// grid's edge take the checked path.
//
// Measured on GB300 (Heat 4096^2, reverse steps back to back over distinct
// u_t): 38.4 us per step against 29-31 us for a plain kernel that reads two
// grids and writes one; the previous form of this step (scalar FMAs, every
// load checked, gradient per lambda point with a u_t window) took 47.3 us at
// about 235 warp instructions per output row, this one issues about 120.  More
// rows in flight
// (5 or 8 ahead in registers: fewer CTAs per SM; or a per-warp shared-memory
// ring fed by bulk copies, 5 or 8 rows ahead), 7, 22, 25, 28 or 31 rows per
// warp, and the warps of a CTA side by side instead of stacked all measured
// the same or slower; evict-first loads of the rows that die with the step
// gained ~7 %.  Two reverse steps per pass (lambda_{t-1} from lambda_{t+1} in
// registers, the middle 120 of each warp's 128 columns stored: 8 B per
// point-step instead of 12, bit-identical lambda) ran 37.2-40.3 us per step
// against 36.8-38.1 for the single step (136 registers and 3 CTAs per SM, or
// 128 with spills and 4): the step is bound by the latency of each warp's row
// walk, not by the bytes it moves.
constexpr int kAdsWarps = 4;    // warps per CTA, stacked vertically
constexpr int kAdsRows = 16;    // output rows per warp
constexpr int kAdsCols = 128;   // strip width (32 lanes x 4 columns)
constexpr int kAdsAhead = 2;    // rows loaded ahead of their use
constexpr int kAdsHint = 1;     // L2 policy of the row loads and stores (AdsPolicy)

template <int R>
struct AdsRow {
    float4 v;     // the lane's 4 columns
    float h[R];   // lane 0: columns x0 - R .. x0 - 1; lane 31: x0 + 128 .. x0 + 127 + R
};

// Grid row y of g as lane `lane` of the strip at x0 needs it; zero outside the
// grid, or wrapped.  c = x0 + 4 lane is a multiple of 4 and nx % 4 == 0, so a
// chunk lies wholly inside or wholly outside the grid, and its wrapped image
// is again an aligned chunk.
template <int R>
__device__ __forceinline__ void ads_load(AdsRow<R>& a, const float* __restrict__ g, int y, int c, int x0,
                                         int lane, int ny, int nx, bool periodic) {
    bool rok = true;
    if (periodic) {
        if (y < 0 || y >= ny) y = (y % ny + ny) % ny;
    } else {
        rok = y >= 0 && y < ny;
    }
    const float* row = g + (size_t)(rok ? y : 0) * (size_t)nx;
    int cc = c;
    bool cok = true;
    if (periodic) {
        if (cc >= nx) cc %= nx;
    } else {
        cok = cc < nx;
    }
    a.v = rok && cok ? __ldg(reinterpret_cast<const float4*>(row + cc)) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int xc = lane == 0 ? x0 - R + i : x0 + kAdsCols + i;
        bool ok = rok && (lane == 0 || lane == 31);
        if (periodic) {
            if (xc < 0 || xc >= nx) xc = (xc % nx + nx) % nx;
        } else {
            ok = ok && xc >= 0 && xc < nx;
        }
        a.h[i] = ok ? __ldg(row + xc) : 0.f;
    }
}

// Column pairs of one extended row (radius 1).
struct AdsPairs {
    float2 p0, p1;      // (c0, c1), (c2, c3)
    float2 sm, sc, sp;  // (c-1, c0), (c1, c2), (c3, c4)
};

__device__ __forceinline__ AdsPairs ads_pairs(const AdsRow<1>& a, int lane) {
    const float l = __shfl_up_sync(0xffffffffu, a.v.w, 1);
    const float r = __shfl_down_sync(0xffffffffu, a.v.x, 1);
    AdsPairs e;
    e.p0 = make_float2(a.v.x, a.v.y);
    e.p1 = make_float2(a.v.z, a.v.w);
    e.sm = make_float2(lane == 0 ? a.h[0] : l, a.v.x);
    e.sc = make_float2(a.v.y, a.v.z);
    e.sp = make_float2(a.v.w, lane == 31 ? a.h[0] : r);
    return e;
}

// Columns (2q + s, 2q + 1 + s) of the extended row, s in {-1, 0, 1}.
__device__ __forceinline__ float2 ads_pick(const AdsPairs& e, int q, int s) {
    if (q == 0) return s < 0 ? e.sm : s == 0 ? e.p0 : e.sc;
    return s < 0 ? e.sc : s == 0 ? e.p1 : e.sp;
}

// The lambda update and gradient products of one output row o = yb + k: pair
// q of the row's 4 columns, window slot (jj - R - dy) mod D holding lambda_{t+1}
// row o - dy, uu = u_t row o.
template <int D>
__device__ __forceinline__ float4 ads_products(const AdsPairs (&win)[D], int jj, float4 uu,
                                               const float2 (&wp)[D * D], float2 (&g)[D * D]) {
    constexpr int R = 1;
    const float2 U[2] = {make_float2(uu.x, uu.y), make_float2(uu.z, uu.w)};
    float2 acc[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        acc[q] = make_float2(0.f, 0.f);
#pragma unroll
        for (int dy = -R; dy <= R; ++dy)
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                const int t = (dy + R) * D + (dx + R);
                const float2 L = ads_pick(win[(jj - R - dy + 2 * D) % D], q, -dx);
                acc[q] = __ffma2_rn(wp[t], L, acc[q]);
                g[t] = __ffma2_rn(U[q], L, g[t]);
            }
    }
    return make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
}

// L2 eviction priorities of the reverse step's row traffic (createpolicy and
// .L2::cache_hint, PTX ISA).  lambda_{t+1} and u_t are dead once this step has
// read them; lambda_t is read again by the next reverse step at once and, for
// grids up to about half the L2, can stay there if the dead rows leave first.
// HINT 0: default policy; 1: loads evict-first; 2: loads evict-first and
// stores evict-last; 3: stores evict-last only.
template <int HINT>
struct AdsPolicy {
    unsigned long long first = 0, last = 0;
    __device__ __forceinline__ AdsPolicy() {
        if (HINT == 1 || HINT == 2) asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(first));
        if (HINT >= 2) asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(last));
    }
    __device__ __forceinline__ float4 load4(const float* p) const {
        if (HINT == 1 || HINT == 2) {
            float4 v;
            asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                : "l"(p), "l"(first));
            return v;
        }
        return __ldg(reinterpret_cast<const float4*>(p));
    }
    __device__ __forceinline__ float load1(const float* p) const {
        if (HINT == 1 || HINT == 2) {
            float v;
            asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(first));
            return v;
        }
        return __ldg(p);
    }
    __device__ __forceinline__ void store4(float* p, float4 v) const {
        if (HINT >= 2) {
            asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                         "f"(v.z), "f"(v.w), "l"(last)
                         : "memory");
        } else {
            *reinterpret_cast<float4*>(p) = v;
        }
    }
};

// One warp's walk over its ROWS output rows, rows in flight held in registers
// (AHEAD rows ahead).  EDGE: rows or halo columns may fall outside the grid
// (checked loads, wrap, skipped outputs).
template <bool EDGE, int AHEAD, int ROWS, class POL>
__device__ __forceinline__ void ads_walk(const float* __restrict__ lam_in, const float* __restrict__ u,
                                         float* __restrict__ lam_out, float2 (&g)[9], int ny, int nx,
                                         bool per, const Weights& w, int x0, int yb, int lane, const POL& pol) {
    constexpr int R = 1, D = 3;
    constexpr int NR = ROWS + 2 * R;  // lambda rows walked: yb - R .. yb + ROWS - 1 + R
    constexpr int RING = AHEAD + 1;
    constexpr int G = RING % D == 0 ? RING : D * RING;  // a group: lcm(D, RING) rows (D = 3 is prime)
    static_assert(NR % G == 0, "ring and window indices are static within a group of rows");
    const int c = x0 + 4 * lane;
    const bool col_ok = c < nx;
    const size_t snx = (size_t)nx;
    float2 wp[D * D];  // (w, w) pairs for the packed FMAs
#pragma unroll
    for (int k = 0; k < D * D; ++k) wp[k] = make_float2(w.w[k], w.w[k]);

    AdsRow<1> ra[RING];  // lambda_{t+1} rows in flight, slot = walked row % RING
    float4 ru[RING];     // u_t rows in flight, slot = (output row + 2R) % RING, i.e. the
                         // walked row whose step uses it
    AdsPairs win[D];     // extended lambda_{t+1} rows, slot = walked row % D
    // interior walk: pointers to the next row to load (never formed at EDGE)
    const float* pl = nullptr;
    const float* ph = nullptr;
    const float* pu = nullptr;
    float* po = nullptr;
    if (!EDGE) {
        pl = lam_in + (size_t)(yb - R) * snx + c;
        ph = lam_in + (size_t)(yb - R) * snx + (lane == 0 ? x0 - R : x0 + kAdsCols);
        pu = u + (size_t)yb * snx + c;
        po = lam_out + (size_t)yb * snx + c;
    }
    const bool hl = lane == 0 || lane == 31;
    auto load_lam = [&](AdsRow<1>& a, int i) {  // walked row i
        if (EDGE) {
            ads_load<1>(a, lam_in, yb - R + i, c, x0, lane, ny, nx, per);
        } else {
            a.v = pol.load4(pl);
            a.h[0] = hl ? pol.load1(ph) : 0.f;
            pl += snx;
            ph += snx;
        }
    };
    auto load_u = [&](float4& v, int k) {  // output row yb + k
        if (EDGE) {
            const int y = yb + k;
            v = y < ny && col_ok ? __ldg(reinterpret_cast<const float4*>(u + (size_t)y * snx + c))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            v = pol.load4(pu);
            pu += snx;
        }
    };
    // the rows the first AHEAD steps use (output row k is used at walked row k + 2R)
#pragma unroll
    for (int i = 0; i < AHEAD; ++i) {
        load_lam(ra[i % RING], i);
        if (i - 2 * R >= 0 && i - 2 * R < ROWS) load_u(ru[i % RING], i - 2 * R);
    }
    // A rolled loop over groups of rows (a fully unrolled walk overflows the
    // instruction cache); inside a group every ring and window index is static.
#pragma unroll 1
    for (int s0 = 0; s0 < NR; s0 += G) {
#pragma unroll
        for (int jj = 0; jj < G; ++jj) {
            const int i = s0 + jj;
            if (i + AHEAD < NR) load_lam(ra[(jj + AHEAD) % RING], i + AHEAD);
            const int ku = i + AHEAD - 2 * R;  // used at walked row i + AHEAD
            if (ku >= 0 && ku < ROWS) load_u(ru[(jj + AHEAD) % RING], ku);
            win[jj % D] = ads_pairs(ra[jj % RING], lane);
            // output row o = yb + k, k = i - 2R; lambda_{t+1} row o - dy is walked
            // row i - R - dy, in window slot (jj - R - dy) mod D
            const int k = i - 2 * R, o = yb + k;
            if (k < 0) continue;
            if (EDGE && (o >= ny || !col_ok)) continue;
            const float4 res = ads_products<D>(win, jj % D, ru[jj % RING], wp, g);
            if (EDGE) {
                *reinterpret_cast<float4*>(lam_out + (size_t)o * snx + c) = res;
            } else {
                pol.store4(po, res);
                po += snx;
            }
        }
    }
}

// The reverse step (radius 1; AHEAD, ROWS: see ads_walk; HINT: L2 eviction
// priorities, see AdsPolicy).
template <int R, int AHEAD = kAdsAhead, int ROWS = kAdsRows, int HINT = kAdsHint>
__global__ void __launch_bounds__(kAdsWarps * 32, 5)
    adjoint_stream_kernel(const float* __restrict__ lam_in, const float* __restrict__ u,
                          float* __restrict__ lam_out, double* __restrict__ partials, int ny, int nx,
                          int periodic, Weights w, int tiles_x) {
    static_assert(R == 1, "the row-streaming reverse step is written for radius 1");
    constexpr int D = 2 * R + 1;
    __shared__ float red[kAdsWarps][D * D];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = (blockIdx.x % tiles_x) * kAdsCols;
    const int yb = (blockIdx.x / tiles_x) * (kAdsWarps * ROWS) + warp * ROWS;
    float2 g[D * D];
#pragma unroll
    for (int k = 0; k < D * D; ++k) g[k] = make_float2(0.f, 0.f);
    const AdsPolicy<HINT> pol;
    // interior: the warp's rows yb - R .. yb + ROWS - 1 + R and columns
    // x0 - R .. x0 + 127 + R lie in the grid
    const bool interior = yb >= R && yb + ROWS + R <= ny && x0 >= R && x0 + kAdsCols + R <= nx;
    if (interior)
        ads_walk<false, AHEAD, ROWS>(lam_in, u, lam_out, g, ny, nx, periodic != 0, w, x0, yb, lane, pol);
    else
        ads_walk<true, AHEAD, ROWS>(lam_in, u, lam_out, g, ny, nx, periodic != 0, w, x0, yb, lane, pol);
    // Fixed-order reduction: the pair halves, a butterfly within each warp,
    // then the warps in order.
#pragma unroll
    for (int k = 0; k < D * D; ++k) {
        float v = g[k].x + g[k].y;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < D * D) {
        double s = 0.0;
#pragma unroll
        for (int wv = 0; wv < kAdsWarps; ++wv) s += (double)red[wv][threadIdx.x];
        partials[(size_t)blockIdx.x * D * D + threadIdx.x] += s;
    }
}

// Radius 1 only: at radius 2 the two register windows (5 rows x 8 columns
// each) take the kernel to 225 registers, and the staged-tile step is kept.
static const void* adjoint_stream_kernel_fn(int R) {
    return R == 1 ? (const void*)adjoint_stream_kernel<1> : nullptr;
}

static const void* adjoint_kernel(int R) {
    switch (R) {
        case 1: return (const void*)adjoint_step_kernel<1>;
        case 2: return (const void*)adjoint_step_kernel<2>;
        case 3: return (const void*)adjoint_step_kernel<3>;
        default: return nullptr;
    }
}

}  // namespace gbst

using namespace gbst;

namespace {

thread_local std::string g_adj_error;

stencil_status_t afail(stencil_status_t st, const std::string& msg) {
    g_adj_error = msg;
    return st;
}

#define ACK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return afail(STENCIL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Device scratch of the adjoint, kept by the plan and grown on demand.
struct AdjScratch {
    float* base = nullptr;
    size_t grids = 0;
    double* partials = nullptr;
    size_t npartials = 0;
};

void adj_scratch_free(void* v) {
    AdjScratch* sc = static_cast<AdjScratch*>(v);
    if (sc->base) cudaFree(sc->base);
    if (sc->partials) cudaFree(sc->partials);
    delete sc;
}

stencil_status_t adj_scratch(stencil_plan_t* plan, size_t grids, size_t grid_bytes, size_t npartials,
                             AdjScratch** out) {
    void** slot = plan_aux_slot(plan, 0);
    AdjScratch* sc = static_cast<AdjScratch*>(*slot);
    if (!sc) {
        sc = new (std::nothrow) AdjScratch();
        if (!sc) return afail(STENCIL_ERR_OOM, "host allocation failed");
        *slot = sc;
        plan_set_aux_free(plan, 0, adj_scratch_free);
    }
    if (sc->grids < grids) {
        if (sc->base) cudaFree(sc->base);
        sc->base = nullptr;
        sc->grids = 0;
        if (cudaMalloc(&sc->base, grids * grid_bytes) != cudaSuccess) {
            cudaGetLastError();
            sc->base = nullptr;
            return afail(STENCIL_ERR_OOM, "cudaMalloc of " + std::to_string(grids) + " adjoint grids failed");
        }
        sc->grids = grids;
    }
    if (sc->npartials < npartials) {
        if (sc->partials) cudaFree(sc->partials);
        sc->partials = nullptr;
        sc->npartials = 0;
        if (cudaMalloc(&sc->partials, sizeof(double) * npartials) != cudaSuccess) {
            cudaGetLastError();
            sc->partials = nullptr;
            return afail(STENCIL_ERR_OOM, "cudaMalloc of the gradient partials failed");
        }
        sc->npartials = npartials;
    }
    *out = sc;
    return STENCIL_OK;
}

}  // namespace

extern "C" {

const char* stencil_adjoint_last_error(void) { return g_adj_error.c_str(); }

stencil_status_t stencil_adjoint(stencil_plan_t* plan, const void* u0, const void* grad_uT, int64_t T,
                                 void* grad_u0, double* grad_w, int64_t ckpt_interval,
                                 stencil_stream_t stream) {
    if (!plan || !u0 || !grad_uT || !grad_u0) return afail(STENCIL_ERR_INVALID_ARG, "NULL argument");
    if (T < 0 || ckpt_interval < 0) return afail(STENCIL_ERR_INVALID_ARG, "T and ckpt_interval must be >= 0");
    stencil_plan_info_t info{};
    stencil_status_t s = stencil_plan_info(plan, &info);
    if (s != STENCIL_OK) return afail(s, "stencil_plan_info failed");
    if (info.dtype != STENCIL_F32 || info.compute != STENCIL_COMPUTE_FP32)
        return afail(STENCIL_ERR_UNSUPPORTED, "the adjoint supports FP32 CUDA-core plans only");
    const int R = info.radius, D = 2 * R + 1;
    const int ny = (int)info.ny, nx = (int)info.nx;
    const size_t n = (size_t)ny * (size_t)nx;
    const size_t bytes = n * sizeof(float);
    cudaStream_t st = (cudaStream_t)stream;
    Weights wf{};
    plan_weights(plan, wf.w);
    Weights wadj = wf;  // the step kernels index W directly; the flip is in their loops

    // The row-streaming step where it applies (its 16-byte row chunks need
    // nx % 4 == 0, and the buffers below are then 16-byte aligned), else the
    // staged-tile step.
    const bool streamed = adjoint_stream_kernel_fn(R) != nullptr && nx % 4 == 0;
    const int tiles_x = streamed ? (nx + kAdsCols - 1) / kAdsCols : (nx + kAdjTX - 1) / kAdjTX;
    const int tile_rows = streamed ? kAdsWarps * kAdsRows : kAdjTY;
    const int tiles = tiles_x * ((ny + tile_rows - 1) / tile_rows);
    if (T == 0) {
        if (grad_u0 != grad_uT) ACK(cudaMemcpyAsync(grad_u0, grad_uT, bytes, cudaMemcpyDeviceToDevice, st));
        if (grad_w) ACK(cudaMemsetAsync(grad_w, 0, sizeof(double) * D * D, st));
        return STENCIL_OK;
    }
    const int64_t sgm = ckpt_interval > 0 ? std::min<int64_t>(ckpt_interval, T)
                                          : (int64_t)std::ceil(std::sqrt((double)T));
    const int64_t nseg = (T + sgm - 1) / sgm;
    // Buffers: nseg checkpoints, sgm segment states, two adjoint grids.
    AdjScratch* sc = nullptr;
    const size_t grids = (size_t)nseg + (size_t)sgm + 2;
    s = adj_scratch(plan, grids, bytes, (size_t)(tiles + 1) * D * D, &sc);
    if (s != STENCIL_OK) return s;
    float* ckpt = sc->base;
    float* seg = sc->base + (size_t)nseg * n;
    float* lam[2] = {sc->base + (size_t)(nseg + sgm) * n, sc->base + (size_t)(nseg + sgm + 1) * n};
    double* partials = sc->partials;
    ACK(cudaMemsetAsync(partials, 0, sizeof(double) * (size_t)tiles * D * D, st));

    // Checkpoints u_{j*sgm}, j = 0..nseg-1 (temporally blocked forward).
    ACK(cudaMemcpyAsync(ckpt, u0, bytes, cudaMemcpyDeviceToDevice, st));
    for (int64_t j = 1; j < nseg; ++j) {
        s = stencil_run(plan, ckpt + (size_t)(j - 1) * n, ckpt + (size_t)j * n, sgm, stream);
        if (s != STENCIL_OK) return afail(s, std::string("checkpoint pass: ") + stencil_last_error());
    }
    ACK(cudaMemcpyAsync(lam[0], grad_uT, bytes, cudaMemcpyDeviceToDevice, st));
    int cur = 0;
    const void* kfn = streamed ? adjoint_stream_kernel_fn(R) : adjoint_kernel(R);
    if (!kfn) return afail(STENCIL_ERR_UNSUPPORTED, "no adjoint kernel for this radius");
    const dim3 block = streamed ? dim3(kAdsWarps * 32) : dim3(32, 8);
    int periodic = info.boundary == STENCIL_BOUNDARY_PERIODIC;
    std::vector<float*> segp((size_t)sgm);
    for (int64_t j = nseg - 1; j >= 0; --j) {
        const int64_t t0 = j * sgm;
        const int64_t len = std::min<int64_t>(sgm, T - t0);
        // states u_{t0} .. u_{t0+len-1}: seg[0] is the checkpoint itself; the
        // others come from temporally blocked launches that store every level
        const float* state0 = ckpt + (size_t)j * n;
        if (len > 1) {
            for (int64_t t = 1; t < len; ++t) segp[t - 1] = seg + (size_t)t * n;
            s = plan_run_states(plan, state0, segp.data(), len - 1, st);
            if (s != STENCIL_OK) return afail(s, std::string("segment recompute: ") + stencil_last_error());
        }
        for (int64_t t = len - 1; t >= 0; --t) {
            const float* ut = t == 0 ? state0 : seg + (size_t)t * n;
            const float* lin = lam[cur];
            float* lout = lam[cur ^ 1];
            void* args[] = {(void*)&lin, (void*)&ut, (void*)&lout, (void*)&partials,
                            (void*)&ny, (void*)&nx, (void*)&periodic, (void*)&wadj, (void*)&tiles_x};
            ACK(cudaLaunchKernel(kfn, dim3((unsigned)tiles), block, args, 0, st));
            cur ^= 1;
        }
    }
    ACK(cudaMemcpyAsync(grad_u0, lam[cur], bytes, cudaMemcpyDeviceToDevice, st));
    if (grad_w) {
        const int taps = D * D;
        // grad_w may be host memory: then the sums go to the tail of the
        // partials scratch first and are copied back, synchronising `stream`.
        cudaPointerAttributes pa{};
        const bool host = cudaPointerGetAttributes(&pa, grad_w) != cudaSuccess ||
                          pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeUnregistered;
        (void)cudaGetLastError();
        double* dst = host ? partials + (size_t)tiles * D * D : grad_w;
        reduce_partials_kernel<<<taps, 256, 0, st>>>(partials, tiles, taps, dst);
        ACK(cudaGetLastError());
        if (host) {
            ACK(cudaMemcpyAsync(grad_w, dst, sizeof(double) * taps, cudaMemcpyDeviceToHost, st));
            ACK(cudaStreamSynchronize(st));
        }
    }
    return STENCIL_OK;
}

int64_t stencil_adjoint_launches(const stencil_plan_t* plan, int64_t T, int64_t ckpt_interval) {
    if (!plan || T < 0 || ckpt_interval < 0) return -1;
    if (T == 0) return 0;
    const int64_t sgm = ckpt_interval > 0 ? std::min<int64_t>(ckpt_interval, T)
                                          : (int64_t)std::ceil(std::sqrt((double)T));
    const int64_t nseg = (T + sgm - 1) / sgm;
    int64_t L = (nseg - 1) * stencil_run_launches(plan, sgm);  // checkpoints
    stencil_plan_info_t info{};
    const bool fused = stencil_plan_info(plan, &info) == STENCIL_OK && info.dtype == STENCIL_F32 &&
                       info.nx % 4 == 0;
    for (int64_t j = 0; j < nseg; ++j) {  // segment recompute: all-states launches of 8/4/2/1 steps
        int64_t m = std::min<int64_t>(sgm, T - j * sgm) - 1;
        if (!fused) {
            L += m * stencil_run_launches(plan, 1);
            continue;
        }
        const int top = info.radius == 3 && !info.shape ? 2 : (info.radius == 1 ? 8 : 4);
        for (int d = top; d >= 1 && m > 0; d /= 2)
            while (m >= d) {
                m -= d;
                ++L;
            }
    }
    L += T;      // adjoint steps
    return L + 1;  // reduction
}

}  // extern "C"
