// sweep_stream.cuh -- row-streaming, temporally blocked Jacobi sweep (sm_103a).
//
// Computes K steps of the Jacobi update of Sec. II-C per launch:
//     u^{t+1}[i][j] = sum_{dy,dx} W[dy+R][dx+R] * u~^t[i+dy][j+dx]
// with u~ zero outside the grid (the fixed zero padding of Sec. IV-A) or
// wrapped (periodic).
//
// Decomposition.  A CTA owns an output tile of `by` rows x `bx` columns.  It
// loads a strip of bx + 2H columns (H >= R*K halo columns per side: the GPU
// counterpart of the paper's per-tile halo padding, Sec. IV-A step 3, made K
// times deeper so that K steps need no exchange with other CTAs) and streams
// down the rows from y0 - R*K to y0 + by - 1 + R*K.
//
// Each thread owns 4 adjacent columns, held as two column pairs so that the
// arithmetic runs as packed FP32x2 FMAs (one instruction, two FMAs): (c0, c2)
// and (c1, c3) for radius 1 (every own-column operand is then a register pair
// as it stands), (c0, c1) and (c2, c3) for radius 2 and 3 (measured faster
// there).  Time
// level l+1 is produced from level l as a pipeline along y: when row y of
// level l arrives it is the last contribution to output row y-R of level l+1
// and the first to row y+R.  A thread keeps 2R+1 partial sums per column and
// level in registers (a window sliding down the rows).  A completed
// level-(l+1) row is handed to level l+2 at the NEXT row step, so the K levels
// of one row step are independent: they share one barrier per row step (not
// one per level) and their arithmetic interleaves.  Only the R columns next to
// a thread's 4 columns cross threads: each level publishes its input row's edge
// values to a double-buffered shared-memory array (R = 1: separate left/right
// edge arrays, so every access is conflict-free and unit stride; R = 2, 3: the
// whole 16-byte chunk), does the products that need only its own columns,
// waits at the row step's barrier, then adds the products that need the
// neighbours' edges.
//
// Input rows stream from HBM into a shared-memory ring with cp.async, PF rows
// ahead (VEC kernels: rows are 16-byte aligned; out-of-grid chunks are
// zero-filled by the copy).  Kernels for widths that are not a multiple of 4
// load element by element into registers instead.  Only the level-K row goes
// back to HBM, so HBM traffic is ~(4+4)/K bytes per point-step for FP32 plus
// the overlap of neighbouring tiles' halos.
//
// Boundary.  With the zero rule, every level's values outside the grid are
// forced back to 0 after they are computed (only in tiles that touch the
// boundary), so the halo stays a frozen zero at every sub-step, as the
// padding does in the paper.  With the periodic rule, loads wrap and nothing
// is masked.  Rows before a level's first valid row hold finite garbage that
// never reaches a stored output (a level's valid rows only read valid rows).
//
// Summation order: each output accumulates dy = -R .. R as rows arrive; within
// a row the own-column products come first and the neighbour-column products
// after them, each group in ascending dx.  Star footprints skip the off-axis
// (zero) weights.  The order depends neither on K nor on the tile shape.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "../../include/stencil.h"
#include "common.cuh"

namespace gbst {

constexpr int kStreamMaxThreads = 256;

// Input rows in flight per thread (a power of 2).  Measured on GB300: 8 rows
// for K <= 2 gained nothing for the 13-point star and cost the 49-point box at
// 256-thread CTAs an occupancy step (its ring no longer fit twice per SM).
__host__ __device__ constexpr int stream_prefetch(int) { return 4; }

// Floats of one (level, parity) edge buffer, sized for the largest CTA so
// that every shared-memory offset is a compile-time constant.
__host__ __device__ constexpr int stream_buf_floats(int R) {
    return R == 3 ? 4 * (kStreamMaxThreads + 2) : 2 * R * (kStreamMaxThreads + 2);
}

// TMA-fed kernels: the ring's row mbarriers and the abort flag, after the ring.
constexpr int kStreamTmaCtlBytes = 128;
// Columns of one TMA box (one 512-byte piece of an FP32 ring row).
constexpr int kStreamTmaBox = 128;

// Dynamic shared memory of a launch with CTAs of `nt` threads: the input ring
// (VEC only; one slot of nt 4-element chunks per row in flight), the TMA
// control block (TMA-fed kernels) and 2K edge buffers.
__host__ __device__ constexpr int stream_smem_bytes(int R, int K, int elem_bytes, bool vec, bool tma = false,
                                                    int nt = kStreamMaxThreads) {
    return (vec ? stream_prefetch(K) * nt * 4 * elem_bytes : 0) + (tma ? kStreamTmaCtlBytes : 0) +
           2 * K * stream_buf_floats(R) * 4;
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
// Two scalar FMAs with one weight: the weight comes straight from the constant
// bank, where a packed FMA needs the (w, w) pair in registers.
__device__ __forceinline__ float2 sfma2(float w, float2 b, float2 c) {
    return make_float2(fmaf(w, b.x, c.x), fmaf(w, b.y, c.y));
}

// Weight sources for the tile body.  ParamWeights reads the (w, w) pairs from
// the kernel parameters (the constant bank); RegWeights holds a grid's pairs
// in registers (batched kernel, one weight set per grid).
struct ParamWeights {
    const StreamParams& p;
    __device__ __forceinline__ float2 w2(int i) const { return p.w2.w2[i]; }
};

template <int N>
struct RegWeights {
    float2 w[N];
    __device__ __forceinline__ float2 w2(int i) const { return w[i]; }
};

template <int R, class WS>
__device__ __forceinline__ float2 wgt2(const WS& ws, int m, int dx) {
    return ws.w2(m * (2 * R + 1) + dx + R);
}

// Products with scalar FMAs (weights straight from the constant bank) instead
// of packed FP32x2 FMAs, for footprints whose (w, w) pairs do not stay in
// registers: a packed FMA cannot take its pair from the constant bank, and
// reloading pairs per use runs a microbenchmark at a third of the speed of the
// scalar form (10.4 against 36.6 TFMA/s; pairs held in registers: 31.2).  The
// two forms round identically (a packed FMA is two FMAs).  Used for the 7x7
// box (49 pairs): 16384^2 FP32 478 -> 509 GStencil/s, BF16 storage 469 -> 489,
// and no spills left at k = 1; the 13-point star keeps its 7 off-axis pairs in
// registers and is faster packed (1272 against 1217 at k = 3).
__host__ __device__ constexpr bool stream_scalar_weights(int R, bool STAR) { return R == 3 && !STAR; }

template <int R, bool STAR, class WS>
__device__ __forceinline__ float2 wfma(const WS& ws, int m, int dx, float2 src, float2 acc) {
    if constexpr (stream_scalar_weights(R, STAR)) return sfma2(wgt2<R>(ws, m, dx).x, src, acc);
    else return ffma2(wgt2<R>(ws, m, dx), src, acc);
}

template <int R, bool STAR, class WS>
__device__ __forceinline__ float2 wmul(const WS& ws, int m, int dx, float2 src) {
    if constexpr (stream_scalar_weights(R, STAR)) {
        const float w = wgt2<R>(ws, m, dx).x;
        return make_float2(w * src.x, w * src.y);
    } else {
        return fmul2(wgt2<R>(ws, m, dx), src);
    }
}

// ---- input loading --------------------------------------------------------------

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gsrc, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    const int n = valid ? BYTES : 0;
    if constexpr (BYTES == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(n));
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gsrc), "r"(n));
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ---- TMA-fed ring (FP32 storage, zero rule, rows 16-byte aligned) -------------------
//
// One thread loads each input row of the strip with 2D tensor copies of
// kStreamTmaBox columns x 1 row into the ring slot; out-of-grid columns and
// rows are filled with zeros by the copy engine, which is the zero rule.
// Each slot has an mbarrier that the copies complete; every thread waits on
// it, with a time limit (an expired wait records STENCIL_ERR_TIMEOUT, raises
// the CTA's abort flag and the tile finishes without waiting again).

struct TmaRing {
    const CUtensorMap* map = nullptr;
    unsigned bar0 = 0;             // shared address of slot 0's mbarrier
    volatile int* abort = nullptr;  // CTA-wide flag in shared memory
};

__device__ __forceinline__ unsigned st_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void st_bar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void st_bar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool st_bar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ long long st_now() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void st_tma_row(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Wait for phase `parity` of `bar`; false if the CTA aborted or the limit ran out.
static __device__ __noinline__ bool st_wait_slow(unsigned bar, unsigned parity, volatile int* abort, unsigned* status,
                                          long long limit_ns) {
    const long long t0 = st_now();
    for (unsigned it = 0;; ++it) {
        if (st_bar_try(bar, parity)) return true;
        if (*abort) return false;
        if ((it & 63u) == 63u && (st_now() - t0 > limit_ns || it > (1u << 26))) {
            atomicCAS(status, 0u, (unsigned)STENCIL_ERR_TIMEOUT);
            *abort = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void st_wait(unsigned bar, unsigned parity, volatile int* abort, unsigned* status,
                                        long long limit_ns) {
    if (st_bar_try(bar, parity) || *abort) return;
    st_wait_slow(bar, parity, abort, status, limit_ns);
}

template <typename TS>
__device__ __forceinline__ void smem_chunk_to_f32(const void* src, float (&v)[4]) {
    if constexpr (sizeof(TS) == 4) {
        float4 q = *reinterpret_cast<const float4*>(src);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        uint2 raw = *reinterpret_cast<const uint2*>(src);
        float4 q;
        if constexpr (std::is_same<TS, __nv_bfloat16>::value) {
            float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&raw.x));
            float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&raw.y));
            q = make_float4(a.x, a.y, b.x, b.y);
        } else {
            float2 a = __half22float2(*reinterpret_cast<__half2*>(&raw.x));
            float2 b = __half22float2(*reinterpret_cast<__half2*>(&raw.y));
            q = make_float4(a.x, a.y, b.x, b.y);
        }
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
}

// Element-wise register load of one chunk (widths that are not a multiple of 4).
template <typename TS>
__device__ __forceinline__ void load_chunk_scalar(const StreamParams& p, int y, int c0, bool active,
                                                  float (&v)[4]) {
    const TS* in = static_cast<const TS*>(p.in);
    v[0] = v[1] = v[2] = v[3] = 0.f;
    if (!active) return;
    const int nx = (int)p.nx, ny = (int)p.ny;
    if (p.periodic) {
        const TS* row = in + (size_t)wrap_index(y, ny) * (size_t)p.ld;
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = Storage<TS>::load1(row + (int)wrap_index(c0 + e, nx));
        return;
    }
    if (y < 0 || y >= ny) return;
    const TS* row = in + (size_t)y * (size_t)p.ld;
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (c0 + e >= 0 && c0 + e < nx) v[e] = Storage<TS>::load1(row + c0 + e);
}

// ---- arithmetic -----------------------------------------------------------------
//
// Column pairs.  Radius 1: a thread's 4 columns c0..c3 are held as
// Pa = (c0, c2) and Pb = (c1, c3), and its outputs as A0 = (o0, o2),
// A1 = (o1, o3).  The weight (dy, dx) then updates pair q from the source pair
// (c[q+dx], c[q+dx+2]): for q+dx in {0, 1} that is Pa or Pb itself, so every
// own-column product takes its operands straight from registers; only the
// pairs that straddle a neighbour's columns are assembled.  Radius 2 and 3:
// adjacent pairs Pa = (c0, c1), Pb = (c2, c3) (measured faster there).  In both
// layouts a completed output pair is directly the next level's input pair.
//
// Weight rows.  Row m = dy + R of the weights multiplies the row that arrives
// m rows after the first input row of an output.  The products of one arriving
// row are split by m: rows m >= 1 go into partial sums that hold earlier rows'
// products already; row m = 0 starts a new partial sum (a multiply, no add).

// Own-column products, weight rows MLO..MHI, radius 1 layout.
template <int R, bool STAR, int MLO, int MHI, class WS>
__device__ __forceinline__ void own_products(const WS& p, float2 (&acc)[2 * R + 1][2], float2 Pa,
                                             float2 Pb, int j) {
    constexpr int D = 2 * R + 1;
#pragma unroll
    for (int m = MLO; m <= MHI; ++m) {
        const int slot = (j - m + R + 2 * D) % D;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            bool first = (m == 0);
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                if (STAR && m != R && dx != 0) continue;
                const int c = q + dx;
                if (c != 0 && c != 1) continue;
                const float2 src = c == 0 ? Pa : Pb;
                if (first) {
                    acc[slot][q] = wmul<R, STAR>(p, m, dx, src);
                    first = false;
                } else {
                    acc[slot][q] = wfma<R, STAR>(p, m, dx, src, acc[slot][q]);
                }
            }
        }
    }
}

// Products whose source pair straddles a neighbour column, weight rows
// MLO..MHI, radius 1 layout.  col.pair(c) = (column c, column c + 2) of the
// extended row (left halo, own, right halo).
template <int R, bool STAR, int MLO, int MHI, class WS, class COL>
__device__ __forceinline__ void halo_products(const WS& p, float2 (&acc)[2 * R + 1][2], const COL& col,
                                              int j) {
    constexpr int D = 2 * R + 1;
#pragma unroll
    for (int m = MLO; m <= MHI; ++m) {
        if (STAR && m != R) continue;
        const int slot = (j - m + R + 2 * D) % D;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                const int c = q + dx;
                if (c == 0 || c == 1) continue;
                acc[slot][q] = wfma<R, STAR>(p, m, dx, col.pair(c), acc[slot][q]);
            }
        }
    }
}

// Adjacent layout (radius 2, 3): the source of weight (dy, dx) for output pair
// q is (c[2q+dx], c[2q+dx+1]); own pairs are Pa = (c0,c1), Pb = (c2,c3) and
// mid = (c1, c2).
template <int R, bool STAR, int MLO, int MHI, class WS>
__device__ __forceinline__ void own_products_adj(const WS& p, float2 (&acc)[2 * R + 1][2], float2 Pa,
                                                 float2 Pb, float2 mid, int j) {
    constexpr int D = 2 * R + 1;
#pragma unroll
    for (int m = MLO; m <= MHI; ++m) {
        const int slot = (j - m + R + 2 * D) % D;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            bool first = (m == 0);
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                if (STAR && m != R && dx != 0) continue;
                const int c = 2 * q + dx;
                if (c < 0 || c + 1 > 3) continue;
                const float2 src = (c == 0) ? Pa : (c == 2 ? Pb : mid);
                if (STAR && R == 3 && m == R && !first) {
                    // radius-3 star, centre row: scalar FMAs keep these seven
                    // weights out of the register file (measured faster)
                    acc[slot][q] = sfma2(wgt2<R>(p, m, dx).x, src, acc[slot][q]);
                    continue;
                }
                if (first) {
                    acc[slot][q] = wmul<R, STAR>(p, m, dx, src);
                    first = false;
                } else {
                    acc[slot][q] = wfma<R, STAR>(p, m, dx, src, acc[slot][q]);
                }
            }
        }
    }
}

// Halo products, adjacent layout, general footprint: ext[i] = column i - R of
// the extended row.
template <int R, bool STAR, int MLO, int MHI, class WS>
__device__ __forceinline__ void halo_products_adj(const WS& p, float2 (&acc)[2 * R + 1][2],
                                                  const float (&ext)[4 + 2 * R], int j) {
    constexpr int D = 2 * R + 1;
#pragma unroll
    for (int m = MLO; m <= MHI; ++m) {
        if (STAR && m != R) continue;
        const int slot = (j - m + R + 2 * D) % D;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                const int c = 2 * q + dx;
                if (c >= 0 && c + 1 <= 3) continue;
                const float2 src = make_float2(ext[c + R], ext[c + 1 + R]);
                acc[slot][q] = wfma<R, STAR>(p, m, dx, src, acc[slot][q]);
            }
        }
    }
}

// Halo products of the radius-3 star (only weight row m = 3 reaches across
// columns).  lft = columns -4..-1, rgt = columns 4..7 as loaded from shared
// memory.  Every product runs as a scalar FMA with its weight from the
// constant bank: no pair has to be assembled first and no weight pair has to
// be held in registers.  Per output the products are added in ascending dx,
// the order halo_products_adj uses.
template <class WS>
__device__ __forceinline__ void halo_products_star3(const WS& p, float2 (&acc)[7][2], float4 lft,
                                                    float4 rgt, float2 Pa, float2 Pb, int j) {
    const int slot = (j - 3 + 3 + 14) % 7;
    float2 A0 = acc[slot][0], A1 = acc[slot][1];
    const float wm3 = wgt2<3>(p, 3, -3).x, wm1 = wgt2<3>(p, 3, -1).x;
    const float w1 = wgt2<3>(p, 3, 1).x, w3 = wgt2<3>(p, 3, 3).x;
    // outputs (o0, o1): dx = -3, -2, -1, 3
    A0.x = fmaf(wm3, lft.y, A0.x);
    A0.y = fmaf(wm3, lft.z, A0.y);
    A0 = sfma2(wgt2<3>(p, 3, -2).x, make_float2(lft.z, lft.w), A0);
    A0.x = fmaf(wm1, lft.w, A0.x);
    A0.y = fmaf(wm1, Pa.x, A0.y);
    A0.x = fmaf(w3, Pb.y, A0.x);
    A0.y = fmaf(w3, rgt.x, A0.y);
    // outputs (o2, o3): dx = -3, 1, 2, 3
    A1.x = fmaf(wm3, lft.w, A1.x);
    A1.y = fmaf(wm3, Pa.x, A1.y);
    A1.x = fmaf(w1, Pb.y, A1.x);
    A1.y = fmaf(w1, rgt.x, A1.y);
    A1 = sfma2(wgt2<3>(p, 3, 2).x, make_float2(rgt.x, rgt.y), A1);
    A1.x = fmaf(w3, rgt.y, A1.x);
    A1.y = fmaf(w3, rgt.z, A1.y);
    acc[slot][0] = A0;
    acc[slot][1] = A1;
}

// The extended row of one level-row for R = 1: own pairs plus the
// neighbours' edge columns hl (column -1) and hr (column 4).
template <int R>
struct ExtRow {
    float2 Pa, Pb;
    float hl, hr;
    __device__ __forceinline__ float at(int j) const {
        switch (j) {
            case 0: return Pa.x;
            case 1: return Pb.x;
            case 2: return Pa.y;
            case 3: return Pb.y;
        }
        return j < 0 ? hl : hr;
    }
    // (column c, column c+2)
    __device__ __forceinline__ float2 pair(int c) const { return make_float2(at(c), at(c + 2)); }
};

// Level schedule (see stream_tile): radius 1 forwards a completed row to the
// next level in the same row step; radius 2 and 3 hand it over one row step
// later (measured faster for each: the hand-over frees the K levels of a row
// step from one another but keeps more values live, which costs radius 1's
// deep blocks more occupancy than it gains).
__host__ __device__ constexpr bool stream_handover(int R) { return R >= 2; }

// Input rows a tile's row loop may load beyond its last output row: R*K for
// the halo, K-1 for the hand-over between levels (radius 2, 3), D-1 for
// rounding the loop up to its unroll.  A tile whose rows
// [y0 - R*K, ylast + stream_rows_after) lie in the grid needs no row bounds
// checks.
// The tile of CTA b in a grid of strips x tiles_y tiles.  The edge tiles (top
// and bottom tile rows, left and right strips), which run the slower checked
// path, come first: the block scheduler deals CTAs out to the SMs round-robin,
// so the first ones land on distinct SMs instead of doubling up on some (the
// launch lasts as long as its most loaded SM).  Then the interior tiles, row
// by row.
__device__ __forceinline__ void stream_tile_of(int b, int strips, int tiles_y, int& strip, int& tile) {
    if (strips < 3 || tiles_y < 3) {
        strip = b % strips;
        tile = b / strips;
        return;
    }
    const int ne = 2 * strips + 2 * (tiles_y - 2);
    if (b < 2 * strips) {
        strip = b % strips;
        tile = b < strips ? 0 : tiles_y - 1;
    } else if (b < ne) {
        const int i = b - 2 * strips;
        strip = (i & 1) ? strips - 1 : 0;
        tile = 1 + (i >> 1);
    } else {
        const int i = b - ne;
        strip = 1 + i % (strips - 2);
        tile = 1 + i / (strips - 2);
    }
}

// Edge tiles decide per group of row steps whether completed rows can lie
// outside the grid (two copies of the group body) for radius 1; radius 2 and 3
// check every level row (the second copy pushes the 13-point star at K = 3
// from ~140 to 344 bytes of spills: 1249 -> 1088 GStencil/s, while the
// 9-point box at K = 8 gains 2081 -> 2152).
__host__ __device__ constexpr bool stream_row_gate(int R) { return R == 1; }

__host__ __device__ constexpr int stream_rows_after(int R, int K) {
    return R * K + (stream_handover(R) ? K : 0) + 2 * R + 1;
}

// One CTA's tile.  EDGE = the tile loads rows or columns outside the grid:
// loads are bounds-checked (zero rule) or wrapped (periodic), and with the
// zero rule every level's out-of-grid values are forced to 0.  Interior tiles
// run without any of that.
//
// Schedule.  Level l (l = 0 .. K-1) turns time level l into l+1; level 0 takes
// input row ybeg + s at row step s.  Radius 1 (same-step forwarding): level
// l >= 1 takes the row that level l-1 completes in the same step, after one
// barrier per level.  Radius 2, 3 (hand-over): level l >= 1 takes the row that
// level l-1 completed at step s-1, so the K levels of one row step do not
// depend on one another and share ONE barrier: (A) every level publishes its input row's edge
// columns and adds its own-column products of weight rows 1..2R; barrier;
// (B) from the top level down, every level adds its halo products, then starts
// the partial sum of weight row 0 in the slot its completed row was handed over
// from (the level above has consumed it by then), masks its newly completed
// row (zero rule, edge tiles) and, at the top level, stores it.  Per output the
// products are still added row by row (dy = -R .. R), own columns before
// neighbour columns, so the result does not depend on the schedule or on K.
template <int R, bool STAR, int K, typename TS, bool VEC, bool EDGE, bool TMA = false, bool ALL = false,
          bool SKIPCOL = false, class WS>
__device__ __forceinline__ void stream_tile(const StreamParams& p, const WS& ws, char* ring,
                                            float* ebuf, int NT, int tid, int x0, int y0,
                                            TmaRing tma = TmaRing{}) {
    constexpr int D = 2 * R + 1;
    constexpr int SZ = stream_buf_floats(R);
    constexpr int PF = stream_prefetch(K);
    constexpr int CB = 4 * (int)sizeof(TS);  // bytes of one 4-column chunk
    const int SLOT = NT * CB;                // bytes of one ring slot (one row of the strip)
    const int ny = (int)p.ny, nx = (int)p.nx;
    const size_t ld = (size_t)p.ld;
    const int c0 = x0 - p.H + 4 * tid;  // this thread's first column
    const int ybeg = y0 - R * K;
    const int ylast = min(y0 + p.by, ny);  // one past the last output row
    const bool active = 4 * tid < p.bx + 2 * p.H;
    const bool periodic = EDGE && p.periodic != 0;
    const bool mask = EDGE && !periodic;

    bool col_in[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) col_in[e] = !mask || (c0 + e >= 0 && c0 + e < nx);
    // SKIPCOL (16-byte chunks, edge arrays zeroed when the tile starts): a
    // chunk outside the grid never publishes its edge columns, so its
    // neighbours read the zeros of the edge arrays, and its own values, which
    // nothing else reads or stores, need no mask; only rows outside the grid
    // are masked.
    static_assert(!SKIPCOL || VEC, "SKIPCOL needs whole 16-byte chunks");
    const bool pub = !(EDGE && SKIPCOL && mask) || (c0 >= 0 && c0 < nx);
    const bool store_chunk = active && c0 >= x0 && c0 + 4 <= x0 + p.bx && c0 < nx;

    float2 acc[K][D][2];
#pragma unroll
    for (int l = 0; l < K; ++l)
#pragma unroll
        for (int m = 0; m < D; ++m) acc[l][m][0] = acc[l][m][1] = make_float2(0.f, 0.f);

    // Level K-1 completes output row ybeg + s - (K-1)(R+1) - R at step s with
    // the hand-over, ybeg + s - K*R without.
    constexpr int HAND = stream_handover(R) ? 1 : 0;
    const int nreal = (ylast - y0) + 2 * R * K + HAND * (K - 1);  // row steps that matter
    const int nsteps = (nreal + D - 1) / D * D;            // rounded up to the unroll

    // VEC: the chunk this thread copies for row y.
    const TS* gin = static_cast<const TS*>(p.in);
    const int cw = periodic ? (int)wrap_index(c0, nx) : c0;
    // A whole chunk is copied when it lies inside the row pitch; with the zero
    // rule, columns in [nx, ld) are masked like any other out-of-grid column.
    const bool col_ok = !EDGE || (active && (periodic || (c0 >= 0 && c0 + 4 <= (int)ld)));
    char* my_ring = ring + tid * CB;
    const TS* my_src = gin + (EDGE ? 0 : (ptrdiff_t)ybeg * (ptrdiff_t)ld + c0);
    auto issue_row = [&](int s) {
        if constexpr (TMA) {
            // Warp 0 copies the strip's row ybeg + s into ring slot s % PF: lane b
            // issues box b (kStreamTmaBox columns), lane 0 also arms the slot's
            // mbarrier with the row's byte count.  The slot last held row s - PF,
            // read by every thread at that row step, before a barrier this warp
            // has passed since; each issuing lane's proxy fence orders those reads
            // before the copy engine's writes.
            const int nbox = (NT * 4) / kStreamTmaBox;
            if (tid < nbox && s < nsteps && !*tma.abort) {
                const int slot = s & (PF - 1);
                const unsigned bar = tma.bar0 + 8u * (unsigned)slot;
                const unsigned dst = st_smem(ring + slot * SLOT) + (unsigned)(tid * kStreamTmaBox * 4);
                const int xs = x0 - p.H + tid * kStreamTmaBox;
                // the copy's first column must be 16-byte aligned, and so must its
                // destination (128 bytes: every box starts on a 512-byte boundary)
                if ((xs & 3) || (dst & 127u)) {
                    atomicCAS(p.status, 0u, (unsigned)STENCIL_ERR_DEVICE_CHECK);
                    *tma.abort = 1;
                    return;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (tid == 0) {
                    // (test hook: CTA 0 waits for 16 bytes more than its first row
                    // brings, so that wait runs out and the timeout path is exercised)
                    const unsigned extra = (p.debug_withhold && blockIdx.x == 0 && s == 0) ? 16u : 0u;
                    st_bar_expect_tx(bar, (unsigned)(nbox * kStreamTmaBox * 4) + extra);
                }
                st_tma_row(dst, tma.map, xs, ybeg + s, bar);
            }
            return;
        }
        bool ok = s < nsteps;
        const TS* src;
        if constexpr (EDGE) {
            const int y = ybeg + s;
            int yy = y;
            ok = ok && col_ok;
            if (periodic) {
                yy = (int)wrap_index(y, ny);
            } else {
                ok = ok && y >= 0 && y < ny;
            }
            src = ok ? gin + (size_t)yy * ld + cw : gin;
        } else {
            src = ok ? my_src + (size_t)s * ld : gin;
        }
        cp_async<CB>(my_ring + (s & (PF - 1)) * SLOT, src, ok);
        cp_async_commit();
    };

    float nreg0[4], nreg1[4];  // register prefetch (non-VEC)
    if constexpr (VEC || TMA) {
#pragma unroll
        for (int s = 0; s < PF - 1; ++s) issue_row(s);
    } else {
        load_chunk_scalar<TS>(p, ybeg, c0, active, nreg0);
        load_chunk_scalar<TS>(p, ybeg + 1, c0, active, nreg1);
    }

    // One group of D row steps; MR: some level row the group completes may lie
    // outside the grid (zero rule, edge tiles), so completed rows are checked.
    // Deciding once per group keeps the row checks out of the groups that
    // cannot need them (a branch around whole groups, not per level row).
    auto group = [&](int s0, auto mr) {
        constexpr bool MR = decltype(mr)::value;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const int s = s0 + j;
            const int cin = (j + R) % D;        // slot completed at the previous step
            const int cdone = (j + R + 1) % D;  // slot completed at this step
            float cur[4];                       // level 0's input row
            if constexpr (TMA) {
                issue_row(s + PF - 1);
                st_wait(tma.bar0 + 8u * (unsigned)(s & (PF - 1)), (unsigned)((s / PF) & 1), tma.abort, p.status,
                        p.wait_ns);
                smem_chunk_to_f32<TS>(my_ring + (s & (PF - 1)) * SLOT, cur);
            } else if constexpr (VEC) {
                issue_row(s + PF - 1);
                cp_async_wait<PF - 1>();
                smem_chunk_to_f32<TS>(my_ring + (s & (PF - 1)) * SLOT, cur);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) { cur[e] = nreg0[e]; nreg0[e] = nreg1[e]; }
                if (s + 2 < nsteps) load_chunk_scalar<TS>(p, ybeg + s + 2, c0, active, nreg1);
            }
            float* bpar = ebuf + (s & 1) * SZ;
            if constexpr (!HAND) {
                // Same-step forwarding (radius 1): level l's completed row is
                // level l+1's input row of this step; one barrier per level.
                float2 Pa = make_float2(cur[0], cur[2]), Pb = make_float2(cur[1], cur[3]);
#pragma unroll
                for (int l = 0; l < K; ++l) {
                    float* B = bpar + 2 * l * SZ;
                    if (pub) {
                        B[tid + 1] = Pa.x;                          // column 0
                        B[kStreamMaxThreads + 2 + tid + 1] = Pb.y;  // column 3
                    }
                    own_products<R, STAR, 0, 2 * R>(ws, acc[l], Pa, Pb, j);
                    __syncthreads();
                    ExtRow<R> ext;
                    ext.Pa = Pa;
                    ext.Pb = Pb;
                    ext.hl = B[kStreamMaxThreads + 2 + tid];
                    ext.hr = B[tid + 2];
                    halo_products<R, STAR, 0, 2 * R>(ws, acc[l], ext, j);
                    // Output row (arriving row) - R of level l+1 is complete.
                    Pa = acc[l][cdone][0];
                    Pb = acc[l][cdone][1];
                    if constexpr (EDGE && (MR || !SKIPCOL || !stream_row_gate(R))) {
                        if (mask) {
                            const int yo = ybeg - (l + 1) * R + s;
                            const bool row_out = (unsigned)yo >= (unsigned)ny;
                            if constexpr (SKIPCOL) {
                                if (row_out) Pa = Pb = make_float2(0.f, 0.f);
                            } else {
                                if (row_out || !col_in[0]) Pa.x = 0.f;
                                if (row_out || !col_in[2]) Pa.y = 0.f;
                                if (row_out || !col_in[1]) Pb.x = 0.f;
                                if (row_out || !col_in[3]) Pb.y = 0.f;
                            }
                        }
                    }
                    if constexpr (ALL) {
                        const int yo = ybeg - (l + 1) * R + s;
                        if (l < K - 1 && store_chunk && yo >= y0 && yo < ylast)
                            Storage<TS>::store4(static_cast<TS*>(p.lvl_out[l]) + (size_t)yo * ld + c0,
                                                make_float4(Pa.x, Pb.x, Pa.y, Pb.y));
                    }
                }
                const int yo = ybeg - R * K + s;
                if (store_chunk && yo >= y0 && yo < ylast) {
                    TS* orow = static_cast<TS*>(p.out) + (size_t)yo * ld;
                    const float4 o = make_float4(Pa.x, Pb.x, Pa.y, Pb.y);
                    if (VEC) {
                        Storage<TS>::store4(orow + c0, o);
                    } else {
                        const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (c0 + e < nx) Storage<TS>::store1(orow + c0 + e, ov[e]);
                    }
                }
            } else {
            // Hand-over (radius 2, 3).  The input pairs of level l at this step.
            auto level_in = [&](int l, float2& Pa, float2& Pb) {
                if (l == 0) {
                    if constexpr (R == 1) {
                        Pa = make_float2(cur[0], cur[2]);
                        Pb = make_float2(cur[1], cur[3]);
                    } else {
                        Pa = make_float2(cur[0], cur[1]);
                        Pb = make_float2(cur[2], cur[3]);
                    }
                } else {
                    Pa = acc[l - 1][cin][0];
                    Pb = acc[l - 1][cin][1];
                }
            };
            // (A) publish edges, own-column products of weight rows 1..2R.
#pragma unroll
            for (int l = 0; l < K; ++l) {
                float* B = bpar + 2 * l * SZ;
                float2 Pa, Pb;
                level_in(l, Pa, Pb);
                if constexpr (R == 1) {
                    if (pub) {
                        B[tid + 1] = Pa.x;                          // column 0
                        B[kStreamMaxThreads + 2 + tid + 1] = Pb.y;  // column 3
                    }
                    own_products<R, STAR, 1, 2 * R>(ws, acc[l], Pa, Pb, j);
                } else {
                    if (pub) reinterpret_cast<float4*>(B)[tid + 1] = make_float4(Pa.x, Pa.y, Pb.x, Pb.y);
                    own_products_adj<R, STAR, 1, 2 * R>(ws, acc[l], Pa, Pb, make_float2(Pa.y, Pb.x), j);
                }
            }
            __syncthreads();
            // (B) top level first: halo products, weight row 0, mask, store.
#pragma unroll
            for (int l = K - 1; l >= 0; --l) {
                const float* B = bpar + 2 * l * SZ;
                float2 Pa, Pb;
                level_in(l, Pa, Pb);
                if constexpr (R == 1) {
                    ExtRow<R> ext;
                    ext.Pa = Pa;
                    ext.Pb = Pb;
                    ext.hl = B[kStreamMaxThreads + 2 + tid];
                    ext.hr = B[tid + 2];
                    halo_products<R, STAR, 1, 2 * R>(ws, acc[l], ext, j);
                    own_products<R, STAR, 0, 0>(ws, acc[l], Pa, Pb, j);
                    halo_products<R, STAR, 0, 0>(ws, acc[l], ext, j);
                } else {
                    const float4 a = reinterpret_cast<const float4*>(B)[tid];
                    const float4 b = reinterpret_cast<const float4*>(B)[tid + 2];
                    if constexpr (STAR && R == 3) {
                        halo_products_star3(ws, acc[l], a, b, Pa, Pb, j);
                        own_products_adj<R, STAR, 0, 0>(ws, acc[l], Pa, Pb, make_float2(Pa.y, Pb.x), j);
                    } else {
                        float ext[4 + 2 * R];
                        ext[R + 0] = Pa.x;
                        ext[R + 1] = Pa.y;
                        ext[R + 2] = Pb.x;
                        ext[R + 3] = Pb.y;
                        const float lft[4] = {a.x, a.y, a.z, a.w}, rgt[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            ext[i] = lft[4 - R + i];
                            ext[R + 4 + i] = rgt[i];
                        }
                        halo_products_adj<R, STAR, 1, 2 * R>(ws, acc[l], ext, j);
                        own_products_adj<R, STAR, 0, 0>(ws, acc[l], Pa, Pb, make_float2(Pa.y, Pb.x), j);
                        halo_products_adj<R, STAR, 0, 0>(ws, acc[l], ext, j);
                    }
                }
                // acc[l][cdone] is level l+1's row ybeg + s - l(R+1) - R, complete.
                if constexpr (EDGE && (MR || !SKIPCOL || !stream_row_gate(R))) {
                    if (mask) {
                        const int yo = ybeg + s - l * (R + 1) - R;
                        const bool row_out = (unsigned)yo >= (unsigned)ny;
                        float2& A0 = acc[l][cdone][0];
                        float2& A1 = acc[l][cdone][1];
                        if constexpr (SKIPCOL) {
                            if (row_out) A0 = A1 = make_float2(0.f, 0.f);
                        } else {
                            // element e of the chunk: R == 1 (A0.x, A1.x, A0.y, A1.y),
                            // else (A0.x, A0.y, A1.x, A1.y)
                            constexpr int e_a0y = R == 1 ? 2 : 1, e_a1x = R == 1 ? 1 : 2;
                            if (row_out || !col_in[0]) A0.x = 0.f;
                            if (row_out || !col_in[e_a0y]) A0.y = 0.f;
                            if (row_out || !col_in[e_a1x]) A1.x = 0.f;
                            if (row_out || !col_in[3]) A1.y = 0.f;
                        }
                    }
                }
                if constexpr (ALL) {
                    const int yo = ybeg + s - l * (R + 1) - R;
                    if (l < K - 1 && store_chunk && yo >= y0 && yo < ylast) {
                        const float2 A0 = acc[l][cdone][0], A1 = acc[l][cdone][1];
                        Storage<TS>::store4(static_cast<TS*>(p.lvl_out[l]) + (size_t)yo * ld + c0,
                                            make_float4(A0.x, A0.y, A1.x, A1.y));
                    }
                }
                if (l == K - 1) {
                    const int yo = ybeg + s - (K - 1) * (R + 1) - R;
                    if (store_chunk && yo >= y0 && yo < ylast) {
                        const float2 A0 = acc[l][cdone][0], A1 = acc[l][cdone][1];
                        const float4 o = R == 1 ? make_float4(A0.x, A1.x, A0.y, A1.y)
                                                : make_float4(A0.x, A0.y, A1.x, A1.y);
                        TS* orow = static_cast<TS*>(p.out) + (size_t)yo * ld;
                        if (VEC) {
                            Storage<TS>::store4(orow + c0, o);
                        } else {
                            const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (c0 + e < nx) Storage<TS>::store1(orow + c0 + e, ov[e]);
                        }
                    }
                }
            }
            }  // hand-over
        }
    };
    for (int s0 = 0; s0 < nsteps; s0 += D) {
        if constexpr (EDGE && SKIPCOL && stream_row_gate(R)) {
            // level rows completed in this group: ybeg + s0 - K(R+1) .. ybeg + s0 + D - 1
            if (mask && (ybeg + s0 - K * (R + 1) < 0 || ybeg + s0 + D > ny))
                group(s0, std::true_type{});
            else
                group(s0, std::false_type{});
        } else {
            group(s0, std::true_type{});
        }
    }
    if constexpr (TMA) {
        __syncthreads();  // every thread is done with the ring before the next tile's rows arrive
    } else if constexpr (VEC) {
        cp_async_wait<0>();
    }
}

// Minimum resident 256-thread CTAs per SM the compiler must allow for (2: at
// most 128 registers a thread, 3: 85; 0: no such bound, the compiler's own
// choice, which differs from an explicit 1).  Measured on GB300 at 8192^2 with
// per-instantiation register caps (same bits in every case): a 128-register cap
// lifts the 5-point star at K = 8 from 2359 to 2731 GStencil/s, the 9-point box
// at K = 6 from 1770 to 1842, the 13-point star at K = 3 / 4 from 1108 / 844 to
// 1172 / 971 (it fits 4 CTAs instead of 3 / 2), the 49-point box at K = 2 from
// 388 to 398; an 85-register cap lifts the 49-point box at K = 1 from 335 to
// 353.  The 9-point box at K = 8 and the 13-point star at K = 2 are fastest
// uncapped.
__host__ __device__ constexpr int stream_min_blocks(int R, bool STAR, int K) {
    return (R == 1 && STAR && K >= 6) ? 2
         : (R == 1 && !STAR && K == 6) ? 2
         : (R == 3 && STAR && K >= 3) ? 2
         : (R == 3 && !STAR && K == 2) ? 2
         : (R == 3 && !STAR && K == 1) ? 3
         : 0;
}

// ALL: every time level of the launch is stored (level l+1 to p.lvl_out[l],
// the last to p.out), for callers that need each state (the adjoint's
// recomputation of a segment); VEC kernels only.
template <int R, bool STAR, int K, typename TS, bool VEC, bool ALL = false>
__global__ void __launch_bounds__(kStreamMaxThreads, stream_min_blocks(R, STAR, K))
    sweep_stream_kernel(const __grid_constant__ StreamParams p) {
    constexpr int PF = stream_prefetch(K);
    constexpr int CB = 4 * (int)sizeof(TS);
    extern __shared__ float4 smem_f4[];
    const int NT = blockDim.x;
    char* ring = reinterpret_cast<char*>(smem_f4);
    float* ebuf = reinterpret_cast<float*>(ring + (VEC ? PF * NT * CB : 0));
    const int tid = threadIdx.x;
    int strip, tile;
    stream_tile_of(blockIdx.x, p.strips, gridDim.x / p.strips, strip, tile);
    const int x0 = strip * p.bx;  // first output column of the tile
    const int y0 = tile * p.by;   // first output row of the tile

    for (int i = tid; i < 2 * K * stream_buf_floats(R); i += NT) ebuf[i] = 0.f;
    __syncthreads();

    // Interior: every row this CTA loads (including the rounded-up tail of the
    // row loop) and every column of its strip lies inside the grid.
    const int ny = (int)p.ny, nx = (int)p.nx;
    const int ylast = min(y0 + p.by, ny);
    const bool interior = VEC && y0 - R * K >= 0 && ylast + stream_rows_after(R, K) <= ny &&
                          x0 - p.H >= 0 && x0 - p.H + 4 * NT <= nx;
    const ParamWeights ws{p};
    // (edge tiles of 16-byte-chunk kernels: the edge arrays were zeroed above,
    // so chunks outside the grid may leave them alone, SKIPCOL)
    if (interior)
        stream_tile<R, STAR, K, TS, VEC, false, false, ALL>(p, ws, ring, ebuf, NT, tid, x0, y0);
    else
        stream_tile<R, STAR, K, TS, VEC, true, false, ALL, VEC>(p, ws, ring, ebuf, NT, tid, x0, y0);
}

// The same sweep with the input rows brought in by the tensor-memory-access
// engine (FP32 storage, zero rule, rows of a multiple of 4 elements): `map`
// describes the input grid (nx x ny, row pitch ld, box kStreamTmaBox x 1).
template <int R, bool STAR, int K>
__global__ void __launch_bounds__(kStreamMaxThreads, stream_min_blocks(R, STAR, K))
    sweep_stream_tma_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ StreamParams p) {
    constexpr int PF = stream_prefetch(K);
    constexpr int CB = 16;
    extern __shared__ __align__(1024) float4 smem_tma[];
    const int NT = blockDim.x;
    char* ring = reinterpret_cast<char*>(smem_tma);
    char* ctl = ring + PF * NT * CB;
    float* ebuf = reinterpret_cast<float*>(ctl + kStreamTmaCtlBytes);
    const int tid = threadIdx.x;
    int strip, tile;
    stream_tile_of(blockIdx.x, p.strips, gridDim.x / p.strips, strip, tile);
    const int x0 = strip * p.bx;
    const int y0 = tile * p.by;
    TmaRing tma;
    tma.map = &map;
    tma.bar0 = st_smem(ctl);
    tma.abort = reinterpret_cast<volatile int*>(ctl + 8 * PF);
    if (tid == 0) {
        for (int i = 0; i < PF; ++i) st_bar_init(tma.bar0 + 8u * (unsigned)i, 1);
        *tma.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < 2 * K * stream_buf_floats(R); i += NT) ebuf[i] = 0.f;
    __syncthreads();

    const int ny = (int)p.ny, nx = (int)p.nx;
    const int ylast = min(y0 + p.by, ny);
    const bool interior = y0 - R * K >= 0 && ylast + stream_rows_after(R, K) <= ny && x0 - p.H >= 0 &&
                          x0 - p.H + 4 * NT <= nx;
    const ParamWeights ws{p};
    if (interior)
        stream_tile<R, STAR, K, float, true, false, true>(p, ws, ring, ebuf, NT, tid, x0, y0, tma);
    else
        stream_tile<R, STAR, K, float, true, true, true, false, true>(p, ws, ring, ebuf, NT, tid, x0, y0, tma);
}

// Host-side handle of one instantiation.
struct StreamKernelRef {
    const void* fn;
    int kmax;
};

}  // namespace gbst
