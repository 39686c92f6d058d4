// box49_tc.cu -- the 7x7 box stencil (Box2d-3r) as a tensor-core contraction.
//
// One Jacobi step (Sec. II-C) of a radius-3 box is, for each weight row di,
// a product of row-shifted input with a banded Toeplitz matrix (the idea of
// casting a stencil as a matrix product, Sec. II-D):
//
//   out[r][c0 + n] = sum_di sum_k A_di[r][k] * B_di[k][n],  n = 0..7, k = 0..15,
//   A_di[r][k] = in[r + di - 3][c0 - 4 + k],
//   B_di[k][n] = W[di][k - n - 1]  if 0 <= k - n - 1 <= 6, else 0.
//
// A_di is just the staged input tile read di rows lower, so no im2col copy is
// made: ldmatrix takes any row as the start of a fragment.  The K extent (16)
// starts 4 columns left of the output tile so every fragment row is 16-byte
// aligned; 7 of the 16 B entries per column are non-zero (44 % of the MMA's
// multiply-adds are useful, against 18 % or less for a square-tile GEMM
// formulation).  Each 8-column chunk of A serves as the upper half of one
// output tile's K range and the lower half of the next tile's, so it is
// loaded once and used twice.
//
// Engines (warp-level mma.sync, FP32 accumulate):
//   TF32: m16n8k8, inputs and weights rounded to TF32 (round-to-nearest-even);
//         two MMAs per (tile, di).
//   BF16: m16n8k16, inputs and weights rounded to BF16 (RN-even); one MMA per
//         (tile, di).
//   3xTF32 (accuracy recovery): FP32 storage staged unrounded; every A
//         fragment and weight splits into x = hi + lo with hi = tf32(x),
//         lo = tf32(x - hi), and each product is hi*hi + hi*lo + lo*hi (the
//         lo*lo term, ~2^-22 relative, is dropped), the two small products
//         accumulated first.  Six MMAs per (tile, di); error near FP32.
// CTA: 8 warps, 128x128 outputs; warp w owns rows 16w..16w+15 and all 16
// column tiles.  The staged tile is (128+6) x (128+8) elements, with a row
// pitch padded so the 8 row addresses of every ldmatrix fall in distinct banks.
//
// Two kernels:
//   box49_tc_pipe_kernel (16-byte aligned rows; FP32+TF32 or BF16+BF16): a
//     persistent CTA double-buffers its tiles with cp.async (zero-filled out of
//     the grid, wrapped for periodic), so the next tile streams in while the
//     current one runs on the tensor cores.  Between the steps of one run the
//     FP32 state is kept TF32-rounded (every launch but the last rounds its
//     output), so the staged data is already in MMA format; only the first
//     launch rounds its (caller's) input in shared memory.  Each step's input
//     is thus rounded to TF32 exactly once, as with rounding at load.
//   box49_tc_kernel (any layout and storage/engine pair): one tile per CTA,
//     loads converted in registers while staging.
// One step per launch (HBM-bound: 8 B per point for FP32 storage, 4 for BF16).
#include <cuda_runtime.h>

#include "common.cuh"

namespace gbst {

constexpr int kTcRows = 128, kTcCols = 128;
constexpr int kTcSR = kTcRows + 6;       // staged rows: y0-3 .. y0+130
constexpr int kTcSC = kTcCols + 8;       // staged cols: x0-4 .. x0+131
constexpr int kTcQPR = kTcSC / 4;        // 4-element groups per staged row (34)
constexpr int kTcPitchF32 = kTcSC + 4;   // 140 words: row stride 560 B (= 48 mod 128)
constexpr int kTcPitchB16 = kTcSC + 16;  // 152 halves: row stride 304 B (= 48 mod 128)

struct TcParams {
    const void* in;
    void* out;
    int ny, nx, ld;
    int periodic;
    int tiles_x, tiles;
    int vec;         // 16-byte aligned rows (elements multiple of 4)
    int convert_in;  // pipelined TF32: round the staged input to TF32 (first launch)
    int round_out;   // pipelined TF32: store TF32-rounded values (all but the last launch)
    float w[49];
};

__device__ __forceinline__ unsigned f32_to_tf32(float x) {
    unsigned r;
    asm("cvt.rn.satfinite.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

template <typename TS>
__device__ __forceinline__ float load_elem(const TcParams& p, int y, int x) {
    const TS* in = static_cast<const TS*>(p.in);
    if (p.periodic) {
        y = (y % p.ny + p.ny) % p.ny;
        x = (x % p.nx + p.nx) % p.nx;
    } else if (y < 0 || y >= p.ny || x < 0 || x >= p.nx) {
        return 0.f;
    }
    return Storage<TS>::load1(in + (size_t)y * p.ld + x);
}

// The 7 banded Toeplitz B fragments, B_di[k][n] = W[di][k - n - 1].
// TF32: [kc0 b0, kc0 b1, kc1 b0, kc1 b1]; BF16: [b0, b1, -, -].
template <bool BF16MMA>
__device__ __forceinline__ void make_bfrag(const TcParams& p, int g, int t, unsigned (&bfr)[7][4]) {
    auto bw = [&](int di, int k, int n) -> float {
        const int dj = k - n - 1;
        return (dj >= 0 && dj <= 6) ? p.w[di * 7 + dj] : 0.f;
    };
#pragma unroll
    for (int di = 0; di < 7; ++di) {
        if constexpr (BF16MMA) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(bw(di, 2 * t, g), bw(di, 2 * t + 1, g));
            __nv_bfloat162 hi = __floats2bfloat162_rn(bw(di, 2 * t + 8, g), bw(di, 2 * t + 9, g));
            bfr[di][0] = *reinterpret_cast<unsigned*>(&lo);
            bfr[di][1] = *reinterpret_cast<unsigned*>(&hi);
            bfr[di][2] = bfr[di][3] = 0u;
        } else {
            bfr[di][0] = f32_to_tf32(bw(di, t, g));
            bfr[di][1] = f32_to_tf32(bw(di, t + 4, g));
            bfr[di][2] = f32_to_tf32(bw(di, t + 8, g));
            bfr[di][3] = f32_to_tf32(bw(di, t + 12, g));
        }
    }
}

// 3xTF32: hi / lo parts of the Toeplitz B fragments (TF32 layout).
__device__ __forceinline__ void make_bfrag_split(const TcParams& p, int g, int t, unsigned (&bhi)[7][4],
                                                 unsigned (&blo)[7][4]) {
    auto bw = [&](int di, int k, int n) -> float {
        const int dj = k - n - 1;
        return (dj >= 0 && dj <= 6) ? p.w[di * 7 + dj] : 0.f;
    };
#pragma unroll
    for (int di = 0; di < 7; ++di) {
        const float v[4] = {bw(di, t, g), bw(di, t + 4, g), bw(di, t + 8, g), bw(di, t + 12, g)};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            bhi[di][i] = f32_to_tf32(v[i]);
            blo[di][i] = f32_to_tf32(v[i] - __uint_as_float(bhi[di][i]));
        }
    }
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// All MMAs of one warp's 16x128 output strip from a staged tile at `stile`.
// ldmatrix is issued one chunk ahead of the MMAs that use it.
template <bool BF16MMA>
__device__ __forceinline__ void tile_mma(const void* stile, int warp, int lane, const unsigned (&bfr)[7][4],
                                         float (&acc)[16][4]) {
    const int r0 = 16 * warp;
#pragma unroll
    for (int di = 0; di < 7; ++di) {
        if constexpr (BF16MMA) {
            const int row = r0 + di + (lane & 7) + 8 * ((lane >> 3) & 1);
            const unsigned base = (unsigned)__cvta_generic_to_shared(
                static_cast<const __nv_bfloat16*>(stile) + row * kTcPitchB16);
            unsigned q[2][2];
            asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                         : "=r"(q[0][0]), "=r"(q[0][1]) : "r"(base));
#pragma unroll
            for (int j = 1; j <= 16; ++j) {
                asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                             : "=r"(q[j & 1][0]), "=r"(q[j & 1][1]) : "r"(base + 16 * j));
                mma_bf16(acc[j - 1], q[(j - 1) & 1][0], q[(j - 1) & 1][1], q[j & 1][0], q[j & 1][1],
                         bfr[di][0], bfr[di][1]);
            }
        } else {
            const int m = lane >> 3;
            const int row = r0 + di + (lane & 7) + 8 * (m & 1);
            const unsigned base = (unsigned)__cvta_generic_to_shared(
                static_cast<const unsigned*>(stile) + row * kTcPitchF32 + 4 * (m >> 1));
            unsigned a[2][4];
            asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                         : "=r"(a[0][0]), "=r"(a[0][1]), "=r"(a[0][2]), "=r"(a[0][3]) : "r"(base));
#pragma unroll
            for (int j = 0; j <= 16; ++j) {
                if (j < 16) {
                    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                                 : "=r"(a[(j + 1) & 1][0]), "=r"(a[(j + 1) & 1][1]), "=r"(a[(j + 1) & 1][2]),
                                   "=r"(a[(j + 1) & 1][3])
                                 : "r"(base + 32 * (j + 1)));
                }
                if (j < 16) mma_tf32(acc[j], a[j & 1], bfr[di][0], bfr[di][1]);     // K rows 0..7 of tile j
                if (j > 0) mma_tf32(acc[j - 1], a[j & 1], bfr[di][2], bfr[di][3]);  // K rows 8..15 of tile j-1
            }
        }
    }
}

// 3xTF32: as the TF32 branch of tile_mma, on unrounded FP32 staging.  An MMA
// adds into its accumulator with truncation, which biases a running sum, so
// every hi*hi MMA (8 products) starts from a zero accumulator and is added to
// the running sum with a round-to-nearest FP32 add; the two small correction
// products of a (tile, di), ~2^-11 of the result, share one accumulator.
__device__ __forceinline__ void tile_mma_split(const void* stile, int warp, int lane, const unsigned (&bhi)[7][4],
                                               const unsigned (&blo)[7][4], float (&acc)[16][4]) {
    const int r0 = 16 * warp;
#pragma unroll
    for (int di = 0; di < 7; ++di) {
        const int m = lane >> 3;
        const int row = r0 + di + (lane & 7) + 8 * (m & 1);
        const unsigned base = (unsigned)__cvta_generic_to_shared(
            static_cast<const unsigned*>(stile) + row * kTcPitchF32 + 4 * (m >> 1));
        float small[2][4];  // tile j's correction terms live in small[j & 1] for two steps
        unsigned raw[2][4];
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(raw[0][0]), "=r"(raw[0][1]), "=r"(raw[0][2]), "=r"(raw[0][3]) : "r"(base));
#pragma unroll
        for (int j = 0; j <= 16; ++j) {
            if (j < 16) {
                asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                             : "=r"(raw[(j + 1) & 1][0]), "=r"(raw[(j + 1) & 1][1]), "=r"(raw[(j + 1) & 1][2]),
                               "=r"(raw[(j + 1) & 1][3])
                             : "r"(base + 32 * (j + 1)));
            }
            unsigned hi[4], lo[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float x = __uint_as_float(raw[j & 1][i]);
                hi[i] = f32_to_tf32(x);
                lo[i] = f32_to_tf32(x - __uint_as_float(hi[i]));
            }
            if (j < 16) {  // K rows 0..7 of tile j
                float (&sj)[4] = small[j & 1];
                sj[0] = sj[1] = sj[2] = sj[3] = 0.f;
                mma_tf32(sj, lo, bhi[di][0], bhi[di][1]);
                mma_tf32(sj, hi, blo[di][0], blo[di][1]);
                float big[4] = {0.f, 0.f, 0.f, 0.f};
                mma_tf32(big, hi, bhi[di][0], bhi[di][1]);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[j][i] = __fadd_rn(acc[j][i], big[i]);
            }
            if (j > 0) {  // K rows 8..15 of tile j-1, which completes its row-di terms
                float (&sk)[4] = small[(j - 1) & 1];
                mma_tf32(sk, lo, bhi[di][2], bhi[di][3]);
                mma_tf32(sk, hi, blo[di][2], blo[di][3]);
                float big[4] = {0.f, 0.f, 0.f, 0.f};
                mma_tf32(big, hi, bhi[di][2], bhi[di][3]);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[j - 1][i] = __fadd_rn(__fadd_rn(acc[j - 1][i], big[i]), sk[i]);
            }
        }
    }
}

// C fragment rows g, g+8; columns 2t, 2t+1 of each of the 16 column tiles.
template <typename TS>
__device__ __forceinline__ void store_tile(const TcParams& p, float (&acc)[16][4], int x0, int y0, int r0,
                                           int g, int t, bool round_tf32) {
    TS* out = static_cast<TS*>(p.out);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int x = x0 + 8 * j + 2 * t;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int y = y0 + r0 + g + 8 * h;
            if (y >= p.ny) continue;
            float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
            if (round_tf32) {
                v0 = __uint_as_float(f32_to_tf32(v0));
                v1 = __uint_as_float(f32_to_tf32(v1));
            }
            TS* o = out + (size_t)y * p.ld + x;
            if (x + 1 < p.nx) {
                if constexpr (sizeof(TS) == 4) {
                    if (p.vec) {
                        *reinterpret_cast<float2*>(o) = make_float2(v0, v1);
                        continue;
                    }
                } else {
                    if (p.vec) {
                        *reinterpret_cast<__nv_bfloat162*>(o) = __floats2bfloat162_rn(v0, v1);
                        continue;
                    }
                }
                Storage<TS>::store1(o, v0);
                Storage<TS>::store1(o + 1, v1);
            } else if (x < p.nx) {
                Storage<TS>::store1(o, v0);
            }
        }
    }
}

// ---- one tile per CTA, conversion while staging (any layout) ----------------------

template <typename TS, bool BF16MMA, bool SPLIT = false>
__global__ void __launch_bounds__(256) box49_tc_kernel(const __grid_constant__ TcParams p) {
    static_assert(!SPLIT || (!BF16MMA && sizeof(TS) == 4), "3xTF32 takes FP32 storage");
    extern __shared__ float4 smem_f4[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int x0 = (blockIdx.x % p.tiles_x) * kTcCols;
    const int y0 = (blockIdx.x / p.tiles_x) * kTcRows;

    // Every thread first issues all of its loads (so their DRAM latencies
    // overlap), then converts and stores.  Item i = tid + 256*it covers staged
    // row i / 34, 4-column group i % 34, advanced without division.
    unsigned* s32 = reinterpret_cast<unsigned*>(smem_f4);
    __nv_bfloat16* s16 = reinterpret_cast<__nv_bfloat16*>(smem_f4);
    constexpr int ITERS = (kTcSR * kTcQPR + 255) / 256;
    const TS* gin = static_cast<const TS*>(p.in);
    int r = tid / kTcQPR, q = tid % kTcQPR;
#pragma unroll 2
    for (int it0 = 0; it0 < ITERS; it0 += 6) {
        float v[6][4];
        int rr[6], qq[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            rr[u] = r;
            qq[u] = q;
            const int y = y0 - 3 + r, x = x0 - 4 + 4 * q;
            if ((it0 + u) < ITERS && r < kTcSR) {
                const bool inside = y >= 0 && y < p.ny && x >= 0 && x + 4 <= p.nx;
                if (p.vec && inside) {
                    float4 f = Storage<TS>::load4(gin + (size_t)y * p.ld + x);
                    v[u][0] = f.x; v[u][1] = f.y; v[u][2] = f.z; v[u][3] = f.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) v[u][e] = load_elem<TS>(p, y, x + e);
                }
            }
            q += 256 % kTcQPR;
            r += 256 / kTcQPR;
            if (q >= kTcQPR) {
                q -= kTcQPR;
                ++r;
            }
        }
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            if ((it0 + u) >= ITERS || rr[u] >= kTcSR) continue;
            if constexpr (BF16MMA) {
                __nv_bfloat162 a = __floats2bfloat162_rn(v[u][0], v[u][1]);
                __nv_bfloat162 b = __floats2bfloat162_rn(v[u][2], v[u][3]);
                uint2 raw;
                raw.x = *reinterpret_cast<unsigned*>(&a);
                raw.y = *reinterpret_cast<unsigned*>(&b);
                *reinterpret_cast<uint2*>(s16 + rr[u] * kTcPitchB16 + 4 * qq[u]) = raw;
            } else if constexpr (SPLIT) {  // unrounded: the MMA loop splits hi / lo
                *reinterpret_cast<float4*>(s32 + rr[u] * kTcPitchF32 + 4 * qq[u]) =
                    make_float4(v[u][0], v[u][1], v[u][2], v[u][3]);
            } else {
                *reinterpret_cast<uint4*>(s32 + rr[u] * kTcPitchF32 + 4 * qq[u]) =
                    make_uint4(f32_to_tf32(v[u][0]), f32_to_tf32(v[u][1]), f32_to_tf32(v[u][2]),
                               f32_to_tf32(v[u][3]));
            }
        }
    }
    float acc[16][4];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    if constexpr (SPLIT) {
        unsigned bhi[7][4], blo[7][4];
        make_bfrag_split(p, g, t, bhi, blo);
        __syncthreads();
        tile_mma_split(s32, warp, lane, bhi, blo, acc);
        store_tile<TS>(p, acc, x0, y0, 16 * warp, g, t, false);
    } else {
        unsigned bfr[7][4];
        make_bfrag<BF16MMA>(p, g, t, bfr);
        __syncthreads();
        tile_mma<BF16MMA>(BF16MMA ? (const void*)s16 : (const void*)s32, warp, lane, bfr, acc);
        // FP32 storage, TF32 engine: intermediate states stay TF32-rounded, as
        // the pipelined and tcgen05 engines expect (rounding at load is idempotent).
        store_tile<TS>(p, acc, x0, y0, 16 * warp, g, t, !BF16MMA && sizeof(TS) == 4 && p.round_out);
    }
}

// ---- persistent, double-buffered (16-byte aligned rows) ---------------------------

template <typename TS, bool BF16MMA, bool SPLIT = false>
__global__ void __launch_bounds__(256) box49_tc_pipe_kernel(const __grid_constant__ TcParams p) {
    static_assert(sizeof(TS) == (BF16MMA ? 2 : 4), "pipelined engine needs matching storage");
    static_assert(!SPLIT || !BF16MMA, "3xTF32 splits FP32 operands");
    constexpr int CB = 4 * (int)sizeof(TS);  // bytes per 4-element group
    constexpr int PITCH_B = BF16MMA ? kTcPitchB16 * 2 : kTcPitchF32 * 4;
    constexpr int STAGE_B = kTcSR * PITCH_B;
    extern __shared__ float4 smem_f4[];
    char* smem = reinterpret_cast<char*>(smem_f4);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const TS* gin = static_cast<const TS*>(p.in);

    // B fragments: one set, or hi / lo for 3xTF32 (the unused set stays empty).
    unsigned bfr[7][4], blo[SPLIT ? 7 : 1][4];
    if constexpr (SPLIT) {
        make_bfrag_split(p, g, t, bfr, blo);
    } else {
        make_bfrag<BF16MMA>(p, g, t, bfr);
    }

    // Copy tile `tile`'s groups into stage `st`; out-of-grid groups are zero-filled.
    auto issue = [&](int tile, int st) {
        const int x0 = (tile % p.tiles_x) * kTcCols, y0 = (tile / p.tiles_x) * kTcRows;
        char* base = smem + st * STAGE_B;
        int r = tid / kTcQPR, q = tid % kTcQPR;
        for (int i = tid; i < kTcSR * kTcQPR; i += 256) {
            int y = y0 - 3 + r, x = x0 - 4 + 4 * q;
            bool ok;
            if (p.periodic) {
                y = (y % p.ny + p.ny) % p.ny;
                x = (x % p.nx + p.nx) % p.nx;
                ok = true;
            } else {
                ok = y >= 0 && y < p.ny && x >= 0 && x + 4 <= p.nx;
            }
            const TS* src = ok ? gin + (size_t)y * p.ld + x : gin;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(base + r * PITCH_B + q * CB);
            if constexpr (CB == 16) {
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                             "r"(ok ? 16 : 0));
            } else {
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src),
                             "r"(ok ? 8 : 0));
            }
            q += 256 % kTcQPR;
            r += 256 / kTcQPR;
            if (q >= kTcQPR) {
                q -= kTcQPR;
                ++r;
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };

    int st = 0;
    int tile = blockIdx.x;
    if (tile < p.tiles) issue(tile, 0);
    for (; tile < p.tiles; tile += gridDim.x, st ^= 1) {
        const int next = tile + gridDim.x;
        if (next < p.tiles) {
            issue(next, st ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        __syncthreads();
        char* stage = smem + st * STAGE_B;
        if constexpr (!BF16MMA && !SPLIT) {
            if (p.convert_in) {  // the caller's FP32 input: round to TF32 in place
                for (int i = tid; i < kTcSR * kTcQPR; i += 256) {
                    const int rr = i / kTcQPR, qq = i % kTcQPR;
                    uint4* w = reinterpret_cast<uint4*>(stage + rr * PITCH_B + qq * 16);
                    uint4 u = *w;
                    *w = make_uint4(f32_to_tf32(__uint_as_float(u.x)), f32_to_tf32(__uint_as_float(u.y)),
                                    f32_to_tf32(__uint_as_float(u.z)), f32_to_tf32(__uint_as_float(u.w)));
                }
                __syncthreads();
            }
        }
        float acc[16][4];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        if constexpr (SPLIT) {
            tile_mma_split(stage, warp, lane, bfr, blo, acc);
        } else {
            tile_mma<BF16MMA>(stage, warp, lane, bfr, acc);
        }
        const int x0 = (tile % p.tiles_x) * kTcCols, y0 = (tile / p.tiles_x) * kTcRows;
        store_tile<TS>(p, acc, x0, y0, 16 * warp, g, t, !BF16MMA && !SPLIT && p.round_out);
        __syncthreads();  // every warp is done with `stage` before it is refilled
    }
}

// engine: 0 = TF32, 1 = BF16, 2 = 3xTF32 (FP32 storage only).
const void* get_box49_tc_kernel(int dtype, int engine) {
    if (engine == 2) return dtype == DT_F32 ? (const void*)box49_tc_kernel<float, false, true> : nullptr;
    const bool bf16mma = engine == 1;
    if (dtype == DT_F32) return bf16mma ? (const void*)box49_tc_kernel<float, true>
                                        : (const void*)box49_tc_kernel<float, false>;
    if (dtype == DT_BF16) return bf16mma ? (const void*)box49_tc_kernel<__nv_bfloat16, true>
                                         : (const void*)box49_tc_kernel<__nv_bfloat16, false>;
    return nullptr;
}

// The pipelined kernel for the matching storage/engine pairs, else nullptr.
const void* get_box49_tc_pipe_kernel(int dtype, int engine) {
    if (dtype == DT_F32 && engine == 0) return (const void*)box49_tc_pipe_kernel<float, false>;
    if (dtype == DT_F32 && engine == 2) return (const void*)box49_tc_pipe_kernel<float, false, true>;
    if (dtype == DT_BF16 && engine == 1) return (const void*)box49_tc_pipe_kernel<__nv_bfloat16, true>;
    return nullptr;
}

int box49_tc_smem_bytes(int engine) {
    return engine == 1 ? kTcSR * kTcPitchB16 * 2 : kTcSR * kTcPitchF32 * 4;
}

}  // namespace gbst
