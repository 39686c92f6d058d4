// box49_umma.cu -- the 7x7 box stencil on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory, operands staged by TMA).
//
// The contraction is the one of box49_tc.cu (a stencil step as a matrix
// product, Sec. II-D; the weights of row di form a banded Toeplitz matrix):
//   out[y0 + r][x0 + NT*j + n] = sum_di sum_k A_dij[r][k] * B_di[k][n]
//   A_dij[r][k] = in[y0 + r + di - 3][x0 + NT*j - L + k]
//   B_di[k][n]  = W[di][k - n - (L - 3)]   (0 <= k - n - (L - 3) <= 6, else 0)
// per MMA tile of M = 128 rows and N = NT columns (NT = 16, 32 or 64).  L = 8
// for BF16 operands and 4 for TF32, so every staged column group starts on a
// 16-byte boundary.  K = NT + L + 3 rounded up to the instruction's K step
// (16 for kind::f16, 8 for kind::tf32); 7 of every K products are non-zero.
//
// A staged tile covers 134 rows and the columns x0 - L .. x0 - L + 128 + KE - 1
// in two kinds of K-major operand storage, both filled by 2D TMA boxes with
// zero fill outside the grid (the zero boundary of Sec. IV-A; periodic grids
// use the warp-MMA engine):
//   * 128 columns as 128-byte swizzled atoms (SWIZZLE_128B): one box of
//     128 B x 134 rows per atom, rows 128 B apart, 8-row groups 1024 B apart
//     (SBO), atoms 17 KB apart.  Wide boxes keep the TMA request count low.
//   * the last KE columns as two no-swizzle "planes" of 16 B x 134 rows (rows
//     16 B apart, SBO = 128 B, plane pitch = LBO).
// Every K slice of an instruction starts at a column c that is a multiple of
// KE and lies in one atom (c < 128) or is the plane pair (c = 128).  The row
// shift di is only a descriptor start address: +128 * di bytes in an atom
// or +16 * di bytes in a plane; no data is copied per di.  A tiled
// TMA destination is 1024-byte (swizzled) or 128-byte (plain) aligned: stages
// start on 1024-byte boundaries and the producer checks every destination
// before it issues a copy.
//
// Persistent CTA (one per SM), six warps:
//   warp 0       TMA producer, STAGES-deep ring of staged tiles;
//   warp 1       TMEM allocation and the single-thread MMA issue;
//   warps 2..5   epilogue: tcgen05.ld of the lane quarter warp % 4 (all 128
//                columns, one wait), release of the accumulator, conversion
//                into a 128-byte swizzled staging tile, and one TMA tensor
//                store per 128-byte column atom (clipped at the grid edges).
// Two accumulators of 128 TMEM columns let the epilogue of one tile overlap
// the MMAs of the next; two staging buffers (one where shared memory is
// short) let the TMA store of one tile overlap the epilogue of the next.
// Measured on GB300 (16384^2): the MMAs then cost ~65 cycles each whatever
// their N, i.e. the A operand streams from shared memory at ~64 B per cycle,
// so the widest N that fits (fewest re-reads of the row-shifted A) is the
// fastest: BF16 N = 64 916 GStencil/s, TF32 N = 32 492 (its output tile is
// staged in two column halves to fit).  mbarriers: full / empty per stage, tmem_full /
// tmem_empty per accumulator, one drain barrier.  Every wait is bounded
// (%globaltimer, 2 s by default, and an iteration cap): when one expires the kernel
// stores STENCIL_ERR_TIMEOUT in the status word, raises a CTA-wide abort flag,
// waits (again bounded) for its own TMA loads and MMAs in flight, frees its
// tensor memory and returns.
//
// TF32 engine: kind::tf32 reads the upper 19 bits of each FP32 word, so the
// state it reads must already be TF32-rounded.  The plan keeps it so: the
// first launch of a run (warp-MMA engine) rounds the caller's input, and every
// launch but the last rounds its output (round_out).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/stencil.h"

namespace gbst {

constexpr int kUmRows = 128;            // M: output rows per tile
constexpr int kUmCols = 128;            // output columns per tile
constexpr int kUmSR = kUmRows + 6;      // staged rows y0-3 .. y0+130
constexpr int kUmPlane = 2176;          // plane pitch: 134 rows x 16 B, padded to 128 B
constexpr int kUmAtom = 17408;          // swizzled atom pitch: 134 rows x 128 B, padded to 1 KB
constexpr int kUmThreads = 192;         // 6 warps
constexpr int kUmTmemCols = 256;        // 2 accumulators x 128 FP32 columns

template <bool TF32, int NT>
struct UmCfg {
    static constexpr int EB = TF32 ? 4 : 2;                      // bytes per element
    static constexpr int EPG = 16 / EB;                          // elements per plane row
    static constexpr int L = TF32 ? 4 : 8;                       // K window starts L columns left
    static constexpr int KE = TF32 ? 8 : 16;                     // K of one instruction
    static constexpr int KSTEPS = (NT + L + 3 + KE - 1) / KE;    // instructions per (j, di)
    static constexpr int PPI = KE / EPG;                         // planes per instruction (2)
    static constexpr int PPN = NT / EPG;                         // planes per N-tile step
    static constexpr int JT = kUmCols / NT;                      // N-tiles per tile
    static constexpr int AE = 128 / EB;                          // elements per swizzled atom row
    static constexpr int NA = kUmCols / AE;                      // swizzled atoms (128 columns)
    static constexpr int STAGES = TF32 ? 2 : 3;
    static constexpr int STAGE_BYTES = (NA * kUmAtom + PPI * kUmPlane + 1023) / 1024 * 1024;
    static constexpr int TX_BYTES = NA * kUmSR * 128 + PPI * kUmSR * 16;  // bytes the boxes deliver
    static constexpr int BPLANES = KSTEPS * PPI;                 // K planes of one B_di
    static constexpr int BPLANE = NT * 16;                       // bytes per B plane
    static constexpr int B_BYTES = BPLANES * BPLANE;
    static constexpr int NBARS = 2 * STAGES + 5;
    static constexpr int OUT_BYTES = kUmRows * kUmCols * EB;     // one output tile
    static constexpr int BASE = STAGES * STAGE_BYTES + 7 * B_BYTES + 8 * NBARS;
    // The output tile is staged whole, or in two column halves where shared
    // memory is short; two staging buffers where they fit.
    static constexpr int PARTS = 1024 + BASE + OUT_BYTES <= 227 * 1024 ? 1 : 2;
    static constexpr int PART_BYTES = OUT_BYTES / PARTS;
    static constexpr int STG = 1024 + BASE + 2 * PART_BYTES <= 227 * 1024 ? 2 : 1;
    static constexpr int SMEM = 1024 + BASE + STG * PART_BYTES;  // + alignment slack
    static_assert(kUmCols % NT == 0 && NT % 16 == 0, "N-tile width");
    static_assert(kUmCols + KE >= kUmCols + L + 3, "staged columns cover the footprint");
    static_assert((JT - 1) * NT + (KSTEPS - 1) * KE <= kUmCols, "K slices end in the plane pair");
    static_assert(AE % KE == 0 && PPI == 2, "K slices do not straddle atoms");
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
    static_assert(STAGE_BYTES % 1024 == 0 && PART_BYTES % 1024 == 0 && B_BYTES % 16 == 0,
                  "TMA and descriptor alignment");
};
static_assert(kUmPlane % 128 == 0 && kUmPlane >= kUmSR * 16, "plane pitch");
static_assert(kUmAtom % 1024 == 0 && kUmAtom >= kUmSR * 128, "atom pitch");

struct UmParams {
    void* out;
    int ny, nx, ld;
    int tiles_x, tiles;
    int round_out;      // TF32: store TF32-rounded values
    unsigned* status;   // STENCIL_ERR_TIMEOUT on an expired wait
    long long wait_ns;  // limit of each mbarrier wait
    int withhold;       // test hook: CTA 0 withholds its first accumulator-ready signal
    float w[49];
};

// ---- PTX helpers ------------------------------------------------------------------------

__device__ __forceinline__ unsigned um_smem(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ long long um_now() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void um_bar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void um_bar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void um_bar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool um_bar_try(unsigned bar, unsigned parity) {
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

constexpr unsigned kUmWaitIters = 1u << 26;

// Wait for the phase of `parity` of `bar`.  Gives up when the CTA's abort flag
// is raised, or after `limit_ns` (then records a timeout and raises the flag).
__device__ __forceinline__ bool um_wait(unsigned bar, unsigned parity, volatile int* abort_flag,
                                        unsigned* status, long long limit_ns) {
    const long long t0 = um_now();
    for (unsigned it = 0;; ++it) {
        if (um_bar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((it & 63u) == 63u && (um_now() - t0 > limit_ns || it > kUmWaitIters)) {
            atomicCAS(status, 0u, (unsigned)STENCIL_ERR_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
    }
}

// Bounded wait used while winding down (ignores the abort flag).
__device__ __forceinline__ void um_drain(unsigned bar, unsigned parity, unsigned* status, long long limit_ns) {
    const long long t0 = um_now();
    for (unsigned it = 0;; ++it) {
        if (um_bar_try(bar, parity)) return;
        if ((it & 63u) == 63u && (um_now() - t0 > limit_ns || it > kUmWaitIters)) {
            atomicCAS(status, 0u, (unsigned)STENCIL_ERR_TIMEOUT);
            return;
        }
    }
}

__device__ __forceinline__ void um_tma_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor, K-major: start, LBO and SBO in 16-byte
// units; bits 46..48 hold the fixed value 0b001; no swizzle (layout 0).
__device__ __forceinline__ unsigned long long um_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((saddr >> 4) & 0x3FFFu) |
           ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// The same for the 128-byte swizzle (layout type 2 in bits 61..63): SBO =
// 1024 B between 8-row groups, LBO unused within an atom (set to 16 B).  The
// tensor cores take the swizzle phase from the address bits, as the TMA unit
// does when it writes a 1024-byte aligned atom, so a start address moved by
// whole 128-byte rows (the row shift di) or by 32-byte K steps inside a row
// keeps base offset 0 (bits 49..51); the dyadic-exact tests fail with the
// start address's phase (start >> 7) & 7 in that field instead.
__device__ __forceinline__ unsigned long long um_desc_sw128(unsigned saddr) {
    return um_desc(saddr, 16, 1024) | (2ull << 61);
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A/B format in bits
// 7-9 / 10-12 (BF16 = 1 under kind::f16, TF32 = 2 under kind::tf32), both
// operands K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <bool TF32, int NT>
__device__ __forceinline__ unsigned um_idesc() {
    constexpr unsigned ab = TF32 ? 2u : 1u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((unsigned)(NT >> 3) << 17) | ((unsigned)(kUmRows >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void um_mma(unsigned tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                       unsigned idesc, unsigned accumulate) {
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

// Arrive on `bar` once every tcgen05 operation this thread issued so far is done.
__device__ __forceinline__ void um_commit(unsigned bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane (no wait).
__device__ __forceinline__ void um_ld32(unsigned taddr, unsigned* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void um_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Named barrier 1 over the NTH epilogue threads; returns the AND of `pred`.
template <int NTH = 128>
__device__ __forceinline__ int um_epi_and(int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(pred), "n"(NTH)
        : "memory");
    return r;
}

template <int NTH = 128>
__device__ __forceinline__ void um_epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NTH) : "memory"); }

__device__ __forceinline__ void um_tma_store_2d(const CUtensorMap* map, unsigned src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}

__device__ __forceinline__ void um_st_shared_v4(unsigned addr, unsigned a, unsigned b, unsigned c, unsigned d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

__device__ __forceinline__ unsigned um_tf32(float x) {
    unsigned r;
    asm("cvt.rn.satfinite.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void um_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void um_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- the kernel ---------------------------------------------------------------------------

template <bool TF32, int NT>
__global__ void __launch_bounds__(kUmThreads, 1)
    box49_umma_kernel(const __grid_constant__ CUtensorMap tmap_sw, const __grid_constant__ CUtensorMap tmap_pl,
                      const __grid_constant__ CUtensorMap tmap_out, const __grid_constant__ UmParams p) {
    using C = UmCfg<TF32, NT>;
    extern __shared__ __align__(1024) unsigned char um_dyn[];
    // staging area on a 1024-byte boundary (SMEM includes the slack)
    unsigned char* stages = um_dyn + ((1024u - (um_smem(um_dyn) & 1023u)) & 1023u);
    unsigned char* outstg = stages + C::STAGES * C::STAGE_BYTES;  // output staging, 1024-byte aligned
    unsigned char* bmat = outstg + C::STG * C::PART_BYTES;
    __shared__ unsigned s_tmem;
    __shared__ volatile int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // barriers: full[S], empty[S], tmem_full[2], tmem_empty[2], drain
    const unsigned bar0 = um_smem(bmat + 7 * C::B_BYTES);
    const unsigned full0 = bar0, empty0 = bar0 + 8u * C::STAGES, tfull0 = bar0 + 16u * C::STAGES,
                   tempty0 = tfull0 + 16u, drain = tempty0 + 16u;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < C::STAGES; ++s) {
            um_bar_init(full0 + 8u * s, 1);
            um_bar_init(empty0 + 8u * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            um_bar_init(tfull0 + 8u * b, 1);
            um_bar_init(tempty0 + 8u * b, 4);
        }
        um_bar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B_di in the K-major no-swizzle layout: element (k, n) of B_di at byte
    // di * B_BYTES + (k / EPG) * BPLANE + 16 n + EB * (k % EPG).
    for (int i = threadIdx.x; i < 7 * C::BPLANES * NT * C::EPG; i += kUmThreads) {
        const int e = i % C::EPG;
        const int n = (i / C::EPG) % NT;
        const int pl = (i / (C::EPG * NT)) % C::BPLANES;
        const int di = i / (C::EPG * NT * C::BPLANES);
        const int dj = pl * C::EPG + e - n - (C::L - 3);
        const float v = (dj >= 0 && dj <= 6) ? p.w[di * 7 + dj] : 0.f;
        unsigned char* dst = bmat + di * C::B_BYTES + pl * C::BPLANE + n * 16 + e * C::EB;
        if constexpr (TF32) {
            *reinterpret_cast<unsigned*>(dst) = um_tf32(v);
        } else {
            *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B is read by the tensor cores
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(um_smem(&s_tmem)),
                     "r"(kUmTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    um_fence_before();
    __syncthreads();
    um_fence_after();
    const unsigned tmem = s_tmem;

    if (warp == 0) {
        // ---------------- TMA producer (lane 0 issues, the warp stays converged) ----------------
        int it = 0;
        for (int tile = blockIdx.x; tile < p.tiles; tile += gridDim.x, ++it) {
            const int s = it % C::STAGES;
            int ok = 1;
            if (lane == 0) ok = um_wait(empty0 + 8u * s, ((it / C::STAGES) & 1) ^ 1, &s_abort, p.status, p.wait_ns);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            if (lane == 0) {
                const int x0 = (tile % p.tiles_x) * kUmCols, y0 = (tile / p.tiles_x) * kUmRows;
                const unsigned fb = full0 + 8u * s;
                const unsigned dst = um_smem(stages + s * C::STAGE_BYTES);
                if ((dst & 1023u) != 0u || (fb & 7u) != 0u) {
                    // never issue a misaligned copy: report it and stop the CTA
                    atomicCAS(p.status, 0u, (unsigned)STENCIL_ERR_DEVICE_CHECK);
                    s_abort = 1;
                    ok = 0;
                } else {
                    um_bar_expect_tx(fb, (unsigned)C::TX_BYTES);
                    const int xs = x0 - C::L;
                    for (int a = 0; a < C::NA; ++a)
                        um_tma_2d(dst + (unsigned)(a * kUmAtom), &tmap_sw, xs + C::AE * a, y0 - 3, fb);
                    for (int g = 0; g < C::PPI; ++g)
                        um_tma_2d(dst + (unsigned)(C::NA * kUmAtom + g * kUmPlane), &tmap_pl,
                                  xs + kUmCols + C::EPG * g, y0 - 3, fb);
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
        }
        // Loads still in flight (only after an abort) land before the CTA exits.
        if (lane == 0) {
            for (int i = it - C::STAGES < 0 ? 0 : it - C::STAGES; i < it; ++i)
                um_drain(full0 + 8u * (i % C::STAGES), (i / C::STAGES) & 1, p.status, p.wait_ns);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issue (one thread) ----------------
        const unsigned idesc = um_idesc<TF32, NT>();
        const unsigned long long bdesc0 = um_desc(um_smem(bmat), C::BPLANE, 128);
        int it = 0, issued = 0;
        for (int tile = blockIdx.x; tile < p.tiles; tile += gridDim.x, ++it) {
            const int s = it % C::STAGES, b = it & 1;
            int ok = 1;
            if (lane == 0) {
                ok = um_wait(full0 + 8u * s, (it / C::STAGES) & 1, &s_abort, p.status, p.wait_ns) &&
                     um_wait(tempty0 + 8u * b, ((it >> 1) & 1) ^ 1, &s_abort, p.status, p.wait_ns);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            um_fence_after();
            if (lane == 0) {
                // Base descriptors of this stage; every MMA below adds a compile-time
                // byte offset / 16 to the start-address field (addresses < 256 KB).
                const unsigned sbase = um_smem(stages + s * C::STAGE_BYTES);
                const unsigned long long a_sw = um_desc_sw128(sbase);
                const unsigned long long a_pl = um_desc(sbase + (unsigned)(C::NA * kUmAtom), kUmPlane, 128);
#pragma unroll
                for (int j = 0; j < C::JT; ++j) {
                    const unsigned d = tmem + (unsigned)(b * 128 + NT * j);
#pragma unroll
                    for (int ks = 0; ks < C::KSTEPS; ++ks) {
                        const int c = NT * j + C::KE * ks;  // first column of the K slice (from x0 - L)
#pragma unroll
                        for (int di = 0; di < 7; ++di) {
                            const unsigned long long a =
                                c < kUmCols ? a_sw + (unsigned long long)(((c / C::AE) * kUmAtom + 128 * di +
                                                                           (c % C::AE) * C::EB) >> 4)
                                            : a_pl + (unsigned long long)((16 * di) >> 4);
                            const unsigned long long bd =
                                bdesc0 + (unsigned long long)((di * C::B_BYTES + ks * C::PPI * C::BPLANE) >> 4);
                            um_mma<TF32>(d, a, bd, idesc, (di | ks) != 0);
                        }
                    }
                }
                um_commit(empty0 + 8u * s);  // the stage is free once these MMAs have read it
                if (!(p.withhold && blockIdx.x == 0 && it == 0))
                    um_commit(tfull0 + 8u * b);  // the accumulator is complete
                issued = 1;
            }
            __syncwarp();
        }
        // Every MMA issued is complete before the tensor memory is released.
        if (lane == 0 && issued) {
            um_commit(drain);
            um_drain(drain, 0, p.status, p.wait_ns);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: TMEM lanes 32 q .. 32 q + 31 ----------------
        // Per tile: load the thread's 128 accumulators (one wait), free the
        // TMEM buffer, write the row into a 128-byte swizzled staging tile and
        // let one thread store the tile with TMA (clipped at the grid edges).
        const int q = warp & 3;
        const int r = 32 * q + lane;  // tile row = TMEM lane
        const bool issuer = threadIdx.x == 64;
        constexpr int AEO = 128 / C::EB;            // output columns per staged atom
        constexpr int NAO = kUmCols / AEO;          // staged atoms per tile
        int it = 0;
        for (int tile = blockIdx.x; tile < p.tiles; tile += gridDim.x, ++it) {
            const int b = it & 1;
            int ok = 1;
            if (lane == 0) ok = um_wait(tfull0 + 8u * b, (it >> 1) & 1, &s_abort, p.status, p.wait_ns);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!um_epi_and(ok)) break;  // the four epilogue warps leave together
            um_fence_after();
            unsigned v[kUmCols];
            const unsigned trow = tmem + ((unsigned)(32 * q) << 16) + (unsigned)(b * 128);
#pragma unroll
            for (int c = 0; c < kUmCols / 32; ++c) um_ld32(trow + (unsigned)(32 * c), v + 32 * c);
            um_ld_wait();
            um_fence_before();
            __syncwarp();
            if (lane == 0) um_bar_arrive(tempty0 + 8u * b);  // accumulator free for the MMAs
            const int x0 = (tile % p.tiles_x) * kUmCols, y0 = (tile / p.tiles_x) * kUmRows;
#pragma unroll
            for (int part = 0; part < C::PARTS; ++part) {
                constexpr int APP = NAO / C::PARTS;  // atoms per staged part
                const int sb = C::STG == 2 ? ((it * C::PARTS + part) & 1) : 0;
                // the store that last read this staging buffer has finished reading it
                if (issuer) {
                    if constexpr (C::STG == 2)
                        asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    else
                        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                }
                um_epi_sync();
                const unsigned stg = um_smem(outstg + sb * C::PART_BYTES);
#pragma unroll
                for (int a = 0; a < APP; ++a) {
                    const int A = part * APP + a;  // atom of the tile
#pragma unroll
                    for (int c = 0; c < 8; ++c) {  // 16-byte chunk c of this row in atom A
                        unsigned w[4];
                        if constexpr (TF32) {
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const unsigned u = v[A * 32 + c * 4 + i];
                                w[i] = p.round_out ? um_tf32(__uint_as_float(u)) : u;
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                __nv_bfloat162 h = __floats2bfloat162_rn(
                                    __uint_as_float(v[A * 64 + c * 8 + 2 * i]), __uint_as_float(v[A * 64 + c * 8 + 2 * i + 1]));
                                w[i] = *reinterpret_cast<unsigned*>(&h);
                            }
                        }
                        um_st_shared_v4(stg + (unsigned)(a * kUmRows * 128 + r * 128 + ((c ^ (r & 7)) << 4)), w[0],
                                        w[1], w[2], w[3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // staging is read by TMA
                um_epi_sync();
                if (issuer) {
#pragma unroll
                    for (int a = 0; a < APP; ++a)
                        um_tma_store_2d(&tmap_out, stg + (unsigned)(a * kUmRows * 128), x0 + (part * APP + a) * AEO, y0);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
            }
        }
        // every store has completed (and read its staging) before the CTA exits
        if (issuer) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    }

    um_fence_before();
    __syncthreads();
    um_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUmTmemCols)
                     : "memory");
    }
}

// ---- row-grouped variant ------------------------------------------------------------------
//
// The kernel above reads its A operand (128 rows x one K slice, 4 KB) from
// shared memory once per (N-tile, K step, weight row), and that read, not
// the arithmetic, sets the cost of an MMA.  Here D weight rows share one
// read: the B operand stacks the Toeplitz bands of rows s .. s+D-1 side by
// side (N = D * NT columns) and A is the staged tile shifted by s rows.
// Column block d of the accumulator then holds, in TMEM lane r, what staged
// row r + s contributes through weight row s + d, which belongs to output
// row r - d.  So
//   out[r] = sum_d acc_d[r + d],   r = 0 .. 128 - D,
// a tile has 129 - D output rows, and the epilogue adds the D blocks with
// lane shifts: warp shuffles inside a lane quarter; the last d lanes of a
// quarter take the first d lanes of the next one through shared memory.
// The rows form groups {0..D-1}, {D..2D-1}, ..; the last group may hold
// fewer rows (a narrower MMA that adds into the leading blocks).  Each
// accumulator holds one N-tile (D * NT columns), up to four in flight.
// Measured on GB300 (16384^2, 200 steps): TF32 N = 96 (D = 3) 547 GStencil/s
// against 492 for one row per MMA; BF16 N = 96 784 and N = 128 596 against
// 916.  With the epilogue's shuffles and exchange taken out (a timing copy)
// BF16 reaches only ~940 (D = 3) and ~1130 (D = 4): the wider MMAs cost more
// than the A reads they save, and the D - 1 shuffles per output halve the
// rest.  Eight epilogue warps instead of four, and adding the in-quarter
// terms before the exchange barrier, were both slower.
template <bool TF32, int NT, int D>
struct UmgCfg {
    static constexpr int EB = TF32 ? 4 : 2;
    static constexpr int EPG = 16 / EB;
    static constexpr int L = TF32 ? 4 : 8;
    static constexpr int KE = TF32 ? 8 : 16;
    static constexpr int KSTEPS = (NT + L + 3 + KE - 1) / KE;
    static constexpr int PPI = KE / EPG;
    static constexpr int JT = kUmCols / NT;
    static constexpr int AE = 128 / EB;
    static constexpr int NA = kUmCols / AE;
    static constexpr int NG = (7 + D - 1) / D;                   // row groups
    static constexpr int OUT = kUmRows + 1 - D;                   // output rows per tile
    static constexpr int BUFN = D * NT;                           // TMEM columns of one N-tile
    static constexpr int NBUF = 512 / BUFN < 4 ? 512 / BUFN : 4;  // accumulators in flight
    static constexpr int STAGES = TF32 ? 2 : 3;
    static constexpr int STAGE_BYTES = (NA * kUmAtom + PPI * kUmPlane + 1023) / 1024 * 1024;
    static constexpr int TX_BYTES = NA * kUmSR * 128 + PPI * kUmSR * 16;
    static constexpr int ROW_BYTES = KSTEPS * PPI * NT * 16;      // B bytes per weight row
    static constexpr int B_BYTES = 7 * ROW_BYTES;
    static constexpr int XQ = (D - 1) * (D - 1) * 32;             // exchange floats per lane quarter
    static constexpr int XCH_BYTES = 2 * 4 * XQ * 4;              // two parities x four quarters
    static constexpr int NBARS = 2 * STAGES + 2 * NBUF + 1;
    static constexpr int OUT_BYTES = kUmRows * kUmCols * EB;
    static constexpr int BASE = STAGES * STAGE_BYTES + B_BYTES + XCH_BYTES + 8 * NBARS;
    static constexpr int LIMIT = 227 * 1024 - 1024;               // dynamic bytes next to the static ones
    static constexpr int PARTS = 1024 + BASE + OUT_BYTES <= LIMIT ? 1 : 2;
    static constexpr int PART_BYTES = OUT_BYTES / PARTS;
    static constexpr int STG = 1024 + BASE + 2 * PART_BYTES <= LIMIT ? 2 : 1;
    static constexpr int SMEM = 1024 + BASE + STG * PART_BYTES;
    static __host__ __device__ constexpr int rows(int g) { return 7 - g * D < D ? 7 - g * D : D; }
    static_assert(D >= 2 && D <= 7 && NT % 32 == 0 && BUFN <= 256 && NBUF >= 2, "group shape");
    static_assert((JT - 1) * NT + (KSTEPS - 1) * KE <= kUmCols, "K slices end in the plane pair");
    static_assert(AE % KE == 0 && PPI == 2, "K slices do not straddle atoms");
    static_assert(kUmCols % (kUmCols / PARTS) == 0 && (kUmCols / PARTS) % NT == 0, "parts hold whole N-tiles");
    static_assert(SMEM <= LIMIT, "shared memory per CTA");
    static_assert(STAGE_BYTES % 1024 == 0 && PART_BYTES % 1024 == 0 && ROW_BYTES % 16 == 0 &&
                      (STAGES * STAGE_BYTES + STG * PART_BYTES + B_BYTES) % 16 == 0,
                  "TMA and descriptor alignment");
};

template <bool TF32>
__device__ __forceinline__ unsigned um_idesc_n(int n) {
    constexpr unsigned ab = TF32 ? 2u : 1u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(kUmRows >> 4) << 24);
}

template <bool TF32, int NT, int D>
__global__ void __launch_bounds__(kUmThreads, 1)
    box49_umma_rows_kernel(const __grid_constant__ CUtensorMap tmap_sw, const __grid_constant__ CUtensorMap tmap_pl,
                           const __grid_constant__ CUtensorMap tmap_out, const __grid_constant__ UmParams p) {
    using C = UmgCfg<TF32, NT, D>;
    extern __shared__ __align__(1024) unsigned char um_dyn[];
    unsigned char* stages = um_dyn + ((1024u - (um_smem(um_dyn) & 1023u)) & 1023u);
    unsigned char* outstg = stages + C::STAGES * C::STAGE_BYTES;
    unsigned char* bmat = outstg + C::STG * C::PART_BYTES;
    float* xch = reinterpret_cast<float*>(bmat + C::B_BYTES);
    __shared__ unsigned s_tmem;
    __shared__ volatile int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // barriers: full[S], empty[S], tmem_full[NBUF], tmem_empty[NBUF], drain
    const unsigned bar0 = um_smem(bmat + C::B_BYTES + C::XCH_BYTES);
    const unsigned full0 = bar0, empty0 = bar0 + 8u * C::STAGES, tfull0 = bar0 + 16u * C::STAGES,
                   tempty0 = tfull0 + 8u * C::NBUF, drain = tempty0 + 8u * C::NBUF;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < C::STAGES; ++s) {
            um_bar_init(full0 + 8u * s, 1);
            um_bar_init(empty0 + 8u * s, 1);
        }
        for (int b = 0; b < C::NBUF; ++b) {
            um_bar_init(tfull0 + 8u * b, 1);
            um_bar_init(tempty0 + 8u * b, 4);
        }
        um_bar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B of row group g (rows g*D .. g*D + rows(g) - 1) starts at byte
    // g * D * ROW_BYTES; K-major, no swizzle, plane pitch rows(g) * NT * 16:
    // element (k, n) at (k / EPG) * pitch + 16 n + EB * (k % EPG), where
    // n = d * NT + n' holds W[g*D + d][k - n' - (L - 3)] (0 outside the band).
    for (int i = threadIdx.x; i < 7 * C::KSTEPS * C::PPI * NT * C::EPG; i += kUmThreads) {
        const int e = i % C::EPG;
        const int n1 = (i / C::EPG) % NT;
        const int pl = (i / (C::EPG * NT)) % (C::KSTEPS * C::PPI);
        const int di = i / (C::EPG * NT * C::KSTEPS * C::PPI);
        const int g = di / D, d = di % D;
        const int dj = pl * C::EPG + e - n1 - (C::L - 3);
        const float v = (dj >= 0 && dj <= 6) ? p.w[di * 7 + dj] : 0.f;
        unsigned char* dst = bmat + g * D * C::ROW_BYTES + pl * (C::rows(g) * NT * 16) + (d * NT + n1) * 16 + e * C::EB;
        if constexpr (TF32) {
            *reinterpret_cast<unsigned*>(dst) = um_tf32(v);
        } else {
            *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(um_smem(&s_tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    um_fence_before();
    __syncthreads();
    um_fence_after();
    const unsigned tmem = s_tmem;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        int it = 0;
        for (int tile = blockIdx.x; tile < p.tiles; tile += gridDim.x, ++it) {
            const int s = it % C::STAGES;
            int ok = 1;
            if (lane == 0) ok = um_wait(empty0 + 8u * s, ((it / C::STAGES) & 1) ^ 1, &s_abort, p.status, p.wait_ns);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            if (lane == 0) {
                const int x0 = (tile % p.tiles_x) * kUmCols, y0 = (tile / p.tiles_x) * C::OUT;
                const unsigned fb = full0 + 8u * s;
                const unsigned dst = um_smem(stages + s * C::STAGE_BYTES);
                if ((dst & 1023u) != 0u || (fb & 7u) != 0u) {
                    atomicCAS(p.status, 0u, (unsigned)STENCIL_ERR_DEVICE_CHECK);
                    s_abort = 1;
                    ok = 0;
                } else {
                    um_bar_expect_tx(fb, (unsigned)C::TX_BYTES);
                    const int xs = x0 - C::L;
                    for (int a = 0; a < C::NA; ++a)
                        um_tma_2d(dst + (unsigned)(a * kUmAtom), &tmap_sw, xs + C::AE * a, y0 - 3, fb);
                    for (int g = 0; g < C::PPI; ++g)
                        um_tma_2d(dst + (unsigned)(C::NA * kUmAtom + g * kUmPlane), &tmap_pl,
                                  xs + kUmCols + C::EPG * g, y0 - 3, fb);
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
        }
        if (lane == 0) {
            for (int i = it - C::STAGES < 0 ? 0 : it - C::STAGES; i < it; ++i)
                um_drain(full0 + 8u * (i % C::STAGES), (i / C::STAGES) & 1, p.status, p.wait_ns);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issue (one thread) ----------------
        int it = 0, u = 0, issued = 0;
        bool alive = true;
        for (int tile = blockIdx.x; tile < p.tiles && alive; tile += gridDim.x, ++it) {
            const int s = it % C::STAGES;
            int ok = 1;
            if (lane == 0) ok = um_wait(full0 + 8u * s, (it / C::STAGES) & 1, &s_abort, p.status, p.wait_ns);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            const unsigned sbase = um_smem(stages + s * C::STAGE_BYTES);
            for (int j = 0; j < C::JT; ++j, ++u) {
                const int bf = u % C::NBUF;
                if (lane == 0) ok = um_wait(tempty0 + 8u * bf, ((u / C::NBUF) & 1) ^ 1, &s_abort, p.status, p.wait_ns);
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    alive = false;
                    break;
                }
                um_fence_after();
                if (lane == 0) {
                    const unsigned dcol = tmem + (unsigned)(bf * C::BUFN);
#pragma unroll
                    for (int ks = 0; ks < C::KSTEPS; ++ks) {
                        const int c = NT * j + C::KE * ks;  // first column of the K slice (from x0 - L)
#pragma unroll
                        for (int g = 0; g < C::NG; ++g) {
                            const int sh = g * D;  // row shift of A for this group
                            const unsigned long long a =
                                c < kUmCols ? um_desc_sw128(sbase + (unsigned)((c / C::AE) * kUmAtom + 128 * sh +
                                                                               (c % C::AE) * C::EB))
                                            : um_desc(sbase + (unsigned)(C::NA * kUmAtom + 16 * sh), kUmPlane, 128);
                            const unsigned pitch = (unsigned)(C::rows(g) * NT * 16);
                            const unsigned long long bd =
                                um_desc(um_smem(bmat) + (unsigned)(sh * C::ROW_BYTES) + (unsigned)(ks * C::PPI) * pitch,
                                        pitch, 128);
                            um_mma<TF32>(dcol, a, bd, um_idesc_n<TF32>(C::rows(g) * NT), (ks | g) != 0);
                        }
                    }
                    if (!(p.withhold && blockIdx.x == 0 && u == 0)) um_commit(tfull0 + 8u * bf);
                    issued = 1;
                }
                __syncwarp();
            }
            if (!alive) break;
            if (lane == 0) um_commit(empty0 + 8u * s);  // the stage is free once these MMAs have read it
            __syncwarp();
        }
        if (lane == 0 && issued) {
            um_commit(drain);
            um_drain(drain, 0, p.status, p.wait_ns);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: TMEM lanes 32 q .. 32 q + 31 ----------------
        // Per N-tile: load the D column blocks of the thread's lane (one wait),
        // free the accumulator, pass lanes 0 .. D-2 to the quarter above, add
        // the blocks with lane shifts and write the row into the swizzled
        // staging tile; one thread stores each finished part with TMA.
        const int q = warp & 3;
        const int r = 32 * q + lane;                 // TMEM lane = output row of block 0
        const bool issuer = threadIdx.x == 64;
        constexpr int AEO = 128 / C::EB;             // output columns per staged atom
        constexpr int EPC = 16 / C::EB;              // output columns per 16-byte chunk
        constexpr int CPC = 32 / EPC;                // chunks per 32 columns
        constexpr int PW = kUmCols / C::PARTS;       // columns per staged part
        constexpr int APP = PW / AEO;                // atoms per staged part
        int it = 0, u = 0, xpar = 0;
        bool alive = true;
        for (int tile = blockIdx.x; tile < p.tiles && alive; tile += gridDim.x, ++it) {
            const int x0 = (tile % p.tiles_x) * kUmCols, y0 = (tile / p.tiles_x) * C::OUT;
            for (int j = 0; j < C::JT; ++j, ++u) {
                const int part = (NT * j) / PW;
                const int sb = C::STG == 2 ? ((it * C::PARTS + part) & 1) : 0;
                const unsigned stg = um_smem(outstg + sb * C::PART_BYTES);
                if ((NT * j) % PW == 0) {
                    // the store that last read this staging buffer has finished reading it
                    if (issuer) {
                        if constexpr (C::STG == 2)
                            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                        else
                            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    }
                    um_epi_sync();
                }
                const int bf = u % C::NBUF;
                int ok = 1;
                if (lane == 0) ok = um_wait(tfull0 + 8u * bf, (u / C::NBUF) & 1, &s_abort, p.status, p.wait_ns);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!um_epi_and(ok)) {  // the four epilogue warps leave together
                    alive = false;
                    break;
                }
                um_fence_after();
#pragma unroll 1
                for (int ch = 0; ch < NT / 32; ++ch) {
                    unsigned v[D][32];
                    const unsigned tb = tmem + ((unsigned)(32 * q) << 16) + (unsigned)(bf * C::BUFN + 32 * ch);
#pragma unroll
                    for (int d = 0; d < D; ++d) um_ld32(tb + (unsigned)(d * NT), v[d]);
                    um_ld_wait();
                    if (ch == NT / 32 - 1) {
                        um_fence_before();
                        __syncwarp();
                        if (lane == 0) um_bar_arrive(tempty0 + 8u * bf);  // accumulator free for the MMAs
                    }
                    // lanes l < d of block d feed rows 32 q + l + 32 - d of the quarter below
                    float* xw = xch + (xpar * 4 + q) * C::XQ;
#pragma unroll
                    for (int d = 1; d < D; ++d) {
                        if (lane < d) {
                            float4* dst = reinterpret_cast<float4*>(xw + ((d - 1) * (D - 1) + lane) * 32);
#pragma unroll
                            for (int n = 0; n < 8; ++n)
                                dst[n] = make_float4(__uint_as_float(v[d][4 * n]), __uint_as_float(v[d][4 * n + 1]),
                                                     __uint_as_float(v[d][4 * n + 2]), __uint_as_float(v[d][4 * n + 3]));
                        }
                    }
                    um_epi_sync();
                    // quarter 3 reads quarter 0 here only for rows >= OUT, which are never stored
                    const float* xr = xch + (xpar * 4 + ((q + 1) & 3)) * C::XQ;
                    xpar ^= 1;
                    float o[32];
#pragma unroll
                    for (int n = 0; n < 32; ++n) o[n] = __uint_as_float(v[0][n]);
#pragma unroll
                    for (int d = 1; d < D; ++d) {
                        const bool top = lane + d >= 32;  // row r + d lies in the next quarter
                        const float4* src =
                            reinterpret_cast<const float4*>(xr + ((d - 1) * (D - 1) + (top ? lane + d - 32 : 0)) * 32);
#pragma unroll
                        for (int n = 0; n < 8; ++n) {
                            float s0 = __shfl_down_sync(0xffffffffu, __uint_as_float(v[d][4 * n]), d);
                            float s1 = __shfl_down_sync(0xffffffffu, __uint_as_float(v[d][4 * n + 1]), d);
                            float s2 = __shfl_down_sync(0xffffffffu, __uint_as_float(v[d][4 * n + 2]), d);
                            float s3 = __shfl_down_sync(0xffffffffu, __uint_as_float(v[d][4 * n + 3]), d);
                            if (top) {
                                const float4 t = src[n];
                                s0 = t.x;
                                s1 = t.y;
                                s2 = t.z;
                                s3 = t.w;
                            }
                            o[4 * n] += s0;
                            o[4 * n + 1] += s1;
                            o[4 * n + 2] += s2;
                            o[4 * n + 3] += s3;
                        }
                    }
                    const int col0 = NT * j + 32 * ch;  // tile column of o[0]
                    const int a = (col0 / AEO) % APP;   // atom in the staged part
                    const int c0 = (col0 % AEO) / EPC;  // its first 16-byte chunk in the row
#pragma unroll
                    for (int c = 0; c < CPC; ++c) {
                        unsigned w[4];
                        if constexpr (TF32) {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                w[i] = p.round_out ? um_tf32(o[4 * c + i]) : __float_as_uint(o[4 * c + i]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                __nv_bfloat162 h = __floats2bfloat162_rn(o[8 * c + 2 * i], o[8 * c + 2 * i + 1]);
                                w[i] = *reinterpret_cast<unsigned*>(&h);
                            }
                        }
                        um_st_shared_v4(stg + (unsigned)(a * kUmRows * 128 + r * 128 + (((c0 + c) ^ (r & 7)) << 4)),
                                        w[0], w[1], w[2], w[3]);
                    }
                }
                if ((NT * (j + 1)) % PW == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // staging is read by TMA
                    um_epi_sync();
                    if (issuer) {
#pragma unroll
                        for (int a = 0; a < APP; ++a)
                            um_tma_store_2d(&tmap_out, stg + (unsigned)(a * kUmRows * 128), x0 + (part * APP + a) * AEO,
                                            y0);
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                }
            }
        }
        if (issuer) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    }

    um_fence_before();
    __syncthreads();
    um_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// ---- host side ----------------------------------------------------------------------------

// Kernel for (tf32, nt), or NULL when that pair is not instantiated.
const void* get_box49_umma_kernel(int tf32, int nt) {
    if (tf32) {
        if (nt == 16) return (const void*)box49_umma_kernel<true, 16>;
        if (nt == 32) return (const void*)box49_umma_kernel<true, 32>;
        if (nt == 96) return (const void*)box49_umma_rows_kernel<true, 32, 3>;
        if (nt == 128) return (const void*)box49_umma_rows_kernel<true, 32, 4>;
        return nullptr;  // wider one-row TF32 tiles do not fit shared memory
    }
    if (nt == 16) return (const void*)box49_umma_kernel<false, 16>;
    if (nt == 32) return (const void*)box49_umma_kernel<false, 32>;
    if (nt == 64) return (const void*)box49_umma_kernel<false, 64>;
    if (nt == 96) return (const void*)box49_umma_rows_kernel<false, 32, 3>;
    if (nt == 128) return (const void*)box49_umma_rows_kernel<false, 32, 4>;
    return nullptr;
}

int box49_umma_smem_bytes(int tf32, int nt) {
    if (tf32) {
        if (nt == 96) return UmgCfg<true, 32, 3>::SMEM;
        if (nt == 128) return UmgCfg<true, 32, 4>::SMEM;
        return nt == 16 ? UmCfg<true, 16>::SMEM : UmCfg<true, 32>::SMEM;
    }
    if (nt == 96) return UmgCfg<false, 32, 3>::SMEM;
    if (nt == 128) return UmgCfg<false, 32, 4>::SMEM;
    return nt == 16 ? UmCfg<false, 16>::SMEM : nt == 32 ? UmCfg<false, 32>::SMEM : UmCfg<false, 64>::SMEM;
}

// Output rows per tile: 128 for one weight row per MMA (N <= 64), 129 - D for
// D = N / 32 rows per MMA.
int box49_umma_tile_rows(int nt) { return nt > 64 ? kUmRows + 1 - nt / 32 : kUmRows; }

int box49_umma_threads(int) { return kUmThreads; }

static PFN_cuTensorMapEncodeTiled_v12000 um_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && ptr)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        else
            cudaGetLastError();
    }
    return fn;
}

static CUresult um_encode(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* map, int tf32, const void* src,
                          int ny, int nx, int ld, int box_x, int box_y, CUtensorMapSwizzle swz) {
    const int eb = tf32 ? 4 : 2;
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * (cuuint64_t)eb};
    const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
               const_cast<void*>(src), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// One step src -> dst on at most `ctas` persistent CTAs.  The caller
// guarantees: src and dst 16-byte aligned, ld * element size a multiple of 16
// bytes, ny >= 134 and nx >= 128.  Returns cudaErrorNotSupported when no
// tensor map can be made for this layout.
cudaError_t launch_box49_umma(int tf32, int nt, const void* src, void* dst, int ny, int nx, int ld,
                              int round_out, unsigned* status, const float* w, int ctas, cudaStream_t st,
                              int timeout_ms, int withhold) {
    const void* fn = get_box49_umma_kernel(tf32, nt);
    PFN_cuTensorMapEncodeTiled_v12000 enc = um_encoder();
    if (!fn || !enc) return cudaErrorNotSupported;
    const int eb = tf32 ? 4 : 2;
    alignas(64) CUtensorMap map_sw, map_pl, map_out;
    if (um_encode(enc, &map_sw, tf32, src, ny, nx, ld, 128 / eb, kUmSR, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS ||
        um_encode(enc, &map_pl, tf32, src, ny, nx, ld, 16 / eb, kUmSR, CU_TENSOR_MAP_SWIZZLE_NONE) != CUDA_SUCCESS ||
        um_encode(enc, &map_out, tf32, dst, ny, nx, ld, 128 / eb, box49_umma_tile_rows(nt),
                  CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    UmParams up{};
    up.out = dst;
    up.ny = ny;
    up.nx = nx;
    up.ld = ld;
    up.tiles_x = (nx + kUmCols - 1) / kUmCols;
    up.tiles = up.tiles_x * ((ny + box49_umma_tile_rows(nt) - 1) / box49_umma_tile_rows(nt));
    up.round_out = round_out;
    up.status = status;
    up.wait_ns = (long long)(timeout_ms > 0 ? timeout_ms : 2000) * 1000000LL;
    up.withhold = withhold;
    for (int i = 0; i < 49; ++i) up.w[i] = w[i];
    void* args[] = {&map_sw, &map_pl, &map_out, &up};
    const int grid = ctas < up.tiles ? ctas : up.tiles;
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3((unsigned)box49_umma_threads(nt)), args,
                            (size_t)box49_umma_smem_bytes(tf32, nt), st);
}

}  // namespace gbst
