// plan.cu -- host side of the C ABI: plans, launch sequencing, workspace.
//
// A plan fixes (shape, radius, weights, dtype, boundary) and picks a kernel
// configuration: the temporal-blocking depth k, the CTA size and the tile
// shape of the streaming kernel (sweep_stream.cuh), or the naive kernel.
// stencil_run() then issues ceil(T/k) launches that ping-pong between the
// caller's output and one plan-owned workspace grid, so that the last launch
// writes `out` and `in` is never written.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

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
StreamKernelRef get_stream_states_kernel(int R, int star, int k);
StreamKernelRef get_stream_tma_kernel_r1(int star, int k);
StreamKernelRef get_stream_tma_kernel_r2(int star, int k);
StreamKernelRef get_stream_tma_kernel_r3(int star, int k);
const void* get_naive_kernel(int radius, int dtype);
int lowrank_factor(const float* w, int R, int rank, float col[7][7], float row[7][7], double* sv);
const void* get_lowrank_kernel(int R, int rho);
cudaError_t launch_lowrank(const void* fn, const float* src, float* dst, long long ny, long long nx, int periodic,
                           const float col[7][7], const float row[7][7], int sms, cudaStream_t st);
const void* get_box49_tc_kernel(int dtype, int engine);       // engine: 0 TF32, 1 BF16, 2 3xTF32
const void* get_box49_tc_pipe_kernel(int dtype, int engine);
int box49_tc_smem_bytes(int engine);
const void* get_box49_umma_kernel(int tf32, int nt);
int box49_umma_smem_bytes(int tf32, int nt);
int box49_umma_threads(int nt);
int box49_umma_tile_rows(int nt);
cudaError_t launch_box49_umma(int tf32, int nt, const void* src, void* dst, int ny, int nx, int ld,
                              int round_out, unsigned* status, const float* w, int ctas, cudaStream_t st,
                              int timeout_ms, int withhold);
const void* get_resident_kernel(int radius, int star, int dtype);
int resident_threads();
int resident_max_cluster();
int resident_config(int ny, int nx, int radius, int periodic, int C, int kb, int max_smem, int* rp_out);
cudaError_t launch_resident(const void* fn, int C, int smem, const ResidentParams& prm, cudaStream_t st);
bool resident_cluster_fits(const void* fn, int C, int smem);
struct TcParams {  // must match box49_tc.cu
    const void* in;
    void* out;
    int ny, nx, ld;
    int periodic;
    int tiles_x, tiles;
    int vec;
    int convert_in;
    int round_out;
    float w[49];
};
}  // namespace gbst

using namespace gbst;

static thread_local std::string g_last_error;

static stencil_status_t fail(stencil_status_t st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

#define CK(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            return fail(STENCIL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                            \
    } while (0)

struct stencil_plan {
    int64_t ny = 0, nx = 0;
    int R = 0;
    int star = 0;
    int dtype = 0, boundary = 0, compute = 0;
    Weights w{};
    stencil_options_t opt{};
    int device = 0, sms = 0;
    // chosen configuration
    int kernel = STENCIL_KERNEL_STREAM;
    int k = 1, threads = 0, H = 0, bx = 0, by = 0, strips = 0, tiles_y = 0, smem = 0;
    int per_sm = 0;
    int tma = 0;  // streaming kernel fed by the tensor-memory-access engine
    // separable (low-rank) form of the weights: rank and FP32 factors
    int lr_rank = 0;
    float lr_col[7][7] = {}, lr_row[7][7] = {};
    const void* lr_fn = nullptr;
    const void* tc_pipe = nullptr;  // persistent double-buffered tensor-core kernel
    int tc_pipe_smem = 0, tc_pipe_ctas = 0;
    int umma_n = 0;     // tcgen05 engine in use: N of one MMA (0: warp-MMA engine)
    int umma_ok = 0;    // usable tcgen05 MMA widths, bit n / 16
    int umma_ctas = 0;
    // cluster-resident kernel (sweep_resident.cu): usable cluster sizes (bit log2 C), the one in use
    const void* res_fn = nullptr;
    int res_ok = 0, res_c = 0, res_rp = 0, res_kb = 1, res_smem = 0, res_max_smem = 0;
    unsigned smem_set = 0;  // bit 2k+vec: that kernel's shared-memory attribute is set
    int tuned = 0;
    const void* naive = nullptr;
    // memory
    size_t elem = 4;
    void* ws = nullptr;
    void* host_in = nullptr;
    void* host_out = nullptr;
    unsigned int* status = nullptr;
    cudaStream_t last_stream = nullptr;
    // Scratch of other subsystems (0: adjoint, 1: residual runs), released with the plan.
    void* aux[4] = {nullptr, nullptr, nullptr, nullptr};
    void (*aux_free[4])(void*) = {nullptr, nullptr, nullptr, nullptr};
};

namespace gbst {
void plan_weights(const stencil_plan_t* p, float* w) {
    for (int i = 0; i < kMaxTaps; ++i) w[i] = p->w.w[i];
}
void** plan_aux_slot(stencil_plan_t* p, int id) { return &p->aux[id]; }
void plan_set_aux_free(stencil_plan_t* p, int id, void (*freer)(void*)) { p->aux_free[id] = freer; }
stencil_status_t plan_run_states(stencil_plan_t* p, const void* in, float* const* outs, int64_t n,
                                 cudaStream_t st);
}  // namespace gbst

static size_t elem_size(int dtype) { return dtype == STENCIL_F32 ? 4 : 2; }

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

static StreamKernelRef stream_kernel(int R, int star, int k, int dtype, int vec) {
    typedef StreamKernelRef (*Getter)(int, int, int);
    static const Getter table[3][3] = {
        {get_stream_kernel_r1_f32, get_stream_kernel_r1_bf16, get_stream_kernel_r1_f16},
        {get_stream_kernel_r2_f32, get_stream_kernel_r2_bf16, get_stream_kernel_r2_f16},
        {get_stream_kernel_r3_f32, get_stream_kernel_r3_bf16, get_stream_kernel_r3_f16}};
    if (R < 1 || R > 3 || dtype < 0 || dtype > 2) return {nullptr, 0};
    return table[R - 1][dtype](star, k, vec);
}

// Largest instantiated depth for (R, star), and the largest one <= k.
static int stream_kmax(int R, int star) {
    int m = 0;
    for (int i = 0; i < 8 && kStreamDepths[R - 1][star][i]; ++i) m = kStreamDepths[R - 1][star][i];
    return m;
}

static int stream_depth_at_most(int R, int star, int k) {
    int m = 0;
    for (int i = 0; i < 8 && kStreamDepths[R - 1][star][i]; ++i)
        if (kStreamDepths[R - 1][star][i] <= k) m = kStreamDepths[R - 1][star][i];
    return m;
}

// Default depth before any tuning: deep enough that HBM stops binding for the
// light stencils, 2 for the 49-point box (arithmetic-bound already at k = 1;
// at 16384^2 FP32, k = 2 with 256-thread CTAs 509 GStencil/s against 478 for
// k = 1 with 128 threads).
// These are the best measured choices for 8192^2 FP32 grids on GB300 (the
// 13-point star: k = 3 with its 128-register bound, 4 CTAs per SM, ties k = 2
// at 1173 GStencil/s and moves a third less DRAM traffic; k = 4 needs more
// registers than fit 4 CTAs).
static int default_depth(int R, int star) {
    if (R == 1) return 8;
    if (R == 2) return 4;
    return star ? 3 : 2;
}

// CTA size and row feed before tuning: the configurations the autotuner keeps
// for 8192^2 FP32 grids on GB300 (9-point box at k = 8: 64-thread CTAs, 2354
// GStencil/s against 2256 with 128 threads and TMA rows, 2142 with 128 threads
// and cp.async rows; 13-point star at k = 3: 128 threads, cp.async 1271).  The
// TMA-fed ring is behind the cp.async ring elsewhere (5-point star at k = 6, 8:
// 2772 / 2924 against 2811 / 3050; 9-point box at k = 6 with 128 threads 2012
// against 2107; 13-point star at k = 2, 3, 4: 1060 / 1128 / 780 against 1223 /
// 1244 / 963), so it is never the default and the autotuner times both.
static int default_threads(int R, int star) {
    if (R == 1 && !star) return 64;
    return (R == 3 && !star) ? 256 : 128;
}
static const int kDefaultTma = 0;

// Plans whose rows the TMA-fed streaming kernel can load: FP32 storage, the
// zero rule (the copy engine's zero fill is the zero halo) and rows of a
// multiple of 16 bytes (the tensor map's row pitch).
static bool tma_eligible(const stencil_plan* p) {
    return p->dtype == STENCIL_F32 && p->boundary == STENCIL_BOUNDARY_ZERO && p->nx % 4 == 0;
}

static StreamKernelRef stream_tma_kernel(int R, int star, int k) {
    switch (R) {
        case 1: return get_stream_tma_kernel_r1(star, k);
        case 2: return get_stream_tma_kernel_r2(star, k);
        case 3: return get_stream_tma_kernel_r3(star, k);
        default: return {nullptr, 0};
    }
}

// The depth-`depth` streaming kernel (TMA-fed, VEC or element-wise variant),
// with its shared-memory attribute set on first use.
// `smem` receives the dynamic shared memory of a launch with CTAs of `nt`
// threads; the kernel's attribute allows the largest CTA.
static stencil_status_t stream_fn(stencil_plan* p, int depth, int vec, const void** fn, int* smem,
                                  int tma, int nt) {
    tma = tma && vec;
    StreamKernelRef r = tma ? stream_tma_kernel(p->R, p->star, depth)
                            : stream_kernel(p->R, p->star, depth, p->dtype, vec);
    if (!r.fn) return fail(STENCIL_ERR_UNSUPPORTED, "no streaming kernel for depth " + std::to_string(depth));
    *smem = stream_smem_bytes(p->R, depth, (int)p->elem, vec != 0, tma != 0, nt);
    const unsigned bit = 1u << (2 * depth + (vec ? 1 : 0) + (tma ? 16 : 0));
    if (!(p->smem_set & bit)) {
        CK(cudaFuncSetAttribute(r.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                stream_smem_bytes(p->R, depth, (int)p->elem, vec != 0, tma != 0, kStreamMaxThreads)));
        p->smem_set |= bit;
    }
    *fn = r.fn;
    return STENCIL_OK;
}

// Tensor map of an FP32 grid for the TMA-fed streaming kernel: nx x ny
// elements, row pitch ld, boxes of kStreamTmaBox columns x 1 row, zero fill.
typedef CUresult (*TmaEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static TmaEncodeFn tma_encoder() {
    static TmaEncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && ptr)
            fn = reinterpret_cast<TmaEncodeFn>(ptr);
        else
            cudaGetLastError();
    });
    return fn;
}

static bool stream_tensor_map(CUtensorMap* map, const void* src, int64_t ny, int64_t nx) {
    TmaEncodeFn enc = tma_encoder();
    if (!enc || (uintptr_t)src % 16 != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)nx * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kStreamTmaBox, 1};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(src), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Fill the streaming kernel's tile configuration for depth k and CTA size threads.
static stencil_status_t configure_stream(stencil_plan* p, int k, int threads, int tile_rows) {
    const int kmax = stream_kmax(p->R, p->star);
    if (k < 1 || k > kmax)
        return fail(STENCIL_ERR_UNSUPPORTED,
                    "tb_depth " + std::to_string(k) + " outside 1.." + std::to_string(kmax) +
                        " for radius " + std::to_string(p->R));
    k = stream_depth_at_most(p->R, p->star, k);
    if (threads < 32 || threads > kStreamMaxThreads || threads % 32)
        return fail(STENCIL_ERR_INVALID_ARG, "threads must be a multiple of 32 in 32..256");
    const int vec = p->nx % 4 == 0;
    const int H = (p->R * k + 3) / 4 * 4;
    const int bx_max = 4 * threads - 2 * H;
    if (bx_max < 4) return fail(STENCIL_ERR_UNSUPPORTED, "CTA too narrow for this depth");
    const int64_t strips = ceil_div(p->nx, bx_max);
    const int bx = (int)(ceil_div(ceil_div(p->nx, strips), 4) * 4);
    const int nt = (int)(ceil_div(ceil_div(bx + 2 * H, 4), 32) * 32);
    const void* fn = nullptr;
    int smem = 0;
    stencil_status_t st = stream_fn(p, k, vec, &fn, &smem, p->tma, nt);
    if (st != STENCIL_OK) return st;
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem));
    if (per_sm < 1) return fail(STENCIL_ERR_UNSUPPORTED, "streaming kernel does not fit on an SM");
    int64_t tiles_y;
    int by;
    if (tile_rows > 0) {
        by = tile_rows;
        tiles_y = ceil_div(p->ny, by);
    } else {
        const int64_t resident = (int64_t)per_sm * p->sms;
        const int64_t by_min = std::max<int64_t>(8, 4LL * p->R * k);
        const int64_t want = std::max<int64_t>(1, resident / strips);
        tiles_y = std::max<int64_t>(1, std::min<int64_t>(want, ceil_div(p->ny, by_min)));
        by = (int)ceil_div(p->ny, tiles_y);
        tiles_y = ceil_div(p->ny, by);
    }
    if (strips * tiles_y > 0x7fffffffLL) return fail(STENCIL_ERR_UNSUPPORTED, "grid too large");
    p->kernel = STENCIL_KERNEL_STREAM;
    p->k = k;
    p->threads = nt;
    p->H = H;
    p->bx = bx;
    p->by = by;
    p->strips = (int)strips;
    p->tiles_y = (int)tiles_y;
    p->smem = smem;
    p->per_sm = per_sm;
    return STENCIL_OK;
}

// Default N of one tcgen05 MMA per operand type (BF16, TF32), and whether
// that engine is the default for the tensor-core kernel family (kernel = TC or
// AUTO without autotuning).  Measured on GB300, 16384^2 Box-49, 200 steps:
// BF16 tcgen05 N = 64 916 GStencil/s (N = 32: 856, N = 16: 614; three or four
// weight rows per MMA, N = 96: 784, N = 128: 596) against 708 for the warp-MMA
// engine; TF32 tcgen05 N = 96 547 (N = 32: 492, N = 16: 417, N = 128: 457)
// against 421.  Autotuning times both engines and every width.
static const int kUmmaDefaultN[2] = {64, 96};
// MMA widths of the tcgen05 kernels: N = 16, 32, 64 with one weight row per
// MMA; N = 96 and 128 stack three or four weight rows over 32-column N-tiles.
static const int kUmmaWidths[5] = {16, 32, 64, 96, 128};
static const int kUmmaPreferred[2] = {1, 1};

// The tcgen05 engine (box49_umma.cu) takes zero-boundary grids whose storage is
// the MMA operand type (BF16 storage for TC_BF16, FP32 for TC_TF32), with
// 16-byte aligned rows and at least one full staged tile.  With TF32 the first
// launch of a run stays on the warp-MMA engine, which rounds the caller's
// input (and every output but the last) to TF32.  kernel = TC_UMMA makes the
// engine mandatory, TC_WARP switches it off.  p->umma_ok collects the usable
// MMA widths (bit n / 16), p->umma_n the one in use (0: warp-MMA engine).
static stencil_status_t configure_umma(stencil_plan* p) {
    p->umma_n = 0;
    p->umma_ok = 0;
    const int want = p->opt.kernel;
    if (want == STENCIL_KERNEL_TC_WARP) return STENCIL_OK;
    const int tf32 = p->compute == STENCIL_COMPUTE_TC_TF32;
    const char* why = nullptr;
    if (p->compute == STENCIL_COMPUTE_TC_3XTF32) why = "the tcgen05 engine runs TF32 and BF16 operands only";
    else if (p->boundary != STENCIL_BOUNDARY_ZERO) why = "the tcgen05 engine takes zero-boundary grids";
    else if (tf32 ? p->dtype != STENCIL_F32 : p->dtype != STENCIL_BF16)
        why = "the tcgen05 engine needs FP32 storage for TF32 and BF16 storage for BF16";
    else if ((p->nx * (int64_t)p->elem) % 16 != 0) why = "the tcgen05 engine needs rows of a multiple of 16 bytes";
    else if (p->ny < 134 || p->nx < 128) why = "the tcgen05 engine needs ny >= 134 and nx >= 128";
    else if (p->opt.mma_n > 0 && !get_box49_umma_kernel(tf32, p->opt.mma_n))
        why = "no tcgen05 kernel for this mma_n (BF16: 16, 32, 64, 96, 128; TF32: 16, 32, 96, 128)";
    if (!why) {
        for (int nt : kUmmaWidths) {
            if (p->opt.mma_n > 0 && nt != p->opt.mma_n) continue;
            const void* fn = get_box49_umma_kernel(tf32, nt);
            if (!fn) continue;
            const int smem = box49_umma_smem_bytes(tf32, nt);
            CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            int per_sm = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, box49_umma_threads(nt), smem));
            if (per_sm >= 1) p->umma_ok |= 1 << (nt / 16);
        }
        if (!p->umma_ok) why = "the tcgen05 kernel does not fit an SM";
    }
    if (why) {
        if (want == STENCIL_KERNEL_TC_UMMA) return fail(STENCIL_ERR_UNSUPPORTED, why);
        return STENCIL_OK;
    }
    // One CTA per SM: each holds 256 (one weight row per MMA) or 512 (row
    // groups) tensor-memory columns for its whole life.
    p->umma_ctas = (int)std::min<int64_t>((int64_t)p->sms, (int64_t)p->strips * p->tiles_y);
    const int nt = p->opt.mma_n > 0 ? p->opt.mma_n : kUmmaDefaultN[tf32];
    if (want == STENCIL_KERNEL_TC_UMMA || kUmmaPreferred[tf32]) p->umma_n = (p->umma_ok >> (nt / 16)) & 1 ? nt : 0;
    if (want == STENCIL_KERNEL_TC_UMMA && !p->umma_n) return fail(STENCIL_ERR_UNSUPPORTED, "tcgen05 kernel unusable");
    p->kernel = p->umma_n ? STENCIL_KERNEL_TC_UMMA : STENCIL_KERNEL_TC;
    return STENCIL_OK;
}

static stencil_status_t configure_tc(stencil_plan* p) {
    if (p->R != 3) return fail(STENCIL_ERR_UNSUPPORTED, "tensor-core engines need radius 3 (7x7 weights)");
    if (p->dtype == STENCIL_F16) return fail(STENCIL_ERR_UNSUPPORTED, "tensor-core engines take FP32 or BF16 storage");
    const int engine = p->compute == STENCIL_COMPUTE_TC_BF16 ? 1 : p->compute == STENCIL_COMPUTE_TC_3XTF32 ? 2 : 0;
    if (engine == 2 && p->dtype != STENCIL_F32)
        return fail(STENCIL_ERR_UNSUPPORTED, "3xTF32 splits FP32 values: it takes FP32 storage");
    p->naive = get_box49_tc_kernel(p->dtype, engine);
    if (!p->naive) return fail(STENCIL_ERR_UNSUPPORTED, "no tensor-core kernel for this dtype");
    p->kernel = STENCIL_KERNEL_TC;
    p->k = 1;
    p->threads = 256;
    p->H = 3;
    p->bx = 128;
    p->by = 128;
    p->strips = (int)ceil_div(p->nx, 128);
    p->tiles_y = (int)ceil_div(p->ny, 128);
    p->smem = box49_tc_smem_bytes(engine);
    CK(cudaFuncSetAttribute(p->naive, cudaFuncAttributeMaxDynamicSharedMemorySize, p->smem));
    p->tc_pipe = p->nx % 4 == 0 ? get_box49_tc_pipe_kernel(p->dtype, engine) : nullptr;
    if (p->tc_pipe) {
        p->tc_pipe_smem = 2 * p->smem;
        CK(cudaFuncSetAttribute(p->tc_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, p->tc_pipe_smem));
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->tc_pipe, 256, p->tc_pipe_smem));
        if (per_sm < 1) {
            p->tc_pipe = nullptr;
        } else {
            p->tc_pipe_ctas = (int)std::min<int64_t>((int64_t)per_sm * p->sms, (int64_t)p->strips * p->tiles_y);
        }
    }
    return configure_umma(p);
}

// The cluster-resident kernel holds the grid in the shared memory of one
// cluster of C <= 16 CTAs and runs a whole run in one launch.  It applies when
// some C in {1, 2, 4, 8, 16} gives slabs that fit a CTA's shared memory and
// are at least R rows high (periodic grids also need nx >= R), and the
// cluster can be scheduled.  Sets p->res_ok (bit log2 C per usable C) and
// returns the largest usable C, or 0.
static int resident_candidates(stencil_plan* p, int kb = 1) {
    p->res_ok = 0;
    if (p->compute != STENCIL_COMPUTE_FP32) return 0;
    const int periodic = p->boundary == STENCIL_BOUNDARY_PERIODIC;
    if (periodic && p->nx < p->R) return 0;
    if (p->ny > (1 << 20) || p->nx > (1 << 20)) return 0;
    const void* fn = get_resident_kernel(p->R, p->star, p->dtype);
    if (!fn) return 0;
    int max_smem = 0;
    if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    p->res_max_smem = max_smem;
    int best = 0;
    for (int C = 1; C <= resident_max_cluster(); C *= 2) {
        int rp = 0;
        const int smem = resident_config((int)p->ny, (int)p->nx, p->R, periodic, C, kb, max_smem, &rp);
        if (smem < 0) continue;
        if (!resident_cluster_fits(fn, C, smem)) continue;
        int lg = 0;
        while ((1 << lg) < C) ++lg;
        p->res_ok |= 1 << lg;
        best = C;
    }
    p->res_fn = fn;
    return best;
}

// Switch the plan to the resident kernel with cluster size C and kb steps per
// halo exchange (kb = 1 by default: deeper blocking only pays where a step's
// work is small next to the cluster barrier, which autotuning measures).
static stencil_status_t use_resident(stencil_plan* p, int C, int kb = 1) {
    const int periodic = p->boundary == STENCIL_BOUNDARY_PERIODIC;
    int rp = 0;
    const int smem = resident_config((int)p->ny, (int)p->nx, p->R, periodic, C, kb, p->res_max_smem, &rp);
    if (smem < 0) return fail(STENCIL_ERR_UNSUPPORTED, "grid does not fit the cluster-resident kernel");
    CK(cudaFuncSetAttribute(p->res_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    if (C > 8) CK(cudaFuncSetAttribute(p->res_fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    p->kernel = STENCIL_KERNEL_RESIDENT;
    p->res_c = C;
    p->res_rp = rp;
    p->res_kb = kb;
    p->res_smem = smem;
    return STENCIL_OK;
}

static stencil_status_t configure_naive(stencil_plan* p) {
    p->naive = get_naive_kernel(p->R, p->dtype);
    if (!p->naive) return fail(STENCIL_ERR_UNSUPPORTED, "no naive kernel for this radius");
    p->kernel = STENCIL_KERNEL_NAIVE;
    p->k = 1;
    p->threads = 256;
    p->H = 0;
    p->bx = 32;
    p->by = 8;
    p->strips = (int)ceil_div(p->nx, 32);
    p->tiles_y = (int)std::min<int64_t>(ceil_div(p->ny, 8), 65535);
    p->smem = 0;
    return STENCIL_OK;
}

// Separable form (compute = LOWRANK): factor the weights, one step per launch.
static stencil_status_t configure_lowrank(stencil_plan* p) {
    if (p->dtype != STENCIL_F32) return fail(STENCIL_ERR_UNSUPPORTED, "the low-rank form takes FP32 storage");
    if (p->opt.kernel != STENCIL_KERNEL_AUTO)
        return fail(STENCIL_ERR_UNSUPPORTED, "the low-rank form has its own kernel (kernel must be AUTO)");
    p->lr_rank = lowrank_factor(p->w.w, p->R, p->opt.rank, p->lr_col, p->lr_row, nullptr);
    if (p->lr_rank < 1) p->lr_rank = 1;  // all-zero weights: one zero term
    p->lr_fn = get_lowrank_kernel(p->R, p->lr_rank);
    if (!p->lr_fn) return fail(STENCIL_ERR_UNSUPPORTED, "no low-rank kernel for this rank");
    p->kernel = STENCIL_KERNEL_LOWRANK;
    p->k = 1;
    p->threads = 128;
    p->H = p->R;
    p->bx = 128;
    p->strips = (int)ceil_div(p->nx, 128);
    p->tiles_y = 1;
    p->by = (int)p->ny;
    p->smem = 0;
    return STENCIL_OK;
}

// One launch advancing `nlev` steps from src to dst.  `first` / `last`: this
// launch starts / ends a run (the pipelined TF32 engine rounds its input on
// the first launch and keeps intermediate states TF32-rounded until the last).
static stencil_status_t launch_once(stencil_plan* p, const void* src, void* dst, int nlev,
                                    cudaStream_t st, int first = 1, int last = 1) {
    if (p->kernel == STENCIL_KERNEL_TC || p->kernel == STENCIL_KERNEL_TC_UMMA) {
        TcParams tp{};
        tp.in = src;
        tp.out = dst;
        tp.ny = (int)p->ny;
        tp.nx = (int)p->nx;
        tp.ld = (int)p->nx;
        tp.periodic = p->boundary == STENCIL_BOUNDARY_PERIODIC;
        tp.tiles_x = p->strips;
        tp.tiles = p->strips * p->tiles_y;
        tp.vec = (p->nx % 4 == 0) && ((uintptr_t)src % (4 * p->elem) == 0) &&
                 ((uintptr_t)dst % (4 * p->elem) == 0);
        tp.convert_in = first;
        tp.round_out = !last;
        for (int i = 0; i < 49; ++i) tp.w[i] = p->w.w[i];
        const int tf32 = p->compute == STENCIL_COMPUTE_TC_TF32;
        if (p->umma_n && !(tf32 && first) && (uintptr_t)src % 16 == 0 && (uintptr_t)dst % 16 == 0) {
            const cudaError_t e = launch_box49_umma(tf32, p->umma_n, src, dst, tp.ny, tp.nx, tp.ld,
                                                    tf32 && !last, p->status, p->w.w, p->umma_ctas, st,
                                                    p->opt.timeout_ms, p->opt.debug_withhold);
            if (e == cudaSuccess) return STENCIL_OK;
            if (e != cudaErrorNotSupported) CK(e);
            // no tensor map for this layout: the warp-MMA engine takes the step
        }
        void* args[] = {&tp};
        if (p->tc_pipe && tp.vec) {
            CK(cudaLaunchKernel(p->tc_pipe, dim3((unsigned)p->tc_pipe_ctas), dim3(256), args,
                                (size_t)p->tc_pipe_smem, st));
        } else {
            CK(cudaLaunchKernel(p->naive, dim3((unsigned)tp.tiles), dim3(256), args, (size_t)p->smem, st));
        }
        return STENCIL_OK;
    }
    if (p->kernel == STENCIL_KERNEL_RESIDENT) {
        ResidentParams rp{};
        rp.in = src;
        rp.out = dst;
        rp.ny = (int)p->ny;
        rp.nx = (int)p->nx;
        rp.ld = (int)p->nx;
        rp.T = nlev;
        rp.periodic = p->boundary == STENCIL_BOUNDARY_PERIODIC;
        rp.rp = p->res_rp;
        rp.pitch = (int)p->nx + 2 * p->R;
        rp.kb = p->res_kb;
        rp.H = p->res_kb * p->R;
        rp.w = p->w;
        CK(launch_resident(p->res_fn, p->res_c, p->res_smem, rp, st));
        return STENCIL_OK;
    }
    if (p->kernel == STENCIL_KERNEL_LOWRANK) {
        CK(launch_lowrank(p->lr_fn, static_cast<const float*>(src), static_cast<float*>(dst), p->ny, p->nx,
                          p->boundary == STENCIL_BOUNDARY_PERIODIC, p->lr_col, p->lr_row, p->sms, st));
        return STENCIL_OK;
    }
    if (p->kernel == STENCIL_KERNEL_NAIVE) {
        dim3 block(32, 8), grid((unsigned)p->strips, (unsigned)p->tiles_y);
        long long ny = p->ny, nx = p->nx;
        int periodic = p->boundary;
        void* args[] = {(void*)&src, (void*)&dst, &ny, &nx, &periodic, &p->w};
        CK(cudaLaunchKernel(p->naive, grid, block, args, 0, st));
        return STENCIL_OK;
    }
    StreamParams sp{};
    sp.in = src;
    sp.out = dst;
    sp.ny = p->ny;
    sp.nx = p->nx;
    sp.ld = p->nx;
    sp.nlev = nlev;
    sp.H = p->H;
    sp.bx = p->bx;
    sp.by = p->by;
    sp.strips = p->strips;
    sp.periodic = p->boundary == STENCIL_BOUNDARY_PERIODIC;
    const size_t vec_bytes = 4 * p->elem;
    sp.vec = (p->nx % 4 == 0) && ((uintptr_t)src % vec_bytes == 0) &&
             ((uintptr_t)dst % vec_bytes == 0);
    sp.w = p->w;
    for (int i = 0; i < kMaxTaps; ++i) sp.w2.w2[i] = make_float2(p->w.w[i], p->w.w[i]);
    sp.status = p->status;
    sp.wait_ns = (long long)(p->opt.timeout_ms > 0 ? p->opt.timeout_ms : 2000) * 1000000LL;
    sp.debug_withhold = p->opt.debug_withhold;
    dim3 grid((unsigned)(p->strips * p->tiles_y)), block((unsigned)p->threads);
    const void* fn = nullptr;
    int smem = 0;
    alignas(64) CUtensorMap map;
    // The TMA-fed kernel when the plan uses it and this source has a tensor
    // map (16-byte aligned); otherwise the cp.async kernel, same arithmetic.
    const int tma = p->tma && sp.vec && stream_tensor_map(&map, src, p->ny, p->nx);
    stencil_status_t s = stream_fn(p, nlev, sp.vec, &fn, &smem, tma, p->threads);
    if (s != STENCIL_OK) return s;
    if (tma) {
        void* args[] = {&map, &sp};
        CK(cudaLaunchKernel(fn, grid, block, args, (size_t)smem, st));
    } else {
        void* args[] = {&sp};
        CK(cudaLaunchKernel(fn, grid, block, args, (size_t)smem, st));
    }
    return STENCIL_OK;
}

// Depths of the launches for T steps: full blocks of k, then the remainder
// split greedily into instantiated depths.
static std::vector<int> launch_depths(const stencil_plan* p, int64_t T) {
    std::vector<int> d;
    if (p->kernel == STENCIL_KERNEL_RESIDENT) {  // the whole run in one launch (chunks of 2^30 steps)
        for (int64_t t = 0; t < T; t += (1 << 30)) d.push_back((int)std::min<int64_t>(T - t, 1 << 30));
        return d;
    }
    const int k = p->kernel == STENCIL_KERNEL_STREAM ? p->k : 1;
    for (int64_t t = 0; t < T / k; ++t) d.push_back(k);
    int rem = (int)(T % k);
    while (rem > 0) {
        const int step = p->kernel == STENCIL_KERNEL_STREAM ? stream_depth_at_most(p->R, p->star, rem) : 1;
        d.push_back(step);
        rem -= step;
    }
    return d;
}

// ---- all states of a run (the adjoint's segment recomputation) ------------------------
//
// outs[i] = u_{i+1} for i < n, from u_0 = in: launches of the all-states
// kernels (depths 8 / 4 / 2 / 1 as available), each reading the last state the
// previous launch wrote and storing every level.  FP32 plans whose rows are
// 16-byte aligned; anything else runs one single-step stencil_run per state.
// Each state is the same bits as stencil_run produces (same arithmetic per
// point, independent of the launch depths).

namespace gbst {
stencil_status_t plan_run_states(stencil_plan_t* p, const void* in, float* const* outs, int64_t n,
                                 cudaStream_t st) {
    bool fused = p->dtype == STENCIL_F32 && p->nx % 4 == 0 && (uintptr_t)in % 16 == 0;
    for (int64_t i = 0; i < n && fused; ++i) fused = (uintptr_t)outs[i] % 16 == 0;
    if (!fused) {
        const void* src = in;
        for (int64_t i = 0; i < n; ++i) {
            stencil_status_t s = stencil_run(p, src, outs[i], 1, st);
            if (s != STENCIL_OK) return s;
            src = outs[i];
        }
        return STENCIL_OK;
    }
    const int threads = 128;
    const void* src = in;
    for (int64_t i = 0; i < n;) {
        int d = 8;
        StreamKernelRef r{nullptr, 0};
        for (; d >= 1; d /= 2) {
            if (d > n - i) continue;
            r = get_stream_states_kernel(p->R, p->star, d);
            if (r.fn) break;
        }
        if (!r.fn) return fail(STENCIL_ERR_UNSUPPORTED, "no all-states kernel");
        const int H = (p->R * d + 3) / 4 * 4;
        const int64_t strips = ceil_div(p->nx, 4 * threads - 2 * H);
        const int bx = (int)(ceil_div(ceil_div(p->nx, strips), 4) * 4);
        const int nt = (int)(ceil_div(ceil_div(bx + 2 * H, 4), 32) * 32);
        const int smem = stream_smem_bytes(p->R, d, 4, true, false, nt);
        const unsigned bit = 1u << d;
        static std::mutex mu;
        {
            std::lock_guard<std::mutex> g(mu);
            static unsigned set_bits[3][2] = {};
            if (!(set_bits[p->R - 1][p->star] & bit)) {
                CK(cudaFuncSetAttribute(r.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        stream_smem_bytes(p->R, d, 4, true, false, kStreamMaxThreads)));
                set_bits[p->R - 1][p->star] |= bit;
            }
        }
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, r.fn, nt, smem));
        if (per_sm < 1) return fail(STENCIL_ERR_UNSUPPORTED, "all-states kernel does not fit on an SM");
        const int64_t want = std::max<int64_t>(1, (int64_t)per_sm * p->sms / strips);
        const int64_t by_min = std::max<int64_t>(8, 4LL * p->R * d);
        int64_t tiles_y = std::max<int64_t>(1, std::min<int64_t>(want, ceil_div(p->ny, by_min)));
        const int by = (int)ceil_div(p->ny, tiles_y);
        tiles_y = ceil_div(p->ny, by);
        StreamParams sp{};
        sp.in = src;
        sp.out = outs[i + d - 1];
        sp.ny = p->ny;
        sp.nx = p->nx;
        sp.ld = p->nx;
        sp.nlev = d;
        sp.H = H;
        sp.bx = bx;
        sp.by = by;
        sp.strips = (int)strips;
        sp.periodic = p->boundary == STENCIL_BOUNDARY_PERIODIC;
        sp.vec = 1;
        sp.status = p->status;
        sp.wait_ns = (long long)(p->opt.timeout_ms > 0 ? p->opt.timeout_ms : 2000) * 1000000LL;
        sp.w = p->w;
        for (int t = 0; t < kMaxTaps; ++t) sp.w2.w2[t] = make_float2(p->w.w[t], p->w.w[t]);
        for (int l = 0; l < d - 1; ++l) sp.lvl_out[l] = outs[i + l];
        void* args[] = {&sp};
        CK(cudaLaunchKernel(r.fn, dim3((unsigned)(strips * tiles_y)), dim3((unsigned)nt), args, (size_t)smem, st));
        src = outs[i + d - 1];
        i += d;
    }
    return STENCIL_OK;
}
}  // namespace gbst

// ---- autotuning ---------------------------------------------------------------------
//
// With opt.autotune, the first stencil_run times every instantiated depth k
// with CTAs of 64, 128 and 256 threads (the depth and CTA size the caller
// fixed, if any, stay fixed) and keeps the fastest per step.  Each candidate
// runs one launch from `in` into the plan's workspace, so neither `in` nor
// `out` is touched.  Results are cached per (shape, radius, footprint, dtype,
// boundary, device) for the life of the process.

typedef std::tuple<int64_t, int64_t, int, int, int, int, int> TuneKey;
static std::map<TuneKey, std::pair<int, int>> g_tune_cache;
static std::mutex g_tune_mu;

static stencil_status_t time_launch(stencil_plan* p, const void* in, int reps, cudaStream_t st,
                                    float* ms) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    stencil_status_t s = launch_once(p, in, p->ws, p->k, st);  // warm-up
    if (s == STENCIL_OK) {
        cudaEventRecord(e0, st);
        for (int i = 0; i < reps && s == STENCIL_OK; ++i) s = launch_once(p, in, p->ws, p->k, st);
        cudaEventRecord(e1, st);
    }
    cudaError_t e = cudaEventSynchronize(e1);
    if (s == STENCIL_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != STENCIL_OK) return s;
    if (e != cudaSuccess) return fail(STENCIL_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
    return STENCIL_OK;
}

// Tensor-core plans: time the warp-MMA engine and every usable tcgen05 MMA
// width (one step per launch, `in` into the workspace) and keep the fastest.
// A plan created with kernel = TC_UMMA, or with mma_n set, keeps that choice.
typedef std::tuple<int64_t, int64_t, int, int, int> TcTuneKey;
static std::map<TcTuneKey, int> g_tc_tune_cache;

static stencil_status_t autotune_tc(stencil_plan* p, const void* in, cudaStream_t st) {
    if (!p->umma_ok || p->opt.kernel == STENCIL_KERNEL_TC_UMMA || p->opt.mma_n > 0) return STENCIL_OK;
    const TcTuneKey key(p->ny, p->nx, p->dtype, p->compute, p->device);
    int best_n = -1;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tc_tune_cache.find(key);
        if (it != g_tc_tune_cache.end()) best_n = it->second;
    }
    if (best_n < 0) {
        const int reps = (int)std::max(2.0, std::min(32.0, 4e9 / ((double)p->ny * (double)p->nx)));
        float best = 1e30f;
        for (int c = 0; c <= 5; ++c) {
            const int nt = c ? kUmmaWidths[c - 1] : 0;
            if (nt && !((p->umma_ok >> (nt / 16)) & 1)) continue;
            p->umma_n = nt;
            cudaEvent_t e0, e1;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            stencil_status_t s = launch_once(p, in, p->ws, 1, st, 0, 1);  // warm-up
            if (s == STENCIL_OK) {
                cudaEventRecord(e0, st);
                for (int i = 0; i < reps && s == STENCIL_OK; ++i) s = launch_once(p, in, p->ws, 1, st, 0, 1);
                cudaEventRecord(e1, st);
            }
            cudaError_t e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (s == STENCIL_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (s != STENCIL_OK) return s;
            if (e != cudaSuccess) return fail(STENCIL_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
            if (ms < best) {
                best = ms;
                best_n = nt;
            }
        }
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tc_tune_cache[key] = best_n;
    }
    p->umma_n = best_n;
    p->kernel = best_n ? STENCIL_KERNEL_TC_UMMA : STENCIL_KERNEL_TC;
    return STENCIL_OK;
}

static stencil_status_t autotune(stencil_plan* p, const void* in, cudaStream_t st) {
    const TuneKey key(p->ny, p->nx, p->R, p->star, p->dtype, p->boundary, p->device);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p->tma = it->second.second >> 16;
            return configure_stream(p, it->second.first, it->second.second & 0xffff, p->opt.tile_rows);
        }
    }
    const int ths[3] = {64, 128, 256};
    float best = 1e30f, def_time = -1.f;
    int bk = p->k, bt = p->threads, btma = p->tma;
    const int k0 = p->k, t0 = p->opt.threads > 0 ? p->opt.threads : default_threads(p->R, p->star), tma0 = p->tma;
    const double points = (double)p->ny * (double)p->nx;
    // Row loads: both the cp.async ring and the TMA-fed ring where the plan
    // allows either (load = AUTO), else the one it fixed.
    const int tma_lo = p->opt.load == STENCIL_LOAD_TMA ? 1 : 0;
    const int tma_hi = (p->opt.load != STENCIL_LOAD_CP_ASYNC && tma_eligible(p)) ? 1 : 0;
    for (int tma = tma_lo; tma <= tma_hi; ++tma) {
        p->tma = tma;
        for (int i = 0; i < 8 && kStreamDepths[p->R - 1][p->star][i]; ++i) {
            const int k = kStreamDepths[p->R - 1][p->star][i];
            if (p->opt.tb_depth > 0 && k != p->opt.tb_depth) continue;
            for (int th : ths) {
                if (p->opt.threads > 0 && th != p->opt.threads) continue;
                if (configure_stream(p, k, th, p->opt.tile_rows) != STENCIL_OK) continue;
                // About 2e9 point-steps of work per candidate, at least one launch.
                const int reps = (int)std::max(1.0, std::min(64.0, 2e9 / (points * k)));
                float ms = 0.f;
                stencil_status_t s = time_launch(p, in, reps, st, &ms);
                if (s != STENCIL_OK) return s;
                const float per_step = ms / (float)(reps * k);
                if (k == k0 && th == t0 && tma == tma0) def_time = per_step;
                if (per_step < best) {
                    best = per_step;
                    bk = k;
                    bt = th;
                    btma = tma;
                }
            }
        }
    }
    // Keep the default configuration unless a candidate beats it by more than
    // 2 %: closer timings are within run-to-run noise, and a stable choice
    // keeps launch counts and profiles reproducible.
    if (def_time > 0.f && def_time <= 1.02f * best) {
        bk = k0;
        bt = t0;
        btma = tma0;
    }
    p->tma = btma;
    stencil_status_t s = configure_stream(p, bk, bt, p->opt.tile_rows);
    if (s != STENCIL_OK) return s;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = std::make_pair(bk, bt | (btma << 16));
    return STENCIL_OK;
}

// Small grids (plans that chose the cluster-resident kernel): time that kernel
// at every usable cluster size (runs of 64 steps from `in` into the workspace)
// and the autotuned streaming kernel, per step, and keep the faster.  The
// decision is cached like the streaming kernel's.
static std::map<TuneKey, int> g_res_tune_cache;  // 16 * kb + log2(C) + 1, or 0 for the streaming kernel

static stencil_status_t autotune_resident(stencil_plan* p, const void* in, cudaStream_t st) {
    const TuneKey key(p->ny, p->nx, p->R, p->star, p->dtype, p->boundary, p->device);
    int decision = -1;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_res_tune_cache.find(key);
        if (it != g_res_tune_cache.end()) decision = it->second;
    }
    if (decision < 0) {
        constexpr int S = 64;
        const int reps = (int)std::max(2.0, std::min(16.0, 1e8 / ((double)p->ny * (double)p->nx * S)));
        float best = 1e30f;
        decision = 0;
        for (int lg = 0; (1 << lg) <= resident_max_cluster(); ++lg) {
            if (!((p->res_ok >> lg) & 1)) continue;
            for (int kb = 1; kb <= 8; kb *= 2) {
                int rp = 0;
                const int periodic = p->boundary == STENCIL_BOUNDARY_PERIODIC;
                if (resident_config((int)p->ny, (int)p->nx, p->R, periodic, 1 << lg, kb, p->res_max_smem, &rp) < 0)
                    continue;
                stencil_status_t s = use_resident(p, 1 << lg, kb);
                if (s != STENCIL_OK) return s;
                cudaEvent_t e0, e1;
                CK(cudaEventCreate(&e0));
                CK(cudaEventCreate(&e1));
                s = launch_once(p, in, p->ws, S, st);  // warm-up
                if (s == STENCIL_OK) {
                    cudaEventRecord(e0, st);
                    for (int i = 0; i < reps && s == STENCIL_OK; ++i) s = launch_once(p, in, p->ws, S, st);
                    cudaEventRecord(e1, st);
                }
                cudaError_t e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (s == STENCIL_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (s != STENCIL_OK) return s;
                if (e != cudaSuccess) return fail(STENCIL_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
                const float per_step = ms / (float)(reps * S);
                if (per_step < best) {
                    best = per_step;
                    decision = 16 * kb + lg + 1;
                }
            }
        }
        stencil_status_t s = autotune(p, in, st);  // configures the best streaming kernel
        if (s != STENCIL_OK) return s;
        const int sreps = (int)std::max(2.0, std::min(64.0, 1e8 / ((double)p->ny * (double)p->nx * p->k)));
        float ms = 0.f;
        s = time_launch(p, in, sreps, st, &ms);
        if (s != STENCIL_OK) return s;
        if (ms / (float)(sreps * p->k) < best) decision = 0;
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_res_tune_cache[key] = decision;
    }
    if (decision > 0) return use_resident(p, 1 << ((decision & 15) - 1), decision >> 4);
    return autotune(p, in, st);
}

extern "C" {

const char* stencil_status_string(stencil_status_t s) {
    switch (s) {
        case STENCIL_OK: return "STENCIL_OK";
        case STENCIL_ERR_INVALID_ARG: return "STENCIL_ERR_INVALID_ARG";
        case STENCIL_ERR_UNSUPPORTED: return "STENCIL_ERR_UNSUPPORTED";
        case STENCIL_ERR_CUDA: return "STENCIL_ERR_CUDA";
        case STENCIL_ERR_OOM: return "STENCIL_ERR_OOM";
        case STENCIL_ERR_TIMEOUT: return "STENCIL_ERR_TIMEOUT";
        case STENCIL_ERR_DEVICE_CHECK: return "STENCIL_ERR_DEVICE_CHECK";
        default: return "STENCIL_ERR_UNKNOWN";
    }
}

const char* stencil_last_error(void) { return g_last_error.c_str(); }

int stencil_version(void) { return 100; }

stencil_status_t stencil_plan_create(stencil_plan_t** out, int64_t ny, int64_t nx, int radius,
                                     const float* weights, int dtype, int boundary,
                                     const stencil_options_t* opt) {
    if (!out) return fail(STENCIL_ERR_INVALID_ARG, "plan pointer is NULL");
    *out = nullptr;
    if (ny < 1 || nx < 1) return fail(STENCIL_ERR_INVALID_ARG, "ny and nx must be >= 1");
    if (radius < 1) return fail(STENCIL_ERR_INVALID_ARG, "radius must be >= 1");
    if (radius > kMaxRadius) return fail(STENCIL_ERR_UNSUPPORTED, "radius > 3 is not supported");
    if (ny > (1LL << 30) || nx > (1LL << 30))
        return fail(STENCIL_ERR_UNSUPPORTED, "ny and nx must be <= 2^30");
    if (!weights) return fail(STENCIL_ERR_INVALID_ARG, "weights pointer is NULL");
    if (dtype < STENCIL_F32 || dtype > STENCIL_F16) return fail(STENCIL_ERR_INVALID_ARG, "bad dtype");
    if (boundary != STENCIL_BOUNDARY_ZERO && boundary != STENCIL_BOUNDARY_PERIODIC)
        return fail(STENCIL_ERR_INVALID_ARG, "bad boundary");
    stencil_options_t o{};
    if (opt) o = *opt;
    if (o.compute < 0 || o.compute > STENCIL_COMPUTE_LOWRANK || o.kernel < 0 ||
        o.kernel > STENCIL_KERNEL_RESIDENT || o.tb_depth < 0 || o.threads < 0 || o.tile_rows < 0 ||
        o.mma_n < 0 || o.timeout_ms < 0 || o.debug_withhold < 0 || o.debug_withhold > 1 ||
        o.load < STENCIL_LOAD_AUTO || o.load > STENCIL_LOAD_TMA || o.rank < 0 || o.rank > 2 * radius + 1)
        return fail(STENCIL_ERR_INVALID_ARG, "bad option value");

    stencil_plan* p = new (std::nothrow) stencil_plan();
    if (!p) return fail(STENCIL_ERR_OOM, "host allocation failed");
    p->ny = ny;
    p->nx = nx;
    p->R = radius;
    p->dtype = dtype;
    p->boundary = boundary;
    p->compute = (o.compute == STENCIL_COMPUTE_TC_TF32 || o.compute == STENCIL_COMPUTE_TC_BF16 ||
                  o.compute == STENCIL_COMPUTE_TC_3XTF32 || o.compute == STENCIL_COMPUTE_LOWRANK)
                     ? o.compute : STENCIL_COMPUTE_FP32;
    p->opt = o;
    p->elem = elem_size(dtype);
    const int D = 2 * radius + 1;
    int star = 1;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            const float v = weights[a * D + b];
            if (!std::isfinite(v)) {
                delete p;
                return fail(STENCIL_ERR_INVALID_ARG, "weights must be finite");
            }
            p->w.w[a * D + b] = v;
            if (a != radius && b != radius && v != 0.f) star = 0;
        }
    p->star = star;

    auto bail = [&](stencil_status_t st) {
        stencil_plan_destroy(p);
        return st;
    };
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return fail(STENCIL_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return fail(STENCIL_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    }

    stencil_status_t st;
    const bool tc_kernel = o.kernel == STENCIL_KERNEL_TC || o.kernel == STENCIL_KERNEL_TC_WARP ||
                           o.kernel == STENCIL_KERNEL_TC_UMMA;
    if (p->compute == STENCIL_COMPUTE_LOWRANK) {
        st = configure_lowrank(p);
    } else if (p->compute != STENCIL_COMPUTE_FP32 || tc_kernel) {
        if (p->compute == STENCIL_COMPUTE_FP32) p->compute = STENCIL_COMPUTE_TC_TF32;
        st = configure_tc(p);
    } else if (o.kernel == STENCIL_KERNEL_NAIVE) {
        st = configure_naive(p);
    } else {
        const int k = o.tb_depth > 0 ? o.tb_depth : default_depth(radius, star);
        const int threads = o.threads > 0 ? o.threads : default_threads(radius, star);
        if (o.load == STENCIL_LOAD_TMA && !tma_eligible(p))
            return bail(fail(STENCIL_ERR_UNSUPPORTED,
                             "TMA-fed rows need FP32 storage, the zero rule and nx a multiple of 4"));
        const int k0 = std::min(k, stream_kmax(radius, star));
        p->tma = o.load == STENCIL_LOAD_TMA || (o.load == STENCIL_LOAD_AUTO && tma_eligible(p) && kDefaultTma);
        st = configure_stream(p, k0, threads, o.tile_rows);
        // Small grids: the cluster-resident kernel, unless the caller asked for
        // the streaming kernel or set one of its options.
        // With kernel = RESIDENT, tb_depth is its number of steps per halo exchange.
        const bool stream_opts = o.tb_depth > 0 || o.threads > 0 || o.tile_rows > 0;
        if (st == STENCIL_OK && (o.kernel == STENCIL_KERNEL_RESIDENT ||
                                 (o.kernel == STENCIL_KERNEL_AUTO && !stream_opts))) {
            const int kb = (o.kernel == STENCIL_KERNEL_RESIDENT && o.tb_depth > 0) ? o.tb_depth : 1;
            const int C = resident_candidates(p, kb);
            if (C > 0)
                st = use_resident(p, C, kb);
            else if (o.kernel == STENCIL_KERNEL_RESIDENT)
                st = fail(STENCIL_ERR_UNSUPPORTED, "grid too large for the cluster-resident kernel at this depth");
        }
    }
    if (st != STENCIL_OK) return bail(st);

    const size_t bytes = (size_t)ny * (size_t)nx * p->elem;
    e = cudaMalloc(&p->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        p->ws = nullptr;
        bail(STENCIL_ERR_OOM);
        return fail(STENCIL_ERR_OOM, "cudaMalloc of the workspace failed");
    }
    e = cudaMalloc(&p->status, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(p->status, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        bail(STENCIL_ERR_OOM);
        return fail(STENCIL_ERR_OOM, "cudaMalloc of the status word failed");
    }
    *out = p;
    return STENCIL_OK;
}

void stencil_plan_destroy(stencil_plan_t* p) {
    if (!p) return;
    for (int i = 0; i < 4; ++i)
        if (p->aux[i] && p->aux_free[i]) p->aux_free[i](p->aux[i]);
    if (p->ws) cudaFree(p->ws);
    if (p->host_in) cudaFree(p->host_in);
    if (p->host_out) cudaFree(p->host_out);
    if (p->status) cudaFree(p->status);
    delete p;
}

stencil_status_t stencil_plan_set_weights(stencil_plan_t* p, const float* weights) {
    if (!p || !weights) return fail(STENCIL_ERR_INVALID_ARG, "NULL argument");
    const int R = p->R, D = 2 * R + 1;
    int star = 1;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            const float v = weights[a * D + b];
            if (!std::isfinite(v)) return fail(STENCIL_ERR_INVALID_ARG, "weights must be finite");
            if (a != R && b != R && v != 0.f) star = 0;
        }
    const bool footprint_bound = p->kernel == STENCIL_KERNEL_STREAM || p->kernel == STENCIL_KERNEL_RESIDENT;
    if (footprint_bound && star != p->star)
        return fail(STENCIL_ERR_UNSUPPORTED,
                    "the new weights change the footprint (star / box) the plan's kernel was chosen for");
    if (p->kernel == STENCIL_KERNEL_LOWRANK) {
        float col[7][7], row[7][7];
        int rho = lowrank_factor(weights, R, p->opt.rank, col, row, nullptr);
        if (rho < 1) rho = 1;
        const void* fn = get_lowrank_kernel(R, rho);
        if (!fn) return fail(STENCIL_ERR_UNSUPPORTED, "no low-rank kernel for this rank");
        p->lr_rank = rho;
        p->lr_fn = fn;
        std::memcpy(p->lr_col, col, sizeof(col));
        std::memcpy(p->lr_row, row, sizeof(row));
    }
    for (int i = 0; i < D * D; ++i) p->w.w[i] = weights[i];
    if (!footprint_bound) p->star = star;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_info(const stencil_plan_t* p, stencil_plan_info_t* info) {
    if (!p || !info) return fail(STENCIL_ERR_INVALID_ARG, "NULL argument");
    stencil_plan_info_t i{};
    i.ny = p->ny;
    i.nx = p->nx;
    i.radius = p->R;
    i.shape = p->star;
    i.dtype = p->dtype;
    i.boundary = p->boundary;
    i.compute = p->compute;
    i.kernel = p->kernel;
    i.tb_depth = p->k;
    i.threads = p->threads;
    i.halo_cols = p->H;
    i.tile_cols = p->bx;
    i.tile_rows = p->by;
    i.ctas = p->strips * p->tiles_y;
    i.smem_bytes = p->smem;
    i.workspace_bytes = (int64_t)((size_t)p->ny * p->nx * p->elem);
    i.mma_n = p->umma_n;
    i.load = p->kernel == STENCIL_KERNEL_STREAM ? (p->tma ? STENCIL_LOAD_TMA : STENCIL_LOAD_CP_ASYNC) : 0;
    i.rank = p->kernel == STENCIL_KERNEL_LOWRANK ? p->lr_rank : 0;
    if (p->kernel == STENCIL_KERNEL_RESIDENT) {
        i.tb_depth = 0;  // every step of a run in one launch
        i.threads = resident_threads();
        i.halo_cols = p->R;
        i.tile_cols = (int)p->nx;
        i.tile_rows = p->res_rp;
        i.ctas = p->res_c;
        i.smem_bytes = p->res_smem;
    }
    if (p->umma_n) {
        i.threads = box49_umma_threads(p->umma_n);
        i.ctas = p->umma_ctas;
        i.smem_bytes = box49_umma_smem_bytes(p->compute == STENCIL_COMPUTE_TC_TF32, p->umma_n);
        i.tile_rows = box49_umma_tile_rows(p->umma_n);
    }
    *info = i;
    return STENCIL_OK;
}

int64_t stencil_run_launches(const stencil_plan_t* p, int64_t T) {
    if (!p || T < 0) return -1;
    return (int64_t)launch_depths(p, T).size();
}

stencil_status_t stencil_run(stencil_plan_t* p, const void* in, void* out, int64_t T,
                             stencil_stream_t stream) {
    if (!p) return fail(STENCIL_ERR_INVALID_ARG, "plan is NULL");
    if (!in || !out) return fail(STENCIL_ERR_INVALID_ARG, "in/out is NULL");
    if (T < 0) return fail(STENCIL_ERR_INVALID_ARG, "T must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    p->last_stream = st;
    const size_t bytes = (size_t)p->ny * p->nx * p->elem;
    if (p->opt.autotune && !p->tuned && T > 0 &&
        (p->kernel == STENCIL_KERNEL_TC || p->kernel == STENCIL_KERNEL_TC_UMMA)) {
        stencil_status_t s = autotune_tc(p, in, st);
        if (s != STENCIL_OK) return s;
        p->tuned = 1;
    }
    if (p->opt.autotune && !p->tuned && p->kernel == STENCIL_KERNEL_RESIDENT && T > 0) {
        stencil_status_t s = autotune_resident(p, in, st);
        if (s != STENCIL_OK) return s;
        p->tuned = 1;
    }
    if (p->opt.autotune && !p->tuned && p->kernel == STENCIL_KERNEL_STREAM && T > 0) {
        stencil_status_t s = autotune(p, in, st);
        if (s != STENCIL_OK) return s;
        p->tuned = 1;
    }
    if (T == 0) {
        if (in != out) CK(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st));
        return STENCIL_OK;
    }
    std::vector<int> depths = launch_depths(p, T);
    const void* src = in;
    if (p->kernel == STENCIL_KERNEL_RESIDENT) {
        // one launch reads all of its input before it writes any output
        for (size_t i = 0; i < depths.size(); ++i) {
            stencil_status_t s = launch_once(p, src, out, depths[i], st);
            if (s != STENCIL_OK) return s;
            src = out;
        }
        return STENCIL_OK;
    }
    if (in == out && depths.size() % 2 == 1) {
        // An odd launch count would make launch 1 write the grid it reads.
        // Split one launch in two when possible, else stage the input.
        auto it = std::find_if(depths.begin(), depths.end(), [](int d) { return d >= 2; });
        if (it != depths.end()) {
            const int d = *it;
            *it = d / 2;
            depths.insert(it, d - d / 2);
        } else {
            CK(cudaMemcpyAsync(p->ws, in, bytes, cudaMemcpyDeviceToDevice, st));
            src = p->ws;
        }
    }
    const size_t L = depths.size();
    for (size_t i = 0; i < L; ++i) {
        // Launch i (0-based) writes `out` when L-1-i is even, else the workspace.
        void* dst = ((L - 1 - i) % 2 == 0) ? out : p->ws;
        stencil_status_t s = launch_once(p, src, dst, depths[i], st, i == 0, i + 1 == L);
        if (s != STENCIL_OK) return s;
        src = dst;
    }
    return STENCIL_OK;
}

stencil_status_t stencil_run_host_async(stencil_plan_t* p, const void* in_host, void* out_host,
                                        int64_t T, stencil_stream_t stream) {
    if (!p) return fail(STENCIL_ERR_INVALID_ARG, "plan is NULL");
    if (!in_host || !out_host) return fail(STENCIL_ERR_INVALID_ARG, "in/out is NULL");
    if (T < 0) return fail(STENCIL_ERR_INVALID_ARG, "T must be >= 0");
    const size_t bytes = (size_t)p->ny * p->nx * p->elem;
    if (!p->host_in) {
        if (cudaMalloc(&p->host_in, bytes) != cudaSuccess) {
            cudaGetLastError();
            p->host_in = nullptr;
            return fail(STENCIL_ERR_OOM, "cudaMalloc of the staging input failed");
        }
    }
    if (!p->host_out) {
        if (cudaMalloc(&p->host_out, bytes) != cudaSuccess) {
            cudaGetLastError();
            p->host_out = nullptr;
            return fail(STENCIL_ERR_OOM, "cudaMalloc of the staging output failed");
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(p->host_in, in_host, bytes, cudaMemcpyHostToDevice, st));
    stencil_status_t s = stencil_run(p, p->host_in, p->host_out, T, stream);
    if (s != STENCIL_OK) return s;
    CK(cudaMemcpyAsync(out_host, p->host_out, bytes, cudaMemcpyDeviceToHost, st));
    return STENCIL_OK;
}

stencil_status_t stencil_run_host(stencil_plan_t* p, const void* in_host, void* out_host,
                                  int64_t T, stencil_stream_t stream) {
    stencil_status_t s = stencil_run_host_async(p, in_host, out_host, T, stream);
    if (s != STENCIL_OK) return s;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return STENCIL_OK;
}

stencil_status_t stencil_plan_status(stencil_plan_t* p) {
    if (!p) return fail(STENCIL_ERR_INVALID_ARG, "plan is NULL");
    CK(cudaStreamSynchronize(p->last_stream));
    unsigned int word = 0;
    CK(cudaMemcpy(&word, p->status, sizeof(word), cudaMemcpyDeviceToHost));
    CK(cudaMemset(p->status, 0, sizeof(word)));
    if (word == 0) return STENCIL_OK;
    return word == STENCIL_ERR_TIMEOUT ? STENCIL_ERR_TIMEOUT : STENCIL_ERR_DEVICE_CHECK;
}

}  // extern "C"
