// common.cuh -- definitions shared by the sm_103a kernels and the host plan code.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbst {

constexpr int kMaxRadius = 3;
constexpr int kMaxTaps = (2 * kMaxRadius + 1) * (2 * kMaxRadius + 1);

enum Dtype { DT_F32 = 0, DT_BF16 = 1, DT_F16 = 2 };

// Weight set passed by value as a kernel parameter (lives in the constant bank,
// so FMAs take it as an operand).  w[(dy+R)*(2R+1) + (dx+R)] multiplies
// u[i+dy][j+dx] (cross-correlation, Sec. II-C).
struct Weights {
    float w[kMaxTaps];
};

// The same weights duplicated into (w, w) pairs for the packed FP32x2 FMAs.  A
// packed FMA takes its pair from registers: the kernels keep the pairs they use
// often there and read them from here once (footprints with too many weights
// for that use scalar FMAs on the single weights instead).
struct WeightPairs {
    float2 w2[kMaxTaps];
};

// Parameters of the row-streaming kernel (see sweep_stream.cuh).
struct StreamParams {
    const void* in;
    void* out;
    long long ny, nx;
    long long ld;   // row pitch of in and out, in elements (>= nx; a multiple of 4 when vec)
    int nlev;      // time levels (Jacobi steps) this launch advances, 1..KMAX
    int H;         // halo columns loaded on each side of a strip (multiple of 4, >= R*nlev)
    int bx;        // output columns per strip (multiple of 4)
    int by;        // output rows per tile
    int strips;    // strips along x; blockIdx.x = strip + strips * row_tile
    int periodic;  // 1: wrap indices; 0: zero outside the grid
    int vec;       // 1: rows 16-byte aligned for 4-element vector access
    unsigned* status;   // TMA-fed kernels: device status word (bounded waits), else unused
    long long wait_ns;  // TMA-fed kernels: limit of each wait for a row
    int debug_withhold; // TMA-fed kernels, test hook: CTA 0 expects 16 bytes its first row never brings
    void* lvl_out[8];   // all-states kernels: time level l+1 (l < nlev-1) is also stored to lvl_out[l]
    Weights w;
    WeightPairs w2;
};

// Parameters of the cluster-resident kernel (see sweep_resident.cu).
struct ResidentParams {
    const void* in;
    void* out;
    int ny, nx, ld;
    int T;         // steps of this launch, >= 1
    int periodic;  // 1: wrap; 0: zero outside the grid
    int rp;        // slab rows per CTA
    int pitch;     // floats per staged row (nx + 2R)
    int kb;        // steps per halo exchange (temporal blocking depth)
    int H;         // staged halo rows on each side (kb * R)
    Weights w;
};

// ---- storage <-> FP32 ---------------------------------------------------------------

template <typename TS> struct Storage;

template <> struct Storage<float> {
    static __device__ __forceinline__ float4 load4(const float* p) {
        return __ldg(reinterpret_cast<const float4*>(p));
    }
    static __device__ __forceinline__ float load1(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void store4(float* p, float4 v) {
        *reinterpret_cast<float4*>(p) = v;
    }
    static __device__ __forceinline__ void store1(float* p, float v) { *p = v; }
};

template <> struct Storage<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load4(const __nv_bfloat16* p) {
        uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
        __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&raw.x);
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&raw.y);
        float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ float load1(const __nv_bfloat16* p) {
        return __bfloat162float(p[0]);
    }
    static __device__ __forceinline__ void store4(__nv_bfloat16* p, float4 v) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
        __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
        uint2 raw;
        raw.x = *reinterpret_cast<uint32_t*>(&a);
        raw.y = *reinterpret_cast<uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = raw;
    }
    static __device__ __forceinline__ void store1(__nv_bfloat16* p, float v) {
        *p = __float2bfloat16_rn(v);
    }
};

template <> struct Storage<__half> {
    static __device__ __forceinline__ float4 load4(const __half* p) {
        uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
        __half2 a = *reinterpret_cast<__half2*>(&raw.x);
        __half2 b = *reinterpret_cast<__half2*>(&raw.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ float load1(const __half* p) { return __half2float(p[0]); }
    static __device__ __forceinline__ void store4(__half* p, float4 v) {
        __half2 a = __floats2half2_rn(v.x, v.y);
        __half2 b = __floats2half2_rn(v.z, v.w);
        uint2 raw;
        raw.x = *reinterpret_cast<uint32_t*>(&a);
        raw.y = *reinterpret_cast<uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = raw;
    }
    static __device__ __forceinline__ void store1(__half* p, float v) { *p = __float2half_rn(v); }
};

__device__ __forceinline__ long long wrap_index(long long i, long long n) {
    long long m = i % n;
    return m < 0 ? m + n : m;
}

__device__ __forceinline__ float f4get(const float4& v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

}  // namespace gbst
