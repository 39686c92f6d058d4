// sweep_stream_inst.cuh -- instantiates the streaming kernel for one radius.
// Included by sweep_stream_r{1,2,3}.cu with STREAM_R and STREAM_KMAX_LIST set.
#pragma once
#include "sweep_stream.cuh"

namespace gbst {

template <int R, bool STAR, int KMAX>
static StreamKernelRef pick_dtype(int dtype) {
    switch (dtype) {
        case DT_F32: return {(const void*)sweep_stream_kernel<R, STAR, KMAX, float>, KMAX};
        case DT_BF16: return {(const void*)sweep_stream_kernel<R, STAR, KMAX, __nv_bfloat16>, KMAX};
        case DT_F16: return {(const void*)sweep_stream_kernel<R, STAR, KMAX, __half>, KMAX};
        default: return {nullptr, 0};
    }
}

template <int R, int KMAX>
static StreamKernelRef pick_shape(int star, int dtype) {
    return star ? pick_dtype<R, true, KMAX>(dtype) : pick_dtype<R, false, KMAX>(dtype);
}

}  // namespace gbst
