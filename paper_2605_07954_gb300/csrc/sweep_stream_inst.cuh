// sweep_stream_inst.cuh -- helpers to instantiate the streaming kernel.
#pragma once
#include "sweep_stream.cuh"

namespace gbst {

template <int R, bool STAR, int K, typename TS>
static StreamKernelRef pick_vec(int vec) {
    return vec ? StreamKernelRef{(const void*)sweep_stream_kernel<R, STAR, K, TS, true>, K}
               : StreamKernelRef{(const void*)sweep_stream_kernel<R, STAR, K, TS, false>, K};
}

}  // namespace gbst
