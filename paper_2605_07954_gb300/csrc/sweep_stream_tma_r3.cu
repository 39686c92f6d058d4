// sweep_stream_tma_r3.cu -- TMA-fed streaming-kernel instantiations: radius 3, f32 storage.
#include "sweep_stream.cuh"

namespace gbst {

// TMA-fed kernel advancing exactly k steps per launch ({nullptr, 0} if not instantiated).
StreamKernelRef get_stream_tma_kernel_r3(int star, int k) {
    if (star) {
        switch (k) {
            case 1: return {(const void*)sweep_stream_tma_kernel<3, true, 1>, 1};
            case 2: return {(const void*)sweep_stream_tma_kernel<3, true, 2>, 2};
            case 3: return {(const void*)sweep_stream_tma_kernel<3, true, 3>, 3};
            case 4: return {(const void*)sweep_stream_tma_kernel<3, true, 4>, 4};
            default: return {nullptr, 0};
        }
    }
    switch (k) {
        case 1: return {(const void*)sweep_stream_tma_kernel<3, false, 1>, 1};
        case 2: return {(const void*)sweep_stream_tma_kernel<3, false, 2>, 2};
        default: return {nullptr, 0};
    }
}

}  // namespace gbst
