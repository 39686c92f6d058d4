// sweep_stream_tma_r1.cu -- TMA-fed streaming-kernel instantiations: radius 1, f32 storage.
#include "sweep_stream.cuh"

namespace gbst {

// TMA-fed kernel advancing exactly k steps per launch ({nullptr, 0} if not instantiated).
StreamKernelRef get_stream_tma_kernel_r1(int star, int k) {
    if (star) {
        switch (k) {
            case 1: return {(const void*)sweep_stream_tma_kernel<1, true, 1>, 1};
            case 2: return {(const void*)sweep_stream_tma_kernel<1, true, 2>, 2};
            case 3: return {(const void*)sweep_stream_tma_kernel<1, true, 3>, 3};
            case 4: return {(const void*)sweep_stream_tma_kernel<1, true, 4>, 4};
            case 6: return {(const void*)sweep_stream_tma_kernel<1, true, 6>, 6};
            case 8: return {(const void*)sweep_stream_tma_kernel<1, true, 8>, 8};
            default: return {nullptr, 0};
        }
    }
    switch (k) {
        case 1: return {(const void*)sweep_stream_tma_kernel<1, false, 1>, 1};
        case 2: return {(const void*)sweep_stream_tma_kernel<1, false, 2>, 2};
        case 3: return {(const void*)sweep_stream_tma_kernel<1, false, 3>, 3};
        case 4: return {(const void*)sweep_stream_tma_kernel<1, false, 4>, 4};
        case 6: return {(const void*)sweep_stream_tma_kernel<1, false, 6>, 6};
        case 8: return {(const void*)sweep_stream_tma_kernel<1, false, 8>, 8};
        default: return {nullptr, 0};
    }
}

}  // namespace gbst
