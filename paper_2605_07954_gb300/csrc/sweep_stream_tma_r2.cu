// sweep_stream_tma_r2.cu -- TMA-fed streaming-kernel instantiations: radius 2, f32 storage.
#include "sweep_stream.cuh"

namespace gbst {

// TMA-fed kernel advancing exactly k steps per launch ({nullptr, 0} if not instantiated).
StreamKernelRef get_stream_tma_kernel_r2(int star, int k) {
    switch (k) {
        case 1: return star ? StreamKernelRef{(const void*)sweep_stream_tma_kernel<2, true, 1>, 1}
                            : StreamKernelRef{(const void*)sweep_stream_tma_kernel<2, false, 1>, 1};
        case 2: return star ? StreamKernelRef{(const void*)sweep_stream_tma_kernel<2, true, 2>, 2}
                            : StreamKernelRef{(const void*)sweep_stream_tma_kernel<2, false, 2>, 2};
        case 4: return star ? StreamKernelRef{(const void*)sweep_stream_tma_kernel<2, true, 4>, 4}
                            : StreamKernelRef{(const void*)sweep_stream_tma_kernel<2, false, 4>, 4};
        default: return {nullptr, 0};
    }
}

}  // namespace gbst
