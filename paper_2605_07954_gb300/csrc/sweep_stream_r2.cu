// sweep_stream_r2.cu -- streaming-kernel instantiations for radius 2.
#include "sweep_stream_inst.cuh"

namespace gbst {

// Smallest instantiated KMAX >= kmin for this radius (kmin <= the largest).
StreamKernelRef get_stream_kernel_r2(int star, int kmin, int dtype) {
    if (kmin <= 1) return pick_shape<2, 1>(star, dtype);
    if (kmin <= 2) return pick_shape<2, 2>(star, dtype);
    if (kmin <= 4) return pick_shape<2, 4>(star, dtype);
    return {nullptr, 0};
}

int stream_kmax_r2() { return 4; }

}  // namespace gbst
