// sweep_stream_r3.cu -- streaming-kernel instantiations for radius 3.
#include "sweep_stream_inst.cuh"

namespace gbst {

// Smallest instantiated KMAX >= kmin for this radius (kmin <= the largest).
StreamKernelRef get_stream_kernel_r3(int star, int kmin, int dtype) {
    if (kmin <= 1) return pick_shape<3, 1>(star, dtype);
    if (kmin <= 2) return pick_shape<3, 2>(star, dtype);
    if (kmin <= 4) return pick_shape<3, 4>(star, dtype);
    return {nullptr, 0};
}

int stream_kmax_r3() { return 4; }

}  // namespace gbst
