// sweep_stream_r1.cu -- streaming-kernel instantiations for radius 1.
#include "sweep_stream_inst.cuh"

namespace gbst {

// Smallest instantiated KMAX >= kmin for this radius (kmin <= the largest).
StreamKernelRef get_stream_kernel_r1(int star, int kmin, int dtype) {
    if (kmin <= 1) return pick_shape<1, 1>(star, dtype);
    if (kmin <= 2) return pick_shape<1, 2>(star, dtype);
    if (kmin <= 4) return pick_shape<1, 4>(star, dtype);
    if (kmin <= 8) return pick_shape<1, 8>(star, dtype);
    return {nullptr, 0};
}

int stream_kmax_r1() { return 8; }

}  // namespace gbst
