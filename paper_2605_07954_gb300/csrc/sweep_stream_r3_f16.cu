// sweep_stream_r3_f16.cu -- streaming-kernel instantiations: radius 3, f16 storage.
#include "sweep_stream_inst.cuh"

namespace gbst {

// Kernel advancing exactly k steps per launch ({nullptr, 0} if not instantiated).
StreamKernelRef get_stream_kernel_r3_f16(int star, int k, int vec) {
    if (star) {
        switch (k) {
            case 1: return pick_vec<3, true, 1, __half>(vec);
            case 2: return pick_vec<3, true, 2, __half>(vec);
            case 3: return pick_vec<3, true, 3, __half>(vec);
            case 4: return pick_vec<3, true, 4, __half>(vec);
            default: return {nullptr, 0};
        }
    }
    switch (k) {
        case 1: return pick_vec<3, false, 1, __half>(vec);
        case 2: return pick_vec<3, false, 2, __half>(vec);
        default: return {nullptr, 0};
    }
}

}  // namespace gbst
