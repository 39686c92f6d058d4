// sweep_stream_r1_bf16.cu -- streaming-kernel instantiations: radius 1, bf16 storage.
#include "sweep_stream_inst.cuh"

namespace gbst {

// Kernel advancing exactly k steps per launch ({nullptr, 0} if not instantiated).
StreamKernelRef get_stream_kernel_r1_bf16(int star, int k, int vec) {
    if (star) {
        switch (k) {
            case 1: return pick_vec<1, true, 1, __nv_bfloat16>(vec);
            case 2: return pick_vec<1, true, 2, __nv_bfloat16>(vec);
            case 3: return pick_vec<1, true, 3, __nv_bfloat16>(vec);
            case 4: return pick_vec<1, true, 4, __nv_bfloat16>(vec);
            case 6: return pick_vec<1, true, 6, __nv_bfloat16>(vec);
            case 8: return pick_vec<1, true, 8, __nv_bfloat16>(vec);
            default: return {nullptr, 0};
        }
    }
    switch (k) {
        case 1: return pick_vec<1, false, 1, __nv_bfloat16>(vec);
        case 2: return pick_vec<1, false, 2, __nv_bfloat16>(vec);
        case 3: return pick_vec<1, false, 3, __nv_bfloat16>(vec);
        case 4: return pick_vec<1, false, 4, __nv_bfloat16>(vec);
        case 6: return pick_vec<1, false, 6, __nv_bfloat16>(vec);
        case 8: return pick_vec<1, false, 8, __nv_bfloat16>(vec);
        default: return {nullptr, 0};
    }
}

}  // namespace gbst
