// sweep_stream_states.cu -- all-states streaming kernels (FP32 storage, rows
// 16-byte aligned): every time level of a launch is written out, for the
// adjoint's recomputation of the states of a checkpoint segment.
#include "sweep_stream.cuh"

namespace gbst {

template <int R, bool STAR, int K>
static StreamKernelRef states_ref() {
    return {(const void*)sweep_stream_kernel<R, STAR, K, float, true, true>, K};
}

// All-states kernel advancing exactly k steps ({nullptr, 0} if not instantiated):
// k in {1, 2, 4, 8} for radius 1, {1, 2, 4} for radius 2 and the 13-point star,
// {1, 2} for the 7x7 box.
StreamKernelRef get_stream_states_kernel(int R, int star, int k) {
    switch (R) {
        case 1:
            switch (k) {
                case 1: return star ? states_ref<1, true, 1>() : states_ref<1, false, 1>();
                case 2: return star ? states_ref<1, true, 2>() : states_ref<1, false, 2>();
                case 4: return star ? states_ref<1, true, 4>() : states_ref<1, false, 4>();
                case 8: return star ? states_ref<1, true, 8>() : states_ref<1, false, 8>();
                default: return {nullptr, 0};
            }
        case 2:
            switch (k) {
                case 1: return star ? states_ref<2, true, 1>() : states_ref<2, false, 1>();
                case 2: return star ? states_ref<2, true, 2>() : states_ref<2, false, 2>();
                case 4: return star ? states_ref<2, true, 4>() : states_ref<2, false, 4>();
                default: return {nullptr, 0};
            }
        case 3:
            switch (k) {
                case 1: return star ? states_ref<3, true, 1>() : states_ref<3, false, 1>();
                case 2: return star ? states_ref<3, true, 2>() : states_ref<3, false, 2>();
                case 4: return star ? states_ref<3, true, 4>() : StreamKernelRef{nullptr, 0};
                default: return {nullptr, 0};
            }
        default: return {nullptr, 0};
    }
}

}  // namespace gbst
