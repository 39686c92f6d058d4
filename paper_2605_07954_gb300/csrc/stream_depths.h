// stream_depths.h -- depths instantiated for the streaming kernel (generated with the
// sweep_stream_r*_*.cu files).
#pragma once

namespace gbst {

// Instantiated depths, ascending, 0-terminated: [radius-1][star].
static const int kStreamDepths[3][2][8] = {
    {{1, 2, 3, 4, 6, 8, 0, 0}, {1, 2, 3, 4, 6, 8, 0, 0}},
    {{1, 2, 4, 0, 0, 0, 0, 0}, {1, 2, 4, 0, 0, 0, 0, 0}},
    {{1, 2, 0, 0, 0, 0, 0, 0}, {1, 2, 3, 4, 0, 0, 0, 0}},
};

}  // namespace gbst
