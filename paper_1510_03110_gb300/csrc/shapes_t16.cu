// shapes_t16.cu -- team-width variants: shapes whose default team is 8 lanes,
// compiled again with 16-lane teams (two subproblems per warp), for the
// autotuner to choose between: 4,2,2 6,3,3
#define MHE_TEAM 16
#include "kernels.cuh"

namespace mhe {

int shapes_t16(ShapeEntry* out, int cap)
{
    int k = 0;
    if (k < cap) out[k++] = make_shape<4, 2, 2>();
    if (k < cap) out[k++] = make_shape<6, 3, 3>();
    return k;
}

}  // namespace mhe
