// shapes_t32.cu -- team-width variants: shapes whose default team is 8 or 16
// lanes, compiled again with a warp per subproblem, for the autotuner to choose
// between: 6,3,3 12,6,6
#define MHE_TEAM 32
#include "kernels.cuh"

namespace mhe {

int shapes_t32(ShapeEntry* out, int cap)
{
    int k = 0;
    if (k < cap) out[k++] = make_shape<6, 3, 3>();
    if (k < cap) out[k++] = make_shape<12, 6, 6>();
    return k;
}

}  // namespace mhe
