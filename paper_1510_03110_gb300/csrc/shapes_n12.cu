// shapes_n12.cu -- compiled (nx, nw, ny) shapes with 16-lane teams (two
// subproblems per warp): 12,6,6
#define MHE_TEAM 16
#include "kernels.cuh"

namespace mhe {

int shapes_n12(ShapeEntry* out, int cap)
{
    int k = 0;
    if (k < cap) out[k++] = make_shape<12, 6, 6>();
    return k;
}

}  // namespace mhe
