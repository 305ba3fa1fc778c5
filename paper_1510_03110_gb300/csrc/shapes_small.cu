// shapes_small.cu -- compiled (nx, nw, ny) shapes with 8-lane teams (four
// subproblems per warp; their products have at most 36 outputs):
// 1,1,1 2,1,1 3,2,2 4,2,2 6,3,3
#define MHE_TEAM 8
#include "kernels.cuh"

namespace mhe {

int shapes_small(ShapeEntry* out, int cap)
{
    int k = 0;
    if (k < cap) out[k++] = make_shape<1, 1, 1>();
    if (k < cap) out[k++] = make_shape<2, 1, 1>();
    if (k < cap) out[k++] = make_shape<3, 2, 2>();
    if (k < cap) out[k++] = make_shape<4, 2, 2>();
    if (k < cap) out[k++] = make_shape<6, 3, 3>();
    return k;
}

}  // namespace mhe
