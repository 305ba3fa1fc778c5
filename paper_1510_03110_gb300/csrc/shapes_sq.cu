// shapes_sq.cu -- compiled (nx, nw, ny) shapes: 20,20,20
#include "kernels.cuh"

namespace mhe {

int shapes_sq(ShapeEntry* out, int cap)
{
    int k = 0;
    if (k < cap) out[k++] = make_shape<20, 20, 20>();
    return k;
}

}  // namespace mhe
