// shapes_big.cu -- compiled (nx, nw, ny) shapes: 24,12,12
#include "kernels.cuh"

namespace mhe {

int shapes_big(ShapeEntry* out, int cap)
{
    int k = 0;
    if (k < cap) out[k++] = make_shape<24, 12, 12>();
    return k;
}

}  // namespace mhe
