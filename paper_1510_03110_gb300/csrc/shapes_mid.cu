// shapes_mid.cu -- compiled (nx, nw, ny) shapes: 20,10,10
#include "kernels.cuh"

namespace mhe {

int shapes_mid(ShapeEntry* out, int cap)
{
    int k = 0;
    if (k < cap) out[k++] = make_shape<20, 10, 10>();
    return k;
}

}  // namespace mhe
