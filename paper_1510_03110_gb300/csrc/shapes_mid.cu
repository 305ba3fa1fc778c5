// shapes_mid.cu -- compiled (nx, nw, ny) shapes: 12,6,6 20,10,10
#include "kernels.cuh"

namespace mhe {

int shapes_mid(ShapeEntry* out, int cap)
{
    int k = 0;
    if (k < cap) out[k++] = make_shape<12, 6, 6>();
    if (k < cap) out[k++] = make_shape<20, 10, 10>();
    return k;
}

}  // namespace mhe
