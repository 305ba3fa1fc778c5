// shapes_xl.cu -- compiled (nx, nw, ny) shapes whose subproblems take a team of
// four warps (128 threads): 64,32,32.  A subproblem's FP32 workspace is
// ~168 KB of shared memory (one per SM), so one warp per subproblem would leave
// the SM nearly idle; the team shares each stage's products four times wider.
// Their FP64 workspace does not fit an SM: these shapes run in MHE_FP32_IR.
#define MHE_TEAM 128
#include "kernels.cuh"

namespace mhe {

int shapes_xl(ShapeEntry* out, int cap)
{
    int k = 0;
    if (k < cap) out[k++] = make_shape<64, 32, 32>();
    return k;
}

}  // namespace mhe
