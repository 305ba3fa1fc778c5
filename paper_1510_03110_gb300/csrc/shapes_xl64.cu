// shapes_xl64.cu -- the FP64 passes of the shapes of shapes_xl.cu (64,32,32) in a
// translation unit of their own, compiled in parallel with it.  Their reduction
// workspace (about 342 KB per subproblem in FP64) exceeds an SM's shared memory,
// so the reduction keeps it in global memory (L2-resident); the right-hand-side
// and down passes fit in shared memory.
#define MHE_TEAM 128
#include "kernels.cuh"

namespace mhe {

void shapes_xl_fp64(ShapeOps& o)
{
    set_fp64_global_ops<64, 32>(o);
}

}  // namespace mhe
