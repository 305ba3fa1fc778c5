// shapes_xl.cu -- compiled (nx, nw, ny) shapes whose subproblems take a team of
// four warps (128 threads): 64,32,32.  A subproblem's FP32 workspace is
// ~168 KB of shared memory (one per SM), so one warp per subproblem would leave
// the SM nearly idle; the team shares each stage's products four times wider.
// Their FP64 reduction workspace does not fit an SM: its FP64 passes, with the
// workspace in global memory, come from shapes_xl64.cu.
#define MHE_TEAM 128
#include "kernels.cuh"

namespace mhe {

void shapes_xl_fp64(ShapeOps& o);   // shapes_xl64.cu

// the tries of the tensor-core product waits of this unit's kernels (< 0: the default)
int set_tc_wait_limit(int tries)
{
    const int v = tries < 0 ? -1 : tries;
    return cudaMemcpyToSymbol(tc::g_wait_override, &v, sizeof(int)) == cudaSuccess ? 0 : -1;
}

int shapes_xl(ShapeEntry* out, int cap)
{
    int k = 0;
    if (k < cap) {
        out[k] = make_shape<64, 32, 32>();
        shapes_xl_fp64(out[k].ops);
        ++k;
    }
    return k;
}

}  // namespace mhe
