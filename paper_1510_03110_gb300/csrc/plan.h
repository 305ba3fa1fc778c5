// plan.h -- the tree of subproblems (Algorithm 5's levels and chunk lists).
//
// Level 0 is the UFTOC problem of each instance (stage 0 = arrival stage).  A
// level whose horizon is at most top_len is the instance's top problem and is
// one chunk.  Otherwise the horizon is cut into chunks of length L (leaf_len
// at level 0, branching above), the last chunk taking the remainder; the
// p non-last chunks become the p stages of the next level's master problem
// (Eq. red_mpc_problem) and the last chunk its terminal cost.  The paper
// leaves the chunk lengths to the user (Section VI, remark on batch lengths).
#pragma once
#include <vector>

#include "common.h"

namespace mhe {

struct PlanLevel {
    std::vector<ChunkDesc> chunks;
    std::vector<LevelInst> li;     // per instance (N = 0: absent at this level)
    long long nstages = 0;         // sum of horizons at this level
    long long nstates = 0;         // sum of (horizon + 1)
};

struct Plan {
    int n = 0, m = 0, batch = 0;
    int leaf_len = 0, branching = 0, top_len = 0;
    std::vector<int> N;
    std::vector<long long> in_off;   // caller stage offset of stage t = 1 of each instance
    std::vector<long long> cmp_off;  // the compact offsets (prefix sums of N_b - 1): internal per-stage arrays
    std::vector<long long> w_off;    // caller offset of w_0 of each instance
    std::vector<long long> gs0;      // batch + 1 prefix sums of N (level-0 global stage base)
    long long S_in = 0;              // caller stages: sum (N_b - 1)
    long long W_total = 0;           // caller w entries: sum (n + (N_b - 1) m)
    long long X_total = 0;           // caller x / lambda states: sum (N_b + 1)
    int max_N = 0;
    std::vector<PlanLevel> levels;
};

// Returns 0, or a negative status (argument error) with a message in err.
int make_plan(int n, int m, const int* N, int batch, int leaf_len, int branching, int top_len,
              Plan& plan, const char** err);

// Chunk bounds of a level problem of horizon Nk with chunk length L: all chunks
// have length L except the last (1..L stages); at least two chunks.
void chunk_bounds(int Nk, int L, std::vector<int>& bnd);

}  // namespace mhe
