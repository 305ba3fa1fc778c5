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
// rank_revealing: the master stages are factored with pivoting at their
// numerical rank, so leaf chunks may be shorter than ceil(nx / nw) stages
// (leaf_len >= 1); otherwise leaf_len * nw >= nx is required.
int make_plan(int n, int m, const int* N, int batch, int leaf_len, int branching, int top_len,
              Plan& plan, const char** err, bool rank_revealing = false);

// A plan whose leaf chunks may have a rank-deficient Q^_w: leaf_len * nw < nx.
inline bool needs_rank_revealing(int n, int m, int leaf_len) { return (long long)leaf_len * m < n; }

// Chunk bounds of a level problem of horizon Nk with chunk length L: all chunks
// have length L except the last (1..L stages); at least two chunks.
void chunk_bounds(int Nk, int L, std::vector<int>& bnd);

// ---- receding-horizon serving with factorisation reuse -----------------------
// The tree of an estimator's window with chunk boundaries fixed in absolute
// time: level-0 chunk c holds the samples [cL, (c+1)L) of the estimator's
// measurement stream (the window's first chunk also the arrival stage), and
// level-k chunk g the master stages [gb, (g+1)b), master stage c of level k
// being chunk c of level k-1.  A shift by one sample changes each level's first
// chunk (it loses its oldest stage), its last chunk (the new stage, the new
// terminal) and, when a chunk opens, the chunk that was last; every chunk that
// is interior in two consecutive rounds keeps its data and so its Algorithm 4
// output (its stored factors and its master stage).  Those live in one ring per
// level and estimator whose capacity is a multiple of the level's chunk length,
// so no chunk wraps, followed by a tail into which a top chunk (which spans
// several blocks) may run; master stages whose ring slot is below the tail size
// are also written to the mirrored slot slot + cap.
struct ServeLevelHist {
    long long first = -1, last = -1;   // absolute indices of the level's first and last chunk
    int top = 1;                       // the level was the top (or absent): nothing kept
};

struct ServeWindow {
    int N;                     // UFTOC horizon of the window (N - 1 measured stages)
    long long k0;              // absolute index of the window's first measured sample (stage t = 1)
    long long in_off;          // input offset of stage t = 1 (the resident stage arrays)
    const long long* base;     // per level: the estimator's first slot in the level's store
    const long long* cap;      // per level: ring capacity (a multiple of the level's chunk length)
    int nlev;                  // levels with a ring
    std::vector<ServeLevelHist>* hist;   // previous round's chunk ranges per level; updated
};

// Ring capacities for windows of horizon N: cap[k] per level and the tail every
// ring carries; returns the number of levels (0 on bad arguments).
int serve_caps(int N, int leaf, int br, int top, std::vector<long long>& cap, long long* tail);

// The round's plan over windows w: every level's full chunk list (right-hand
// side and down passes) in plan.levels, and in dirty[k] the chunks of level k
// that must be reduced again; *reduced += the stages of those chunks.  Per-round
// arrays (solutions, terminals, the arrival stage's factors) use the plan's
// per-instance bases as make_plan's do.  Returns 0 or a negative status.
int make_serve_plan(int n, int m, const std::vector<ServeWindow>& w, int leaf, int br, int top, Plan& plan,
                    std::vector<std::vector<ChunkDesc>>& dirty, long long* reduced, const char** err);

}  // namespace mhe
