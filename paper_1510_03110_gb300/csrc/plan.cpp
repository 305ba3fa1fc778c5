// plan.cpp -- builds the per-level chunk lists of the tree (Algorithm 5).
#include "plan.h"

namespace mhe {

void chunk_bounds(int Nk, int L, std::vector<int>& bnd)
{
    if (Nk <= L) L = (Nk + 1) / 2;
    const int c = (Nk + L - 1) / L;
    bnd.clear();
    for (int i = 0; i < c; ++i) bnd.push_back(i * L);
    bnd.push_back(Nk);
}

int make_plan(int n, int m, const int* N, int batch, int leaf_len, int branching, int top_len,
              Plan& plan, const char** err)
{
    static const char* ok = "";
    *err = ok;
    if (n < 1 || m < 1 || batch < 1 || !N) { *err = "nx, nw, batch must be >= 1 and N given"; return -1; }
    const int min_leaf = (n + m - 1) / m;   // leaf chunks need L*nw >= nx for a nonsingular B^
    if (leaf_len < min_leaf) { *err = "leaf_len * nw must be >= nx"; return -1; }
    if (branching < 2) { *err = "branching must be >= 2"; return -1; }
    if (top_len < 1) { *err = "top_len must be >= 1"; return -1; }
    plan = Plan();
    plan.n = n; plan.m = m; plan.batch = batch;
    plan.leaf_len = leaf_len; plan.branching = branching; plan.top_len = top_len;
    plan.N.assign(N, N + batch);
    plan.in_off.resize(batch);
    plan.w_off.resize(batch);
    plan.gs0.resize(batch + 1);
    long long so = 0, wo = 0, g0 = 0, xo = 0;
    for (int b = 0; b < batch; ++b) {
        if (N[b] < 1) { *err = "every horizon N must be >= 1"; return -1; }
        plan.in_off[b] = so;
        plan.w_off[b] = wo;
        plan.gs0[b] = g0;
        so += N[b] - 1;
        wo += n + (long long)(N[b] - 1) * m;
        g0 += N[b];
        xo += N[b] + 1;
        if (N[b] > plan.max_N) plan.max_N = N[b];
    }
    plan.gs0[batch] = g0;
    plan.cmp_off = plan.in_off;
    plan.S_in = so;
    plan.W_total = wo;
    plan.X_total = xo;

    std::vector<int> bnd;
    for (int b = 0; b < batch; ++b) {
        int Nk = N[b];
        for (int k = 0;; ++k) {
            if ((int)plan.levels.size() <= k) {
                plan.levels.emplace_back();
                plan.levels.back().li.assign(batch, LevelInst{0, 0, 0, 0});
            }
            PlanLevel& L = plan.levels[k];
            LevelInst& li = L.li[b];
            li.gs = L.nstages;
            li.gx = L.nstates;
            li.N = Nk;
            L.nstages += Nk;
            L.nstates += Nk + 1;
            const int len = (k == 0) ? leaf_len : branching;
            bool top = Nk <= top_len;
            if (!top) {
                chunk_bounds(Nk, len, bnd);
                // at level 0 every non-last chunk except the first needs L*nw >= nx
                if (k == 0 && bnd.size() > 3 && (bnd[2] - bnd[1]) < min_leaf) top = true;
            }
            if (top) {
                li.top = 1;
                ChunkDesc cd;
                cd.inst = b; cd.t0 = 0; cd.len = Nk;
                cd.flags = CH_LAST | CH_TOP | (k == 0 ? CH_ARRIVAL : 0);
                cd.g0 = li.gs; cd.parent = -1; cd.px = -1;
                L.chunks.push_back(cd);
                break;
            }
            const int p = (int)bnd.size() - 2;   // chunks 0..p, p is the last
            // the next level exists for this instance; its bases are the current counters
            if ((int)plan.levels.size() <= k + 1) {
                plan.levels.emplace_back();
                plan.levels.back().li.assign(batch, LevelInst{0, 0, 0, 0});
            }
            PlanLevel& U = plan.levels[k + 1];
            PlanLevel& L2 = plan.levels[k];   // re-take: emplace_back may move
            const long long gs_up = U.nstages, gx_up = U.nstates;
            for (int i = 0; i <= p; ++i) {
                ChunkDesc cd;
                cd.inst = b;
                cd.t0 = bnd[i];
                cd.len = bnd[i + 1] - bnd[i];
                cd.flags = (i == p ? CH_LAST : 0) | ((k == 0 && i == 0) ? CH_ARRIVAL : 0);
                cd.g0 = L2.li[b].gs + bnd[i];
                cd.parent = (i < p) ? gs_up + i : -1;
                cd.px = gx_up + i;
                L2.chunks.push_back(cd);
            }
            Nk = p;
        }
    }
    return 0;
}

}  // namespace mhe
