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
              Plan& plan, const char** err, bool rank_revealing)
{
    static const char* ok = "";
    *err = ok;
    if (n < 1 || m < 1 || batch < 1 || !N) { *err = "nx, nw, batch must be >= 1 and N given"; return -1; }
    // leaf chunks need L*nw >= nx for a nonsingular B^, unless the master stages are rank-revealing
    const int min_leaf = rank_revealing ? 1 : (n + m - 1) / m;
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
                cd.g0 = li.gs; cd.parent = -1; cd.px = -1; cd.pw = -1; cd.parent2 = -1;
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
                cd.pw = cd.parent;
                cd.parent2 = -1;
                cd.px = gx_up + i;
                L2.chunks.push_back(cd);
            }
            Nk = p;
        }
    }
    return 0;
}

namespace {
// slots after each ring's capacity: the longest top chunk (top_len stages, or one
// block of leaf or branching stages, and never more than the window's N stages)
// starting at any slot of the ring fits
long long serve_tail(int leaf, int br, int top, int N)
{
    long long t = top > leaf ? top : leaf;
    if (br > t) t = br;
    if (N < t) t = N;
    return t + 1;
}
}  // namespace

int serve_caps(int N, int leaf, int br, int top, std::vector<long long>& cap, long long* tail)
{
    cap.clear();
    if (N < 2 || leaf < 1 || br < 2 || top < 1) return 0;
    *tail = serve_tail(leaf, br, top, N);
    // level 0: the N - 1 samples meet at most ceil((N-1)/L) + 1 blocks
    long long nb = (N - 1 + leaf - 1) / leaf;
    cap.push_back((long long)leaf * (nb + 2));
    long long Nk = nb;   // master stages of level 1, at most
    int len = br;
    while (true) {
        const long long blocks = (Nk + len - 1) / len;
        cap.push_back((long long)len * (blocks + 2));
        if (Nk <= top || cap.size() > 60) break;
        Nk = blocks;
    }
    return (int)cap.size();
}

int make_serve_plan(int n, int m, const std::vector<ServeWindow>& w, int leaf, int br, int top, Plan& plan,
                    std::vector<std::vector<ChunkDesc>>& dirty, long long* reduced, const char** err)
{
    static const char* ok = "";
    *err = ok;
    const int batch = (int)w.size();
    if (n < 1 || m < 1 || batch < 1) { *err = "nx, nw, batch must be >= 1"; return -1; }
    const int min_leaf = (n + m - 1) / m;
    if (leaf < min_leaf) { *err = "leaf_len * nw must be >= nx"; return -1; }
    if (br < 2 || top < 1) { *err = "branching must be >= 2 and top_len >= 1"; return -1; }
    plan = Plan();
    plan.n = n; plan.m = m; plan.batch = batch;
    plan.leaf_len = leaf; plan.branching = br; plan.top_len = top;
    plan.N.resize(batch);
    plan.in_off.resize(batch);
    plan.cmp_off.resize(batch);
    plan.w_off.resize(batch);
    plan.gs0.resize(batch + 1);
    long long so = 0, wo = 0, g0s = 0, xo = 0;
    for (int b = 0; b < batch; ++b) {
        if (w[b].N < 2) { *err = "every window horizon N must be >= 2"; return -1; }
        plan.N[b] = w[b].N;
        plan.in_off[b] = w[b].in_off;
        plan.cmp_off[b] = so;
        plan.w_off[b] = wo;
        plan.gs0[b] = g0s;
        so += w[b].N - 1;
        wo += n + (long long)(w[b].N - 1) * m;
        g0s += w[b].N;
        xo += w[b].N + 1;
        if (w[b].N > plan.max_N) plan.max_N = w[b].N;
    }
    plan.gs0[batch] = g0s;
    plan.S_in = so;
    plan.W_total = wo;
    plan.X_total = xo;
    dirty.clear();
    auto level = [&](int k) -> PlanLevel& {
        while ((int)plan.levels.size() <= k) {
            plan.levels.emplace_back();
            plan.levels.back().li.assign(batch, LevelInst{0, 0, 0, 0});
            dirty.emplace_back();
        }
        return plan.levels[k];
    };
    for (int b = 0; b < batch; ++b) {
        const ServeWindow& W = w[b];
        std::vector<ServeLevelHist>& H = *W.hist;
        // level k: stages t = 0 .. Nk - 1; at level 0 stage t >= 1 is sample k0 + t - 1 and
        // stage 0 the arrival stage, at level k >= 1 stage t is master stage f + t
        long long f = W.k0;          // absolute index of stage 1 (level 0) or stage 0 (k >= 1)
        long long Nk = W.N;          // the level's horizon
        int k = 0;
        for (;; ++k) {
            if (k >= W.nlev) { *err = "the window needs more levels than its rings provide"; return -1; }
            if ((int)H.size() <= k) H.resize(k + 1);
            PlanLevel& L = level(k);
            LevelInst& li = L.li[b];
            li.gs = L.nstages;
            li.gx = L.nstates;
            li.N = (int)Nk;
            L.nstages += Nk;
            L.nstates += Nk + 1;
            const int len = k == 0 ? leaf : br;
            const long long capk = W.cap[k], basek = W.base[k];
            // absolute chunk indices of the first and last chunk (level 0: the blocks of the samples)
            const long long lo = f, hi = k == 0 ? f + Nk - 2 : f + Nk - 1;
            const long long c0 = lo / len, cl = hi / len;
            auto ring = [&](long long idx) { return basek + idx % capk; };
            if (Nk <= top || c0 == cl) {
                // the top problem: one chunk, reduced every round (its factors may run into the tail)
                li.top = 1;
                ChunkDesc cd;
                cd.inst = b; cd.t0 = 0; cd.len = (int)Nk;
                cd.flags = CH_LAST | CH_TOP | (k == 0 ? CH_ARRIVAL : 0);
                cd.g0 = k == 0 ? ring(f) - 1 : ring(f);
                cd.parent = -1; cd.px = -1; cd.pw = -1; cd.parent2 = -1;
                L.chunks.push_back(cd);
                dirty[k].push_back(cd);
                *reduced += Nk;
                H[k].first = H[k].last = -1;
                H[k].top = 1;
                break;
            }
            if (k + 1 >= W.nlev) { *err = "the window needs more levels than its rings provide"; return -1; }
            PlanLevel& U = level(k + 1);
            PlanLevel& L2 = plan.levels[k];   // re-take: level() may move the vector
            const long long gs_up = U.nstages, gx_up = U.nstates;
            const long long capu = W.cap[k + 1], baseu = W.base[k + 1];
            const long long tailu = serve_tail(leaf, br, top, W.N);
            const ServeLevelHist prev = H[k];
            for (long long c = c0; c <= cl; ++c) {
                ChunkDesc cd;
                cd.inst = b;
                const long long start = c == c0 ? lo : c * len, end = c == cl ? hi : (c + 1) * len - 1;
                if (k == 0) {
                    cd.t0 = c == c0 ? 0 : (int)(start - f + 1);
                    cd.len = (int)(end - start + 1) + (c == c0 ? 1 : 0);
                    cd.g0 = c == c0 ? ring(start) - 1 : ring(start);
                } else {
                    cd.t0 = (int)(start - f);
                    cd.len = (int)(end - start + 1);
                    cd.g0 = ring(start);
                }
                cd.flags = (c == cl ? CH_LAST : 0) | ((k == 0 && c == c0) ? CH_ARRIVAL : 0);
                const long long i = c - c0;   // master stage index within the level above
                if (c < cl) {
                    cd.parent = baseu + c % capu;
                    cd.parent2 = (c % capu) < tailu ? baseu + capu + c % capu : -1;
                    cd.pw = gs_up + i;
                } else {
                    cd.parent = -1; cd.parent2 = -1; cd.pw = -1;
                }
                cd.px = gx_up + i;
                L2.chunks.push_back(cd);
                const bool kept = prev.top == 0 && c > prev.first && c < prev.last && c > c0 && c < cl;
                if (!kept) {
                    dirty[k].push_back(cd);
                    *reduced += cd.len;
                }
            }
            H[k].first = c0;
            H[k].last = cl;
            H[k].top = 0;
            f = c0;
            Nk = cl - c0;
        }
        // levels above this round's top: nothing of them is kept
        for (size_t j = (size_t)k + 1; j < H.size(); ++j) H[j] = ServeLevelHist();
    }
    return 0;
}

}  // namespace mhe
