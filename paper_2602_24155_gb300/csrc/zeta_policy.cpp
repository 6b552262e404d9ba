// Reduction policies (arXiv 2602.24155, Sec. 3.4 and Sec. 4) played on the
// host as the abstract game: only exponent vectors move, no linear algebra.
// The result is a plan the device executes (zeta_kernels.cu): for every term
// the chunks (v, k) of move 1 and the merge destination of move 2.
//
//  depth-first  (Sec. 4.2): each start term alone, greedy v (Algorithm 3),
//               largest k with v in V_full(u, k) and |u - k v| >= |S| - 1;
//               never merges.
//  p-chunk      (Sec. 4.1): all terms of the largest pole order K = p t are
//               reduced by p (by p - n when K = p), then terms with equal u
//               are combined; the start terms of pole order p(t-1) join.
//               Reading: when the greedy direction v admits fewer than p
//               steps, the chunk of size p is completed with further greedy
//               directions, so that all terms stay on the pole orders p t.
//  var-by-var   (Sec. 4.3): phase t = n..0 reduces every term with greedy
//               chunks until u_t = 0 (or pole order n), then combines.
//  cover        (this library, a search over move 2 of the game): the levels
//               of p-chunk, but every term of a level chooses its destination
//               so that terms land together.  Every step lowers each nonzero
//               coordinate in S by at least 1, so after L steps a term with
//               U_i >= L for i in S can reach exactly the V with
//               0 <= V <= U - L 1_S and |V| = |U| - d L; a group of terms can
//               share a destination iff the positive part of the
//               componentwise minimum of their boxes U - L 1_S still sums to
//               |V|.  Terms first join the next level's start terms they
//               dominate, then groups grow greedily on the compatibility graph
//               (seeds in decreasing degree, members keeping the most mass of
//               the common box); the destination is the point of the common
//               box proportional to it.  Terms with a coordinate below L, and
//               the last level (pole order n, no merging), play Algorithm 3.
#include <algorithm>
#include <array>
#include <cstring>
#include <functional>
#include <unordered_map>

#include "zeta_internal.h"

namespace zeta {

namespace {

// Algorithm 3: S scanned in ascending order (Smask, bit t = t in S), the count
// tested before every increment of the round-robin loop.
void greedy_v(const int32_t *U, int nv, int d, int *v, uint32_t Smask) {
    int i = d;
    for (int t = 0; t < nv; t++) v[t] = 0;
    for (int t = 0; t < nv && i > 0; t++)
        if (((Smask >> t) & 1u) && U[t] != 0) { v[t] = 1; i--; }
    while (i > 0)
        for (int t = 0; t < nv && i > 0; t++)
            if (v[t] < U[t]) { v[t]++; i--; }
}

int norm(const int32_t *U, int nv) {
    int s = 0;
    for (int t = 0; t < nv; t++) s += U[t];
    return s;
}

// largest k with U - k v >= 0 and |U - k v| >= base (= |S| - 1, the norm at pole order n)
int k_max(const int32_t *U, const int *v, int nv, int base, int d) {
    int k = (norm(U, nv) - base) / d;
    for (int t = 0; t < nv; t++)
        if (v[t] > 0) k = std::min(k, U[t] / v[t]);
    return k;
}

uint64_t pack(const int32_t *U, int nv) {
    uint64_t key = 0;
    for (int t = 0; t < nv; t++) key = (key << 12) | (uint64_t)U[t];
    return key;
}

// Greedy chunks from U until `stop` says so; appends to plan.chunks; U updated.
// first (optional): direction of the first chunk instead of Algorithm 3.
// choose (optional): proposes the direction of a chunk (U, steps left) instead of Algorithm 3.
template <typename Stop>
void play_chunks(Instance &X, int32_t *U, uint64_t live, Stop stop, int max_steps,
                 const std::function<bool(const int32_t *, int, int *)> &choose = nullptr) {
    const int nv = (int)X.nv, base = (int)X.base, d = (int)X.d;
    int left = max_steps;
    X.cur_live = live;
    while (norm(U, nv) > base && left > 0 && !stop(U)) {
        int v[kMaxVars];
        if (!(choose && choose(U, left, v))) greedy_v(U, nv, d, v, X.Smask);
        int k = std::min(k_max(U, v, nv, base, d), left);
        if (k <= 0) break;
        PlanChunk c;
        std::memset(&c, 0, sizeof(c));
        for (int t = 0; t < nv; t++) c.v[t] = (int8_t)v[t];
        c.k = k;
        X.plan.chunks.push_back(c);
        for (int t = 0; t < nv; t++) U[t] -= k * v[t];
        left -= k;
        X.plan.chunks_played++;
        X.plan.steps += k;
        X.plan.column_steps += (uint64_t)k * __builtin_popcountll(live);
        X.plan.work += (uint64_t)k * __builtin_popcountll(live) * X.s * X.s;
    }
}

// Chunks of a path of L steps from U to V = U - L 1_S - E (E >= 0, |E| = (d - |S|) L,
// U_i >= L for i in S): step j lowers every coordinate in S by 1 and takes
// d - |S| extra units from the list of E's units sorted by coordinate; equal
// consecutive steps form one chunk.  Every step is legal: the coordinates in S
// stay >= 1 until the last step (the condition of Prop. 3.3 holds) and the
// pole order stays >= n.
void path_chunks(Instance &X, int32_t *U, const int32_t *V, int L, uint64_t live) {
    const int nv = (int)X.nv, x = (int)X.d - (int)X.base - 1;
    int inS[kMaxVars];
    for (int t = 0; t < nv; t++) inS[t] = (int)((X.Smask >> t) & 1u);
    int rem[kMaxVars];
    int cur = 0;
    for (int t = 0; t < nv; t++) rem[t] = U[t] - L * inS[t] - V[t];
    int prev[kMaxVars];
    int run = 0;
    auto flush = [&]() {
        if (!run) return;
        PlanChunk c;
        std::memset(&c, 0, sizeof(c));
        for (int t = 0; t < nv; t++) c.v[t] = (int8_t)prev[t];
        c.k = run;
        X.plan.chunks.push_back(c);
        for (int t = 0; t < nv; t++) U[t] -= run * prev[t];
        X.plan.chunks_played++;
        X.plan.steps += run;
        X.plan.column_steps += (uint64_t)run * __builtin_popcountll(live);
        X.plan.work += (uint64_t)run * __builtin_popcountll(live) * X.s * X.s;
        run = 0;
    };
    for (int j = 0; j < L; j++) {
        int v[kMaxVars];
        for (int t = 0; t < nv; t++) v[t] = inS[t];
        for (int u = 0; u < x; u++) {
            while (cur < nv && rem[cur] == 0) cur++;
            if (cur >= nv) break;  // cannot happen (the units sum to x L); validate_plan rejects the plan
            v[cur]++;
            rem[cur]--;
        }
        bool same = run > 0;
        for (int t = 0; t < nv && same; t++) same = v[t] == prev[t];
        if (!same) {
            flush();
            std::memcpy(prev, v, sizeof(v));
        }
        run++;
    }
    flush();
}

uint64_t chain_live(const Instance &X, const Chain &ch) {
    uint64_t m = 0;
    for (uint32_t t = ch.term_begin; t < ch.term_end; t++) m |= 1ull << X.terms[t].col;
    return m;
}

// Destinations of the entries [e0, e1) of a cover level (L steps each): see
// the policy's description above.  Returns, per entry, its destination V or
// an empty vector (Algorithm 3).
std::vector<std::vector<int32_t>> cover_destinations(
    const Instance &X, const Plan &P, size_t e0, size_t e1, const std::vector<int> &next_starts, int L,
    const std::function<bool(const int32_t *, int, int *)> &choose) {
    const int nv = (int)X.nv, d = (int)X.d;
    const size_t E = e1 - e0;
    std::vector<std::vector<int32_t>> out(E);
    if (E == 0) return out;
    const int target = norm(P.entries[e0].U, nv) - d * L;
    std::vector<int> freeidx;
    std::vector<std::array<int32_t, kMaxVars>> box(E);
    for (size_t i = 0; i < E; i++) {
        const PlanEntry &e = P.entries[e0 + i];
        bool ok = norm(e.U, nv) - d * L == target;
        for (int t = 0; t < nv; t++) {
            box[i][t] = e.U[t] - (((X.Smask >> t) & 1u) ? L : 0);
            if (box[i][t] < 0) ok = false;
        }
        if (ok) freeidx.push_back((int)i);
    }
    auto mass = [&](const int32_t *m) {
        int s = 0;
        for (int t = 0; t < nv; t++) {
            if (m[t] < 0) return -1;
            s += m[t];
        }
        return s;
    };
    // 1. join a term already bound for the next level that the box dominates (most shared columns): the
    //    next level's start terms and the destinations of this level's other terms (Algorithm 3, or the
    //    network's directions under the learned policy)
    std::vector<std::array<int32_t, kMaxVars>> fixedV;
    std::vector<uint64_t> fixedLive;
    for (int c : next_starts) {
        std::array<int32_t, kMaxVars> V{};
        for (int t = 0; t < nv; t++) V[t] = X.chains[c].U[t];
        fixedV.push_back(V);
        fixedLive.push_back(chain_live(X, X.chains[c]));
    }
    {
        std::vector<char> is_free(E, 0);
        for (int i : freeidx) is_free[i] = 1;
        for (size_t i = 0; i < E; i++) {
            if (is_free[i]) continue;
            std::array<int32_t, kMaxVars> u{};
            for (int t = 0; t < nv; t++) u[t] = P.entries[e0 + i].U[t];
            int leftsteps = L;
            while (leftsteps > 0 && norm(u.data(), nv) > (int)X.base) {
                int v[kMaxVars];  // the direction the level will play (the same chooser as play_chunks)
                X.cur_live = P.entries[e0 + i].live;
                if (!(choose && choose(u.data(), leftsteps, v))) greedy_v(u.data(), nv, d, v, X.Smask);
                const int k = std::min(k_max(u.data(), v, nv, (int)X.base, d), leftsteps);
                if (k <= 0) break;
                for (int t = 0; t < nv; t++) u[t] -= k * v[t];
                leftsteps -= k;
            }
            if (norm(u.data(), nv) == target) {
                fixedV.push_back(u);
                fixedLive.push_back(P.entries[e0 + i].live);
            }
        }
    }
    std::vector<int> left;
    for (int i : freeidx) {
        const PlanEntry &e = P.entries[e0 + i];
        int best = -1, best_overlap = -1;
        for (size_t f = 0; f < fixedV.size(); f++) {
            bool dom = true;
            for (int t = 0; t < nv && dom; t++) dom = fixedV[f][t] <= box[i][t];
            if (!dom) continue;
            const int ov = __builtin_popcountll(fixedLive[f] & e.live);
            if (ov > best_overlap) { best_overlap = ov; best = (int)f; }
        }
        if (best >= 0) out[i].assign(fixedV[best].begin(), fixedV[best].end());
        else left.push_back(i);
    }
    // 2. compatibility graph on the rest, greedy group growth
    const size_t R = left.size();
    std::vector<std::vector<int>> comp(R);
    for (size_t a = 0; a < R; a++)
        for (size_t b = a + 1; b < R; b++) {
            int32_t m[kMaxVars];
            for (int t = 0; t < nv; t++) m[t] = std::min(box[left[a]][t], box[left[b]][t]);
            if (mass(m) >= target) {
                comp[a].push_back((int)b);
                comp[b].push_back((int)a);
            }
        }
    std::vector<int> order(R);
    for (size_t a = 0; a < R; a++) order[a] = (int)a;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return comp[a].size() > comp[b].size(); });
    std::vector<char> taken(R, 0);
    for (int a : order) {
        if (taken[a]) continue;
        taken[a] = 1;
        std::vector<int> grp{a};
        int32_t m[kMaxVars] = {0};
        for (int t = 0; t < nv; t++) m[t] = box[left[a]][t];
        std::vector<int> cand;
        for (int b : comp[a])
            if (!taken[b]) cand.push_back(b);
        while (!cand.empty()) {
            int best = -1, best_mass = -1;
            for (int b : cand) {
                int32_t mm[kMaxVars];
                for (int t = 0; t < nv; t++) mm[t] = std::min(m[t], box[left[b]][t]);
                const int ms = mass(mm);
                if (ms > best_mass) { best_mass = ms; best = b; }
            }
            if (best_mass < target) break;
            for (int t = 0; t < nv; t++) m[t] = std::min(m[t], box[left[best]][t]);
            taken[best] = 1;
            grp.push_back(best);
            std::vector<int> keep;
            for (int b : cand) {
                if (taken[b]) continue;
                int32_t mm[kMaxVars];
                for (int t = 0; t < nv; t++) mm[t] = std::min(m[t], box[left[b]][t]);
                if (mass(mm) >= target) keep.push_back(b);
            }
            cand.swap(keep);
        }
        // destination: the point of the common box m with |V| = target proportional to m
        const int tot = mass(m);
        std::vector<int32_t> V(kMaxVars, 0);
        int sum = 0;
        for (int t = 0; t < nv; t++) {
            V[t] = (int32_t)((int64_t)m[t] * target / tot);
            sum += V[t];
        }
        for (int t = 0; sum < target; t = (t + 1) % nv)
            if (V[t] < m[t]) { V[t]++; sum++; }
        for (int b : grp) out[left[b]] = V;
    }
    return out;
}

}  // namespace

zeta_status schedule_policy(Instance &X, zeta_policy policy) {
    Plan &P = X.plan;
    P = Plan();
    if (X.b > 64) { X.error = "more than 64 basis columns"; return X.status = ZETA_ERR_UNSUPPORTED; }
    const int nv = (int)X.nv, n = (int)X.n, d = (int)X.d, p = (int)X.p, base = (int)X.base;
    if (X.Smask != (1u << nv) - 1 && (policy == ZETA_POLICY_LEARNED || X.hook)) {
        X.error = "the learned policy takes S = {0..n} only";
        return X.status = ZETA_ERR_UNSUPPORTED;
    }
    // a term of pole order K has |u| = |S| - 1 + d (K - n)
    auto pole = [&](const int32_t *U) { return (norm(U, nv) - base) / d + n; };
    auto new_entry = [&](const int32_t *U) {
        PlanEntry e;
        std::memset(&e, 0, sizeof(e));
        for (int t = 0; t < nv; t++) e.U[t] = U[t];
        e.arrival = -1;
        e.start_chain = -1;
        e.dest = -1;
        return e;
    };

    if (policy == ZETA_POLICY_DEPTH_FIRST) {
        P.phase_begin.push_back(0);
        for (size_t c = 0; c < X.chains.size(); c++) {
            PlanEntry e = new_entry(X.chains[c].U);
            e.start_chain = (int32_t)c;
            e.live = chain_live(X, X.chains[c]);
            int32_t U[kMaxVars];
            std::memcpy(U, e.U, sizeof(U));
            e.chunk_begin = (uint32_t)P.chunks.size();
            play_chunks(X, U, e.live, [](const int32_t *) { return false; }, 1 << 30);
            e.chunk_end = (uint32_t)P.chunks.size();
            P.entries.push_back(e);
        }
        P.phase_begin.push_back((uint32_t)P.entries.size());
        P.cap = 0;
        return ZETA_OK;
    }

    // phases with merging.  `cur` maps exponent -> (arrival block, live mask).
    struct Arr { int32_t block; uint64_t live; };
    std::unordered_map<uint64_t, Arr> cur, nxt;
    std::vector<std::vector<int32_t>> curU, nxtU;  // exponents of arrival blocks by index
    auto phase = [&](const std::vector<int> &starts, auto stop_for, auto max_steps,
                     const std::function<bool(const int32_t *, int, int *)> &choose = nullptr,
                     const std::vector<int> *cover_next = nullptr, int cover_L = 0) {
        // entries: arrivals of this phase, then start chains (merged into an arrival if equal u)
        P.phase_begin.push_back((uint32_t)P.entries.size());
        std::unordered_map<uint64_t, size_t> entry_of;
        for (size_t bi = 0; bi < curU.size(); bi++) {
            const int32_t *U = curU[bi].data();
            PlanEntry e = new_entry(U);
            e.arrival = (int32_t)bi;
            e.live = cur[pack(U, nv)].live;
            entry_of[pack(U, nv)] = P.entries.size();
            P.entries.push_back(e);
        }
        for (int c : starts) {
            const int32_t *U = X.chains[c].U;
            uint64_t key = pack(U, nv);
            auto it = entry_of.find(key);
            if (it != entry_of.end()) {
                P.entries[it->second].start_chain = c;
                P.entries[it->second].live |= chain_live(X, X.chains[c]);
                P.merges++;
            } else {
                PlanEntry e = new_entry(U);
                e.start_chain = c;
                e.live = chain_live(X, X.chains[c]);
                entry_of[key] = P.entries.size();
                P.entries.push_back(e);
            }
        }
        // play each entry, route to the next phase
        nxt.clear();
        nxtU.clear();
        const size_t e0 = P.phase_begin.back(), e1 = P.entries.size();
        std::vector<std::vector<int32_t>> dest_of;  // cover: chosen destination per entry (empty = Algorithm 3)
        if (cover_next) dest_of = cover_destinations(X, P, e0, e1, *cover_next, cover_L, choose);
        for (size_t ei = e0; ei < e1; ei++) {
            PlanEntry &e = P.entries[ei];
            int32_t U[kMaxVars];
            std::memcpy(U, e.U, sizeof(U));
            e.chunk_begin = (uint32_t)P.chunks.size();
            if (cover_next && !dest_of[ei - e0].empty()) path_chunks(X, U, dest_of[ei - e0].data(), cover_L, e.live);
            else play_chunks(X, U, e.live, stop_for, max_steps(e), choose);
            e.chunk_end = (uint32_t)P.chunks.size();
            if (norm(U, nv) == base) {
                e.dest = -1;
                continue;
            }
            uint64_t key = pack(U, nv);
            auto it = nxt.find(key);
            if (it == nxt.end()) {
                Arr a{(int32_t)nxtU.size(), e.live};
                nxt.emplace(key, a);
                nxtU.push_back(std::vector<int32_t>(U, U + kMaxVars));
                e.dest = a.block;
                e.flags |= 1u;
            } else {
                e.dest = it->second.block;
                it->second.live |= e.live;
                P.merges++;
            }
        }
        P.cap = std::max<uint32_t>(P.cap, (uint32_t)nxtU.size());
        cur.swap(nxt);
        curU.swap(nxtU);
    };

    if (policy == ZETA_POLICY_LEARNED && X.net.w) {
        // the network sees the terms of the p-chunk game played with Algorithm 3
        zeta_status st = reference_contributions(X);
        if (st) return st;
        X.plan = Plan();
    }
    if (policy == ZETA_POLICY_PCHUNK || policy == ZETA_POLICY_LEARNED || policy == ZETA_POLICY_COVER) {
        int tmax = 0;
        std::vector<std::vector<int>> by_level;
        for (size_t c = 0; c < X.chains.size(); c++) {
            int K = pole(X.chains[c].U);
            if (K % p) { X.error = "start pole order not a multiple of p"; return X.status = ZETA_ERR_INTERNAL; }
            int t = K / p;
            if ((int)by_level.size() <= t) by_level.resize(t + 1);
            by_level[t].push_back((int)c);
            tmax = std::max(tmax, t);
        }
        for (int t = tmax; t >= 1; t--) {
            const int steps = (t >= 2) ? p : p - n;  // to pole order p(t-1), or to n
            std::function<bool(const int32_t *, int, int *)> choose = nullptr;
            if (policy == ZETA_POLICY_LEARNED)
                choose = [&X, t, tmax](const int32_t *U, int left, int *v) {
                    return learned_direction(X, U, left, t, tmax, v);
                };
            else if (policy == ZETA_POLICY_COVER && X.hook)
                choose = [&X, t](const int32_t *U, int left, int *v) { return X.hook(U, left, t, v); };
            // the learned policy plays on the cover levels: searched destinations where a term's box allows,
            // the network's directions for the others
            const bool cover = (policy == ZETA_POLICY_COVER || (policy == ZETA_POLICY_LEARNED && X.net.w)) &&
                               t >= 2 && d > base;
            const std::vector<int> none;
            phase(t < (int)by_level.size() ? by_level[t] : none, [](const int32_t *) { return false; },
                  [&](const PlanEntry &) { return steps; }, choose,
                  cover ? (t - 1 < (int)by_level.size() ? &by_level[t - 1] : &none) : nullptr, steps);
        }
    } else if (policy == ZETA_POLICY_VAR_BY_VAR) {
        std::vector<int> all(X.chains.size());
        for (size_t c = 0; c < all.size(); c++) all[c] = (int)c;
        for (int t = n; t >= 0; t--) {
            phase(t == n ? all : std::vector<int>(), [t](const int32_t *U) { return U[t] == 0; },
                  [](const PlanEntry &) { return 1 << 30; });
        }
        if (!curU.empty()) { X.error = "var-by-var left terms above pole order n"; return X.status = ZETA_ERR_INTERNAL; }
    } else {
        X.error = "unknown policy";
        return X.status = ZETA_ERR_ARG;
    }
    P.phase_begin.push_back((uint32_t)P.entries.size());
    return validate_plan(X);
}

// Every chunk of the plan is a legal move of the game (Prop. 3.3: |v| = d,
// v <= u, u_i != 0 => v_i != 0 for i in S, k >= 1, pole order >= n after the
// chunk, i.e. |u| >= |S| - 1) and every entry ends where its routing says: at
// the exponent of its destination block, or at pole order n.
zeta_status validate_plan(Instance &X) {
    const Plan &P = X.plan;
    const int nv = (int)X.nv, base = (int)X.base, d = (int)X.d;
    for (size_t ph = 0; ph + 1 < P.phase_begin.size(); ph++) {
        std::unordered_map<int32_t, std::vector<int32_t>> dest_U;
        for (uint32_t ei = P.phase_begin[ph]; ei < P.phase_begin[ph + 1]; ei++) {
            const PlanEntry &e = P.entries[ei];
            int32_t U[kMaxVars];
            std::memcpy(U, e.U, sizeof(U));
            for (uint32_t ci = e.chunk_begin; ci < e.chunk_end; ci++) {
                const PlanChunk &c = P.chunks[ci];
                int sv = 0;
                bool ok = c.k >= 1;
                for (int t = 0; t < nv; t++) {
                    sv += c.v[t];
                    if (c.v[t] < 0 || U[t] - c.k * c.v[t] < 0 || (((X.Smask >> t) & 1u) && U[t] != 0 && c.v[t] == 0))
                        ok = false;
                }
                if (!ok || sv != d) {
                    X.error = "plan has an illegal chunk";
                    return X.status = ZETA_ERR_INTERNAL;
                }
                for (int t = 0; t < nv; t++) U[t] -= c.k * c.v[t];
                if (norm(U, nv) < base) {
                    X.error = "plan goes below pole order n";
                    return X.status = ZETA_ERR_INTERNAL;
                }
            }
            if (e.dest < 0) {
                if (norm(U, nv) != base) {
                    X.error = "plan leaves a term above pole order n";
                    return X.status = ZETA_ERR_INTERNAL;
                }
                continue;
            }
            auto it = dest_U.find(e.dest);
            if (it == dest_U.end()) dest_U.emplace(e.dest, std::vector<int32_t>(U, U + nv));
            else if (!std::equal(U, U + nv, it->second.begin())) {
                X.error = "plan merges different exponents";
                return X.status = ZETA_ERR_INTERNAL;
            }
        }
        // the next phase's arrivals start where their block's entries ended
        if (ph + 2 < P.phase_begin.size())
            for (uint32_t ei = P.phase_begin[ph + 1]; ei < P.phase_begin[ph + 2]; ei++) {
                const PlanEntry &e = P.entries[ei];
                if (e.arrival < 0) continue;
                auto it = dest_U.find(e.arrival);
                if (it == dest_U.end() || !std::equal(e.U, e.U + nv, it->second.begin())) {
                    X.error = "plan arrival does not match its block";
                    return X.status = ZETA_ERR_INTERNAL;
                }
            }
    }
    return ZETA_OK;
}

}  // namespace zeta
