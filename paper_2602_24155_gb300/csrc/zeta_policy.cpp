// Reduction policies (arXiv 2602.24155, Sec. 3.4 and Sec. 4) played on the
// host as the abstract game: only exponent vectors move, no linear algebra.
// The result is a plan the device executes (zeta_kernels.cu): for every term
// the chunks (v, k) of move 1 and the merge destination of move 2.
//
//  depth-first  (Sec. 4.2): each start term alone, greedy v (Algorithm 3),
//               largest k with v in V_full(u, k) and |u - k v| >= n; never merges.
//  p-chunk      (Sec. 4.1): all terms of the largest pole order K = p t are
//               reduced by p (by p - n when K = p), then terms with equal u
//               are combined; the start terms of pole order p(t-1) join.
//               Reading: when the greedy direction v admits fewer than p
//               steps, the chunk of size p is completed with further greedy
//               directions, so that all terms stay on the pole orders p t.
//  var-by-var   (Sec. 4.3): phase t = n..0 reduces every term with greedy
//               chunks until u_t = 0 (or pole order n), then combines.
#include <algorithm>
#include <cstring>
#include <functional>
#include <unordered_map>

#include "zeta_internal.h"

namespace zeta {

namespace {

// Algorithm 3 with S = {0..n}: S scanned in ascending order, the count tested
// before every increment of the round-robin loop.
void greedy_v(const int32_t *U, int nv, int d, int *v) {
    int i = d;
    for (int t = 0; t < nv; t++) v[t] = 0;
    for (int t = 0; t < nv && i > 0; t++)
        if (U[t] != 0) { v[t] = 1; i--; }
    while (i > 0)
        for (int t = 0; t < nv && i > 0; t++)
            if (v[t] < U[t]) { v[t]++; i--; }
}

int norm(const int32_t *U, int nv) {
    int s = 0;
    for (int t = 0; t < nv; t++) s += U[t];
    return s;
}

// largest k with U - k v >= 0 and |U - k v| >= n
int k_max(const int32_t *U, const int *v, int nv, int n, int d) {
    int k = (norm(U, nv) - n) / d;
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
void play_chunks(Instance &X, int32_t *U, uint32_t live, Stop stop, int max_steps,
                 const std::function<bool(const int32_t *, int, int *)> &choose = nullptr) {
    const int nv = (int)X.nv, n = (int)X.n, d = (int)X.d;
    int left = max_steps;
    while (norm(U, nv) > n && left > 0 && !stop(U)) {
        int v[kMaxVars];
        if (!(choose && choose(U, left, v))) greedy_v(U, nv, d, v);
        int k = std::min(k_max(U, v, nv, n, d), left);
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
        X.plan.column_steps += (uint64_t)k * __builtin_popcount(live);
        X.plan.work += (uint64_t)k * __builtin_popcount(live) * X.s * X.s;
    }
}

uint32_t chain_live(const Instance &X, const Chain &ch) {
    uint32_t m = 0;
    for (uint32_t t = ch.term_begin; t < ch.term_end; t++) m |= 1u << X.terms[t].col;
    return m;
}

}  // namespace

zeta_status schedule_policy(Instance &X, zeta_policy policy) {
    Plan &P = X.plan;
    P = Plan();
    if (X.b > 32) { X.error = "more than 32 basis columns"; return X.status = ZETA_ERR_UNSUPPORTED; }
    const int nv = (int)X.nv, n = (int)X.n, d = (int)X.d, p = (int)X.p;
    auto pole = [&](const int32_t *U) { return (norm(U, nv) - n) / d + n; };
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
    struct Arr { int32_t block; uint32_t live; };
    std::unordered_map<uint64_t, Arr> cur, nxt;
    std::vector<std::vector<int32_t>> curU, nxtU;  // exponents of arrival blocks by index
    auto phase = [&](const std::vector<int> &starts, auto stop_for, auto max_steps,
                     const std::function<bool(const int32_t *, int, int *)> &choose = nullptr) {
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
        for (size_t ei = e0; ei < e1; ei++) {
            PlanEntry &e = P.entries[ei];
            int32_t U[kMaxVars];
            std::memcpy(U, e.U, sizeof(U));
            e.chunk_begin = (uint32_t)P.chunks.size();
            play_chunks(X, U, e.live, stop_for, max_steps(e), choose);
            e.chunk_end = (uint32_t)P.chunks.size();
            if (norm(U, nv) == n) {
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
    if (policy == ZETA_POLICY_PCHUNK || policy == ZETA_POLICY_LEARNED) {
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
            else if (X.teacher)
                choose = [&X](const int32_t *U, int left, int *v) { return teacher_direction(X, U, left, v); };
            phase(t < (int)by_level.size() ? by_level[t] : std::vector<int>(),
                  [](const int32_t *) { return false; }, [&](const PlanEntry &) { return steps; }, choose);
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
    return ZETA_OK;
}

}  // namespace zeta
