// Learned direction policy for the reduction game (arXiv 2602.24155,
// Sec. 3.4; Sec. 4.4 notes that the paper's policies never inspect U and
// that better policies are open).  The network scores the legal directions v
// of every chunk decision the cover levels leave to a direction rule (the
// terms whose destination is not searched, Sec. 4.1 p-chunks) and the best is
// played; any choice yields the same cohomology classes, only the game's cost
// changes.
//
// Training data comes from the game itself.  The cover game is played with
// Algorithm 3 and its chunk decisions with two or more legal directions are
// recorded; for a sample of them (kDatasetDecisions per instance) every legal
// direction is tried in a full rollout of the rest of the game (the same
// cover game, Algorithm 3 elsewhere), and its cost is that plan's column steps
// plus kChunkCost per chunk played.  The label is the cheapest direction (ties
// to Algorithm 3's choice), and costs[row] is the row's cost above it.  The
// network sees only local features, so it stands in for the rollouts, whose
// cost grows with the game, in the scheduler.
//
// Features of a candidate (u, v), with w the exponent reached at the end of the
// p-chunk (v first, then Algorithm 3):
//   u_i/|u|, v_i/d, w_i/|w| for four coordinates (zero-padded),
//   k/left (this chunk's length over the steps left), t/tmax (level),
//   [v is Algorithm 3's choice],
//   and what the policy sees of U: the number c of other terms that reach w in
//   the reference game (the cover game with Algorithm 3), as min(c, 4)/4 and
//   [c > 0], and the share of the term's columns those terms carry to w.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstring>
#include <functional>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "zeta_internal.h"

namespace zeta {

namespace {

int norm(const int32_t *U, int nv) {
    int s = 0;
    for (int t = 0; t < nv; t++) s += U[t];
    return s;
}

uint64_t pack(const int32_t *U, int nv) {
    uint64_t key = 0;
    for (int t = 0; t < nv; t++) key = (key << 12) | (uint64_t)U[t];
    return key;
}

void greedy_dir(const int32_t *U, int nv, int d, int *v) {
    int i = d;
    for (int t = 0; t < nv; t++) v[t] = 0;
    for (int t = 0; t < nv && i > 0; t++)
        if (U[t] != 0) { v[t] = 1; i--; }
    while (i > 0)
        for (int t = 0; t < nv && i > 0; t++)
            if (v[t] < U[t]) { v[t]++; i--; }
}

int kmax(const int32_t *U, const int *v, int nv, int n, int d) {
    int k = (norm(U, nv) - n) / d;
    for (int t = 0; t < nv; t++)
        if (v[t] > 0) k = std::min(k, U[t] / v[t]);
    return k;
}

// All v with |v| = d, v <= U, U_i != 0 => v_i >= 1 (Sec. 3.4, V_full) and k_max >= 1,
// Algorithm 3's choice first; compositions of d enumerated with an explicit stack.
void legal_dirs(const int32_t *U, int nv, int n, int d, std::vector<std::array<int, kMaxVars>> &out) {
    out.clear();
    int g[kMaxVars];
    greedy_dir(U, nv, d, g);
    std::array<int, kMaxVars> ga{};
    for (int t = 0; t < nv; t++) ga[t] = g[t];
    out.push_back(ga);
    std::array<int, kMaxVars> v{};
    int lo[kMaxVars], hi[kMaxVars];
    for (int t = 0; t < nv; t++) {
        lo[t] = U[t] != 0 ? 1 : 0;
        hi[t] = std::min<int>(U[t], d);
    }
    // odometer over v_0..v_{nv-2}; v_{nv-1} = d - (sum of the others)
    int pos = 0, rem = d;
    v[0] = lo[0] - 1;
    while (pos >= 0) {
        if (pos == nv - 1) {
            v[pos] = rem;
            if (rem >= lo[pos] && rem <= hi[pos] && kmax(U, v.data(), nv, n, d) >= 1 && v != ga) out.push_back(v);
            pos--;
            continue;
        }
        // next value of v[pos]
        if (v[pos] >= lo[pos]) rem += v[pos];
        v[pos]++;
        if (v[pos] > hi[pos] || v[pos] > rem) {
            v[pos] = lo[pos] - 1;
            pos--;
            continue;
        }
        rem -= v[pos];
        pos++;
        if (pos < nv - 1) v[pos] = lo[pos] - 1;
    }
}

// Exponent reached after `left` steps: first chunk in direction v, then Algorithm 3.
void p_chunk_dest(const int32_t *U, const int *v, int left, int nv, int n, int d, int32_t *W, int *k_first) {
    for (int t = 0; t < nv; t++) W[t] = U[t];
    bool first = true;
    *k_first = 0;
    while (left > 0 && norm(W, nv) > n) {
        int dir[kMaxVars];
        if (first) for (int t = 0; t < nv; t++) dir[t] = v[t];
        else greedy_dir(W, nv, d, dir);
        int k = std::min(left, kmax(W, dir, nv, n, d));
        if (k <= 0) break;
        if (first) *k_first = k;
        first = false;
        for (int t = 0; t < nv; t++) W[t] -= k * dir[t];
        left -= k;
    }
}

void features(const int32_t *U, const int *v, const int32_t *W, int k_first, int left, int t, int tmax, int nv, int d,
              bool is_greedy, int others, float overlap, float *f) {
    const float nu = (float)std::max(1, norm(U, nv)), nw = (float)std::max(1, norm(W, nv));
    for (int i = 0; i < 4; i++) {
        f[i] = i < nv ? U[i] / nu : 0.f;
        f[4 + i] = i < nv ? (float)v[i] / d : 0.f;
        f[8 + i] = i < nv ? W[i] / nw : 0.f;
    }
    f[12] = left > 0 ? (float)k_first / left : 0.f;
    f[13] = tmax > 0 ? (float)t / tmax : 0.f;
    f[14] = is_greedy ? 1.f : 0.f;
    f[15] = (float)std::min(std::max(others, 0), 4) / 4.f;
    f[16] = others > 0 ? 1.f : 0.f;
    f[17] = overlap;
}

// Other terms of the reference game that reach W at level t - 1, for the term at U
// (its own Algorithm 3 destination `own` is not counted).
int others_at(const Instance &X, int t, const int32_t *W, uint64_t own) {
    if (t - 1 < 1 || t - 1 >= (int)X.ref_contrib.size()) return 0;
    const uint64_t key = pack(W, (int)X.nv);
    auto it = X.ref_contrib[t - 1].find(key);
    int c = it == X.ref_contrib[t - 1].end() ? 0 : it->second;
    return key == own ? c - 1 : c;
}

// Share of the term's columns (live) that other terms of the reference game carry to W at level t - 1: the
// columns a merge there would save (the term's own contribution is not counted when W is its own destination).
float overlap_at(const Instance &X, int t, const int32_t *W, uint64_t own, uint64_t live) {
    if (!live || t - 1 < 1 || t - 1 >= (int)X.ref_cols.size()) return 0.f;
    const uint64_t key = pack(W, (int)X.nv);
    auto it = X.ref_cols[t - 1].find(key);
    if (it == X.ref_cols[t - 1].end()) return 0.f;
    int shared = 0;
    for (int col = 0; col < 64; col++)
        if ((live >> col & 1ull) && (int)it->second[col] - (key == own ? 1 : 0) > 0) shared++;
    return (float)shared / (float)__builtin_popcountll(live);
}

}  // namespace

float policy_score(const PolicyNet &net, const float *x) {
    const int F = kPolicyFeatures, H = net.hidden;
    const float *W1 = net.w, *b1 = W1 + F * H, *W2 = b1 + H, *b2 = W2 + H * H, *w3 = b2 + H, *b3 = w3 + H;
    float h1[512], h2[512];
    for (int j = 0; j < H; j++) {
        float a = b1[j];
        for (int i = 0; i < F; i++) a += x[i] * W1[i * H + j];
        h1[j] = a > 0.f ? a : 0.f;
    }
    float out = b3[0];
    for (int j = 0; j < H; j++) {
        float a = b2[j];
        for (int i = 0; i < H; i++) a += h1[i] * W2[i * H + j];
        h2[j] = a > 0.f ? a : 0.f;
        out += h2[j] * w3[j];
    }
    return out;
}



size_t policy_param_count(int hidden) {
    const size_t F = kPolicyFeatures, H = hidden;
    return F * H + H + H * H + H + H + 1;
}

bool learned_direction(const Instance &X, const int32_t *U, int left, int t, int tmax, int *v) {
    if (!X.net.w || X.net.hidden <= 0 || X.net.hidden > 512 || X.nv > 4) return false;
    const int nv = (int)X.nv, n = (int)X.n, d = (int)X.d;
    std::vector<std::array<int, kMaxVars>> cand;
    legal_dirs(U, nv, n, d, cand);
    if (cand.size() < 2) return false;
    int32_t own_w[kMaxVars];
    int kf0;
    p_chunk_dest(U, cand[0].data(), left, nv, n, d, own_w, &kf0);
    const uint64_t own = pack(own_w, nv);
    float best = -INFINITY;
    size_t arg = 0;
    for (size_t c = 0; c < cand.size(); c++) {
        int32_t W[kMaxVars];
        int kf;
        p_chunk_dest(U, cand[c].data(), left, nv, n, d, W, &kf);
        float f[kPolicyFeatures];
        features(U, cand[c].data(), W, kf, left, t, tmax, nv, d, c == 0, others_at(X, t, W, own),
                 overlap_at(X, t, W, own, X.cur_live), f);
        float sc = policy_score(X.net, f);
        if (sc > best) { best = sc; arg = c; }
    }
    for (int q = 0; q < nv; q++) v[q] = cand[arg][q];
    return true;
}

zeta_status reference_contributions(Instance &X) {
    // the game the network plays in, with Algorithm 3 for every choice it would make
    std::function<bool(const int32_t *, int, int, int *)> saved = X.hook;
    X.hook = nullptr;
    zeta_status st = schedule_policy(X, ZETA_POLICY_COVER);
    X.hook = saved;
    if (st) return st;
    const int nv = (int)X.nv;
    const Plan &P = X.plan;
    const int nph = (int)P.phase_begin.size() - 1;
    const int tmax = nph;  // phase i plays level tmax - i
    X.ref_contrib.assign(tmax + 1, {});
    X.ref_cols.assign(tmax + 1, {});
    auto add = [&](int t, uint64_t key, uint64_t live) {
        X.ref_contrib[t][key] += 1;
        auto &cnt = X.ref_cols[t][key];
        for (int col = 0; col < 64; col++)
            if (live >> col & 1ull) cnt[col]++;
    };
    for (int ph = 0; ph + 1 < nph; ph++) {
        const int tn = tmax - ph - 1;  // next level
        std::vector<uint64_t> block_key;
        for (uint32_t e = P.phase_begin[ph + 1]; e < P.phase_begin[ph + 2]; e++) {
            const PlanEntry &E = P.entries[e];
            const uint64_t key = pack(E.U, nv);
            if (E.start_chain >= 0) {
                const Chain &C = X.chains[E.start_chain];
                uint64_t live = 0;
                for (uint32_t t = C.term_begin; t < C.term_end; t++) live |= 1ull << X.terms[t].col;
                add(tn, key, live);
            }
            if (E.arrival >= 0) {
                if ((int)block_key.size() <= E.arrival) block_key.resize(E.arrival + 1, 0);
                block_key[E.arrival] = key;
            }
        }
        for (uint32_t e = P.phase_begin[ph]; e < P.phase_begin[ph + 1]; e++)
            if (P.entries[e].dest >= 0) add(tn, block_key[P.entries[e].dest], P.entries[e].live);
    }
    return ZETA_OK;
}

// Training decisions labelled by rollouts (see the file comment).
zeta_status policy_dataset(Instance &X, std::vector<float> &feat, std::vector<uint32_t> &group_off,
                           std::vector<uint32_t> &labels, std::vector<int32_t> &costs) {
    if (X.nv > 4) { X.error = "the policy features cover at most four variables"; return X.status = ZETA_ERR_UNSUPPORTED; }
    if (X.Smask != (1u << X.nv) - 1) { X.error = "the learned policy takes S = {0..n} only"; return X.status = ZETA_ERR_UNSUPPORTED; }
    zeta_status st = reference_contributions(X);  // what the network sees of U
    if (st) return st;
    const int nv = (int)X.nv, n = (int)X.n, d = (int)X.d, p = (int)X.p;
    int tmax = 0;
    for (const Chain &c : X.chains) tmax = std::max(tmax, ((norm(c.U, nv) - (int)X.base) / d + n) / p);
    auto cost = [](const Plan &P) { return (int64_t)P.column_steps + (int64_t)kChunkCost * (int64_t)P.chunks_played; };
    struct Dec {
        int t, left;
        uint64_t live;
        std::array<int32_t, kMaxVars> U;
    };
    // 1. the cover game with Algorithm 3; its decisions (a term's first call may come from the level's search,
    //    the second from play: both are the same decision)
    std::vector<Dec> decs;
    std::unordered_set<uint64_t> seen;
    std::vector<std::array<int, kMaxVars>> cand;
    X.hook = [&](const int32_t *U, int left, int t, int *) {
        legal_dirs(U, nv, n, d, cand);
        if (cand.size() >= 2) {
            const uint64_t key = (pack(U, nv) << 12) ^ ((uint64_t)left << 6) ^ (uint64_t)t;
            if (seen.insert(key).second) {
                Dec D;
                D.t = t;
                D.left = left;
                D.live = X.cur_live;
                D.U.fill(0);
                for (int q = 0; q < nv; q++) D.U[q] = U[q];
                decs.push_back(D);
            }
        }
        return false;
    };
    st = schedule_policy(X, ZETA_POLICY_COVER);
    X.hook = nullptr;
    if (st) return st;
    const int64_t base_cost = cost(X.plan);
    // 2. every legal direction of a sample of the decisions, each in a rollout of the whole game
    group_off.assign(1, 0);
    const size_t stride = std::max<size_t>(1, (decs.size() + kDatasetDecisions - 1) / kDatasetDecisions);
    for (size_t di = 0; di < decs.size(); di += stride) {
        const Dec &D = decs[di];
        std::vector<std::array<int, kMaxVars>> cands;
        legal_dirs(D.U.data(), nv, n, d, cands);
        std::vector<int64_t> c_of(cands.size(), base_cost);
        for (size_t c = 1; c < cands.size(); c++) {
            X.hook = [&](const int32_t *U, int left, int t, int *v) {
                if (t != D.t || left != D.left) return false;
                for (int q = 0; q < nv; q++)
                    if (U[q] != D.U[q]) return false;
                for (int q = 0; q < nv; q++) v[q] = cands[c][q];
                return true;
            };
            st = schedule_policy(X, ZETA_POLICY_COVER);
            X.hook = nullptr;
            if (st) return st;
            c_of[c] = cost(X.plan);
        }
        size_t lab = 0;
        for (size_t c = 1; c < cands.size(); c++)
            if (c_of[c] < c_of[lab]) lab = c;
        int32_t own_w[kMaxVars];
        int kf0;
        p_chunk_dest(D.U.data(), cands[0].data(), D.left, nv, n, d, own_w, &kf0);
        const uint64_t own = pack(own_w, nv);
        for (size_t c = 0; c < cands.size(); c++) {
            int32_t W[kMaxVars];
            int kf;
            p_chunk_dest(D.U.data(), cands[c].data(), D.left, nv, n, d, W, &kf);
            float f[kPolicyFeatures];
            features(D.U.data(), cands[c].data(), W, kf, D.left, D.t, tmax, nv, d, c == 0, others_at(X, D.t, W, own),
                     overlap_at(X, D.t, W, own, D.live), f);
            feat.insert(feat.end(), f, f + kPolicyFeatures);
            costs.push_back((int32_t)std::min<int64_t>(c_of[c] - c_of[lab], INT32_MAX));
        }
        labels.push_back((uint32_t)lab);
        group_off.push_back((uint32_t)(feat.size() / kPolicyFeatures));
    }
    return ZETA_OK;
}

}  // namespace zeta
