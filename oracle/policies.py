"""Tweak, greedy directions and the reduction policies (oracle; test infrastructure only).

Sec. 3.1 Algorithm 1 (Tweak), Sec. 4 Algorithm 3 (greedy v), the abstract
reduction game of Sec. 3.4 and the three policies of Sec. 4.1-4.3.
Exponent vectors are tuples in N^{n+1}.  A term of pole order K has
|u| = |S| - 1 + d (K - n): its numerator x^u g / x^S, g in Homog_{dn-n}, has
degree dK - n - 1.  For S = {0..n} that is n + d (K - n); the game ends at
|u| = |S| - 1 (pole order n).
"""


def tweak(I, m):
    """Algorithm 1: remove m units from the front of I (lowest index first).

    Returns (I', J) with I = I' + J and |J| = min(m, |I|).
    """
    out = list(I)
    J = [0] * len(I)
    left = m
    for i in range(len(out)):
        if left == 0:
            break
        take = min(out[i], left)
        out[i] -= take
        J[i] += take
        left -= take
    return tuple(out), tuple(J)


def greedy_v(d, u, S):
    """Algorithm 3: v with |v| = d and v <= u, v_s >= 1 for s in S with u_s != 0.

    Readings of the printed algorithm: S is scanned in ascending order, the
    count i is tested before every increment of the round-robin loop, and
    the vector built (v) is what is returned.
    """
    v = [0] * len(u)
    i = d
    for s in sorted(S):
        if u[s] != 0:
            v[s] = 1
            i -= 1
            if i == 0:
                break
    while i > 0:
        progressed = False
        for m in range(len(u)):
            if i > 0 and v[m] < u[m]:
                v[m] += 1
                i -= 1
                progressed = True
        if not progressed:
            raise ValueError("|u| < d: no direction")
    return tuple(v)


def in_V_full(u, v, k, S):
    """v in V_S(u, k) intersected with V_full: |v| = d implied by caller.

    u - k v >= 0, and for i in S: u_i != 0 implies v_i != 0 (the condition
    of Prop. 3.3 on the exponent before the step).
    """
    for i in range(len(u)):
        if u[i] - k * v[i] < 0:
            return False
        if i in S and u[i] != 0 and v[i] == 0:
            return False
    return True


def k_max(u, v, n, d, base=None):
    """Largest k with u - k v >= 0 and |u - k v| >= base (Sec. 4.2); base = |S| - 1,
    n for S = {0..n}."""
    base = n if base is None else base
    k = (sum(u) - base) // d
    for i in range(len(u)):
        if v[i] > 0:
            k = min(k, u[i] // v[i])
    return k


def pole_order(u, n, d, base=None):
    base = n if base is None else base
    return (sum(u) - base) // d + n


def sub_kv(u, v, k):
    return tuple(a - k * b for a, b in zip(u, v))


class GameLog:
    """Cost bookkeeping of the reduction game (Sec. 3.4): M k + S per chunk, D per duplicate."""

    def __init__(self):
        self.chunks = 0
        self.steps = 0          # sum of k over chunks (one per term per pole order)
        self.column_steps = 0   # steps times the number of live columns of the term
        self.merges = 0         # duplicates removed

    def cost(self, cM, cS, cD):
        return cM * self.steps + cS * self.chunks + cD * self.merges


def merge_terms(terms, add, log):
    """Move 2: combine terms with equal u.  terms: list of (u, payload)."""
    out = {}
    order = []
    for u, w in terms:
        if u in out:
            out[u] = add(out[u], w)
            log.merges += 1
        else:
            out[u] = w
            order.append(u)
    return [(u, out[u]) for u in order]


def play(policy, terms, n, d, p, S, reduce_chunk, add, log):
    """Run a policy on the initial term list; returns the terms at pole order n
    (|u| = |S| - 1).

    reduce_chunk(u, v, k, payload) -> payload after k steps in direction v.
    add(a, b) -> merged payload.
    """
    S = set(S)
    base = len(S) - 1
    if policy == "depth_first":
        out = []
        for u, w in terms:
            while sum(u) > base:
                v = greedy_v(d, u, S)
                k = k_max(u, v, n, d, base)
                assert k >= 1 and in_V_full(u, v, k, S)
                w = reduce_chunk(u, v, k, w)
                u = sub_kv(u, v, k)
            out.append((u, w))
        return out
    if policy == "p_chunk":
        # Reading of Sec. 4.1: every term of the largest pole order K is reduced
        # by a chunk of size p (p - n when K = p, i.e. down to pole order n);
        # when the greedy direction admits fewer steps, the chunk is completed
        # with further greedy directions, so all terms stay on pole orders p t.
        live = merge_terms(terms, add, log)
        done = []
        while live:
            L = max(sum(u) for u, _ in live)
            nxt = []
            for u, w in live:
                if sum(u) == L:
                    K = pole_order(u, n, d, base)
                    left = K - max(K - p, n)
                    while left > 0:
                        v = greedy_v(d, u, S)
                        k = min(left, k_max(u, v, n, d, base))
                        assert k >= 1 and in_V_full(u, v, k, S)
                        w = reduce_chunk(u, v, k, w)
                        u = sub_kv(u, v, k)
                        left -= k
                nxt.append((u, w))
            # terms at pole order n leave the game (their numerators are summed
            # by the final reduction); the others are combined
            done += [(u, w) for u, w in nxt if sum(u) == base]
            live = merge_terms([(u, w) for u, w in nxt if sum(u) > base], add, log)
        return done
    if policy == "var_by_var":
        live = merge_terms(terms, add, log)
        done = []
        for t in range(n, -1, -1):
            nxt = []
            for u, w in live:
                while sum(u) > base and u[t] > 0:
                    v = greedy_v(d, u, S)
                    k = k_max(u, v, n, d, base)
                    assert k >= 1 and in_V_full(u, v, k, S)
                    w = reduce_chunk(u, v, k, w)
                    u = sub_kv(u, v, k)
                nxt.append((u, w))
            done += [(u, w) for u, w in nxt if sum(u) == base]
            live = merge_terms([(u, w) for u, w in nxt if sum(u) > base], add, log)
        # after the u_0 phase every term has |u| = |S| - 1
        assert not live
        return done
    raise ValueError("unknown policy %r" % policy)
