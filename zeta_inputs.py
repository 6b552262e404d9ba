"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the reduction method.  It only draws
candidate coefficient vectors of homogeneous forms f in F_p[x_0..x_n]_d from
a counter-based generator (splitmix64, Steele/Lea/Flood 2014) so that every
consumer sees the same candidates.  Whether a candidate is accepted (the
smoothness test of the Jacobian criterion) is decided by the caller's own
predicate: the oracle and the product each bring their own.

Coefficient order: monomials of degree d in n+1 variables in descending
lexicographic order of the exponent vector, x_0 first.  For n = 2, d = 2 this
is x0^2, x0 x1, x0 x2, x1^2, x1 x2, x2^2.
"""
from math import comb

MASK64 = (1 << 64) - 1

PRIMES_QUINTIC_CURVES = (7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47)
PRIMES_K3 = (7, 11, 13)


def splitmix64(state):
    """One step of splitmix64: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class Stream:
    """Counter-based stream keyed by (seed, instance, attempt)."""

    def __init__(self, seed, instance, attempt):
        s = 0
        for word in (seed, instance, attempt):
            s, out = splitmix64(s ^ (word & MASK64))
            s = out
        self.state = s

    def next64(self):
        self.state, out = splitmix64(self.state)
        return out

    def below(self, bound):
        """Uniform integer in [0, bound) by rejection (no modulo bias)."""
        limit = (1 << 64) - ((1 << 64) % bound)
        while True:
            z = self.next64()
            if z < limit:
                return z % bound


def num_monomials(nvars, deg):
    return comb(deg + nvars - 1, nvars - 1)


def dense_candidate(n, d, p, seed, instance, attempt):
    """All C(n+d, n) coefficients uniform in F_p."""
    st = Stream(seed, instance, attempt)
    return [st.below(p) for _ in range(num_monomials(n + 1, d))]


def sparse_candidate(n, d, p, seed, instance, attempt, kmin=4, kmax=8):
    """k in [kmin, kmax] distinct monomials, nonzero coefficients uniform in F_p^*."""
    st = Stream(seed, instance, attempt)
    nm = num_monomials(n + 1, d)
    k = kmin + st.below(kmax - kmin + 1)
    chosen = []
    while len(chosen) < k:
        i = st.below(nm)
        if i not in chosen:
            chosen.append(i)
    coeffs = [0] * nm
    for i in chosen:
        coeffs[i] = 1 + st.below(p - 1)
    return coeffs


def fermat(n, d):
    """x_0^d + ... + x_n^d in the coefficient order above."""
    nm = num_monomials(n + 1, d)
    coeffs = [0] * nm
    # x_i^d sits at the position of the exponent vector d*e_i.
    idx = 0
    pos = []
    for exps in _monomials(n + 1, d):
        if max(exps) == d:
            pos.append(idx)
        idx += 1
    for i in pos:
        coeffs[i] = 1
    return coeffs


def _monomials(nvars, deg):
    if nvars == 1:
        yield (deg,)
        return
    for e0 in range(deg, -1, -1):
        for rest in _monomials(nvars - 1, deg - e0):
            yield (e0,) + rest


# ---------------------------------------------------------------------------
# Workload recipes (shapes and distributions of the paper's examples).
# ---------------------------------------------------------------------------
WORKLOADS = {
    # one dense plane quartic (genus 3) over F_11, seed 0
    "quartic_curve_f11": dict(n=2, d=4, count=1, seed=0),
    # dense plane quintics (genus 6), p cycling over 12 primes
    "quintic_curves": dict(n=2, d=5, count=4096, seed=1),
    # quartic K3 surfaces in P^3 over F_7, F_11, F_13, 10% sparse (4-8 terms)
    "quartic_k3": dict(n=3, d=4, count=512, seed=2),
    # dense quintic surfaces in P^3 over F_7
    "quintic_surfaces": dict(n=3, d=5, count=256, seed=3),
    # dense cubic surfaces in P^3 over F_7, F_11, F_13 (d < n + 1: reduction with S = {3})
    "cubic_surfaces": dict(n=3, d=3, count=1024, seed=4),
}


def instance_shape(workload, i):
    """(n, d, p, sparse) of instance i of a workload."""
    w = WORKLOADS[workload]
    if workload == "quartic_curve_f11":
        return 2, 4, 11, False
    if workload == "quintic_curves":
        return 2, 5, PRIMES_QUINTIC_CURVES[i % len(PRIMES_QUINTIC_CURVES)], False
    if workload == "quartic_k3":
        return 3, 4, PRIMES_K3[i % 3], (i % 10) == 9
    if workload == "quintic_surfaces":
        return 3, 5, 7, False
    if workload == "cubic_surfaces":
        return 3, 3, PRIMES_K3[i % 3], False
    raise KeyError(workload)


def draw_instance(workload, i, accept, max_attempts=100000):
    """First candidate of instance i accepted by `accept(n, d, p, coeffs)`.

    Returns (n, d, p, coeffs, attempts).  `accept` is the caller's smoothness
    test; candidates are drawn in attempt order 0, 1, 2, ...
    """
    n, d, p, sparse = instance_shape(workload, i)
    seed = WORKLOADS[workload]["seed"]
    for attempt in range(max_attempts):
        if sparse:
            c = sparse_candidate(n, d, p, seed, i, attempt)
        else:
            c = dense_candidate(n, d, p, seed, i, attempt)
        if accept(n, d, p, c):
            return n, d, p, c, attempt + 1
    raise RuntimeError("no accepted candidate for %s[%d]" % (workload, i))


# The mixed stream: 64 instances of uneven size for one persistent launch (curves, surfaces, threefolds), as
# (workload, index) pairs of the workloads above, plus diagonal forms ("fermat", (n, d, p)).  The paper's cubic
# fourfolds (s = 3003) are not among them: the library refuses s > 512.
MIXED_STREAM = ([("quartic_curve_f11", 0)] + [("quintic_curves", i) for i in range(24)] +
                [("cubic_surfaces", i) for i in range(16)] + [("quartic_k3", i) for i in range(21)] +
                [("fermat", (4, 3, 7)), ("fermat", (4, 3, 13))])


def draw_mixed(k, accept):
    """Instance k of MIXED_STREAM as (n, d, p, coeffs)."""
    workload, x = MIXED_STREAM[k]
    if workload == "fermat":
        n, d, p = x
        return n, d, p, fermat(n, d)
    return draw_instance(workload, x, accept)[:4]


def random_residues(seed, count, modulus):
    """`count` residues uniform in [0, modulus) (kernel-level parity inputs)."""
    st = Stream(seed, 0xABCDEF, count)
    if modulus <= (1 << 63):
        return [st.below(modulus) for _ in range(count)]
    out = []
    for _ in range(count):
        # compose from 64-bit words, then reject above the largest multiple
        words = (modulus.bit_length() + 63) // 64
        top = 1 << (64 * words)
        limit = top - top % modulus
        while True:
            z = 0
            for _ in range(words):
                z = (z << 64) | st.next64()
            if z < limit:
                out.append(z % modulus)
                break
    return out
