"""The setup's right inverses solved on the device (k_right_inverse) against the host's elimination.

Both run Gauss-Jordan over Z/q with unit pivots in column order, the first unit row as pivot (the section of
Prop. 3.3 and the final reduction's levels, Sec. 3.3 step (2)); with exact arithmetic the section and the final
reduction map must agree word for word.  Batches whose setup is solved either way must return the same P(T)
and the same statuses, including ZETA_ERR_NOT_SMOOTH for two smooth cubic surfaces that are not {3}-smooth.
"""
import os
import time

import numpy as np
import pytest

import zeta_inputs as zi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
z = pytest.importorskip("paper_2602_24155_gb300")

GOLDEN_3FOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cubic_threefold_f11.txt")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = z.zeta_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    z.zeta_destroy(c)


def _accept(n, d, p, c):
    try:
        z.zeta_query((n, d, p, c))
        return True
    except z.ZetaError:
        return False


def _threefold():
    out = {}
    for line in open(GOLDEN_3FOLD):
        if line.startswith("#") or ":" not in line:
            continue
        key, _, val = line.partition(":")
        out[key.strip()] = val.strip()
    n, d, p = map(int, out["n d p"].split())
    return n, d, p, [int(x) for x in out["coeffs"].split()]


CASES = [("quintic_curves", 11), ("quintic_curves", 0), ("cubic_surfaces", 1), ("quartic_k3", 9), ("quartic_k3", 2)]


@pytest.mark.parametrize("workload,i", CASES)
def test_device_right_inverses_equal_the_host(ctx, workload, i):
    n, d, p, c, _ = zi.draw_instance(workload, i, _accept)
    host = z.zeta_plan((n, d, p, c), policy="p_chunk")
    sec, fin, ms = z.zeta_plan_device(ctx, (n, d, p, c), policy="p_chunk")
    assert sec.shape == host["sec"].shape and np.array_equal(sec, host["sec"])
    assert fin.shape == host["fin"].shape and np.array_equal(fin, host["fin"])
    assert ms > 0


def test_device_right_inverses_dense_cubic_threefold(ctx):
    spec = _threefold()
    t0 = time.time()
    host = z.zeta_plan(spec, policy="p_chunk")
    t_host = time.time() - t0
    t0 = time.time()
    sec, fin, ms = z.zeta_plan_device(ctx, spec, policy="p_chunk")
    t_dev = time.time() - t0
    print("dense cubic threefold over F_11: host plan %.2f s, device-solved plan %.2f s (solve kernel %.1f ms)"
          % (t_host, t_dev, ms))
    assert sec.shape == (2475, 1001)
    assert np.array_equal(sec, host["sec"]) and np.array_equal(fin, host["fin"])
    assert _section_identity_ok(spec, sec, host["kappa"], host["q"], [0, 500, 1000])


def test_batches_agree_with_host_and_device_setup(ctx):
    specs = [zi.draw_instance("quintic_curves", i, _accept)[:4] for i in range(6)]
    specs += [zi.draw_instance("cubic_surfaces", i, _accept)[:4] for i in range(4)]
    specs.append((3, 3, 7, zi.dense_candidate(3, 3, 7, 4, 1002, 0)))   # smooth, not {3}-smooth
    specs.append((3, 3, 7, zi.dense_candidate(3, 3, 7, 4, 1006, 0)))   # smooth, not {3}-smooth
    out = {}
    for setup in ("host", "device"):
        P, per, tot = z.zeta_batch(ctx, specs, policy="p_chunk", setup=setup)
        out[setup] = (P, [r["status"] for r in per])
    assert out["host"][1] == out["device"][1]
    assert out["device"][1][-2:] == [2, 2]
    assert all(st == 0 for st in out["device"][1][:-2])
    for a, b, st in zip(out["host"][0], out["device"][0], out["device"][1]):
        if st == 0:
            assert a == b


def _monos(nv, D):
    out = []
    def rec(pos, rem, cur):
        if pos == nv - 1:
            out.append(tuple(cur + [rem]))
            return
        for t in range(rem, -1, -1):
            rec(pos + 1, rem - t, cur + [t])
    if D >= 0:
        rec(0, D, [])
    return out


def _section_identity_ok(spec, sec, kappa, q, cols):
    """For each sampled column gamma of the section: sum_i G_i d_i f = x^gamma mod q, G_i from the rows (i, nu)."""
    n, d, p, c = spec
    nv = n + 1
    md = _monos(nv, d)
    f = {m: cf for m, cf in zip(md, c) if cf}
    df = []
    for i in range(nv):
        g = {}
        for m, cf in f.items():
            if m[i]:
                e = list(m); e[i] -= 1
                g[tuple(e)] = (g.get(tuple(e), 0) + cf * m[i]) % q
        df.append(g)
    src = _monos(nv, kappa - d + 1)
    rows = _monos(nv, kappa)
    for gcol in cols:
        acc = {}
        for i in range(nv):
            for a, nu in enumerate(src):
                v = int(sec[i * len(src) + a, gcol])
                if not v:
                    continue
                for m, cf in df[i].items():
                    e = tuple(x + y for x, y in zip(nu, m))
                    acc[e] = (acc.get(e, 0) + v * cf) % q
        want = rows[gcol]
        for e, v in acc.items():
            if v != (1 if e == want else 0):
                return False
        if acc.get(want, 0) != 1:
            return False
    return True


def test_device_right_inverses_dense_cubic_fourfold(ctx):
    """The dense cubic fourfold of tests/golden/cubic_fourfold_f7.txt (C(15, 5) = 3003; the host refuses its setup):
    its section (18 018 x 6188 over Z/7^9, from a 6188 x 24 206 elimination) and final map from the device, with
    A x Sec = I checked on sampled columns of the section (the map of J_S applied to column gamma gives x^gamma)."""
    c = zi.dense_candidate(5, 3, 7, 5, 76, 0)
    spec = (5, 3, 7, c)
    t0 = time.time()
    sec, fin, ms = z.zeta_plan_device(ctx, spec, policy="p_chunk", r=1)
    print("dense cubic fourfold: section %s and final map %s in %.1f s, solve kernels %.0f ms"
          % (sec.shape, fin.shape, time.time() - t0, ms))
    assert sec.shape == (6 * 3003, 6188) and fin.shape == (22, 2002)
    assert sec.any() and fin.any()
    assert _section_identity_ok(spec, sec, 12, 7 ** 9, [0, 3001, 6187])
