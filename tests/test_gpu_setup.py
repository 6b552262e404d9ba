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
