"""The whole-GPU executor (zeta_large.cuh) against the persistent executors, and the cubic fourfold it is built for.

 - Quintic curves, cubic surfaces (S = {3}), a K3 surface and a cubic threefold (S = {4}) at relative precision 1:
   the same batch run with ZETA_FLAG_WHOLE_GPU and without gives the same P(T) word for word (the same plan in exact
   arithmetic, so the same numerators H).
 - The Fermat cubic fourfold over F_7 (s = C(15, 5) = 3003, b = 22, S = {5}) at relative precision 1 (M = 9): its
   P(T) agrees with Weil's Gauss-sum closed form (computed without any of the reduction) modulo p^(1 + H(i)) in
   every coefficient, H the Hodge polygon (0, 1, 3, ..., 41, 44); its height is 1 (p = 1 mod 3: ordinary).
"""
import os

import pytest

import zeta_inputs as zi
from oracle import pins

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


def test_whole_gpu_executor_equals_the_persistent_ones(ctx):
    specs = [zi.draw_instance("quintic_curves", i, _accept)[:4] for i in (0, 5, 11)]
    specs += [zi.draw_instance("cubic_surfaces", i, _accept)[:4] for i in (0, 1)]
    specs.append(zi.draw_instance("quartic_k3", 9, _accept)[:4])
    specs.append(_threefold())
    P0, per0, tot0 = z.zeta_batch(ctx, specs, policy="p_chunk", r=1)
    P1, per1, tot1 = z.zeta_batch(ctx, specs, policy="p_chunk", r=1, whole_gpu=True)
    assert [x["status"] for x in per0] == [0] * len(specs)
    assert [x["status"] for x in per1] == [0] * len(specs)
    assert P0 == P1
    assert tot1["column_steps"] == tot0["column_steps"]
    print("whole-GPU executor: %d launches, %.1f ms; persistent: %.1f ms"
          % (tot1["kernel_launches"], tot1["ms_kernel"], tot0["ms_kernel"]))


def test_fermat_cubic_fourfold_f7_relative_precision_one(ctx):
    from paper_2602_24155_gb300.newton import fourfold_height, hodge_polygon
    n, d, p = 5, 3, 7
    P, per, tot = z.zeta_batch(ctx, [(n, d, p, zi.fermat(n, d))], policy="p_chunk", r=1)
    st = per[0]
    print("Fermat cubic fourfold over F_7, r = 1: status %d, s %d, b %d, M %d; %d chunks, %d steps, %d column steps; "
          "setup %.0f ms, kernels %.0f ms in %d launches" % (st["status"], st["s"], st["b"], st["M"], tot["chunks"],
                                                            tot["steps"], tot["column_steps"], tot["ms_host_setup"],
                                                            tot["ms_kernel"], tot["kernel_launches"]))
    assert st["status"] == 0 and st["s"] == 3003 and st["b"] == 22 and st["M"] == 9
    exact = pins.fermat_charpoly(n, d, p)
    H = hodge_polygon(n, d)
    assert len(P[0]) == len(exact) == 23 and P[0][0] == 1
    for i in range(1, 23):
        mod = p ** (1 + H[i])
        assert (P[0][i] - exact[i]) % mod == 0, i
    assert fourfold_height(P[0], p) == 1


def test_every_run_of_a_prepared_batch_launches_again(ctx):
    """zeta_batch_run may be called again on a plan and runs the batch again each time (how the bench times
    resident inputs): three runs of a batch holding a persistent-executor instance and a whole-GPU one give the
    same P(T) as one, with three persistent launches."""
    specs = [zi.draw_instance("quintic_curves", i, _accept)[:4] for i in (0, 1)]
    specs.append((3, 5, 11, zi.fermat(3, 5)))          # b = 52: the whole-GPU executor
    plan = z.zeta_batch_prepare(ctx, specs, policy="p_chunk", r=1)
    plan.run()
    P1, _, tot1 = plan.finish()
    for _ in range(3):
        plan.run()
    P3, _, tot3 = plan.finish()
    plan.release()
    assert P1 == P3
    assert tot3["kernel_launches"] > tot1["kernel_launches"] and tot3["ms_kernel"] > tot1["ms_kernel"]


def test_pipelined_batch_with_device_setup_equals_one_plan(ctx):
    """zeta_batch on 256 instances or more splits them into sub-batches; when one holds an instance with s > 128 the
    setup's right inverses of all sub-batches are solved on the device before the first launch.  256 quartic K3
    surfaces at relative precision 1 through that path give the same P(T) and statuses as one prepared plan."""
    def accept(n, d, p, c):
        try:
            z.zeta_query((n, d, p, c), r=1)
            return True
        except z.ZetaError as e:
            if e.status == 2:
                return False
            raise
    specs = [zi.draw_instance("quartic_k3", i, accept)[:4] for i in range(256)]
    P1, per1, _ = z.zeta_batch(ctx, specs, policy="p_chunk", r=1)
    plan = z.zeta_batch_prepare(ctx, specs, policy="p_chunk", r=1)
    plan.run()
    P2, per2, _ = plan.finish()
    plan.release()
    assert [st["status"] for st in per1] == [st["status"] for st in per2] == [0] * 256
    assert P1 == P2


def test_single_instance_call_on_a_cubic_fourfold(ctx):
    """zeta_frobenius on an instance with C(dn, n) > 512 solves its right inverses on the device and runs it on the
    whole-GPU executor: the Fermat cubic fourfold at series order 2 (a short plan; the columns Y are a truncation)
    gives the same Y under two policies, as Y depends on neither."""
    spec = (5, 3, 7, zi.fermat(5, 3))
    F1, Y1, st1 = z.zeta_frobenius(ctx, spec, r=1, N=2, y_only=True, policy="p_chunk")
    F2, Y2, st2 = z.zeta_frobenius(ctx, spec, r=1, N=2, y_only=True, policy="depth_first")
    assert st1["s"] == 3003 and st1["b"] == 22 and st1["column_steps"] != st2["column_steps"]
    assert (Y1 == Y2).all() and Y1.any()
