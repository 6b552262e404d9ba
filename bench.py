"""Benchmark: zeta functions of a batch of smooth plane quintics on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--policy depth_first] [--path vector]

A step is one pass of the whole hot path over one batch: every reduction
chain of every instance run to pole order n by the recurrence kernel, then
the per-instance sums.  `value` is zeta functions per second with the
inputs (start terms, sections, tables: larger than L2) resident in HBM;
`e2e` is the same metric through zeta_batch with host buffers (host setup,
uploads, kernels, download and host finish all inside the timed region).
Under torchrun every rank runs its own batch of the same size (weak
scaling, no collective on the data path).  `--impl reference` times the
CPU oracle on a bounded sample of the same workload on the host cores.
"""
import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import zeta_inputs as zi  # noqa: E402

METRIC = "exact zeta funcs/s + reduction steps/s mod p^N on 1 GB300; learned vs plain policy"

# DRAM bytes (read + written) per instance of the executor k_execute on the quintic-curve workload under the
# learned policy: dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of the current kernels on 456
# instances of the workload (bench.py --count 456 --path vector), scaled by the instance count; traffic grows in
# proportion to the instances (the merge blocks and inputs of each are written and read once).
DRAM_BYTES_PER_INSTANCE = (2.312358e9 + 2.177106e9) / 456
WORKLOAD = "quintic_curves"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _instances(rank, count):
    """Instances rank*count .. rank*count+count-1 of the quintic-curve workload, filtered by the oracle's
    smoothness test: for the reference arm (the oracle) and the multi-process tests only; the timed path draws
    the same instances through the library (_instances_lib)."""
    from oracle.cohomology import is_smooth  # the oracle's smoothness predicate only filters
    out = []
    for i in range(rank * count, rank * count + count):
        n, d, p, c, _ = zi.draw_instance(WORKLOAD, i, is_smooth)
        out.append((n, d, p, c))
    return out


def _instances_range(start, count, z):
    """Instances start .. start+count-1, accepted by the library's own smoothness test."""
    def accept(n, d, p, c):
        try:
            z.zeta_query((n, d, p, c))
            return True
        except z.ZetaError as e:
            if e.status == 2:
                return False
            raise
    return [zi.draw_instance(WORKLOAD, i, accept)[:4] for i in range(start, start + count)]


def _instances_lib(rank, count, z):
    return _instances_range(rank * count, count, z)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.index = index
        # raw samples (the JSON line carries their summary); directory from ZETA_BENCH_OUT
        out_dir = os.environ.get("ZETA_BENCH_OUT", os.path.join(ROOT, "bench_out"))
        self.path = os.path.join(out_dir, "clocks_rank%d.csv" % index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_one(spec):
    from oracle import zeta as oz
    n, d, p, c = spec
    t = time.perf_counter()
    res = oz.compute_zeta(n, d, p, c)
    return time.perf_counter() - t, res.log.column_steps, res.P


def oracle_sample(specs, cores):
    """Time the oracle on `specs` with one process per instance over `cores` processes."""
    from oracle import zeta as oz
    oz.build_helper()
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_one, specs)
    wall = time.perf_counter() - t0
    return wall, res


def _workload_config(count):
    """The workload of the main line, shared by both arms so that they name the same config."""
    return {"workload": "quintic_curves_4096", "n": 2, "d": 5, "count_per_gpu": count,
            "primes": list(zi.PRIMES_QUINTIC_CURVES), "l2": "inputs larger than L2 (HBM-resident)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    sample_n = max(1, min(cores, 16))
    specs = _instances(0, sample_n)
    # warm-up: the same process pool on the genus-3 quartic over F_11 (module imports, the C helper, the pool)
    from oracle.cohomology import is_smooth
    small = zi.draw_instance("quartic_curve_f11", 0, is_smooth)[:4]
    for _ in range(args.warmup):
        oracle_sample([small] * min(cores, sample_n), cores)
    walls = []
    steps = 0
    for _ in range(max(1, args.steps)):
        wall, res = oracle_sample(specs, cores)
        walls.append(wall)
        steps = sum(r[1] for r in res)
    wall = statistics.median(walls)
    value = sample_n / wall
    sample = ("first %d instances of %s (primes %s), %d processes, oracle as it stands; each warm-up step runs "
              "the pool on the genus-3 quartic over F_11" % (
                  sample_n, WORKLOAD, sorted(set(s[2] for s in specs)), min(cores, sample_n)))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "zeta/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int (exact big integers)", "data": "synthetic",
        "steps_per_s": steps / wall,
        "config": _workload_config(args.count),
        "cpu_baseline": {"value": value, "unit": "zeta/s", "cores": min(cores, sample_n), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "zeta/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _k3_survey(z, ctx, stream, torch):
    """The 512 quartic K3 surfaces over F_7, F_11, F_13 (every tenth sparse) at relative precision 1 in one persistent
    launch: a_i mod p^i, which decides every finite height (paper_2602_24155_gb300.newton.k3_height)."""
    from paper_2602_24155_gb300.newton import k3_height

    def accept(n, d, p, c):
        try:
            z.zeta_query((n, d, p, c))
            return True
        except z.ZetaError as e:
            if e.status == 2:
                return False
            raise
    count = zi.WORKLOADS["quartic_k3"]["count"]
    specs = [zi.draw_instance("quartic_k3", i, accept)[:4] for i in range(count)]
    plan = z.zeta_batch_prepare(ctx, specs, policy="p_chunk", r=1)
    plan.run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.run()
    e1.record(stream)
    torch.cuda.synchronize()
    P, per, tot = plan.finish()
    plan.release()
    ms = e0.elapsed_time(e1)
    hist = {}
    for (n, d, p, c), Pi in zip(specs, P):
        h = "failed" if Pi is None else (k3_height(Pi, p) or "inf")
        hist[str(h)] = hist.get(str(h), 0) + 1
    return {"workload": "quartic_k3_%d" % count, "primes": [7, 11, 13], "precision": "r = 1 (a_i mod p^i)",
            "s": 220, "b": 21, "ms_per_launch": ms, "instances_per_s": count / (ms / 1000.0), "launches": 1,
            "column_steps": tot["column_steps"], "heights": dict(sorted(hist.items()))}


def _k3_full(z, ctx, stream, torch, count, N=0):
    """Quartic K3 surfaces (n = 3, d = 4: s = 220, b = 21) over F_7, F_11, F_13 (every tenth sparse) at the full
    precision of the library's rules, the first `count` of the 512-surface workload in one persistent launch on
    thread-block clusters (each cluster reduces one surface; its CTAs hold row slices of the step matrices)."""

    def accept(n, d, p, c):
        try:
            z.zeta_query((n, d, p, c))
            return True
        except z.ZetaError as e:
            if e.status == 2:
                return False
            raise
    specs = [zi.draw_instance("quartic_k3", i, accept)[:4] for i in range(count)]
    t0 = time.perf_counter()
    # N > 0: every series order truncated to N (a small case for profiling; P(T) is then not the zeta function)
    plan = z.zeta_batch_prepare(ctx, specs, policy="p_chunk", **(dict(N=N, r=4, y_only=True) if N else {}))
    setup_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.run()
    e1.record(stream)
    torch.cuda.synchronize()
    P, per, tot = plan.finish()
    plan.release()
    ms = e0.elapsed_time(e1)
    s = 220
    ok = sum(1 for x in per if x["status"] == 0)
    heights = {}
    from paper_2602_24155_gb300.newton import k3_height
    for (n, d, p, c), Pi in zip(specs, P):
        h = "failed" if Pi is None else (k3_height(Pi, p) or "inf")
        heights[str(h)] = heights.get(str(h), 0) + 1
    # every modulus here is below 2^56: four mad.wide.u32 per modular multiply-add (28-bit limbs)
    madw = 4 * tot["column_steps"] * s * s
    peak = 152 * 64 * 2070.0 * 1e6 / 1e12
    achieved = madw / (ms / 1000.0) / 1e12
    return {"workload": "quartic_k3_%d of 512" % count, "primes": [7, 11, 13],
            "precision": ("full (r_m, N_m of the library's rules; exact P(T) of degree 21)" if not N else
                          "truncated: N_m = %d, r = 4, unnormalised columns only (profiling case)" % N),
            "s": s, "b": 21, "ms_per_launch": ms,
            "zeta_per_s": count / (ms / 1000.0), "launches": 1, "completed": "%d/%d" % (ok, count),
            "column_steps": tot["column_steps"], "column_steps_per_s": tot["column_steps"] / (ms / 1000.0),
            "modmac_per_s": tot["column_steps"] * s * s / (ms / 1000.0), "host_setup_s": setup_s,
            "heights": dict(sorted(heights.items())),
            "roofline": {"bound": "alu", "kernel": "k_execute_cluster", "achieved": achieved, "peak": peak,
                         "unit": "T mad.wide.u32/s", "frac": achieved / peak,
                         "peak_basis": "152 SM x 64 mad.wide.u32/clk at 2070 MHz (nominal); 4 per modular "
                                       "multiply-add (28-bit limbs, q < 2^56)"}}


def _mixed_stream(z, ctx, stream, torch):
    """The 64-instance mixed stream of zeta_inputs.MIXED_STREAM (a quartic curve, 24 quintic curves, 16 cubic
    surfaces, 21 quartic K3 surfaces and two Fermat cubic threefolds: s = 28 ... 495) at full precision in one
    persistent launch; per-instance device latency from the kernel's own %globaltimer stamps."""

    def accept(n, d, p, c):
        try:
            z.zeta_query((n, d, p, c))
            return True
        except z.ZetaError as e:
            if e.status == 2:
                return False
            raise
    specs = [zi.draw_mixed(k, accept) for k in range(len(zi.MIXED_STREAM))]
    plan = z.zeta_batch_prepare(ctx, specs, policy="p_chunk")
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.run()
    e1.record(stream)
    torch.cuda.synchronize()
    P, per, tot = plan.finish()
    plan.release()
    ms = e0.elapsed_time(e1)
    lat = sorted(st["ms_dev_end"] for st in per)

    def pct(q):
        return lat[min(len(lat) - 1, int(q * len(lat)))]
    by_class = {}
    for (n, d, p, c), st in zip(specs, per):
        key = "n%d_d%d_s%d" % (n, d, st["s"])
        by_class.setdefault(key, []).append(st["ms_dev_end"] - st["ms_dev_start"])
    return {"workload": "mixed_stream_64", "composition": "1 quartic curve, 24 quintic curves, 16 cubic surfaces, "
            "21 quartic K3 surfaces, 2 Fermat cubic threefolds (no cubic fourfolds: s = 3003 is refused)",
            "precision": "full", "launches": tot["kernel_launches"], "ms_per_launch": ms,
            "zeta_per_s": len(specs) / (ms / 1000.0),
            "completed": "%d/%d" % (sum(1 for st in per if st["status"] == 0), len(specs)),
            "latency_ms": {"p50": pct(0.5), "p99": pct(0.99), "max": lat[-1],
                           "meaning": "device time from the launch's first block start to the instance's "
                                      "numerators written back"},
            "busy_ms_median_by_class": {k: statistics.median(v) for k, v in sorted(by_class.items())}}


def _mixed_stream_r1(z, ctx, stream, torch):
    """A 64-instance stream at relative precision 1 with every size the library takes: the mixed stream's quartic
    curve, 24 quintic curves, 16 cubic surfaces, the first 16 of its K3 surfaces and its 2 Fermat cubic threefolds in
    one persistent launch, then 4 quintic surfaces (b = 52) and the Fermat cubic fourfold (s = 3003) on the whole-GPU
    executor, all from one zeta_batch_run.  Latency per instance: device time inside the persistent launch (cluster
    executor stamps) for the first 59, host time after the run call for the other 5."""
    accept = _accept_r1(z)
    ks = list(range(1 + 24 + 16 + 16)) + [len(zi.MIXED_STREAM) - 2, len(zi.MIXED_STREAM) - 1]
    specs = [zi.draw_mixed(k, accept) for k in ks]
    specs += [zi.draw_instance("quintic_surfaces", i, accept)[:4] for i in range(4)]
    specs.append((5, 3, 7, zi.fermat(5, 3)))
    plan = z.zeta_batch_prepare(ctx, specs, policy="p_chunk", r=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.run()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    P, per, tot = plan.finish()
    plan.release()
    lat = sorted(st["ms_dev_end"] for st in per)

    def pct(q):
        return lat[min(len(lat) - 1, int(q * len(lat)))]
    by_class = {}
    for (n, d, p, c), st in zip(specs, per):
        key = "n%d_d%d_s%d_b%d" % (n, d, st["s"], st["b"])
        by_class.setdefault(key, []).append(st["ms_dev_end"])
    return {"workload": "mixed_stream_64_r1", "composition": "1 quartic curve, 24 quintic curves, 16 cubic "
            "surfaces, 16 quartic K3 surfaces, 2 Fermat cubic threefolds (persistent launch), 4 quintic surfaces "
            "and the Fermat cubic fourfold (whole-GPU executor)", "precision": "relative precision r = 1",
            "wall_s": wall, "zeta_per_s": len(specs) / wall,
            "completed": "%d/%d" % (sum(1 for st in per if st["status"] == 0), len(specs)),
            "latency_ms": {"p50": pct(0.5), "p99": pct(0.99), "max": lat[-1],
                           "meaning": "completion after the run call: device clock inside the persistent launch, "
                                      "host clock on the whole-GPU executor"},
            "completion_ms_median_by_class": {k: statistics.median(v) for k, v in sorted(by_class.items())}}


def _accept_r1(z):
    def accept(n, d, p, c):
        try:
            z.zeta_query((n, d, p, c), r=1)
            return True
        except z.ZetaError as e:
            if e.status == 2:
                return False
            raise
    return accept


def _quintic_surfaces(z, ctx, stream, torch, count, train_count):
    """Dense quintic surfaces over F_7 (n = 3, d = 5: b = 52 columns, s = 455) at relative precision 1 (M = 3: P(T)
    mod p, the unit-root part; the full precision needs p^M = 7^49, beyond 64-bit residues), on the whole-GPU
    executor, with the learned policy (a network trained here on rollouts of the surfaces' own cover games, indices
    past the batch) against the method without it (cover) and p-chunk.  P(T) mod p of these surfaces equals the
    Hasse-Witt closed form in tests/test_gpu_quintic_surfaces.py."""
    from paper_2602_24155_gb300.newton import unit_roots_mod_p
    from paper_2602_24155_gb300.policy_train import train_policy
    accept = _accept_r1(z)
    specs = [zi.draw_instance("quintic_surfaces", i, accept)[:4] for i in range(count)]
    train = [zi.draw_instance("quintic_surfaces", 100000 + i, accept)[:4] for i in range(train_count)]
    t0 = time.perf_counter()
    weights, loss, decisions = train_policy(ctx, train, hidden=8, epochs=60, opt=dict(r=1))
    out = {"workload": "quintic_surfaces_%d" % count, "precision": "relative precision r = 1 (M = 3)",
           "training": {"instances": train_count, "decisions": decisions, "loss": loss,
                        "s": time.perf_counter() - t0}}
    P_ref = None
    for pol in ("learned", "cover", "p_chunk"):
        o = dict(policy=pol, r=1)
        if pol == "learned":
            o.update(weights=weights, hidden=8)
        plan = z.zeta_batch_prepare(ctx, specs, **o)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run()
        e1.record(stream)
        torch.cuda.synchronize()
        P, per, tot = plan.finish()
        plan.release()
        ms = e0.elapsed_time(e1)
        if P_ref is None:
            P_ref = P
        assert P == P_ref, "policies disagree"
        out[pol] = {"zeta_per_s": len(specs) / (ms / 1000.0), "ms": ms, "column_steps": tot["column_steps"],
                    "chunks": tot["chunks"], "steps": tot["steps"], "kernel_launches": tot["kernel_launches"],
                    "ms_host_setup": tot["ms_host_setup"]}
    out["network_gain_over_cover"] = {
        "column_steps": 1 - out["learned"]["column_steps"] / out["cover"]["column_steps"],
        "time": 1 - out["learned"]["ms"] / out["cover"]["ms"]}
    hist = {}
    for P in P_ref:
        k = unit_roots_mod_p(P, 7)
        hist[k] = hist.get(k, 0) + 1
    out["unit_roots_histogram"] = dict(sorted(hist.items()))
    return out


def _cubic_fourfolds(z, ctx, stream, torch, dense, N=0):
    """Cubic fourfolds over F_7 (n = 5, d = 3: s = C(15, 5) = 3003, b = 22, S = {5}) at relative precision 1 (M = 9;
    the full precision needs 7^25, beyond 64-bit residues) on the whole-GPU executor: the Fermat cubic fourfold and,
    with `dense`, the dense one of tests/golden/cubic_fourfold_f7.txt (dense_candidate seed 5, instance 76).  The
    height (first slope 2 - 1/h) is what relative precision 1 decides.  Checks: tests/test_gpu_whole.py (Gauss-sum
    closed form) and tests/test_gpu_fourfold.py (point counts over F_7 and F_49)."""
    from paper_2602_24155_gb300.newton import fourfold_height
    cases = [("fermat", zi.fermat(5, 3))]
    if dense:
        cases.append(("dense_seed5_76", zi.dense_candidate(5, 3, 7, 5, 76, 0)))
    out = {}
    for name, c in cases:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P, per, tot = z.zeta_batch(ctx, [(5, 3, 7, c)], policy="p_chunk", r=1, **({"N": N, "y_only": True} if N else {}))
        wall = time.perf_counter() - t0
        out[name] = {"status": per[0]["status"], "wall_s": wall, "ms_host_setup": tot["ms_host_setup"],
                     "ms_kernel": tot["ms_kernel"], "kernel_launches": tot["kernel_launches"],
                     "chunks": tot["chunks"], "steps": tot["steps"], "column_steps": tot["column_steps"],
                     "column_steps_per_s": tot["column_steps"] / (tot["ms_kernel"] / 1000.0),
                     "modmac_per_s": tot["column_steps"] * 3003.0 * 3003.0 / (tot["ms_kernel"] / 1000.0),
                     "height": fourfold_height(P[0], 7) if P[0] and not N else None}
    return out


def _cubic_survey(z, ctx, stream, torch):
    """1024 dense cubic surfaces over F_7, F_11, F_13 at full precision in one persistent launch: d = 3 < n + 1, so
    the reduction runs with S = {3} (Prop. 3.3 for a smaller index set; same kernel, section of J_S).  Parity with
    the oracle, point counts and the Gauss-sum closed form is in tests/test_gpu_general_s.py."""

    def accept(n, d, p, c):
        try:
            z.zeta_query((n, d, p, c))       # smooth and {3}-smooth
            return True
        except z.ZetaError as e:
            if e.status == 2:
                return False
            raise
    count = zi.WORKLOADS["cubic_surfaces"]["count"]
    specs = [zi.draw_instance("cubic_surfaces", i, accept)[:4] for i in range(count)]
    s = 84
    alu_peak = 152 * 64 * 2070.0 * 1e6 / 1e12      # mad.wide.u32 at the maximum SM clock, as the main line

    def timed(policy):
        plan = z.zeta_batch_prepare(ctx, specs, policy=policy)
        plan.run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run()
        e1.record(stream)
        torch.cuda.synchronize()
        P, per, tot = plan.finish()
        plan.release()
        ms = e0.elapsed_time(e1)
        ok = sum(1 for x in per if x["status"] == 0)
        # every modulus here is below 2^56: four mad.wide.u32 per modular multiply-add
        achieved = 4 * tot["column_steps"] * s * s / (ms / 1000.0) / 1e12
        return P, {"policy": policy, "ms_per_launch": ms, "zeta_per_s": count / (ms / 1000.0), "launches": 1,
                   "column_steps": tot["column_steps"], "completed": "%d/%d" % (ok, count),
                   "ms_host_setup": tot["ms_host_setup"],
                   "modmac_per_s": tot["column_steps"] * s * s / (ms / 1000.0),
                   "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "T mad.wide.u32/s",
                                "frac": achieved / alu_peak}}
    P, line = timed("p_chunk")
    out = {"workload": "cubic_surfaces_%d" % count, "primes": [7, 11, 13], "S": [3], "s": s, "b": 6}
    out.update(line)
    try:
        P_cover, line_cover = timed("cover")
        line_cover["same_P_as_p_chunk"] = P_cover == P
        out["cover"] = line_cover
    except Exception as exc:    # reported, never a reason to lose the p-chunk line
        out["cover"] = {"error": repr(exc)[:200]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--policy", default="learned",
                    help="learned (trained here on instances disjoint from the batch; it plays on the cover levels), "
                         "cover, p_chunk, depth_first, var_by_var")
    ap.add_argument("--train-count", type=int, default=96)
    ap.add_argument("--path", default="auto", choices=["auto", "vector", "gemm"],
                    help="auto: the autotuner times the launch configurations on a sample of the batch first")
    ap.add_argument("--count", type=int, default=zi.WORKLOADS[WORKLOAD]["count"])
    ap.add_argument("--policy-count", type=int, default=1024,
                    help="instances of the sub-batch on which every policy is timed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-k3", action="store_true", help="skip the K3 height survey (512 surfaces, precision 1)")
    ap.add_argument("--k3-count", type=int, default=76,
                    help="quartic K3 surfaces of the 512-surface workload run at full precision (0: skip)")
    ap.add_argument("--k3-N", type=int, default=0,
                    help="truncate the K3 line's series orders to N (small profiling case; 0 = full precision)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 64-instance mixed stream")
    ap.add_argument("--no-fourfold", action="store_true", help="skip the cubic fourfold line (Fermat, r = 1)")
    ap.add_argument("--only", default=None, choices=["fourfold", "surfaces", "mixed_r1"],
                    help="run only this line (profiling a small case of its kernels) and print it")
    ap.add_argument("--fourfold-N", type=int, default=0,
                    help="series order override of the --only fourfold run (a small case; 0 = the rule)")
    ap.add_argument("--fourfold-dense", action="store_true",
                    help="add the dense cubic fourfold to the fourfold line (several minutes)")
    ap.add_argument("--surface-count", type=int, default=256,
                    help="quintic surfaces over F_7 at r = 1 with learned / cover / p-chunk (0 = skip)")
    ap.add_argument("--no-cubic", action="store_true",
                    help="skip the cubic-surface line (1024 surfaces, S = {3}, full precision)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    import paper_2602_24155_gb300 as z

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    stream = torch.cuda.current_stream()
    ctx = z.zeta_create(local, stream.cuda_stream)
    if args.only == "fourfold":
        print(json.dumps({"cubic_fourfolds": _cubic_fourfolds(z, ctx, stream, torch, args.fourfold_dense,
                                                              args.fourfold_N)}))
        z.zeta_destroy(ctx)
        return
    if args.only == "mixed_r1":
        print(json.dumps({"mixed_stream_r1": _mixed_stream_r1(z, ctx, stream, torch)}))
        z.zeta_destroy(ctx)
        return
    if args.only == "surfaces":
        print(json.dumps({"quintic_surfaces": _quintic_surfaces(z, ctx, stream, torch, args.surface_count, 24)}))
        z.zeta_destroy(ctx)
        return
    specs = _instances_lib(rank, args.count, z)
    opt = dict(policy=args.policy, path=args.path)
    learned = None
    if args.policy == "learned":
        # training instances: the same workload recipe, indices past every rank's batch
        from paper_2602_24155_gb300.policy_train import train_policy
        train = _instances_range(world * args.count, args.train_count, z)
        t0 = time.perf_counter()
        weights, train_loss, decisions = train_policy(ctx, train, hidden=8, epochs=60)
        learned = {"train_s": time.perf_counter() - t0, "decisions": decisions, "loss": train_loss,
                   "hidden": 8, "train_instances": len(train)}
        opt.update(weights=weights, hidden=8)

    tuning = None
    if args.path == "auto":
        # before the timed region, like the training: time the candidates on a sample of the batch
        t0 = time.perf_counter()
        tuning = z.zeta_autotune(ctx, specs, **opt)
        tuning["tune_s"] = time.perf_counter() - t0

    # device-resident inputs: prepare once, then time the kernels
    plan = z.zeta_batch_prepare(ctx, specs, **opt)
    for _ in range(args.warmup):
        plan.run()
    torch.cuda.synchronize()
    P_warm, per, tot_warm = plan.finish()
    assert all(P is not None for P in P_warm), "an instance failed"

    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.run()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    P_timed, _, tot = plan.finish()   # kernel-event timing of the timed launches
    assert P_timed == P_warm
    plan.release()
    ms_t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    ms_per_step = ms_max / args.steps
    total_instances = args.count * world
    value = total_instances / (ms_per_step / 1000.0)
    column_steps = tot["column_steps"] * world
    s = per[0]["s"]

    # the learned policy against the method without the network (cover) and the paper's three policies
    # (Sec. 4.1-4.3), all on one sub-batch of the same workload, one device-resident launch each
    policies = {"batch": "first %d instances of the main batch" % min(args.policy_count, args.count),
                args.policy + "_full_batch": {"zeta_per_s": value, "column_steps": column_steps,
                                              "ms_per_step": ms_per_step}}
    if learned is not None:
        policies[args.policy + "_full_batch"].update(learned)
    sub = specs[:min(args.policy_count, args.count)]
    P_sub = None
    for pol in ("learned", "cover", "p_chunk", "depth_first", "var_by_var"):
        if pol == "learned" and learned is None:
            continue
        o = dict(opt, policy=pol, path=args.path if args.path != "auto" else "vector")
        if pol != "learned":
            o.pop("weights", None)
            o.pop("hidden", None)
        plan2 = z.zeta_batch_prepare(ctx, sub, **o)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan2.run()
        e1.record(stream)
        torch.cuda.synchronize()
        P_pol, _, tot_pol = plan2.finish()
        plan2.release()
        if P_sub is None:
            P_sub = P_pol
        assert P_pol == P_sub == P_warm[:len(sub)], "policies disagree"
        ms_pol = e0.elapsed_time(e1)
        policies[pol] = {"zeta_per_s": len(sub) / (ms_pol / 1000.0), "column_steps": tot_pol["column_steps"],
                         "chunks": tot_pol["chunks"], "steps": tot_pol["steps"], "ms_per_launch": ms_pol,
                         "column_steps_per_s": tot_pol["column_steps"] / (ms_pol / 1000.0)}
    if "learned" in policies and "cover" in policies:
        policies["network_gain_over_cover"] = {
            "column_steps": 1 - policies["learned"]["column_steps"] / policies["cover"]["column_steps"],
            "time": 1 - policies["learned"]["ms_per_launch"] / policies["cover"]["ms_per_launch"]}

    # the other recurrence path on the same batch and policy (limb-split GEMM on the tensor cores against the
    # modular matrix-vector steps on the CUDA cores)
    chosen = tuning["best"]["path"] if tuning else args.path
    paths = {chosen: {"zeta_per_s": value, "ms_per_step": ms_per_step}}
    other = "gemm" if chosen == "vector" else "vector"
    plan3 = z.zeta_batch_prepare(ctx, specs, **dict(opt, path=other))
    plan3.run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan3.run()
    e1.record(stream)
    torch.cuda.synchronize()
    P_other, _, _ = plan3.finish()
    plan3.release()
    assert P_other == P_warm, "paths disagree"
    ms_other = e0.elapsed_time(e1)
    paths[other] = {"zeta_per_s": args.count / (ms_other / 1000.0), "ms_per_step": ms_other}
    for v in paths.values():
        v["modmac_per_s"] = tot["column_steps"] * s * s / (v["ms_per_step"] / 1000.0)

    # end to end through the C ABI with host buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P_e2e, per_e2e, tot_e2e = z.zeta_batch(ctx, specs, **opt)
    e2e_s = time.perf_counter() - t0
    assert P_e2e == P_warm
    e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = total_instances / float(e2e_t.item())
    coeff_bytes = sum(4 * len(sp[3]) for sp in specs)

    # roofline of the recurrence kernel: modular multiply-adds (s^2 per column step)
    peaks = _peaks()
    traffic = DRAM_BYTES_PER_INSTANCE * args.count if (DRAM_BYTES_PER_INSTANCE and args.policy == "learned"
                                                        and chosen == "vector") else None
    ms_kernel = tot["ms_kernel"] / max(1, tot["kernel_launches"])
    macs_per_launch = tot["column_steps"] * s * s
    # mad.wide.u32 per launch as the executor computes them: four per modular multiply-add when q = p^M < 2^56
    # (28-bit limbs), six otherwise (20-bit x 30-bit limbs)
    madw_per_launch = sum(st["column_steps"] * st["s"] ** 2 * (4 if sp[2] ** st["M"] < (1 << 56) else 6)
                          for sp, st in zip(specs, per))
    achieved = madw_per_launch / (ms_kernel / 1000.0) / 1e12
    # ALU peak: 152 SMs x 64 mad.wide.u32 per SM per clock (nominal) at the maximum SM clock
    alu_peak = 152 * 64 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "zeta/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "steps_per_s": column_steps / (ms_per_step / 1000.0),
        "config": _workload_config(args.count),
        "run": {"policy": args.policy, "path": chosen,
                "block_threads": tuning["best"]["block_threads"] if tuning else 0,
                "resident_bytes": tot["bytes_h2d"], "column_steps_per_step": column_steps},
        "e2e": {"value": e2e_value, "unit": "zeta/s", "h2d_bytes_per_step": coeff_bytes + tot_e2e["bytes_h2d"],
                "d2h_bytes_per_step": tot_e2e["bytes_d2h"] + 16 * sum(len(P) for P in P_e2e)},
        "gpu_launches": args.steps,
        "policies": policies,
        "paths": paths,
        "autotune": tuning,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "T mad.wide.u32/s",
                     "frac": achieved / alu_peak, "traffic": traffic,
                     "kernel": "k_execute", "ms_per_launch": ms_kernel,
                     "modmac_per_s": macs_per_launch / (ms_kernel / 1000.0),
                     "madw_per_launch": madw_per_launch,
                     "peak_basis": ("152 SM x 64 mad.wide.u32/clk (nominal) at %.0f MHz; achieved counts 4 per "
                                    "modular multiply-add for q < 2^56 (28-bit limbs), 6 above (20 x 30-bit limbs)"
                                    % peaks.get("sm_max_mhz", 2070.0))
                                   + ("" if chosen == "vector" else "; tensor-core path: its CUDA-core epilogue "
                                      "(digit fold and reduction) bounds it, the tensor pipe is the minor share")},
        "clocks": clk,
        "host": {"ms_setup": tot_e2e["ms_host_setup"], "ms_finish": tot_e2e["ms_host_finish"],
                 "e2e_s": e2e_s},
    }
    if rank == 0 and world == 1 and not args.no_k3:
        line["k3_heights"] = _k3_survey(z, ctx, stream, torch)
    if rank == 0 and world == 1 and args.k3_count > 0:
        try:
            line["k3_full"] = _k3_full(z, ctx, stream, torch, args.k3_count, args.k3_N)
        except Exception as exc:   # reported, never a reason to lose the main line
            line["k3_full"] = {"error": repr(exc)[:200]}
    if rank == 0 and world == 1 and not args.no_mixed:
        try:
            line["mixed_stream"] = _mixed_stream(z, ctx, stream, torch)
        except Exception as exc:   # reported, never a reason to lose the main line
            line["mixed_stream"] = {"error": repr(exc)[:200]}
    if rank == 0 and world == 1 and not args.no_cubic:
        try:
            line["cubic_surfaces"] = _cubic_survey(z, ctx, stream, torch)
        except Exception as exc:   # reported, never a reason to lose the main line
            line["cubic_surfaces"] = {"error": repr(exc)[:200]}
    if rank == 0 and world == 1 and args.surface_count > 0:
        try:
            line["quintic_surfaces"] = _quintic_surfaces(z, ctx, stream, torch, args.surface_count, 24)
        except Exception as exc:   # reported, never a reason to lose the main line
            line["quintic_surfaces"] = {"error": repr(exc)[:200]}
    if rank == 0 and world == 1 and not args.no_mixed:
        try:
            line["mixed_stream_r1"] = _mixed_stream_r1(z, ctx, stream, torch)
        except Exception as exc:   # reported, never a reason to lose the main line
            line["mixed_stream_r1"] = {"error": repr(exc)[:200]}
    if rank == 0 and world == 1 and not args.no_fourfold:
        try:
            line["cubic_fourfolds"] = _cubic_fourfolds(z, ctx, stream, torch, args.fourfold_dense)
        except Exception as exc:   # reported, never a reason to lose the main line
            line["cubic_fourfolds"] = {"error": repr(exc)[:200]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        sample_n = max(1, min(cores, 16))
        wall, res = oracle_sample(specs[:sample_n], cores)
        for (P_o, (_, _, P_ref)) in zip(P_warm[:sample_n], res):
            assert P_o == P_ref, "GPU result differs from the oracle"
        line["cpu_baseline"] = {"value": sample_n / wall, "unit": "zeta/s", "cores": min(cores, sample_n),
                                "kind": "oracle",
                                "sample": "first %d instances (all %d primes cycle), one process each; "
                                          "results also checked equal to the GPU's" % (sample_n, min(sample_n, 12))}
    if rank == 0:
        print(json.dumps(line))
    z.zeta_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
