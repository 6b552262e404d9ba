"""Reader of tests/golden/quartic_k3_full.txt (written by make_golden.py k3 from the oracle alone)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def load():
    """List of dicts: instance, n, d, p, coeffs, P (the oracle's full-precision P(T))."""
    out, cur = [], None
    for line in open(os.path.join(HERE, "quartic_k3_full.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, _, val = line.partition(":")
        val = val.strip()
        if key == "instance":
            cur = {"instance": int(val)}
            out.append(cur)
        elif key == "n d p":
            cur["n"], cur["d"], cur["p"] = map(int, val.split())
        elif key == "coeffs":
            cur["coeffs"] = [int(x) for x in val.split()]
        elif key == "P":
            cur["P"] = [int(x) for x in val.split()]
    return out
