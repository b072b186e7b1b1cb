"""Comparison of Bragg amplitudes for the parity tests.

Two figures over the propagating orders of both sides, [c; d] stacked in order:
  norm-wise   ||a - b|| / ||b||              (the 1e-9 target of the FP64 path)
  element-wise max_n |a_n - b_n| / |b_n|     (every single amplitude, the weakest included)
The orders themselves must agree exactly (integer decisions, taken in FP64 on both sides)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    """{(side, order): amplitude} from tests/golden/<name>_bragg.txt (written from the oracle)."""
    ref = {}
    for ln in open(os.path.join(GOLDEN, f"{name}_bragg.txt")):
        if ln.startswith("#"):
            continue
        s, n, a, b = ln.split()
        ref[(s, int(n))] = complex(float(a), float(b))
    return ref


def as_dict(br):
    got = {("c", int(n)): v for n, v in zip(br["n_top"], br["c"])}
    got.update({("d", int(n)): v for n, v in zip(br["n_bot"], br["d"])})
    return got


def errors(got, ref):
    """(norm-wise, element-wise) relative errors of `got` against `ref`; both are Bragg results
    (dicts from GratingSolver.bragg or load_golden).  Raises if the propagating orders differ."""
    g = got if "n_top" not in got else as_dict(got)
    r = ref if "n_top" not in ref else as_dict(ref)
    assert set(g) == set(r), (sorted(set(g) ^ set(r)))
    keys = sorted(r)
    a = np.array([g[k] for k in keys])
    b = np.array([r[k] for k in keys])
    return float(np.linalg.norm(a - b) / np.linalg.norm(b)), float(np.max(np.abs(a - b) / np.abs(b)))


def check(got, ref, tol=1e-9, elem_tol=1e-9):
    """Asserts both figures; returns them."""
    nw, ew = errors(got, ref)
    assert nw <= tol, ("norm-wise", nw)
    assert ew <= elem_tol, ("element-wise", ew)
    return nw, ew
