"""Helpers shared by the GPU parity tests (no method arithmetic)."""
import numpy as np


def rel_err(got, ref):
    """max over rows of ||got - ref||_inf / max over rows of ||ref||_inf (the per-result metric)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))
