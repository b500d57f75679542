"""Exact network solve by dense factorisation (oracle; test infrastructure).

The inverse-based rewrite v = G^{-1} i of Eq. 2 has a unique answer because G
is symmetric positive definite (every bus has a shunt to ground). This module
computes it the plain way: a dense Cholesky factorisation, refactored after
every change of G ("explicit recomputation").
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


class DenseSolver:
    """v = G^{-1} i of Eq. 2 by a dense Cholesky factorisation of G (the explicit recomputation
    that Sec. IV's local modification is measured against)."""

    def __init__(self, G: np.ndarray):
        self.G = np.array(G, dtype=float)
        self.cf = sla.cho_factor(self.G, lower=True)

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        """G^{-1} rhs (Eq. 2)."""
        return sla.cho_solve(self.cf, rhs)

    def inverse(self) -> np.ndarray:
        """The exact G^{-1} that the stores of Sec. III are compared with."""
        return sla.cho_solve(self.cf, np.eye(self.G.shape[0]))


def inverse(G: np.ndarray) -> np.ndarray:
    """The exact G^{-1} (Eq. 2); also Algorithm 1's "direct compute" of a leaf block."""
    return DenseSolver(G).inverse()


def sherman_morrison(Ginv: np.ndarray, u: np.ndarray, delta: float) -> np.ndarray:
    """(G + delta u u^T)^{-1} = G^{-1} - (delta/d) z z^T, z = G^{-1} u, d = 1 + delta u^T z: the
    global rank-one form of a single change G' = G + delta u u^T of Sec. IV."""
    z = Ginv @ u
    d = 1.0 + delta * float(u @ z)
    return Ginv - (delta / d) * np.outer(z, z)


def woodbury(Ginv: np.ndarray, U: np.ndarray, deltas: np.ndarray) -> np.ndarray:
    """(G + U diag(delta) U^T)^{-1} by the Woodbury identity: several simultaneous changes of
    Sec. IV, and the form the EXACT node cores of Sec. III take."""
    Z = Ginv @ U
    K = np.diag(1.0 / np.asarray(deltas, float)) + U.T @ Z
    return Ginv - Z @ np.linalg.solve(K, Z.T)
