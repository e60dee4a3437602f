"""Relative reconstruction error, eq. (4): RRE = ||X - G F||_F / ||X||_F.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""

from __future__ import annotations

import numpy as np


def rre(X, G, F) -> float:
    X = np.asarray(X, dtype=np.float64)
    return float(np.linalg.norm(X - np.asarray(G, dtype=np.float64) @ np.asarray(F, dtype=np.float64))
                 / np.linalg.norm(X))


def rre_history(X, history) -> np.ndarray:
    """RRE after each recorded outer iteration, history = [(G, F), ...]."""
    X = np.asarray(X, dtype=np.float64)
    nx = np.linalg.norm(X)
    return np.array([np.linalg.norm(X - G @ F) / nx for G, F in history])
