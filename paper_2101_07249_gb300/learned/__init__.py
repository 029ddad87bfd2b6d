"""Learned sketch proposal: the gate that decides whether the network's start
block replaces the Gaussian sketch.

The proposal is an aid to the randomised range finder (Alg. 3), so it is
judged the way Rayleigh-Ritz judges any subspace.  For a subspace of
dimension m the sum of its k largest Ritz values is at most the sum of A's k
largest eigenvalues (Ky Fan), with equality when the subspace contains the
leading invariant subspace; a larger sum therefore means a better captured
dominant subspace, which is what the spectral LMP needs.  The learned block
[S_nn, G_l] is accepted only when its top-k Ritz sum is at least `ratio`
(default 1: never worse) times that of the Gaussian block of the same width;
otherwise the Gaussian sketch is used.
"""
from __future__ import annotations

import numpy as np


def accept(theta_learned, theta_gauss, k=None, ratio=1.0):
    """Gate of the learned proposal: sum of the top-k Ritz values of the
    learned block >= ratio x that of the Gaussian block (both decreasing
    arrays from the same REVD on blocks of the same width)."""
    tl = np.sort(np.asarray(theta_learned, dtype=np.float64))[::-1]
    tg = np.sort(np.asarray(theta_gauss, dtype=np.float64))[::-1]
    k = min(len(tl), len(tg)) if k is None else int(k)
    if k < 1 or len(tl) < k or len(tg) < k:
        raise ValueError("need at least k Ritz values from each block")
    sl, sg = float(np.sum(tl[:k])), float(np.sum(tg[:k]))
    if not (np.isfinite(sl) and np.isfinite(sg)):
        return False
    return sl >= ratio * sg
