"""Training of the per-bond rank predictor on rank traces the method generates.

`collect_traces` runs the QTT Moulinec-Suquet solver (`ms_homogenize`) with
trace recording on and returns the (features, log2 rank) rows of every
sketched rounding; `train` fits the device-side network with its own
forward/backward/Adam kernels (all arithmetic in libqtt.so; this module only
batches host arrays).
"""
from __future__ import annotations

import numpy as np

from . import qtt as Q


def collect_traces(ctx: "Q.Context", problems, cap: int = 200000):
    """problems: iterable of dicts with keys indicator, kind, moduli, C0 and the
    ms_homogenize keyword arguments (tol, max_rank, eps, max_iter, ...)."""
    rows = []
    for pb in problems:
        kw = dict(pb)
        ind = kw.pop("indicator")
        kind = kw.pop("kind")
        moduli = kw.pop("moduli")
        C0 = kw.pop("C0")
        _, rep = Q.ms_homogenize(ctx, ind, kind, moduli, C0, trace_cap=cap, **kw)
        rows.append(rep.trace_rows)
    data = np.concatenate(rows, axis=0) if rows else np.zeros((0, Q.MLP_FEATURES + 1), np.float32)
    return data[:, :Q.MLP_FEATURES], data[:, Q.MLP_FEATURES]


def train(net: "Q.MLP", X, t, epochs: int = 300, batch: int = 512, lr: float = 3e-3, alpha: float = 4.0,
          seed: int = 0):
    """Mini-batch Adam on the asymmetric loss (under-prediction weighted by
    alpha); returns the loss history (one value per epoch, the last batch)."""
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    hist = []
    for _ in range(epochs):
        perm = rng.permutation(n)
        last = None
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            last = net.train_step(X[idx], t[idx], alpha=alpha, lr=lr)
        hist.append(last)
    return hist
