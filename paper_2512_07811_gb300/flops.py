"""Flop model of SVD-based tensor-train rounding, shared by every measured path.

"tt_round TFLOP/s" is this model's count divided by time, the same count for
the GPU paths and the CPU oracle, so that the rates compare like for like.
Per core k (0-based, modes p_k, input ranks r, ranks after the
orthogonalisation sweep R, output ranks t), real flops, complex x4:

  orthogonalisation sweep, k = 0..d-2, m = R_k p_k, n = r_{k+1}:
      absorb R:   2 R_k r_k p_k r_{k+1}
      QR:         2 m n^2 - 2/3 n^3        (m >= n; general form below)
      form Q:     the same again
  truncation sweep, k = d-1..1:
      SVD of R_k x (p_k t_{k+1}):   4 R_k (p_k t_{k+1})^2 + 8 (p_k t_{k+1})^3
      absorb U S into core k-1:     2 p_{k-1} R_{k-1} R_k t_k
"""
from __future__ import annotations


def _qr(m: float, n: float) -> float:
    k = min(m, n)
    return 2.0 * m * n * k - (m + n) * k * k + 2.0 * k ** 3 / 3.0


def round_flops(modes, ranks_in, ranks_out, complex_values: bool = True) -> float:
    d = len(modes)
    R = [1] * (d + 1)
    for k in range(d - 1):
        R[k + 1] = min(R[k] * modes[k], ranks_in[k + 1])
    f = 0.0
    for k in range(d - 1):
        m = R[k] * modes[k]
        n = ranks_in[k + 1]
        f += 2.0 * R[k] * ranks_in[k] * modes[k] * ranks_in[k + 1]
        f += 2.0 * _qr(m, n)
    for k in range(d - 1, 0, -1):
        pt = modes[k] * ranks_out[k + 1]
        f += 4.0 * R[k] * pt * pt + 8.0 * pt ** 3
        f += 2.0 * modes[k - 1] * R[k - 1] * R[k] * ranks_out[k]
    return 4.0 * f if complex_values else f
