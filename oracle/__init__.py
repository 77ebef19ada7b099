"""CPU oracle for the QTT Moulinec-Suquet hot path.

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 / complex128 NumPy code written
from the paper's definitions (arXiv 2512.07811, Sections 2-3 and Appendix A)
and from the textbook definitions it cites.  Only the test-suite, the smoke
check and the benchmark's CPU-baseline leg may import anything from here; the
GPU library neither imports nor links it, and it imports nothing from the GPU
library (the seeded input generators are a separate module without any of the
method's arithmetic).

Modules
-------
tt      tensor-train algebra, orthogonalisation, SVD rounding, TT-SVD
qft     the superfast Fourier transform Q_n as an operator train
ms      dense FFT Moulinec-Suquet (Algorithm 1) and QTT Moulinec-Suquet
        (Algorithm 2), Green operators, effective tensors, closed forms
mlp     the per-bond rank predictor (3 hidden layers of width 64) with
        hand-written forward and backward passes
randround  randomize-then-orthogonalize TT rounding (not in the
        paper) used to check the GPU sketch path
"""
