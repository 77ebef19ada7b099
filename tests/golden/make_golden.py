"""Writes the stored expected values under tests/golden/ from closed forms in
the oracle (nothing here runs the GPU library).

scalar_laminate_keff.json
    Two-phase laminate, layers normal to x, phase fraction 1/2, k1 = 1,
    k2 = 10: the exact effective conductivity is the harmonic mean across the
    layers (20/11) and the arithmetic mean along them (11/2); the
    Moulinec-Suquet fixed point with k0 = (k1 + k2)/2 reproduces it on any
    grid (Sec. 3.1, Algorithm 1; Appendix A for the column-by-column read-out).
elastic_laminate_ceff.json
    The same layout with isotropic phases E = 1 and E = 10, nu = 0.3:
    Backus-type laminate averages in Voigt form, engineering shears.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ms as MS  # noqa: E402


def lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def main():
    k1, k2 = 1.0, 10.0
    K = MS.scalar_laminate_keff(k1, k2, 0.5, axis=0)
    with open(os.path.join(HERE, "scalar_laminate_keff.json"), "w") as f:
        json.dump({"source": "closed form: harmonic mean across layers, arithmetic along",
                   "k1": k1, "k2": k2, "fraction2": 0.5, "keff": K.tolist(),
                   "keff_xx_exact": "20/11", "keff_yy_exact": "11/2"}, f, indent=1)
    l1, m1 = lame(1.0, 0.3)
    l2, m2 = lame(10.0, 0.3)
    C = MS.elastic_laminate_ceff([l2, l1], [m2, m1], [0.5, 0.5])
    with open(os.path.join(HERE, "elastic_laminate_ceff.json"), "w") as f:
        json.dump({"source": "Backus-type laminate averages, layers normal to x",
                   "E": [1.0, 10.0], "nu": 0.3, "fraction2": 0.5,
                   "voigt_order": "11,22,33,23,13,12", "ceff": C.tolist()}, f, indent=1)


if __name__ == "__main__":
    main()
