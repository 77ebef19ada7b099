"""Parity of Algorithm 2's final contract() (the local field of a strain
train) with the oracle: random trains on anisotropic grids in both site
orders, the laminate's closed-form local gradient, and the dense FFT
solver's local field on a plane box."""
import numpy as np
import pytest

from oracle import ms as MS
from paper_2512_07811_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2512_07811_gb300 import qtt
    return qtt


@pytest.fixture(scope="module")
def ctx(Q):
    return Q.Context(0)


@pytest.mark.parametrize("nb", [(3, 2, 1), (2, 3, 0)])
@pytest.mark.parametrize("ordering", ["interleaved", "grouped"])
def test_contract_random_train_equals_oracle(Q, ctx, nb, ordering):
    rng = np.random.default_rng(sum(nb) + len(ordering))
    d = sum(nb)
    ranks = [1] + [3] * d + [1]
    modes = [6] + [2] * d
    x = [rng.standard_normal((ranks[k], modes[k], ranks[k + 1])) + 1j * rng.standard_normal((ranks[k], modes[k], ranks[k + 1]))
         for k in range(d + 1)]
    want = MS.contract(x, nb, ordering)
    got = Q.contract_voxels(ctx, Q.TT.from_cores(ctx, x), nb, interleaved=ordering == "interleaved")
    np.testing.assert_allclose(got, want, atol=1e-13 * np.abs(want).max())
    got32 = Q.contract_voxels(ctx, Q.TT.from_cores(ctx, x, Q.C64), nb, interleaved=ordering == "interleaved")
    np.testing.assert_allclose(got32, want, atol=1e-5 * np.abs(want).max())


def test_local_strain_laminate_closed_form(Q, ctx):
    """16^3 laminate, E = e_x: the local gradient is 20/11 in phase 1, 2/11 in
    phase 2, zero across the layers."""
    ind = I.laminate_indicator(16)
    C, rep = Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), tol=1e-13, max_rank=32, eps=1e-10,
                             max_iter=20, prec=Q.PREC_F64, load_mask=1, return_strain=True)
    loc = Q.contract_voxels(ctx, rep.strain, (4, 4, 4))
    want = np.where(ind == 1.0, 2.0 / 11.0, 20.0 / 11.0)
    np.testing.assert_allclose(loc[0].real, want, atol=1e-9)
    assert np.abs(loc[1:]).max() < 1e-9


def test_local_strain_plane_box_equals_dense_field(Q, ctx):
    pb = MS.scalar_problem(I.box_indicator_2d(16, 0.25), 1.0, 10.0)
    E = np.array([1.0, 0.0, 0.0])
    dense = MS.ms_dense(pb, E, tol=1e-11, max_iter=500, keep_field=True)
    C, rep = Q.ms_homogenize(ctx, pb.indicator, "scalar", (1.0, 10.0), pb.C0, tol=1e-11, max_rank=64, eps=1e-11,
                             max_iter=300, oversample=16, prec=Q.PREC_F64, load_mask=1, return_strain=True)
    loc = Q.contract_voxels(ctx, rep.strain, (4, 4, 0))
    assert np.abs(loc - dense.eps_field).max() < 1e-6
