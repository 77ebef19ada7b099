"""The library's site order (host logic, no GPU) equals the oracle's: the
sites holding each dimension's bits, level by level, for cubes, anisotropic
grids, plane grids and both orders."""
import pytest

from oracle import ms as MS
from paper_2512_07811_gb300 import qtt as Q


@pytest.mark.parametrize("nb", [(3, 3, 3), (3, 2, 1), (2, 3, 0), (0, 4, 1), (5, 0, 0), (18, 18, 0), (12, 12, 12)])
@pytest.mark.parametrize("ordering", ["interleaved", "grouped"])
def test_site_order_equals_oracle(nb, ordering):
    dim, pos = Q.site_order(nb, interleaved=ordering == "interleaved")
    assert len(dim) == sum(nb)
    for d in range(3):
        sites = MS.dim_positions(nb, ordering, d)
        assert [p for p in range(len(dim)) if dim[p] == d] == sites
        assert [pos[p] for p in sites] == list(range(nb[d]))


def test_site_order_rejects_bad_grids():
    with pytest.raises(Q.QTTError):
        Q.site_order((21, 0, 0))
    with pytest.raises(Q.QTTError):
        Q.site_order((-1, 2, 2))
