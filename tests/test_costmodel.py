"""The cost model of Eqs. 6-9 (host arithmetic, no GPU): the break-even R0 of
Eq. 6 reduces to the bound of Eq. 7 when the modes are free and every solve
costs the same, and Eq. 9's bound is R1 / (2 R1 + N)."""
import pytest

from paper_2201_09729_gb300 import costmodel as cm


@pytest.mark.parametrize("n,r1", [(32, 8), (128, 8), (640, 24), (4, 1)])
def test_free_modes_give_eq7(n, r1):
    # t_lap = 0, equal time per solve: R0 = 2 R1 + N exactly (the equality of Eq. 7)
    assert cm.r0_equivalent(0.0, n, 0.37, r1) == pytest.approx(2 * r1 + n, rel=1e-15)
    # any Laplacian time raises R0 above the bound, by t_lap / t_D
    assert cm.r0_equivalent(1.1, n, 0.5, r1) == pytest.approx(2 * r1 + n + 2.2, rel=1e-15)


@pytest.mark.parametrize("n,r1", [(32, 8), (640, 24), (4, 4)])
def test_eq9_bound(n, r1):
    assert cm.rest_fraction_bound(n, r1) == pytest.approx(r1 / (2 * r1 + n), rel=1e-15)
    # a remainder exactly at the bound pays off with free modes, one just above does not
    r0 = cm.r0_equivalent(0.0, n, 1.0, r1)
    b = cm.rest_fraction_bound(n, r1)
    assert cm.pays_off(1.0 - b + 1e-12, r1, r0)
    assert not cm.pays_off(1.0 - b - 1e-9, r1, r0)


def test_limits():
    assert cm.pays_off(1.0, 8, 100.0)            # C = C_dist: nothing stochastic left
    assert not cm.pays_off(0.0, 8, 100.0)        # no distillation signal at all
    with pytest.raises(ValueError):
        cm.r0_equivalent(1.0, 4, 0.0, 1)
