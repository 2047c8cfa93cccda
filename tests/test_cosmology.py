"""The product's expansion histories (used by the drivers to supply a and adot per step)
against the oracle's independent ones: the Lambda-free models of Table 1 (Einstein-de Sitter
and open, Peebles' cycloid) and flat LCDM, including a(t(z)) = 1/(1+z) round trips."""
import math

import pytest

from oracle import constants as K
from oracle import cosmology as OC
from paper_0908_2654_gb300 import cosmology as PC


@pytest.mark.parametrize("q0,h", [(0.5, 0.5), (0.05, 1.0)])
def test_lambda_free_matches_oracle(q0, h):
    p = PC.LambdaFree(q0=q0, h=h)
    o = OC.OpenNoLambda(q0, h * K.H100)
    for z in (10.0, 4.0, 1.0, 0.0):
        t = p.t_of_z(z)
        assert t == pytest.approx(o.t_of_a(1.0 / (1.0 + z)), rel=1e-12)
        assert p.a(t) == pytest.approx(1.0 / (1.0 + z), rel=1e-12)
        assert p.a(t) == pytest.approx(o.a(t), rel=1e-12)
        assert p.adot(t) == pytest.approx(o.adot(t), rel=1e-11)
    # early times: the open model tends to Einstein-de Sitter with H0^2 Om
    t = 1e-6 / p.H0
    assert p.a(t) == pytest.approx((1.5 * math.sqrt(2 * q0) * p.H0 * t) ** (2 / 3), rel=1e-3)


def test_flat_lcdm_matches_oracle():
    p = PC.from_dict(dict(Omega_m=0.3, Omega_L=0.7, h=0.7))
    o = OC.FlatLCDM(0.3, 0.7, 0.7)
    for z in (10.0, 4.0, 0.0):
        t = p.t_of_z(z)
        assert t == pytest.approx(o.t_of_z(z), rel=1e-12)
        assert p.a(t) == pytest.approx(1.0 / (1.0 + z), rel=1e-12)
        assert p.adot(t) == pytest.approx(o.adot(t), rel=1e-12)
