"""The CUDA discrete adjoint (rt_adjoint_step behind a torch.autograd.Function) against the
oracle's dense adjoint on 8^3 grids and against central finite differences of the GPU forward
run on 8 source emissivities.  The adjoint covers periodic and reflecting faces (the Stromgren
case here reflects at every face); a grid with outflow faces is rejected."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import adjoint as OA  # noqa: E402

TIGHT = dict(precision="fp64", newton_tol=1e-11, lin_rtol=1e-12, max_newton=60, max_lin=400)


def _grad(w, nsteps, **opt):
    from paper_0908_2654_gb300.adjoint import ionized_fraction
    ndot = torch.tensor(np.asarray(w["src_ndot"], float), dtype=torch.float64, requires_grad=True)
    clump = torch.tensor(np.asarray(w["clump"], np.float32), requires_grad=True)
    J = ionized_fraction(ndot, clump, w, nsteps, **opt)
    J.backward()
    return float(J.detach()), ndot.grad.cpu().numpy(), clump.grad.cpu().numpy()


@pytest.mark.parametrize("name,make,nsteps", [
    ("reion8_nonisothermal", lambda: W.reionization_field(n=8, nsrc=2, box_mpc=14.4 * 8 / 256, ndot_total=4e49,
                                                          dt_myr=0.3), 2),
    ("stromgren8_isothermal", lambda: W.stromgren_static(n=8, dt_over_trec=1e-3, bc=("reflect",) * 6), 2),
])
def test_adjoint_matches_oracle_dense_adjoint(name, make, nsteps):
    w = make()
    J, g_ndot, g_clump = _grad(w, nsteps, **TIGHT)
    Jo, go_ndot, go_clump = OA.gradient(w, np.asarray(w["src_ndot"], float), np.asarray(w["clump"], float), nsteps)
    assert J == pytest.approx(Jo, rel=1e-9)
    np.testing.assert_allclose(g_ndot, go_ndot, rtol=1e-6)
    scale = np.abs(go_clump).max()
    assert np.max(np.abs(g_clump - go_clump)) <= 1e-6 * scale


def test_adjoint_matches_finite_differences_on_8_emissivities():
    """Mixed-precision forward (FP32 multigrid in FP64 Newton/CG), 16^3 field, 8 sources."""
    from paper_0908_2654_gb300.adjoint import ionized_fraction
    w = W.reionization_field(n=16, nsrc=8, box_mpc=14.4 * 16 / 256, ndot_total=1e52 * 8 / 2000, dt_myr=1.0)
    opt = dict(TIGHT, precision="mixed")
    nsteps = 3
    J, g_ndot, _ = _grad(w, nsteps, **opt)
    ndot0 = np.asarray(w["src_ndot"], float)
    clump = torch.tensor(np.asarray(w["clump"], np.float32))
    for s in range(8):
        h = 1e-3 * ndot0[s]
        vals = []
        for sign in (1, -1):
            p = ndot0.copy()
            p[s] += sign * h
            vals.append(float(ionized_fraction(torch.tensor(p), clump, w, nsteps, **opt)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert g_ndot[s] == pytest.approx(fd, rel=1e-5), (s, g_ndot[s], fd)


def test_adjoint_rejects_outflow_faces():
    from paper_0908_2654_gb300 import _rt
    w = W.stromgren_static(n=8, dt_over_trec=1e-3)          # outflow at the upper faces
    with pytest.raises(_rt.RTError) as e:
        _grad(w, 1, **TIGHT)
    assert e.value.code == _rt.RT_EINVAL
