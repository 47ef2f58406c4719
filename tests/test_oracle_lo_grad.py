"""Pins of the oracle's lo_grad option (CPU): a medium vertex's outgoing radiance depends on x
through the HG phase of the light it scatters toward x (the extension beyond Sec. 4's
grad L_o = 0 that Sec. 7 discusses; Eq. reducedRadianceDerivatives with grad L_o kept).

L_o(x) = L_o(x_c) f(l . w(x)) / f(l . w(x_c)): l the light's propagation direction at the
vertex, w(x) the unit direction from the vertex to x, x_c the record centre.  Pinned by:
central differences of the oracle's own frozen-vertex value function (its gradient and
Hessian), the isotropic case (f constant: nothing changes), the surface shell (Lambertian:
nothing changes), and the values at the centre (the factor is 1 there)."""
import numpy as np

import oracle as O
import workloads as W
from workloads.configs import replace
from workloads.scenes import Medium

from tests.test_oracle_pins import fd_grad, fd_hess_from_grad, rel


def _setup(g=0.5):
    c1 = W.config1()
    c1.scene.medium = Medium(0.5, 0.05, g)
    return c1, O.OracleScene(c1.scene)


def test_derivatives_vs_frozen_vertex_finite_differences(oracle_lib):
    c1, os_ = _setup(0.5)
    rp = replace(c1.params, lo_grad=1)
    pos = c1.positions()
    for r in (0, 7):
        x0 = pos[r].astype(np.float64)
        fL = lambda xx: O.frozen_eval(os_, rp, pos[r], xx, rec=r, which=2)[0][0]
        fg = lambda xx: O.frozen_eval(os_, rp, pos[r], xx, rec=r, which=2)[1][0]
        L, g, H = O.frozen_eval(os_, rp, pos[r], x0, rec=r, which=2)
        for c in range(3):
            assert rel(g[0, c], fd_grad(lambda xx: fL(xx)[c], x0)) < 1e-6
            assert rel(H[0, c], fd_hess_from_grad(lambda xx: fg(xx)[c], x0)) < 1e-6
        # the factor changes the derivatives, not the value at the centre
        L0, g0, H0 = O.frozen_eval(os_, c1.params, pos[r], x0, rec=r, which=2)
        assert np.allclose(L, L0, rtol=1e-13)
        assert rel(g[0], g0[0]) > 1e-4 and rel(H[0], H0[0]) > 1e-4
        # away from the centre the value moves too (the vertex radiance toward x changes)
        xe = x0 + np.array([0.01, -0.005, 0.007])
        assert rel(O.frozen_eval(os_, rp, pos[r], xe, rec=r, which=2)[0],
                   O.frozen_eval(os_, c1.params, pos[r], xe, rec=r, which=2)[0]) > 1e-6


def test_isotropic_medium_and_surface_shell_are_unchanged(oracle_lib):
    c1, os_ = _setup(0.0)
    pos = c1.positions()[:6]
    a = O.records(os_, c1.params, pos)
    b = O.records(os_, replace(c1.params, lo_grad=1), pos)
    for k in ("L", "grad", "hess", "L_ff", "radius"):
        assert np.allclose(a[k], b[k], rtol=1e-13, atol=1e-15), k
    c1, os_ = _setup(0.5)
    a = O.records(os_, c1.params, pos)
    b = O.records(os_, replace(c1.params, lo_grad=1), pos)
    for k in ("L", "L_ss", "L_ms", "grad_ss", "hess_ss", "L_ff"):
        assert np.allclose(a[k], b[k], rtol=1e-13, atol=1e-15), k
    assert not np.allclose(a["hess_ms"], b["hess_ms"], rtol=1e-6)
