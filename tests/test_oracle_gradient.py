"""The oracle's tangent-linear gradient of the frozen liquid window against central finite
differences of the oracle itself (the gradient's definition).  J = sum over the window's
steps of the x-force on all spheres (Eqs. netforce, momentum_transfer); parameters: the
relaxation time tau (lambda_+ = -1/tau, lambda_- from the magic relation) and the gravity g."""
import numpy as np
import pytest

G0 = np.array([2e-5, -1e-5, 5e-6])


def _make(orc, tau=0.7, g=G0):
    return orc.Sim(nx=14, ny=12, nz=13, tau=tau, g=g, bc=(1, 1, 1), sphere_mode=0,
                   spheres=[(5.3, 6.1, 6.2, 2.5, 1.5, 0.002, 0.0, -0.001, 0.0, 0.001, 0.0), (10.2, 5.7, 6.4, 2.0, 1.5)])


@pytest.mark.parametrize("which", ["tau", "gx", "gz"])
def test_tangent_matches_finite_differences(orc, which):
    n = 40
    if which == "tau":
        J, dJ = _make(orc).tangent_window(n, dtau=1.0)
        h = 1e-4
        fd = (_make(orc, tau=0.7 + h).window_objective(n) - _make(orc, tau=0.7 - h).window_objective(n)) / (2 * h)
        tol = 1e-6
    else:
        e = np.array([1.0, 0, 0]) if which == "gx" else np.array([0, 0, 1.0])
        J, dJ = _make(orc).tangent_window(n, dg=e)
        h = 1e-7
        fd = (_make(orc, g=G0 + h * e).window_objective(n) - _make(orc, g=G0 - h * e).window_objective(n)) / (2 * h)
        tol = 1e-8
    assert abs(dJ - fd) <= tol * abs(dJ), (dJ, fd)
    assert abs(J - _make(orc).window_objective(n)) <= 1e-12 * abs(J)
