"""Pins of the oracle's WENO5 reconstruction against definitions that do not
reuse its formulas: reconstruction polynomials from cell-average conditions,
Jiang-Shu smoothness indicators from their integral definition, and the
exactness orders of finite-difference WENO (Jiang & Shu 1996, the paper's WENO
reference in "Numerical approximation")."""
import numpy as np
import pytest

import oracle
from tests.analytic import jiang_shu_beta, stencil_face_value

D = np.array([0.1, 0.6, 0.3])


def _poly_values(coef, x):
    return sum(c * x ** k for k, c in enumerate(coef))


@pytest.mark.parametrize("seed", range(8))
def test_weights_and_value_match_definition(seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=5) * rng.choice([1e-3, 1.0, 30.0])
    eps = 1e-6
    beta = jiang_shu_beta(v)
    a = D / (eps + beta) ** 2
    w_ref = a / a.sum()
    p_ref = stencil_face_value(v)
    val, w = oracle.weno5(v, eps)
    assert np.allclose(w, w_ref, rtol=1e-10, atol=1e-14)
    assert val == pytest.approx(float(w_ref @ p_ref), rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_quadratics_exact_for_any_weights(seed):
    # For point values f of a quadratic, FD-WENO reconstructs H with
    # cell-averages f, i.e. H = f - f''/24 (dx = 1), at the face x = 1/2.
    rng = np.random.default_rng(100 + seed)
    c = rng.normal(size=3)
    x = np.arange(-2, 3, dtype=np.float64)
    v = _poly_values(c, x)
    H_face = _poly_values(c, 0.5) - 2 * c[2] / 24.0
    val, _ = oracle.weno5(v, 1e-6)
    assert val == pytest.approx(H_face, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_quartics_exact_with_linear_weights(seed):
    # With eps >> beta the weights are the linear ones (0.1, 0.6, 0.3) and the
    # reconstruction is exact for degree 4: H = f - f''/24 + 7 f''''/5760.
    rng = np.random.default_rng(200 + seed)
    c = rng.normal(size=5)
    x = np.arange(-2, 3, dtype=np.float64)
    v = _poly_values(c, x)
    d2 = lambda z: 2 * c[2] + 6 * c[3] * z + 12 * c[4] * z * z
    H_face = _poly_values(c, 0.5) - d2(0.5) / 24.0 + 7.0 * 24.0 * c[4] / 5760.0
    val, w = oracle.weno5(v, 1e30)
    assert np.allclose(w, D, rtol=1e-12)
    assert val == pytest.approx(H_face, rel=1e-11, abs=1e-11)


def test_step_picks_smooth_stencil():
    val, w = oracle.weno5([0.0, 0.0, 0.0, 1.0, 1.0], 1e-6)
    assert w[0] > 0.999 and abs(val) < 1e-6
    val, w = oracle.weno5([0.0, 0.0, 1.0, 1.0, 1.0], 1e-6)
    assert w[2] > 0.999 and abs(val - 1.0) < 1e-6


@pytest.mark.parametrize("seed", range(4))
def test_odd_symmetry_exact(seed):
    # W(-v) = -W(v) bit for bit: what makes the wall mass flux exactly zero.
    v = np.random.default_rng(300 + seed).normal(size=5)
    assert oracle.weno5(-v)[0] == -oracle.weno5(v)[0]
