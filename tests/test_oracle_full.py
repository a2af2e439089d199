"""Pins of the oracle's full-system solve by even/odd reduction (CPU only).

The solvers of Sec. 3 work on the even-site system M_ee x_e = 2m b_e - D_eo b_o
(M_ee = 4m^2 - D_eo D_oe); the full solution of (2m + D) x = b follows from
x_o = (b_o - D_oe x_e)/(2m).  Pinned here against what the block algebra of
M = [[2m, D_eo], [D_oe, 2m]] fixes, using only the separately pinned stencil
and operators:

* a known solution is recovered: for b = M x* the Schur source equals
  M_ee x*_e and the reconstruction from x*_e returns x*_o;
* for any x_e the reconstructed full residual vanishes on the odd sites and
  is the Schur residual over 2m on the even ones;
* the whole solve agrees with a dense LU solve of the full M (the oracle's own
  LU, cross-checked against numpy elsewhere) on 2^4 and 4^4, where the
  three-hop term aliases, and reaches its target true residual;
* a wrong sign of the D_eo term, a dropped 2m or a wrong parity fails each of
  these.
"""
import numpy as np
import pytest

from paper_2302_09224_gb300 import synth


def cvec(a):
    a = np.asarray(a)
    return (a[..., 0] + 1j * a[..., 1]).reshape(-1)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("dims,m", [((2, 2, 2, 2), 0.1), ((4, 4, 4, 6), 0.05), ((6, 4, 4, 8), -0.07)])
def test_known_solution_is_recovered(orc, dims, m):
    fat, lng = synth.gauge_pair(dims, seed=3)
    xs = synth.spinor(dims, 1200, full=True).numpy()
    b = orc.mfull(dims, fat, lng, m, xs)
    bt = orc.schur_source(dims, fat, lng, m, b)
    assert rel(bt, orc.mee(dims, fat, lng, m, xs[0])) <= 1e-13
    xo = orc.reconstruct_odd(dims, fat, lng, m, b[1], xs[0])
    assert rel(xo, xs[1]) <= 1e-13


@pytest.mark.parametrize("dims,m", [((4, 4, 4, 4), 0.1), ((4, 6, 4, 8), 0.02)])
def test_reconstructed_residual_identity(orc, dims, m):
    fat, lng = synth.gauge_pair(dims, seed=4)
    b = synth.spinor(dims, 1300, full=True).numpy()
    xe = synth.spinor(dims, 1301).numpy()      # any even field, not a solution
    xo = orc.reconstruct_odd(dims, fat, lng, m, b[1], xe)
    x = np.stack([xe, xo])
    r = b - orc.mfull(dims, fat, lng, m, x)
    assert np.linalg.norm(r[1]) <= 1e-13 * np.linalg.norm(b)
    rs = orc.schur_source(dims, fat, lng, m, b) - orc.mee(dims, fat, lng, m, xe)
    assert rel(r[0], rs / (2 * m)) <= 1e-12


@pytest.mark.parametrize("dims,m", [((2, 2, 2, 2), 0.1), ((4, 4, 4, 4), 0.05), ((4, 4, 4, 4), -0.03)])
def test_solve_full_vs_dense(orc, dims, m):
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1400, full=True).numpy()
    a = orc.dense(dims, fat, lng, "mfull", m=m)
    xd = orc.lu_solve(a, cvec(b))
    sv = np.linalg.svd(a, compute_uv=False)
    kappa = sv.max() / sv.min()
    tol = 1e-12
    x, st, it, tr = orc.solve_full(dims, fat, lng, m, b, tol)
    assert st == 0 and tr <= tol
    assert np.linalg.norm(cvec(x) - xd) <= kappa * tol * np.linalg.norm(xd)


def test_zero_source_and_status(orc):
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_pair(dims, seed=0)
    x, st, it, tr = orc.solve_full(dims, fat, lng, 0.1, np.zeros((2, 128, 3, 2)), 1e-10)
    assert st == 0 and it == 0 and tr == 0.0 and not x.any()
    b = synth.spinor(dims, 1401, full=True).numpy()
    x, st, it, tr = orc.solve_full(dims, fat, lng, 0.01, b, 1e-12, maxiter=3)
    assert st == 1 and it == 3 and tr > 1e-6
