"""Pins of the oracle's Krylov solvers (CPU only).

* CG (textbook Hestenes-Stiefel) against a dense direct solve of M_ee by the
  oracle's own LU, itself cross-checked against numpy;
* multi-shift CG (Sec. 3.2, co-linear shifted residuals) against dense solves
  per shift, the co-linearity invariant ``b - (A + s_i) x_i = zeta_i r`` and
  the single-shift case, which must reproduce CG;
* BiCGStab(l) (Sec. 6.1) against a dense solve of the full ``2m + D`` and, at
  l = 1, against the textbook BiCGStab iterates written here from
  van der Vorst's recurrences (a different algorithm that coincides at l = 1);
* the stabilised mixed-precision CG with emulated sloppy storage (Sec. 3.1):
  with FP64 storage, exact links, no reliable update before convergence and
  Fletcher-Reeves beta it is textbook CG, bit for bit; in every storage format
  it reaches the FP64 true residual; and it reproduces the ordering Sec. 3.1
  argues for: at a light mass the Polak-Ribiere, re-projected recurrence
  converges where the plain Fletcher-Reeves one stalls;
* the multi-shift stage with emulated sloppy storage (Sec. 3.2): with FP64
  storage and no reliable update it is the FP64 multi-shift CG, bit for bit,
  on every shifted system; and, as Table 3 reports, a 30-bit stage leaves the
  shifted systems (those not yet at their target) with residuals more than an
  order of magnitude below those of an FP32 stage;
* BiCGStab(l) with emulated sloppy storage and reliable updates at the end of
  a cycle (Sec. 6.1): with FP64 storage it is the FP64 BiCGStab(l), bit for
  bit; at a light mass 20-bit storage needs fewer operator applications than
  16-bit storage, the ordering of Table 2.
"""
import math

import numpy as np
import pytest

from paper_2302_09224_gb300 import synth


def cvec(a):
    a = np.asarray(a)
    return (a[..., 0] + 1j * a[..., 1]).reshape(-1)


def rvec(v, shape):
    return np.stack([v.real, v.imag], axis=-1).reshape(shape)


def test_lu_matches_numpy(orc):
    g = np.random.Generator(np.random.Philox(key=1))
    a = g.standard_normal((40, 40)) + 1j * g.standard_normal((40, 40))
    b = g.standard_normal(40) + 1j * g.standard_normal(40)
    np.testing.assert_allclose(orc.lu_solve(a, b), np.linalg.solve(a, b), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims,m", [((2, 2, 2, 2), 0.1), ((4, 4, 4, 4), 0.1), ((4, 4, 4, 4), 0.02)])
def test_cg_vs_dense(orc, dims, m):
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, synth.rhs_seed(0)).numpy()
    a = orc.dense(dims, fat, lng, "mee", m=m)
    xd = orc.lu_solve(a, cvec(b))
    ev = np.linalg.eigvalsh(a)
    kappa = ev.max() / ev.min()
    tol = 1e-12
    x, st, it, tr = orc.cg(dims, fat, lng, m, b, tol)
    assert st == 0 and tr <= 10 * tol
    err = np.linalg.norm(cvec(x) - xd) / np.linalg.norm(xd)
    assert err <= kappa * 10 * tol
    assert it <= len(a) * 3


def test_cg_initial_guess_and_status(orc):
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1001).numpy()
    x, st, it, tr = orc.cg(dims, fat, lng, 0.05, b, 1e-12, maxiter=5)
    assert st == 1 and it == 5 and tr > 1e-6
    x2, st2, it2, tr2 = orc.cg(dims, fat, lng, 0.05, b, 1e-12, x0=x)
    assert st2 == 0 and tr2 <= 1e-11


def test_multishift_vs_dense(orc):
    dims = (4, 4, 4, 4)
    m = 0.05
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1000).numpy()
    sig = synth.shifts_logspaced(6, 1e-3, 1.0)
    tols = [1e-12] * 6
    x, st, its, z, r = orc.multishift_cg(dims, fat, lng, m, sig, tols, b)
    assert st == 0
    for i, s in enumerate(sig):
        a = orc.dense(dims, fat, lng, "mee", m=m, sigma=s)
        xd = np.linalg.solve(a, cvec(b))
        assert np.linalg.norm(cvec(x[i]) - xd) <= 1e-9 * np.linalg.norm(xd)
    # heavier shifts converge first
    assert all(its[i] >= its[i + 1] for i in range(5))


def test_multishift_colinearity(orc):
    dims = (4, 4, 4, 6)
    m = 0.02
    fat, lng = synth.gauge_pair(dims, seed=1)
    b = synth.spinor(dims, 1003).numpy()
    sig = [0.0, 0.01, 0.1, 0.7]
    x, st, its, z, r = orc.multishift_cg(dims, fat, lng, m, sig, [0.0] * 4, b, maxiter=25)
    assert st == 1 and all(i == 25 for i in its)
    bn = np.linalg.norm(cvec(b))
    for i, s in enumerate(sig):
        res = cvec(b) - cvec(orc.mee(dims, fat, lng, m, x[i], sigma=s))
        assert np.linalg.norm(res - z[i] * cvec(r)) <= 1e-10 * bn
    assert z[0] == 1.0
    assert all(abs(z[i + 1]) < abs(z[i]) for i in range(3))


def test_multishift_single_shift_is_cg(orc):
    dims = (4, 4, 4, 4)
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1000).numpy()
    xs, st, its, z, r = orc.multishift_cg(dims, fat, lng, 0.05, [0.2], [1e-11], b)
    xc, stc, itc, trc = orc.cg(dims, fat, lng, 0.05, b, 1e-11, sigma=0.2)
    assert its[0] == itc
    np.testing.assert_allclose(xs[0], xc, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dims,l", [((2, 2, 2, 2), 4), ((4, 4, 4, 4), 4), ((4, 4, 4, 4), 2)])
def test_bicgstabl_vs_dense(orc, dims, l):
    m = 0.1
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1000, full=True).numpy()
    a = orc.dense(dims, fat, lng, "mfull", m=m)
    xd = orc.lu_solve(a, cvec(b))
    x, st, mv, tr = orc.bicgstabl(dims, fat, lng, m, b, l, 1e-12)
    assert st == 0 and tr <= 1e-11
    assert np.linalg.norm(cvec(x) - xd) <= 1e-8 * np.linalg.norm(xd)
    assert mv % (2 * l) == 0


def _textbook_bicgstab(apply, b, iters):
    x = np.zeros_like(b)
    r = b.copy()
    rh = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for _ in range(iters):
        rho_new = np.vdot(rh, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply(p)
        alpha = rho_new / np.vdot(rh, v)
        s = r - alpha * v
        t = apply(s)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
    return x


@pytest.mark.parametrize("m,k", [(2.0, 12), (0.05, 2)])
def test_bicgstabl_l1_is_bicgstab(orc, m, k):
    # M = 2m + D has a spectrum 2m + i*lambda; at light mass BiCGStab's
    # minimal-residual step is nearly singular and rounding differences grow
    # chaotically, so the iterate comparison runs at a heavy mass for many
    # cycles and at a light mass for the first cycles only
    dims = (4, 4, 4, 6)
    fat, lng = synth.gauge_pair(dims, seed=2)
    b = synth.spinor(dims, 1005, full=True).numpy()
    shape = b.shape

    def apply(v):
        return cvec(orc.mfull(dims, fat, lng, m, rvec(v, shape)))

    xt = _textbook_bicgstab(apply, cvec(b), k)
    x, st, mv, tr = orc.bicgstabl(dims, fat, lng, m, b, 1, 0.0, max_matvecs=2 * k)
    assert mv == 2 * k
    assert np.linalg.norm(cvec(x) - xt) <= 1e-11 * np.linalg.norm(xt)


def test_mixed_cg_reduces_to_textbook_cg(orc):
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000).numpy()
    x0, st0, it0, _ = orc.cg(dims, fat, lng, m, b, 1e-10)
    # FP64 storage, exact links, delta = 0 (one reliable update, at convergence), FR beta: the same recurrence
    x, st, it, ru, tr, hist = orc.mixed_cg(dims, fat, lng, m, b, "f64", 1e-10, delta=0.0, pr=False,
                                           reproject=False)
    assert st == st0 == 0 and it == it0 and ru == 1
    np.testing.assert_array_equal(x, x0)
    assert hist[0] == pytest.approx(1.0) and hist[-1] <= 1e-10
    # Polak-Ribiere equals Fletcher-Reeves in exact arithmetic (r_new is orthogonal to r_old)
    x, st, it, ru, tr, _ = orc.mixed_cg(dims, fat, lng, m, b, "f64", 1e-10, delta=0.0, pr=True, reproject=True)
    assert st == 0 and abs(it - it0) <= 1 and tr <= 1e-10
    assert np.linalg.norm(x - x0) / np.linalg.norm(x0) <= 1e-9


@pytest.mark.parametrize("sfmt", ["f32", "half", "int20", "int30", "int14"])
def test_mixed_cg_emulated_formats_converge(orc, sfmt):
    dims, m = (8, 8, 8, 8), 0.05
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000).numpy()
    gf = "fix32" if sfmt == "int30" else ("f32" if sfmt == "f32" else "fix16")
    fs = orc.gauge_emulate(dims, fat, gf, 18, False)
    ls = orc.gauge_emulate(dims, lng, gf, 12, True)
    _, _, it0, _ = orc.cg(dims, fat, lng, m, b, 1e-10)
    x, st, it, ru, tr, hist = orc.mixed_cg(dims, fat, lng, m, b, sfmt, 1e-10, fat_s=fs, lng_s=ls)
    assert st == 0 and tr <= 1e-10
    assert ru >= 2  # delta = 0.1 fires before convergence
    assert it <= 1.1 * it0
    r = b - orc.mee(dims, fat, lng, m, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) == pytest.approx(tr, rel=1e-6)


def test_mixed_cg_stabilisation_ordering(orc):
    dims, m = (6, 6, 6, 6), 0.002
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000).numpy()
    fs = orc.gauge_emulate(dims, fat, "fix16", 18, False)
    ls = orc.gauge_emulate(dims, lng, "fix16", 12, True)
    _, st_s, it_s, _, tr_s, _ = orc.mixed_cg(dims, fat, lng, m, b, "half", 1e-10, fat_s=fs, lng_s=ls, pr=True,
                                             reproject=True, maxiter=8000)
    _, st_p, it_p, _, tr_p, _ = orc.mixed_cg(dims, fat, lng, m, b, "half", 1e-10, fat_s=fs, lng_s=ls, pr=False,
                                             reproject=False, maxiter=8000)
    assert st_s == 0 and tr_s <= 1e-10
    assert st_p == 1 and tr_p > 1e-10


def ms_case():
    dims, m = (8, 8, 8, 8), 0.01
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000).numpy()
    return dims, m, fat, lng, b, synth.shifts_logspaced(6, 1e-4, 1.0), synth.shift_tolerances(6, 1e-10, 1e-7)


def test_mixed_multishift_reduces_to_multishift_cg(orc):
    dims, m, fat, lng, b, sig, tols = ms_case()
    x0, st0, its0, _, _ = orc.multishift_cg(dims, fat, lng, m, sig, tols, b)
    x, st, it, ru, its, res = orc.mixed_multishift(dims, fat, lng, m, sig, tols, b, "f64", delta=0.0)
    assert st == st0 == 0 and ru == 0
    assert it == max(its0[1:])  # the stage ends when the last shifted system stops
    for i in range(1, len(sig)):
        assert its[i] == its0[i]
        np.testing.assert_array_equal(x[i], x0[i])
        assert res[i] <= 2 * tols[i]


def test_mixed_multishift_int30_beats_fp32(orc):
    dims, m, fat, lng, b, sig, tols = ms_case()
    res = {}
    for sfmt, gfmt in (("int30", "fix32"), ("f32", "f32")):
        f32 = sfmt == "f32"  # the 30-bit triplet decodes its 32-bit links in FP64
        fs = orc.gauge_emulate(dims, fat, gfmt, 18, False, compute_f32=f32)
        ls = orc.gauge_emulate(dims, lng, gfmt, 12, True, compute_f32=f32)
        _, st, _, ru, _, r = orc.mixed_multishift(dims, fat, lng, m, sig, tols, b, sfmt, fat_s=fs, lng_s=ls)
        assert st == 0 and ru >= 1
        res[sfmt] = r
    open_shifts = [i for i in range(1, len(sig)) if res["int30"][i] > tols[i]]
    assert len(open_shifts) >= 3
    for i in open_shifts:
        assert res["f32"][i] > 10 * res["int30"][i]


def test_mixed_bicgstabl_reduces_to_bicgstabl(orc):
    dims, m = (4, 4, 4, 8), 0.1
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000, full=True).numpy()
    x0, st0, mv0, tr0 = orc.bicgstabl(dims, fat, lng, m, b, 4, 1e-10)
    x, st, mv, ru, tr = orc.mixed_bicgstabl(dims, fat, lng, m, b, 4, "f64", 1e-10, delta=0.0)
    assert st == st0 == 0 and mv == mv0 and ru == 1 and tr == tr0
    np.testing.assert_array_equal(x, x0)


def test_mixed_bicgstabl_int20_beats_half(orc):
    dims, m = (4, 4, 4, 8), 0.002
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000, full=True).numpy()
    fs = orc.gauge_emulate(dims, fat, "fix16", 18, False)
    ls = orc.gauge_emulate(dims, lng, "fix16", 12, True)
    mv = {}
    for sfmt in ("int20", "half"):
        _, st, mv[sfmt], ru, tr = orc.mixed_bicgstabl(dims, fat, lng, m, b, 4, sfmt, 1e-10, fat_s=fs, lng_s=ls,
                                                      max_matvecs=40000)
        assert st == 0 and tr <= 1e-10 and ru >= 2
    assert mv["int20"] < mv["half"]


def test_mixed_cg_error_estimate_trigger_limits(orc):
    """The error-estimate trigger (the footnote of Sec. 3, after van der Vorst
    and Ye's residual replacement) with a vanishing precision never fires
    before convergence, so the run is the delta = 0 run bit for bit.  With FP64
    storage the estimate only grows with the precision it is given: the
    coarser that precision, the earlier d crosses sqrt(eps) |r|, so the more
    reliable updates, while the iterates (FP64 everywhere) stay those of CG."""
    dims, m = (4, 4, 4, 4), 0.1
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000).numpy()
    x0, st0, it0, ru0, tr0, h0 = orc.mixed_cg(dims, fat, lng, m, b, "f64", 1e-10, delta=0.0)
    x1, st1, it1, ru1, tr1, h1 = orc.mixed_cg(dims, fat, lng, m, b, "f64", 1e-10, dyn_eps=1e-300)
    assert st0 == st1 == 0 and it0 == it1 and ru0 == ru1 == 1
    np.testing.assert_array_equal(x0, x1)
    np.testing.assert_array_equal(h0, h1)
    rus = []
    for e in (2.0 ** -53, 2.0 ** -24, 2.0 ** -15):
        _, st2, it2, ru2, tr2, _ = orc.mixed_cg(dims, fat, lng, m, b, "f64", 1e-10, dyn_eps=e)
        assert st2 == 0 and abs(it2 - it0) <= 4 and tr2 <= 1e-10
        rus.append(ru2)
    assert rus[0] < rus[1] < rus[2]


@pytest.mark.parametrize("sfmt,gf,eps", [("half", "fix16", 2.0 ** -15), ("int20", "fix16", 2.0 ** -15),
                                         ("int30", "fix32", 2.0 ** -29)])
def test_mixed_cg_error_estimate_trigger_converges(orc, sfmt, gf, eps):
    """At the light mass where Fletcher-Reeves without re-projection stalls,
    the stabilised CG driven by the error-estimate trigger reaches the FP64
    true residual; its history shows the recomputed residual at each reliable
    update, and updates come more often the coarser the sloppy format."""
    dims, m = (6, 6, 6, 6), 0.002
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000).numpy()
    fs = orc.gauge_emulate(dims, fat, gf, 18, False)
    ls = orc.gauge_emulate(dims, lng, gf, 12, True)
    x, st, it, ru, tr, hist = orc.mixed_cg(dims, fat, lng, m, b, sfmt, 1e-10, fat_s=fs, lng_s=ls, dyn_eps=eps,
                                           maxiter=8000)
    assert st == 0 and tr <= 1e-10 and ru >= 2
    assert hist[-1] == pytest.approx(tr, rel=1e-12)
    r = b - orc.mee(dims, fat, lng, m, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) == pytest.approx(tr, rel=1e-6)


@pytest.mark.parametrize("rho,c,eps", [(0.9, 0.5, 2.0 ** -15), (0.8, 2.0, 2.0 ** -19), (0.95, 0.1, 2.0 ** -29),
                                       (0.7, 0.0, 2.0 ** -24)])
def test_ru_trigger_closed_form(orc, rho, c, eps):
    """The error-estimate trigger's rule on a geometric sequence |r_k| = rho^k with |alpha_k| |A p_k| =
    c rho^k: the drift estimate is d_k = eps (1 + A (1 - rho^k)), A = (rho + c) / (1 - rho), which
    first exceeds sqrt(eps) |r_m| at the smallest m with rho^m < Q = sqrt(eps) (1 + A) / (1 + sqrt(eps) A);
    the trigger fires in the step that ends there, k = m - 1 (with d_m far above 1.1 d_0)."""
    A = (rho + c) / (1 - rho)
    h = math.sqrt(eps)
    Q = h * (1 + A) / (1 + h * A)
    t = math.log(Q) / math.log(rho)
    assert abs(t - round(t)) > 1e-6  # not on the boundary, where rounding would decide
    m = math.floor(t) + 1
    n = m + 10
    r = rho ** np.arange(n + 1, dtype=float)
    aa = c * rho ** np.arange(n, dtype=float)
    assert orc.ru_trigger_first(r, aa, eps) == m - 1


def test_ru_trigger_guards(orc):
    """A drift that crosses sqrt(eps) |r| within its first 10 % never fires (it starts above the
    threshold from then on), and as eps vanishes the estimate never crosses it."""
    r = 0.01 ** np.arange(6, dtype=float)
    assert orc.ru_trigger_first(r, np.zeros(5), 0.01) == -1
    r = 0.9 ** np.arange(101, dtype=float)
    assert orc.ru_trigger_first(r, 0.5 * r[:-1], 1e-300) == -1
