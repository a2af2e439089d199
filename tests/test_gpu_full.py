"""GPU full-lattice solve (2m + D) x = b by even/odd reduction (hisq_solve_full),
the error-estimate reliable-update trigger and the CG residual history.

* hisq_solve_full against the oracle's dense LU solve of the full M on 2^4 and
  4^4, and against the oracle-recomputed FP64 full residual |b - M x|/|b| on
  larger lattices in every sloppy format, negative mass included; the
  library's own full residual agrees with the oracle's;
* batched right-hand sides (nrhs > 1) give each system's bits independent of
  its companions, and host pointers give the device pointers' bits;
* the error-estimate trigger (the Sec. 3 footnote's dynamic choice) reaches
  the FP64 true residual in every format and makes reliable updates; in a
  batch it runs per right-hand side;
* the residual history (Fig. 1's quantity): entry 0 is 1 for x = 0, its
  length is the iteration count plus one, its last entry is the final true
  residual, and at a light mass the naive double-half CG (reliable updates
  only) stalls where the stabilised one converges, the ordering Sec. 3.1
  reports with Fig. 1.
"""
import numpy as np
import pytest
import torch

from paper_2302_09224_gb300 import hisq, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = hisq.hisq_create(0)
    yield c
    hisq.hisq_destroy(c)


def cvec(a):
    a = np.asarray(a)
    return (a[..., 0] + 1j * a[..., 1]).reshape(-1)


def full_res(orc, dims, fat, lng, m, b, x):
    r = np.asarray(b) - orc.mfull(dims, fat, lng, m, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def solve_full(ctx, dims, fat, lng, m, bs, name="int20", tol=1e-10, on_device=True, **kw):
    g = hisq.hisq_load_gauge(ctx, dims, torch.as_tensor(fat).cuda(), torch.as_tensor(lng).cuda())
    try:
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.on_device = m, tol, int(on_device)
        p.sloppy = hisq.prec(name, 12)
        p.nrhs = len(bs)
        for k, v in kw.items():
            setattr(p, k, v)
        b = np.ascontiguousarray(np.stack(bs))
        if on_device:
            bd = torch.from_numpy(b).cuda()
            x = torch.zeros_like(bd)
            st, info = hisq.hisq_solve_full(ctx, g, p, bd, x)
            return st, info, x.cpu().numpy()
        x = np.zeros_like(b)
        st, info = hisq.hisq_solve_full(ctx, g, p, b, x)
        return st, info, x
    finally:
        hisq.hisq_free_gauge(ctx, g)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
@pytest.mark.parametrize("name", ["f64", "int20"])
def test_full_vs_dense(ctx, orc, dims, name):
    m, tol = 0.1, 1e-11
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1500, full=True).numpy()
    a = orc.dense(dims, fat, lng, "mfull", m=m)
    xd = orc.lu_solve(a, cvec(b))
    sv = np.linalg.svd(a, compute_uv=False)
    st, info, x = solve_full(ctx, dims, fat, lng, m, [b], name, tol=tol)
    assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
    tr = full_res(orc, dims, fat, lng, m, b, x[0])
    assert tr <= tol
    assert abs(info.true_residual - tr) <= 0.05 * tr + 1e-15
    assert np.linalg.norm(cvec(x[0]) - xd) <= 10 * (sv.max() / sv.min()) * tol * np.linalg.norm(xd)


@pytest.mark.parametrize("name", ["f64", "f32", "half", "int20", "int30", "int30f32"])
@pytest.mark.parametrize("dims,m", [((8, 8, 8, 8), 0.05), ((6, 4, 4, 10), -0.03)])
def test_full_true_residual(ctx, orc, name, dims, m):
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1501, full=True).numpy()
    st, info, x = solve_full(ctx, dims, fat, lng, m, [b], name)
    assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
    tr = full_res(orc, dims, fat, lng, m, b, x[0])
    assert tr <= 1e-10, (name, tr)
    assert abs(info.true_residual - tr) <= 0.05 * tr + 1e-15
    # the even half solves the Schur system the oracle defines
    xo = orc.reconstruct_odd(dims, fat, lng, m, b[1], x[0][0])
    assert np.linalg.norm(xo - x[0][1]) <= 1e-12 * np.linalg.norm(xo)


def test_full_batched_and_host(ctx, orc):
    dims, m = (8, 8, 8, 16), 0.03
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=1))
    bs = [synth.spinor(dims, 1600 + k, full=True).numpy() for k in range(4)]
    st, info, x4 = solve_full(ctx, dims, fat, lng, m, bs, "int20", rhs_tile=2)
    assert st == hisq.HISQ_OK
    for b, x in zip(bs, x4):
        assert full_res(orc, dims, fat, lng, m, b, x) <= 1e-10
    _, _, x2 = solve_full(ctx, dims, fat, lng, m, bs[:2], "int20", rhs_tile=2)
    np.testing.assert_array_equal(x4[:2], x2)
    st, _, xh = solve_full(ctx, dims, fat, lng, m, bs[:1], "int20", on_device=False)
    _, _, xd = solve_full(ctx, dims, fat, lng, m, bs[:1], "int20", on_device=True)
    assert st == hisq.HISQ_OK
    np.testing.assert_array_equal(xh, xd)


def test_full_refusals(ctx):
    dims = (4, 4, 4, 4)
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1502, full=True).numpy()
    with pytest.raises(hisq.HisqError, match="nonzero"):
        solve_full(ctx, dims, fat, lng, 0.0, [b])
    st, info, x = solve_full(ctx, dims, fat, lng, 0.1, [np.zeros_like(b)])
    assert st == hisq.HISQ_OK and not x.any() and info.true_residual == 0.0


def cg(ctx, dims, fat, lng, m, b, name, hist=None, **kw):
    g = hisq.hisq_load_gauge(ctx, dims, torch.as_tensor(fat).cuda(), torch.as_tensor(lng).cuda())
    try:
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.on_device = m, 1e-10, 1
        p.sloppy = hisq.prec(name, 12)
        for k, v in kw.items():
            setattr(p, k, v)
        if hist is not None:
            hisq.set_history(p, hist)
        bd = torch.as_tensor(b).cuda()
        x = torch.zeros_like(bd)
        st, info = hisq.hisq_cg(ctx, g, p, bd, x)
        return st, info, x.cpu().numpy()
    finally:
        hisq.hisq_free_gauge(ctx, g)


def true_res(orc, dims, fat, lng, m, b, x):
    r = np.asarray(b) - orc.mee(dims, fat, lng, m, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


@pytest.mark.parametrize("name", ["f32", "half", "int20", "int30", "int30f32"])
def test_error_estimate_trigger(ctx, orc, name):
    dims, m = (8, 8, 8, 16), 0.01
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000).numpy()
    st, info, x = cg(ctx, dims, fat, lng, m, b, name, ru_trigger=1)
    assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
    assert true_res(orc, dims, fat, lng, m, b, x) <= 1e-10
    assert info.reliable_updates >= 2
    st0, info0, _ = cg(ctx, dims, fat, lng, m, b, name, ru_trigger=0)
    assert info.iters <= 1.5 * info0.iters + 16


def test_error_estimate_trigger_batched(ctx, orc):
    dims, m = (8, 8, 8, 16), 0.01
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    bs = [synth.spinor(dims, synth.rhs_seed(k)).numpy() for k in range(4)]
    st, info, xs = cg(ctx, dims, fat, lng, m, np.stack(bs), "int20", ru_trigger=1, nrhs=4, rhs_tile=2)
    assert st == hisq.HISQ_OK
    for b, x in zip(bs, xs):
        assert true_res(orc, dims, fat, lng, m, b, x) <= 1e-10


def test_history_and_fig1_ordering(ctx, orc):
    dims, m, cap = (6, 6, 6, 6), 0.002, 8000
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000).numpy()
    runs = {}
    for label, name, kw in [("double", "f64", {}), ("stabilised", "half", {}),
                            ("naive", "half", dict(pr_beta=0, reproject=0))]:
        h = np.full(cap + 1, np.nan)
        st, info, x = cg(ctx, dims, fat, lng, m, b, name, hist=h, maxiter=cap, **kw)
        n = min(info.iters + 1, h.size)
        assert np.isfinite(h[:n]).all() and np.isnan(h[n:]).all()
        assert h[0] == pytest.approx(1.0, rel=1e-12)
        runs[label] = (st, info, h[:n], x)
    for label in ("double", "stabilised"):
        st, info, h, x = runs[label]
        assert st == hisq.HISQ_OK, (label, hisq.STATUS_NAMES[st], info.iters, info.true_residual)
        assert h[-1] == pytest.approx(info.true_residual, rel=1e-9)
        assert true_res(orc, dims, fat, lng, m, b, x) <= 1e-10
    # 1/kappa (about 3e-7 here) is far below the 16-bit epsilon, the regime Sec. 3.3 names as the limit
    # of reduced precision: the stabilised solve converges, with more iterations than FP64, while the
    # naive one (reliable updates only) does not within the cap, or needs more still
    st, info, h, x = runs["naive"]
    assert st == hisq.HISQ_ENOTCONV or info.iters > runs["stabilised"][1].iters
    assert runs["stabilised"][1].iters >= runs["double"][1].iters
