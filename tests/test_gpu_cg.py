"""GPU CG (plain FP64 and stabilised mixed precision, Sec. 3.1) against the oracle.

* 2^4 and 4^4: the solution against the oracle's dense direct solve;
* larger lattices: the FP64 true residual of the returned x, recomputed by the
  CPU oracle, must reach the requested tolerance for every sloppy format;
* the paper's claim that re-projection and Polak-Ribiere keep mixed CG close
  to the FP64 iteration count is checked as an ordering (iterations of the
  stabilised half-precision solve within a small factor of FP64 CG);
* graph and direct launches give bitwise identical solutions (deterministic
  reductions), host and device pointers agree, maxiter gives ENOTCONV with the
  best x, bad inputs give EINVAL.
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


def true_res(orc, dims, fat, lng, m, b, x, sigma=0.0):
    r = np.asarray(b) - orc.mee(dims, fat, lng, m, x, sigma=sigma)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def solve(ctx, dims, fat, lng, m, b, name="int20", tol=1e-10, **kw):
    g = hisq.hisq_load_gauge(ctx, dims, torch.as_tensor(fat).cuda(), torch.as_tensor(lng).cuda())
    try:
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.on_device = m, tol, 1
        p.sloppy = hisq.prec(name, 12)
        for k, v in kw.items():
            setattr(p, k, v)
        bd = torch.as_tensor(b).cuda()
        x = torch.zeros_like(bd)
        st, info = hisq.hisq_cg(ctx, g, p, bd, x)
        return st, info, x.cpu().numpy()
    finally:
        hisq.hisq_free_gauge(ctx, g)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
@pytest.mark.parametrize("name", ["f64", "int20", "half"])
def test_cg_vs_dense(ctx, orc, dims, name):
    m = 0.1
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1000).numpy()
    a = orc.dense(dims, fat, lng, "mee", m=m)
    xd = orc.lu_solve(a, cvec(b))
    st, info, x = solve(ctx, dims, fat, lng, m, b, name, tol=1e-11)
    assert st == hisq.HISQ_OK
    ev = np.linalg.eigvalsh(a)
    assert np.linalg.norm(cvec(x) - xd) <= 10 * (ev.max() / ev.min()) * 1e-11 * np.linalg.norm(xd)
    assert true_res(orc, dims, fat, lng, m, b, x) <= 1e-11
    assert abs(info.true_residual - true_res(orc, dims, fat, lng, m, b, x)) < 1e-12


@pytest.mark.parametrize("name", ["f64", "f32", "half", "int20", "int30", "int30f32", "int14", "int20se"])
def test_cg_true_residual_8x4(ctx, orc, name):
    """The config-1 lattice (8^4, m = 0.1, tol 1e-10) in every sloppy format."""
    dims, m = (8, 8, 8, 8), 0.1
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, synth.rhs_seed(0)).numpy()
    st, info, x = solve(ctx, dims, fat, lng, m, b, name)
    assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
    tr = true_res(orc, dims, fat, lng, m, b, x)
    assert tr <= 1e-10
    assert info.true_residual <= 1e-10
    if name != "f64":
        assert info.reliable_updates >= 1


def test_cg_light_mass_orderings(ctx, orc):
    """m = 0.01 on 8^3 x 16: stabilised mixed CG converges with few extra iterations."""
    dims, m = (8, 8, 8, 16), 0.01
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1000).numpy()
    res = {}
    for name in ("f64", "half", "int20"):
        st, info, x = solve(ctx, dims, fat, lng, m, b, name, tol=1e-10)
        assert st == hisq.HISQ_OK
        assert true_res(orc, dims, fat, lng, m, b, x) <= 1e-10
        res[name] = info.iters
    assert res["int20"] <= 1.5 * res["f64"]
    assert res["half"] <= 2.0 * res["f64"]


def test_graph_matches_direct_and_is_deterministic(ctx):
    dims, m = (8, 8, 8, 8), 0.05
    fat, lng = synth.gauge_pair(dims, seed=1)
    b = synth.spinor(dims, 1001).numpy()
    _, i1, x1 = solve(ctx, dims, fat, lng, m, b, "int20", use_graph=1)
    _, i2, x2 = solve(ctx, dims, fat, lng, m, b, "int20", use_graph=0)
    _, i3, x3 = solve(ctx, dims, fat, lng, m, b, "int20", use_graph=1)
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(x1, x3)
    assert i1.iters == i2.iters == i3.iters


def test_profiler_sampling(ctx):
    """With a sample period of 4 the CG graphs time one block of iterations in
    four: the solution is bitwise the unprofiled one, the timed stencil
    launches are about a quarter of those timed with period 1, and every
    timed launch is accounted with its algorithmic bytes; period 0 is EINVAL."""
    dims, m = (8, 8, 8, 8), 0.05
    fat, lng = synth.gauge_pair(dims, seed=1)
    b = synth.spinor(dims, 1001).numpy()
    _, i0, x0 = solve(ctx, dims, fat, lng, m, b, "int20", use_graph=1)
    counts = {}
    try:
        for every in (1, 4):
            hisq.hisq_profile_sample(ctx, every)
            hisq.hisq_profile_reset(ctx)
            hisq.hisq_profile_enable(ctx, True)
            _, i1, x1 = solve(ctx, dims, fat, lng, m, b, "int20", use_graph=1)
            st = hisq.hisq_profile_read(ctx, hisq.HISQ_PROF_STENCIL)
            hisq.hisq_profile_enable(ctx, False)
            np.testing.assert_array_equal(x1, x0)
            assert i1.iters == i0.iters
            assert st.launches > 0 and st.ms > 0
            assert abs(st.bytes / st.launches - counts.get("per", st.bytes / st.launches)) < 1e-6 * st.bytes / st.launches
            counts["per"] = st.bytes / st.launches
            counts[every] = st.launches
    finally:
        hisq.hisq_profile_sample(ctx, 1)
    assert counts[4] < counts[1]
    assert counts[4] >= counts[1] // 4 - 16  # one block in four (blocks of 8 iterations, 2 passes each)
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        hisq.hisq_profile_sample(ctx, 0)


def test_host_pointers(ctx, orc):
    dims, m = (4, 4, 4, 8), 0.1
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1000).numpy()
    g = hisq.hisq_load_gauge(ctx, dims, fat, lng)
    try:
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.on_device = m, 1e-10, 0
        x = np.zeros_like(b)
        st, info = hisq.hisq_cg(ctx, g, p, b, x)
        assert st == hisq.HISQ_OK
        assert true_res(orc, dims, fat, lng, m, b, x) <= 1e-10
        # initial guess: already converged -> no iterations
        p.use_init_guess = 1
        st, info2 = hisq.hisq_cg(ctx, g, p, b, x)
        assert st == hisq.HISQ_OK and info2.iters == 0
    finally:
        hisq.hisq_free_gauge(ctx, g)


def test_maxiter_and_invalid(ctx, orc):
    dims, m = (8, 8, 8, 8), 0.01
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1000).numpy()
    st, info, x = solve(ctx, dims, fat, lng, m, b, "int20", maxiter=16)
    assert st == hisq.HISQ_ENOTCONV
    assert 16 <= info.iters <= 16 + 8
    tr = true_res(orc, dims, fat, lng, m, b, x)
    assert abs(tr - info.true_residual) <= 1e-6 * tr and tr < 1.0
    bad = b.copy()
    bad[2, 1, 0] = np.nan
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        solve(ctx, dims, fat, lng, m, bad)
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        solve(ctx, dims, fat, lng, m, b, nbuf=0)
    st, info, x = solve(ctx, dims, fat, lng, m, np.zeros_like(b))
    assert st == hisq.HISQ_OK and not x.any()


@pytest.mark.parametrize("name", ["f32", "int20", "half", "int30"])
def test_split_scalars(ctx, orc, name):
    """alpha and beta summed from the block partials by every block of the
    kernel that uses them (the default) or once, by a one-block launch and a
    last block: both reach the tolerance by the oracle's FP64 residual, with
    iteration counts within a few percent (they sum in different block shapes,
    so their rounding differs); the split chain is deterministic (graph and
    direct launches bitwise equal) and carries the error-estimate trigger,
    whose finisher reads the alpha record that block 0 writes."""
    dims, m = (8, 8, 8, 16), 0.01
    fat, lng = (f.numpy() for f in synth.gauge_pair(dims, seed=0))
    b = synth.spinor(dims, 1000).numpy()
    prev = hisq.hisq_cg_split_scalars(0)
    try:
        st0, i0, x0 = solve(ctx, dims, fat, lng, m, b, name)
        assert hisq.hisq_cg_split_scalars(1) == 0
        st1, i1, x1 = solve(ctx, dims, fat, lng, m, b, name)
        st2, i2, x2 = solve(ctx, dims, fat, lng, m, b, name, use_graph=0)
        st3, i3, x3 = solve(ctx, dims, fat, lng, m, b, name, ru_trigger=1)
    finally:
        hisq.hisq_cg_split_scalars(prev)
    # the solver stops on its own FP64 evaluation of |b - M x| / |b| <= 1e-10 and the oracle evaluates
    # it again in FP64: at m = 0.01 |x| is about 50 |b| per component and each component of M x sums
    # terms of about 10^3 |b|, so the two roundings may differ by about 1e-13 |b|, 1e-3 of the target
    for st, x in ((st0, x0), (st1, x1), (st3, x3)):
        assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
        assert true_res(orc, dims, fat, lng, m, b, x) <= 1e-10 * (1 + 1e-3)
    np.testing.assert_array_equal(x1, x2)
    assert i1.iters == i2.iters and i1.reliable_updates == i2.reliable_updates
    assert abs(i1.iters - i0.iters) <= 0.03 * i0.iters + 4, (i0.iters, i1.iters)
    assert i3.reliable_updates >= 2
    assert hisq.hisq_cg_split_scalars(2) == -2


def test_programmatic_launch_same_bits(ctx):
    """Kernels launched with programmatic dependent launch (each waiting for its
    predecessor's results before touching them) give the same solution, bit
    for bit, as kernels launched one after another, in graphs and directly."""
    dims, m = (8, 8, 8, 16), 0.02
    fat, lng = synth.gauge_pair(dims, seed=2)
    b = synth.spinor(dims, 1002).numpy()
    prev = hisq.hisq_programmatic_launch(0)
    try:
        ref = [solve(ctx, dims, fat, lng, m, b, name, use_graph=g)[2] for name in ("int20", "int30") for g in (0, 1)]
        hisq.hisq_programmatic_launch(1)
        got = [solve(ctx, dims, fat, lng, m, b, name, use_graph=g)[2] for name in ("int20", "int30") for g in (0, 1)]
    finally:
        hisq.hisq_programmatic_launch(prev)
    for a, r in zip(got, ref):
        np.testing.assert_array_equal(a, r)
    assert hisq.hisq_programmatic_launch(3) == -2
