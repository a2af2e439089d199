"""GPU BiCGStab(l) (Sec. 6.1) on the full-lattice operator 2m + D against the oracle.

* 2^4 and 4^4: the solution against the oracle's dense direct solve;
* 8^4 and 8^3 x 16: the FP64 true residual of x recomputed by the CPU oracle
  reaches the target in every sloppy format, for l = 1, 2 and 4;
* Table 2's finding as an ordering at light mass: the 20-bit sloppy solve needs
  fewer operator applications than the 16-bit one.
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


def run(ctx, dims, fat, lng, m, b, name="int20", l=4, tol=1e-10, **kw):
    g = hisq.hisq_load_gauge(ctx, dims, torch.as_tensor(fat).cuda(), torch.as_tensor(lng).cuda())
    try:
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.on_device, p.l = m, tol, 1, l
        p.sloppy = hisq.prec(name, 12)
        for k, v in kw.items():
            setattr(p, k, v)
        bd = torch.as_tensor(b).cuda()
        x = torch.zeros_like(bd)
        st, info = hisq.hisq_bicgstabl(ctx, g, p, bd, x)
        return st, info, x.cpu().numpy()
    finally:
        hisq.hisq_free_gauge(ctx, g)


def true_res(orc, dims, fat, lng, m, b, x):
    r = b - orc.mfull(dims, fat, lng, m, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_vs_dense(ctx, orc, dims):
    m = 0.1
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1000, full=True).numpy()
    a = orc.dense(dims, fat, lng, "mfull", m=m)
    xd = orc.lu_solve(a, cvec(b))
    st, info, x = run(ctx, dims, fat, lng, m, b, "f64", tol=1e-11)
    assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
    sv = np.linalg.svd(a, compute_uv=False)
    assert np.linalg.norm(cvec(x) - xd) <= 10 * sv[0] / sv[-1] * 1e-11 * np.linalg.norm(xd)
    assert true_res(orc, dims, fat, lng, m, b, x) <= 1e-11


@pytest.mark.parametrize("name", ["f64", "f32", "half", "int20", "int30", "int14"])
@pytest.mark.parametrize("l", [1, 2, 4])
def test_true_residual(ctx, orc, name, l):
    dims, m = (8, 8, 8, 8), 0.1
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1000, full=True).numpy()
    st, info, x = run(ctx, dims, fat, lng, m, b, name, l=l)
    assert st == hisq.HISQ_OK, (hisq.STATUS_NAMES[st], info.true_residual)
    tr = true_res(orc, dims, fat, lng, m, b, x)
    assert tr <= 1e-10
    assert abs(tr - info.true_residual) <= 1e-3 * tr
    assert info.matvecs % (2 * l) == 0


def test_light_mass_int20_vs_half(ctx, orc):
    dims, m = (8, 8, 8, 16), 0.01
    fat, lng = synth.gauge_pair(dims, seed=0)
    b = synth.spinor(dims, 1000, full=True).numpy()
    mv = {}
    for name in ("f64", "int20", "half"):
        st, info, x = run(ctx, dims, fat, lng, m, b, name, l=4)
        assert st == hisq.HISQ_OK, (name, hisq.STATUS_NAMES[st])
        assert true_res(orc, dims, fat, lng, m, b, x) <= 1e-10
        mv[name] = info.matvecs
    assert mv["int20"] <= mv["half"]


def test_graph_matches_direct(ctx):
    dims, m = (4, 4, 8, 8), 0.05
    fat, lng = synth.gauge_pair(dims, seed=3)
    b = synth.spinor(dims, 1002, full=True).numpy()
    _, i1, x1 = run(ctx, dims, fat, lng, m, b, "int20", use_graph=1)
    _, i2, x2 = run(ctx, dims, fat, lng, m, b, "int20", use_graph=0)
    np.testing.assert_array_equal(x1, x2)
    assert i1.matvecs == i2.matvecs


def u3_links(lng, seed):
    """Long links times a random phase per link: unitary, no longer a sign times SU(3)."""
    u = lng[..., 0] + 1j * lng[..., 1]
    g = np.random.Generator(np.random.Philox(key=seed))
    w = u * np.exp(1j * g.uniform(-np.pi, np.pi, u.shape[:-2]))[..., None, None]
    return np.ascontiguousarray(np.stack([w.real, w.imag], axis=-1))


@pytest.mark.parametrize("name,recon", [("f32", 13), ("half", 13), ("int14", 12)])
def test_bicgstab_other_formats(ctx, orc, name, recon):
    """BiCGStab(2) on 2m + D with U(3) long links in 13 reals, and with the 12-byte 14-bit fermion:
    the FP64 true residual recomputed by the oracle meets the target."""
    dims, m = (8, 8, 8, 8), 0.05
    fat, lng = (t.numpy() for t in synth.gauge_pair(dims, seed=0))
    if recon == 13:
        lng = u3_links(lng, 11)
    b = synth.spinor(dims, 1000, full=True).numpy()
    g = hisq.hisq_load_gauge(ctx, dims, torch.as_tensor(fat).cuda(), torch.as_tensor(lng).cuda())
    try:
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.on_device, p.l = m, 1e-10, 1, 2
        p.sloppy = hisq.prec(name, recon)
        bd = torch.as_tensor(b).cuda()
        x = torch.zeros_like(bd)
        st, info = hisq.hisq_bicgstabl(ctx, g, p, bd, x)
    finally:
        hisq.hisq_free_gauge(ctx, g)
    assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
    assert true_res(orc, dims, fat, lng, m, b, x.cpu().numpy()) <= 1e-10


def test_programmatic_launch_same_bits(ctx):
    """BiCGStab's kernel chain launched with programmatic dependent launch (every kernel waits for its
    predecessor's results before touching them) gives the same solution, bit for bit, as kernels
    launched one after another, in graphs and directly."""
    dims, m = (8, 8, 8, 8), 0.05
    fat, lng = (t.numpy() for t in synth.gauge_pair(dims, seed=2))
    b = synth.spinor(dims, 1002, full=True).numpy()
    prev = hisq.hisq_programmatic_launch(0)
    try:
        ref = [run(ctx, dims, fat, lng, m, b, name, l=2, use_graph=g)[2] for name in ("int20", "int30") for g in (0, 1)]
        hisq.hisq_programmatic_launch(1)
        got = [run(ctx, dims, fat, lng, m, b, name, l=2, use_graph=g)[2] for name in ("int20", "int30") for g in (0, 1)]
    finally:
        hisq.hisq_programmatic_launch(prev)
    for a, r in zip(got, ref):
        np.testing.assert_array_equal(a, r)
