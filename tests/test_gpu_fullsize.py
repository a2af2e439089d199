"""The solvers at the 32^3 x 64 lattice of the headline measurement, each
solution checked by the CPU oracle.

At this size every BLAS kernel loops over sites more than once per thread
(grids are capped at a few blocks per SM), the reductions run over thousands
of blocks, and the solves take thousands of iterations with many reliable
updates: the paths a small lattice never reaches.  For each solve the FP64
true residual of the returned x is recomputed by the oracle (its own FP64
stencil, no code shared with the library) and must meet the requested target
(Sec. 3.1 for CG, Sec. 3.2 and Table 3 for the 12-shift solve, Sec. 6.1 and
Table 2 for BiCGStab(4)).

Inputs: the synthetic 32^3 x 64 links (near-identity SU(3), eps = 0.3, fat
x 0.8, staggered phases) and Gaussian sources, as in the benchmark.
"""
import numpy as np
import pytest
import torch

from paper_2302_09224_gb300 import hisq, synth

pytestmark = pytest.mark.gpu

DIMS = (32, 32, 32, 64)


@pytest.fixture(scope="module")
def env():
    ctx = hisq.hisq_create(0)
    fat, lng = synth.gauge_pair(DIMS, seed=0, device="cuda")
    g = hisq.hisq_load_gauge(ctx, DIMS, fat, lng)
    host = (fat.cpu().numpy(), lng.cpu().numpy())
    del fat, lng
    torch.cuda.empty_cache()
    yield ctx, g, host
    hisq.hisq_free_gauge(ctx, g)
    hisq.hisq_destroy(ctx)


def rel_res(r, b):
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def test_mixed_cg_int20(env, orc):
    ctx, g, (fat, lng) = env
    m, tol = 0.01, 1e-10
    b = synth.spinor(DIMS, synth.rhs_seed(0))
    p = hisq.hisq_default_params()
    p.mass, p.tol, p.on_device = m, tol, 1
    p.sloppy = hisq.prec("int20", 12)
    x = torch.zeros_like(b).cuda()
    st, info = hisq.hisq_cg(ctx, g, p, b.cuda(), x)
    assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
    bn = b.numpy()
    tr = rel_res(bn - orc.mee(DIMS, fat, lng, m, x.cpu().numpy()), bn)
    assert tr <= tol, tr
    # the library's own FP64 true residual agrees with the oracle's
    assert abs(info.true_residual - tr) <= 0.05 * tr + 1e-13
    assert info.reliable_updates >= 2 and info.iters > 500


def test_multishift_12_shifts_int20(env, orc):
    ctx, g, (fat, lng) = env
    m = 0.005
    sig = synth.shifts_logspaced(12, 1e-4, 1.0)
    tols = synth.shift_tolerances(12, 1e-10, 1e-7)
    b = synth.spinor(DIMS, synth.rhs_seed(1))
    p = hisq.hisq_default_params()
    p.mass, p.on_device = m, 1
    p.sloppy = hisq.prec("int20", 12)
    p.refine = hisq.prec("int20", 12)
    xs = [torch.zeros_like(b).cuda() for _ in sig]
    st, info = hisq.hisq_multishift_cg(ctx, g, p, sig, tols, b.cuda(), xs)
    assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
    bn = b.numpy()
    for i, (s, t) in enumerate(zip(sig, tols)):
        tr = rel_res(bn - orc.mee(DIMS, fat, lng, m, xs[i].cpu().numpy(), sigma=s), bn)
        assert tr <= t, (i, s, tr, t)
        assert abs(info.shift_resid[i] - tr) <= 0.05 * tr + 1e-13, (i, info.shift_resid[i], tr)


def test_bicgstab4_int20(env, orc):
    ctx, g, (fat, lng) = env
    m, tol = 0.01, 1e-10
    b = synth.spinor(DIMS, synth.rhs_seed(2), full=True)
    p = hisq.hisq_default_params()
    p.mass, p.tol, p.on_device, p.l = m, tol, 1, 4
    p.sloppy = hisq.prec("int20", 12)
    x = torch.zeros_like(b).cuda()
    st, info = hisq.hisq_bicgstabl(ctx, g, p, b.cuda(), x)
    assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
    bn = b.numpy()
    tr = rel_res(bn - orc.mfull(DIMS, fat, lng, m, x.cpu().numpy()), bn)
    assert tr <= tol, tr
    assert abs(info.true_residual - tr) <= 0.05 * tr + 1e-13
