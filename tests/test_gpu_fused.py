"""GPU: the fused M_ee pass (D_oe and D_eo swept over t-slices in one
persistent kernel) against the two separate stencil passes, inside the CG
solver: for every FP32-compute storage triplet and both long-link storages,
on lattices with Lt below and above the seven-slice reach of the three-hop
term and with ragged last chunks, the fused solve meets the oracle-recomputed
FP64 true residual, agrees with the two-pass solve within the tolerance the
iteration allows, and reports no exhausted wait."""
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


def solve(ctx, dims, m, name, recon, fused, anti=False, tol=1e-10, maxiter=100000):
    fat, lng = synth.gauge_pair(dims, seed=0, antiperiodic_t=anti)
    g = hisq.hisq_load_gauge(ctx, dims, fat.cuda(), lng.cuda(), flags=1 if anti else 0)
    prev = hisq.hisq_mee_fused(1 if fused else 0)
    try:
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.on_device, p.maxiter = m, tol, 1, maxiter
        p.sloppy = hisq.prec(name, recon)
        b = synth.spinor(dims, synth.rhs_seed(0)).cuda()
        x = torch.zeros_like(b)
        st, info = hisq.hisq_cg(ctx, g, p, b, x)
        return st, info, b.cpu().numpy(), x.cpu().numpy(), fat.numpy(), lng.numpy()
    finally:
        hisq.hisq_mee_fused(prev)
        hisq.hisq_free_gauge(ctx, g)


@pytest.mark.parametrize("dims,anti", [((4, 4, 4, 4), False), ((6, 4, 4, 6), True), ((4, 6, 4, 8), True),
                                        ((8, 8, 8, 16), False), ((6, 6, 4, 10), True)])
@pytest.mark.parametrize("name,recon", [("int20", 12), ("int20", 18), ("half", 12), ("f32", 18), ("int30f32", 12)])
def test_fused_matches_two_pass(ctx, orc, dims, anti, name, recon):
    m = 0.05
    st1, i1, b, x1, fat, lng = solve(ctx, dims, m, name, recon, True, anti)
    assert st1 == hisq.HISQ_OK, hisq.STATUS_NAMES[st1]
    r = b - orc.mee(dims, fat, lng, m, x1)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    st0, i0, _, x0, _, _ = solve(ctx, dims, m, name, recon, False, anti)
    assert st0 == hisq.HISQ_OK
    d = np.linalg.norm(x1 - x0) / np.linalg.norm(x0)
    assert d <= 1e-7  # both solutions meet 1e-10 on an operator with condition number < 1e3
    assert abs(i1.iters - i0.iters) <= max(3, i0.iters // 20)


def test_fused_switch(ctx):
    prev = hisq.hisq_mee_fused(1)
    assert hisq.hisq_mee_fused(prev) == 1
    assert hisq.hisq_mee_fused(5) == -2


def test_exhausted_wait_returns_ecuda_and_context_recovers(ctx, orc):
    """The fused pass's waits are bounded: with every wait's target made
    unreachable (a count no block ever reaches) and a short poll limit, each
    wait gives up, the kernel flags the error and finishes, and the solver
    returns ECUDA instead of hanging; with normal waits restored the same
    context solves the system."""
    dims, m = (8, 8, 8, 16), 0.05
    hisq.hisq_mee_fused_wait_test(4, True)
    try:
        with pytest.raises(hisq.HisqError, match="ECUDA"):
            solve(ctx, dims, m, "int20", 12, True, maxiter=64)
    finally:
        hisq.hisq_mee_fused_wait_test(0, False)
    st, info, b, x, fat, lng = solve(ctx, dims, m, "int20", 12, True)
    assert st == hisq.HISQ_OK
    r = b - orc.mee(dims, fat, lng, m, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
