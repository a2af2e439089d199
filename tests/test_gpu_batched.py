"""GPU batched (multi right-hand side) CG: one stencil launch per tile of
right-hand sides shares each link load (Sec. 1, block solvers).

* every right-hand side's FP64 true residual, recomputed by the CPU oracle,
  meets the target, for each batched sloppy format and tile size;
* a right-hand side's iterates do not depend on which others share its batch:
  the same system solved in a batch of four and in a batch of two (same tile)
  gives bitwise identical solutions; against the single-RHS solver (another
  stencil kernel, so other rounding) both solutions meet the tolerance, so
  their difference is within twice the tolerance in the residual norm
  |M_ee (x_a - x_b)| / |b|;
* nor on its tile or the kernel: tiles of 1, 2 and 4 with both kernels (and
  1, 4 and 16 right-hand sides per tile) give bitwise identical solutions;
* the batched stencil equals the single-RHS stencil through the oracle check of
  the solutions; bad tile sizes give EINVAL.
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


_fields = {}


def lattice(dims):
    if dims not in _fields:
        _fields[dims] = tuple(f.numpy() for f in synth.gauge_pair(dims, seed=0))
    return _fields[dims]


def solve(ctx, dims, m, bs, name="int20", tile=0, tol=1e-10, **kw):
    fat, lng = lattice(dims)
    g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda())
    try:
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.on_device = m, tol, 1
        p.sloppy = hisq.prec(name, 12)
        p.nrhs = len(bs)
        p.rhs_tile = tile
        for k, v in kw.items():
            setattr(p, k, v)
        b = torch.from_numpy(np.stack(bs)).cuda().contiguous()
        x = torch.zeros_like(b)
        st, info = hisq.hisq_cg(ctx, g, p, b, x)
        return st, info, x.cpu().numpy()
    finally:
        hisq.hisq_free_gauge(ctx, g)


def true_res(orc, dims, m, b, x):
    fat, lng = lattice(dims)
    r = b - orc.mee(dims, fat, lng, m, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


@pytest.mark.parametrize("name,tile", [("int20", 0), ("int20", 1), ("half", 2), ("f32", 4)])
def test_batched_true_residuals(ctx, orc, name, tile):
    dims, m = (8, 8, 8, 8), 0.05
    bs = [synth.spinor(dims, synth.rhs_seed(k)).numpy() for k in range(4)]
    st, info, xs = solve(ctx, dims, m, bs, name, tile)
    assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
    for b, x in zip(bs, xs):
        assert true_res(orc, dims, m, b, x) <= 1e-10
    assert info.true_residual <= 1e-10


def test_same_alone_and_in_the_mix(ctx, orc):
    dims, m, tol = (8, 8, 8, 16), 0.02, 1e-10
    bs = [synth.spinor(dims, synth.rhs_seed(k)).numpy() for k in range(4)]
    _, _, x4 = solve(ctx, dims, m, bs, "int20", tile=2, tol=tol)
    _, _, x2 = solve(ctx, dims, m, bs[:2], "int20", tile=2, tol=tol)
    np.testing.assert_array_equal(x4[:2], x2)
    _, _, x1 = solve(ctx, dims, m, bs[:1], "int20", tol=tol)  # the single-RHS solver
    # x is fixed only up to the tolerance: both meet it, so in the residual
    # norm the two solutions differ by at most 2 tol (triangle inequality)
    fat, lng = lattice(dims)
    d = np.linalg.norm(orc.mee(dims, fat, lng, m, x4[0] - x1[0])) / np.linalg.norm(bs[0])
    assert d <= 2 * tol, d


def test_iterates_independent_of_tile(ctx):
    """A right-hand side's iterates do not depend on its tile or on the
    kernel: pairs of right-hand sides on the packed FP32 pipe and a tile of
    one run the same operations per lane, both kernels share that arithmetic,
    and every tile's partial sums are reduced in the same order, so the
    solutions are bitwise identical for every tile size and kernel."""
    dims, m = (8, 8, 8, 16), 0.02
    bs = [synth.spinor(dims, synth.rhs_seed(k)).numpy() for k in range(4)]
    ref = None
    for tile in (1, 2, 4):
        for kernel in (1, 2):
            st, _, x = solve(ctx, dims, m, bs, "int20", tile=tile, rhs_kernel=kernel)
            assert st == hisq.HISQ_OK
            if ref is None:
                ref = x
            else:
                np.testing.assert_array_equal(x, ref)
    dims, m = (4, 4, 8, 8), 0.1
    bs = [synth.spinor(dims, synth.rhs_seed(k)).numpy() for k in range(16)]
    sols = [solve(ctx, dims, m, bs, "half", tile=t, rhs_kernel=2)[2] for t in (1, 4, 16)]
    np.testing.assert_array_equal(sols[1], sols[0])
    np.testing.assert_array_equal(sols[2], sols[0])


def test_sixteen_rhs_and_invalid(ctx, orc):
    dims, m = (4, 4, 8, 8), 0.1
    bs = [synth.spinor(dims, synth.rhs_seed(k)).numpy() for k in range(16)]
    st, info, xs = solve(ctx, dims, m, bs, "half", tile=16)
    assert st == hisq.HISQ_OK
    for b, x in zip(bs, xs):
        assert true_res(orc, dims, m, b, x) <= 1e-10
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        solve(ctx, dims, m, bs[:3], "half", tile=2)
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        solve(ctx, dims, m, bs[:2], "int30", tile=1)


@pytest.mark.parametrize("name", ["int20", "half"])
@pytest.mark.parametrize("tile", [1, 2, 4, 8, 16])
def test_register_and_staged_kernels(ctx, orc, name, tile):
    """Both batched stencil kernels (registers; staged neighbour loads through
    shared memory) at every tile size: every right-hand side meets the target
    and the two kernels' solutions agree (same arithmetic in the same order).
    The 6x4x4x8 lattice has a ragged last block (384 sites per parity)."""
    dims, m = (6, 4, 4, 8), 0.08
    bs = [synth.spinor(dims, synth.rhs_seed(k)).numpy() for k in range(16)]
    sols = []
    for kernel in (1, 2):
        st, info, xs = solve(ctx, dims, m, bs, name, tile, rhs_kernel=kernel)
        assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
        for b, x in zip(bs, xs):
            assert true_res(orc, dims, m, b, x) <= 1e-10
        sols.append(xs)
    d = max(np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(*sols))
    assert d <= 1e-9


def test_staged_kernel_refuses_other_formats(ctx):
    dims = (4, 4, 4, 8)
    bs = [synth.spinor(dims, synth.rhs_seed(k)).numpy() for k in range(2)]
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        solve(ctx, dims, 0.1, bs, "f32", tile=2, rhs_kernel=2)


def test_adaptive_tile_same_bits(ctx, orc):
    """With the tile left to the library, a batch whose systems stop at very
    different iterations switches to smaller tiles as they finish and launches
    only tiles that still hold an iterating system; every solution is bitwise
    the one of a fixed tile (the per-RHS arithmetic does not depend on the
    tile) and meets the target.  Half of the systems start from a guess close
    to their solution, so they stop after a few iterations."""
    dims, m = (8, 8, 8, 16), 0.03
    fat, lng = lattice(dims)
    bs = [synth.spinor(dims, synth.rhs_seed(k)).numpy() for k in range(8)]
    _, _, x_ref = solve(ctx, dims, m, bs, "int20", tile=4, rhs_kernel=1)
    guess = x_ref.copy()
    guess[1::2] = 0.0                   # odd systems from zero, even ones from near their solution
    guess[0::2] *= 1.0 + 1e-7
    g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda())
    try:
        sols = []
        for tile, kernel in ((0, 0), (4, 1), (2, 2), (8, 1)):
            p = hisq.hisq_default_params()
            p.mass, p.tol, p.on_device, p.use_init_guess = m, 1e-10, 1, 1
            p.sloppy = hisq.prec("int20", 12)
            p.nrhs, p.rhs_tile, p.rhs_kernel = 8, tile, kernel
            b = torch.from_numpy(np.stack(bs)).cuda().contiguous()
            x = torch.from_numpy(guess).cuda().contiguous()
            st, info = hisq.hisq_cg(ctx, g, p, b, x)
            assert st == hisq.HISQ_OK
            sols.append(x.cpu().numpy())
    finally:
        hisq.hisq_free_gauge(ctx, g)
    for s_ in sols[1:]:
        np.testing.assert_array_equal(s_, sols[0])
    for k in range(8):
        assert true_res(orc, dims, m, bs[k], sols[0][k]) <= 1e-10
