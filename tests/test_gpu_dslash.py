"""GPU stencil against the FP64 oracle, per precision triplet (Sec. 4, Sec. 5.2).

For every triplet the C-ABI ``hisq_dslash`` (input rounded into the spinor
format, links in the gauge format, arithmetic in the compute precision,
output repacked) is compared with

* the exact FP64 stencil (the oracle's O3), relative L2 within the stated
  per-format bound, and
* the oracle's format emulation (fields rounded exactly as stored, then the
  FP64 stencil): the remaining difference is compute rounding plus the
  rounding of the stored output, bounded per format,

on lattices that exercise a ragged last block, the 2^4 and 4^4 aliasing of the
three-hop term, non-cubic extents and antiperiodic time.  The orderings the
paper reports for the deviation (Sec. 5.2: 30-bit with FP64 compute about two
orders below FP32; 20-bit only modestly better than half) are checked too.
"""
import numpy as np
import pytest
import torch

from paper_2302_09224_gb300 import hisq, synth

pytestmark = pytest.mark.gpu

# relative L2 bounds against the exact FP64 stencil
BOUND_EXACT = {"f64": 1e-12, "f32": 1e-6, "half": 1e-3, "int20": 3e-4, "int30": 1e-8, "int30f32": 2e-6,
               "int14": 1e-3, "int20se": 3e-4}
# relative L2 bounds against the format emulation (compute + output rounding)
# (the output is stored in the spinor format: for half and int14 its rounding dominates)
BOUND_EMUL = {"f64": 1e-13, "f32": 1e-6, "half": 5e-5, "int20": 3e-6, "int30": 3e-9, "int30f32": 1e-6,
              "int14": 2e-4, "int20se": 3e-6}
SPINOR = {"f64": "f64", "f32": "f32", "half": "half", "int20": "int20", "int30": "int30", "int30f32": "int30",
          "int14": "int14", "int20se": "int20"}
GAUGE = {"f64": "f64", "f32": "f32", "half": "fix16", "int20": "fix16", "int30": "fix32", "int30f32": "fix32",
         "int14": "fix16", "int20se": "se15"}
COMPUTE_F32 = {"f64": False, "f32": True, "half": True, "int20": True, "int30": False, "int30f32": True,
               "int14": True, "int20se": True}


@pytest.fixture(scope="module")
def ctx():
    c = hisq.hisq_create(0)
    yield c
    hisq.hisq_destroy(c)


_cache = {}


def lattice(dims, anti):
    key = (dims, anti)
    if key not in _cache:
        fat, lng = synth.gauge_pair(dims, seed=0, antiperiodic_t=anti)
        _cache[key] = (fat.numpy(), lng.numpy())
    return _cache[key]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def run_gpu(ctx, dims, anti, name, recon, parity, a, on_device=True):
    fat, lng = lattice(dims, anti)
    flags = hisq.HISQ_GAUGE_ANTIPERIODIC_T if anti else 0
    g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda(), flags)
    try:
        full = parity == 2
        x = synth.spinor(dims, 1000, full=full).numpy()
        y = synth.spinor(dims, 1001, full=full).numpy()
        if on_device:
            xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
            out = torch.empty_like(xd)
            hisq.hisq_dslash(ctx, g, hisq.prec(name, recon), parity, a, yd if a else None, xd, out, True)
            torch.cuda.synchronize()
            out = out.cpu().numpy()
        else:
            out = np.empty_like(x)
            hisq.hisq_dslash(ctx, g, hisq.prec(name, recon), parity, a, y if a else None, x, out, False)
    finally:
        hisq.hisq_free_gauge(ctx, g)
    return x, y, out


def oracle_apply(orc, dims, fat, lng, parity, a, x, y):
    if parity == 2:
        d = np.stack([orc.dslash(dims, fat, lng, 0, x[1]), orc.dslash(dims, fat, lng, 1, x[0])])
    else:
        d = orc.dslash(dims, fat, lng, parity, x)
    return a * y - d if a else d


CASES = [
    ((4, 4, 4, 4), False, 0, 0.0),
    ((6, 4, 4, 10), False, 1, 0.0),     # Vh = 480: ragged last block
    ((4, 6, 8, 10), True, 2, 0.0),      # non-cubic, antiperiodic, full lattice
    ((2, 2, 2, 2), False, 1, 0.3),      # every hop aliases
    ((8, 8, 8, 8), False, 0, 0.7),      # several blocks, xpay
]


@pytest.mark.parametrize("name", list(BOUND_EXACT))
@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("dims,anti,parity,a", CASES)
def test_dslash_parity(ctx, orc, name, recon, dims, anti, parity, a):
    fat, lng = lattice(dims, anti)
    x, y, out = run_gpu(ctx, dims, anti, name, recon, parity, a)
    exact = oracle_apply(orc, dims, fat, lng, parity, a, x, y)
    err = rel(out, exact)
    assert err <= BOUND_EXACT[name], (name, recon, err)
    # format emulation: the fields exactly as the kernel sees them
    sf = SPINOR[name]
    c32 = COMPUTE_F32[name]
    fe = orc.gauge_emulate(dims, fat, GAUGE[name], 18, long_link=False, antiperiodic_t=anti, compute_f32=c32)
    le = orc.gauge_emulate(dims, lng, GAUGE[name], recon, long_link=True, antiperiodic_t=anti, compute_f32=c32)
    xe = orc.spinor_emulate(x, sf).reshape(x.shape)
    ye = orc.spinor_emulate(y, sf).reshape(y.shape)
    emul = oracle_apply(orc, dims, fe, le, parity, a, xe, ye)
    assert rel(out, emul) <= BOUND_EMUL[name], (name, recon, rel(out, emul))


def test_host_pointers_match_device(ctx):
    dims = (4, 4, 4, 8)
    _, _, o1 = run_gpu(ctx, dims, False, "int20", 12, 0, 0.5, on_device=True)
    _, _, o2 = run_gpu(ctx, dims, False, "int20", 12, 0, 0.5, on_device=False)
    np.testing.assert_array_equal(o1, o2)


def test_deviation_orderings(ctx, orc):
    """Sec. 5.2: 30-bit + FP64 ~100x below FP32; 30-bit + FP32 ~ FP32; 20-bit < half."""
    dims = (8, 8, 8, 8)
    fat, lng = lattice(dims, False)
    err = {}
    for name in ("f32", "half", "int20", "int30", "int30f32"):
        x, y, out = run_gpu(ctx, dims, False, name, 12, 0, 0.0)
        err[name] = rel(out, orc.dslash(dims, fat, lng, 0, x))
    assert err["int30"] * 30 < err["f32"]
    assert 0.2 < err["int30f32"] / err["f32"] < 5
    assert err["int20"] < err["half"]


def test_r12_refused_for_fat_and_nonunitary(ctx):
    dims = (4, 4, 4, 4)
    fat, lng = lattice(dims, False)
    bad = lng.copy()
    bad[0, 0, 0, 0, 0, 2, 2, 0] += 0.5   # breaks unitarity of one long link
    g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(bad).cuda())
    try:
        x = synth.spinor(dims, 1).cuda()
        out = torch.empty_like(x)
        with pytest.raises(hisq.HisqError, match="EINVAL"):
            hisq.hisq_dslash(ctx, g, hisq.prec("half", 12), 0, 0.0, None, x, out, True)
        hisq.hisq_dslash(ctx, g, hisq.prec("half", 18), 0, 0.0, None, x, out, True)
        p = hisq.prec("half", 18)
        p.fat_recon = 12
        with pytest.raises(hisq.HisqError, match="EINVAL"):
            hisq.hisq_dslash(ctx, g, p, 0, 0.0, None, x, out, True)
    finally:
        hisq.hisq_free_gauge(ctx, g)


def test_invalid_inputs(ctx):
    dims = (4, 4, 4, 4)
    fat, lng = lattice(dims, False)
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        hisq.hisq_load_gauge(ctx, (4, 4, 3, 4), torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda())
    nan = fat.copy()
    nan[1, 1, 1, 1, 1, 0, 0, 1] = np.nan
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(nan).cuda(), torch.from_numpy(lng).cuda())
    g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda())
    try:
        x = synth.spinor(dims, 1).cuda()
        x[3, 1, 0] = float("inf")
        out = torch.empty_like(x)
        with pytest.raises(hisq.HisqError, match="non-finite"):
            hisq.hisq_dslash(ctx, g, hisq.prec("int20"), 0, 0.0, None, x, out, True)
        bad = hisq.prec("int20")
        bad.compute = hisq.HISQ_COMPUTE_F64
        with pytest.raises(hisq.HisqError, match="unsupported"):
            hisq.hisq_dslash(ctx, g, bad, 0, 0.0, None, x, out, True)
    finally:
        hisq.hisq_free_gauge(ctx, g)


@pytest.mark.parametrize("name", ["f64", "half", "int20"])
def test_full_size_sampled(ctx, orc, name):
    """32^3 x 64 (the benchmark lattice), whole-lattice launch, sampled sites vs the oracle."""
    dims = (32, 32, 32, 64)
    fat, lng = synth.gauge_pair(dims, seed=0, device="cuda")
    g = hisq.hisq_load_gauge(ctx, dims, fat, lng)
    try:
        x = synth.spinor(dims, 1000, device="cuda")
        out = torch.empty_like(x)
        hisq.hisq_dslash(ctx, g, hisq.prec(name, 12), 1, 0.0, None, x, out, True)
        torch.cuda.synchronize()
        vh = x.shape[0]
        cbs = np.unique(np.concatenate([np.arange(64), vh - 1 - np.arange(64),
                                        np.random.Generator(np.random.Philox(key=9)).integers(0, vh, 2000)]))
        ref = orc.dslash_sites(dims, fat.cpu(), lng.cpu(), 1, x.cpu(), cbs)
        got = out.cpu().numpy()[cbs]
        assert rel(got, ref) <= BOUND_EXACT[name]
    finally:
        hisq.hisq_free_gauge(ctx, g)
        del fat, lng
        torch.cuda.empty_cache()


@pytest.mark.parametrize("cfg", range(5))
@pytest.mark.parametrize("name", ["int20", "half", "f32", "f64"])
def test_every_launch_shape(ctx, orc, cfg, name):
    """Each stencil launch shape the tuner may pick gives the same parity (ragged and aliased lattices)."""
    prev = hisq.hisq_stencil_config(cfg)
    try:
        for dims, anti, parity, a in [((6, 4, 4, 10), True, 2, 0.4), ((2, 2, 2, 2), False, 1, 0.0)]:
            fat, lng = lattice(dims, anti)
            x, y, out = run_gpu(ctx, dims, anti, name, 12, parity, a)
            exact = oracle_apply(orc, dims, fat, lng, parity, a, x, y)
            assert rel(out, exact) <= BOUND_EXACT[name], (cfg, name, dims)
    finally:
        hisq.hisq_stencil_config(prev)


def test_launch_shape_controls(ctx):
    """Forced shapes per pass are reported by the in-use query; invalid values are refused."""
    dims = (4, 4, 4, 8)
    fat, lng = lattice(dims, False)
    g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda())
    p = hisq.prec("int20", 12)
    prev = hisq.hisq_stencil_config(2)
    prev_r = hisq.hisq_stencil_config_reduce(3)
    try:
        assert hisq.hisq_stencil_config_in_use(g, p, False) == 2
        assert hisq.hisq_stencil_config_in_use(g, p, True) == 3
        hisq.hisq_stencil_config_reduce(-1)  # the reducing pass follows the plain one again
        assert hisq.hisq_stencil_config_in_use(g, p, True) == 2
        assert hisq.hisq_stencil_config(7) == -2 and hisq.hisq_stencil_config_reduce(-5) == -2
    finally:
        hisq.hisq_stencil_config(prev)
        hisq.hisq_stencil_config_reduce(prev_r)
        hisq.hisq_free_gauge(ctx, g)


# largest input magnitude each triplet stores without loss of range: FP32 max
# for the FP32-compute triplets (and the FP32-pair arithmetic of 30-bit/FP64),
# FP64 max for plain FP64
HUGE = {"f64": 1.7e308, "f32": 3.3e38, "half": 3.3e38, "int20": 3.3e38, "int30": 3.3e38, "int30f32": 3.3e38,
        "int14": 3.3e38, "int20se": 3.3e38}


@pytest.mark.parametrize("name", list(BOUND_EXACT))
def test_unstorable_output_is_reported(ctx, name):
    """Finite inputs whose stencil result overflows the compute precision:
    the input packs, the output cannot be stored, and the call returns ERANGE
    instead of a silently zeroed site; the next call on the context works."""
    dims = (4, 4, 4, 8)
    fat, lng = lattice(dims, False)
    g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda())
    try:
        p = hisq.prec(name, 12)
        x = synth.spinor(dims, 1).cuda()
        big = x / x.abs().max() * HUGE[name]
        out = torch.empty_like(x)
        with pytest.raises(hisq.HisqError, match="ERANGE"):
            hisq.hisq_dslash(ctx, g, p, 0, 0.0, None, big, out, True)
        ref = torch.empty_like(x)
        hisq.hisq_dslash(ctx, g, p, 0, 0.0, None, x, ref, True)
        hisq.hisq_dslash(ctx, g, p, 0, 0.0, None, x, out, True)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all() and torch.equal(out, ref)
    finally:
        hisq.hisq_free_gauge(ctx, g)


@pytest.mark.parametrize("name", ["f32", "half", "int20"])
@pytest.mark.parametrize("dims,anti,parity,a", CASES)
def test_dslash_r13_parity(ctx, orc, name, dims, anti, parity, a):
    """13-real long links (rows 0, 1 and the phase of det U; row 2 rebuilt as
    e^{i pi t} conj(row0 x row1) in registers) against the exact stencil and
    the oracle's emulation of the same storage, within the 12-real bounds."""
    fat, lng = lattice(dims, anti)
    x, y, out = run_gpu(ctx, dims, anti, name, 13, parity, a)
    exact = oracle_apply(orc, dims, fat, lng, parity, a, x, y)
    assert rel(out, exact) <= BOUND_EXACT[name], (name, rel(out, exact))
    fe = orc.gauge_emulate(dims, fat, GAUGE[name], 18, long_link=False, antiperiodic_t=anti)
    le = orc.gauge_emulate(dims, lng, GAUGE[name], 13, long_link=True, antiperiodic_t=anti)
    xe = orc.spinor_emulate(x, SPINOR[name]).reshape(x.shape)
    ye = orc.spinor_emulate(y, SPINOR[name]).reshape(y.shape)
    emul = oracle_apply(orc, dims, fe, le, parity, a, xe, ye)
    assert rel(out, emul) <= BOUND_EMUL[name], (name, rel(out, emul))


def u3_long_links(lng, seed):
    """Long links times a random phase per link: unitary, no longer a sign times SU(3)."""
    u = lng[..., 0] + 1j * lng[..., 1]
    g = np.random.Generator(np.random.Philox(key=seed))
    ph = np.exp(1j * g.uniform(-np.pi, np.pi, u.shape[:-2]))[..., None, None]
    w = u * ph
    return np.ascontiguousarray(np.stack([w.real, w.imag], axis=-1))


@pytest.mark.parametrize("name", ["f32", "int20"])
def test_r13_u3_links_and_refusals(ctx, orc, name):
    """U(3) long links (a random phase on each): 12-real compression is refused,
    13 reals reproduce them; a 13-real request on FP64 or 30-bit triplets, or
    for a batched solve, is refused; a CG solve with 13-real links meets the
    oracle's true residual."""
    dims = (4, 6, 4, 8)
    fat, lng0 = lattice(dims, False)
    lng = u3_long_links(lng0, 17)
    g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda())
    try:
        x = synth.spinor(dims, 1000)
        out = torch.empty_like(x).cuda()
        with pytest.raises(hisq.HisqError, match="12-real"):
            hisq.hisq_dslash(ctx, g, hisq.prec(name, 12), 0, 0.0, None, x.cuda(), out, True)
        hisq.hisq_dslash(ctx, g, hisq.prec(name, 13), 0, 0.0, None, x.cuda(), out, True)
        torch.cuda.synchronize()
        exact = orc.dslash(dims, fat, lng, 0, x.numpy())
        assert rel(out.cpu().numpy(), exact) <= BOUND_EXACT[name]
        for bad in ("f64", "int30"):
            with pytest.raises(hisq.HisqError, match="EINVAL"):
                hisq.hisq_dslash(ctx, g, hisq.prec(bad, 13), 0, 0.0, None, x.cuda(), out, True)
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.on_device = 0.05, 1e-10, 1
        p.sloppy = hisq.prec(name, 13)
        b = x.cuda()
        sol = torch.zeros_like(b)
        st, info = hisq.hisq_cg(ctx, g, p, b, sol)
        assert st == hisq.HISQ_OK
        r = x.numpy() - orc.mee(dims, fat, lng, 0.05, sol.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(x.numpy()) <= 1e-10
        p.nrhs = 2
        b2 = torch.stack([b, b]).contiguous()
        with pytest.raises(hisq.HisqError, match="EINVAL"):
            hisq.hisq_cg(ctx, g, p, b2, torch.zeros_like(b2))
    finally:
        hisq.hisq_free_gauge(ctx, g)


def rotated_long_links(lng):
    """Long links times one fixed SU(3) matrix on the left whose elements all have |.|^2 = 1/3: still a
    sign times SU(3), but far from diagonal, where the 8-real rebuild is well conditioned."""
    w = np.exp(2j * np.pi / 3)
    f = np.array([[1, 1, 1], [1, w, w * w], [1, w * w, w]]) / np.sqrt(3)
    f = f / np.linalg.det(f) ** (1.0 / 3.0)
    u = lng[..., 0] + 1j * lng[..., 1]
    r = np.einsum("ij,...jk->...ik", f, u)
    return np.ascontiguousarray(np.stack([r.real, r.imag], axis=-1))


def run_fields(ctx, dims, anti, fat, lng, name, recon, parity, a):
    flags = hisq.HISQ_GAUGE_ANTIPERIODIC_T if anti else 0
    g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda(), flags)
    try:
        full = parity == 2
        x = synth.spinor(dims, 1000, full=full).numpy()
        y = synth.spinor(dims, 1001, full=full).numpy()
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        out = torch.empty_like(xd)
        hisq.hisq_dslash(ctx, g, hisq.prec(name, recon), parity, a, yd if a else None, xd, out, True)
        torch.cuda.synchronize()
        return x, y, out.cpu().numpy()
    finally:
        hisq.hisq_free_gauge(ctx, g)


BOUND_EXACT_R8 = {"f32": 2e-6, "half": 1e-3, "int20": 4e-4}
BOUND_EMUL_R8 = {"f32": 1e-5, "half": 6e-5, "int20": 1e-5}


@pytest.mark.parametrize("name", ["f32", "half", "int20"])
@pytest.mark.parametrize("rotate", [True, False])
@pytest.mark.parametrize("dims,anti,parity,a", CASES)
def test_dslash_r8_parity(ctx, orc, name, rotate, dims, anti, parity, a):
    """8-real long links (Sec. 1: 18 -> 8; V = sign U parametrised by arg V00, arg V20, V01, V02, V10 and
    rebuilt in registers from unitarity and det V = 1), on the synthetic long links (near the identity) and
    on the same links rotated far from it: against the oracle's emulation of the same storage within the
    compute rounding, and against the exact stencil."""
    fat, lng = lattice(dims, anti)
    if rotate:
        lng = rotated_long_links(lng)
    x, y, out = run_fields(ctx, dims, anti, fat, lng, name, 8, parity, a)
    exact = oracle_apply(orc, dims, fat, lng, parity, a, x, y)
    assert rel(out, exact) <= BOUND_EXACT_R8[name], (name, rel(out, exact))
    fe = orc.gauge_emulate(dims, fat, GAUGE[name], 18, long_link=False, antiperiodic_t=anti)
    le = orc.gauge_emulate(dims, lng, GAUGE[name], 8, long_link=True, antiperiodic_t=anti)
    xe = orc.spinor_emulate(x, SPINOR[name]).reshape(x.shape)
    ye = orc.spinor_emulate(y, SPINOR[name]).reshape(y.shape)
    emul = oracle_apply(orc, dims, fe, le, parity, a, xe, ye)
    assert rel(out, emul) <= BOUND_EMUL_R8[name], (name, rel(out, emul))


def test_r8_refusals_and_solve(ctx, orc):
    """8 reals are refused for U(3) long links and for the free field (V00 = 1: N = 0, no rebuild), and on
    FP64 or 30-bit triplets; a CG solve with 8-real long links meets the oracle's true residual."""
    dims = (4, 6, 4, 8)
    fat, lng = lattice(dims, False)
    x = synth.spinor(dims, 1000)
    free = synth.gauge_field(dims, "long", seed=0, eps=0.0).numpy()
    for bad in (u3_long_links(lng, 5), free):
        g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(bad).cuda())
        try:
            out = torch.empty_like(x).cuda()
            with pytest.raises(hisq.HisqError, match="8-real"):
                hisq.hisq_dslash(ctx, g, hisq.prec("int20", 8), 0, 0.0, None, x.cuda(), out, True)
        finally:
            hisq.hisq_free_gauge(ctx, g)
    g = hisq.hisq_load_gauge(ctx, dims, torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda())
    try:
        out = torch.empty_like(x).cuda()
        for bad in ("f64", "int30"):
            with pytest.raises(hisq.HisqError, match="EINVAL"):
                hisq.hisq_dslash(ctx, g, hisq.prec(bad, 8), 0, 0.0, None, x.cuda(), out, True)
        p = hisq.hisq_default_params()
        p.mass, p.tol, p.on_device = 0.05, 1e-10, 1
        p.sloppy = hisq.prec("int20", 8)
        b = x.cuda()
        sol = torch.zeros_like(b)
        st, info = hisq.hisq_cg(ctx, g, p, b, sol)
        assert st == hisq.HISQ_OK
        r = x.numpy() - orc.mee(dims, fat, lng, 0.05, sol.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(x.numpy()) <= 1e-10
    finally:
        hisq.hisq_free_gauge(ctx, g)
