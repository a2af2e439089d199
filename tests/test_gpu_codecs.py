"""GPU storage-format codecs against the oracle's codecs, bit for bit.

Every kernel of the library stores and loads fields through the same device
codecs; ``hisq_spinor_pack`` / ``hisq_spinor_unpack`` expose them.  Packed
records must equal the oracle's byte for byte (the planar device layout is
re-assembled into per-site records first), including zeros, ties, extreme
exponents and non-finite inputs, which both sides count and store as zero.
"""
import numpy as np
import pytest
import torch

from paper_2302_09224_gb300 import hisq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = hisq.hisq_create(0)
    yield c
    hisq.hisq_destroy(c)


def sites(n, seed):
    g = np.random.Generator(np.random.Philox(key=seed))
    v = g.standard_normal((n, 6)) * np.exp(g.uniform(-20, 20, size=(n, 1)))
    v[::7, 3] = 0.0
    v[5] = 0.0
    v[6] = [1, 0.5, -0.25, 0, 0, 0]                                   # ties
    v[7] = [1, 5.7220458984375e-06, 9.5367431640625e-06, -5.7220458984375e-06, 0, 0]
    v[8] = [3e-39, -1e-40, 0, 0, 0, 2e-45]                            # below FP32 normal
    v[9] = [3.0e38, -1e38, 0, 1, 0, 0]                                # near FP32 max
    v[10, 2] = np.nan
    v[11, 0] = np.inf
    return v


def device_pack(ctx, fmt, v):
    n = len(v)
    x = torch.from_numpy(np.ascontiguousarray(v)).cuda()
    buf = torch.zeros(hisq.hisq_spinor_bytes(fmt, n), dtype=torch.uint8, device="cuda")
    bad = hisq.hisq_spinor_pack(ctx, fmt, n, x, buf)
    return buf.cpu().numpy(), bad


@pytest.mark.parametrize("n", [1, 37, 4096 + 13])
def test_half_bit_exact(ctx, orc, n):
    v = sites(max(n, 16), n)[:max(n, 16)]
    buf, bad = device_pack(ctx, hisq.HISQ_SPINOR_HALF16, v)
    rec, obad = orc.half_pack(v.astype(np.float32))
    assert bad == obad
    np.testing.assert_array_equal(buf.reshape(-1, 16), rec)


@pytest.mark.parametrize("n", [16, 4096 + 13])
def test_int20_bit_exact(ctx, orc, n):
    v = sites(n, 100 + n)
    buf, bad = device_pack(ctx, hisq.HISQ_SPINOR_INT20, v)
    w, obad = orc.int20_pack(v.astype(np.float32))
    assert bad == obad
    np.testing.assert_array_equal(buf.view(np.uint32).reshape(-1, 4), w)


def int14_words(buf, n):
    """The device's two planes (8 + 4 bytes per site) as per-site records of three words."""
    a = buf[:8 * n].view(np.uint32).reshape(n, 2)
    b = buf[8 * n:12 * n].view(np.uint32).reshape(n, 1)
    return np.concatenate([a, b], axis=1)


@pytest.mark.parametrize("n", [16, 4096 + 13])
def test_int14_bit_exact(ctx, orc, n):
    v = sites(n, 500 + n)
    v[12] = [1.999755859375, 0, 0, 0, 0, -1.999755859375]   # t = 2^-12 exactly, q = rint(4095.5)
    buf, bad = device_pack(ctx, hisq.HISQ_SPINOR_INT14, v)
    w, obad = orc.int14_pack(v.astype(np.float32))
    assert bad == obad >= 2
    np.testing.assert_array_equal(int14_words(buf, n), w)
    # the FP32-input store path, and the decode
    with np.errstate(over="ignore"):
        f = v.astype(np.float32)
    x = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    buf32 = torch.zeros(hisq.hisq_spinor_bytes(hisq.HISQ_SPINOR_INT14, n), dtype=torch.uint8, device="cuda")
    assert hisq.hisq_spinor_pack32(ctx, hisq.HISQ_SPINOR_INT14, n, x, buf32) == obad
    np.testing.assert_array_equal(int14_words(buf32.cpu().numpy(), n), w)
    out = torch.empty((n, 6), dtype=torch.float64, device="cuda")
    hisq.hisq_spinor_unpack(ctx, hisq.HISQ_SPINOR_INT14, 0, n, buf32, out)
    np.testing.assert_array_equal(out.cpu().numpy(), orc.int14_unpack(w).astype(np.float64))


@pytest.mark.parametrize("n", [16, 4096 + 13])
def test_int30_bit_exact(ctx, orc, n):
    v = sites(n, 200 + n)
    v[12] = [1e300, 0, 0, 0, 0, 0]    # beyond the 8-bit exponent: flagged on both sides
    buf, bad = device_pack(ctx, hisq.HISQ_SPINOR_INT30, v)
    w, obad = orc.int30_pack(v)
    assert bad == obad >= 3
    a = buf[:16 * n].view(np.uint32).reshape(n, 4)
    b = buf[16 * n:].view(np.uint32).reshape(n, 2)
    np.testing.assert_array_equal(np.concatenate([a, b], axis=1), w)


@pytest.mark.parametrize("n", [16, 4096 + 13])
def test_fp32_store_path_bit_exact(ctx, orc, n):
    """The FP32-input store (what FP32-compute kernels write) against the
    oracle's FP64 codecs on the same FP32-exact values: 30-bit records are
    derived there without FP64 arithmetic and must still match bit for bit."""
    v = sites(n, 300 + n)
    v[9] = [1e-30, 2e-44, 0, 0, 0, 0]                 # tiny site maximum: exponent clamped to 1
    v[13] = [np.nextafter(np.float32(2), np.float32(0)), 1, 0, 0, 0, 0]   # largest FP32 significand
    with np.errstate(over="ignore"):
        f = v.astype(np.float32)
    x = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    for fmt in (hisq.HISQ_SPINOR_INT30, hisq.HISQ_SPINOR_INT20, hisq.HISQ_SPINOR_HALF16):
        buf = torch.zeros(hisq.hisq_spinor_bytes(fmt, n), dtype=torch.uint8, device="cuda")
        bad = hisq.hisq_spinor_pack32(ctx, fmt, n, x, buf)
        got = buf.cpu().numpy()
        if fmt == hisq.HISQ_SPINOR_INT30:
            w, obad = orc.int30_pack(f.astype(np.float64))
            a = got[:16 * n].view(np.uint32).reshape(n, 4)
            b = got[16 * n:].view(np.uint32).reshape(n, 2)
            np.testing.assert_array_equal(np.concatenate([a, b], axis=1), w)
        elif fmt == hisq.HISQ_SPINOR_INT20:
            w, obad = orc.int20_pack(f)
            np.testing.assert_array_equal(got.view(np.uint32).reshape(-1, 4), w)
        else:
            w, obad = orc.half_pack(f)
            np.testing.assert_array_equal(got.reshape(-1, 16), w)
        assert bad == obad


@pytest.mark.parametrize("n", [16, 4096 + 13])
def test_pair_store_path_bit_exact(ctx, orc, n):
    """The 30-bit store from FP32 pairs (what the FP64-class kernels write,
    without FP64 arithmetic) against the oracle's FP64 codec on the values
    hi + lo: exponents from power-of-two hi with tails of either sign, and
    exact ties after scaling, bit for bit."""
    g = np.random.Generator(np.random.Philox(key=400 + n))
    hi = (g.standard_normal((n, 6)) * np.exp(g.uniform(-30, 30, size=(n, 1)))).astype(np.float32)
    hi[::3, 0] = np.float32(2.0) ** g.integers(-60, 60, size=hi[::3, 0].shape).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (g.uniform(-0.5, 0.5, size=(n, 6)) * ulp * 10.0 ** -g.integers(0, 8, size=(n, 6))).astype(np.float32)
    lo[::5] = (np.sign(g.standard_normal((len(lo[::5]), 6))) * ulp[::5] / 2).astype(np.float32)  # ties
    hi[2] = 0.0
    lo[2] = 0.0
    # power-of-two site maxima with opposite-sign tails above and below 2^(p-29)
    hi[1] = [1.0, 0.25, 0, 0, 0, 0]
    lo[1] = [-2.0 ** -25, 0, 0, 0, 0, 0]
    hi[3] = [0, -2.0, 0, 0, 0.5, 0]
    lo[3] = [0, 2.0 ** -40, 0, 0, 0, 0]
    lo = np.where(np.abs(lo.astype(np.float64)) <= ulp / 2, lo, np.float32(0))
    # keep only tails whose sum with hi is exact in FP64 (the reference below)
    exact = (hi.astype(np.float64) + lo.astype(np.float64)) - hi.astype(np.float64) == lo.astype(np.float64)
    lo = np.where(exact, lo, np.float32(0))
    pairs = np.stack([hi, lo], axis=-1)
    x = torch.from_numpy(np.ascontiguousarray(pairs)).cuda()
    buf = torch.zeros(hisq.hisq_spinor_bytes(hisq.HISQ_SPINOR_INT30, n), dtype=torch.uint8, device="cuda")
    bad = hisq.hisq_spinor_pack_pair_int30(ctx, n, x, buf)
    d = hi.astype(np.float64) + lo.astype(np.float64)  # exact (filtered above)
    w, obad = orc.int30_pack(d)
    got = buf.cpu().numpy()
    a = got[:16 * n].view(np.uint32).reshape(n, 4)
    b = got[16 * n:].view(np.uint32).reshape(n, 2)
    np.testing.assert_array_equal(np.concatenate([a, b], axis=1), w)
    assert bad == obad == 0


def test_f32_f64_layouts(ctx):
    n = 1000
    v = sites(n, 7)[20:]
    n = len(v)
    buf, _ = device_pack(ctx, hisq.HISQ_SPINOR_F32, v)
    f = v.astype(np.float32)
    np.testing.assert_array_equal(buf[:16 * n].view(np.float32).reshape(n, 4), f[:, :4])
    np.testing.assert_array_equal(buf[16 * n:].view(np.float32).reshape(n, 2), f[:, 4:])
    buf, _ = device_pack(ctx, hisq.HISQ_SPINOR_F64, v)
    d = buf.view(np.float64).reshape(3, n, 2)
    np.testing.assert_array_equal(d.transpose(1, 0, 2).reshape(n, 6), v)


@pytest.mark.parametrize("fmt,compute", [("half", 0), ("int20", 0), ("int30", 1), ("int30", 0), ("f32", 0)])
def test_unpack_matches_oracle(ctx, orc, fmt, compute):
    n = 3000
    v = sites(n, 300)
    v = v[np.all(np.isfinite(v), axis=1)]
    v = v[np.abs(v).max(axis=1) < 1e30]
    n = len(v)
    code = hisq.SPINOR_FMT[fmt]
    x = torch.from_numpy(np.ascontiguousarray(v)).cuda()
    buf = torch.zeros(hisq.hisq_spinor_bytes(code, n), dtype=torch.uint8, device="cuda")
    hisq.hisq_spinor_pack(ctx, code, n, x, buf)
    out = torch.empty_like(x)
    hisq.hisq_spinor_unpack(ctx, code, compute, n, buf, out)
    got = out.cpu().numpy()
    if fmt == "half":
        ref = orc.half_unpack(orc.half_pack(v.astype(np.float32))[0]).astype(np.float64)
    elif fmt == "int20":
        ref = orc.int20_unpack(orc.int20_pack(v.astype(np.float32))[0]).astype(np.float64)
    elif fmt == "int30":
        ref = orc.int30_unpack(orc.int30_pack(v)[0])
        if compute == 0:  # FP32 decode: round the integer, scale exactly
            ref = ref.astype(np.float32).astype(np.float64)
    else:
        ref = v.astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(got, ref)
