"""Pins of the oracle's storage formats (CPU only).

* bit patterns derived by hand from the paper's codec rules
  (``tests/golden/*_vectors.txt``: Appendix A, Listing 4 for 20-bit;
  Sec. 2, Listing 1 for 16-bit; our stated reading of Listing 3 for 30-bit;
  the Appendix A rule with scale 2^13-1 for our 12-byte 14-bit width; the
  30-bit rule with scale 2^14-1 per link for the shared-exponent link format);
* round-trip error within the format's epsilon (Sec. 2: 2^-15 relative to the
  site maximum for the two's-complement 16-bit format; Sec. 4: about 2^-19
  for 20-bit and 2^-29 for 30-bit);
* idempotence ``pack(unpack(pack(v))) == pack(v)`` and exact round trip of
  vectors that are already on the format's grid;
* fixed-point gauge and reconstruct-12 round trips on random SU(3) links.
"""
import os

import numpy as np
import pytest

from paper_2302_09224_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, b = line.split("|")
            rows.append(([float(v) for v in a.split()], b.split()))
    return rows


def test_int20_golden(orc):
    for vals, words in _read("int20_vectors.txt"):
        w, bad = orc.int20_pack(np.array([vals], dtype=np.float32))
        assert bad == 0
        assert [int(x, 16) for x in words] == [int(x) for x in w[0]], vals


def test_int30_golden(orc):
    for vals, words in _read("int30_vectors.txt"):
        w, bad = orc.int30_pack(np.array([vals]))
        assert bad == 0
        assert [int(x, 16) for x in words] == [int(x) for x in w[0]], vals


def test_int14_golden(orc):
    for vals, words in _read("int14_vectors.txt"):
        w, bad = orc.int14_pack(np.array([vals], dtype=np.float32))
        assert bad == 0
        assert [int(x, 16) for x in words] == [int(x) for x in w[0]], vals


def test_se15_golden(orc):
    for vals, halves in _read("se15_vectors.txt"):
        h, bad = orc.se15_pack(np.array([vals]), len(vals))
        assert bad == 0
        assert [int(x, 16) for x in halves] == [int(x) for x in h[0]], vals


@pytest.mark.parametrize("nr", [18, 12])
def test_se15_roundtrip_bound_exact_grid_and_nonfinite(orc, nr):
    g = np.random.Generator(np.random.Philox(key=11))
    # links of very different magnitudes (smeared fat links have no common scale)
    v = g.standard_normal((5000, nr)) * np.exp(g.uniform(-20, 20, size=(5000, 1)))
    h, bad = orc.se15_pack(v, nr)
    assert bad == 0
    u = orc.se15_unpack(h, nr)
    mx = np.abs(v).max(axis=1, keepdims=True)
    # step 2^(E-127) <= 2 mx / (2^14 - 1): every real within half a step
    assert np.all(np.abs(u - v) <= mx / 16383.0 * (1 + 1e-12))
    # per-link relative precision, whatever the link's magnitude
    assert np.all(np.abs(u - v) <= mx * 2.0 ** -14)
    # values on a link's grid come back exactly; zero links stay zero
    q = g.integers(-16000, 16001, size=(200, nr))
    q[:, 0] = 16000  # max |q| in [2^13, 2^14 - 1): the scale is exactly 2^-30
    w = q * 2.0 ** -30
    np.testing.assert_array_equal(orc.se15_unpack(orc.se15_pack(w, nr)[0], nr), w)
    z, _ = orc.se15_pack(np.zeros((1, nr)), nr)
    assert np.all(orc.se15_unpack(z, nr) == 0)
    bad_links = np.ones((3, nr))
    bad_links[1, 3] = np.nan
    bad_links[2, 0] = np.inf
    hb, nb = orc.se15_pack(bad_links, nr)
    assert nb == 2 and np.all(orc.se15_unpack(hb, nr)[1:] == 0)


def test_se15_gauge_emulate(orc):
    """The emulated field keeps each link's relative precision (2^-14 of its own largest element),
    where 16-bit fixed point with one global scale loses the small links."""
    dims = (4, 4, 4, 4)
    fat = synth.gauge_field(dims, "fat", seed=3).numpy()
    g = np.random.Generator(np.random.Philox(key=12))
    fat = fat * np.exp(g.uniform(-8, 0, size=fat.shape[:-3]))[..., None, None, None]  # magnitudes over 2^11
    e = orc.gauge_emulate(dims, fat, "se15", 18, long_link=False)
    f = orc.gauge_emulate(dims, fat, "fix16", 18, long_link=False)
    links = fat.reshape(-1, 18)
    mx = np.abs(links).max(axis=1)
    err_se = np.abs(e.reshape(-1, 18) - links).max(axis=1) / mx
    err_fx = np.abs(f.reshape(-1, 18) - links).max(axis=1) / mx
    assert np.all(err_se <= 2.0 ** -14)
    assert np.median(err_fx) > 10 * np.median(err_se)


def test_half_golden(orc):
    for vals, fields in _read("half_vectors.txt"):
        rec, bad = orc.half_pack(np.array([vals], dtype=np.float32))
        assert bad == 0
        q = np.frombuffer(rec[0, :12].tobytes(), dtype=np.int16)
        norm = np.frombuffer(rec[0, 12:].tobytes(), dtype=np.float32)[0]
        assert list(q) == [int(v) for v in fields[:6]], vals
        assert norm == np.float32(float(fields[6]))


def _random_sites(n, seed):
    g = np.random.Generator(np.random.Philox(key=seed))
    v = g.standard_normal((n, 6)) * np.exp(g.uniform(-30, 30, size=(n, 1)))
    v[::17, 2] = 0.0           # sites with zero components
    v[::31] *= 1e-15          # tiny sites; max/(2^19-1) stays an FP32 normal
    return v


def test_int20_roundtrip_bound_and_idempotence(orc):
    v = _random_sites(20000, 1).astype(np.float32)
    w, bad = orc.int20_pack(v)
    assert bad == 0
    u = orc.int20_unpack(w)
    mx = np.abs(v).max(axis=1, keepdims=True)
    # step 2^(E-127) <= 2 max/(2^19-1): error <= max/(2^19-1) (+ FP32 rounding of t)
    assert np.all(np.abs(u - v) <= mx / 524287.0 * (1 + 1e-6))
    w2, _ = orc.int20_pack(u)
    np.testing.assert_array_equal(w, w2)


def test_int20_exact_grid_and_zero(orc):
    g = np.random.Generator(np.random.Philox(key=4))
    q = g.integers(-300000, 300001, size=(500, 6))
    q[:, 0] = 300000  # max |q| in [2^18, 2^19): the scale is exactly 2^-10
    v = (q * 2.0 ** -10).astype(np.float32)
    u = orc.int20_unpack(orc.int20_pack(v)[0])
    np.testing.assert_array_equal(u, v)
    w, _ = orc.int20_pack(np.zeros((1, 6), np.float32))
    assert np.all(orc.int20_unpack(w) == 0)


def test_int20_exponent_floor(orc):
    # the smallest exponent is E = 1 (scale 2^-126): sites below the FP32
    # normal range round onto that grid rather than keeping 20 bits
    v = np.array([[3e-39, -1e-40, 0, 0, 0, 2e-45]], np.float32)
    w, _ = orc.int20_pack(v)
    assert w[0, 3] >> 24 == 1
    assert np.all(np.abs(orc.int20_unpack(w) - v) <= 2.0 ** -127)


def test_int20_nonfinite_flagged(orc):
    v = np.ones((3, 6), np.float32)
    v[1, 4] = np.nan
    v[2, 0] = np.inf
    _, bad = orc.int20_pack(v)
    assert bad == 2


def test_int14_roundtrip_bound_and_idempotence(orc):
    v = _random_sites(20000, 8).astype(np.float32)
    w, bad = orc.int14_pack(v)
    assert bad == 0
    assert np.all((w[:, 2] & 0x00030003) == 0)  # halves 4 and 5 carry no exponent bits
    u = orc.int14_unpack(w)
    mx = np.abs(v).max(axis=1, keepdims=True)
    # step 2^(E-127) <= 2 max/(2^13-1): error <= max/(2^13-1) (+ FP32 rounding of t)
    assert np.all(np.abs(u - v) <= mx / 8191.0 * (1 + 1e-6))
    # re-encoding the decoded site gives the same record, except where the
    # largest integer rounded up to 2^13 - 1: there t = 2^(E-127) exactly and
    # the rule picks the next exponent
    w2, _ = orc.int14_pack(u)
    def expo(ww):
        return sum(((ww[:, k // 2].astype(np.int64) >> (16 * (k % 2))) & 3) << (2 * k) for k in range(4))
    E = expo(w)
    qmax = np.rint(np.abs(u).max(axis=1) / np.ldexp(1.0, E - 127)).astype(np.int64)
    top = qmax == 8191
    np.testing.assert_array_equal(w[~top], w2[~top])
    assert np.all(expo(w2)[top] == E[top] + 1)


def test_int14_exact_grid_zero_floor_and_nonfinite(orc):
    g = np.random.Generator(np.random.Philox(key=9))
    q = g.integers(-8000, 8001, size=(500, 6))
    q[:, 1] = 8000  # max |q| in [2^12, 2^13 - 1): the scale is exactly 2^-7
    v = (q * 2.0 ** -7).astype(np.float32)
    np.testing.assert_array_equal(orc.int14_unpack(orc.int14_pack(v)[0]), v)
    w, _ = orc.int14_pack(np.zeros((1, 6), np.float32))
    assert np.all(orc.int14_unpack(w) == 0)
    # E = 1 (scale 2^-126) is the floor: FP32 subnormal sites land on that grid
    v = np.array([[3e-39, -1e-40, 0, 0, 0, 2e-45]], np.float32)
    w, _ = orc.int14_pack(v)
    e = sum(((int(w[0, k // 2]) >> (16 * (k % 2))) & 3) << (2 * k) for k in range(4))
    assert e == 1
    assert np.all(np.abs(orc.int14_unpack(w) - v) <= 2.0 ** -127)
    v = np.ones((3, 6), np.float32)
    v[1, 4] = np.nan
    v[2, 0] = -np.inf
    w, bad = orc.int14_pack(v)
    assert bad == 2 and np.all(orc.int14_unpack(w)[1:] == 0)


def test_half_roundtrip_bound_and_idempotence(orc):
    v = _random_sites(20000, 2).astype(np.float32)
    rec, bad = orc.half_pack(v)
    assert bad == 0
    u = orc.half_unpack(rec)
    mx = np.abs(v).max(axis=1, keepdims=True)
    # half a step of max/32767 plus FP32 rounding of the scale and product
    assert np.all(np.abs(u - v) <= mx * (0.5 / 32767.0 + 3 * 2.0 ** -24))
    assert np.all(np.abs(u - v) <= mx * 2.0 ** -15)   # the epsilon of Sec. 2
    # the decoded maximum is max*(1 +- 2^-23), so a second pass may move a
    # component by one step of the 16-bit grid, never more
    rec2, _ = orc.half_pack(u)
    q1 = rec[:, :12].copy().view(np.int16).astype(np.int64)
    q2 = rec2[:, :12].copy().view(np.int16).astype(np.int64)
    assert np.abs(q1 - q2).max() <= 1


def test_int30_roundtrip_bound_and_idempotence(orc):
    v = _random_sites(20000, 3)
    w, bad = orc.int30_pack(v)
    assert bad == 0
    u = orc.int30_unpack(w)
    mx = np.abs(v).max(axis=1, keepdims=True)
    assert np.all(np.abs(u - v) <= mx / 536870911.0 * (1 + 1e-12))
    assert np.all(np.abs(u - v) <= mx * 2.0 ** -29)
    w2, _ = orc.int30_pack(u)
    np.testing.assert_array_equal(w, w2)


def test_int30_exact_grid(orc):
    g = np.random.Generator(np.random.Philox(key=5))
    # max |q| in [2^28, 2^29 - 1): t = max/(2^29-1) lies in [2^-41, 2^-40),
    # so the scale is exactly 2^-40 (a max of 2^29-1 would give t = 2^-40
    # and round the scale up to 2^-39)
    q = g.integers(-(2 ** 29 - 2), 2 ** 29 - 1, size=(300, 6))
    q[:, 3] = 2 ** 29 - 2
    v = q * 2.0 ** -40
    np.testing.assert_array_equal(orc.int30_unpack(orc.int30_pack(v)[0]), v)


def test_spinor_emulate_orders(orc):
    """Format error ordering of Sec. 4: int30 << f32 < int20 < half < int14."""
    v = synth.spinor((4, 4, 4, 4), 7).numpy().reshape(-1, 6)
    err = {}
    for f in ("f32", "half", "int20", "int30", "int14"):
        e = orc.spinor_emulate(v, f)
        err[f] = np.linalg.norm(e - v) / np.linalg.norm(v)
    assert err["int30"] < 1e-8 < err["f32"] < 1e-6 < err["int20"] < err["half"] < 1e-4
    assert err["half"] / err["int20"] > 8     # 4 more bits
    assert 2 < err["int14"] / err["half"] < 8  # 13 bits against the 16-bit format's 15
    np.testing.assert_array_equal(orc.spinor_emulate(v, "f64"), v)


@pytest.mark.parametrize("bits", [16, 32])
def test_fixed_point_gauge(orc, bits):
    dims = (4, 4, 4, 4)
    fat = synth.gauge_field(dims, "fat", seed=9).numpy()
    gmax = orc.absmax(fat)
    assert 0.5 < gmax <= 0.8 + 1e-12
    q = orc.fix_pack(fat, gmax, bits)
    qm = 32767 if bits == 16 else 2 ** 31 - 1
    assert np.abs(q).max() == qm
    d = orc.fix_unpack(q, gmax, bits, compute_f32=False)
    assert np.abs(d - fat.reshape(-1)).max() <= 0.5 * gmax / qm * (1 + 1e-9)
    d32 = orc.fix_unpack(q, gmax, bits, compute_f32=True)
    np.testing.assert_array_equal(d32, (q.astype(np.float32) * np.float32(gmax / qm)).astype(np.float64))


def test_reconstruct12(orc):
    dims = (4, 4, 4, 6)
    for anti in (False, True):
        lng = synth.gauge_field(dims, "long", seed=4, antiperiodic_t=anti).numpy()
        e = orc.gauge_emulate(dims, lng, "f64", 12, long_link=True, antiperiodic_t=anti)
        assert np.abs(e - lng).max() <= 1e-14
        # with the wrong boundary sign the t-boundary links come back negated
        bad = orc.gauge_emulate(dims, lng, "f64", 12, long_link=True, antiperiodic_t=not anti)
        assert np.abs(bad - lng).max() > 1.0
    fat = synth.gauge_field(dims, "fat", seed=4).numpy()
    # fat links are 0.8 eta U: not in SU(3) up to a sign, so row 2 is not rebuilt by r12
    e = orc.gauge_emulate(dims, fat, "f64", 12, long_link=False)
    assert np.abs(e - fat).max() > 0.1
    lng = synth.gauge_field(dims, "long", seed=4).numpy()
    e32 = orc.gauge_emulate(dims, lng, "f32", 12, long_link=True)
    assert np.abs(e32 - lng).max() <= 1e-6
    e16 = orc.gauge_emulate(dims, lng, "fix16", 12, long_link=True, compute_f32=False)
    assert np.abs(e16 - lng).max() <= 4.0 / 32767


def test_half_floor(orc):
    # 32767/max overflows FP32 below ~1e-34: such sites are stored as zero
    v = np.array([[1e-35, 0, 0, 0, 0, -2e-36], [2.0 ** -109, 0, 0, 0, 0, 0]], np.float32)
    rec, bad = orc.half_pack(v)
    assert bad == 0
    u = orc.half_unpack(rec)
    assert np.all(u[0] == 0)
    assert abs(u[1, 0] - 2.0 ** -109) <= 2.0 ** -109 / 32767
