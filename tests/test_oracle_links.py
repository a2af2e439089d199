"""Pins of the oracle's compressed long-link formats (CPU only).

* 8 reals (Sec. 1: 18 -> 8 for SU(3) links): the parameters (arg V00, arg V20,
  V01, V02, V10) of V = sign * U and the rebuild from unitarity and det V = 1.
  In FP64 the rebuild returns every Haar-random SU(3) matrix (and sign times
  one) to rounding; two matrices whose rebuild is worked out by hand (a
  rotation in the (0, 1) plane and the cyclic permutation) come back exactly;
  with FP32 or 16-bit storage of the 8 reals the error follows the format's
  rounding, amplified where the rebuild divides by N = 1 - |V00|^2 or takes
  sqrt(N - |V10|^2) (links near diagonal).
* 13 reals (12 + 1, for long links in U(3)): rows 0 and 1 and the phase of
  det U; row 2 = det(U) conj(row0 x row1).  Exact in FP64 for U(3) matrices
  with any phase; for sign times SU(3) the stored phase is 0 or 1 (times pi)
  in every format, so the rebuild is the 12-real one.
"""
import numpy as np
import pytest

from paper_2302_09224_gb300 import synth


def haar_su3(n, seed):
    g = np.random.Generator(np.random.Philox(key=seed))
    z = g.standard_normal((n, 3, 3)) + 1j * g.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    return q / np.linalg.det(q)[:, None, None] ** (1.0 / 3.0)


def to_real(u):
    return np.stack([u.real, u.imag], axis=-1)


def to_cplx(a):
    a = np.asarray(a)
    return a[..., 0] + 1j * a[..., 1]


def test_r8_fp64_roundtrip_haar(orc):
    u = haar_su3(4000, 5)
    sign = np.where(np.arange(4000) % 3 == 0, -1.0, 1.0)
    links = to_real(u * sign[:, None, None])
    p = orc.link_r8_pack(links, sign)
    back = to_cplx(orc.link_r8_unpack(p, sign))
    err = np.abs(back - u * sign[:, None, None]).max(axis=(1, 2))
    n = np.abs(u[:, 0, 1]) ** 2 + np.abs(u[:, 0, 2]) ** 2
    assert np.all(err <= 1e-12 / np.minimum(n, 1.0))


@pytest.mark.parametrize("case", ["rotation", "cyclic"])
def test_r8_hand_derived_cases(orc, case):
    if case == "rotation":
        c, s = np.cos(np.pi / 6), 0.5
        v = np.array([[c, s, 0], [-s, c, 0], [0, 0, 1]], dtype=complex)
        # V00 = c (phase 0), V20 = 0 (phase 0), V01 = 1/2, V02 = 0, V10 = -1/2
        want = [0.0, 0.0, 0.5, 0.0, 0.0, 0.0, -0.5, 0.0]
    else:
        v = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], dtype=complex)
        # V00 = 0 (phase taken as 0), V20 = 1 (phase 0), V01 = 1, V02 = 0, V10 = 0
        want = [0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    p = orc.link_r8_pack(to_real(v[None]), np.ones(1))
    np.testing.assert_allclose(p[0], want, atol=1e-15)
    back = to_cplx(orc.link_r8_unpack(np.array([want]), np.ones(1)))[0]
    np.testing.assert_allclose(back, v, atol=1e-15)


def test_r8_reduced_storage_error(orc):
    u = haar_su3(20000, 6)
    ones = np.ones(len(u))
    p = orc.link_r8_pack(to_real(u), ones)
    p32 = p.astype(np.float32).astype(np.float64)
    err = np.abs(to_cplx(orc.link_r8_unpack(p32, ones)) - u).max(axis=(1, 2))
    assert np.median(err) <= 1e-6 and np.percentile(err, 99) <= 5e-6
    # 16-bit: angles and elements to 1/32767 of their range
    p16 = np.rint(p * 32767.0) / 32767.0
    err16 = np.abs(to_cplx(orc.link_r8_unpack(p16, ones)) - u).max(axis=(1, 2))
    assert np.median(err16) <= 3e-4 and np.median(err16) >= 1e-6


def test_gauge_emulate_r13_r8_fp64(orc):
    dims = (4, 4, 4, 6)
    lng = synth.gauge_field(dims, "long", seed=2, eps=1.2).numpy()
    for recon, bound in ((13, 1e-14), (8, 1e-10)):
        e = orc.gauge_emulate(dims, lng, "f64", recon, long_link=True)
        assert np.abs(e - lng).max() <= bound, recon
    # sign times SU(3): the 13-real phase is 0 or pi, stored exactly in 16 bits, so the rebuild is the
    # 12-real one
    e13 = orc.gauge_emulate(dims, lng, "fix16", 13, long_link=True)
    e12 = orc.gauge_emulate(dims, lng, "fix16", 12, long_link=True)
    assert np.abs(e13 - e12).max() <= 1e-15


def test_r13_u3_phase(orc):
    dims = (2, 2, 2, 2)
    lng = synth.gauge_field(dims, "long", seed=3).numpy()
    u = to_cplx(lng.reshape(-1, 3, 3, 2))
    g = np.random.Generator(np.random.Philox(key=9))
    ph = np.exp(1j * g.uniform(-np.pi, np.pi, len(u)))
    w = to_real(u * ph[:, None, None]).reshape(lng.shape)     # U(3): any phase of det
    e = orc.gauge_emulate(dims, w, "f64", 13, long_link=True)
    assert np.abs(e - w).max() <= 1e-14
    e16 = orc.gauge_emulate(dims, w, "fix16", 13, long_link=True, gmax=1.0)
    # rows 0, 1 to 1/65534 of the scale, row 2 also through the phase rounded to pi/65534
    assert np.abs(e16 - w).max() <= 4 * np.pi / 65534
