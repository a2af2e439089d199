"""Pins of the oracle's HISQ stencil (CPU only).

The stencil is only named in the paper (Sec. 1, Sec. 5.2); the oracle reads
it as the one-hop fat plus three-hop Naik staggered operator with phased links.
These tests fix that reading by properties a mistake would break:

* free field: with links ``c1 eta_mu`` (fat) and ``c3 eta_mu`` (long) a plane
  wave is mapped to ``2i e^{ipx} sum_mu eta_mu(x) (c1 sin p_mu + c3 sin 3p_mu)``
  times itself, and M_ee has eigenvalue ``4m^2 + 4 sum_mu (c1 sin p_mu +
  c3 sin 3p_mu)^2`` (the eta cross terms cancel in D^2);
* anti-hermiticity ``D_oe = -D_eo^+``;
* gauge covariance ``D[U^Omega](Omega psi) = Omega D[U] psi``;
* dense-matrix identities at 2^4 and 4^4 (where the +3 hop aliases the -1 hop).
"""
import numpy as np
import pytest
import torch

from paper_2302_09224_gb300 import synth


def lex_of_cb(dims, parity):
    """lex index of every checkerboard site of the given parity."""
    lx, ly, lz, lt = dims
    vh = lx * ly * lz * lt // 2
    lex = 2 * np.arange(vh)
    x = lex % lx
    y = (lex // lx) % ly
    z = (lex // (lx * ly)) % lz
    t = lex // (lx * ly * lz)
    par = (x + y + z + t) % 2
    return lex + (par != parity)


def coords(dims, lex):
    lx, ly, lz, lt = dims
    return (lex % lx, (lex // lx) % ly, (lex // (lx * ly)) % lz, lex // (lx * ly * lz))


def eta(mu, c):
    x, y, z, t = c
    s = [0 * x, x, x + y, x + y + z][mu]
    return 1.0 - 2.0 * (s % 2)


def to_c(a):
    a = np.asarray(a)
    return a[..., 0] + 1j * a[..., 1]


def to_r(a):
    return np.stack([a.real, a.imag], axis=-1)


def plane_wave(dims, parity, k, chi, antiperiodic=False):
    lex = lex_of_cb(dims, parity)
    c = coords(dims, lex)
    p = [2 * np.pi * k[mu] / dims[mu] for mu in range(4)]
    if antiperiodic:
        p[3] = (2 * k[3] + 1) * np.pi / dims[3]
    ph = np.exp(1j * sum(p[mu] * c[mu] for mu in range(4)))
    return ph[:, None] * np.asarray(chi)[None, :], p, c


@pytest.mark.parametrize("dims,k,anti", [
    ((4, 6, 8, 10), (1, 2, 3, 1), False),
    ((4, 4, 4, 4), (1, 3, 2, 1), False),
    ((6, 4, 4, 8), (1, 1, 0, 2), True),
    ((8, 8, 4, 6), (3, 1, 1, 0), True),
])
def test_free_field_plane_wave(orc, dims, k, anti):
    c1, c3 = 0.7, -0.35
    fat = synth.unit_gauge(dims, c1, antiperiodic_t=anti, long_link=False)
    lng = synth.unit_gauge(dims, c3, antiperiodic_t=anti, long_link=True)
    chi = np.array([1.0 + 0.5j, -0.3 + 0.2j, 0.25 - 1.0j])
    for out_par in (0, 1):
        psi, p, _ = plane_wave(dims, 1 - out_par, k, chi, anti)
        out = to_c(orc.dslash(dims, fat, lng, out_par, to_r(psi)))
        wave_out, _, cout = plane_wave(dims, out_par, k, chi, anti)
        f = sum(eta(mu, cout) * (c1 * np.sin(p[mu]) + c3 * np.sin(3 * p[mu])) for mu in range(4))
        expect = 2j * f[:, None] * wave_out
        np.testing.assert_allclose(out, expect, atol=1e-13 * np.abs(expect).max() + 1e-14)


@pytest.mark.parametrize("dims,k,anti", [((4, 6, 8, 10), (1, 2, 3, 4), False), ((4, 4, 4, 6), (1, 0, 3, 1), True)])
def test_free_field_mee_eigenvalue(orc, dims, k, anti):
    c1, c3, m, sigma = 0.8, -0.2, 0.05, 0.3
    fat = synth.unit_gauge(dims, c1, antiperiodic_t=anti)
    lng = synth.unit_gauge(dims, c3, antiperiodic_t=anti, long_link=True)
    chi = np.array([0.3 - 0.1j, 1.0, -0.5j])
    psi, p, _ = plane_wave(dims, 0, k, chi, anti)
    out = to_c(orc.mee(dims, fat, lng, m, to_r(psi), sigma=sigma))
    lam = 4 * m * m + sigma + 4 * sum((c1 * np.sin(q) + c3 * np.sin(3 * q)) ** 2 for q in p)
    np.testing.assert_allclose(out, lam * psi, atol=1e-13 * lam)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 6, 2, 8)])
def test_anti_hermiticity(orc, dims):
    fat, lng = synth.gauge_pair(dims, seed=3)
    x = synth.spinor(dims, 11).numpy()
    y = synth.spinor(dims, 12).numpy()
    deo_x = to_c(orc.dslash(dims, fat, lng, 0, x))   # even <- odd
    doe_y = to_c(orc.dslash(dims, fat, lng, 1, y))   # odd <- even
    lhs = np.vdot(to_c(y), deo_x)
    rhs = -np.vdot(doe_y, to_c(x))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def _random_su3_field(dims, seed):
    vol = int(np.prod(dims))
    nrm = np.random.Generator(np.random.Philox(key=seed + 99)).standard_normal((vol, 18))
    u = synth._su3_from_normals(torch.from_numpy(nrm), 3.0).numpy()
    lx, ly, lz, lt = dims
    return u.reshape(lt, lz, ly, lx, 3, 3)


@pytest.mark.parametrize("dims", [(4, 6, 8, 6), (8, 4, 4, 4)])
def test_gauge_covariance(orc, dims):
    fat, lng = synth.gauge_pair(dims, seed=5, antiperiodic_t=True)
    lx, ly, lz, lt = dims
    F = to_c(fat.numpy())  # [mu][t][z][y][x][3][3]
    G = to_c(lng.numpy())
    om = _random_su3_field(dims, 1)
    axis = {0: 3, 1: 2, 2: 1, 3: 0}
    Fp = np.empty_like(F)
    Gp = np.empty_like(G)
    for mu in range(4):
        o1 = np.roll(om, -1, axis=axis[mu]).conj().swapaxes(-1, -2)
        o3 = np.roll(om, -3, axis=axis[mu]).conj().swapaxes(-1, -2)
        Fp[mu] = om @ F[mu] @ o1
        Gp[mu] = om @ G[mu] @ o3
    omf = om.reshape(-1, 3, 3)
    psi_o = to_c(synth.spinor(dims, 21).numpy())
    lo = lex_of_cb(dims, 1)
    le = lex_of_cb(dims, 0)
    psi_o_t = np.einsum("sij,sj->si", omf[lo], psi_o)
    out = to_c(orc.dslash(dims, fat, lng, 0, to_r(psi_o)))
    out_t = to_c(orc.dslash(dims, to_r(Fp), to_r(Gp), 0, to_r(psi_o_t)))
    np.testing.assert_allclose(out_t, np.einsum("sij,sj->si", omf[le], out), atol=1e-12)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_dense_identities(orc, dims):
    m = 0.07
    fat, lng = synth.gauge_pair(dims, seed=8)
    deo = orc.dense(dims, fat, lng, "deo")
    doe = orc.dense(dims, fat, lng, "doe")
    np.testing.assert_allclose(doe, -deo.conj().T, atol=1e-14)
    mee = orc.dense(dims, fat, lng, "mee", m=m)
    np.testing.assert_allclose(mee, 4 * m * m * np.eye(len(mee)) - deo @ doe, atol=1e-12)
    np.testing.assert_allclose(mee, mee.conj().T, atol=1e-12)
    ev = np.linalg.eigvalsh(mee)
    assert ev.min() >= 4 * m * m - 1e-10
    mf = orc.dense(dims, fat, lng, "mfull", m=m)
    nh = len(mee)
    # M^+ M = 4m^2 - D^2; its even block is M_ee
    np.testing.assert_allclose((mf.conj().T @ mf)[:nh, :nh], mee, atol=1e-11)
    # the full operator is 2m plus the two stencil blocks
    np.testing.assert_allclose(mf[:nh, nh:], deo, atol=1e-14)
    np.testing.assert_allclose(mf[nh:, :nh], doe, atol=1e-14)
    np.testing.assert_allclose(np.diag(mf), 2 * m, atol=1e-14)


def test_sampled_sites_match_full(orc):
    dims = (4, 4, 6, 8)
    fat, lng = synth.gauge_pair(dims, seed=2)
    x = synth.spinor(dims, 3).numpy()
    full = orc.dslash(dims, fat, lng, 1, x)
    cbs = np.array([0, 5, 17, len(full) - 1])
    np.testing.assert_array_equal(orc.dslash_sites(dims, fat, lng, 1, x, cbs), full[cbs])
