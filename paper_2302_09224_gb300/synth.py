"""Seeded synthetic inputs for the HISQ stencil and its solvers.

This module is the one place where inputs are made.  Both the CUDA path
(tests, benchmark) and the CPU oracle consume what it returns; it holds none
of the stencil, storage-format or solver arithmetic of either side.

Recipe (the paper's gauge ensembles are not available, so synthetic fields of
the same structure stand in for them):

* Random numbers: numpy's Philox-4x64 counter-based generator (Salmon et al.,
  SC'11), keyed by ``(seed, field, chunk)`` so any chunk can be regenerated on
  its own and the stream does not depend on the device or on chunking.
* Link field: per link a 3x3 complex Gaussian ``G`` (unit variance for the real
  and the imaginary part), ``H = (G + G^+)/2 - tr/3``, ``U = exp(i eps H)`` with
  ``eps = 0.3`` (12th-order Taylor of ``exp(A/4)`` squared twice, error below
  1e-16 for these norms), then re-unitarised: Gram-Schmidt on rows 0 and 1 and
  row 2 = conj(row0 x row1), so ``U`` is in SU(3) to rounding.
* Fat links ``F_mu(x) = 0.8 * eta_mu(x) * U_f``; long (Naik) links
  ``L_mu(x) = eta_mu(x) * U_l``, staggered phases ``eta_0 = 1``,
  ``eta_1 = (-1)^x``, ``eta_2 = (-1)^(x+y)``, ``eta_3 = (-1)^(x+y+z)``; with
  antiperiodic time, links that cross the t boundary carry an extra -1 (fat at
  ``t = Lt-1``, long at ``t >= Lt-3``).
* Right-hand sides: Gaussian complex 3-vectors (unit variance per real part)
  on the sites of one parity, seed ``1000 + k`` for the k-th vector.

Array layouts (the C ABI's host layouts):

* gauge: float64 ``[mu][t][z][y][x][row][col][re,im]``;
* half-lattice spinor: float64 ``[cb][color][re,im]`` where ``cb = lex // 2``
  and ``lex = ((t*Lz + z)*Ly + y)*Lx + x``;
* full-lattice spinor: ``[parity][cb][color][re,im]``, even parity first.
"""
from __future__ import annotations

import math

import numpy as np
import torch

EPS_DEFAULT = 0.3
FAT_SCALE = 0.8
GAUGE_SEED = 0
LINKS_PER_CHUNK = 1 << 16
_FIELD_FAT = 1
_FIELD_LONG = 2
_FIELD_SPINOR = 3


def _philox(seed: int, field: int, chunk: int) -> np.random.Generator:
    key = (int(seed) & 0xFFFFFFFF) | (int(field) << 32) | (int(chunk) << 64)
    return np.random.Generator(np.random.Philox(key=key))


def volume(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def check_dims(dims):
    if len(dims) != 4 or any(int(d) < 2 or int(d) % 2 for d in dims):
        raise ValueError(f"lattice extents must be four even numbers >= 2, got {dims}")


def _link_normals(seed: int, field: int, n_links: int, start: int, count: int) -> np.ndarray:
    """18 normals per link for links [start, start+count) of one field."""
    out = np.empty((count, 18), dtype=np.float64)
    c0 = start // LINKS_PER_CHUNK
    c1 = (start + count - 1) // LINKS_PER_CHUNK
    for c in range(c0, c1 + 1):
        lo = c * LINKS_PER_CHUNK
        hi = min(lo + LINKS_PER_CHUNK, n_links)
        blk = _philox(seed, field, c).standard_normal((hi - lo) * 18).reshape(hi - lo, 18)
        a = max(lo, start)
        b = min(hi, start + count)
        out[a - start:b - start] = blk[a - lo:b - lo]
    return out


def _su3_from_normals(nrm: torch.Tensor, eps: float) -> torch.Tensor:
    """(n,18) normals -> (n,3,3) complex128 SU(3) matrices near the identity."""
    g = torch.complex(nrm[:, 0::2], nrm[:, 1::2]).reshape(-1, 3, 3)
    h = 0.5 * (g + g.conj().transpose(1, 2))
    tr = (h[:, 0, 0] + h[:, 1, 1] + h[:, 2, 2]) / 3.0
    eye = torch.eye(3, dtype=h.dtype, device=h.device)
    h = h - tr[:, None, None] * eye
    a = (1j * eps / 4.0) * h
    e = eye.expand_as(a).clone()
    for k in range(12, 0, -1):  # Horner form of sum_k a^k/k!
        e = eye + torch.matmul(a, e) / k
    e = torch.matmul(e, e)
    e = torch.matmul(e, e)
    r0 = e[:, 0, :]
    r0 = r0 / torch.linalg.vector_norm(r0, dim=1, keepdim=True)
    r1 = e[:, 1, :]
    r1 = r1 - (r0.conj() * r1).sum(1, keepdim=True) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=1, keepdim=True)
    r2 = torch.linalg.cross(r0, r1, dim=1).conj()
    return torch.stack([r0, r1, r2], dim=1)


def _coords(dims, lex: torch.Tensor):
    lx, ly, lz, _ = (int(d) for d in dims)
    x = lex % lx
    r = lex // lx
    y = r % ly
    r = r // ly
    z = r % lz
    t = r // lz
    return x, y, z, t


def link_signs(dims, mu: int, lex: torch.Tensor, long_link: bool, antiperiodic_t: bool) -> torch.Tensor:
    """Staggered phase times boundary sign for links (mu, lex): +-1 float64."""
    x, y, z, t = _coords(dims, lex)
    if mu == 0:
        s = torch.zeros_like(x)
    elif mu == 1:
        s = x
    elif mu == 2:
        s = x + y
    else:
        s = x + y + z
    sign = 1.0 - 2.0 * (s % 2).to(torch.float64)
    if antiperiodic_t and mu == 3:
        lt = int(dims[3])
        cross = (t >= lt - 3) if long_link else (t == lt - 1)
        sign = torch.where(cross, -sign, sign)
    return sign


def gauge_field(dims, kind: str = "fat", seed: int = GAUGE_SEED, eps: float = EPS_DEFAULT,
                antiperiodic_t: bool = False, device="cpu", chunk_links: int = 1 << 20) -> torch.Tensor:
    """One synthetic link field, float64 ``[mu][t][z][y][x][3][3][2]`` on ``device``."""
    check_dims(dims)
    if kind not in ("fat", "long"):
        raise ValueError(kind)
    field = _FIELD_FAT if kind == "fat" else _FIELD_LONG
    vol = volume(dims)
    n_links = 4 * vol
    out = torch.empty((n_links, 3, 3, 2), dtype=torch.float64, device=device)
    scale = FAT_SCALE if kind == "fat" else 1.0
    for start in range(0, n_links, chunk_links):
        cnt = min(chunk_links, n_links - start)
        nrm = torch.from_numpy(_link_normals(seed, field, n_links, start, cnt)).to(device)
        u = _su3_from_normals(nrm, eps)
        idx = torch.arange(start, start + cnt, device=device, dtype=torch.int64)
        mu_of = idx // vol
        lex = idx % vol
        sign = torch.empty(cnt, dtype=torch.float64, device=device)
        for mu in range(4):
            m = mu_of == mu
            if bool(m.any()):
                sign[m] = link_signs(dims, mu, lex[m], kind == "long", antiperiodic_t)
        u = u * (scale * sign)[:, None, None]
        out[start:start + cnt] = torch.view_as_real(u)
    lx, ly, lz, lt = (int(d) for d in dims)
    return out.reshape(4, lt, lz, ly, lx, 3, 3, 2)


def gauge_pair(dims, seed: int = GAUGE_SEED, eps: float = EPS_DEFAULT, antiperiodic_t: bool = False,
               device="cpu"):
    """(fat, long) synthetic link fields for one lattice."""
    return (gauge_field(dims, "fat", seed, eps, antiperiodic_t, device),
            gauge_field(dims, "long", seed, eps, antiperiodic_t, device))


def unit_gauge(dims, c: float, antiperiodic_t: bool = False, long_link: bool = False) -> torch.Tensor:
    """Free field: ``c * eta_mu(x) * identity`` on every link (float64, CPU)."""
    check_dims(dims)
    vol = volume(dims)
    lex = torch.arange(vol, dtype=torch.int64)
    out = torch.zeros((4, vol, 3, 3, 2), dtype=torch.float64)
    for mu in range(4):
        s = link_signs(dims, mu, lex, long_link, antiperiodic_t) * c
        for i in range(3):
            out[mu, :, i, i, 0] = s
    lx, ly, lz, lt = (int(d) for d in dims)
    return out.reshape(4, lt, lz, ly, lx, 3, 3, 2)


def spinor(dims, seed: int, full: bool = False, device="cpu") -> torch.Tensor:
    """Gaussian source: ``[Vh][3][2]`` (or ``[2][Vh][3][2]`` if ``full``) float64."""
    check_dims(dims)
    vh = volume(dims) // 2
    n = (2 * vh if full else vh) * 6
    v = _philox(seed, _FIELD_SPINOR, 0).standard_normal(n)
    t = torch.from_numpy(v).to(device)
    return t.reshape((2, vh, 3, 2) if full else (vh, 3, 2))


def rhs_seed(k: int) -> int:
    """Seed of the k-th right-hand side."""
    return 1000 + int(k)


def shifts_logspaced(n: int, lo: float = 1e-4, hi: float = 1.0):
    """Rational-approximation-style shifts: n values log-spaced in [lo, hi]."""
    if n == 1:
        return [lo]
    return [lo * (hi / lo) ** (i / (n - 1)) for i in range(n)]


def shift_tolerances(n: int, lo: float = 1e-10, hi: float = 1e-7):
    """Per-shift targets, log-spaced from ``lo`` (smallest shift) to ``hi``."""
    return shifts_logspaced(n, lo, hi)


def poisson_requests(n: int, rate_hz: float = 200.0, seed: int = 1,
                     volumes=((8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 48), (32, 32, 32, 64)),
                     mass_range=(1e-3, 1e-1), tols=(1e-6, 1e-8, 1e-10), frac_multishift=0.3,
                     nshift=8):
    """A seeded Poisson stream of solve requests (arrival time, kind and parameters)."""
    g = _philox(seed, 7, 0)
    t = 0.0
    reqs = []
    for i in range(n):
        t += g.exponential(1.0 / rate_hz)
        vol = volumes[int(g.integers(len(volumes)))]
        m = math.exp(g.uniform(math.log(mass_range[0]), math.log(mass_range[1])))
        tol = tols[int(g.integers(len(tols)))]
        ms = bool(g.uniform() < frac_multishift)
        reqs.append({"t": t, "dims": tuple(vol), "mass": m, "tol": tol, "multishift": ms,
                     "shifts": shifts_logspaced(nshift) if ms else None, "rhs_seed": rhs_seed(i)})
    return reqs
