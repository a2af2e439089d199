"""The seeded input generator: determinism and the structure of its fields."""
import numpy as np
import torch

from paper_2302_09224_gb300 import synth


def test_links_are_phased_su3():
    dims = (4, 2, 4, 6)
    for anti in (False, True):
        lng = synth.gauge_field(dims, "long", seed=3, antiperiodic_t=anti)
        u = torch.view_as_complex(lng.contiguous()).reshape(4, -1, 3, 3)
        eye = torch.eye(3, dtype=u.dtype)
        assert torch.allclose(u @ u.conj().transpose(-1, -2), eye.expand_as(u), atol=1e-14)
        det = torch.linalg.det(u)
        vol = int(np.prod(dims))
        lex = torch.arange(vol)
        for mu in range(4):
            s = synth.link_signs(dims, mu, lex, True, anti)
            assert torch.allclose(det[mu], s.to(det.dtype), atol=1e-13)
    fat = synth.gauge_field(dims, "fat", seed=3)
    f = torch.view_as_complex(fat.contiguous()).reshape(4, -1, 3, 3) / 0.8
    assert torch.allclose(f @ f.conj().transpose(-1, -2), torch.eye(3, dtype=f.dtype).expand_as(f), atol=1e-13)


def test_near_identity_and_deterministic():
    dims = (4, 4, 4, 4)
    a = synth.gauge_field(dims, "long", seed=0)
    b = synth.gauge_field(dims, "long", seed=0, chunk_links=1000)
    assert torch.equal(a, b)
    c = synth.gauge_field(dims, "long", seed=1)
    assert not torch.equal(a, c)
    u = torch.view_as_complex(a.contiguous()).reshape(4, -1, 3, 3)
    tr = (u[0, :, 0, 0] + u[0, :, 1, 1] + u[0, :, 2, 2]).real / 3   # mu = 0 carries no phase
    assert 0.8 < float(tr.mean()) < 1.0
    s = synth.spinor(dims, 1000)
    assert s.shape == (128, 3, 2) and torch.equal(s, synth.spinor(dims, 1000))
    assert abs(float(s.std()) - 1.0) < 0.1


def test_poisson_stream():
    r = synth.poisson_requests(400, seed=1)
    assert r == synth.poisson_requests(400, seed=1)
    dt = np.diff([q["t"] for q in r])
    assert 150 < 1.0 / dt.mean() < 260
    ms = np.mean([q["multishift"] for q in r])
    assert 0.2 < ms < 0.4
