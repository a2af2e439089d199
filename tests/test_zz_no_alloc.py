"""hisq_dslash_noalloc: the stencil for callers that may not allocate device memory.

It must give the same result as hisq_dslash (the allocating entry point) on
the same inputs, call after call, although all its calls share one fixed
scratch array; sizes beyond its limit, missing gauge copies and non-finite
inputs are refused with EINVAL, a result that cannot be stored in the
spinor format returns ERANGE, and none of these poisons the next call.  This file is
collected last so that a failure here stops a -x run only after every other
test has run.
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


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("name,dims,parity,a", [
    ("int20", (8, 8, 8, 8), 0, 0.0),
    ("half", (16, 16, 16, 16), 2, 0.0),     # full lattice at the size limit
    ("f64", (4, 6, 8, 10), 1, 0.6),
    ("int30", (6, 4, 4, 10), 2, 0.3),
    ("f64", (16, 16, 16, 16), 2, 0.7),      # widest format at the limit: the scratch filled to its end
    ("int30", (16, 16, 16, 16), 2, -0.4),
])
def test_matches_allocating_entry_point(ctx, name, dims, parity, a):
    fat, lng = synth.gauge_pair(dims, seed=0, device="cuda")
    g = hisq.hisq_load_gauge(ctx, dims, fat, lng)
    try:
        p = hisq.prec(name, 12)
        for call in range(2):  # two calls in a row, different inputs each time
            full = parity == 2
            x = synth.spinor(dims, 1000 + call, full=full, device="cuda")
            y = synth.spinor(dims, 2000 + call, full=full, device="cuda")
            ref = torch.empty_like(x)
            hisq.hisq_dslash(ctx, g, p, parity, a, y if a else None, x, ref, True)
            out = torch.full_like(x, float("nan"))
            hisq.hisq_dslash_noalloc(ctx, g, p, parity, a, y if a else None, x, out)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert rel(out, ref) <= 1e-12, (name, call)
    finally:
        hisq.hisq_free_gauge(ctx, g)


def test_refusals_and_recovery(ctx):
    dims = (8, 8, 8, 8)
    fat, lng = synth.gauge_pair(dims, seed=1, device="cuda")
    g = hisq.hisq_load_gauge(ctx, dims, fat, lng)
    try:
        x = synth.spinor(dims, 5, device="cuda")
        out = torch.empty_like(x)
        # no stored copy for this precision yet: refused rather than allocated
        with pytest.raises(hisq.HisqError, match="no stored copy"):
            hisq.hisq_dslash_noalloc(ctx, g, hisq.prec("f32", 18), 0, 0.0, None, x, out)
        ref = torch.empty_like(x)
        hisq.hisq_dslash(ctx, g, hisq.prec("f32", 18), 0, 0.0, None, x, ref, True)
        bad = x.clone()
        bad[7, 2, 1] = float("nan")
        with pytest.raises(hisq.HisqError, match="non-finite"):
            hisq.hisq_dslash_noalloc(ctx, g, hisq.prec("f32", 18), 0, 0.0, None, bad, out)
        hisq.hisq_dslash_noalloc(ctx, g, hisq.prec("f32", 18), 0, 0.0, None, x, out)
        torch.cuda.synchronize()
        assert rel(out, ref) <= 1e-12
    finally:
        hisq.hisq_free_gauge(ctx, g)
    big = (16, 16, 16, 18)   # 36864 sites per parity > the fixed scratch
    fat, lng = synth.gauge_pair(big, seed=2, device="cuda")
    g = hisq.hisq_load_gauge(ctx, big, fat, lng)
    try:
        x = synth.spinor(big, 5, device="cuda")
        out = torch.empty_like(x)
        hisq.hisq_dslash(ctx, g, hisq.prec("int20"), 0, 0.0, None, x, out, True)
        with pytest.raises(hisq.HisqError, match="exceed"):
            hisq.hisq_dslash_noalloc(ctx, g, hisq.prec("int20"), 0, 0.0, None, x, out)
    finally:
        hisq.hisq_free_gauge(ctx, g)


@pytest.mark.parametrize("name", ["f64", "f32", "int20", "int30"])
def test_unstorable_output_is_reported(ctx, name):
    """Finite inputs whose stencil result overflows the compute precision give
    ERANGE (not a silently zeroed site), and the next call is correct."""
    dims = (4, 4, 4, 8)
    fat, lng = synth.gauge_pair(dims, seed=0, device="cuda")
    g = hisq.hisq_load_gauge(ctx, dims, fat, lng)
    try:
        p = hisq.prec(name, 12)
        x = synth.spinor(dims, 1, device="cuda")
        big = x / x.abs().max() * (1.7e308 if name == "f64" else 3.3e38)
        ref = torch.empty_like(x)
        hisq.hisq_dslash(ctx, g, p, 0, 0.0, None, x, ref, True)
        out = torch.empty_like(x)
        with pytest.raises(hisq.HisqError, match="ERANGE"):
            hisq.hisq_dslash_noalloc(ctx, g, p, 0, 0.0, None, big, out)
        hisq.hisq_dslash_noalloc(ctx, g, p, 0, 0.0, None, x, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    finally:
        hisq.hisq_free_gauge(ctx, g)
