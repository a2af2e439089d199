"""Failure detection made on the host (no GPU fault): a device-memory budget
too small for the context's own buffers, or for a gauge field, is refused
with ENOMEM; the accounting returns to its level before the refused
allocation and the context stays usable.  (NaN inputs and maxiter are covered
in the stencil and CG tests.)"""
import numpy as np
import pytest
import torch

from paper_2302_09224_gb300 import hisq, synth

pytestmark = pytest.mark.gpu


def test_budget_too_small():
    # 1 MiB holds less than the context's reduction buffers (about 16.8 MB)
    with pytest.raises(hisq.HisqError, match="ENOMEM"):
        hisq.hisq_create(0, 1 << 20)
    c = hisq.hisq_create(0, 64 << 20)
    ref = hisq.hisq_create(0)
    try:
        # the FP64 copies of a 16^4 field (2 x 37.7 MB) exceed the 64 MiB budget left after the buffers
        big = (16, 16, 16, 16)
        fat, lng = synth.gauge_pair(big, seed=0, device="cuda")
        used = hisq.hisq_mem_used(c)
        with pytest.raises(hisq.HisqError, match="ENOMEM"):
            hisq.hisq_load_gauge(c, big, fat, lng)
        assert hisq.hisq_mem_used(c) == used
        assert "budget" in hisq.hisq_last_error(c)
        del fat, lng
        # a smaller field then loads and its stencil agrees with a context of the default budget
        dims = (8, 8, 8, 8)
        fat, lng = synth.gauge_pair(dims, seed=0, device="cuda")
        x = synth.spinor(dims, 1000, device="cuda")
        outs = []
        for ctx in (c, ref):
            g = hisq.hisq_load_gauge(ctx, dims, fat, lng)
            try:
                out = torch.empty_like(x)
                hisq.hisq_dslash(ctx, g, hisq.prec("int20", 12), 0, 0.0, None, x, out, True)
                torch.cuda.synchronize()
                outs.append(out.cpu().numpy())
            finally:
                hisq.hisq_free_gauge(ctx, g)
        assert np.isfinite(outs[0]).all()
        d = np.linalg.norm(outs[0] - outs[1]) / np.linalg.norm(outs[1])
        assert d <= 1e-6
        assert hisq.hisq_mem_used(c) >= used
    finally:
        hisq.hisq_destroy(c)
        hisq.hisq_destroy(ref)
