"""The C-ABI library loads and exports every function include/hisq.h declares (CPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    with open(os.path.join(ROOT, "include", "hisq.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"HISQ_API\s+[\w\s\*]*?\b(hisq_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2302_09224_gb300 import build, hisq

    build.build()
    return hisq.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2302_09224_gb300 import hisq

    assert set(declared()) <= set(hisq._SIGS), set(declared()) - set(hisq._SIGS)


def test_pure_host_calls(lib):
    from paper_2302_09224_gb300 import hisq

    assert hisq.hisq_spinor_bytes(hisq.HISQ_SPINOR_HALF16, 10) == 160
    assert hisq.hisq_spinor_bytes(hisq.HISQ_SPINOR_INT30, 10) == 240
    assert hisq.hisq_spinor_bytes(hisq.HISQ_SPINOR_INT14, 10) == 120
    assert hisq.hisq_spinor_bytes(hisq.HISQ_SPINOR_F64, 3) == 144
    assert hisq.hisq_spinor_bytes(9, 3) == 0
    p = hisq.hisq_default_params()
    assert p.delta == 0.1 and p.nbuf == 8 and p.pr_beta == 1 and p.reproject == 1 and p.l == 4
    assert p.sloppy.spinor == hisq.HISQ_SPINOR_INT20 and p.sloppy.long_recon == 12


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2302_09224_gb300 import hisq

    monkeypatch.setattr(hisq, "_lib", None)
    monkeypatch.setattr(hisq, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        hisq.lib()


def test_host_controls_and_refusals(lib):
    """Calls that need no device: the launch-shape and fused-pass controls
    return their previous value and refuse out-of-range values (-2) without
    changing the setting; null contexts are refused, not dereferenced."""
    from paper_2302_09224_gb300 import hisq

    old = hisq.hisq_stencil_config(2)
    try:
        assert hisq.hisq_stencil_config(99) == -2 and hisq.hisq_stencil_config(-5) == -2
        assert hisq.hisq_stencil_config(3) == 2  # the refused calls left 2 in place
    finally:
        hisq.hisq_stencil_config(old)
    old = hisq.hisq_stencil_config_reduce(-1)
    try:
        assert hisq.hisq_stencil_config_reduce(99) == -2
        assert hisq.hisq_stencil_config_reduce(old) == -1
    finally:
        hisq.hisq_stencil_config_reduce(old)
    old = hisq.hisq_mee_fused(0)
    try:
        assert hisq.hisq_mee_fused(2) == -2 and hisq.hisq_mee_fused(-1) == -2
        assert hisq.hisq_mee_fused(old) == 0
    finally:
        hisq.hisq_mee_fused(old)
    for control in (hisq.hisq_programmatic_launch, hisq.hisq_cg_split_scalars):
        old = control(0)
        try:
            assert old in (0, 1)
            assert control(2) == -2 and control(-1) == -2
            assert control(1) == 0  # the refused calls left 0 in place
        finally:
            control(old)
    assert hisq.hisq_mem_used(None) == 0 and hisq.hisq_launch_count(None) == 0
    assert hisq.hisq_last_error(None) == "null context"
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        hisq.hisq_profile_sample(None, 1)


def test_create_without_a_device_is_refused(lib):
    """On a host without a GPU the library loads (every entry point is there)
    and hisq_create refuses cleanly instead of falling back to the CPU."""
    import torch

    from paper_2302_09224_gb300 import hisq

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        hisq.hisq_create(0)
