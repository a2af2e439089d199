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
