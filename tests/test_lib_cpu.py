"""Host-side checks of the CUDA library that need no GPU: it builds for
sm_103a, loads, and exports every entry point that include/nair.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "nair.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nair_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    from paper_1704_05001_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(nair_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_library_loads_and_binding_names_match(built):
    import paper_1704_05001_gb300 as nair
    L = nair.lib()
    for name in declared_symbols():
        assert hasattr(L, name)
    assert sorted(nair.EXPORTS) == declared_symbols()


def test_default_params_without_gpu(built):
    import paper_1704_05001_gb300 as nair
    p = nair.default_params()
    assert p.strength_theta == 0.1 and p.filter_tol == 1e-4 and p.neumann_degree == 1
    assert p.gmres_restart == 50 and p.tol == 1e-10 and p.max_levels == 25


def test_no_cpu_fallback_when_library_missing(monkeypatch):
    import paper_1704_05001_gb300 as nair
    monkeypatch.setattr(nair, "_lib", None)
    monkeypatch.setattr(nair, "LIB_PATH", "/nonexistent/libnair.so")
    with pytest.raises(RuntimeError):
        nair.lib()
