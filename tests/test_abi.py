"""The C-ABI library builds, loads, and exports every entry point include/qaoa.h declares.
No compute calls: these run without a GPU."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qaoa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_0-9]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2506_10531_gb300 import build
    return build.build()


def test_header_declarations_found():
    names = declared_functions()
    assert "qaoa_run_layers" in names and "dqaoa_merge" in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    import paper_2506_10531_gb300 as q
    assert sorted(q.EXPORTS) == declared_functions()
    L = q.lib()
    for name in q.EXPORTS:
        assert hasattr(L, name)
        assert callable(getattr(q, name)), name


def test_invalid_arguments_rejected_before_any_launch(libpath):
    # NULL context and out-of-range sizes fail validation without touching CUDA
    import paper_2506_10531_gb300 as q
    L = q.lib()
    assert L.qaoa_run_layers(None, 10, 1, None, None, None, None, 1, None) == q.QAOA_E_INVALID
    assert L.dqaoa_merge(None, 0, None, 0, 0, None, 0, None, None, None) == q.QAOA_E_INVALID
    assert L.dqaoa_session_cycle_sampled(None, None, 0, None, 0, 0, 16, None, None, None, None) == q.QAOA_E_INVALID
    assert L.dqaoa_session_shots(None, None, None, None) == q.QAOA_E_INVALID
    assert L.qaoa_server_cancel(None, 1) == q.QAOA_E_INVALID
    assert L.qaoa_server_fail_admissions(None, 1, None) == q.QAOA_E_INVALID
    assert b"bad" in L.qaoa_last_error() or len(L.qaoa_last_error()) > 0
    assert q.qaoa_workspace_bytes(0) == 0 and q.qaoa_workspace_bytes(31) == 0
    assert q.qaoa_workspace_bytes(30) > q.qaoa_workspace_bytes(20) > 0
