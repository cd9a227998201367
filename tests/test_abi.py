"""The C-ABI library builds, loads and exports every entry point that
include/sem.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sem.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"SEM_API\s+[\w\s\*]+?\b(sem_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib_path():
    import paper_2207_07098_gb300 as P
    return P.build()


def test_header_declares_entry_points():
    names = _declared()
    for required in ("sem_setup", "sem_ax", "sem_gs", "sem_cg_solve", "sem_destroy", "sem_setup_batch",
                     "sem_cg_solve_batch", "sem_dot", "sem_mass"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_header(lib_path):
    import paper_2207_07098_gb300 as P
    P.load(lib_path)
    assert set(_declared()) == set(P.exported_symbols())


def test_no_oracle_in_product_path():
    """The product package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2207_07098_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt and "sem_oracle" not in txt, f
