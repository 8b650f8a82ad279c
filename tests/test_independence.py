"""The oracle and the CUDA product share no code and neither uses the other:
the package and its C sources never name the oracle, and the oracle's C
file includes only its own header and the C library.  Only the tests, the
smoke check and the bench's CPU legs load the oracle."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2302_07499_gb300")


def _sources(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_never_names_the_oracle():
    files = list(_sources(PKG, (".py", ".cu", ".cuh", ".h"))) + list(_sources(os.path.join(ROOT, "include"), (".h",)))
    assert files
    for f in files:
        assert not re.search(r"\boracle\b|liboracle|nl_oracle", open(f).read(), re.I), f


def test_oracle_includes_only_its_header_and_libc():
    src = open(os.path.join(ROOT, "oracle", "nl_oracle.c")).read()
    local = re.findall(r'#include\s+"([^"]+)"', src)
    assert local == ["nl_oracle.h"]
    system = set(re.findall(r"#include\s+<([^>]+)>", src))
    assert not {h for h in system if "cuda" in h or h.startswith("nl")}
    py = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_2302_07499_gb300" not in py and "libnlfem" not in py


def test_oracle_loaded_only_by_tests_smoke_and_bench():
    for f in _sources(ROOT, (".py",)):
        rel = os.path.relpath(f, ROOT)
        if rel.startswith(("tests" + os.sep, "oracle" + os.sep, "_work" + os.sep, "baseline" + os.sep)):
            continue
        if re.search(r"^\s*(import oracle|from oracle)", open(f).read(), re.M):
            assert rel in ("bench.py", "__graft_entry__.py"), rel
