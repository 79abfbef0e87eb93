"""The C-ABI library loads and exports every entry point include/goac.h
declares, and the binding declares a signature for each (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "goac.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(goac_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build_library_only()
    from paper_2409_08808_gb300 import _lib
    names = _declared()
    assert len(names) >= 20
    lib = ctypes.CDLL(_lib.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES)


def test_version_and_error_string():
    from paper_2409_08808_gb300 import _lib
    assert _lib.lib.goac_version() == 100
    assert _lib.lib.goac_last_error() is not None


def test_oracle_shares_no_code_with_the_library():
    """The oracle and the CUDA package do not import or include each other."""
    pkg = os.path.join(ROOT, "paper_2409_08808_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "goac_oracle" not in src, f
    src = open(os.path.join(ROOT, "oracle", "goac_oracle.c")).read() + open(
        os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "import paper_2409_08808_gb300" not in src and "from paper_2409_08808_gb300" not in src
    assert "#include" not in src.replace("#include <math.h>", "").replace("#include <stdint.h>", "").replace(
        "#include <stdlib.h>", "").replace("#include <string.h>", "")


def test_binding_context_and_problem_lifetime_methods():
    """Context and Problem expose close() as methods of the class (a context's
    close destroys its problems first, then the context), and using a closed
    context or problem raises GoacError instead of passing a stale handle."""
    import __graft_entry__
    __graft_entry__.build_library_only()
    import paper_2409_08808_gb300 as g
    for cls in (g.Context, g.Problem):
        assert callable(getattr(cls, "close", None)), cls
        assert callable(getattr(cls, "__del__", None)), cls
    assert isinstance(g.Context.__dict__["closed"], property)
    assert not hasattr(g.launch_count, "close")
    # a context object whose handle is gone behaves as closed (no device needed)
    c = g.Context.__new__(g.Context)
    c._h = None
    c._problems = set()
    assert c.closed
    c.close()                       # closing a closed context is a no-op
    try:
        c.sync_stream()
    except g.GoacError as e:
        assert e.status == -1 and "closed" in str(e)
    else:
        raise AssertionError("a closed context was used")
    p = g.Problem.__new__(g.Problem)
    p._h = None
    p.ctx = c
    p.close()
    try:
        p.handle
    except g.GoacError as e:
        assert "closed" in str(e)
    else:
        raise AssertionError("a closed problem was used")
