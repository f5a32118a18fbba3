"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/ep.h declares, and validates arguments."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_01701_gb300 import build as B
    B.build()
    import paper_2305_01701_gb300 as P
    return P.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:ep_status|const char \*)\s*(ep_\w+)\s*\(", src, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_symbol():
    from paper_2305_01701_gb300 import _native
    bound = {n for n, _, _ in _native.SIGNATURES}
    assert _declared() <= bound


def test_workspace_bytes_and_argument_errors(lib):
    import paper_2305_01701_gb300 as P
    a = P.workspace_bytes(2, (64, 64), P.FP64)
    b = P.workspace_bytes(2, (64, 64), P.FP32_MIXED)
    assert 0 < b < a
    with pytest.raises(P.EPError):
        P.workspace_bytes(4, (1, 1, 1), P.FP64)
    with pytest.raises(P.EPError):
        P.workspace_bytes(2, (0, 4), P.FP64)


def test_layout_of_fields_matches_the_oracle():
    import oracle as O
    from paper_2305_01701_gb300 import _native
    for nd, n in ((2, (5, 3)), (3, (4, 3, 2))):
        for f in _native.FIELDS:
            if nd == 2 and f in ("vz", "uz", "v0z", "tzz", "ezz", "txz", "tyz", "exz", "eyz"):
                continue
            assert _native.field_shape(nd, n, f) == O.field_shape(nd, n, f), f
        assert _native.FIELD_ID == {k: v for k, v in O.FIELD_ID.items() if k in _native.FIELD_ID}


def _c_layout(struct, fields):
    """sizeof and offsetof of a struct of include/ep.h, from a C compiler."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    body = 'printf("%%zu", sizeof(%s));' % struct
    body += "".join('printf(" %%zu", offsetof(%s, %s));' % (struct, f) for f in fields)
    src = ('#include <stddef.h>\n#include <stdio.h>\n#include "ep.h"\n'
           "int main(void) { %s printf(\"\\n\"); return 0; }\n" % body)
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("cls,struct", [("SolverOpts", "ep_solver_opts"), ("SolveInfo", "ep_solve_info")])
def test_binding_structs_match_the_header_layout(cls, struct):
    """The ctypes mirrors of the option and result structs have the C
    compiler's size and field offsets (a field added on one side only, or in
    another order, fails here rather than as garbage on the GPU)."""
    from paper_2305_01701_gb300 import _native
    import ctypes
    S = getattr(_native, cls)
    names = [n for n, _ in S._fields_]
    size, offs = _c_layout(struct, names)
    assert ctypes.sizeof(S) == size
    assert [getattr(S, n).offset for n in names] == offs


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: without libep.so the binding raises instead of
    computing anything."""
    from paper_2305_01701_gb300 import _native
    saved_path, saved_lib = _native.LIB_PATH, _native._lib
    try:
        _native.LIB_PATH = str(tmp_path / "libep.so")
        _native._lib = None
        with pytest.raises(ImportError):
            _native.lib()
        with pytest.raises(ImportError):
            _native.Grid(2, (8, 8))
    finally:
        _native.LIB_PATH, _native._lib = saved_path, saved_lib
