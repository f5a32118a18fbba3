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
