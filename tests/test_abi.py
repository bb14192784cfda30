"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol include/combsieve.h declares, and rejects the same parameter sets
as the oracle before touching the device."""
import os
import re

import pytest

import oracle.oracle as O
import paper_2012_03771_gb300 as cs
from paper_2012_03771_gb300 import workloads
from tests.conftest import ROOT


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cs_\w+)\s*\(", text, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2012_03771_gb300 import build
    build.build()
    return cs.load()


def test_header_declares_exports(lib):
    declared = _declared()
    assert declared, "no declarations parsed"
    assert declared == set(cs.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_rejections_match_oracle(lib):
    seen = 0
    for prm in workloads.tiny_cases(200):
        rc = cs.cs_plan_status(*prm.as_tuple())
        bad = O.validate(*prm.as_tuple()) != 0
        assert (rc == cs.CS_EINVAL) == bad, (prm, rc, cs.cs_last_error())
        seen += bad
    assert seen > 5
    for args in ((503, 4, 1, 10, 100, 10**6), (7, 11, 1, 10, 100, 10**6), (503, 210, 0, 10, 100, 10**6),
                 (1, 1, 5, 10, 4, 100), (503, 210, 1, 10, 100, 2**40 + 1), (503, 210, 1, 10, 2**20 + 1, 10**6),
                 (503, 0, 1, 10, 100, 10**6), (503, 210, 1, 2**31, 100, 10**6)):
        assert cs.cs_plan_status(*args) == cs.CS_EINVAL
        assert O.validate(*args) == O.EINVAL


def test_bad_tuning_rejected(lib):
    t = cs.make_tuning(threshold=100)          # below 2*SL
    assert cs.cs_plan_status(503, 210, 1, 10, 1000, 10**6, t) == cs.CS_EINVAL
    t = cs.make_tuning(tile_rows=3)
    assert cs.cs_plan_status(503, 210, 1, 10, 1000, 10**6, t) in (cs.CS_EINVAL, cs.CS_EDEVICE)


def test_bad_walk_and_layout_knobs_rejected(lib):
    for kw in (dict(m_classes=4), dict(layout=2)):
        t = cs.make_tuning(**kw)
        assert cs.cs_plan_status(503, 210, 1, 10, 1000, 10**6, t) == cs.CS_EINVAL, kw


def test_environment_knobs_reach_the_plan(lib, monkeypatch):
    """Tuning fields left at 0 are read from the environment when a plan is made: an
    out-of-range value set only there is rejected like the same value in the struct."""
    args = (503, 210, 1, 10, 1000, 10**6)
    for name, bad in (("CS_M_CLASSES", "4"), ("CS_THRESHOLD", "100")):
        monkeypatch.setenv(name, bad)
        assert cs.cs_plan_status(*args, cs.make_tuning()) == cs.CS_EINVAL, name
        monkeypatch.delenv(name)
    # a value given in the struct wins over the environment: the plan gets past the
    # knob checks (and, without a GPU, stops at the first device call)
    monkeypatch.setenv("CS_M_CLASSES", "4")
    assert cs.cs_plan_status(*args, cs.make_tuning(m_classes=1)) != cs.CS_EINVAL
    monkeypatch.delenv("CS_M_CLASSES")


def _header_struct(name):
    """(type, field) pairs of `typedef struct { ... } name;` in the header, arrays as (type, field[n])."""
    text = open(os.path.join(ROOT, "include", "combsieve.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    return re.findall(r"(uint\d+_t)\s+(\w+(?:\[\d+\])?)\s*;", m.group(1))


@pytest.mark.parametrize("name, cls", [("cs_tuning", "cs_tuning"), ("cs_info_t", "cs_info_t"),
                                       ("cs_stats_t", "cs_stats_t")])
def test_binding_structs_match_header(name, cls):
    """The ctypes mirrors of the ABI structs have the header's fields, in order and with the
    same widths, so that the library and the binding agree on every offset."""
    import ctypes
    import paper_2012_03771_gb300._binding as b
    want = _header_struct(name)
    got = getattr(b, cls)._fields_
    assert len(got) == len(want), (name, got, want)
    width = {"uint32_t": 4, "uint64_t": 8}
    for (ctype, field), (gname, gtype) in zip(want, got):
        base = field.split("[")[0]
        n = int(field.split("[")[1][:-1]) if "[" in field else 1
        assert gname == base, (name, gname, base)
        assert ctypes.sizeof(gtype) == width[ctype] * n, (name, base)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2012_03771_gb300._binding as b
    monkeypatch.setattr(b, "_lib", None)
    with pytest.raises(ImportError):
        b.load(str(tmp_path / "nope.so"))


def test_null_arguments(lib):
    import ctypes
    assert lib.cs_plan(503, 210, 1, 10, 100, 10**6, None, None) == cs.CS_EINVAL
    assert lib.cs_sieve(None, None) == cs.CS_EINVAL
    assert lib.cs_destroy(None) == cs.CS_OK
    assert lib.cs_info(None, None) == cs.CS_EINVAL
    h = ctypes.c_uint64(0)
    assert lib.cs_primes(10, 2**41, None, 0, ctypes.byref(h), None) == cs.CS_EINVAL
