"""libpes builds for sm_103a, loads without a GPU and exports every entry point
that include/pes.h declares; host-side argument checks run without a GPU."""
import os
import re

import pytest

from paper_2101_10881_gb300 import pes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    pes.build()


def declared():
    text = open(os.path.join(ROOT, "include", "pes.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pes_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    L = pes.lib()
    names = declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(pes.EXPORTS)


def test_status_strings():
    L = pes.lib()
    for code in range(8):
        assert L.pes_status_string(code)
    assert b"unknown" in L.pes_status_string(99)


def test_md_costs():
    assert pes.md_costs(10) == (3089.0, 397.0)
    for k in (1, 2, 3, 4, 5, 8):
        m, a = pes.md_costs(k)
        assert m >= a >= 1
    with pytest.raises(pes.PesError):
        pes.md_costs(6)
