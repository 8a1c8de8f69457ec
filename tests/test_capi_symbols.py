"""The C-ABI library loads and exports every function include/eat.h declares (no GPU calls)."""
import ctypes
import os
import re

from paper_1912_00966_gb300 import eat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "eat.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eat_[a-z_]+)\s*\(", text)))


def test_header_declares_the_expected_api():
    names = _declared()
    for n in ("eat_build", "eat_free", "eat_query", "eat_query_batch", "eat_query_batch_multi",
              "eat_workspace_bytes", "eat_next_departure", "eat_get_stats", "eat_net_host_view",
              "eat_last_error", "eat_version"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(eat.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing
    assert set(eat.EXPORTED) >= set(_declared())


def test_version_and_error_string():
    assert eat.eat_version() >= 100
    assert isinstance(eat.eat_last_error(), str)
