"""The C ABI: libctm.so builds, loads without a GPU and exports every symbol
declared in include/*.h; the binding declares a signature for each of them."""
import glob
import os
import re

from paper_2306_08212_gb300 import build as B
from paper_2306_08212_gb300 import ctm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(ctm_\w+)\s*\(", text, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(ctm.LIB_PATH):
        B.build()
    lib = ctm.load()
    names = declared_symbols()
    assert "ctm_move" in names and "ctm_init_env" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in ctm.SIGNATURES, n


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: a missing libctm.so is an error, not a silent substitute."""
    import pytest
    with pytest.raises(FileNotFoundError):
        ctm.load(str(tmp_path / "libctm.so"))


def test_every_declaration_cites_its_passage_or_says_it_has_none():
    """Each entry point's comment names the section, figure or equation it follows, or
    states that the paper has no counterpart (bookkeeping, measurement, test hooks,
    batching, allocation-free calls)."""
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        for m in re.finditer(r"/\*(.*?)\*/\s*([^;{]*?\b(ctm_\w+)\s*\()", text, flags=re.S):
            comment, name = m.group(1), m.group(3)
            assert re.search(r"Sec\.|Fig\.|Eq\.|Appendix|no counterpart", comment), name
