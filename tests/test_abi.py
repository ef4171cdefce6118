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
