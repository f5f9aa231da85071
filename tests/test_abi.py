"""The C-ABI library loads and exports every symbol include/rambo.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

from paper_1910_04358_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def _declared():
    names = set()
    for f in os.listdir(HEADER):
        if f.endswith(".h"):
            text = open(os.path.join(HEADER, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rambo_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_builds_and_exports_header_symbols():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert {"rambo_create", "rambo_query_seqs", "rambo_query_kmers", "rambo_insert"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_needs_no_device():
    lib = ctypes.CDLL(build.build())
    lib.rambo_strerror.restype = ctypes.c_char_p
    assert lib.rambo_strerror(0) == b"ok"
    assert lib.rambo_strerror(-4) == b"document id out of range"
    lib.rambo_mask_words.restype = ctypes.c_uint32
    assert lib.rambo_mask_words(None) == 0
