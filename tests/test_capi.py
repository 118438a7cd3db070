"""The C-ABI library builds and exports every symbol include/kbisim.h declares
(no GPU needed: nothing is called that touches a device)."""
import os
import re

from paper_2204_05821_gb300 import _build, _capi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kbisim.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kb_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    _build.build()
    lib = _capi.load()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(n for n, _, _ in _capi.SIGNATURES)


def test_option_presets_and_status_strings():
    lib = _capi.load()
    o = lib.kb_options_default()
    assert (o.direction, o.use_vertex_labels, o.use_edge_labels, o.early_stop, o.validate) == (0, 1, 1, 1, 1)
    s = lib.kb_options_schaetzle()
    assert (s.direction, s.use_vertex_labels, s.use_edge_labels) == (0, 0, 1)
    k = lib.kb_options_kaushik()
    assert (k.direction, k.use_vertex_labels, k.use_edge_labels) == (1, 1, 0)
    assert lib.kb_status_string(0) == b"ok"
    assert lib.kb_status_string(3) == b"block table full"
