"""The C-ABI library builds and exports every symbol include/kbisim.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
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
    assert o.rekey_all == 0 and o.reorder == 0 and o.subject == 0
    assert lib.kb_status_string(0) == b"ok"
    assert lib.kb_status_string(3) == b"block table full"


C_SIZES = {"int64_t": 8, "int32_t": 4, "uint64_t": 8, "uint32_t": 4, "float": 4, "double": 8, "size_t": 8}


def header_structs():
    """{typedef name: [(field, bytes)]} for the plain structs of the header."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(kb_[a-z_]+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(?:const )?([a-z_0-9]+)\s*(\*?)\s*(.+)$", decl)
            assert m, decl
            ctype, ptr, names = m.groups()
            for item in names.split(","):
                n = re.match(r"\s*([a-z_0-9]+)(?:\[(\d+)\])?\s*$", item)
                assert n, decl
                size = 8 if ptr else C_SIZES[ctype]
                fields.append((n.group(1), size * int(n.group(2) or 1)))
        out[name] = fields
    return out


def test_ctypes_structs_match_the_header():
    structs = header_structs()
    pairs = {"kb_graph": _capi.KbGraph, "kb_options": _capi.KbOptions,
             "kb_server_config": _capi.KbServerConfig, "kb_server_stats": _capi.KbServerStats,
             "kb_tuning": _capi.KbTuning, "kb_prepared_info": _capi.KbPreparedInfo}
    assert set(pairs) <= set(structs)
    for cname, py in pairs.items():
        want = structs[cname]
        got = [(name, ctypes.sizeof(t)) for name, t in py._fields_]
        assert got == want, (cname, got, want)
        assert ctypes.sizeof(py) == sum(sz for _, sz in want), cname
