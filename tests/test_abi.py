"""The C ABI without a GPU: the library loads, exports every symbol that
include/genga.h declares, and rejects bad arguments on the host before
touching a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def lib():
    import paper_2309_08217_gb300 as g
    g.build()
    return g.load()


def declared_functions():
    names = []
    for h in sorted(os.listdir(HEADER_DIR)):
        if h.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(genga_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("genga_create", "genga_destroy", "genga_kick", "genga_drift", "genga_encounters",
                     "genga_step", "genga_energy", "genga_get_status", "genga_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_status_strings(lib):
    import paper_2309_08217_gb300 as g
    for code in range(8):
        assert len(g.genga_status_string(code)) > 0
        assert g.genga_status_string(code) != "unknown status"
    assert g.genga_status_string(99) == "unknown status"


def _struct_fields(name):
    text = open(os.path.join(HEADER_DIR, "genga.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", text).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        names = decl.split(None, 1)[1]
        fields += [n.strip().lstrip("*") for n in names.split(",")]
    return fields


def test_binding_structs_match_the_header():
    import paper_2309_08217_gb300 as g
    assert [f[0] for f in g.genga_params._fields_] == _struct_fields("genga_params")
    assert [f[0] for f in g.genga_system._fields_] == _struct_fields("genga_system")


def test_host_argument_checks_without_device(lib):
    import paper_2309_08217_gb300 as g
    p = g.make_params(G=1.0)
    sysc = g.genga_system(0, None, None, None, None, None, None, None)
    # NULL context / system / params are rejected on the host
    assert lib.genga_kick(None, C.byref(sysc), C.byref(p), 0.0, None, None) == g.GENGA_ERR_INVALID_ARG
    assert lib.genga_drift(None, C.byref(sysc), C.byref(p), 1.0, None) == g.GENGA_ERR_INVALID_ARG
    assert lib.genga_step(None, C.byref(sysc), C.byref(p), 1, None) == g.GENGA_ERR_INVALID_ARG
    assert lib.genga_encounters(None, C.byref(sysc), C.byref(p), None, 0, None, None) == g.GENGA_ERR_INVALID_ARG
    assert lib.genga_last_encounters(None, None, 0, None, None) == g.GENGA_ERR_INVALID_ARG
    assert lib.genga_get_status(None, None) == g.GENGA_ERR_INVALID_ARG
    h = C.c_void_p()
    assert lib.genga_create(None, 10, 0) == g.GENGA_ERR_INVALID_ARG
    assert lib.genga_create(C.byref(h), -1, 0) == g.GENGA_ERR_INVALID_ARG
    lib.genga_destroy(None)                                   # no-op
