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


def test_build_can_be_called_again(lib):
    """build() stays the package's function after it has run (its compiler
    driver is a submodule of another name), so a process may call it twice,
    as the build step followed by the smoke test does."""
    import paper_2309_08217_gb300 as g
    assert callable(g.build)
    assert g.build() == g.build()
    assert callable(g.build)


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


def test_noalloc_argument_checks_without_device(lib):
    """genga_kick_noalloc rejects bad sizes and parameters on the host,
    before any CUDA call (each case below fails one check)."""
    import paper_2309_08217_gb300 as g
    fake = 0x1000  # never dereferenced: every call is rejected first
    ok = dict(G=2.959122082855911e-4, Mstar=1.0, dt=6.0, precision=g.GENGA_FP64)

    def call(N=100, tau=0.0, **kw):
        p = g.make_params(**{**ok, **kw})
        s = g.genga_system(N, *([fake] * 7), None)
        return lib.genga_kick_noalloc(C.byref(s), C.byref(p), tau, None, None)

    inf, nan = float("inf"), float("nan")
    assert call(N=g.GENGA_NOALLOC_MAX_N + 1) == g.GENGA_ERR_INVALID_ARG
    assert call(N=-1) == g.GENGA_ERR_INVALID_ARG
    assert call(precision=g.GENGA_FP32) == g.GENGA_ERR_INVALID_ARG
    assert call(rcrit_mode=7) == g.GENGA_ERR_INVALID_ARG
    assert call(changeover=5) == g.GENGA_ERR_INVALID_ARG
    assert call(n_big=-2) == g.GENGA_ERR_INVALID_ARG
    assert call(tau=inf) == g.GENGA_ERR_INVALID_ARG
    assert call(tau=nan) == g.GENGA_ERR_INVALID_ARG
    for name in ("G", "Mstar", "dt", "n1", "n2"):
        for bad in (inf, nan):
            assert call(**{name: bad}) == g.GENGA_ERR_INVALID_ARG, (name, bad)
    assert call(G=-1.0) == g.GENGA_ERR_INVALID_ARG
    assert call(Mstar=0.0) == g.GENGA_ERR_INVALID_ARG
    assert call(n1=-1.0) == g.GENGA_ERR_INVALID_ARG
    s = g.genga_system(10, None, *([fake] * 6), None)   # a NULL state array
    p = g.make_params(**ok)
    assert lib.genga_kick_noalloc(C.byref(s), C.byref(p), 0.0, None, None) == g.GENGA_ERR_INVALID_ARG
    assert lib.genga_kick_noalloc(None, C.byref(p), 0.0, None, None) == g.GENGA_ERR_INVALID_ARG
    assert lib.genga_kick_noalloc(C.byref(s), None, 0.0, None, None) == g.GENGA_ERR_INVALID_ARG


def test_variant_info_and_test_hook_without_device(lib):
    import paper_2309_08217_gb300 as g
    kinds = set()
    v = 0
    while True:
        try:
            info = g.genga_kernel_variant_info(v)
        except g.GengaError as e:
            assert e.code == g.GENGA_ERR_INVALID_ARG
            break
        assert info["kind"] in (0, 1) and info["warps"] >= 1 and info["bodies_per_thread"] >= 1
        kinds.add(info["kind"])
        v += 1
    assert kinds == {0, 1}
    with pytest.raises(g.GengaError):
        g.genga_kernel_variant_info(-1)
    assert lib.genga_set_test_waits(None, 20, 1) == g.GENGA_ERR_INVALID_ARG
