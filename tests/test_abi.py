"""CPU-side checks of the C ABI: the library loads and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "lair.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lair_[A-Za-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lair_setup", "lair_solve", "lair_adjoint", "lair_grad_A", "lair_precond_apply",
                     "lair_options_default", "lair_free"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair
    lib = ctypes.CDLL(lair.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_options_defaults_and_status_strings():
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair
    o = lair.options()
    assert o.cf_mode == lair.CF_AUTO and o.distance == 1 and o.theta == 0.25 and o.lump_tol == 1e-3
    assert o.coarse_max == 128 and o.max_levels == 25 and o.rs_block == 4096 and o.fgmres_restart == 30
    assert o.autotune == 1 and o.nodal == 0 and o.restriction == lair.R_LAIR
    assert lair.lib.lair_status_string(0) == b"LAIR_OK"
    assert lair.lib.lair_status_string(13) == b"LAIR_ERR_UNSUPPORTED"


def test_setup_rejects_bad_arguments_without_a_gpu():
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair
    h = ctypes.c_void_p()
    assert lair.lib.lair_setup(None, None, ctypes.byref(h)) == 1
    o = lair.options(distance=5)
    A = lair.lair_csr(4, 4, None, None, None, 0)
    st = lair.lib.lair_setup(ctypes.byref(A), ctypes.byref(o), ctypes.byref(h))
    assert st == 1
    assert b"distance" in lair.lib.lair_last_error(h)
    lair.lib.lair_free(h)


@pytest.mark.parametrize("kw,code,word", [
    (dict(restriction=2), 1, b"restriction"),
    (dict(nodal=-1), 1, b"nodal"),
    (dict(nodal=9), 13, b"nodal"),
    (dict(nodal=6, block_size=6), 1, b"block_size"),
    (dict(nodal=2, restriction=1), 13, b"lAIR"),
    (dict(nodal=3), 1, b"multiple of nodal"),      # n = 4 is not a multiple of 3
    (dict(autotune=2), 1, b"autotune"),
    (dict(wait_polls=-1), 1, b"wait_polls"),
])
def test_setup_rejects_option_combinations_without_a_gpu(kw, code, word):
    """Option checks run before any device call: unknown values, nodal with block scaling or the Neumann
    restriction, and a size that is not a multiple of the node size."""
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair
    h = ctypes.c_void_p()
    o = lair.options(**kw)
    A = lair.lair_csr(4, 4, None, None, None, 0)
    st = lair.lib.lair_setup(ctypes.byref(A), ctypes.byref(o), ctypes.byref(h))
    assert st == code
    assert word in lair.lib.lair_last_error(h)
    lair.lib.lair_free(h)


def test_refresh_rejects_a_handle_without_a_hierarchy():
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair
    lair.lib.lair_refresh.restype = ctypes.c_int
    lair.lib.lair_refresh.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lair.lib.lair_refresh(None, None) == 1
    h = ctypes.c_void_p()
    o = lair.options(distance=5)
    A = lair.lair_csr(4, 4, None, None, None, 0)
    assert lair.lib.lair_setup(ctypes.byref(A), ctypes.byref(o), ctypes.byref(h)) == 1
    val = (ctypes.c_double * 4)()
    assert lair.lib.lair_refresh(h, val) == 1
    assert b"no hierarchy" in lair.lib.lair_last_error(h)
    lair.lib.lair_free(h)


def test_nodal_user_splitting_must_agree_within_nodes():
    """With nodal = k the k unknowns of a node share one label: a user splitting that gives a node's unknowns
    different labels is rejected before any device call, by the library and by the oracle alike."""
    import numpy as np
    import __graft_entry__ as g
    g.build()
    from paper_1708_06065_gb300 import lair
    from oracle import oracle as O
    import workloads as W
    cfu = np.array([1, 1, 0, 0, 1, 0], np.int8)           # node 2 (unknowns 4, 5) disagrees
    h = ctypes.c_void_p()
    o = lair.options(nodal=2, cf_mode=lair.CF_USER)
    o.cf_user = cfu.ctypes.data_as(ctypes.c_void_p).value
    A = lair.lair_csr(6, 6, None, None, None, 0)
    assert lair.lib.lair_setup(ctypes.byref(A), ctypes.byref(o), ctypes.byref(h)) == 1
    assert b"node 2" in lair.lib.lair_last_error(h)
    lair.lib.lair_free(h)
    s = W.upwind_chain(6)
    assert O.Hierarchy(s, cf_user=cfu, nodal=2).status == 1
    cfu[5] = 1
    assert O.Hierarchy(s, cf_user=cfu, nodal=2).status == 0


def test_binding_structs_match_the_header():
    """Every ctypes structure of the binding has the C layout of its header struct: the same size and
    the same offset for every field (compiled with the host C compiler)."""
    import shutil
    import subprocess
    import tempfile
    from paper_1708_06065_gb300 import lair
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"lair_options": lair.lair_options, "lair_report": lair.lair_report,
               "lair_level_info": lair.lair_level_info, "lair_csr": lair.lair_csr}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lair.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'    printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["    return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
