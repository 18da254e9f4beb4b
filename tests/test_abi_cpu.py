"""The C ABI library loads and exports what include/submat.h declares
(no compute calls: this runs without a GPU)."""
import ctypes as C
import glob
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "submat.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2004_10811_gb300 import submat
    return submat.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(submat_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    from paper_2004_10811_gb300 import EXPORTS
    assert sorted(EXPORTS) == names


def test_struct_layouts_match_the_header(lib):
    from paper_2004_10811_gb300.submat import Options, Stats
    src = ('#include "submat.h"\n#include <stdio.h>\n#include <stddef.h>\n'
           'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(submat_options), sizeof(submat_stats),'
           ' offsetof(submat_options, refine_rounds), offsetof(submat_stats, kernel_exec));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "probe")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == C.sizeof(Options)
    assert int(out[1]) == C.sizeof(Stats)
    assert int(out[2]) == Options.refine_rounds.offset
    assert int(out[3]) == Stats.kernel_exec.offset


def test_options_default(lib):
    from paper_2004_10811_gb300.submat import Options
    o = Options()
    o.prec = 7
    lib.submat_options_default(C.byref(o))
    assert o.prec == 0 and o.tol == 0.0 and o.max_iter == 0


def _create(lib, bs, rp, ci, **opts):
    from paper_2004_10811_gb300.submat import Options
    bs = np.ascontiguousarray(bs, np.int32)
    rp = np.ascontiguousarray(rp, np.int64)
    ci = np.ascontiguousarray(ci, np.int32)
    h = C.c_void_p()
    o = Options()
    lib.submat_options_default(C.byref(o))
    for k, v in opts.items():
        setattr(o, k, v)
    st = lib.submat_plan_create(len(bs), bs.ctypes.data_as(C.POINTER(C.c_int32)),
                                rp.ctypes.data_as(C.POINTER(C.c_int64)),
                                ci.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(o), None, C.byref(h))
    return st, lib.submat_last_error().decode()


@pytest.mark.parametrize("bs,rp,ci,what", [
    ([2, 2], [0, 2, 3], [0, 1, 1], "symmetric"),            # (0,1) stored, (1,0) not
    ([2, 2], [0, 1, 2], [0, 2], "out of range"),             # column 2 of 2
    ([2, 2, 2], [0, 2, 4, 5], [1, 0, 0, 1, 2], "increasing"),  # unsorted row 0
    ([2, 2], [0, 1, 2], [1, 0], "diagonal"),                 # no diagonal blocks
])
def test_bad_patterns_rejected_on_host(lib, bs, rp, ci, what):
    st, msg = _create(lib, bs, rp, ci)
    assert st == 2, (st, msg)
    assert what in msg


def test_bad_block_size_rejected(lib):
    st, msg = _create(lib, [2, 0], [0, 1, 2], [0, 1])
    assert st == 1 and "block_sizes" in msg


def test_null_arguments_rejected(lib):
    h = C.c_void_p()
    assert lib.submat_plan_create(0, None, None, None, None, None, C.byref(h)) == 1
    assert lib.submat_sign(None, None, 0.0, None, None) == 1
    assert lib.submat_trace(None, None, None, None) == 1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2004_10811_gb300 import submat
    monkeypatch.setattr(submat, "_lib", None)
    with pytest.raises(submat.SubmatLibraryMissing):
        submat.load(str(tmp_path / "nope.so"))


@pytest.mark.parametrize("opts,status,what", [
    (dict(tile_n_ns=192), 1, "tile widths"),
    (dict(iteration=2), 1, "iteration"),
    (dict(prec=0, iteration=1), 9, "mixed path only"),   # third order: mixed path only
    (dict(prec=1, iteration=1), 9, "mixed path only"),
    (dict(adjoint_mode=2), 1, "adjoint_mode"),
    (dict(prec=0, adjoint_mode=1), 9, "mixed path only"),  # tensor-core adjoint: mixed plans only
])
def test_bad_options_rejected_on_host(lib, opts, status, what):
    st, msg = _create(lib, [2, 2], [0, 2, 4], [0, 1, 0, 1], **opts)
    assert st == status, (st, msg)
    assert what in msg


@pytest.mark.parametrize("groups,what", [
    ([0, 2, 2], "has no block column"),
    ([0, -1, 1], "outside"),
    ([0, 3, 1], "outside"),
])
def test_bad_groups_rejected_on_host(lib, groups, what):
    """Grouped plans (Section IV-C): group ids must be 0 .. ngroups - 1, all
    used; checked on the host before any device allocation."""
    from paper_2004_10811_gb300.submat import Options
    bs = np.ascontiguousarray([2, 2, 2], np.int32)
    rp = np.ascontiguousarray([0, 2, 4, 5], np.int64)
    ci = np.ascontiguousarray([0, 1, 0, 1, 2], np.int32)
    gr = np.ascontiguousarray(groups, np.int32)
    opt = Options()
    lib.submat_options_default(C.byref(opt))
    h = C.c_void_p()
    st = lib.submat_plan_create_grouped(3, bs.ctypes.data_as(C.POINTER(C.c_int32)),
                                        rp.ctypes.data_as(C.POINTER(C.c_int64)),
                                        ci.ctypes.data_as(C.POINTER(C.c_int32)),
                                        gr.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(opt), None, C.byref(h))
    assert st == 1
    assert what in lib.submat_last_error().decode()
