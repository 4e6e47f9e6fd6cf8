"""C-ABI checks that need no GPU: the library loads and exports every
function include/pprpa.h declares, the binding mirrors the header, and host
argument validation returns error codes instead of crashing."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pprpa.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pprpa_[A-Za-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2512_12515_gb300 import _lib

    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pprpa_create", "pprpa_destroy", "pprpa_set_orbitals", "pprpa_set_active",
                     "pprpa_set_ao", "pprpa_set_mo", "pprpa_sigma", "pprpa_diag",
                     "pprpa_build_matrix", "pprpa_solve", "pprpa_grad"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_mirrors_header():
    from paper_2512_12515_gb300 import _lib

    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_error_strings(lib):
    assert lib.pprpa_strerror(0) == b"ok"
    for code in range(-1, -9, -1):
        assert lib.pprpa_strerror(code) != b"unknown error"


def test_null_context_is_an_argument_error(lib):
    assert lib.pprpa_set_orbitals(None, 3, None, None) == -1
    assert lib.pprpa_solve(None, None, None, None, None, None, None) == -1
    lib.pprpa_destroy(None)


def test_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.pprpa_create(ctypes.byref(h), 0, None)
    assert rc in (-1, -2) and not h.value
    assert len(lib.pprpa_last_error()) > 0


def test_options_struct_layout_matches_header(tmp_path):
    """The ctypes mirrors of pprpa_options and pprpa_info have the C header's size and field
    offsets (read from a small C program compiled against include/pprpa.h)."""
    import shutil
    import subprocess

    from paper_2512_12515_gb300 import _lib

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pprpa.h"', "int main(void) {"]
    for cname, cls in (("pprpa_options", _lib.Options), ("pprpa_info", _lib.Info)):
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, cls in (("pprpa_options", _lib.Options), ("pprpa_info", _lib.Info)):
        assert int(got[cname]) == ctypes.sizeof(cls)
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_binding_pair_counts_match_the_oracle_pair_lists():
    import oracle
    from paper_2512_12515_gb300 import _lib

    for no, nv in ((0, 3), (2, 5), (5, 20)):
        for mult in (1, 3):
            nvv, noo = _lib.pair_counts(no, nv, mult)
            assert nvv == len(oracle.pair_list(nv, mult)) and noo == len(oracle.pair_list(no, mult))


def test_binding_refuses_wrong_extents():
    import numpy as np
    import pytest
    from paper_2512_12515_gb300 import _lib

    _lib._need(np.empty((2, 3)), (2, 3), "x")
    with pytest.raises(ValueError):
        _lib._need(np.empty((2, 3)), (3, 2), "x")
    assert _lib._vectors(np.empty(7), 7, "z") == 1
    assert _lib._vectors(np.empty((4, 7)), 7, "z") == 4
    for bad in (np.empty(6), np.empty((4, 6)), np.empty((2, 2, 7))):
        with pytest.raises(ValueError):
            _lib._vectors(bad, 7, "z")
