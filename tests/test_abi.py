"""The C-ABI library builds, loads and exports every entry point declared in include/*.h
(CPU only: no call here launches device work)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        hdr = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        syms |= set(re.findall(r"\b(bandred_[a-z0-9_]+)\s*\(", hdr))
    return sorted(syms)


@pytest.fixture(scope="module")
def L():
    import paper_1709_00302_gb300 as br

    br.build()
    return br.lib()


def test_every_declared_symbol_is_exported(L):
    syms = declared_symbols()
    assert len(syms) >= 28
    assert "bandred_mlp_loss_grad" in syms
    for s in syms:
        assert hasattr(L, s), s


def test_default_opts_and_status_strings(L):
    import paper_1709_00302_gb300 as br

    o = br.bandred_opts()
    L.bandred_default_opts(ctypes.byref(o))
    assert o.b == 0 and o.lookahead == -1 and o.precision == 0 and o.debug == 0
    assert all(r == 0 for r in o.reserved)
    assert br.bandred_status_string(0) == "success"
    assert "timed out" in br.bandred_status_string(1)
    assert "argument" in br.bandred_status_string(-3)


def test_invalid_arguments_are_rejected_before_any_device_work(L):
    i64 = ctypes.c_int64
    null = ctypes.c_void_p(0)
    # sy2sb: n < 0, w < 1, A missing, lda < n, tau missing
    assert L.bandred_sy2sb_ex(-1, 4, null, 1, null, None, null, 0, null, null) == -1
    assert L.bandred_sy2sb_ex(10, 0, null, 10, null, None, null, 0, null, null) == -2
    assert L.bandred_sy2sb_ex(10, 4, null, 10, null, None, null, 0, null, null) == -3
    fake = ctypes.c_void_p(4096)
    assert L.bandred_sy2sb_ex(10, 4, fake, 9, fake, None, null, 0, null, null) == -4
    assert L.bandred_sy2sb_ex(10, 4, fake, 10, null, None, null, 0, null, null) == -5
    import paper_1709_00302_gb300 as br

    bad = br.bandred_opts()
    L.bandred_default_opts(ctypes.byref(bad))
    bad.b = 5  # b > w
    assert L.bandred_sy2sb_ex(10, 4, fake, 10, fake, ctypes.byref(bad), null, 0, null, null) == -6
    bad.b = 2
    bad.reserved[3] = 1
    assert L.bandred_sy2sb_ex(10, 4, fake, 10, fake, ctypes.byref(bad), null, 0, null, null) == -6
    bad.reserved[3] = 0
    bad.depth = 3  # look-ahead depth beyond 2
    assert L.bandred_sy2sb_ex(10, 4, fake, 10, fake, ctypes.byref(bad), null, 0, null, null) == -6
    # ge2gb: n < 0, w < 1, lda < m (n > m is the wide case: allowed)
    assert L.bandred_ge2gb_ex(4, -5, 1, fake, 4, fake, fake, None, null, 0, null, null) == -2
    assert L.bandred_ge2gb_ex(6, 5, 0, fake, 6, fake, fake, None, null, 0, null, null) == -3
    assert L.bandred_ge2gb_ex(6, 5, 1, fake, 5, fake, fake, None, null, 0, null, null) == -5
    assert L.bandred_ge2gb_ex(6, 5, 1, fake, 6, null, fake, None, null, 0, null, null) == -6
    assert L.bandred_ge2gb_ex(6, 5, 1, fake, 6, fake, null, None, null, 0, null, null) == -7
    # ge2bb: m < 0, n < 0, w < 1, lda < m, tauq / taup missing where reflectors exist
    assert L.bandred_ge2bb_ex(-1, 5, 1, fake, 4, fake, fake, None, null, 0, null, null) == -1
    assert L.bandred_ge2bb_ex(6, -5, 1, fake, 6, fake, fake, None, null, 0, null, null) == -2
    assert L.bandred_ge2bb_ex(6, 5, 0, fake, 6, fake, fake, None, null, 0, null, null) == -3
    assert L.bandred_ge2bb_ex(6, 5, 1, fake, 5, fake, fake, None, null, 0, null, null) == -5
    assert L.bandred_ge2bb_ex(6, 5, 1, fake, 6, null, fake, None, null, 0, null, null) == -6
    assert L.bandred_ge2bb_ex(6, 5, 1, fake, 6, fake, null, None, null, 0, null, null) == -7
    assert L.bandred_ge2bb_ex(6, 5, 6, fake, 6, null, null, None, null, 0, null, null) == -9  # no reflectors
    # second stage: sb2st, sterf, gb2bd, bdsv (argument order, bandwidth limit, workspace)
    unsupported = -1003  # BANDRED_ERR_UNSUPPORTED
    assert L.bandred_sb2st(-1, 4, fake, 1, fake, fake, None, fake, 1 << 20, null, null) == -1
    assert L.bandred_sb2st(10, 0, fake, 10, fake, fake, None, fake, 1 << 20, null, null) == -2
    assert L.bandred_sb2st(10, 129, fake, 10, fake, fake, None, fake, 1 << 20, null, null) == unsupported
    assert L.bandred_sb2st(10, 4, null, 10, fake, fake, None, fake, 1 << 20, null, null) == -3
    assert L.bandred_sb2st(10, 4, fake, 9, fake, fake, None, fake, 1 << 20, null, null) == -4
    assert L.bandred_sb2st(10, 4, fake, 10, null, fake, None, fake, 1 << 20, null, null) == -5
    assert L.bandred_sb2st(10, 4, fake, 10, fake, null, None, fake, 1 << 20, null, null) == -6
    assert L.bandred_sb2st(10, 4, fake, 10, fake, fake, None, null, 1 << 20, null, null) == -8
    assert L.bandred_sb2st(10, 4, fake, 10, fake, fake, None, ctypes.c_void_p(4096 + 16), 1 << 20, null, null) == -8
    assert L.bandred_sb2st(10, 4, fake, 10, fake, fake, None, fake, 8, null, null) == -9
    assert L.bandred_sterf(-1, fake, fake, fake, fake, 1 << 20, null) == -1
    assert L.bandred_sterf(10, null, fake, fake, fake, 1 << 20, null) == -2
    assert L.bandred_sterf(10, fake, null, fake, fake, 1 << 20, null) == -3
    assert L.bandred_sterf(10, fake, fake, null, fake, 1 << 20, null) == -4
    assert L.bandred_sterf(10, fake, fake, fake, null, 1 << 20, null) == -5
    assert L.bandred_sterf(10, fake, fake, fake, fake, 8, null) == -6
    assert L.bandred_gb2bd(-1, 4, fake, 1, fake, fake, None, fake, 1 << 20, null, null) == -1
    assert L.bandred_gb2bd(10, 0, fake, 10, fake, fake, None, fake, 1 << 20, null, null) == -2
    assert L.bandred_gb2bd(10, 129, fake, 10, fake, fake, None, fake, 1 << 20, null, null) == unsupported
    assert L.bandred_gb2bd(10, 4, null, 10, fake, fake, None, fake, 1 << 20, null, null) == -3
    assert L.bandred_gb2bd(10, 4, fake, 9, fake, fake, None, fake, 1 << 20, null, null) == -4
    assert L.bandred_gb2bd(10, 4, fake, 10, null, fake, None, fake, 1 << 20, null, null) == -5
    assert L.bandred_gb2bd(10, 4, fake, 10, fake, null, None, fake, 1 << 20, null, null) == -6
    assert L.bandred_gb2bd(10, 4, fake, 10, fake, fake, None, null, 1 << 20, null, null) == -8
    assert L.bandred_gb2bd(10, 4, fake, 10, fake, fake, None, ctypes.c_void_p(4096 + 16), 1 << 20, null, null) == -8
    assert L.bandred_gb2bd(10, 4, fake, 10, fake, fake, None, fake, 8, null, null) == -9
    assert L.bandred_gb2bd_workspace(10, 129) == 0 and L.bandred_gb2bd_workspace(10, 4) >= 3 * 4 * 10 * 8
    assert L.bandred_bdsv(-1, fake, fake, fake, fake, 1 << 20, null) == -1
    assert L.bandred_bdsv(10, null, fake, fake, fake, 1 << 20, null) == -2
    assert L.bandred_bdsv(10, fake, null, fake, fake, 1 << 20, null) == -3
    assert L.bandred_bdsv(10, fake, fake, null, fake, 1 << 20, null) == -4
    assert L.bandred_bdsv(10, fake, fake, fake, null, 1 << 20, null) == -5
    assert L.bandred_bdsv(10, fake, fake, fake, fake, 8, null) == -6
    assert L.bandred_bdsv_workspace(10) >= L.bandred_sterf_workspace(20)
    # cost model: shape limits, missing pointers
    assert L.bandred_mlp_param_count(8, 32) == 8 * 32 + 32 + 32 * 32 + 3 * 32 + 1 - 32
    assert L.bandred_mlp_param_count(0, 4) == 0 and L.bandred_mlp_param_count(4, 65) == 0
    assert L.bandred_mlp_forward(33, 4, null, null, 0, null, null) == -1
    assert L.bandred_mlp_forward(4, 0, null, null, 0, null, null) == -2
    assert L.bandred_mlp_forward(4, 4, null, null, 0, null, null) == -3
    assert L.bandred_mlp_loss_grad(4, 4, fake, fake, fake, 0, fake, fake, fake, 1 << 20, null) == -6
    assert L.bandred_mlp_loss_grad(4, 4, fake, fake, fake, 10, fake, fake, fake, 8, null) == -9
    assert L.bandred_mlp_adam(4, fake, fake, fake, fake, 0, ctypes.c_float(0.1), ctypes.c_float(0.9),
                              ctypes.c_float(0.999), ctypes.c_float(1e-8), null) == -6


def test_product_path_does_not_import_the_oracle():
    import subprocess
    import sys

    code = ("import sys; import paper_1709_00302_gb300 as br; br.lib(); "
            "assert 'oracle' not in sys.modules, 'oracle imported by the product path'")
    subprocess.run([sys.executable, "-c", code], check=True, cwd=ROOT)


def test_python_opts_struct_mirrors_the_header(L):
    """The binding's bandred_opts has the header's fields, in order, all int, and the same
    size (a layout slip would shift every option the library reads)."""
    import paper_1709_00302_gb300 as br

    hdr = open(os.path.join(ROOT, "include", "bandred.h")).read()
    body = re.search(r"typedef struct bandred_opts \{(.*?)\} bandred_opts;", hdr, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\bint\s+([a-z_]+)(?:\[(\d+)\])?\s*;", body)
    assert [name for name, _ in fields] == [name for name, _ in br.bandred_opts._fields_]
    count = sum(int(n) if n else 1 for _, n in fields)
    assert ctypes.sizeof(br.bandred_opts) == 4 * count
    for (name, n), (pname, ptype) in zip(fields, br.bandred_opts._fields_):
        want = ctypes.c_int * int(n) if n else ctypes.c_int
        assert ctypes.sizeof(ptype) == ctypes.sizeof(want), name


def test_panel_group_is_validated(L):
    import paper_1709_00302_gb300 as br

    fake = ctypes.c_void_p(4096)
    null = ctypes.c_void_p(0)
    for bad_group in (3, 8, -2):
        o = br.make_opts(b=2, panel_group=bad_group)
        assert L.bandred_sy2sb_ex(10, 4, fake, 10, fake, ctypes.byref(o), null, 0, null, null) == -6
