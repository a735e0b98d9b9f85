"""The C-ABI library loads and exports every function include/*.h declares;
host-side validation rejects bad arguments before any CUDA call (CPU only)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return")))


@pytest.fixture(scope="module")
def ngf():
    from paper_1804_10541_b300 import build
    build.build()
    from paper_1804_10541_b300 import ngf as m
    return m


def test_every_declared_symbol_is_exported(ngf):
    decl = _declared_functions()
    assert len(decl) >= 17
    for name in decl:
        assert hasattr(ngf.lib, name), name
    assert sorted(ngf.EXPORTS) == decl


def test_struct_layouts_match_header(ngf, tmp_path):
    """The ctypes mirrors have the size and field offsets the C compiler gives
    the header's structs."""
    import subprocess
    structs = {"ngf_level_desc": ngf.LevelDesc, "ngf_pcg_state": ngf.PcgState, "ngf_options": ngf.Options,
               "ngf_report": ngf.Report, "ngf_pcg_info": ngf.PcgInfo, "ngf_net_desc": ngf.NetDesc}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ngf.h"', '#include "ngf_cnn.h"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


@pytest.mark.parametrize("m,n,tau,rho,alpha,what", [
    ((8, 8, 8), (10, 5, 5), 0.1, 0.1, 1.0, "finer than the image grid"),
    ((8, 8, 8), (1, 5, 5), 0.1, 0.1, 1.0, "nodes n must be >= 2"),
    ((0, 8, 8), (2, 5, 5), 0.1, 0.1, 1.0, "cells m must be >= 1"),
    ((8, 8, 8), (5, 5, 5), 0.0, 0.1, 1.0, "tau and rho"),
    ((8, 8, 8), (5, 5, 5), 0.1, 0.1, -1.0, "alpha"),
])
def test_plan_validation_rejects_before_any_launch(ngf, m, n, tau, rho, alpha, what):
    d = ngf.level_desc(m, (1, 1, 1), n, alpha=alpha, tau=tau, rho=rho)
    h = C.c_void_p()
    st = ngf.lib.ngf_plan_create(C.byref(h), C.byref(d), None)
    assert st == -1 and not h.value
    assert what in ngf.ngf_last_error(None)


def test_null_plan_is_an_error(ngf):
    D, S = C.c_double(), C.c_double()
    assert ngf.lib.ngf_objective(None, None, None, None, C.byref(D), C.byref(S)) == -1
    assert "plan is NULL" in ngf.ngf_last_error(None)
    assert ngf.lib.ngf_plan_destroy(None) == 0


def test_register_multilevel_validates_options(ngf):
    d = ngf.level_desc((8, 8, 8), (1, 1, 1), (5, 5, 5))
    o = ngf.options(levels=0)
    rep = ngf.Report()
    buf = (C.c_float * 512)()
    st = ngf.lib.register_multilevel(C.byref(d), C.byref(o), buf, buf, buf, C.byref(rep), None)
    assert st == -1 and "levels" in ngf.ngf_last_error(None)


def test_size_limit_and_distance_validation(ngf):
    """Rejections that come before any CUDA call: grids past the 2^31 index
    range, an unknown distance, an unknown method, an empty batch."""
    h = C.c_void_p()
    big = ngf.level_desc((2048, 2048, 1024), (1, 1, 1), (65, 65, 33))
    assert ngf.lib.ngf_plan_create(C.byref(h), C.byref(big), None) == -8 and not h.value
    assert "2^31" in ngf.ngf_last_error(None)
    bad = ngf.level_desc((8, 8, 8), (1, 1, 1), (5, 5, 5), distance=3)
    assert ngf.lib.ngf_plan_create(C.byref(h), C.byref(bad), None) == -1
    assert "distance" in ngf.ngf_last_error(None)
    ok = ngf.level_desc((8, 8, 8), (1, 1, 1), (5, 5, 5))
    buf = (C.c_float * 600)()
    rep = ngf.Report()
    opts = ngf.options(2, method=5)
    assert ngf.lib.register_multilevel(C.byref(ok), C.byref(opts), buf, buf, buf, C.byref(rep), None) == -1
    assert "method" in ngf.ngf_last_error(None)
    opts = ngf.options(2, method=ngf.NGF_METHOD_LBFGS, lbfgs_memory=0)
    assert ngf.lib.register_multilevel(C.byref(ok), C.byref(opts), buf, buf, buf, C.byref(rep), None) == -1
    bh = C.c_void_p()
    assert ngf.lib.ngf_batch_create(C.byref(bh), 0, C.byref(ok), 0, None) == -1 and not bh.value


def test_preconditioner_schedule_validation(ngf):
    """A negative refresh interval of the Jacobi diagonal is rejected by the
    single and the batched registration before any CUDA call."""
    ok = ngf.level_desc((8, 8, 8), (1, 1, 1), (5, 5, 5))
    buf = (C.c_float * 600)()
    rep = ngf.Report()
    opts = ngf.options(2, diag_every=-1)
    assert ngf.lib.register_multilevel(C.byref(ok), C.byref(opts), buf, buf, buf, C.byref(rep), None) == -1
    assert "diag_every" in ngf.ngf_last_error(None)
    ptrs = (C.c_void_p * 1)(C.addressof(buf))
    reps = (ngf.Report * 1)()
    assert ngf.lib.register_batch(1, C.byref(ok), C.byref(opts), ptrs, ptrs, ptrs, reps, 0, None) == -1
    assert "diag_every" in ngf.ngf_last_error(None)


def test_tile_depth_and_convolution_validation(ngf):
    """A negative z-chunk length and convolution shapes outside the documented
    limits are rejected before any CUDA call."""
    h = C.c_void_p()
    ok = ngf.level_desc((8, 8, 8), (1, 1, 1), (5, 5, 5))
    assert ngf.lib.ngf_plan_create_ex(C.byref(h), C.byref(ok), -1, None) == -1 and not h.value
    assert "zc" in ngf.ngf_last_error(None)
    buf = (C.c_float * 600)()
    rep = ngf.Report()
    opts = ngf.options(2, zc=-2)
    assert ngf.lib.register_multilevel(C.byref(ok), C.byref(opts), buf, buf, buf, C.byref(rep), None) == -1
    assert "zc" in ngf.ngf_last_error(None)
    conv = ngf.lib.ngf_conv3d_fwd
    for cin, cout in ((8, 16), (80, 16), (16, 8), (16, 24), (16, 272)):
        assert conv(buf, buf, None, buf, 1, 2, 2, 2, cin, cout, 0, None) == -1, (cin, cout)
    assert conv(buf, buf, None, buf, 1, -1, 2, 2, 16, 16, 0, None) == -1
    assert conv(buf, buf, None, buf, 1, 2048, 2048, 1024, 16, 16, 0, None) == -8
    assert conv(None, None, None, None, 1, 0, 4, 4, 16, 16, 0, None) == 0  # empty volume


def test_net_parameter_count_and_validation(ngf):
    """The network's parameter count is the sum over its seven layers of
    27 Cin Cout weights and Cout biases; bad descriptors are refused before
    any CUDA call."""
    d = ngf.net_desc(32, 2, -500.0, 1.0 / 500.0, 5.0)
    layers = [(16, 16), (16, 32), (32, 64), (64, 128), (128, 64), (64, 64), (64, 16)]
    assert ngf.ngf_net_param_count(d) == sum(27 * ci * co + co for ci, co in layers)
    for bad in (ngf.net_desc(12, 1, 0.0, 1.0, 1.0), ngf.net_desc(16, 0, 0.0, 1.0, 1.0),
                ngf.net_desc(16, 1, 0.0, 1.0, 0.0), ngf.net_desc(16, 1, 0.0, 0.0, 1.0)):
        assert ngf.lib.ngf_net_param_count(C.byref(bad)) == -1
        h = C.c_void_p()
        assert ngf.lib.ngf_net_create(C.byref(h), C.byref(bad), None) == -1 and not h.value
