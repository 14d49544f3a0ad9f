"""The C-ABI library builds, loads and exports every symbol the header
declares (no GPU needed: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "netsolve.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(net[q]?_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def so():
    from paper_1908_03301_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["net_create", "net_solve", "net_flux", "net_get_pressure", "net_get_labels",
              "net_destroy", "net_solve_batch", "netq_create", "netq_submit", "netq_poll",
              "netq_wait", "netq_cancel", "netq_stats", "netq_destroy", "net_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(so):
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    from paper_1908_03301_gb300 import netsolve as ns

    assert sorted(ns.EXPORTS) == declared_functions()


def test_host_side_validation_without_gpu(so):
    """Descriptor checks happen on the host before any device work."""
    from paper_1908_03301_gb300 import netsolve as ns

    ns._lib = None
    L = ns.lib()
    h = ctypes.c_void_p()
    ptrs = (ctypes.c_void_p * 3)()
    for dims, fa in [((2, 8), 0), ((8, 8), 2), ((0, 8), 0)]:
        d = ns.make_desc(dims, flow_axis=fa)
        assert L.net_create(ctypes.byref(d), ptrs, ctypes.byref(h)) == ns.NET_EINVAL
        assert L.net_last_error()
    # periodic boundaries: only y / z, never the flow axis, extent >= 3,
    # no axis beyond ndim
    for dims, fa, per in [((8, 8), 0, (0,)), ((8, 8), 1, (1,)), ((8, 8), 0, (2,)),
                          ((8, 2), 0, (1,)), ((6, 6, 6), 2, (2,)), ((6, 6, 2), 0, (1, 2))]:
        d = ns.make_desc(dims, flow_axis=fa, periodic=per)
        assert L.net_create(ctypes.byref(d), ptrs, ctypes.byref(h)) == ns.NET_EINVAL, (dims, fa, per)
        assert L.net_last_error()
    d = ns.make_desc((8, 8), p_in=1.0, p_out=1.0)
    assert L.net_create(ctypes.byref(d), ptrs, ctypes.byref(h)) == ns.NET_EINVAL
    assert L.net_solve(None, None, None) == ns.NET_EINVAL
    assert L.net_destroy(None) == ns.NET_OK
    assert L.net_autotune(None, 0, None, None) == ns.NET_EINVAL
    L.net_tune_clear()
    # FBM generator: descriptor checks before any device work
    one = ctypes.c_void_p(16)
    for nd, n, H, beta in [(1, (8, 1, 1), 0.7, (1, 1, 1)), (2, (8, 8, 2), 0.7, (1, 1, 1)),
                           (2, (8, 8, 1), float("nan"), (1, 1, 1)), (2, (8, 8, 1), 0.7, (0, 1, 1)),
                           (3, (8, 8, 0), 0.7, (1, 1, 1))]:
        fd = ns.net_fbm_desc(nd, (ctypes.c_int64 * 3)(*n), H, (ctypes.c_double * 3)(*beta), 0, None)
        assert L.net_fbm_field(ctypes.byref(fd), one, one) == ns.NET_EINVAL
        assert L.net_last_error()


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of net_desc, net_opts, net_result and net_tune have
    the header's field offsets and sizes (compiled with the host C compiler)."""
    from paper_1908_03301_gb300 import netsolve as ns

    structs = {"net_desc": ns.net_desc, "net_opts": ns.net_opts, "net_result": ns.net_result,
               "net_tune": ns.net_tune, "net_fbm_desc": ns.net_fbm_desc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "netsolve.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess

    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        cname, field, val = line.split()
        py = structs[cname]
        expect = ctypes.sizeof(py) if field == "sizeof" else getattr(py, field).offset
        assert int(val) == expect, (cname, field, int(val), expect)
        seen += 1
    assert seen == sum(len(p._fields_) + 1 for p in structs.values())


def test_periodic_plane_sizes_checked_by_binding(so):
    """A periodic axis has one bond per node along it; the binding refuses
    planes of the no-flow size before calling the library."""
    from paper_1908_03301_gb300 import netgen
    from paper_1908_03301_gb300 import netsolve as ns

    assert ns.plane_elems((8, 6), 1, periodic=(1,)) == 48
    assert ns.plane_elems((8, 6), 1) == 40
    assert ns.periodic_mask((1, 2)) == 6
    with pytest.raises(ValueError):
        ns.Network((8, 6), netgen.uniform((8, 6)), periodic=(1,))
