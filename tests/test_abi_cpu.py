"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, and exports every function include/dpso.h declares."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "dpso.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dpso_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1706_04399_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("dpso_cost_matrix", "dpso_init", "dpso_step", "dpso_plan"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(libpath):
    from paper_1706_04399_gb300 import dpso
    p = dpso.default_params()
    assert (p.w, p.phi1, p.phi2, p.mut_period, p.det_frac_pct) == (1.0, 0.4, 0.4, 3, 10)
    assert p.flags == dpso.FLAGS_ALL
    assert dpso.default_cost_params().blocked_penalty_mm == 1_000_000
    assert dpso.status_string(dpso.ERR_RANGE) == "value out of range"


def test_argument_errors_need_no_device(libpath):
    from paper_1706_04399_gb300 import dpso
    L = dpso.lib()
    # rejected before any CUDA call
    assert L.dpso_cost_matrix(None, 10, None, 0, ctypes.byref(dpso.default_cost_params()),
                              None, None) == dpso.ERR_ARG
    assert L.dpso_step(None, 1, None) == dpso.ERR_ARG
    bad = dpso.default_params(swarm=0)
    h = ctypes.c_void_p()
    assert L.dpso_init(ctypes.byref(h), 1, 10, None, ctypes.byref(bad), 1, None) == dpso.ERR_ARG
    big = dpso.default_params(swarm=70000)
    assert L.dpso_init(ctypes.byref(h), 1, 10, None, ctypes.byref(big), 1, None) == dpso.ERR_RANGE
    # the probes check their arguments before touching a device
    g = ctypes.c_double(0.0)
    assert L.dpso_probe_l2_gather_gbs(1024, 4, ctypes.byref(g), None) == dpso.ERR_ARG
    assert L.dpso_probe_l2_gather_gbs(8 << 20, 0, ctypes.byref(g), None) == dpso.ERR_ARG
    assert L.dpso_probe_l2_gather_gbs(8 << 20, 4, None, None) == dpso.ERR_ARG
    assert L.dpso_probe_l2_read_gbs(1024, 4, ctypes.byref(g), None) == dpso.ERR_ARG
    ok = dpso.default_params()
    assert L.dpso_init(ctypes.byref(h), 1, dpso.MAX_N + 1, None, ctypes.byref(ok), 1,
                       None) == dpso.ERR_RANGE


def test_server_host_side_checks(libpath):
    from paper_1706_04399_gb300 import dpso, inputs
    L = dpso.lib()
    sp = dpso.default_server_params()
    assert (sp.memory_budget_bytes, sp.max_active, sp.generations_per_tick, sp.policy,
            sp.lanes) == (0, 64, 8, dpso.SERVE_ARRIVAL_ORDER, 4)
    h = ctypes.c_void_p()
    for bad in (dpso.default_server_params(max_active=0),
                dpso.default_server_params(generations_per_tick=0),
                dpso.default_server_params(policy=2), dpso.default_server_params(lanes=9),
                dpso.default_server_params(lanes=-1)):
        assert L.dpso_server_create(ctypes.byref(h), ctypes.byref(bad)) == dpso.ERR_ARG
    state = ctypes.c_int32(0)
    assert L.dpso_server_poll(None, 1, ctypes.byref(state), None, 0, None, None) == dpso.ERR_ARG
    assert L.dpso_server_wait(None, 1, 0.0, ctypes.byref(state)) == dpso.ERR_ARG
    L.dpso_server_destroy(None)

    # admission footprint: grows with n, swarm and budget; the 2-opt copies count
    inst = inputs.random_instance(200, 3, 1)
    cp = dpso.default_cost_params()

    def fp(n_inst, **kw):
        p = dpso.default_params(swarm=kw.pop("swarm", 64))
        for k, v in kw.items():
            setattr(p, k, v)
        return dpso.dpso_server_footprint(n_inst.xyz, n_inst.boxes, n_inst.tags, cp, p, 1, 50)

    base = fp(inst)
    assert base >= 200 * 224 * 4 + 4 * 200 * 212 * 4 + 3 * 64 * 200 * 2
    assert fp(inputs.random_instance(400, 3, 1)) > 3 * base
    assert fp(inst, swarm=128) > base
    assert fp(inst, flags=dpso.FLAG_DET_INIT) < base - 4 * 200 * 200 * 4
    r, _keep = dpso.make_request(inst.xyz, inst.boxes, inst.tags, cp, dpso.default_params(), 1, 5)
    r.n = 2
    out = ctypes.c_uint64(0)
    assert L.dpso_server_footprint(ctypes.byref(r), ctypes.byref(out)) == dpso.ERR_ARG
    r.n = dpso.MAX_N + 1
    assert L.dpso_server_footprint(ctypes.byref(r), ctypes.byref(out)) == dpso.ERR_RANGE


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the Python binding mirrors has the header's size and field
    offsets (a C program compiled against include/dpso.h prints them)."""
    import shutil
    import subprocess
    from paper_1706_04399_gb300 import dpso
    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [getattr(dpso, name) for name in dir(dpso)
               if name.startswith("dpso_") and isinstance(getattr(dpso, name), type)
               and issubclass(getattr(dpso, name), ctypes.Structure)]
    assert len(structs) >= 9
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dpso.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'printf("{s.__name__} %zu\\n", sizeof({s.__name__}));')
        for f, _ in s._fields_:
            lines.append(f'printf("{s.__name__}.{f} %zu\\n", offsetof({s.__name__}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in
               subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
               if line)
    for s in structs:
        assert int(got[s.__name__]) == ctypes.sizeof(s), s.__name__
        for f, _ in s._fields_:
            assert int(got[f"{s.__name__}.{f}"]) == getattr(s, f).offset, (s.__name__, f)


def test_default_two_opt_shapes(libpath):
    # host-only: the launch shapes used when none is pinned (results never
    # depend on the shape; these pin the documented choice)
    from paper_1706_04399_gb300 import dpso
    shape = dpso.dpso_two_opt_default_shape
    assert shape(200, 1024, 152) == (32, 2, 1)       # short tours: two per CTA
    assert shape(400, 1024, 152) == (32, 1, 2)       # the facade: two tiles in flight
    assert shape(1992, 4096, 152) == (8, 1, 1)       # the bridge: 8-row tiles, two CTAs per SM
    assert shape(1992, 152, 152) == (16, 1, 1)       # too few tours to pair them
    assert shape(1992, 303, 152) == (16, 1, 1)
    assert shape(1992, 304, 152) == (8, 1, 1)
    assert shape(2600, 4096, 152)[0] == 16           # two 8-row tours no longer fit
    assert shape(6600, 10, 152) == (0, 0, 0)         # beyond the tiled kernel
    L = dpso.lib()
    out = dpso.dpso_two_opt_shape()
    assert L.dpso_two_opt_default_shape(2, 1, 152, ctypes.byref(out)) == dpso.ERR_ARG
    assert L.dpso_two_opt_default_shape(400, 1, 0, ctypes.byref(out)) == dpso.ERR_ARG
    assert L.dpso_two_opt_default_shape(400, 1, 152, None) == dpso.ERR_ARG
