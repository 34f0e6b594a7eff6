"""The C ABI library: builds, loads, exports every declared entry point, and
checks its host-side arguments without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include"))
           if h.endswith(".h")]


def _declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(sss_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2606_27604_b300 import build as b
    b.build()
    from paper_2606_27604_b300 import api
    return api


def test_header_declares_the_walk_calls():
    names = _declared_functions()
    for f in ("sss_walk", "sss_walk_bwd", "sss_walk_workspace_size", "sss_read_status",
              "sss_status_string"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    raw = C.CDLL(lib.LIB_PATH)
    missing = [f for f in _declared_functions() if not hasattr(raw, f)]
    assert not missing, missing


def test_defaults_and_sizes(lib):
    o = lib.Opts()
    lib.lib.sss_walk_opts_default(C.byref(o))
    assert o.nbins == 64 and abs(o.r_max_mm - 10.0) < 1e-6 and o.max_steps == 65536
    assert o.entry_fresnel == 1 and o.want_sumsq == 1 and o.mode == 0
    assert lib.tally_count(64, 3, 1) == 64 + 6 + 3 + 65
    assert lib.tally_count(32, 3, 0) == 32 + 6 + 3
    assert lib.abi_version() == 3
    # workspace size: header + accumulators, with a prefix table for uneven budgets
    p = lib.Params(C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), None,
                   4096, None, 1.4, 3, 1000)
    n1 = lib.lib.sss_walk_workspace_size(C.byref(p), C.byref(o))
    assert n1 >= 256 + 1000 * lib.tally_count(64, 3, 1) * 8
    p.n_paths = C.c_void_p(512)
    n2 = lib.lib.sss_walk_workspace_size(C.byref(p), C.byref(o))
    assert n2 >= n1 + 1001 * 8
    nb = lib.lib.sss_walk_bwd_workspace_size(C.byref(p), C.byref(o))
    assert nb >= 4 * 3 * 1000 * 8


def test_host_side_argument_errors(lib):
    o = lib.Opts()
    lib.lib.sss_walk_opts_default(C.byref(o))
    ok = lib.Params(C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), None,
                    16, None, 1.0, 3, 10)
    t = lib.Tallies()
    bad_cases = []
    p = lib.Params.from_buffer_copy(ok); p.K = 0; bad_cases.append((p, o))
    p = lib.Params.from_buffer_copy(ok); p.K = 5; bad_cases.append((p, o))
    p = lib.Params.from_buffer_copy(ok); p.alpha = None; bad_cases.append((p, o))
    p = lib.Params.from_buffer_copy(ok); p.alpha = C.c_void_p(258); bad_cases.append((p, o))
    p = lib.Params.from_buffer_copy(ok); p.n_rel = 0.5; bad_cases.append((p, o))
    for field, val in (("nbins", 0), ("nbins", 5000), ("r_max_mm", -1.0), ("mode", 3),
                       ("max_steps", 0), ("schedule", 7), ("block_threads", 48),
                       ("regroup", 33)):
        oo = lib.Opts.from_buffer_copy(o)
        setattr(oo, field, val)
        bad_cases.append((ok, oo))
    for p, oo in bad_cases:
        assert lib.lib.sss_walk_workspace_size(C.byref(p), C.byref(oo)) == 0
        rc = lib.lib.sss_walk(C.byref(p), C.byref(oo), C.c_void_p(4096), 1 << 30, C.byref(t),
                              None)
        assert rc == 1, (rc, field)
    # misaligned or missing workspace, too small workspace
    assert lib.lib.sss_walk(C.byref(ok), C.byref(o), None, 1 << 30, C.byref(t), None) == 1
    assert lib.lib.sss_walk(C.byref(ok), C.byref(o), C.c_void_p(4100), 1 << 30, C.byref(t),
                            None) == 1
    assert lib.lib.sss_walk(C.byref(ok), C.byref(o), C.c_void_p(4096), 16, C.byref(t),
                            None) == 3
    assert lib.lib.sss_walk_bwd(C.byref(ok), C.byref(o), C.c_void_p(4096), 1 << 30, None,
                                None, None) == 1
    for code in range(8):
        assert lib.lib.sss_status_string(code)


def test_no_device_is_reported_not_hidden(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    o = lib.Opts()
    lib.lib.sss_walk_opts_default(C.byref(o))
    p = lib.Params(C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), None,
                   16, None, 1.0, 3, 10)
    t = lib.Tallies()
    rc = lib.lib.sss_walk(C.byref(p), C.byref(o), C.c_void_p(4096), 1 << 30, C.byref(t), None)
    assert rc == 7  # SSS_ERR_UNSUPPORTED: no sm_103a device, nothing computed elsewhere
