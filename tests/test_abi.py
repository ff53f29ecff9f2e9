"""The C-ABI library loads on a machine without a GPU and exports every entry point of include/ld.h; its
host-side tables and defaults agree with the oracle's independent construction.  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ldmod():
    from paper_1807_02752_gb300 import build, ld
    build.build()
    ld._libs.clear()
    return ld


def test_header_declarations_are_exported(ldmod):
    hdr = open(os.path.join(ROOT, "include", "ld.h")).read()
    declared = sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(ld_\w+)\s*\(", hdr, flags=re.M)))
    assert declared, "no declarations found"
    L = ctypes.CDLL(ldmod.LIB_PATH)
    for name in declared:
        assert hasattr(L, name), f"{name} declared in ld.h but not exported"
    assert sorted(ldmod.EXPORTED) == declared


def test_defaults_match_oracle(ldmod, oracle_mod):
    a = ldmod.default_params().as_dict()
    b = oracle_mod.default_params().as_dict()
    assert a == b


def test_tables_match_oracle(ldmod, oracle_mod):
    for kw in ({}, {"sigma_r": 0.2, "sigma_s": 5.0, "bf_rho": 3}, {"sigma_g": 2.0}, {"wg_gaussian": 1},
               {"wg_gaussian": 1, "sigma_g": 2.0}):
        ws, wr, wg = ldmod.tables(ldmod.default_params(**kw))
        ows, owr, owg = oracle_mod.tables(oracle_mod.default_params(**kw))
        assert (ws == ows).all() and (wr == owr).all() and (wg == owg).all()


def test_n_starts(ldmod, oracle_mod):
    L = ldmod.load()
    p = ldmod.default_params()
    for w in (16, 17, 320, 1241, 1242, 1920):
        assert L.ld_n_starts(ctypes.byref(p), w) == oracle_mod.n_starts(w)


def test_invalid_params_rejected_without_device(ldmod):
    L = ldmod.load()
    h = ctypes.c_void_p()
    for kw in ({"bf_rho": 6}, {"tau_x": 8}, {"n_disp": 300}, {"ransac_hyps": 0}, {"max_lanes": 9}, {"bilateral": 3},
               {"wg_gaussian": 2}, {"thr_abs": 5}, {"dp_literal": 2},
               {"band_literal_bottom": 2}):
        p = ldmod.default_params(**kw)
        assert L.ld_create(ctypes.byref(p), 1242, 375, 4, None, ctypes.byref(h)) == ldmod.E_ARG
        assert h.value is None
        assert L.ld_last_error(None)
    p = ldmod.default_params()
    for size in ((8, 375, 1), (1242, 2000, 1), (1242, 375, 0), (5000, 375, 1)):
        assert L.ld_create(ctypes.byref(p), *size, None, ctypes.byref(h)) == ldmod.E_ARG
    assert L.ld_destroy(None) is None


def test_object_entry_points_reject_null_handles_without_device(ldmod):
    """The network and stereo objects refuse a missing handle before touching the device."""
    L = ldmod.load()
    out = ctypes.c_void_p()
    assert L.ld_net_create(None, 0, ctypes.byref(out)) == ldmod.E_ARG and out.value is None
    assert L.ld_net_last_error(None)
    sp = ldmod.stereo_params()
    assert (sp.rho, sp.tau, sp.d_max, sp.tr_lrc) == (3, 1, -1, 3)
    assert L.ld_stereo_create(None, ctypes.byref(sp), ctypes.byref(out)) == ldmod.E_ARG and out.value is None
    assert L.ld_stereo_last_error(None)
    assert L.ld_net_param_count() == ldmod.NET_PARAMS
    for fn in (L.ld_net_status, L.ld_net_destroy, L.ld_stereo_destroy):
        fn(None)
    assert L.ld_server_set_learned(None, None, 0) == ldmod.E_ARG
    assert L.ld_detect_groups(None, None, 1) == ldmod.E_ARG
    assert ctypes.sizeof(ldmod.Group) == 40


def test_checked_build_loads_and_exports(ldmod):
    """The bounds-checked variant builds from the same sources and exports the same entry points."""
    from paper_1807_02752_gb300 import build
    build.build(checked=True)
    L = ldmod.load(checked=True)
    assert L.ld_checked_build() == 1
    assert ldmod.load().ld_checked_build() == 0
    for name in ldmod.EXPORTED:
        assert hasattr(L, name), f"{name} missing from the checked library"
    assert L.ld_check_site_name(1) == b"selftest" and L.ld_check_site_name(10 ** 6) == b"?"


def test_size_limits_match_header(ldmod):
    hdr = open(os.path.join(ROOT, "include", "ld.h")).read()
    for name, val in (("LD_MAX_W", ldmod.MAX_W), ("LD_MAX_H", ldmod.MAX_H), ("LD_MAX_D", ldmod.MAX_D),
                      ("LD_MAX_LANES", ldmod.MAX_LANES)):
        assert int(re.search(r"#define %s (\d+)" % name, hdr).group(1)) == val, name
