"""CPU checks of the CUDA library: it builds for sm_103a, loads, and exports
every entry point that include/stratego.h declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "stratego.h")).read()
    return sorted(set(re.findall(r"^(?:st_status|const char\*)\s+(st_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("st_env_create", "st_env_destroy", "st_env_reset", "st_env_step", "st_env_run",
                     "st_env_export", "st_env_import", "st_obs_encode", "st_belief_sample", "st_rollout",
                     "st_last_error"):
        assert required in names


def test_library_builds_and_exports_all_symbols():
    from paper_2511_07312_gb300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(st_\w+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n)
    lib.st_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.st_version()


def test_argument_errors_are_reported_without_a_gpu():
    import paper_2511_07312_gb300 as st
    L = st.lib()
    cfg = st.st_env_config(0, 1, st.make_rules(), 0, 0, None)
    h = ctypes.c_void_p()
    assert L.st_env_create(ctypes.byref(cfg), ctypes.byref(h)) == 1      # num_games 0 -> ST_ERR_INVALID
    assert b"num_games" in L.st_last_error()
    bad = st.st_env_config(8, 1, st.make_rules(k=0), 0, 0, None)
    assert L.st_env_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    # st_search: sizes and coefficients are checked before anything is enqueued
    r = st.make_rules()
    nulls = [None] * 7
    for P, S, depth, alpha, beta, what in ((1, 4, 0, 0.002, 0.02, b"depth"), (1, -1, 4, 0.002, 0.02, b"S must"),
                                           (70000, 4, 4, 0.002, 0.02, b"P must"), (1, 4, 4, 0.0, 0.0, b"alpha"),
                                           (1, 4, 4, -1.0, 0.5, b"alpha")):
        assert L.st_search(None, P, S, depth, 1, None, None, None, alpha, beta, ctypes.byref(r), *nulls, None) == 1
        assert what in L.st_last_error()
    assert L.st_search(None, 0, 4, 4, 1, None, None, None, 0.002, 0.02, ctypes.byref(r), *nulls, None) == 0
    # the rollout-policy bit is for rollouts only: the env refuses it
    magnet = st.st_env_config(8, 1, st.make_rules(flags=st.RULES_ALL | st.ROLLOUT_MAGNET), 0, 0, None)
    assert L.st_env_create(ctypes.byref(magnet), ctypes.byref(h)) == 1
    # env configuration calls check their arguments before touching the env
    assert L.st_env_set_setup_pool(None, None, 0, 0) == 1
    assert L.st_env_pin(None, None, 0, None) == 1
    assert L.st_env_enable_history(None, 10) == 1
    assert L.st_env_history_positions(None, 0, None, None, None, None) == 1
    assert L.st_positions_mask(None, 1, ctypes.byref(st.make_rules(k=0)), None, None, None, None, None) == 1
