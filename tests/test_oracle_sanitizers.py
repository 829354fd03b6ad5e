"""The oracle under gcc's sanitizers.

The oracle is the authority every GPU output is compared with, so an
out-of-bounds access or undefined operation in it would put wrong expected
values into the parity tests.  This builds the same C sources with
UndefinedBehaviorSanitizer (every report fatal) and, separately, with
AddressSanitizer, and drives every entry point of the oracle through each
build in a child process: games to their end, the environment loop with
auto-reset, a setup pool with mirroring and pinned restarts, replay,
observation planes, legal moves and the brute-force enumerator, perft,
belief marginals and samples, rollouts with both rollout policies, and the
search."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKOUT = r'''
import numpy as np
import oracle

g = oracle.play_games(5, 3)
setups, actions, lengths = g["setups"], g["actions"], g["lengths"]
games = np.array([0, 0, 1, 2, 2], np.int32)
plies = np.array([0, min(50, lengths[0] - 1), min(10, lengths[1] - 1), 0, min(300, lengths[2] - 1)], np.int16)
pos = oracle.replay_positions(setups, actions, games, plies)
u8, bf, mask = oracle.obs_encode(setups, actions, games, plies, player=np.array([-1, 0, 1, -1, 1], np.int8))
for p in pos:
    assert oracle.import_check(p) == 0
    mv = oracle.legal_moves(p)
    assert sorted(oracle.legal_moves(p, physical=True)) == sorted(oracle.brute_moves(p))
    oracle.two_square_applies(p)
    oracle.start_check(p)
    oracle.marginals(p, 0)
    oracle.marginals(p, 1)
    oracle.policy_pick(p, 12345, 67890, magnet=True)
    oracle.policy_pick(p, 12345, 67890, magnet=False)
    if len(mv):
        oracle.apply(p, mv[:1], planes=True)
assert oracle.perft(pos[0], 2) == oracle.perft(pos[0], 2, brute=True)
types = oracle.belief_sample(pos, 8, 3)
oracle.rollout(pos, 8, 24, 7)
oracle.rollout(pos, 8, 24, 7, types=types, want_outcomes=True)
oracle.rollout(pos, 8, 24, 7, flags=oracle.ALL_RULES | oracle.ROLLOUT_MAGNET)
oracle.search(pos[1:3], 2, 8, 11)
oracle.search(pos[1:2], 2, 8, 11, flags=oracle.ALL_RULES | oracle.ROLLOUT_MAGNET,
              pi_theta=np.full((1, 10000), 1e-3, np.float32))
oracle.env_run(3, 4, 400)
pool = np.stack([np.stack([oracle.setup_types(9, m)[40 * s:40 * s + 40] for m in range(3)]) for s in range(2)])
oracle.env_run(4, 3, 300, pool=pool, mirror=True, pins={1: pos[4]}, want_final=True)
oracle.env_run(6, 2, 200, k=200, cap=4000)
bfr, u8r = oracle.ratio_batch(np.arange(1, 50), np.full(49, 7))
print("workout ok")
'''


def _run(tmp_path, flags, env_extra):
    import oracle.build as ob
    out = str(tmp_path / ("liboracle_%s.so" % "_".join(f.strip("-").replace("=", "_") for f in flags)))
    try:
        ob.build(force=True, out=out, extra=flags)
    except subprocess.CalledProcessError as exc:
        pytest.skip("sanitizer build unavailable: %s" % exc)
    env = dict(os.environ, STRATEGO_ORACLE_LIB=out, PYTHONPATH=ROOT, **env_extra)
    r = subprocess.run([sys.executable, "-c", WORKOUT], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=600)
    report = r.stdout + r.stderr
    assert r.returncode == 0 and "workout ok" in r.stdout, report[-4000:]
    assert "runtime error" not in report, report[-4000:]
    assert "ERROR: AddressSanitizer" not in report, report[-4000:]


def test_oracle_under_ubsan(tmp_path):
    _run(tmp_path, ["-fsanitize=undefined", "-fno-sanitize-recover=all", "-g"], {})


def test_oracle_under_asan(tmp_path):
    libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not libasan or not os.path.isabs(libasan) or not os.path.exists(libasan):
        pytest.skip("libasan not found")
    _run(tmp_path, ["-fsanitize=address", "-fno-omit-frame-pointer", "-g"],
         {"LD_PRELOAD": libasan, "ASAN_OPTIONS": "detect_leaks=0:abort_on_error=0"})
