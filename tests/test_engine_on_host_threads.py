"""The CUDA kernels' source run on host threads under sanitizers.

compute-sanitizer is not available to this project, so the device code of
the env (csrc/engine.cuh; the reset, pin, plain, persistent and recording
step, history-position, history-record and export kernels of csrc/env.cu), of the observation planes (k_replay, k_obs_emit), of the
belief samples and rollouts (k_belief, k_roots, k_draw_samples,
k_rollout_flat), of the snapshot masks (k_positions_mask), of a serving
batch (k_serve_roots, k_serve_rollouts) and of the search
(k_search_prep, k_search_offsets, k_search_rollouts, k_search_policy) is
also compiled with g++ against a host stand-in for the CUDA features it uses
(tests/simt_host: one std::thread per lane, warp collectives as rendezvous
of the lanes in their mask, block barriers, per-block static shared
variables, bulk copies performed at their wait) and run under
ThreadSanitizer and under AddressSanitizer with UndefinedBehaviorSanitizer.
Every output must equal the oracle's.  Only the bulk-copy inline assembly
and the shared-memory declarations are rewritten for the host.

Any sanitizer report fails the test.  A planted missing team barrier must
be reported."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_07312_gb300", "csrc")
HARNESS = os.path.join(ROOT, "tests", "simt_host")


def _host_source(text):
    """The CUDA source with its shared-memory declarations and its bulk-copy
    inline assembly replaced by the harness's host equivalents."""
    text = text.replace("extern __shared__ __align__(16) unsigned char smem[];",
                        "unsigned char* const smem = emu::block_smem();")
    # a static __shared__ variable becomes a reference to the block's object
    text = re.sub(r"(?<!extern )__shared__\s+([A-Za-z_][\w ]*?)\s+([A-Za-z_]\w*)((?:\[[^\]]+\])*)\s*;",
                  lambda m: "auto& %s = *emu::block_static<%s%s>(__LINE__);" % (m.group(2), m.group(1), m.group(3)),
                  text)
    # the persistent step's bulk copy of a mask staging buffer and its waits
    text = text.replace('asm volatile("fence.proxy.async.shared::cta;" ::: "memory");', ";")
    text = re.sub(r'const uint32_t src = static_cast<uint32_t>\(__cvta_generic_to_shared\(staged\)\);\s*'
                  r'asm volatile\("cp\.async\.bulk\.global\.shared::cta\.bulk_group \[%0\], \[%1\], %2;"\s*'
                  r'::\s*"l"\(dst\), "r"\(src\), "r"\(\(uint32_t\)kMaskBytes\) : "memory"\);\s*'
                  r'asm volatile\("cp\.async\.bulk\.commit_group;" ::: "memory"\);',
                  "emu::bulk_copy(dst, staged, kMaskBytes);", text)
    text = text.replace('asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");', "emu::bulk_wait();")
    text = text.replace('asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");', "emu::bulk_wait();")
    assert "asm" not in re.sub(r"//.*", "", text), "inline assembly the harness does not know"
    return text


def _device_part(name):
    """The kernels of a .cu file without its C entry points: env.cu up to its
    host helpers (env_args onwards), obs.cu and search.cu up to their first
    extern "C" function."""
    text = open(os.path.join(CSRC, name)).read().replace('#include "host_common.h"', '#include "stratego.h"')
    lines = text.split("\n")
    keep = lambda l: True
    if name == "env.cu":
        start = next(i for i, l in enumerate(lines) if l.startswith("namespace {"))
        end = next(i for i, l in enumerate(lines) if l.startswith("EnvArgs env_args("))
        pre = [l for l in lines[:start] if (l.startswith("#include") or l.startswith("using namespace")) and keep(l)]
        return "\n".join(pre + lines[start:end]) + "\n}  // namespace\n"
    if name == "serve.cu":   # the kernels' namespace only (the server's host state follows)
        end = next(i for i, l in enumerate(lines) if l.startswith("}  // namespace")) + 1
    else:
        end = next(i for i, l in enumerate(lines) if l.startswith('extern "C"'))
    return "\n".join(l for l in lines[:end] if keep(l)) + "\n"


def _prepare(dst, edit=None):
    for f in ("engine.cuh", "snapshot.cuh", "rollout.cuh", "features.cuh"):
        text = _host_source(open(os.path.join(CSRC, f)).read())
        if edit is not None:
            text = edit(f, text)
        with open(os.path.join(dst, f), "w") as o:
            o.write(text)
    for f, dev in (("env.cu", "env_dev.cu"), ("obs.cu", "obs_dev.cu"), ("search.cu", "search_dev.cu"),
                   ("serve.cu", "serve_dev.cu")):
        with open(os.path.join(dst, dev), "w") as o:
            o.write(_host_source(_device_part(f)))


def _build(tmp, flags, name, edit=None, driver="env_on_host.cpp"):
    src = os.path.join(tmp, "src")
    os.makedirs(src, exist_ok=True)
    _prepare(src, edit)
    exe = os.path.join(tmp, name)
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-pthread", "-w", "-I", os.path.join(HARNESS, "include"),
           "-I", src, "-I", os.path.join(ROOT, "include"), os.path.join(HARNESS, driver), "-o", exe] + flags
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        if "sanitize" in r.stderr or "cannot find" in r.stderr:
            pytest.skip("sanitizer runtime unavailable: %s" % r.stderr[-300:])
        raise AssertionError(r.stderr[-4000:])
    return exe


def _line_of(src_dir, name, text, after=None):
    """1-based line of `text` in the prepared file `name` (the first one
    after the line containing `after`, if given)."""
    lines = open(os.path.join(src_dir, name)).read().split("\n")
    start = 0 if after is None else next(i for i, l in enumerate(lines) if after in l)
    return "%s:%d" % (name, next(i for i in range(start, len(lines)) if text in lines[i]) + 1)


def _check_report(r, known=()):
    """No sanitizer report other than the races listed in `known` (pairs of
    the two accesses' innermost file:line); the kernels' own runs list none."""
    report = r.stdout + r.stderr
    if r.returncode != 0 and "FATAL: ThreadSanitizer" in report and "memory" in report:
        pytest.skip("ThreadSanitizer cannot start here: %s" % report[-300:])
    assert "runtime error" not in report and "ERROR: AddressSanitizer" not in report, report[-6000:]
    # collectives: lanes of one mask always meet at the same kind of
    # collective from the same source line
    assert "EMU FAILURE" not in report and "EMU WARNING" not in report, report[-6000:]
    races = report.split("WARNING: ThreadSanitizer: data race")[1:]
    for block in races:
        tops = re.findall(r"(?:Read|Write|read|write) of size \d+ at .*?\n\s+#0 \S+ .*?([\w.]+\.(?:cuh|cu|cpp|h):\d+)",
                          block)
        assert tuple(sorted(tops)) in set(known), "unexpected data race:" + block[:5000]
    assert r.returncode == (66 if races else 0), report[-6000:]
    return report


def _run_and_compare(exe, tmp, N, S, L, wpb, gpf, blocks, seed, env=None):
    out = os.path.join(tmp, "o_%d_%d_%d_%d" % (L, wpb, gpf, blocks))
    r = subprocess.run([exe, str(N), str(S), str(L), str(wpb), str(gpf), str(blocks), str(seed), out],
                       capture_output=True, text=True, timeout=900, env=dict(os.environ, **(env or {})))
    report = _check_report(r)
    assert "status 0 " in r.stdout, report[-2000:]
    ref = oracle.env_run(seed, N, S)
    for k, dt in (("action", np.int16), ("reward", np.int8), ("done", np.uint8), ("ply", np.int16)):
        got = np.fromfile(out + "." + k, dtype=dt).reshape(S, N)
        bad = np.argwhere(got != ref[k])
        assert bad.size == 0, "%s differs first at (ply, slot) %s" % (k, bad[0])
    mask = np.fromfile(out + ".mask", dtype=np.uint8).reshape(S, N, oracle.MASK_BYTES)
    bad = np.argwhere((mask != ref["mask"]).any(-1))
    assert bad.size == 0, "mask differs first at (ply, slot) %s" % bad[0]
    stats = np.fromfile(out + ".stats", dtype=np.uint32).reshape(N, 8)
    np.testing.assert_array_equal(stats, ref["stats"])


@pytest.fixture(scope="module")
def built(tmp_path_factory):
    """build(driver, flags) -> (executable, prepared source dir), each
    (driver, flags) pair compiled once per test module."""
    cache = {}

    def get(driver, flags):
        key = (driver, tuple(flags))
        if key not in cache:
            tmp = str(tmp_path_factory.mktemp(driver.split(".")[0]))
            cache[key] = (_build(tmp, list(flags), "exe", driver=driver), os.path.join(tmp, "src"))
        return cache[key]
    return get


@pytest.fixture(scope="module")
def tsan_exe(built):
    exe, src = built("env_on_host.cpp", ["-fsanitize=thread"])
    return exe, os.path.dirname(src)


@pytest.mark.parametrize("L,wpb,gpf,blocks,nsplit", [(8, 1, 1, 1, 1), (4, 1, 2, 1, 2), (16, 2, 1, 2, 1),
                                                      (32, 2, 1, 1, 3), (8, 1, 2, 1, 2)])
def test_step_kernel_under_threadsanitizer(tsan_exe, L, wpb, gpf, blocks, nsplit):
    # nsplit > 1: each slot's plies in parts claimed as separate work units,
    # a later part waiting for the earlier one's release
    exe, tmp = tsan_exe
    _run_and_compare(exe, tmp, 8, 120, L, wpb, gpf, blocks, 7,
                     env={"TSAN_OPTIONS": "halt_on_error=0", "NSPLIT": str(nsplit)})


def test_step_kernel_under_address_and_ub_sanitizers(tmp_path, built):
    exe, _ = built("env_on_host.cpp", SANITIZERS[1][0])
    for L, wpb, gpf, blocks, nsplit in ((8, 2, 1, 2, 1), (4, 1, 1, 1, 2)):
        _run_and_compare(exe, str(tmp_path), 8, 150, L, wpb, gpf, blocks, 11,
                         env={"ASAN_OPTIONS": "detect_leaks=0", "NSPLIT": str(nsplit)})


def test_part_wait_runs_out_and_latches_a_timeout(tmp_path, built):
    # two parts per slot, the queue starting at the second parts: no first
    # part ever runs, so every wait (bounded at 200 polls here) runs out,
    # latches ST_ERR_TIMEOUT (5) for the lowest slot and skips the unit; the
    # launch returns
    exe, _ = built("env_on_host.cpp", SANITIZERS[1][0] + ["-DST_PART_SPIN_LIMIT=200"])
    N, S = 8, 120
    out = str(tmp_path / "o")
    r = subprocess.run([exe, str(N), str(S), "8", "1", "1", "1", "3", out], capture_output=True, text=True,
                       timeout=600, env=dict(os.environ, ASAN_OPTIONS="detect_leaks=0", NSPLIT="2", QUEUE0=str(N)))
    _check_report(r)
    assert "status 5 0" in r.stdout, r.stdout[-2000:]
    # nothing was played: the counters stay zero
    assert not np.fromfile(out + ".stats", dtype=np.uint32).any()


def test_harness_reports_a_planted_missing_sync(tmp_path):
    # the check itself: without the team barrier between clearing the board
    # and placing the pieces, ThreadSanitizer must report a race
    sync = ("    for (int s = T.tl; s < 112; s += L) G->board[s] = (s < 100 && is_lake(s)) ? kLake : kEmpty;\n"
            "    T.sync();")

    def drop_sync(name, text):
        if name != "engine.cuh":
            return text
        assert sync in text
        return text.replace(sync, sync.split("\n")[0])

    exe = _build(str(tmp_path), ["-fsanitize=thread"], "env_race", edit=drop_sync)
    r = subprocess.run([exe, "4", "20", "8", "1", "1", "1", "7", str(tmp_path / "o")], capture_output=True,
                       text=True, timeout=600, env=dict(os.environ, TSAN_OPTIONS="halt_on_error=1"))
    report = r.stdout + r.stderr
    if r.returncode != 0 and "FATAL: ThreadSanitizer" in report and "memory" in report:
        pytest.skip("ThreadSanitizer cannot start here")
    assert "WARNING: ThreadSanitizer: data race" in report and "build_board" in report, report[-3000:]
    with pytest.raises(AssertionError, match="unexpected data race"):
        _check_report(r, ())


def test_harness_reports_mismatched_collectives(tmp_path):
    # plant, on the host only, a team whose lanes reach different kinds of
    # collective with one mask: the odd lanes reduce, the even lanes ballot
    # (undefined on the hardware); the harness must stop with a report that
    # names both collectives
    total = "    const int total = T.sum(cnt);\n    T.sync();\n    return total;"

    def mismatch(name, text):
        if name != "engine.cuh":
            return text
        assert total in text
        return text.replace(total, "    const int total = (T.tl & 1) ? T.sum(cnt) : (int)T.ballot(cnt > 0);\n"
                                   "    T.sync();\n    return total;")

    exe = _build(str(tmp_path), [], "env_mismatch", edit=mismatch)
    r = subprocess.run([exe, "4", "5", "8", "1", "1", "1", "7", str(tmp_path / "o")], capture_output=True,
                       text=True, timeout=600)
    report = r.stdout + r.stderr
    assert r.returncode != 0
    assert "different collectives: " in report and "reduce" in report and "ballot" in report, report[-3000:]


def _run_driver(exe, args, env, known=()):
    r = subprocess.run([exe] + [str(a) for a in args], capture_output=True, text=True, timeout=900,
                       env=dict(os.environ, **env))
    report = _check_report(r, known)
    assert "done" in r.stdout, report[-6000:]
    return r.stdout


SANITIZERS = [
    (["-fsanitize=thread"], {"TSAN_OPTIONS": "halt_on_error=0"}),
    (["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined"], {"ASAN_OPTIONS": "detect_leaks=0"}),
]


@pytest.mark.parametrize("san", [0, 1], ids=["tsan", "asan_ubsan"])
def test_observation_kernels_under_sanitizers(tmp_path, built, san):
    # k_replay (chunks of 4 items per warp) then k_obs_emit: planes, bf16
    # planes and masks of every item, the acting or a given player's view;
    # two items that cannot be replayed come back with status 1 and zeros
    flags, env = SANITIZERS[san]
    exe, src = built("obs_on_host.cpp", flags)
    g = oracle.play_games(41, 6)
    rng = np.random.default_rng(3)
    B = 30
    games = rng.integers(0, 6, B).astype(np.int32)
    plies = np.array([rng.integers(0, min(300, g["lengths"][k] - 1) + 1) for k in games], np.int16)
    order = np.lexsort((plies, games))
    games, plies = games[order], plies[order]
    player = (np.arange(B) % 3 - 1).astype(np.int8)
    bad = np.array([7, 19])
    games_in, plies_in = games.copy(), plies.copy()
    games_in[7] = 9                                # no such log
    plies_in[19] = g["actions"].shape[1] + 1       # beyond the log
    inp = str(tmp_path / "in")
    g["setups"].tofile(inp + ".setups")
    g["actions"].tofile(inp + ".actions")
    games_in.tofile(inp + ".game")
    plies_in.tofile(inp + ".ply")
    player.tofile(inp + ".player")
    out = str(tmp_path / "out")
    _run_driver(exe, [inp, 6, g["actions"].shape[1], B, 4, out], env)
    status = np.fromfile(out + ".status", np.uint8)
    u8 = np.fromfile(out + ".planes", np.uint8).reshape(B, oracle.NCHAN, 100)
    bf = np.fromfile(out + ".bf16", np.uint16).reshape(B, oracle.NCHAN, 100)
    mask = np.fromfile(out + ".mask", np.uint8).reshape(B, oracle.MASK_BYTES)
    assert (status[bad] == 1).all() and (np.delete(status, bad) == 0).all()
    assert not u8[bad].any() and not bf[bad].any() and not mask[bad].any()
    good = np.delete(np.arange(B), bad)
    r8, rbf, rmask = oracle.obs_encode(g["setups"], g["actions"], games[good], plies[good], player=player[good])
    np.testing.assert_array_equal(u8[good], r8)
    np.testing.assert_array_equal(bf[good], rbf)
    np.testing.assert_array_equal(mask[good], rmask)


@pytest.mark.parametrize("san", [0, 1], ids=["tsan", "asan_ubsan"])
def test_rollout_kernels_under_sanitizers(tmp_path, built, san):
    # k_roots, then k_rollout_flat on two resident blocks striding over the
    # units (each team's chase store reused from unit to unit), with samples
    # drawn in the kernel or ahead by k_draw_samples, uniform and magnet
    # rollout policies; then k_belief and k_positions_mask
    flags, env = SANITIZERS[san]
    exe, src = built("rollout_on_host.cpp", flags)
    g = oracle.play_games(43, 4)
    rng = np.random.default_rng(5)
    games = np.repeat(np.arange(4), 2).astype(np.int32)
    plies = np.array([rng.integers(0, min(400, g["lengths"][k] - 1) + 1) for k in games], np.int16)
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    P, K, depth, seed = len(pos), 12, 24, 77
    inp = str(tmp_path / "in")
    pos.tofile(inp + ".pos")
    for draw_ahead, rflags in ((0, oracle.ALL_RULES), (1, oracle.ALL_RULES),
                               (0, oracle.ALL_RULES | oracle.ROLLOUT_MAGNET)):
        out = str(tmp_path / ("out%d_%d" % (draw_ahead, rflags)))
        _run_driver(exe, [inp, P, K, depth, seed, draw_ahead, 2, rflags, out], env)
        assert (np.fromfile(out + ".status", np.uint8) == 0).all()
        tallies = np.fromfile(out + ".tallies", np.int32).reshape(P, 4)
        np.testing.assert_array_equal(tallies, oracle.rollout(pos, K, depth, seed, flags=rflags))
    # the belief samples of st_belief_sample and the masks of st_positions_mask
    types = np.fromfile(out + ".types", np.uint8).reshape(P, K, 40)
    np.testing.assert_array_equal(types, oracle.belief_sample(pos, K, seed))
    mask = np.fromfile(out + ".mask", np.uint8).reshape(P, oracle.MASK_BYTES)
    n_legal = np.fromfile(out + ".n_legal", np.int32)
    two = np.fromfile(out + ".two_square", np.uint8)
    for i in range(P):
        moves = oracle.legal_moves(pos[i])
        bits = np.unpackbits(mask[i], bitorder="little")
        assert set(np.nonzero(bits)[0]) == set(moves.tolist()) and n_legal[i] == len(moves)
        assert two[i] == oracle.two_square_applies(pos[i])


@pytest.mark.parametrize("san", [0, 1], ids=["tsan", "asan_ubsan"])
def test_search_kernels_under_sanitizers(tmp_path, built, san):
    # k_search_prep, the single-block offsets scan (__syncthreads), samples
    # drawn ahead, k_search_rollouts on two resident blocks and the policy
    # update; the host's exp and log stand in for the device's, so pi is
    # compared within the GPU tests' 1e-12 relative bound
    flags, env = SANITIZERS[san]
    exe, src = built("search_on_host.cpp", flags)
    g = oracle.play_games(47, 3)
    rng = np.random.default_rng(5)
    games = np.repeat(np.arange(3), 2).astype(np.int32)
    plies = np.array([rng.integers(0, min(400, g["lengths"][k] - 1) + 1) for k in games], np.int16)
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    P, S, depth, seed = len(pos), 3, 8, 2024
    inp = str(tmp_path / "in")
    pos.tofile(inp + ".pos")
    for rflags in (oracle.ALL_RULES, oracle.ALL_RULES | oracle.ROLLOUT_MAGNET):
        out = str(tmp_path / ("out%d" % rflags))
        _run_driver(exe, [inp, P, S, depth, seed, 2, rflags, out], env, ())
        ref = oracle.search(pos, S, depth, seed, flags=rflags)
        M = oracle.SEARCH_MAX_MOVES
        for k, dt, shape in (("n_moves", np.int32, (P,)), ("actions", np.int16, (P, M)),
                             ("tallies", np.int32, (P, M, 4)), ("q", np.float64, (P, M)),
                             ("chosen", np.int16, (P,)), ("status", np.uint8, (P,))):
            np.testing.assert_array_equal(np.fromfile(out + "." + k, dt).reshape(shape), ref[k], err_msg=k)
        np.testing.assert_allclose(np.fromfile(out + ".pi", np.float64).reshape(P, M), ref["pi"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("san", [0, 1], ids=["tsan", "asan_ubsan"])
def test_plain_step_with_supplied_actions_under_sanitizers(tmp_path, built, san):
    # the plain path (one k_env_step launch per ply) with actions supplied for
    # most slots and plies and the random policy for the rest
    flags, env = SANITIZERS[san]
    exe, src = built("env_on_host.cpp", flags)
    N, S, seed = 8, 60, 5
    ref = oracle.env_run(seed, N, S)
    acts = ref["action"].astype(np.int16)
    acts[::3, ::2] = -1
    acts.tofile(str(tmp_path / "acts"))
    out = str(tmp_path / "o")
    r = subprocess.run([exe, str(N), str(S), "32", "4", "1", "1", str(seed), out, str(tmp_path / "acts")],
                       capture_output=True, text=True, timeout=900, env=dict(os.environ, **env))
    _check_report(r, ())
    for k, dt in (("action", np.int16), ("reward", np.int8), ("done", np.uint8), ("ply", np.int16)):
        np.testing.assert_array_equal(np.fromfile(out + "." + k, dt).reshape(S, N), ref[k], err_msg=k)
    mask = np.fromfile(out + ".mask", np.uint8).reshape(S, N, oracle.MASK_BYTES)
    np.testing.assert_array_equal(mask, ref["mask"])


@pytest.mark.parametrize("san", [0, 1], ids=["tsan", "asan_ubsan"])
def test_reset_sources_and_history_under_sanitizers(tmp_path, built, san):
    # history on, a mirrored setup pool, two pinned slots (a forced flag
    # capture and a mid-game position), the recording persistent step on two
    # blocks, then positions rebuilt at four past steps, the records of those
    # steps and the snapshots of every slot (k_env_export)
    from tests.helpers import BOMB, FLAG, MINER, SERGEANT, make_position, sq
    flags, env = SANITIZERS[san]
    exe, src = built("env_sources_on_host.cpp", flags)
    N, S, H, seed, M = 16, 200, 200, 23, 3
    pool = np.zeros((2, M, 40), np.uint8)
    for m in range(M):
        t = oracle.setup_types(3000, m)
        pool[0, m], pool[1, m] = t[:40], t[40:]
    g = oracle.play_games(72, 1)
    mid = oracle.replay_positions(g["setups"], g["actions"], np.array([0]),
                                  np.array([min(200, g["lengths"][0] - 1)], np.int16))[0]
    forced = make_position([(0, MINER, sq("e8"), 0), (0, BOMB, sq("d8"), 0), (0, BOMB, sq("f8"), 0),
                            (0, BOMB, sq("e7"), 0), (0, FLAG, sq("a1"), 0), (1, FLAG, sq("e9"), 0),
                            (1, SERGEANT, sq("j9"), 0)], ply=300, battleless=12)
    pins = {3: forced, 7: mid}
    inp, out = str(tmp_path / "in"), str(tmp_path / "o")
    pool.tofile(inp + ".pool")
    np.stack([pins[i] for i in sorted(pins)]).tofile(inp + ".pins")
    np.array(sorted(pins), np.int32).tofile(inp + ".idx")
    steps = [200, 150, 60, 0]
    stdout = _run_driver(exe, [inp, out, N, S, 8, 2, 1, 2, seed, H, M, 1, len(pins)] + steps, env, ())
    assert "status 0 " in stdout, stdout[-2000:]
    ref = oracle.env_run(seed, N, S, pool=pool, mirror=True, episode0=1, pins=pins)
    for k, dt in (("action", np.int16), ("reward", np.int8), ("done", np.uint8), ("ply", np.int16)):
        np.testing.assert_array_equal(np.fromfile(out + "." + k, dt).reshape(S, N), ref[k], err_msg=k)
    np.testing.assert_array_equal(np.fromfile(out + ".mask", np.uint8).reshape(S, N, oracle.MASK_BYTES), ref["mask"])
    np.testing.assert_array_equal(np.fromfile(out + ".stats", np.uint32).reshape(N, 8), ref["stats"])
    for t in steps:
        status = np.fromfile(out + ".hist%d.status" % t, np.uint8)
        pos = np.fromfile(out + ".hist%d.pos" % t, np.uint8).reshape(N, oracle.POS_BYTES)
        assert (status == 0).all(), (t, status)
        fin = oracle.env_run(seed, N, t, want_mask=False, want_final=True, pool=pool, mirror=True, episode0=1,
                             pins=pins)["final"]
        np.testing.assert_array_equal(pos, fin, err_msg="step %d" % t)
        if t < S:
            for k, dt in (("action", np.int16), ("done", np.uint8), ("reward", np.int8)):
                np.testing.assert_array_equal(np.fromfile(out + ".steps%d.%s" % (t, k), dt), ref[k][t],
                                              err_msg="step record %d %s" % (t, k))
    now = oracle.env_run(seed, N, S, want_mask=False, want_final=True, pool=pool, mirror=True, episode0=1,
                         pins=pins)["final"]
    np.testing.assert_array_equal(np.fromfile(out + ".export", np.uint8).reshape(N, oracle.POS_BYTES), now[::-1])


@pytest.mark.parametrize("san", [0, 1], ids=["tsan", "asan_ubsan"])
def test_serving_batch_under_sanitizers(tmp_path, built, san):
    # one batch of the server: k_serve_roots, then k_serve_rollouts on two
    # resident blocks; each request's last unit publishes its tallies and
    # completion word; a request with no samples is published by the roots
    # kernel, one with a corrupt position with -1 tallies
    flags, env = SANITIZERS[san]
    exe, src = built("serve_on_host.cpp", flags)
    g = oracle.play_games(44, 3)
    rng = np.random.default_rng(9)
    games = np.array([0, 1, 2, 0, 1], np.int32)
    plies = np.array([rng.integers(0, min(300, g["lengths"][k] - 1) + 1) for k in games], np.int16)
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    bad = pos[0].copy()
    bad[0] = 99
    pos = np.concatenate([pos, bad[None]])
    R = len(pos)
    #                K  depth seed-lo seed-hi stream
    req = np.array([[9, 200, 77, 0, 5], [0, 12, 78, 0, 6], [13, 20, 79, 1, 7], [5, 1, 80, 0, 8],
                    [11, 160, 81, 0, 9], [4, 8, 82, 0, 10]], np.int32)
    inp, out = str(tmp_path / "in"), str(tmp_path / "o")
    pos.tofile(inp + ".pos")
    req.tofile(inp + ".req")
    _run_driver(exe, [inp, R, 2, out], env, ())
    tallies = np.fromfile(out + ".tallies", np.int32).reshape(R, 4)
    np.testing.assert_array_equal(np.fromfile(out + ".done", np.uint32), 1000 + np.arange(R))
    for i in range(R - 1):
        K, depth, lo, hi, sid = (int(v) for v in req[i])
        seed = (hi << 32) | (lo & 0xFFFFFFFF)
        ref = (oracle.rollout(pos[i:i + 1], K, depth, seed, stream_ids=np.array([sid], np.uint32))[0] if K > 0
               else np.zeros(4, np.int32))
        np.testing.assert_array_equal(tallies[i], ref, err_msg="request %d" % i)
    assert (tallies[R - 1] == -1).all()
