"""GPU parity of the environment kernels (plain per-ply launch and the
persistent launch) with the oracle, bit for bit, through the C ABI."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2511_07312_gb300 as st  # noqa: E402


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _plain_steps(env, n_steps):
    outs = {k: [] for k in ("action", "reward", "done", "ply", "mask")}
    for _ in range(n_steps):
        o = env.step()
        for k in outs:
            outs[k].append(o[k].clone())
    env.stream.synchronize()
    return {k: torch.stack(v).cpu().numpy() for k, v in outs.items()}


def _compare(gpu, ref, slots=None, steps=None):
    for k in ("action", "reward", "done", "ply"):
        g = gpu[k] if slots is None else gpu[k][:, slots]
        r = ref[k]
        if steps is not None:
            g, r = g[steps], r[steps]
        mism = np.argwhere(g != r)
        assert mism.size == 0, "%s differs first at (step, slot) %s: gpu %s oracle %s" % (
            k, mism[0], g[tuple(mism[0])], r[tuple(mism[0])])
    if gpu.get("mask") is not None and ref.get("mask") is not None:
        g = gpu["mask"] if slots is None else gpu["mask"][:, slots]
        r = ref["mask"]
        if steps is not None:
            g, r = g[steps], r[steps]
        mism = np.argwhere((g != r).any(-1))
        assert mism.size == 0, "mask differs first at (step, slot) %s" % (mism[0],)


def test_plain_step_64_games_1000_plies_bit_exact():
    # 64 games, seed 1, to the end or the 1000-ply cap, auto-reset afterwards
    env = st.Env(64, seed=1)
    gpu = _plain_steps(env, 1000)
    ref = oracle.env_run(1, 64, 1000)
    _compare(gpu, ref)
    stats = _np(env.stats())
    np.testing.assert_array_equal(stats, ref["stats"].astype(np.int32))


def test_plain_step_ragged_slots_sampled():
    # 1,000 slots (the plain step runs 32 per block: a ragged last block),
    # 300 one-launch plies; sampled slots against the oracle
    N, S = 1000, 300
    env = st.Env(N, seed=13)
    gpu = _plain_steps(env, S)
    slots = np.array([0, 1, 31, 32, 500, 991, 992, 998, 999] + list(range(45, N, 89)))
    for s in slots:
        r = oracle.env_run(13, 1, S, slot0=int(s))
        for k in ("action", "reward", "done", "ply"):
            np.testing.assert_array_equal(gpu[k][:, s], r[k][:, 0], err_msg="%s slot %d" % (k, s))
        np.testing.assert_array_equal(gpu["mask"][:, s], r["mask"][:, 0], err_msg="mask slot %d" % s)


@pytest.mark.parametrize("gpw", [1, 2, 4, 8])
def test_persistent_run_matches_plain_and_oracle(gpw):
    env = st.Env(64, seed=1)
    env.set_launch(4, 0, 1, games_per_warp=gpw)
    out = env.run(1000)
    env.stream.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle.env_run(1, 64, 1000)
    _compare(gpu, ref)


@pytest.mark.parametrize("wpb,gpf,gpw", [(1, 1, 1), (4, 3, 1), (8, 1, 1), (8, 7, 1), (1, 1, 2), (4, 3, 2),
                                         (8, 1, 2), (8, 5, 2), (1, 1, 4), (4, 3, 4), (8, 1, 4), (8, 2, 4),
                                         (1, 1, 8), (2, 3, 8), (4, 1, 8), (8, 2, 8)])
def test_persistent_launch_shapes_ragged(wpb, gpf, gpw):
    # 1,000 slots (not a multiple of any block), 300 plies, ring of 7 rows
    N, S, R = 1000, 300, 7
    env = st.Env(N, seed=5)
    env.set_launch(wpb, 0, gpf, games_per_warp=gpw)
    out = env.run(S, R)
    env.stream.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in out.items()}
    slots = np.array([0, 1, 2, 499, 500, 998, 999] + list(range(37, N, 97)))
    # oracle per sampled slot (slots are independent)
    rows = [(S - R + i) for i in range(R)]
    for s in slots:
        r = oracle.env_run(5, 1, S, slot0=int(s))
        for j, row in enumerate(rows):
            ring_row = row % R
            for k in ("action", "reward", "done", "ply"):
                assert gpu[k][ring_row, s] == r[k][row, 0], (k, s, row)
            assert np.array_equal(gpu["mask"][ring_row, s], r["mask"][row, 0]), ("mask", s, row)
    stats = _np(env.stats())
    for s in slots:
        r = oracle.env_run(5, 1, S, slot0=int(s), want_mask=False)
        np.testing.assert_array_equal(stats[s], r["stats"][0].astype(np.int32))


@pytest.mark.parametrize("wpb,gpf,gpw", [(1, 1, 1), (4, 3, 2), (2, 2, 4)])
def test_persistent_launch_in_parts_per_slot(wpb, gpf, gpw):
    # one block per SM and 1.25 waves of slots (R resident games, N = R +
    # R/4 + 3): with 800 plies each slot's plies run as three work units of
    # 267, 267 and 266 plies, later parts claimed after every earlier one;
    # ring of 7 rows, then a second launch continuing the same slots
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    R = sms * wpb * gpw
    N, S, K = R + R // 4 + 3, 800, 7
    env = st.Env(N, seed=9)
    env.set_launch(wpb, 1, gpf, games_per_warp=gpw)
    out = env.run(S, K)
    env.stream.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in out.items()}
    stats = _np(env.stats())
    slots = np.array([0, 1, R - 1, R, N - 2, N - 1] + list(range(61, N, max(1, N // 9))))
    pos = _np(env.export(torch.from_numpy(slots).to(torch.int32)))
    for j, s in enumerate(slots):
        r = oracle.env_run(9, 1, S, slot0=int(s), want_final=True)
        for row in range(S - K, S):
            for k in ("action", "reward", "done", "ply"):
                assert gpu[k][row % K, s] == r[k][row, 0], (k, s, row)
            assert np.array_equal(gpu["mask"][row % K, s], r["mask"][row, 0]), ("mask", s, row)
        np.testing.assert_array_equal(stats[s], r["stats"][0].astype(np.int32))
        np.testing.assert_array_equal(pos[j], r["final"][0])
    env.run(S, K)
    st2 = _np(env.stats())
    for s in slots[:4]:
        r = oracle.env_run(9, 1, 2 * S, slot0=int(s), want_mask=False)
        np.testing.assert_array_equal(st2[s], r["stats"][0].astype(np.int32))


def test_oversized_launch_shape_is_rejected_and_leaves_no_error_behind():
    env = st.Env(64, seed=1)
    with pytest.raises(st.StrategoError):
        env.set_launch(16, 0, 1, games_per_warp=8)   # more warps per block than the persistent kernel allows
    out = env.run(50)   # the previous shape is kept
    env.stream.synchronize()
    ref = oracle.env_run(1, 64, 50)
    _compare({k: v.cpu().numpy() for k, v in out.items()}, ref)
    st.Env(64, seed=2).close()


def test_launch_shape_reports_the_clamped_blocks_per_sm():
    env = st.Env(64, seed=1)
    env.set_launch(8, 0, 1, games_per_warp=4)
    full = env.launch_shape()
    assert full["warps_per_block"] == 8 and full["games_per_warp"] == 4 and full["games_per_fetch"] == 1
    assert full["blocks_per_sm"] >= 1
    env.set_launch(8, 64, 3, games_per_warp=4)   # far above what fits: clamped to the occupancy limit
    assert env.launch_shape() == dict(full, games_per_fetch=3)
    env.set_launch(8, 1, 1, games_per_warp=4)
    assert env.launch_shape()["blocks_per_sm"] == 1
    out = env.run(50)
    env.stream.synchronize()
    _compare({k: v.cpu().numpy() for k, v in out.items()}, oracle.env_run(1, 64, 50))
    env.close()


def test_full_size_65536_games_2000_plies_sampled_slots():
    # the benchmark workload in the benchmark's launch shape: 65,536 slots,
    # 2,000 plies in one persistent launch, a 16-row ring; sampled slots are
    # checked against the oracle (counters, final snapshot, last 16 plies)
    from paper_2511_07312_gb300 import autotune
    N, S, R = 65536, 2000, 16
    best = autotune.tune(N, final_plies=S)
    env = st.Env(N, seed=1)
    env.set_launch(best["warps_per_block"], best["blocks_per_sm"], best["games_per_fetch"],
                   games_per_warp=best["games_per_warp"])
    out = env.run(S, R)
    env.sync()
    stats = _np(env.stats())
    slots = np.array([0, 1, 151, 152, 4095, 4096, 32767, 32768, 65534, 65535] +
                     list(np.random.default_rng(0).integers(0, N, 22)))
    pos = env.export(torch.from_numpy(slots).to(torch.int32))
    env.sync()
    pos = pos.cpu().numpy()
    ring = {k: v.cpu().numpy() for k, v in out.items()}
    assert (stats[:, 5] <= S).all() and stats[:, 5].sum() > 0.99 * N * S
    for j, s in enumerate(slots):
        r = oracle.env_run(1, 1, S, slot0=int(s), want_final=True)
        np.testing.assert_array_equal(stats[s], r["stats"][0].astype(np.int32))
        np.testing.assert_array_equal(pos[j], r["final"][0])
        for row in range(S - R, S):
            for k in ("action", "reward", "done", "ply"):
                assert ring[k][row % R, s] == r[k][row, 0], (k, s, row)
            assert np.array_equal(ring["mask"][row % R, s], r["mask"][row, 0]), ("mask", s, row)


def test_full_size_all_65536_slots_counters_and_final_positions():
    # the same launch; every slot's counters (games ended by each code,
    # plies, wins per side) and final snapshot against the oracle, the
    # oracle stepping disjoint slots on every host thread
    import os
    import threading
    from paper_2511_07312_gb300 import autotune
    N, S = 65536, 2000
    best = autotune.tune(N, final_plies=S)
    env = st.Env(N, seed=1)
    env.set_launch(best["warps_per_block"], best["blocks_per_sm"], best["games_per_fetch"],
                   games_per_warp=best["games_per_warp"])
    env.run(S, 16)
    env.sync()
    stats = _np(env.stats())
    pos = _np(env.export(torch.arange(N, dtype=torch.int32)))
    chunk, nxt, bad = 256, [0], []
    lock = threading.Lock()

    def worker():
        while True:
            with lock:
                s0 = nxt[0]
                nxt[0] += chunk
            if s0 >= N:
                return
            r = oracle.env_run(1, chunk, S, slot0=s0, want_mask=False, want_final=True)
            st_ok = np.array_equal(stats[s0:s0 + chunk], r["stats"].astype(np.int32))
            pos_ok = np.array_equal(pos[s0:s0 + chunk], r["final"])
            if not (st_ok and pos_ok):
                with lock:
                    bad.append((s0, st_ok, pos_ok))

    threads = [threading.Thread(target=worker) for _ in range(max(1, len(os.sched_getaffinity(0))))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not bad, "chunks (first slot, counters equal, final positions equal) that differ: %s" % sorted(bad)[:8]


def test_supplied_actions_and_illegal_action_latch():
    env = st.Env(16, seed=3)
    ref = oracle.env_run(3, 16, 40)
    acts = torch.from_numpy(ref["action"]).cuda()
    outs = []
    for t in range(40):
        outs.append({k: v.clone() for k, v in env.step(acts[t].contiguous()).items()})
    env.sync()
    gpu = {k: torch.stack([o[k] for o in outs]).cpu().numpy() for k in outs[0]}
    _compare(gpu, ref)
    # an illegal action leaves that slot unchanged and is latched
    before = env.export(torch.arange(16))
    bad = torch.full((16,), -1, dtype=torch.int16, device="cuda")
    bad[5] = 0
    o = env.step(bad)
    with pytest.raises(st.StrategoError) as ei:
        env.sync()
    assert ei.value.code == 4
    after = env.export(torch.arange(16))
    torch.cuda.synchronize()
    assert torch.equal(before[5], after[5])
    assert int(o["action"][5]) == -1
    env.sync()   # the latch was cleared


def test_export_matches_oracle_snapshots_and_import_roundtrip():
    N, S = 48, 257
    env = st.Env(N, seed=9)
    env.run(S, 1, want=())
    pos = env.export(torch.arange(N))
    env.sync()
    ref = oracle.env_run(9, N, S, want_mask=False, want_final=True)
    np.testing.assert_array_equal(pos.cpu().numpy(), ref["final"])
    # import into other slots and continue: same as continuing in place
    env2 = st.Env(N, seed=9)
    env2.import_(torch.arange(N).flip(0), pos)
    env2.sync()
    back = env2.export(torch.arange(N).flip(0))
    env2.sync()
    np.testing.assert_array_equal(back.cpu().numpy(), ref["final"])


def test_import_of_oracle_positions_then_step_with_given_actions():
    g = oracle.play_games(13, 8)
    games = np.repeat(np.arange(8), 4)
    plies = np.concatenate([np.linspace(0, g["lengths"][i] - 2, 4).astype(np.int16) for i in range(8)])
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    n = len(pos)
    env = st.Env(n, seed=2, autoreset=False)
    env.import_(torch.arange(n), torch.from_numpy(pos).cuda())
    acts = np.array([g["actions"][games[i], plies[i]] for i in range(n)], np.int16)
    o = env.step(torch.from_numpy(acts).cuda())
    env.sync()
    nxt = oracle.replay_positions(g["setups"], g["actions"], games, plies + 1)
    after = env.export(torch.arange(n))
    env.sync()
    np.testing.assert_array_equal(after.cpu().numpy(), nxt)
    for i in range(n):
        moves = oracle.legal_moves(nxt[i])
        bits = np.unpackbits(o["mask"][i].cpu().numpy(), bitorder="little")
        assert set(np.nonzero(bits)[0]) == set(moves.tolist())


def test_bad_snapshot_is_rejected_without_fault():
    env = st.Env(4, seed=1)
    pos = env.export(torch.arange(4))
    env.sync()
    bad = pos.clone()
    bad[0, 0] = 99                 # type code out of range
    bad[1, 80] = 42                # a piece on a lake
    bad[2, 245] = 7                # chaser neither 0, 1 nor none
    env.import_(torch.arange(4), bad)
    with pytest.raises(st.StrategoError) as ei:
        env.sync()
    assert ei.value.code == 8
    now = env.export(torch.arange(4))
    env.sync()
    assert torch.equal(now[:3], pos[:3])


def test_sampled_actions_are_the_next_random_plies():
    # App. B.1 SampleRandomLegalAction: the random policy's action at the
    # current state, not played; the next step with actions NULL plays it
    for autoreset in (True, False):
        env = st.Env(48, seed=12, autoreset=autoreset)
        ref = oracle.env_run(12, 48, 400, autoreset=autoreset, want_mask=False)
        for t in range(400):
            sampled = _np(env.sample_actions())
            np.testing.assert_array_equal(sampled, ref["action"][t])
            out = env.step(want_mask=False)
            np.testing.assert_array_equal(_np(out["action"]), sampled)
        env.close()
