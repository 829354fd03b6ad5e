"""GPU parity at the benchmark's full sizes, in the launch configuration the
benchmark times: every one of the 16,384 observation items (planes, bf16
planes, masks), every one of the 4,096 positions of the 256-sample x
depth-32 rollouts, and every slot of the 16,384-slot history query, each
against the oracle, which works through disjoint chunks on all host
threads.  Bit for bit."""
import os
import threading

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2511_07312_gb300 as st  # noqa: E402


def _workload3():
    # 64 games of seed 1 to their end or 1,000 plies; 16,384 items at plies
    # uniform in [0, min(600, length - 1)], sorted by (game, ply)
    g = oracle.play_games(1, 64)
    rng = np.random.default_rng(3)
    games = rng.integers(0, 64, 16384).astype(np.int32)
    plies = np.array([rng.integers(0, min(600, max(1, g["lengths"][k]) - 1) + 1) for k in games], np.int16)
    order = np.lexsort((plies, games))
    return g, games[order], plies[order]


def _on_host_threads(n, chunk, check):
    """check(lo, hi) for chunks [lo, hi) of range(n) on every host thread;
    returns the chunks whose check returned something other than None."""
    nxt, bad = [0], []
    lock = threading.Lock()

    def worker():
        while True:
            with lock:
                lo = nxt[0]
                nxt[0] += chunk
            if lo >= n:
                return
            r = check(lo, min(n, lo + chunk))
            if r is not None:
                with lock:
                    bad.append((lo, r))

    threads = [threading.Thread(target=worker) for _ in range(max(1, len(os.sched_getaffinity(0))))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    return sorted(bad)


def test_observations_all_16384_items():
    g, games, plies = _workload3()
    dev = torch.device("cuda", 0)
    o = st.obs_encode(torch.from_numpy(g["setups"]).to(dev), torch.from_numpy(g["actions"]).to(dev),
                      torch.from_numpy(games).to(dev), torch.from_numpy(plies).to(dev))
    torch.cuda.synchronize()
    assert (o["status"].cpu().numpy() == 0).all()
    u8_all = o["planes"].cpu().numpy()
    bf_all = o["planes_bf16"].view(torch.int16).cpu().numpy().view(np.uint16)
    mask_all = o["mask"].cpu().numpy()

    def check(lo, hi):
        u8, bf, mask = oracle.obs_encode(g["setups"], g["actions"], games[lo:hi], plies[lo:hi])
        ok = (np.array_equal(u8_all[lo:hi], u8), np.array_equal(bf_all[lo:hi], bf),
              np.array_equal(mask_all[lo:hi], mask))
        return None if all(ok) else ok

    bad = _on_host_threads(16384, 256, check)
    assert not bad, "chunks (first item, (planes, bf16, mask) equal) that differ: %s" % bad[:8]


def test_rollouts_all_4096_positions_256_samples_depth_32():
    g, games, plies = _workload3()
    sel = np.linspace(0, 16383, 4096).astype(np.int64)
    pos = oracle.replay_positions(g["setups"], g["actions"], games[sel], plies[sel])
    tallies, status = st.rollout(torch.from_numpy(pos).cuda(), 256, 32, seed=7)
    torch.cuda.synchronize()
    t = tallies.cpu().numpy()
    assert (status.cpu().numpy() == 0).all() and (t.sum(1) == 256).all()
    pick = np.array([0, 1, 511, 512, 2047, 3000, 4094, 4095])
    ref = oracle.rollout(pos[pick], 256, 32, 7, stream_ids=pick.astype(np.uint32))
    np.testing.assert_array_equal(t[pick], ref)

    # every position
    def check(lo, hi):
        r = oracle.rollout(pos[lo:hi], 256, 32, 7, stream_ids=np.arange(lo, hi, dtype=np.uint32))
        return None if np.array_equal(t[lo:hi], r) else int(np.argwhere((t[lo:hi] != r).any(1))[0, 0]) + lo

    bad = _on_host_threads(4096, 64, check)
    assert not bad, "chunks (first position, first differing position): %s" % bad[:8]


def test_history_all_16384_slots():
    N, H = 16384, 1000
    env = st.Env(N, seed=5)
    env.set_launch(4, 0, 1, games_per_warp=4)
    env.enable_history(H)
    env.run(H)
    t = env.current_step() - 300
    hp = env.history_positions(t)
    torch.cuda.synchronize()
    status = hp["status"].cpu().numpy()
    pos = hp["pos"].cpu().numpy()
    assert (status == 0).all()
    for g in (0, 1, 151, 152, 8191, 16383):
        ref = oracle.env_run(5, 1, t, slot0=g, want_mask=False, want_final=True)["final"][0]
        np.testing.assert_array_equal(pos[g], ref)
    env.close()

    # every slot
    def check(lo, hi):
        ref = oracle.env_run(5, hi - lo, t, slot0=lo, want_mask=False, want_final=True)["final"]
        return None if np.array_equal(pos[lo:hi], ref) else int(np.argwhere((pos[lo:hi] != ref).any(1))[0, 0]) + lo

    bad = _on_host_threads(N, 256, check)
    assert not bad, "chunks (first slot, first differing slot): %s" % bad[:8]
