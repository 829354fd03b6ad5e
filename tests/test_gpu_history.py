"""GPU parity of the env's historical queries (App. B.1: the simulator keeps
a circular buffer of past steps and rebuilds past positions, masks and
information states on demand) with the oracle, bit for bit.  The oracle's
expected state at step t is its own environment run for t steps."""
import numpy as np
import pytest

import oracle
from tests.helpers import BOMB, FLAG, MINER, SERGEANT, make_position, sq

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2511_07312_gb300 as st  # noqa: E402


def _games_at(done, t, episode0=0, start0=0):
    """Per slot: the step at which the game holding it at step t began, and
    its episode number, from the oracle's ending codes (auto-reset)."""
    N = done.shape[1]
    start = np.full(N, start0, np.int64)
    ep = np.full(N, episode0, np.int64)
    for s in range(t):
        ended = done[s] != 0
        start[ended] = s + 1
        ep[ended] += 1
    return start, ep


def _final(seed, N, t, **kw):
    return oracle.env_run(seed, N, t, want_mask=False, want_final=True, **kw)["final"]


def test_positions_steps_and_logs_with_auto_reset():
    N, S, H, seed = 64, 700, 300, 21
    env = st.Env(N, seed=seed)
    env.enable_history(H)
    for _ in range(50):
        env.step()
    env.run(S - 50)
    assert env.current_step() == S
    ref = oracle.env_run(seed, N, S, want_mask=False)
    lo = S - H
    for t in (S, S - 1, 600, 450, lo + 1, lo):
        hp = env.history_positions(t)
        torch.cuda.synchronize()
        status = hp["status"].cpu().numpy()
        start, _ = _games_at(ref["done"], t)
        want = np.where(start < lo, 2, 0) if t < S else np.zeros(N)
        np.testing.assert_array_equal(status, want)
        ok = status == 0
        assert ok.any() or t <= lo + 1          # at the window's edge few games began inside it
        np.testing.assert_array_equal(hp["pos"].cpu().numpy()[ok], _final(seed, N, t)[ok])
        assert (hp["ended"].cpu().numpy() == 0).all() and (hp["since"].cpu().numpy() == 0).all()
    for t in (S - 1, 550, lo):
        hs = env.history_steps(t)
        torch.cuda.synchronize()
        start, _ = _games_at(ref["done"], t)
        np.testing.assert_array_equal(hs["action"].cpu().numpy(), ref["action"][t])
        np.testing.assert_array_equal(hs["done"].cpu().numpy(), ref["done"][t])
        np.testing.assert_array_equal(hs["reward"].cpu().numpy(), ref["reward"][t])
        np.testing.assert_array_equal(hs["start"].cpu().numpy(), (start == t).astype(np.uint8))
    # setups and action logs of the games at step t, then their planes
    t, L = 640, 1000
    hl = env.history_logs(t, L)
    torch.cuda.synchronize()
    start, ep = _games_at(ref["done"], t)
    status = hl["status"].cpu().numpy()
    np.testing.assert_array_equal(status, np.where(start < lo, 2, 0))
    setups, logs, plies = hl["setups"].cpu().numpy(), hl["logs"].cpu().numpy(), hl["plies"].cpu().numpy()
    ok = np.flatnonzero(status == 0)
    for g in ok:
        np.testing.assert_array_equal(setups[g], oracle.setup_types(seed, int(g), int(ep[g])))
        n = t - start[g]
        assert plies[g] == n
        np.testing.assert_array_equal(logs[g, :n], ref["action"][start[g]:t, g])
        assert (logs[g, n:] == -1).all()
    o = st.obs_encode(hl["setups"], hl["logs"], torch.from_numpy(ok.astype(np.int32)).cuda(),
                      hl["plies"][torch.from_numpy(ok).cuda()].contiguous())
    torch.cuda.synchronize()
    u8, _, mask = oracle.obs_encode(setups, logs, ok.astype(np.int32), plies[ok])
    np.testing.assert_array_equal(o["planes"].cpu().numpy(), u8)
    np.testing.assert_array_equal(o["mask"].cpu().numpy(), mask)
    env.close()


def test_ended_games_without_auto_reset():
    N, S, seed = 32, 900, 22
    env = st.Env(N, seed=seed, autoreset=False)
    env.enable_history(1000)
    env.run(S)
    ref = oracle.env_run(seed, N, S, autoreset=False, want_mask=False)
    assert (ref["done"] != 0).any(axis=0).sum() > N // 2
    for t in (S, 700, 300, 1):
        hp = env.history_positions(t)
        torch.cuda.synchronize()
        assert (hp["status"].cpu().numpy() == 0).all()
        np.testing.assert_array_equal(hp["pos"].cpu().numpy(), _final(seed, N, t, autoreset=False))
        ended, since = hp["ended"].cpu().numpy(), hp["since"].cpu().numpy()
        for g in range(N):
            e = np.flatnonzero(ref["done"][:t, g])
            if e.size:
                assert (ended[g], since[g]) == (ref["done"][e[0], g], t - e[0])
            else:
                assert (ended[g], since[g]) == (0, 0)
    env.close()


def test_window_edges_and_late_enable():
    N, seed = 16, 24
    env = st.Env(N, seed=seed)
    env.run(100)
    env.enable_history(50)
    env.run(80)
    now = env.current_step()
    assert now == 180
    for bad in (129, 181):
        with pytest.raises(st.StrategoError):
            env.history_positions(bad)
    with pytest.raises(st.StrategoError):
        env.history_steps(180)                   # no record of the current step yet
    ref = oracle.env_run(seed, N, 180, want_mask=False)
    hp = env.history_positions(130)
    torch.cuda.synchronize()
    start, _ = _games_at(ref["done"], 130)
    status = hp["status"].cpu().numpy()
    np.testing.assert_array_equal(status, np.where(start < 130, 2, 0))
    ok = status == 0
    np.testing.assert_array_equal(hp["pos"].cpu().numpy()[ok], _final(seed, N, 130)[ok])
    env.close()


def _forced_capture():
    return make_position([(0, MINER, sq("e8"), 0), (0, BOMB, sq("d8"), 0), (0, BOMB, sq("f8"), 0),
                          (0, BOMB, sq("e7"), 0), (0, FLAG, sq("a1"), 0), (1, FLAG, sq("e9"), 0),
                          (1, SERGEANT, sq("j9"), 0)], ply=300, battleless=12)


def test_history_with_pool_pins_imports_and_given_setups():
    N, seed = 16, 23
    pool = np.zeros((2, 3, 40), np.uint8)
    for m in range(3):
        t = oracle.setup_types(3000, m)
        pool[0, m], pool[1, m] = t[:40], t[40:]
    g = oracle.play_games(72, 1)
    mid = oracle.replay_positions(g["setups"], g["actions"], np.array([0]),
                                  np.array([min(200, g["lengths"][0] - 1)], np.int16))[0]
    pins = {3: _forced_capture(), 7: mid}
    env = st.Env(N, seed=seed)
    env.enable_history(400)
    env.set_setup_pool(torch.from_numpy(pool), mirror=True)
    env.pin(torch.tensor(sorted(pins), dtype=torch.int32),
            torch.from_numpy(np.stack([pins[i] for i in sorted(pins)])).cuda())
    env.reset()
    env.run(300)
    for t in (300, 250, 120, 0):
        hp = env.history_positions(t)
        torch.cuda.synchronize()
        assert (hp["status"].cpu().numpy() == 0).all()
        np.testing.assert_array_equal(hp["pos"].cpu().numpy(),
                                      _final(seed, N, t, episode0=1, pool=pool, mirror=True, pins=pins))
    hl = env.history_logs(250, 400)
    torch.cuda.synchronize()
    status = hl["status"].cpu().numpy()
    assert status[3] == 4 and status[7] == 4 and (np.delete(status, [3, 7]) == 0).all()
    # an import and a reset to given setups start games that cannot be rebuilt
    env.import_(torch.tensor([2]), torch.from_numpy(mid[None].copy()).cuda())
    which = torch.zeros(N, dtype=torch.uint8)
    which[5] = 1
    setups = torch.from_numpy(np.tile(oracle.setup_types(5, 5), (N, 1))).cuda()
    env.reset(setups, which.cuda())
    env.run(20)
    hp = env.history_positions(310)
    torch.cuda.synchronize()
    status = hp["status"].cpu().numpy()
    assert status[2] == 3 and status[5] == 3
    hp = env.history_positions(320)                  # the current step is always answered
    torch.cuda.synchronize()
    assert (hp["status"].cpu().numpy() == 0).all()
    env.close()


def test_masks_of_past_positions():
    N, seed = 32, 25
    env = st.Env(N, seed=seed)
    env.enable_history(500)
    env.run(400)
    hp = env.history_positions(333)
    m = st.positions_mask(hp["pos"])
    torch.cuda.synchronize()
    pos = hp["pos"].cpu().numpy()
    mask = m["mask"].cpu().numpy()
    for g in range(N):
        want = np.zeros(1264, np.uint8)
        moves = oracle.legal_moves(pos[g])
        for a in moves:
            want[a >> 3] |= 1 << (a & 7)
        np.testing.assert_array_equal(mask[g], want)
        assert m["n_legal"][g].item() == len(moves)
        assert m["two_square"][g].item() == oracle.two_square_applies(pos[g])
    env.close()


def test_history_recorded_by_a_persistent_launch_in_two_parts():
    # one block of one warp per SM and 1.25 waves of slots: a 700-ply launch
    # runs each slot's plies as two parts of 350, the second part of a slot
    # recording into the history ring where its first part stopped
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    N, S, H, seed = sms + sms // 4 + 3, 700, 500, 33
    env = st.Env(N, seed=seed)
    env.set_launch(1, 1, 1, games_per_warp=1)
    env.enable_history(H)
    env.run(S)
    assert env.current_step() == S
    ref = oracle.env_run(seed, N, S, want_mask=False)
    lo = S - H
    for t in (S, 600, 351, 349, lo + 1):
        hp = env.history_positions(t)
        torch.cuda.synchronize()
        status = hp["status"].cpu().numpy()
        start, _ = _games_at(ref["done"], t)
        want = np.where(start < lo, 2, 0) if t < S else np.zeros(N)
        np.testing.assert_array_equal(status, want)
        ok = status == 0
        np.testing.assert_array_equal(hp["pos"].cpu().numpy()[ok], _final(seed, N, t)[ok])
    for t in (S - 1, 351, 350, 349, lo):
        hs = env.history_steps(t)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(hs["action"].cpu().numpy(), ref["action"][t])
        np.testing.assert_array_equal(hs["done"].cpu().numpy(), ref["done"][t])
        np.testing.assert_array_equal(hs["reward"].cpu().numpy(), ref["reward"][t])
    np.testing.assert_array_equal(env.stats().cpu().numpy(), ref["stats"].astype(np.int32))
    env.close()
