"""GPU parity of the env's reset sources with the oracle, bit for bit: a
setup pool per side with left-right orientation randomisation (Sec. "Data
Collection", App. "Learned Setups") and restarts from pinned non-initial
positions with their history and chase state (App. B.3-B.4)."""
import numpy as np
import pytest

import oracle
from tests.helpers import BOMB, CAPTAIN, FLAG, MINER, SERGEANT, action, make_position, sq

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2511_07312_gb300 as st  # noqa: E402


def _pool(M, seed=0):
    pool = np.zeros((2, M, 40), np.uint8)
    for m in range(M):
        t = oracle.setup_types(2000 + seed, m)
        pool[0, m] = t[:40]
        pool[1, m] = t[40:]
    return pool


def _compare(gpu, ref, keys=("action", "reward", "done", "ply", "mask")):
    for k in keys:
        g = gpu[k].cpu().numpy() if hasattr(gpu[k], "cpu") else gpu[k]
        mism = np.argwhere(g != ref[k]) if k != "mask" else np.argwhere((g != ref[k]).any(-1))
        assert mism.size == 0, "%s differs first at (step, slot) %s" % (k, mism[0])


def _plain(env, n):
    outs = {k: [] for k in ("action", "reward", "done", "ply", "mask")}
    for _ in range(n):
        o = env.step()
        for k in outs:
            outs[k].append(o[k].clone())
    env.stream.synchronize()
    return {k: torch.stack(v).cpu().numpy() for k, v in outs.items()}


def _pins():
    forced = make_position([(0, MINER, sq("e8"), 0), (0, BOMB, sq("d8"), 0), (0, BOMB, sq("f8"), 0),
                            (0, BOMB, sq("e7"), 0), (0, FLAG, sq("a1"), 0), (1, FLAG, sq("e9"), 0),
                            (1, SERGEANT, sq("j9"), 0)], ply=300, battleless=12)
    chase0 = make_position([(0, CAPTAIN, sq("a2"), 0), (0, CAPTAIN, sq("j2"), 0), (0, FLAG, sq("f1"), 0),
                            (1, SERGEANT, sq("b3"), 0), (1, SERGEANT, sq("i3"), 0), (1, FLAG, sq("f10"), 0)])
    seq = [action("a2", "b2"), action("b3", "a3"), action("j2", "i2"), action("i3", "j3"),
           action("b2", "a2"), action("a3", "b3"), action("i2", "j2"), action("j3", "i3")]
    chase, _, _ = oracle.apply(chase0, seq)
    g = oracle.play_games(71, 2)
    mid = oracle.replay_positions(g["setups"], g["actions"], np.arange(2),
                                  np.minimum(g["lengths"] - 1, [150, 333]).astype(np.int16))
    return {3: forced, 10: chase, 11: mid[0], 40: mid[1], 63: mid[1]}


@pytest.mark.parametrize("mirror", [False, True])
def test_pool_plain_steps(mirror):
    pool = _pool(5)
    env = st.Env(64, seed=11)
    env.set_setup_pool(torch.from_numpy(pool), mirror=mirror)
    env.reset()
    gpu = _plain(env, 300)
    ref = oracle.env_run(11, 64, 300, pool=pool, mirror=mirror, episode0=1)
    _compare(gpu, ref)
    env.close()


@pytest.mark.parametrize("gpw", [1, 4])
def test_pool_and_pins_persistent_run(gpw):
    pool = _pool(7, seed=1)
    pins = _pins()
    env = st.Env(64, seed=12)
    env.set_setup_pool(torch.from_numpy(pool), mirror=True)
    idx = torch.tensor(sorted(pins), dtype=torch.int32)
    env.pin(idx, torch.from_numpy(np.stack([pins[i] for i in sorted(pins)])).cuda())
    env.reset()
    env.set_launch(4, 0, 1, games_per_warp=gpw)
    out = env.run(1200)
    env.stream.synchronize()
    stats = env.stats().cpu().numpy()
    ref = oracle.env_run(12, 64, 1200, pool=pool, mirror=True, episode0=1, pins=pins)
    _compare(out, ref)
    np.testing.assert_array_equal(stats, ref["stats"].astype(np.int32))
    # slot 3 wins at once, every ply, from its pin
    assert (ref["done"][:, 3] == 1).all() and (ref["ply"][:, 3] == 300).all()
    env.close()


def test_pins_replace_and_clear():
    pins = _pins()
    env = st.Env(16, seed=13)
    env.pin(torch.tensor([3]), torch.from_numpy(pins[3][None].copy()).cuda())
    env.pin(torch.tensor([5, 5]), torch.from_numpy(np.stack([pins[11], pins[3]])).cuda())   # later entry wins
    env.reset()
    gpu = _plain(env, 40)
    ref = oracle.env_run(13, 16, 40, episode0=1, pins={5: pins[3]})
    _compare(gpu, ref)
    env.pin()                                            # cleared: slot 5 restarts from Philox setups
    env.reset()
    gpu = _plain(env, 40)
    assert (gpu["ply"][0] == 0).all()
    env.close()


def test_bad_pin_and_bad_pool_are_rejected():
    env = st.Env(8, seed=14)
    bad = _pins()[11].copy()
    bad[0] = 77
    env.pin(torch.tensor([2, 9]), torch.from_numpy(np.stack([bad, _pins()[3]])).cuda())
    with pytest.raises(st.StrategoError):
        env.sync()                                       # both entries latched, neither pinned
    env.reset()
    gpu = _plain(env, 5)
    ref = oracle.env_run(14, 8, 5, episode0=1)
    _compare(gpu, ref)
    pool = _pool(2)
    pool[1, 1, 0] = 11 if pool[1, 1, 0] != 11 else 10    # one entry with a wrong piece count
    with pytest.raises(st.StrategoError):
        env.set_setup_pool(torch.from_numpy(pool))
    env.close()
