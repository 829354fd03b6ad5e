"""Pins of the oracle's reset sources: a pool of setups per side (Sec. "Data
Collection"), left-right orientation randomisation of those setups (App.
"Learned Setups"), and restarts from a fixed non-initial position with its
history and chase state (App. B.3-B.4).  CPU only."""
import numpy as np

import oracle
from tests.helpers import (BOMB, CAPTAIN, FLAG, MINER, SERGEANT, action, make_position, sq)


def _pool(M, seed=0):
    # M valid setups per side, from the oracle's seeded setup shuffle
    pool = np.zeros((2, M, 40), np.uint8)
    for m in range(M):
        t = oracle.setup_types(1000 + seed, m)
        pool[0, m] = t[:40]
        pool[1, m] = t[40:]
    return pool


def _start_types(final):
    # at ply 0 piece id i of red stands on square i, id 40+i of blue on 60+i
    return final[:, :40], final[:, 40:80]


def _mirror(entry):
    return entry.reshape(4, 10)[:, ::-1].reshape(40)


def test_single_entry_pool_starts_every_game_from_it():
    pool = _pool(1)
    r = oracle.env_run(3, 50, 0, pool=pool, want_mask=False, want_final=True, episode0=2)
    red, blue = _start_types(r["final"])
    assert (red == pool[0, 0]).all() and (blue == pool[1, 0]).all()
    sq_ = r["final"][:, 80:160]
    assert (sq_[:, :40] == np.arange(40)).all() and (sq_[:, 40:] == np.arange(60, 100)).all()


def test_pool_index_is_uniform_and_follows_its_counter():
    M = 3
    pool = _pool(M)
    seed, n = 17, 3000
    r = oracle.env_run(seed, n, 0, pool=pool, want_mask=False, want_final=True, episode0=5)
    red, blue = _start_types(r["final"])
    key = np.array([seed, 0], np.uint32)
    got = np.zeros((2, M))
    for slot in range(n):
        for side, types in ((0, red[slot]), (1, blue[slot])):
            idx = [m for m in range(M) if (pool[side, m] == types).all()]
            assert len(idx) == 1
            w = oracle.philox(np.array([[slot, 5, 0, (7 << 24) | side]], np.uint32), key)[0, 0]
            assert idx[0] == (int(w) * M) >> 32
            got[side, idx[0]] += 1
    for side in (0, 1):
        chi2 = ((got[side] - n / M) ** 2 / (n / M)).sum()
        assert chi2 < 18.4   # 2 degrees of freedom: p < 1e-4


def test_mirroring_reverses_files_half_of_the_time():
    pool = _pool(1, seed=7)
    assert not (_mirror(pool[0, 0]) == pool[0, 0]).all()
    n = 4000
    r = oracle.env_run(21, n, 0, pool=pool, mirror=True, want_mask=False, want_final=True)
    red, blue = _start_types(r["final"])
    for side, types in ((0, red), (1, blue)):
        plain = (types == pool[side, 0]).all(1)
        flipped = (types == _mirror(pool[side, 0])).all(1)
        assert (plain ^ flipped).all()
        # binomial(4000, 1/2): 4.4 standard deviations
        assert abs(flipped.sum() - n / 2) < 140
    # without mirroring nothing is flipped
    r = oracle.env_run(21, 200, 0, pool=pool, want_mask=False, want_final=True)
    assert (r["final"][:, :40] == pool[0, 0]).all()


def _forced_capture():
    # red's only legal move: the Miner on e8 takes blue's Flag on e9
    return make_position([(0, MINER, sq("e8"), 0), (0, BOMB, sq("d8"), 0), (0, BOMB, sq("f8"), 0),
                          (0, BOMB, sq("e7"), 0), (0, FLAG, sq("a1"), 0), (1, FLAG, sq("e9"), 0),
                          (1, SERGEANT, sq("j9"), 0)], ply=300, battleless=12)


def test_pinned_slot_restarts_from_its_position():
    pin = _forced_capture()
    assert oracle.legal_moves(pin).tolist() == [action("e8", "e9")]
    r = oracle.env_run(5, 3, 20, pins={1: pin})
    # slot 1 wins at once, every step, restarting from the pin
    assert (r["action"][:, 1] == action("e8", "e9")).all()
    assert (r["done"][:, 1] == 1).all() and (r["reward"][:, 1] == 1).all()
    assert (r["ply"][:, 1] == 300).all()
    want = np.zeros(1264, np.uint8)
    a = action("e8", "e9")
    want[a >> 3] = 1 << (a & 7)
    assert (r["mask"][:, 1] == want).all()
    assert r["stats"][1].tolist() == [20, 0, 0, 0, 0, 20, 20, 0]
    # the other slots play their Philox games
    ref = oracle.env_run(5, 3, 20)
    for s in (0, 2):
        np.testing.assert_array_equal(r["action"][:, s], ref["action"][:, s])


def test_pinned_restart_keeps_the_chase_history():
    chase = make_position([(0, CAPTAIN, sq("a2"), 0), (0, CAPTAIN, sq("j2"), 0), (0, FLAG, sq("f1"), 0),
                           (1, SERGEANT, sq("b3"), 0), (1, SERGEANT, sq("i3"), 0), (1, FLAG, sq("f10"), 0)])
    seq = [action("a2", "b2"), action("b3", "a3"), action("j2", "i2"), action("i3", "j3"),
           action("b2", "a2"), action("a3", "b3"), action("i2", "j2"), action("j3", "i3")]
    pin, _, _ = oracle.apply(chase, seq)
    repeat = action("a2", "b2")
    legal = set(oracle.legal_moves(pin).tolist())
    assert repeat not in legal
    n = 300
    r = oracle.env_run(8, n, 1, pins={i: pin for i in range(n)}, want_mask=False, want_final=True)
    first = r["action"][0]
    assert set(first.tolist()) <= legal and repeat not in set(first.tolist())
    assert len(set(first.tolist())) == len(legal)          # every legal move is drawn by some slot
    # zero steps: the slot holds the pinned position itself
    r0 = oracle.env_run(8, 1, 0, pins={0: pin}, want_mask=False, want_final=True)
    np.testing.assert_array_equal(r0["final"][0], pin)
