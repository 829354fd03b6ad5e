"""Pins of the oracle's rollout policies: uniform over the legal moves, and
the magnet policy rho (Tab. notation: a piece with a legal move uniformly,
then one of its legal moves uniformly), as a rollout and search policy.
CPU only."""
import numpy as np

import oracle
from tests.helpers import FLAG, MARSHAL, SERGEANT, F_MOVED, action, make_position, sq

MAGNET = oracle.ROLLOUT_MAGNET


def _pos_two_pieces():
    # red to move: Sergeant a1 (a2, b1), Marshal e4 (e3, d4, f4, e5), Flag j1
    return make_position([(0, MARSHAL, sq("e4"), F_MOVED), (0, SERGEANT, sq("a1"), 0), (0, FLAG, sq("j1"), 0),
                          (1, FLAG, sq("j10"), 0), (1, SERGEANT, sq("a10"), 0)])


def test_magnet_pick_boundaries():
    # pieces in ascending square order: Sergeant a1 (square 0), Marshal e4
    # (square 34); word 0 splits [0, 2^32) in halves between them, word 1
    # splits the piece's moves (ascending) evenly
    pos = _pos_two_pieces()
    serg = sorted([action("a1", "a2"), action("a1", "b1")])
    mars = sorted([action("e4", t) for t in ("e3", "d4", "f4", "e5")])
    H = 1 << 31
    assert oracle.policy_pick(pos, 0, 0) == serg[0]
    assert oracle.policy_pick(pos, H - 1, H) == serg[1]
    assert oracle.policy_pick(pos, H, 0) == mars[0]
    for q in range(4):
        assert oracle.policy_pick(pos, 0xFFFFFFFF, q << 30) == mars[q]
        assert oracle.policy_pick(pos, 0xFFFFFFFF, (q << 30) + (1 << 30) - 1) == mars[q]
    # the uniform policy ignores word 1 and takes the idx-th of the six moves
    allm = sorted(serg + mars)
    for i in range(6):
        w0 = (i * (1 << 32) + 5) // 6 + 1
        assert oracle.policy_pick(pos, w0, 12345, magnet=False) == allm[(w0 * 6) >> 32]


def test_magnet_frequencies_follow_rho():
    pos = _pos_two_pieces()
    rng = np.random.default_rng(11)
    N = 20000
    w = rng.integers(0, 1 << 32, size=(N, 2), dtype=np.uint64)
    picks = np.array([oracle.policy_pick(pos, a, b) for a, b in w])
    want = {action("a1", "a2"): 0.25, action("a1", "b1"): 0.25}
    want.update({action("e4", t): 0.125 for t in ("e3", "d4", "f4", "e5")})
    assert set(picks.tolist()) == set(want)
    chi2 = sum((np.sum(picks == a) - N * p) ** 2 / (N * p) for a, p in want.items())
    assert chi2 < 25.0   # 5 degrees of freedom: p < 1e-4


def _first_run_lengths(moves):
    frm = moves // 100
    starts = np.flatnonzero(np.r_[True, frm[1:] != frm[:-1]])
    return starts, np.diff(np.r_[starts, len(moves)])


def _magnet_by_hand(moves, w0, w1):
    starts, lens = _first_run_lengths(moves)
    piece = (int(w0) * len(starts)) >> 32
    return moves[starts[piece] + ((int(w1) * int(lens[piece])) >> 32)]


def test_magnet_rollouts_rederived_step_by_step():
    g = oracle.play_games(9, 4)
    plies = np.minimum(g["lengths"] - 1, [10, 60, 120, 200]).astype(np.int16)
    pos = oracle.replay_positions(g["setups"], g["actions"], np.arange(4), plies)
    K, D, seed = 4, 20, 4242
    types = oracle.belief_sample(pos, K, seed)
    tallies, outcomes = oracle.rollout(pos, K, D, seed, flags=oracle.ALL_RULES | MAGNET, want_outcomes=True)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    for b in range(len(pos)):
        searcher = int(np.frombuffer(pos[b, 240:242].tobytes(), np.int16)[0]) & 1
        for s in range(K):
            p = pos[b].copy()
            p[40 * (1 - searcher):40 * (1 - searcher) + 40] = types[b, s]
            code, winner = oracle.start_check(p)
            d = 0
            while not code and d < D:
                moves = np.sort(oracle.legal_moves(p))
                w = oracle.philox(np.array([[b, s, d, 4 << 24]], np.uint32), key)[0]
                p, code, winner = oracle.apply(p, [_magnet_by_hand(moves, w[0], w[1])])
                d += 1
            want = 3 if not code else (2 if winner < 0 else (0 if winner == searcher else 1))
            assert outcomes[b, s] == want


def test_magnet_search_rollouts_use_the_search_counter():
    g = oracle.play_games(10, 2)
    plies = np.minimum(g["lengths"] - 1, [40, 90]).astype(np.int16)
    pos = oracle.replay_positions(g["setups"], g["actions"], np.arange(2), plies)
    S, D, seed = 2, 10, 31
    r = oracle.search(pos, S, D, seed, flags=oracle.ALL_RULES | MAGNET)
    types = oracle.belief_sample(pos, S, seed)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    for b in range(2):
        searcher = int(np.frombuffer(pos[b, 240:242].tobytes(), np.int16)[0]) & 1
        for j in range(r["n_moves"][b]):
            tally = [0, 0, 0, 0]
            for s in range(S):
                p = pos[b].copy()
                p[40 * (1 - searcher):40 * (1 - searcher) + 40] = types[b, s]
                p, code, winner = oracle.apply(p, [r["actions"][b, j]])
                d = 1
                while not code and d < D:
                    moves = np.sort(oracle.legal_moves(p))
                    w = oracle.philox(np.array([[b, j * S + s, d, 5 << 24]], np.uint32), key)[0]
                    p, code, winner = oracle.apply(p, [_magnet_by_hand(moves, w[0], w[1])])
                    d += 1
                tally[3 if not code else (2 if winner < 0 else (0 if winner == searcher else 1))] += 1
            assert r["tallies"][b, j].tolist() == tally
