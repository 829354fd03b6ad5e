"""Pins of the oracle's App. E search: per-candidate-move rollouts with a
forced first move, mean values, the magnet policy and the tabular MMD update,
and the sampled move.  CPU only."""
import numpy as np
import pytest

import oracle
from tests.helpers import FLAG, MARSHAL, MINER, SERGEANT, F_MOVED, F_REVEALED, action, make_position, sq

ALPHA, BETA = oracle.SEARCH_ALPHA, oracle.SEARCH_BETA


def _pos_two_pieces():
    # red to move: Marshal e4 (four moves), Sergeant a1 (a2, b1), Flag j1;
    # blue: Flag j10 and a Sergeant at a10 that can move
    return make_position([(0, MARSHAL, sq("e4"), F_MOVED), (0, SERGEANT, sq("a1"), 0), (0, FLAG, sq("j1"), 0),
                          (1, FLAG, sq("j10"), 0), (1, SERGEANT, sq("a10"), 0)])


def _dense(actions, values):
    d = np.zeros((1, 10000), np.float32)
    for a, v in zip(actions, values):
        d[0, a] = v
    return d


def test_magnet_policy_on_a_hand_position_and_the_fixed_point():
    # rho (Tab. notation): a piece with a move uniformly, then one of its moves
    # uniformly: 1/(2*4) for each Marshal move, 1/(2*2) for each Sergeant move.
    # With no rollouts q = 0, and with pi_theta = rho the update's optimum is
    # rho itself ([rho^a rho^b]^(1/(a+b)) = rho).
    pos = _pos_two_pieces()
    marshal = [action("e4", t) for t in ("e3", "d4", "f4", "e5")]
    sergeant = [action("a1", t) for t in ("a2", "b1")]
    want = {a: 0.125 for a in marshal}
    want.update({a: 0.25 for a in sergeant})
    acts = sorted(want)
    r = oracle.search(pos, 0, 1, 3, pi_theta=_dense(acts, [want[a] for a in acts]))
    n = r["n_moves"][0]
    assert n == 6 and sorted(r["actions"][0, :n].tolist()) == acts
    got = dict(zip(r["actions"][0, :n].tolist(), r["pi"][0, :n]))
    for a in acts:
        assert got[a] == pytest.approx(want[a], rel=1e-12)
    assert (r["q"][0, :n] == 0).all() and (r["tallies"][0, :n] == 0).all()


def _objective(pi, q, rho, pt):
    m = pi > 0
    return (pi * q).sum() - ALPHA * (pi[m] * np.log(pi[m] / rho[m])).sum() - BETA * (pi[m] * np.log(pi[m] / pt[m])).sum()


def test_update_maximizes_the_regularized_objective():
    # App. E step 4: pi_search = argmax <q, pi> - alpha KL(pi, rho) - beta KL(pi, pi_theta).
    # Checked through optimality, not through the closed form: stationarity on
    # the support and no gain from random moves on the simplex.
    g = oracle.play_games(11, 3)
    plies = np.minimum(g["lengths"] - 1, [20, 40, 60]).astype(np.int16)
    pos = oracle.replay_positions(g["setups"], g["actions"], np.arange(3), plies)
    rng = np.random.default_rng(0)
    for b in range(3):
        r0 = oracle.search(pos[b], 0, 1, 5)
        n = r0["n_moves"][0]
        acts = r0["actions"][0, :n]
        pt_vals = rng.dirichlet(np.ones(n))
        r = oracle.search(pos[b], 6, 6, 5, pi_theta=_dense(acts, pt_vals))
        q = r["q"][0, :n]
        pi = r["pi"][0, :n]
        pt = pt_vals.astype(np.float32).astype(np.float64)
        # rho from the move list: pieces with a move, moves per piece
        frm = acts // 100
        per = {f: (frm == f).sum() for f in set(frm.tolist())}
        rho = np.array([1.0 / (len(per) * per[f]) for f in frm])
        # stationarity: q - alpha (ln(pi/rho) + 1) - beta (ln(pi/pt) + 1) is one constant
        g_ = q - ALPHA * (np.log(pi / rho) + 1) - BETA * (np.log(pi / pt) + 1)
        assert np.ptp(g_) < 1e-9 * max(1.0, np.abs(g_).max())
        f0 = _objective(pi, q, rho, pt)
        for _ in range(200):
            eps = rng.normal(size=n) * 1e-3
            alt = pi * np.exp(eps)
            alt /= alt.sum()
            assert _objective(alt, q, rho, pt) <= f0 + 1e-15


def test_forced_first_move_and_mean_values():
    # depth 1: only the forced move is played.  Red's Miner j9 takes blue's
    # revealed Flag j10 (a win in every configuration: a revealed piece keeps
    # its type in the belief samples); every other move leaves the game
    # running (unfinished, value 0).
    pos = make_position([(0, MINER, sq("j9"), F_MOVED), (0, FLAG, sq("a1"), 0), (1, FLAG, sq("j10"), F_REVEALED),
                         (1, SERGEANT, sq("a10"), 0)])
    S = 5
    r = oracle.search(pos, S, 1, 42)
    n = r["n_moves"][0]
    acts = r["actions"][0, :n].tolist()
    win = action("j9", "j10")
    assert win in acts
    for j, a in enumerate(acts):
        want = [S, 0, 0, 0] if a == win else [0, 0, 0, S]
        assert r["tallies"][0, j].tolist() == want
        assert r["q"][0, j] == (1.0 if a == win else 0.0)
    # the winning move dominates the update
    assert r["chosen"][0] == win and r["pi"][0, acts.index(win)] > 0.99


def _search_rollout_by_hand(pos, types, seed, stream, j, S, s, depth, first):
    """Re-derive one search rollout with the oracle's primitives and the key
    layout: forced first move, then counter (stream, j*S+s, d, 5<<24)."""
    p = pos.copy()
    searcher = int(np.frombuffer(p[240:242].tobytes(), np.int16)[0]) & 1
    opp = 1 - searcher
    p[40 * opp:40 * opp + 40] = types
    p, code, winner = oracle.apply(p, [first])
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    d = 1
    while not code and d < depth:
        moves = np.sort(oracle.legal_moves(p))
        w = oracle.philox(np.array([[stream, j * S + s, d, 5 << 24]], np.uint32), key)[0, 0]
        a = moves[(int(w) * len(moves)) >> 32]
        p, code, winner = oracle.apply(p, [a])
        d += 1
    if not code:
        return 3
    return 2 if winner < 0 else (0 if winner == searcher else 1)


def test_rollouts_match_step_by_step_rederivation():
    g = oracle.play_games(5, 2)
    plies = np.minimum(g["lengths"] - 1, [30, 80]).astype(np.int16)
    pos = oracle.replay_positions(g["setups"], g["actions"], np.arange(2), plies)
    S, D, seed = 3, 12, 99
    r = oracle.search(pos, S, D, seed)
    types = oracle.belief_sample(pos, S, seed)
    for b in range(2):
        n = r["n_moves"][b]
        for j in range(n):
            tally = [0, 0, 0, 0]
            for s in range(S):
                tally[_search_rollout_by_hand(pos[b], types[b, s], seed, b, j, S, s, D, r["actions"][b, j])] += 1
            assert r["tallies"][b, j].tolist() == tally


def test_sampled_move_follows_pi():
    # with S = 0 the update is the same for every seed; the played move is
    # drawn from it, so over many seeds its frequencies match pi (chi-square)
    pos = _pos_two_pieces()
    acts = sorted([action("e4", t) for t in ("e3", "d4", "f4", "e5")] + [action("a1", "a2"), action("a1", "b1")])
    pt = _dense(acts, [0.05, 0.1, 0.15, 0.2, 0.2, 0.3])
    r = oracle.search(pos, 0, 1, 0, pi_theta=pt)
    pi = r["pi"][0, :6]
    order = r["actions"][0, :6].tolist()
    N = 4000
    counts = np.zeros(6)
    for seed in range(N):
        c = oracle.search(pos, 0, 1, seed + 1, pi_theta=pt)["chosen"][0]
        counts[order.index(int(c))] += 1
    exp = N * pi
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 25.0   # 5 degrees of freedom: p < 1e-4


def test_zero_prior_moves_and_degenerate_inputs():
    pos = _pos_two_pieces()
    acts = sorted([action("e4", t) for t in ("e3", "d4", "f4", "e5")] + [action("a1", "a2"), action("a1", "b1")])
    # a legal move with pi_theta = 0 gets probability 0 and is never played
    pt = _dense(acts, [0.0, 0.2, 0.2, 0.2, 0.2, 0.2])
    for seed in range(50):
        r = oracle.search(pos, 2, 4, seed, pi_theta=pt)
        assert r["pi"][0, 0] == 0.0 and r["chosen"][0] != acts[0]
        assert r["pi"][0, :6].sum() == pytest.approx(1.0, abs=1e-12)
    # pi_theta zero on every legal move: rejected
    r = oracle.search(pos, 2, 4, 1, pi_theta=np.zeros((1, 10000), np.float32))
    assert r["status"][0] == 2 and r["chosen"][0] == -1
    # a side without legal moves searches nothing
    stuck = make_position([(0, FLAG, sq("a1"), 0), (1, FLAG, sq("j10"), 0), (1, SERGEANT, sq("a10"), 0)])
    r = oracle.search(stuck, 3, 4, 1)
    assert r["n_moves"][0] == 0 and r["chosen"][0] == -1 and r["status"][0] == 0
    # an invalid snapshot is reported
    bad = pos.copy()
    bad[0] = 99
    assert oracle.search(bad, 3, 4, 1)["status"][0] == 1


def test_given_values_replace_the_rollouts():
    # step 3 with a value estimate per move given by action (the value
    # network's role): no rollout runs, q is the given value, and the update
    # is still the maximiser of the regularised objective
    pos = _pos_two_pieces()
    acts = sorted([action("e4", t) for t in ("e3", "d4", "f4", "e5")] + [action("a1", "a2"), action("a1", "b1")])
    qv = np.zeros((1, 10000), np.float32)
    vals = np.array([0.01, -0.02, 0.0, 0.03, -0.005, 0.015], np.float32)
    qv[0, acts] = vals
    qv[0, 9999] = 5.0                       # an illegal action's entry is never read
    r = oracle.search(pos, 8, 20, 3, q_values=qv)
    n = r["n_moves"][0]
    assert n == 6 and (r["tallies"][0] == 0).all()
    order = r["actions"][0, :n]
    np.testing.assert_array_equal(r["q"][0, :n], qv[0, order].astype(np.float64))
    q = r["q"][0, :n]
    pi = r["pi"][0, :n]
    rho = np.array([0.25 if a // 100 == 0 else 0.125 for a in order])
    pt = np.full(n, 1.0 / n)
    g_ = q - ALPHA * (np.log(pi / rho) + 1) - BETA * (np.log(pi / pt) + 1)
    assert np.ptp(g_) < 1e-9
    # the move with the largest value gains the most over the prior
    best = int(np.argmax(q))
    assert pi[best] / (rho[best] ** (ALPHA / (ALPHA + BETA)) * pt[best] ** (BETA / (ALPHA + BETA))) == pytest.approx(
        np.max(pi / (rho ** (ALPHA / (ALPHA + BETA)) * pt ** (BETA / (ALPHA + BETA)))), rel=1e-12)
