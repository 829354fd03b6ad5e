"""Pins of the oracle's belief posterior and sampler (App. E "Search", step 1,
with the uniform posterior in place of the belief network) and of the random
rollouts (App. E, step 2)."""
import itertools
from collections import Counter
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.helpers import (BOMB, CAPTAIN, COUNTS, FLAG, F_MOVED, F_REVEALED, F_SCOUT, MARSHAL, MINER,
                           SCOUT, SERGEANT, SPY, make_position, sq)


def _tiny_position():
    """Blue (the opponent of red, who is to move) has 7 hidden pieces left:
    four unmoved (one is the flag), two moved, one known scout; everything
    else of blue is captured and therefore known."""
    blue = [(1, FLAG, sq("a10"), 0), (1, BOMB, sq("b10"), 0), (1, BOMB, sq("c10"), 0),
            (1, MINER, sq("d10"), 0),
            (1, SERGEANT, sq("e8"), F_MOVED), (1, CAPTAIN, sq("f8"), F_MOVED),
            (1, SCOUT, sq("g7"), F_MOVED | F_SCOUT),
            (1, MARSHAL, sq("h8"), F_MOVED | F_REVEALED)]
    red = [(0, MARSHAL, sq("e2"), 0), (0, FLAG, sq("a1"), 0)]
    return make_position(red + blue, ply=10)


def _enumerate(pos):
    """All type assignments of blue's hidden pieces consistent with the
    public information, by brute force; returns list of dict pid->type."""
    flags = pos[160:240]
    types = pos[:80]
    hidden = []
    remaining = Counter()
    for t, c in enumerate(COUNTS):
        remaining[t] = c
    for k in range(40):
        pid = 40 + k
        alive = flags[pid] & 1
        if not alive or flags[pid] & F_REVEALED:
            remaining[types[pid]] -= 1
        elif flags[pid] & F_SCOUT:
            remaining[SCOUT] -= 1
        else:
            hidden.append(pid)
    multiset = [t for t, c in remaining.items() for _ in range(c)]
    assert len(multiset) == len(hidden)
    out = set()
    for perm in itertools.permutations(multiset):
        ok = all(not (flags[pid] & F_MOVED and t in (FLAG, BOMB)) for pid, t in zip(hidden, perm))
        if ok:
            out.add(tuple(perm))
    return hidden, sorted(out)


def test_closed_form_marginals_equal_exact_enumeration():
    pos = _tiny_position()
    hidden, assignments = _enumerate(pos)
    num, den = oracle.marginals(pos, 1)
    for i, pid in enumerate(hidden):
        counts = Counter(a[i] for a in assignments)
        for t in range(12):
            exact = Fraction(counts[t], len(assignments))
            assert Fraction(int(num[pid - 40, t]), int(den[pid - 40, t])) == exact, (pid, t)


def test_sampler_frequencies_match_enumeration():
    pos = _tiny_position()
    hidden, assignments = _enumerate(pos)
    K = 20000
    samples = oracle.belief_sample(pos, K, seed=1234)[0]
    # known pieces carry their known type in every sample
    for k in range(40):
        pid = 40 + k
        if pid not in hidden:
            expected = SCOUT if pos[160 + pid] & F_SCOUT and not pos[160 + pid] & F_REVEALED else pos[pid]
            assert (samples[:, k] == expected).all()
    got = Counter(tuple(int(s[pid - 40]) for pid in hidden) for s in samples)
    assert set(got) <= set(assignments)
    expected = K / len(assignments)
    chi2 = sum((got[a] - expected) ** 2 / expected for a in assignments)
    dof = len(assignments) - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof) + 10


def test_samples_are_consistent_on_game_positions():
    g = oracle.play_games(31, 12)
    games = np.repeat(np.arange(12), 6)
    plies = np.concatenate([np.linspace(1, g["lengths"][i] - 1, 6).astype(np.int16) for i in range(12)])
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    samples = oracle.belief_sample(pos, 64, seed=99)
    for b in range(len(pos)):
        p = pos[b]
        opp = 1 - (int(plies[b]) & 1)
        flags = p[160:240]
        for s in samples[b]:
            assert np.array_equal(np.bincount(s, minlength=12), COUNTS)
            for k in range(40):
                pid = 40 * opp + k
                f = flags[pid]
                if not (f & 1) or f & F_REVEALED:
                    assert s[k] == p[pid]
                elif f & F_SCOUT:
                    assert s[k] == SCOUT
                elif f & F_MOVED:
                    assert s[k] not in (FLAG, BOMB)
        # different samples differ (the sampler is not stuck)
        if ((flags[40 * opp:40 * opp + 40] & 1) & ~(flags[40 * opp:40 * opp + 40] >> 1) & 1).sum() > 3:
            assert len({bytes(s) for s in samples[b]}) > 1


def test_stream_ids_select_independent_streams():
    pos = _tiny_position()
    a = oracle.belief_sample(np.stack([pos, pos]), 16, seed=5)
    assert not np.array_equal(a[0], a[1])        # positions 0 and 1 use streams 0 and 1
    b = oracle.belief_sample(np.stack([pos, pos]), 16, seed=5, stream_ids=[1, 1])
    np.testing.assert_array_equal(b[0], a[1])
    np.testing.assert_array_equal(b[1], a[1])


# ------------------------------------------------------------------ rollouts

def _rollout_by_hand(pos, types, seed, stream, sample, depth):
    """Re-derive one rollout by stepping the position one legal move at a
    time with the oracle's primitives and the random-policy key layout."""
    p = pos.copy()
    ply = int(np.frombuffer(p[240:242].tobytes(), np.int16)[0])
    searcher = ply & 1
    opp = 1 - searcher
    p[40 * opp:40 * opp + 40] = types
    code, winner = oracle.start_check(p)
    d = 0
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    while not code and d < depth:
        moves = np.sort(oracle.legal_moves(p))
        w = oracle.philox(np.array([[stream, sample, d, 4 << 24]], np.uint32), key)[0, 0]
        a = moves[(int(w) * len(moves)) >> 32]
        p, code, winner = oracle.apply(p, [a])
        d += 1
    if not code:
        return 3
    if winner < 0:
        return 2
    return 0 if winner == searcher else 1


def test_rollout_matches_step_by_step_rederivation():
    g = oracle.play_games(8, 6)
    games = np.arange(6)
    plies = np.minimum(g["lengths"] - 1, 150).astype(np.int16)
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    K, D, seed = 6, 24, 777
    types = oracle.belief_sample(pos, K, seed)
    tallies, outcomes = oracle.rollout(pos, K, D, seed, want_outcomes=True)
    assert (tallies.sum(1) == K).all()
    for b in range(len(pos)):
        for s in range(K):
            assert outcomes[b, s] == _rollout_by_hand(pos[b], types[b, s], seed, b, s, D)
    # supplying the same samples gives the same tallies
    np.testing.assert_array_equal(oracle.rollout(pos, K, D, seed, types=types), tallies)


def test_rollout_depth_zero_and_long():
    g = oracle.play_games(8, 4)
    pos = oracle.replay_positions(g["setups"], g["actions"], np.arange(4), np.zeros(4, np.int16))
    t0 = oracle.rollout(pos, 5, 0, 1)
    assert (t0[:, 3] == 5).all()
    t = oracle.rollout(pos, 5, 2000, 1)
    assert (t[:, 3] == 0).all() and (t.sum(1) == 5).all()
