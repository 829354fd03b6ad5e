"""Pins of the oracle's rule engine against what the paper fixes (App. A,
Tab. pieces, Tab. chase, App. D.1) and against closed forms, hand positions,
invariants and an independent brute-force move enumerator."""
import os

import numpy as np
import pytest

import oracle
from tests.helpers import (BOMB, CAPTAIN, FLAG, F_MOVED, F_REVEALED, GENERAL, LAKES, MARSHAL, MINER,
                           SCOUT, SERGEANT, SPY, action, field, make_position, sq)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NAMES = ["Spy", "Scout", "Miner", "Sergeant", "Lieutenant", "Captain", "Major", "Colonel",
         "General", "Marshal", "Flag", "Bomb"]


# ------------------------------------------------------------------ battles

def test_battle_table_matches_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "battle_table.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 10
    code = {"W": 1, "L": 2, "T": 3}
    for ta, row in enumerate(rows):
        assert row[0] == NAMES[ta]
        assert len(row) == 13
        for td in range(12):
            assert oracle.battle(ta, td) == code[row[1 + td]], (NAMES[ta], NAMES[td])


def test_battle_in_play_reveals_and_removes():
    # red Spy attacks the blue Marshal: Spy wins (only when attacking)
    pos = make_position([(0, SPY, sq("e4"), 0), (0, FLAG, sq("a1"), 0),
                         (1, MARSHAL, sq("e5"), 0), (1, FLAG, sq("j10"), 0), (1, BOMB, sq("j9"), 0)])
    out, ending, _ = oracle.apply(pos, [action("e4", "e5")])
    spy = 0
    marshal = 40
    assert out[160 + spy] & 1 and out[80 + spy] == sq("e5") and out[160 + spy] & F_REVEALED
    assert not (out[160 + marshal] & 1) and (out[160 + marshal] >> 4) == 6  # hidden defender died
    # blue has only immovable pieces left -> red wins by no-moves
    assert ending == 2
    # the Marshal attacking the Spy wins by rank
    pos = make_position([(0, SPY, sq("e4"), 0), (0, FLAG, sq("a1"), 0), (0, SCOUT, sq("a2"), 0),
                         (1, MARSHAL, sq("e5"), 0), (1, FLAG, sq("j10"), 0)], ply=1)
    out, ending, _ = oracle.apply(pos, [action("e5", "e4")])
    assert not (out[160 + 0] & 1) and (out[160 + 0] >> 4) == 6
    assert out[160 + 40] & 1 and out[80 + 40] == sq("e4")


# ------------------------------------------------------------------ movement

def _lone(side, t, square, ply=0):
    # one movable piece plus both flags tucked into corners far away
    pcs = [(side, t, square, 0), (0, FLAG, sq("j1") if square != sq("j1") else sq("i1"), 0),
           (1, FLAG, sq("j10"), 0)]
    return make_position(pcs, ply=ply)


@pytest.mark.parametrize("square,t,expected", [
    ("a1", SCOUT, 18 - 1),   # a1..a10 and b1..j1, minus the flag parked on j1
    ("c4", SCOUT, 12),       # below the c5 lake
    ("e5", SCOUT, 10),       # between the lakes
    ("e2", MARSHAL, 4),
    ("e2", BOMB, 0),
    ("e2", FLAG, 0),
])
def test_hand_move_counts(square, t, expected):
    if t == FLAG:
        pos = make_position([(0, FLAG, sq(square), 0), (1, FLAG, sq("j10"), 0)])
    else:
        pos = _lone(0, t, sq(square))
    assert len(oracle.legal_moves(pos)) == expected


def test_scout_a1_open_board_is_18():
    # flag on j2 leaves rank 1 and file a open: 9 + 9 moves
    pos = make_position([(0, SCOUT, sq("a1"), 0), (0, FLAG, sq("j2"), 0), (1, FLAG, sq("j10"), 0)])
    moves = oracle.legal_moves(pos)
    assert len(moves) == 18
    assert set(moves % 100) == {sq("a%d" % r) for r in range(2, 11)} | {sq(c + "1") for c in "bcdefghij"}


def test_scout_stops_at_first_enemy_and_before_own():
    pos = make_position([(0, SCOUT, sq("a1"), 0), (0, FLAG, sq("a5"), 0), (1, SERGEANT, sq("d1"), 0),
                         (1, FLAG, sq("j10"), 0)])
    dests = set(oracle.legal_moves(pos) % 100)
    assert dests == {sq("a2"), sq("a3"), sq("a4"), sq("b1"), sq("c1"), sq("d1")}


def front_count(types_red):
    # closed form for red's first move: only the six squares of rank 4 that
    # face open squares can move (b..c and g..h of rank 5 are lakes)
    total = 0
    for s in (30, 31, 34, 35, 38, 39):
        t = types_red[s]
        total += 0 if t in (FLAG, BOMB) else (3 if t == SCOUT else 1)
    return total


@pytest.mark.parametrize("seed", [1, 2, 3, 99, 12345])
def test_initial_position_closed_form_and_perft(seed):
    for slot in range(8):
        types = oracle.setup_types(seed, slot)
        pos = oracle.initial_position(types)
        assert len(oracle.legal_moves(pos)) == front_count(types)
    types = oracle.setup_types(seed, 0)
    pos = oracle.initial_position(types)
    for depth in (1, 2, 3):
        assert oracle.perft(pos, depth) == oracle.perft(pos, depth, brute=True)
    assert oracle.perft(pos, 1) == front_count(types)


def test_generator_matches_brute_enumerator_midgame():
    g = oracle.play_games(7, 16)
    rng = np.random.default_rng(0)
    games = np.repeat(np.arange(16), 12)
    plies = np.array([rng.integers(0, max(1, g["lengths"][i])) for i in games], np.int16)
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    for p in pos:
        phys = oracle.legal_moves(p, physical=True)
        assert np.array_equal(np.sort(phys), oracle.brute_moves(p))


def test_setup_counts_and_uniformity():
    n = 3000
    freq = np.zeros((2, 40, 12))
    for slot in range(n):
        types = oracle.setup_types(11, slot)
        for side in (0, 1):
            assert np.array_equal(np.bincount(types[40 * side:40 * side + 40], minlength=12),
                                  [1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6])
            freq[side, np.arange(40), types[40 * side:40 * side + 40]] += 1
    expected = n * np.array([1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6]) / 40.0
    chi2 = ((freq - expected) ** 2 / expected).sum()
    dof = 2 * 40 * 11
    assert chi2 < dof + 6 * np.sqrt(2 * dof)


# ------------------------------------------------------------------ two-square rule

def test_two_square_one_step_piece():
    # red Captain went e2-e3-e2-e3 on its last three turns: e3-e2 is forbidden, e3-f3 is not
    pos = make_position([(0, CAPTAIN, sq("e3"), F_MOVED), (0, FLAG, sq("a1"), 0), (1, FLAG, sq("j10"), 0),
                         (1, SCOUT, sq("j9"), F_MOVED)],
                        ply=6, ts={0: (0, [sq("e2"), sq("e3"), sq("e2"), sq("e3")])})
    dests = set(oracle.legal_moves(pos) % 100)
    assert sq("e2") not in dests and sq("f3") in dests and sq("d3") in dests and sq("e4") in dests
    assert oracle.two_square_applies(pos) == 1
    off = set(oracle.legal_moves(pos, flags=oracle.RULE_CHASE) % 100)
    assert sq("e2") in off


def test_two_square_scout_pin():
    # scout on rank 1 went a -> c -> b -> d (cols 0,2,1,3): d -> a or b forbidden, d -> c allowed
    pos = make_position([(0, SCOUT, 3, F_MOVED), (0, FLAG, sq("a10"), 0), (1, FLAG, sq("j10"), 0),
                         (1, SCOUT, sq("j9"), F_MOVED)],
                        ply=6, ts={0: (0, [0, 2, 1, 3])})
    dests = set(oracle.legal_moves(pos) % 100)
    assert 0 not in dests and 1 not in dests and 2 in dests and 4 in dests


def _blocked_literal(seq):
    # literal reading: the set of square boundaries each move crosses; the
    # fourth move is forbidden when one boundary is in all four sets
    sets = []
    for a, b in zip(seq[:-1], seq[1:]):
        lo, hi = min(a, b), max(a, b)
        sets.append({x + 0.5 for x in range(lo, hi)})
    return len(set.intersection(*sets)) > 0


def test_two_square_interval_test_vs_boundary_sets():
    # every 3-move history of a scout on an empty rank 1, every 4th move
    rng = np.random.default_rng(3)
    seqs = set()
    while len(seqs) < 400:
        s = [int(rng.integers(0, 10))]
        while len(s) < 4:
            t = int(rng.integers(0, 10))
            if t != s[-1]:
                s.append(t)
        seqs.add(tuple(s))
    for s in seqs:
        pos = make_position([(0, SCOUT, s[3], F_MOVED), (0, FLAG, sq("a10"), 0), (1, FLAG, sq("j10"), 0),
                             (1, SCOUT, sq("j9"), F_MOVED)], ply=6, ts={0: (0, list(s))})
        dests = set(int(m % 100) for m in oracle.legal_moves(pos) if m // 100 == s[3])
        for d in range(10):
            if d == s[3]:
                continue
            assert (d in dests) == (not _blocked_literal(list(s) + [d])), (s, d)


def test_two_square_state_through_play():
    pos = make_position([(0, CAPTAIN, sq("e2"), 0), (0, FLAG, sq("a1"), 0), (1, SERGEANT, sq("e9"), 0),
                         (1, FLAG, sq("j10"), 0)])
    seq = [action("e2", "e3"), action("e9", "e8"), action("e3", "e2"), action("e8", "e9"),
           action("e2", "e3"), action("e9", "e8")]
    out, ending, _ = oracle.apply(pos, seq)
    assert ending == 0
    dests = set(int(m % 100) for m in oracle.legal_moves(out))
    assert sq("e2") not in dests and sq("d3") in dests
    # moving another piece in between resets the count
    pos2 = make_position([(0, CAPTAIN, sq("e2"), 0), (0, GENERAL, sq("a2"), 0), (0, FLAG, sq("a1"), 0),
                          (1, SERGEANT, sq("e9"), 0), (1, FLAG, sq("j10"), 0)])
    seq2 = [action("e2", "e3"), action("e9", "e8"), action("a2", "a3"), action("e8", "e7"),
            action("e3", "e2"), action("e7", "e8"), action("e2", "e3"), action("e8", "e9")]
    out2, ending, _ = oracle.apply(pos2, seq2)
    assert sq("e2") in set(int(m % 100) for m in oracle.legal_moves(out2) if m // 100 == sq("e3"))


# ------------------------------------------------------------------ continuous chasing

def _chase_position():
    # red Captains R1 (b2->..) and R2 (j2), blue Sergeants B1 (b3) and B2 (i3)
    return make_position([(0, CAPTAIN, sq("a2"), 0), (0, CAPTAIN, sq("j2"), 0), (0, FLAG, sq("f1"), 0),
                          (1, SERGEANT, sq("b3"), 0), (1, SERGEANT, sq("i3"), 0), (1, FLAG, sq("f10"), 0)])


def test_chase_repeat_with_two_chasers_is_forbidden():
    seq = [action("a2", "b2"),   # R1 threatens B1 on b3: chase starts
           action("b3", "a3"),   # B1 evades
           action("j2", "i2"),   # R2 threatens B2 on i3
           action("i3", "j3"),   # B2 evades
           action("b2", "a2"),   # R1 threatens B1 on a3
           action("a3", "b3"),   # B1 evades
           action("i2", "j2"),   # R2 threatens B2 on j3
           action("j3", "i3")]   # B2 evades
    out, ending, _ = oracle.apply(_chase_position(), seq)
    assert ending == 0
    assert out[245] == 0 and out[246] == 8      # red chases, 8 plies long
    repeat = action("a2", "b2")                 # recreates the position after the first threat
    assert repeat not in set(oracle.legal_moves(out))
    assert repeat in set(oracle.legal_moves(out, flags=oracle.RULE_TWO_SQUARE))
    # moving the piece moved last turn back to its square is the exception
    assert action("j2", "i2") in set(oracle.legal_moves(out))


def test_chase_return_to_previous_square_is_allowed():
    seq = [action("a2", "b2"), action("b3", "a3"), action("b2", "a2"), action("a3", "b3")]
    out, ending, _ = oracle.apply(_chase_position(), seq)
    assert out[245] == 0 and out[246] == 4
    assert action("a2", "b2") in set(oracle.legal_moves(out))


def test_chase_ends_on_a_quiet_move_and_position_roundtrip():
    seq = [action("a2", "b2"), action("b3", "a3"), action("j2", "j1")]
    out, ending, _ = oracle.apply(_chase_position(), seq)
    assert out[245] == 0xFF and out[246] == 0
    # snapshot round trip rebuilds the chase positions from the history
    seq = [action("a2", "b2"), action("b3", "a3"), action("j2", "i2"), action("i3", "j3"),
           action("b2", "a2"), action("a3", "b3"), action("i2", "j2"), action("j3", "i3")]
    mid, _, _ = oracle.apply(_chase_position(), seq[:4])
    out_a, _, _ = oracle.apply(mid, seq[4:])
    assert action("a2", "b2") not in set(oracle.legal_moves(out_a))


# ------------------------------------------------------------------ endings

def test_ending_flag_capture():
    pos = make_position([(0, MINER, sq("e8"), 0), (0, FLAG, sq("a1"), 0), (1, FLAG, sq("e9"), 0),
                         (1, SCOUT, sq("j9"), 0)])
    _, ending, winner = oracle.apply(pos, [action("e8", "e9")])
    assert (ending, winner) == (1, 0)


def test_ending_no_moves_and_neither_can_move():
    pos = make_position([(0, MARSHAL, sq("e4"), 0), (0, FLAG, sq("a1"), 0), (1, FLAG, sq("j10"), 0),
                         (1, BOMB, sq("j9"), 0)])
    _, ending, winner = oracle.apply(pos, [action("e4", "e5")])
    assert (ending, winner) == (2, 0)
    # both Sergeants die; nobody has a movable piece: draw
    pos = make_position([(0, SERGEANT, sq("e4"), 0), (0, FLAG, sq("a1"), 0), (1, SERGEANT, sq("e5"), 0),
                         (1, FLAG, sq("j10"), 0)])
    _, ending, winner = oracle.apply(pos, [action("e4", "e5")])
    assert (ending, winner) == (3, -1)
    # a fresh position whose acting player cannot move ends at once
    pos = make_position([(0, FLAG, sq("a1"), 0), (0, BOMB, sq("a2"), 0), (1, SCOUT, sq("j9"), 0),
                         (1, FLAG, sq("j10"), 0)])
    assert oracle.start_check(pos) == (2, 1)
    pos = make_position([(0, FLAG, sq("a1"), 0), (1, FLAG, sq("j10"), 0)])
    assert oracle.start_check(pos) == (3, -1)


def test_ending_k_rule_and_cap():
    pcs = [(0, MARSHAL, sq("e4"), 0), (0, FLAG, sq("a1"), 0), (1, SCOUT, sq("j9"), 0), (1, FLAG, sq("j10"), 0)]
    _, ending, _ = oracle.apply(make_position(pcs, ply=120, battleless=99), [action("e4", "e5")])
    assert ending == 4
    _, ending, _ = oracle.apply(make_position(pcs, ply=120, battleless=98), [action("e4", "e5")])
    assert ending == 0
    _, ending, _ = oracle.apply(make_position(pcs, ply=998, battleless=98), [action("e4", "e5")], cap=999)
    assert ending == 5
    # the k-rule is checked before the cap
    _, ending, _ = oracle.apply(make_position(pcs, ply=998, battleless=99), [action("e4", "e5")], cap=999)
    assert ending == 4
    # a battle resets the counter
    pcs2 = [(0, MARSHAL, sq("e4"), 0), (0, FLAG, sq("a1"), 0), (1, SCOUT, sq("e5"), 0),
            (1, SCOUT, sq("j9"), 0), (1, FLAG, sq("j10"), 0)]
    out, ending, _ = oracle.apply(make_position(pcs2, ply=120, battleless=99), [action("e4", "e5")])
    assert ending == 0 and field(out, "battleless") == 0


# ------------------------------------------------------------------ invariants over random play

def _check_invariants(pos, start=None):
    assert oracle.import_check(pos) == 0
    types, squares, flags = pos[:80], pos[80:160], pos[160:240]
    alive = flags & 1
    occupied = squares[alive == 1]
    assert len(set(occupied.tolist())) == len(occupied)
    assert not (set(occupied.tolist()) & LAKES)
    for pid in range(80):
        home = pid if pid < 40 else 60 + pid - 40
        if types[pid] in (FLAG, BOMB) and alive[pid]:
            assert squares[pid] == home and not (flags[pid] & F_MOVED)
        if not alive[pid]:
            assert 1 <= (flags[pid] >> 4) <= 6 and flags[pid] & F_REVEALED


def test_invariants_along_random_games():
    g = oracle.play_games(5, 24)
    assert (g["lengths"] <= 1000).all() and (g["lengths"] >= 1).all()
    assert set(np.unique(g["endings"])) <= {1, 2, 3, 4, 5}
    games = np.repeat(np.arange(24), 20)
    plies = np.concatenate([np.linspace(0, g["lengths"][i], 20).astype(np.int16) for i in range(24)])
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    for p in pos:
        _check_invariants(p)
    # type counts never rise: captured pieces only accumulate along a game
    for i in range(24):
        dead = [(pos[20 * i + j][160:240] & 1 == 0).sum() for j in range(20)]
        assert all(a <= b for a, b in zip(dead[:-1], dead[1:]))


def test_env_run_matches_play_games_first_episode():
    g = oracle.play_games(9, 8)
    r = oracle.env_run(9, 8, 1200, want_mask=False)
    for i in range(8):
        L = g["lengths"][i]
        np.testing.assert_array_equal(r["action"][:L, i], g["actions"][i, :L])
        assert r["done"][L - 1, i] == g["endings"][i]
        assert (r["done"][:L - 1, i] == 0).all()
        assert r["reward"][L - 1, i] == g["rewards"][i]
    # rewards and ending counters agree
    assert r["stats"][:, :5].sum() == (r["done"] > 0).sum()
    assert r["stats"][:, 6].sum() == (r["reward"] > 0).sum()


def test_supplied_actions_are_validated():
    r = oracle.env_run(3, 2, 5, want_mask=True)
    acts = r["action"].copy()
    r2 = oracle.env_run(3, 2, 5, actions=acts)
    np.testing.assert_array_equal(r2["mask"], r["mask"])
    bad = acts.copy()
    bad[2, 1] = 0   # a1 -> a1 is never legal
    with pytest.raises(ValueError):
        oracle.env_run(3, 2, 5, actions=bad)


def test_snapshot_roundtrip():
    g = oracle.play_games(4, 6)
    games = np.repeat(np.arange(6), 5)
    plies = np.concatenate([np.linspace(0, g["lengths"][i] - 1, 5).astype(np.int16) for i in range(6)])
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    for p in pos:
        out, _, _ = oracle.apply(p, [])
        np.testing.assert_array_equal(out, p)
    # continuing from an imported snapshot equals replaying further
    for j, p in enumerate(pos):
        i, t = games[j], plies[j]
        L = g["lengths"][i]
        n = min(L - t, 7)
        if n <= 0:
            continue
        out, _, _ = oracle.apply(p, g["actions"][i, t:t + n])
        ref = oracle.replay_positions(g["setups"], g["actions"], [i], [t + n])[0]
        np.testing.assert_array_equal(out, ref)


def test_import_rejects_corrupt_rule_state():
    # the snapshot checks the GPU import makes (App. B.2 two-square record;
    # chase history), one corrupt field at a time on a valid position
    pcs = [(0, MARSHAL, sq("e4"), F_MOVED), (0, FLAG, sq("a1"), 0), (1, SCOUT, sq("e6"), F_MOVED),
           (1, FLAG, sq("j10"), 0)]
    good = make_position(pcs, ply=4, battleless=4, ts={0: (0, [sq("e3"), sq("e4")])})
    assert oracle.import_check(good) == 0
    bad = good.copy(); bad[248] = 100                    # two-square piece id beyond the 80 pieces
    assert oracle.import_check(bad) == -8
    bad = good.copy(); bad[253] = 100                    # a two-square square off the board
    assert oracle.import_check(bad) == -8
    bad = good.copy(); bad[253] = sq("c5")               # a two-square square in a lake
    assert oracle.import_check(bad) == -8
    # a chase whose history move starts off the board
    chase = make_position(pcs, ply=4, battleless=4, chaser=0, chase_plies=1, hist=[65000])
    assert oracle.import_check(chase) == -12


def test_online_200_move_rule_and_the_rule_fractions():
    # App. A "Additional rule for online play" and App. D.1: the online game
    # draws after 200 battleless moves, and channels 41-42 (App. C.1) give
    # ply / max plies and battleless / k.  Values below are worked by hand:
    # 151/200 -> uint8 floor(255*151/200 + 1/2) = 193, bf16 193/256 = 0x3F41;
    # 161/4000 -> uint8 floor(10.26 + 1/2) = 10, bf16 165/4096 = 0x3D25.
    pcs = [(0, MARSHAL, sq("e4"), 0), (0, FLAG, sq("a1"), 0), (1, SCOUT, sq("j9"), 0), (1, FLAG, sq("j10"), 0)]
    mv = [action("e4", "e5")]
    out, ending, _, u8, bf = oracle.apply(make_position(pcs, ply=160, battleless=150), mv, k=200, cap=4000,
                                          planes=True)
    assert ending == 0 and field(out, "battleless") == 151
    assert (u8[42] == 193).all() and (bf[42] == 0x3F41).all()
    assert (u8[41] == 10).all() and (bf[41] == 0x3D25).all()
    # the same move ends the game under the 100-move rule, and under the
    # 200-move rule once 200 battleless plies are reached
    _, ending, _ = oracle.apply(make_position(pcs, ply=160, battleless=150), mv, k=100)
    assert ending == 4
    _, ending, _ = oracle.apply(make_position(pcs, ply=300, battleless=199), mv, k=200, cap=4000)
    assert ending == 4
    _, ending, _ = oracle.apply(make_position(pcs, ply=300, battleless=198), mv, k=200, cap=4000)
    assert ending == 0
