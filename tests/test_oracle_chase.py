"""The continuous-chasing rule (App. A, Tab. chase and the rule under it;
App. B.3) re-derived from the move list alone and compared with the oracle.

A second, literal tracker written here in plain Python replays each game
from its setup and action list with the hand-written battle table of
tests/golden: it keeps the board of piece ids, classifies every move as a
battle, evade, threat or quiet move, runs the chase state (chaser, chase
length, the positions after each of the chaser's threats) and lists the
moves the rule forbids.  Nothing of it comes from the oracle: at every ply
its board, chaser and chase length must equal the oracle's snapshot, and
the oracle's legal moves under the chasing rule alone must equal the
oracle's brute-force enumerator of physical moves (a separate code path)
minus the moves this tracker forbids.

Readings (the paper states the rule in prose): a threat is a non-battle
move ending orthogonally next to an enemy piece; an evade is a non-battle
move of a piece that stood next to where the opponent's previous move
ended (that move not a battle), to a square not next to it; evade takes
precedence.  A threat by the chaser continues the chase, any other threat
starts one; an evade by the chased side keeps it; anything else ends it.
A chase position is the piece-id occupancy after one of the chaser's
threats; while P chases, a threat recreating one is forbidden unless it
moves the piece P moved last turn back to that move's from-square.
"""
import os

import numpy as np
import pytest

import oracle
from tests.helpers import CAPTAIN, FLAG, SERGEANT, action, make_position, sq

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BATTLE, QUIET, THREAT, EVADE = 0, 1, 2, 3


def _battle_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "battle_table.txt")) if l.strip() and l[0] != "#"]
    return [[r[1 + d] for d in range(12)] for r in rows]


TABLE = _battle_table()


def _nbrs(s):
    r, c = divmod(s, 10)
    out = []
    if r > 0:
        out.append(s - 10)
    if r < 9:
        out.append(s + 10)
    if c > 0:
        out.append(s - 1)
    if c < 9:
        out.append(s + 1)
    return out


def _adjacent(a, b):
    return b in _nbrs(a)


class ChaseTracker:
    """Board of piece ids (-1 empty) and the chase state, from the moves."""

    def __init__(self, types):
        self.types = [int(t) for t in types]
        self.board = [-1] * 100
        for pid in range(80):
            self.board[pid if pid < 40 else pid + 20] = pid
        self.ply = 0
        self.prev = None          # (to, was_battle) of the previous ply
        self.last = [None, None]  # (from, to) of each player's previous move
        self.chaser = None
        self.length = 0
        self.positions = []

    def side(self, pid):
        return pid // 40

    def enemy_at(self, s, P):
        p = self.board[s]
        return p >= 0 and self.side(p) != P

    def classify(self, frm, to):
        P = self.ply & 1
        if self.board[to] >= 0:
            return BATTLE
        if self.prev is not None:
            pto, pbattle = self.prev
            if not pbattle and self.enemy_at(pto, P) and _adjacent(frm, pto) and not _adjacent(to, pto):
                return EVADE
        if any(self.enemy_at(n, P) for n in _nbrs(to)):
            return THREAT
        return QUIET

    def after(self, frm, to):
        """Board tuple after a non-battle move."""
        b = list(self.board)
        b[to], b[frm] = b[frm], -1
        return tuple(b)

    def forbidden(self, moves):
        """The moves of the player to move that the chasing rule forbids."""
        P = self.ply & 1
        if self.chaser != P or not self.positions:
            return set()
        seen = set(self.positions)
        out = set()
        back = self.last[P]
        for a in moves:
            frm, to = divmod(int(a), 100)
            if self.classify(frm, to) != THREAT:
                continue
            if back is not None and frm == back[1] and to == back[0]:
                continue
            if self.after(frm, to) in seen:
                out.add(int(a))
        return out

    def play(self, a):
        P = self.ply & 1
        frm, to = divmod(int(a), 100)
        cls = self.classify(frm, to)
        X = self.board[frm]
        assert X >= 0 and self.side(X) == P
        if cls == BATTLE:
            D = self.board[to]
            res = TABLE[self.types[X]][self.types[D]]
            self.board[frm] = -1
            self.board[to] = X if res == "W" else (D if res == "L" else -1)
        else:
            self.board[to], self.board[frm] = X, -1
        if cls == THREAT:
            if self.chaser == P:
                self.positions.append(tuple(self.board))
                self.length += 1
            else:
                self.chaser, self.positions, self.length = P, [tuple(self.board)], 1
        elif cls == EVADE and self.chaser == 1 - P:
            self.length += 1
        else:
            self.chaser, self.positions, self.length = None, [], 0
        self.prev = (to, cls == BATTLE)
        self.last[P] = (frm, to)
        self.ply += 1


def _board_of(pos):
    b = [-1] * 100
    for pid in range(80):
        if pos[160 + pid] & 1:
            b[int(pos[80 + pid])] = pid
    return b


def _check_game(setup, acts):
    """Step one game; returns the number of moves the rule forbade."""
    T = ChaseTracker(setup)
    L = len(acts)
    pos = oracle.replay_positions(setup[None, :], acts[None, :], np.zeros(L + 1, np.int32),
                                  np.arange(L + 1, dtype=np.int16))
    blocked = 0
    for t in range(L + 1):
        p = pos[t]
        assert _board_of(p) == T.board, t
        assert p[245] == (0xFF if T.chaser is None else T.chaser), t
        assert p[246] == T.length, t
        phys = oracle.brute_moves(p)
        forb = T.forbidden(phys)
        blocked += len(forb)
        want = sorted(set(int(a) for a in phys) - forb)
        got = sorted(int(a) for a in oracle.legal_moves(p, flags=oracle.RULE_CHASE))
        assert got == want, (t, sorted(forb))
        if t < L:
            T.play(acts[t])
    return blocked


def test_chase_state_over_random_games():
    # uniform random play (the oracle's own games): state and legal moves
    # agree at every ply
    for seed in (3, 17):
        g = oracle.play_games(seed, 25)
        for i in range(25):
            L = min(int(g["lengths"][i]), 400)
            _check_game(g["setups"][i], g["actions"][i, :L].copy())


def _chasing_game(seed, plies):
    """A game whose players seek cycles of chasing: each side plays a threat
    or an evade whenever the full rules allow one, preferring to replay its
    move of four turns ago or to take back its move of two turns ago or of
    last turn (two pieces taking turns in such a loop recreate the chase
    positions), else any legal move; a numpy generator of the given seed
    decides among equals.  Returns (setup, actions)."""
    rng = np.random.default_rng(seed)
    setup = oracle.setup_types(seed, 0)
    pos = oracle.initial_position(setup)
    T = ChaseTracker(setup)
    acts = []
    own = [[], []]
    for _ in range(plies):
        legal = [int(a) for a in oracle.legal_moves(pos)]
        if not legal:
            break
        P = T.ply & 1
        h = own[P]
        cand = [a for a in legal if T.classify(a // 100, a % 100) in (THREAT, EVADE)] or legal
        prefs = []
        if len(h) >= 4:
            prefs.append(h[-4])
        if len(h) >= 2:
            prefs.append((h[-2] % 100) * 100 + h[-2] // 100)
        if h:
            prefs.append((h[-1] % 100) * 100 + h[-1] // 100)
        pick = None
        for a in prefs:
            if a in cand and rng.random() < 0.9:
                pick = a
                break
        if pick is None:
            pick = cand[int(rng.integers(len(cand)))]
        pos, ending, _ = oracle.apply(pos, [pick])
        T.play(pick)
        acts.append(pick)
        own[P].append(pick)
        if ending:
            break
    return setup, np.array(acts, np.int16)


def test_chase_state_and_forbidden_moves_over_chasing_games():
    # 50 games played by chase-seeking players, every ply compared; the rule
    # must have forbidden moves in this sample
    blocked = 0
    for seed in range(50):
        setup, acts = _chasing_game(1000 + seed, 200)
        blocked += _check_game(setup, acts)
    assert blocked > 0


def _hand_setup_game(pcs, moves):
    """A hand position stepped through `moves`, checked ply by ply."""
    pos = make_position(pcs)
    T = ChaseTracker(pos[:80])
    T.board = _board_of(pos)
    blocked = 0
    cur = pos
    for t in range(len(moves) + 1):
        assert _board_of(cur) == T.board
        assert cur[245] == (0xFF if T.chaser is None else T.chaser)
        assert cur[246] == T.length
        phys = oracle.brute_moves(cur)
        forb = T.forbidden(phys)
        blocked += len(forb)
        got = sorted(int(a) for a in oracle.legal_moves(cur, flags=oracle.RULE_CHASE))
        assert got == sorted(set(int(a) for a in phys) - forb)
        if t < len(moves):
            cur, ending, _ = oracle.apply(cur, [moves[t]])
            assert ending == 0
            T.play(moves[t])
    return blocked, T


def test_hand_chase_loop_forbids_the_repeat():
    pcs = [(0, CAPTAIN, sq("a2"), 0), (0, CAPTAIN, sq("j2"), 0), (0, FLAG, sq("f1"), 0),
           (1, SERGEANT, sq("b3"), 0), (1, SERGEANT, sq("i3"), 0), (1, FLAG, sq("f10"), 0)]
    seq = [action("a2", "b2"), action("b3", "a3"), action("j2", "i2"), action("i3", "j3"),
           action("b2", "a2"), action("a3", "b3"), action("i2", "j2"), action("j3", "i3")]
    blocked, T = _hand_setup_game(pcs, seq)
    assert T.chaser == 0 and T.length == 8
    # recreating the position after the first threat is forbidden; moving the
    # piece moved last turn back to its square is the exception
    assert T.forbidden([action("a2", "b2"), action("j2", "i2")]) == {action("a2", "b2")}
    assert blocked >= 1


def test_tracker_classes_on_hand_moves():
    # the tracker's own classes, worked by hand
    pcs = [(0, CAPTAIN, sq("a2"), 0), (0, FLAG, sq("f1"), 0), (1, SERGEANT, sq("b3"), 0), (1, FLAG, sq("f10"), 0)]
    pos = make_position(pcs)
    T = ChaseTracker(pos[:80])
    T.board = _board_of(pos)
    assert T.classify(sq("a2"), sq("b2")) == THREAT     # ends next to b3
    assert T.classify(sq("a2"), sq("a3")) == THREAT     # ends next to b3
    assert T.classify(sq("a2"), sq("a1")) == QUIET
    T.play(action("a2", "b2"))
    assert T.classify(sq("b3"), sq("a3")) == EVADE      # b3 stood next to b2, a3 is not next to b2
    assert T.classify(sq("b3"), sq("c3")) == EVADE
    assert T.classify(sq("b3"), sq("b4")) == EVADE
    assert T.classify(sq("b3"), sq("b2")) == BATTLE
    T.play(action("b3", "b4"))
    assert T.chaser == 0 and T.length == 2
    assert T.classify(sq("b2"), sq("b3")) == THREAT     # next to b4
