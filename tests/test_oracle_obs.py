"""Pins of the oracle's observation planes (App. C): exact rounding of the
ratio channels, hand scenarios for the feature groups, and invariants that
hold on every position."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.helpers import (BOMB, CAPTAIN, FLAG, F_MOVED, F_REVEALED, F_SCOUT, LAKES, MARSHAL, MINER,
                           SCOUT, SERGEANT, SPY, action, make_position, sq)


# ------------------------------------------------------------------ value encodings

def _bf16_from_f64(x):
    # round-to-nearest-even of a float64 to bf16 by integer arithmetic on its bits
    bits = np.asarray(x, np.float64).view(np.uint64)
    sign = (bits >> 63).astype(np.uint64)
    exp = ((bits >> 52) & 0x7FF).astype(np.int64)
    man = (bits & ((1 << 52) - 1)).astype(np.uint64)
    keep = man >> 45                      # top 7 mantissa bits
    rest = man & ((1 << 45) - 1)
    half = np.uint64(1 << 44)
    up = (rest > half) | ((rest == half) & ((keep & 1) == 1))
    keep = keep + up.astype(np.uint64)
    exp = exp + (keep >> 7).astype(np.int64)
    keep = keep & 0x7F
    out = (sign << 15) | ((exp - 1023 + 127).astype(np.uint64) << 7) | keep
    out = np.where(np.asarray(x) == 0, 0, out)
    return out.astype(np.uint16)


def test_ratio_encodings_exhaustive_small_denominators():
    den = np.concatenate([np.full(d + 1, d) for d in range(1, 401)]).astype(np.uint32)
    num = np.concatenate([np.arange(d + 1) for d in range(1, 401)]).astype(np.uint32)
    bf, u8 = oracle.ratio_batch(num, den)
    np.testing.assert_array_equal(bf, _bf16_from_f64(num / den))
    # uint8 = round half up of 255*num/den
    ref = np.floor(255.0 * num / den + 0.5).astype(np.uint8)
    exact_half = (510 * num.astype(np.int64)) % (2 * den) == den
    np.testing.assert_array_equal(u8[~exact_half], ref[~exact_half])
    for n, d in zip(num[exact_half][:200], den[exact_half][:200]):
        assert oracle.u8_ratio(n, d) == int(Fraction(255 * int(n), int(d)) + Fraction(1, 2))


def test_ratio_fp32_double_rounding_is_exact_for_plane_denominators():
    # IEEE fp32 division followed by RNE to bf16 gives the exactly rounded
    # value for every num <= den <= 1600 (the largest plane denominator is 40*33)
    torch = pytest.importorskip("torch")
    den = np.concatenate([np.full(d + 1, d) for d in range(1, 1601)]).astype(np.uint32)
    num = np.concatenate([np.arange(d + 1) for d in range(1, 1601)]).astype(np.uint32)
    bf, _ = oracle.ratio_batch(num, den)
    q = (torch.from_numpy(num.astype(np.float32)) / torch.from_numpy(den.astype(np.float32)))
    gpu_style = q.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(bf, gpu_style)


# ------------------------------------------------------------------ invariants on random positions

def _positions(seed=21, n_games=10, per_game=8):
    g = oracle.play_games(seed, n_games)
    games = np.repeat(np.arange(n_games), per_game)
    plies = np.concatenate([np.linspace(0, g["lengths"][i] - 1, per_game).astype(np.int16)
                            for i in range(n_games)])
    return g, games, plies


def test_plane_invariants():
    g, games, plies = _positions()
    u8, bf, mask = oracle.obs_encode(g["setups"], g["actions"], games, plies)
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    for b in range(len(games)):
        P = int(plies[b]) & 1
        p = pos[b]
        types, squares, flags = p[:80], p[80:160], p[160:240]
        alive = (flags & 1) == 1
        revealed = (flags & F_REVEALED) != 0
        x = u8[b].reshape(487, 100)
        y = bf[b].reshape(487, 100)
        # u8 and bf16 agree on indicator and history values
        ind = np.r_[0:12, 36:41, 43:355, 355:487]
        assert np.array_equal(y[ind] == 0x3F80, x[ind] == 1)
        assert np.array_equal(y[ind] == 0xBF80, x[ind] == 255)
        assert set(np.unique(x[ind])) <= {0, 1, 255}
        own = np.zeros(100, bool)
        opp = np.zeros(100, bool)
        for pid in range(80):
            if alive[pid]:
                (own if pid // 40 == P else opp)[squares[pid]] = True
        # 0-11: one type bit per own square, nothing elsewhere
        assert np.array_equal(x[0:12].sum(0), own.astype(int))
        for pid in range(80):
            if alive[pid] and pid // 40 == P:
                assert x[types[pid], squares[pid]] == 1
        # 12-23 sum to 1 on opponent squares (exact rationals), 24-35 on own squares
        for side, base, occ in ((1 - P, 12, opp), (P, 24, own)):
            num, den = oracle.marginals(p, side)
            for k in range(40):
                pid = side * 40 + k
                if not alive[pid]:
                    continue
                assert sum(Fraction(int(num[k, t]), int(den[k, t])) for t in range(12)) == 1
                for t in range(12):
                    assert x[base + t, squares[pid]] == oracle.u8_ratio(num[k, t], den[k, t])
                    assert y[base + t, squares[pid]] == oracle.bf16_ratio(num[k, t], den[k, t])
            assert (x[base:base + 12][:, ~occ] == 0).all()
        # partition: own hidden, opp hidden, empty, own revealed, opp revealed, lake
        cls = x[36].astype(int) + x[37] + x[38]
        for pid in range(80):
            if alive[pid] and revealed[pid]:
                cls[squares[pid]] += 1
        for s in LAKES:
            cls[s] += 1
        assert (cls == 1).all()
        # 355-454: one start square per occupied square
        assert np.array_equal(x[355:455].sum(0), (own | opp).astype(int))
        for pid in range(80):
            if alive[pid]:
                start = pid if pid < 40 else 60 + pid - 40
                assert x[355 + start, squares[pid]] == 1
        # constant fraction planes
        assert (x[41] == oracle.u8_ratio(int(plies[b]), 1000)).all()
        # history: one +1 and one -1 for each of the last min(ply, 32) moves
        for j in range(32):
            plane = x[455 + j]
            if j < plies[b]:
                assert (plane == 1).sum() == 1 and (plane == 255).sum() == 1
            else:
                assert (plane == 0).all()
        # captured planes count every dead piece except flags
        for side, base in ((P, 109), (1 - P, 120)):
            dead = [pid for pid in range(side * 40, side * 40 + 40) if not alive[pid] and types[pid] != FLAG]
            assert x[base:base + 11].sum() == len(dead)
        # mask: the acting player's legal moves
        moves = oracle.legal_moves(p)
        bits = np.unpackbits(mask[b], bitorder="little")
        assert set(np.nonzero(bits)[0]) == set(moves.tolist())


# ------------------------------------------------------------------ hand scenarios

def _planes_after(pcs, seq, **kw):
    pos = make_position(pcs, **kw)
    out, ending, winner, u8, bf = oracle.apply(pos, seq, planes=True)
    return out, u8


def test_threat_and_evade_channels():
    pcs = [(0, CAPTAIN, sq("a2"), 0), (0, FLAG, sq("f1"), 0), (1, SERGEANT, sq("b3"), 0),
           (1, FLAG, sq("f10"), 0)]
    # red Captain threatens the hidden Sergeant; planes seen by blue (to move)
    out, x = _planes_after(pcs, [action("a2", "b2")])
    assert x[76 + 10, sq("b2")] == 1          # opponent piece threatened a hidden piece
    assert x[43:76].sum() == 0
    # blue evades: from red's view (to move) the opponent piece evaded a hidden threatener
    out, x = _planes_after(pcs, [action("a2", "b2"), action("b3", "a3")])
    assert x[43 + 10, sq("b2")] == 1          # own threat bit persists
    assert x[87 + 10, sq("a3")] == 1          # opponent evade from hidden
    # a revealed threatener is recorded by rank
    pcs_r = [(0, CAPTAIN, sq("a2"), F_REVEALED), (0, FLAG, sq("f1"), 0), (1, SERGEANT, sq("b3"), 0),
             (1, FLAG, sq("f10"), 0)]
    out, x = _planes_after(pcs_r, [action("a2", "b2"), action("b3", "a3")])
    assert x[87 + CAPTAIN, sq("a3")] == 1


def test_active_adjacency_channel():
    # red Marshal next to a hidden blue Scout and a revealed blue Sergeant; red plays elsewhere
    pcs = [(0, MARSHAL, sq("e4"), 0), (0, CAPTAIN, sq("a1"), 0), (0, FLAG, sq("j1"), 0),
           (1, SCOUT, sq("e5"), 0), (1, SERGEANT, sq("f4"), F_REVEALED), (1, FLAG, sq("j10"), 0)]
    out, x = _planes_after(pcs, [action("a1", "a2")])
    # seen by blue: the opponent's Marshal was actively adjacent to hidden and to a Sergeant
    assert x[98 + 10, sq("e4")] == 1 and x[98 + SERGEANT, sq("e4")] == 1
    # playing the attack does not mark the chosen target
    out, x = _planes_after(pcs, [action("e4", "f4")])
    assert x[98 + 10, sq("f4")] == 1 and x[98 + SERGEANT, sq("f4")] == 0


def test_protection_channels():
    # red Captain A threatens blue Sergeant B; blue Miner C steps next to B
    pcs = [(0, CAPTAIN, sq("d2"), 0), (0, FLAG, sq("j1"), 0),
           (1, SERGEANT, sq("e3"), 0), (1, MINER, sq("g4"), 0), (1, FLAG, sq("j10"), 0)]
    out, x = _planes_after(pcs, [action("d2", "e2"), action("g4", "f4"), action("e2", "d2")])
    # planes seen by blue (to move): own C at f4, own B at e3
    assert out[240] == 3
    # f4 is adjacent to e3?  no: f4 = (3,5), e3 = (2,4) -> diagonal, so nothing yet
    assert x[251:355].sum() == 0
    out, x = _planes_after(pcs, [action("d2", "e2"), action("g4", "f4")])
    pcs2 = [(0, CAPTAIN, sq("d2"), 0), (0, FLAG, sq("j1"), 0),
            (1, SERGEANT, sq("e3"), 0), (1, MINER, sq("g3"), 0), (1, FLAG, sq("j10"), 0)]
    out, x = _planes_after(pcs2, [action("d2", "e2"), action("g3", "f3"), action("e2", "d2")])
    # blue's view: own Miner C (f3) protected a hidden piece and an empty square
    # (f2, next to e2, empty and newly adjacent), against a hidden piece
    assert x[263, sq("f3")] == 1
    assert x[262, sq("f3")] == 1
    assert x[276, sq("f3")] == 1
    # own Sergeant B (e3) was protected by a hidden piece, against a hidden piece
    assert x[289, sq("e3")] == 1 and x[302, sq("e3")] == 1
    assert x[275].sum() == 0 and x[288].sum() == 0 and x[301].sum() == 0


def test_death_and_capture_channels():
    # red Sergeant attacks a hidden blue Captain and dies: cause 3 for red, at e5
    pcs = [(0, SERGEANT, sq("e4"), 0), (0, SCOUT, sq("a1"), 0), (0, FLAG, sq("j1"), 0),
           (1, CAPTAIN, sq("e5"), 0), (1, SCOUT, sq("a10"), 0), (1, FLAG, sq("j10"), 0)]
    out, x = _planes_after(pcs, [action("e4", "e5")])
    # seen by blue: opponent death, cause 3, Sergeant, at e5; captured on its start square (pid 0 -> a1)
    assert x[191 + 20 + SERGEANT, sq("e5")] == 1
    assert x[120 + SERGEANT, 0] == 1
    # now the Captain is revealed; a red Marshal... a red Scout attacks it and dies: cause 1
    pcs2 = [(0, SERGEANT, sq("e4"), 0), (0, SCOUT, sq("e7"), F_MOVED), (0, FLAG, sq("j1"), 0),
            (1, CAPTAIN, sq("e5"), 0), (1, SCOUT, sq("a10"), 0), (1, FLAG, sq("j10"), 0)]
    out, x = _planes_after(pcs2, [action("e4", "e5"), action("a10", "a9"), action("e7", "e6"),
                                  action("a9", "a10"), action("e6", "e5")])
    assert x[191 + 0 + SCOUT, sq("e5")] == 1 and x[191 + 20 + SERGEANT, sq("e5")] == 1
    # blue Captain survived twice and is revealed: not hidden (37 from red... blue to move: own hidden 36)
    assert x[36, sq("e5")] == 0


def test_history_planes_orientation():
    pcs = [(0, CAPTAIN, sq("a2"), 0), (0, FLAG, sq("f1"), 0), (1, SERGEANT, sq("b3"), 0),
           (1, FLAG, sq("f10"), 0)]
    out, x = _planes_after(pcs, [action("a2", "b2"), action("b3", "a3")])
    assert x[455, sq("a3")] == 1 and x[455, sq("b3")] == 255
    assert x[456, sq("b2")] == 1 and x[456, sq("a2")] == 255
    assert x[457].sum() == 0


# ------------------------------------------------------------------ causes of death, one per case

def _deaths_at(x, square):
    """(channel, value) of every death channel (131-250) set at `square`."""
    return sorted((int(c), int(x[c, square])) for c in range(131, 251) if x[c, square])


# App. C.1 "Causes of death": the attacker A dies by cause 1 (defender
# revealed, A lost), 2 (defender revealed, a tie) or 3 (defender hidden, A
# lost or tied); the defender D dies by cause 4 (D revealed, lost), 5 (D
# revealed, a tie) or 6 (D hidden).  Channel 131 + 10*(cause-1) + rank index
# for own pieces, 191 + ... for the opponent's, at the battle square.
@pytest.mark.parametrize("name,att,dfn,d_flags,red_cause,blue_cause", [
    ("revealed defender wins", SERGEANT, CAPTAIN, F_REVEALED, 1, None),
    ("tie with a revealed defender", CAPTAIN, CAPTAIN, F_REVEALED, 2, 5),
    ("hidden defender wins", SERGEANT, CAPTAIN, 0, 3, None),
    ("tie with a hidden defender", CAPTAIN, CAPTAIN, 0, 3, 6),
    ("revealed defender loses", MARSHAL, CAPTAIN, F_REVEALED, None, 4),
    ("hidden defender loses", MARSHAL, CAPTAIN, 0, None, 6),
])
def test_death_cause_of_each_case(name, att, dfn, d_flags, red_cause, blue_cause):
    pcs = [(0, att, sq("e4"), 0), (0, SCOUT, sq("a2"), 0), (0, FLAG, sq("j1"), 0),
           (1, dfn, sq("e5"), d_flags), (1, SCOUT, sq("a9"), 0), (1, FLAG, sq("j10"), 0)]
    red, blue = 0, 40                      # the attacker and the defender are each side's first piece
    out, x = _planes_after(pcs, [action("e4", "e5")])
    # the snapshot keeps the cause in flag bits 4-6 and the battle square
    for pid, cause in ((red, red_cause), (blue, blue_cause)):
        if cause is None:
            assert out[160 + pid] & 1 and out[160 + pid] & F_REVEALED, name
        else:
            assert not (out[160 + pid] & 1), name
            assert (out[160 + pid] >> 4) & 7 == cause, name
            assert out[80 + pid] == sq("e5"), name
    # blue (the defender's side) to move: own deaths 131.., opponent deaths 191..
    want_blue = []
    if blue_cause is not None:
        want_blue.append((131 + 10 * (blue_cause - 1) + dfn, 1))
    if red_cause is not None:
        want_blue.append((191 + 10 * (red_cause - 1) + att, 1))
    assert _deaths_at(x, sq("e5")) == sorted(want_blue), name
    # red's view after a quiet blue move: the same deaths with own and opponent swapped
    out, x = _planes_after(pcs, [action("e4", "e5"), action("a9", "a8")])
    want_red = []
    if red_cause is not None:
        want_red.append((131 + 10 * (red_cause - 1) + att, 1))
    if blue_cause is not None:
        want_red.append((191 + 10 * (blue_cause - 1) + dfn, 1))
    assert _deaths_at(x, sq("e5")) == sorted(want_red), name


def test_bomb_death_has_no_death_channel_but_a_capture_plane():
    # a Miner defuses a revealed Bomb: cause 4 in the snapshot; the death
    # channels list ten ranks per cause (Bomb dropped), the captured planes
    # 109-130 keep the Bomb (index 10) on its start square
    pcs = [(0, MINER, sq("e4"), 0), (0, FLAG, sq("j1"), 0),
           (1, BOMB, sq("e5"), F_REVEALED), (1, SCOUT, sq("a9"), 0), (1, FLAG, sq("j10"), 0)]
    out, x = _planes_after(pcs, [action("e4", "e5")])
    assert not (out[160 + 40] & 1) and (out[160 + 40] >> 4) & 7 == 4
    assert _deaths_at(x, sq("e5")) == []
    assert x[109 + 10, 60] == 1           # blue's own captured Bomb at the start square of piece 40 (a7)
