"""Builders for hand-made test positions in the 784-byte snapshot layout.

The layout (documented with the oracle and in include/stratego.h):
type[80] | square[80] | flags[80] | int16 ply | int16 battleless |
last_battle | chaser | chase_plies | 0 | ts_pid[2] | ts_len[2] | ts_sq[2][4] |
12 zero bytes | uint16 hist[256].
"""
import numpy as np

COUNTS = [1, 8, 5, 4, 4, 4, 3, 2, 1, 1, 1, 6]
SPY, SCOUT, MINER, SERGEANT, LIEUTENANT, CAPTAIN, MAJOR, COLONEL, GENERAL, MARSHAL, FLAG, BOMB = range(12)
LAKES = {42, 43, 46, 47, 52, 53, 56, 57}
F_ALIVE, F_REVEALED, F_MOVED, F_SCOUT = 1, 2, 4, 8


def sq(name):
    """Algebraic square name (file a-j, rank 1-10) -> index 10*row + col."""
    col = ord(name[0]) - ord("a")
    row = int(name[1:]) - 1
    return 10 * row + col


def make_position(pieces, ply=0, battleless=0, last_battle=0, chaser=0xFF, chase_plies=0,
                  ts=None, hist=()):
    """pieces: list of (side, type, square, flags).  Every other piece of each
    side is dead (captured) with a type that completes the side's counts; dead
    pieces sit at their start square with cause 0xFF-free flags (revealed)."""
    pos = np.zeros(784, np.uint8)
    left = [list(COUNTS), list(COUNTS)]
    slots = [[], []]
    for side, t, s, fl in pieces:
        left[side][t] -= 1
        assert left[side][t] >= 0, "too many pieces of a type"
        slots[side].append((t, s, fl))
    for side in (0, 1):
        k = 0
        for t, s, fl in slots[side]:
            pid = side * 40 + k
            pos[pid] = t
            pos[80 + pid] = s
            pos[160 + pid] = fl | F_ALIVE
            k += 1
        for t in range(12):
            for _ in range(left[side][t]):
                pid = side * 40 + k
                pos[pid] = t
                pos[80 + pid] = 0
                pos[160 + pid] = F_REVEALED | (4 << 4)  # captured (cause 4)
                k += 1
        assert k == 40
    pos[240:242] = np.frombuffer(np.int16(ply).tobytes(), np.uint8)
    pos[242:244] = np.frombuffer(np.int16(battleless).tobytes(), np.uint8)
    pos[244] = last_battle
    pos[245] = chaser
    pos[246] = chase_plies
    pos[248:250] = 0xFF
    pos[252:260] = 0xFF
    if ts:
        for player, (pid, squares) in ts.items():
            pos[248 + player] = pid
            pos[250 + player] = len(squares)
            for i, s in enumerate(squares):
                pos[252 + 4 * player + i] = s
    h = np.full(256, 0xFFFF, np.uint16)
    for i, a in enumerate(hist):
        h[i] = a
    pos[272:] = np.frombuffer(h.tobytes(), np.uint8)
    return pos


def pid_at(pos, square):
    for pid in range(80):
        if pos[160 + pid] & F_ALIVE and pos[80 + pid] == square:
            return pid
    return None


def field(pos, name):
    if name == "ply":
        return int(np.frombuffer(pos[240:242].tobytes(), np.int16)[0])
    if name == "battleless":
        return int(np.frombuffer(pos[242:244].tobytes(), np.int16)[0])
    if name == "hist":
        return np.frombuffer(pos[272:].tobytes(), np.uint16)
    raise KeyError(name)


def action(a, b):
    return sq(a) * 100 + sq(b)
