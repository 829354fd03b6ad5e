"""Python access to the Stratego oracle (plain single-threaded C).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports this package, and this package never imports the product.

Every function takes and returns numpy arrays; positions are the 784-byte
snapshot layout documented in ``rules.c``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

POS_BYTES = 784
MASK_BYTES = 1264
NCHAN = 487
RULE_TWO_SQUARE = 1
RULE_CHASE = 2
ALL_RULES = RULE_TWO_SQUARE | RULE_CHASE
ROLLOUT_MAGNET = 0x100   # rollouts and search: the magnet policy instead of uniform

_lib = None


def lib():
    """The oracle library: liboracle.so built here, or the file that
    STRATEGO_ORACLE_LIB names (a sanitizer build, for the tests)."""
    global _lib
    if _lib is None:
        path = os.environ.get("STRATEGO_ORACLE_LIB") or _build.build()
        _lib = ctypes.CDLL(path)
        _declare(_lib)
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _declare(L):
    vp, i32, u64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32
    L.orx_env_run.argtypes = [u64, i32, i32, i32, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp, i32,
                              i32, vp, vp]
    L.orx_play_games.argtypes = [u64, i32, i32, i32, i32, vp, vp, vp, vp, vp]
    L.orx_replay_positions.argtypes = [vp, vp, i32, vp, vp, i32, i32, i32, i32, vp]
    L.orx_obs_encode.argtypes = [vp, vp, i32, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp]
    L.orx_belief_sample.argtypes = [vp, i32, i32, u64, vp, vp]
    L.orx_rollout.argtypes = [vp, i32, i32, i32, u64, vp, vp, i32, i32, i32, vp, vp]
    L.orx_legal_moves.argtypes = [vp, i32, i32, i32, i32, vp]
    L.orx_brute_moves.argtypes = [vp, vp]
    L.orx_policy_pick.argtypes = [vp, i32, i32, i32, u32, u32]
    L.orx_apply.argtypes = [vp, i32, i32, i32, vp, i32, vp, vp, vp, vp, vp]
    L.orx_start_check.argtypes = [vp, i32, i32, i32, vp]
    L.orx_two_square_applies.argtypes = [vp, i32, i32, i32]
    L.orx_import_check.argtypes = [vp]
    L.orx_marginals.argtypes = [vp, i32, vp, vp]
    L.orx_perft.argtypes = [vp, i32, i32, i32, i32, i32]
    L.orx_perft.restype = u64
    L.orx_setup_types.argtypes = [u64, u32, u32, vp]
    L.orx_initial_position.argtypes = [vp, vp]
    L.orx_philox.argtypes = [vp, vp, vp, i32]
    L.orx_battle.argtypes = [i32, i32]
    L.orx_bf16_ratio.argtypes = [u32, u32]
    L.orx_bf16_ratio.restype = ctypes.c_uint16
    L.orx_u8_ratio.argtypes = [u32, u32]
    L.orx_u8_ratio.restype = ctypes.c_uint8
    L.orx_ratio_batch.argtypes = [vp, vp, i32, vp, vp]
    L.orx_search.argtypes = [vp, i32, i32, i32, u64, vp, vp, vp, ctypes.c_double, ctypes.c_double, i32, i32, i32,
                             vp, vp, vp, vp, vp, vp, vp]


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------- primitives

def philox(ctr, key):
    """ctr: [n,4] uint32, key: [2] uint32 -> [n,4] uint32."""
    ctr = _c(np.atleast_2d(ctr), np.uint32)
    key = _c(key, np.uint32)
    out = np.zeros_like(ctr)
    lib().orx_philox(_p(ctr), _p(key), _p(out), ctr.shape[0])
    return out


def battle(ta, td):
    return lib().orx_battle(int(ta), int(td))


def bf16_ratio(num, den):
    return lib().orx_bf16_ratio(int(num), int(den))


def u8_ratio(num, den):
    return lib().orx_u8_ratio(int(num), int(den))


def ratio_batch(num, den):
    """Vectorised bf16 bits and uint8 codes of num/den."""
    num = _c(num, np.uint32)
    den = _c(den, np.uint32)
    bf = np.zeros(num.shape, np.uint16)
    u8 = np.zeros(num.shape, np.uint8)
    lib().orx_ratio_batch(_p(num), _p(den), num.size, _p(bf), _p(u8))
    return bf, u8


def setup_types(seed, slot, episode=0):
    out = np.zeros(80, np.uint8)
    lib().orx_setup_types(seed, slot, episode, _p(out))
    return out


def initial_position(types):
    types = _c(types, np.uint8)
    out = np.zeros(POS_BYTES, np.uint8)
    lib().orx_initial_position(_p(types), _p(out))
    return out


# --------------------------------------------------------------- positions

def import_check(pos):
    return lib().orx_import_check(_p(_c(pos, np.uint8)))


def legal_moves(pos, k=100, cap=1000, flags=ALL_RULES, physical=False):
    pos = _c(pos, np.uint8)
    buf = np.zeros(400, np.int32)
    n = lib().orx_legal_moves(_p(pos), k, cap, flags, int(physical), _p(buf))
    if n < 0:
        raise ValueError("invalid position")
    return buf[:n].copy()


def policy_pick(pos, w0, w1, magnet=True, k=100, cap=1000, flags=ALL_RULES):
    """The rollout policy's move in `pos` for Philox words (w0, w1)."""
    pos = _c(pos, np.uint8)
    f = (flags | ROLLOUT_MAGNET) if magnet else (flags & ~ROLLOUT_MAGNET)
    a = lib().orx_policy_pick(_p(pos), k, cap, f, int(w0) & 0xFFFFFFFF, int(w1) & 0xFFFFFFFF)
    if a == -2:
        raise ValueError("invalid position")
    return a


def brute_moves(pos):
    pos = _c(pos, np.uint8)
    buf = np.zeros(400, np.int32)
    n = lib().orx_brute_moves(_p(pos), _p(buf))
    if n < 0:
        raise ValueError("invalid position")
    return buf[:n].copy()


def apply(pos, actions, k=100, cap=1000, flags=ALL_RULES, planes=False):
    """Apply actions; returns (position, ending, winner[, planes_u8, planes_bf16])."""
    pos = _c(pos, np.uint8)
    acts = _c(actions, np.int16)
    out = np.zeros(POS_BYTES, np.uint8)
    ending = ctypes.c_int(0)
    winner = ctypes.c_int(-1)
    u8 = np.zeros((NCHAN, 100), np.uint8) if planes else None
    bf = np.zeros((NCHAN, 100), np.uint16) if planes else None
    r = lib().orx_apply(_p(pos), k, cap, flags, _p(acts), len(acts), _p(out),
                        ctypes.byref(ending), ctypes.byref(winner), _p(u8), _p(bf))
    if r != 0:
        raise ValueError("illegal action at index %d (code %d)" % (-r - 1, r))
    if planes:
        return out, ending.value, winner.value, u8, bf
    return out, ending.value, winner.value


def start_check(pos, k=100, cap=1000, flags=ALL_RULES):
    w = ctypes.c_int(-1)
    code = lib().orx_start_check(_p(_c(pos, np.uint8)), k, cap, flags, ctypes.byref(w))
    return code, w.value


def two_square_applies(pos, k=100, cap=1000, flags=ALL_RULES):
    return lib().orx_two_square_applies(_p(_c(pos, np.uint8)), k, cap, flags)


def marginals(pos, side):
    num = np.zeros((40, 12), np.uint32)
    den = np.zeros((40, 12), np.uint32)
    if lib().orx_marginals(_p(_c(pos, np.uint8)), side, _p(num), _p(den)):
        raise ValueError("invalid position")
    return num, den


def perft(pos, depth, brute=False, k=100, cap=1000, flags=ALL_RULES):
    return int(lib().orx_perft(_p(_c(pos, np.uint8)), depth, int(brute), k, cap, flags))


# --------------------------------------------------------------- drivers

def env_run(seed, n_slots, n_steps, slot0=0, k=100, cap=1000, flags=ALL_RULES, autoreset=True,
            actions=None, want_mask=True, want_final=False, episode0=0, pool=None, mirror=False, pins=None):
    """Oracle environment loop; outputs are [n_steps, n_slots] (mask [..., 1264]).

    pool: [2, M, 40] uint8 setups per side (types on the side's setup
    squares in ascending order); mirror: left-right orientation
    randomisation of pool setups; pins: {slot index i: 784-byte snapshot}
    for slots that start and restart from a fixed position."""
    shape = (n_steps, n_slots)
    act = np.zeros(shape, np.int16)
    rew = np.zeros(shape, np.int8)
    done = np.zeros(shape, np.uint8)
    ply = np.zeros(shape, np.int16)
    mask = np.zeros(shape + (MASK_BYTES,), np.uint8) if want_mask else None
    stats = np.zeros((n_slots, 8), np.uint32)
    final = np.zeros((n_slots, POS_BYTES), np.uint8) if want_final else None
    ain = None if actions is None else _c(actions, np.int16)
    pl = None if pool is None else _c(pool, np.uint8)
    pin_pos = pinned = None
    if pins:
        pin_pos = np.zeros((n_slots, POS_BYTES), np.uint8)
        pinned = np.zeros(n_slots, np.uint8)
        for i, p in pins.items():
            pin_pos[i] = p
            pinned[i] = 1
    r = lib().orx_env_run(seed, slot0, n_slots, n_steps, k, cap, flags, int(autoreset), _p(ain),
                          _p(act), _p(rew), _p(done), _p(ply), _p(mask), _p(stats), _p(final), int(episode0),
                          _p(pl), 0 if pl is None else pl.shape[1], int(bool(mirror)), _p(pin_pos), _p(pinned))
    if r != 0:
        if -r - 1 >= n_steps * n_slots:
            raise ValueError("corrupt pinned snapshot for slot %d" % (-r - 1 - n_steps * n_slots))
        raise ValueError("illegal supplied action (flat index %d)" % (-r - 1))
    return dict(action=act, reward=rew, done=done, ply=ply, mask=mask, stats=stats, final=final)


def play_games(seed, n_games, k=100, cap=1000, flags=ALL_RULES):
    setups = np.zeros((n_games, 80), np.uint8)
    actions = np.zeros((n_games, cap), np.int16)
    lengths = np.zeros(n_games, np.int32)
    endings = np.zeros(n_games, np.uint8)
    rewards = np.zeros(n_games, np.int8)
    lib().orx_play_games(seed, n_games, k, cap, flags, _p(setups), _p(actions), _p(lengths),
                         _p(endings), _p(rewards))
    return dict(setups=setups, actions=actions, lengths=lengths, endings=endings, rewards=rewards)


def replay_positions(setups, actions, game, ply, k=100, cap=1000, flags=ALL_RULES):
    setups = _c(setups, np.uint8)
    actions = _c(actions, np.int16)
    game = _c(game, np.int32)
    ply = _c(ply, np.int16)
    out = np.zeros((len(game), POS_BYTES), np.uint8)
    r = lib().orx_replay_positions(_p(setups), _p(actions), actions.shape[1], _p(game), _p(ply),
                                   len(game), k, cap, flags, _p(out))
    if r != 0:
        raise ValueError("replay failed for item %d" % (-r - 1))
    return out


def obs_encode(setups, actions, game, ply, player=None, k=100, cap=1000, flags=ALL_RULES,
               want_u8=True, want_bf16=True, want_mask=True):
    setups = _c(setups, np.uint8)
    actions = _c(actions, np.int16)
    game = _c(game, np.int32)
    ply = _c(ply, np.int16)
    B = len(game)
    pl = None if player is None else _c(player, np.int8)
    u8 = np.zeros((B, NCHAN, 100), np.uint8) if want_u8 else None
    bf = np.zeros((B, NCHAN, 100), np.uint16) if want_bf16 else None
    mask = np.zeros((B, MASK_BYTES), np.uint8) if want_mask else None
    r = lib().orx_obs_encode(_p(setups), _p(actions), actions.shape[1], _p(game), _p(ply), _p(pl), B,
                             k, cap, flags, _p(u8), _p(bf), _p(mask))
    if r != 0:
        raise ValueError("replay failed for item %d" % (-r - 1))
    return u8, bf, mask


def belief_sample(pos, K, seed, stream_ids=None):
    pos = _c(np.atleast_2d(pos), np.uint8)
    P = pos.shape[0]
    sid = None if stream_ids is None else _c(stream_ids, np.uint32)
    out = np.zeros((P, K, 40), np.uint8)
    r = lib().orx_belief_sample(_p(pos), P, K, seed, _p(sid), _p(out))
    if r != 0:
        raise ValueError("invalid position %d" % (-r - 1))
    return out


def rollout(pos, K, depth, seed, stream_ids=None, types=None, k=100, cap=1000, flags=ALL_RULES,
            want_outcomes=False):
    pos = _c(np.atleast_2d(pos), np.uint8)
    P = pos.shape[0]
    sid = None if stream_ids is None else _c(stream_ids, np.uint32)
    ty = None if types is None else _c(types, np.uint8)
    tallies = np.zeros((P, 4), np.int32)
    outc = np.zeros((P, K), np.int8) if want_outcomes else None
    r = lib().orx_rollout(_p(pos), P, K, depth, seed, _p(sid), _p(ty), k, cap, flags, _p(tallies), _p(outc))
    if r != 0:
        raise ValueError("invalid position %d" % (-r - 1))
    return (tallies, outc) if want_outcomes else tallies


SEARCH_MAX_MOVES = 256
SEARCH_ALPHA, SEARCH_BETA = 0.002, 0.02   # App. E, Tab. search-hyper


def search(pos, S, depth, seed, stream_ids=None, pi_theta=None, alpha=SEARCH_ALPHA, beta=SEARCH_BETA, k=100,
           cap=1000, flags=ALL_RULES, q_values=None):
    """App. E search: per-candidate-move rollouts (S configurations, depth
    plies with the forced first move) and the tabular MMD update.  Returns a
    dict of n_moves [P], actions [P, 256], tallies [P, 256, 4], q and pi
    [P, 256] (float64), chosen [P], status [P]."""
    pos = _c(np.atleast_2d(pos), np.uint8)
    P = pos.shape[0]
    M = SEARCH_MAX_MOVES
    sid = None if stream_ids is None else _c(stream_ids, np.uint32)
    pt = None if pi_theta is None else _c(pi_theta, np.float32)
    qv = None if q_values is None else _c(q_values, np.float32)
    out = dict(n_moves=np.zeros(P, np.int32), actions=np.zeros((P, M), np.int16),
               tallies=np.zeros((P, M, 4), np.int32), q=np.zeros((P, M)), pi=np.zeros((P, M)),
               chosen=np.zeros(P, np.int16), status=np.zeros(P, np.uint8))
    r = lib().orx_search(_p(pos), P, S, depth, seed, _p(sid), _p(pt), _p(qv), float(alpha), float(beta), k, cap, flags,
                         _p(out["n_moves"]), _p(out["actions"]), _p(out["tallies"]), _p(out["q"]), _p(out["pi"]),
                         _p(out["chosen"]), _p(out["status"]))
    if r != 0:
        raise ValueError("position %d has more than %d legal moves" % (-r - 1, M))
    return out
