"""Python binding of the GB300 Stratego engine (libstratego_gb300.so).

Argument marshalling only: every step of the game engine runs in the CUDA
kernels behind the C ABI of include/stratego.h.  PyTorch supplies device
memory and streams; tensors are passed by data pointer.  The library is
required: if it cannot be loaded every entry point raises.
"""
import ctypes
import os

import torch

from . import build as _build

MASK_BYTES = 1264
NCHAN = 487
POS_BYTES = 784
RULE_TWO_SQUARE = 1
RULE_CHASE = 2
RULES_ALL = RULE_TWO_SQUARE | RULE_CHASE
POOL_MIRROR = 1          # st_env_set_setup_pool: left-right orientation randomisation
ROLLOUT_MAGNET = 0x100   # rollouts, search, server: the magnet policy as the rollout policy
AUTORESET = 4

ST_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "cuda error", 4: "illegal action",
                5: "timeout", 6: "busy", 7: "not ready", 8: "bad position"}


class StrategoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(code, "error"), code, msg))
        self.code = code


class st_rules(ctypes.Structure):
    _fields_ = [("battleless_limit", ctypes.c_int16), ("max_plies", ctypes.c_int16), ("flags", ctypes.c_uint32)]


class st_env_config(ctypes.Structure):
    _fields_ = [("num_games", ctypes.c_int32), ("seed", ctypes.c_uint64), ("rules", st_rules),
                ("env_flags", ctypes.c_uint32), ("device", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class st_position(ctypes.Structure):
    _fields_ = [("raw", ctypes.c_uint8 * POS_BYTES)]


class st_request(ctypes.Structure):
    _fields_ = [("pos", st_position), ("K", ctypes.c_int32), ("depth", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("stream_id", ctypes.c_uint32)]


class st_serve_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_requests", ctypes.c_int32), ("sample_slots", ctypes.c_int32),
                ("max_batches", ctypes.c_int32), ("rules", st_rules)]


class st_timing(ctypes.Structure):
    _fields_ = [("submit_ns", ctypes.c_uint64), ("admit_ns", ctypes.c_uint64), ("done_ns", ctypes.c_uint64)]


class st_serve_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "admitted", "completed", "batches", "max_batch_requests",
                                               "queued", "running")]


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load (building first if the sources are newer) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    vp, i32, i16, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int16, ctypes.c_uint64
    L.st_version.restype = ctypes.c_char_p
    L.st_last_error.restype = ctypes.c_char_p
    for name, args in {
        "st_env_create": [ctypes.POINTER(st_env_config), ctypes.POINTER(vp)],
        "st_env_destroy": [vp],
        "st_env_reset": [vp, vp, vp],
        "st_env_step": [vp, vp, vp, vp, vp, vp, vp],
        "st_env_run": [vp, i32, i32, vp, vp, vp, vp, vp],
        "st_env_set_launch": [vp, i32, i32, i32, i32],
        "st_env_get_launch": [vp, vp],
        "st_env_sync": [vp],
        "st_env_stats": [vp, vp],
        "st_env_export": [vp, vp, i32, vp],
        "st_env_import": [vp, vp, i32, vp],
        "st_env_set_setup_pool": [vp, vp, i32, ctypes.c_uint32],
        "st_env_pin": [vp, vp, i32, vp],
        "st_env_sample_actions": [vp, vp],
        "st_env_enable_history": [vp, i32],
        "st_env_current_step": [vp, ctypes.POINTER(ctypes.c_int64)],
        "st_env_history_positions": [vp, ctypes.c_int64, vp, vp, vp, vp],
        "st_env_history_steps": [vp, ctypes.c_int64, vp, vp, vp, vp],
        "st_env_history_logs": [vp, ctypes.c_int64, i32, vp, vp, vp, vp],
        "st_positions_mask": [vp, i32, ctypes.POINTER(st_rules), vp, vp, vp, vp, vp],
        "st_replay_positions": [vp, vp, i32, i32, vp, vp, i32, ctypes.POINTER(st_rules), vp, vp, vp],
        "st_replay_set_chunk": [i32],
        "st_obs_encode": [vp, vp, i32, i32, vp, vp, vp, i32, ctypes.POINTER(st_rules), vp, vp, vp, vp, vp],
        "st_obs_encode_static": [vp, vp, i32, i32, vp, vp, vp, i32, ctypes.POINTER(st_rules), vp, vp, vp, vp, vp],
        "st_belief_sample": [vp, i32, i32, u64, vp, vp, vp, vp],
        "st_rollout": [vp, i32, i32, i32, u64, vp, vp, ctypes.POINTER(st_rules), vp, vp, vp],
        "st_search": [vp, i32, i32, i32, u64, vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(st_rules),
                      vp, vp, vp, vp, vp, vp, vp, vp],
        "st_serve_create": [ctypes.POINTER(st_serve_config), ctypes.POINTER(vp)],
        "st_serve_submit": [vp, ctypes.POINTER(st_request), ctypes.POINTER(ctypes.c_uint64)],
        "st_serve_poll": [vp, ctypes.c_uint64, vp, ctypes.POINTER(st_timing)],
        "st_serve_wait": [vp, ctypes.c_uint64, i32, vp, ctypes.POINTER(st_timing)],
        "st_serve_get_stats": [vp, ctypes.POINTER(st_serve_stats)],
        "st_serve_destroy": [vp],
    }.items():
        if hasattr(L, name):
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int


def _check(code):
    if code != ST_OK:
        raise StrategoError(code, lib().st_last_error().decode())


def _ptr(t, dtype=None, name="tensor", numel=None):
    """Device address of a contiguous CUDA tensor of the given dtype.  numel:
    the elements the call reads or writes through it; a smaller tensor is
    refused here, since the C entry points get bare pointers and cannot
    check extents themselves."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if numel is not None and t.numel() < numel:
        raise ValueError("%s holds %d elements; the call uses %d" % (name, t.numel(), numel))
    if not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def set_replay_chunk(items_per_block):
    _check(lib().st_replay_set_chunk(int(items_per_block)))


def make_rules(k=100, cap=1000, flags=RULES_ALL):
    return st_rules(int(k), int(cap), int(flags))


def version():
    return lib().st_version().decode()


class Env:
    """N game slots on one GPU (App. B.1).  All outputs are CUDA tensors."""

    def __init__(self, num_games, seed=1, k=100, cap=1000, flags=RULES_ALL, autoreset=True, device=0,
                 stream=None):
        self.device = torch.device("cuda", device)
        self.N = int(num_games)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        cfg = st_env_config(self.N, int(seed) & 0xFFFFFFFFFFFFFFFF, make_rules(k, cap, flags),
                            AUTORESET if autoreset else 0, int(device), self.stream.cuda_stream)
        h = ctypes.c_void_p()
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        _check(lib().st_env_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.release_to_current()

    def close(self):
        if getattr(self, "_h", None):
            lib().st_env_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, shape, dtype):
        with torch.cuda.device(self.device):
            return torch.empty(shape, dtype=dtype, device=self.device)

    def wait_for_current(self):
        """The env's stream waits for the caller's current stream (inputs
        ready, output buffers free)."""
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def release_to_current(self):
        """The caller's current stream waits for the env's stream (results
        visible to whatever the caller enqueues next)."""
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _launch(self, fn, *a):
        self.wait_for_current()
        _check(fn(*a))
        self.release_to_current()

    def step(self, actions=None, want_mask=True, out=None):
        """One ply in every slot; returns dict(action, reward, done, ply, mask)."""
        if out is None:
            out = dict(action=self._empty(self.N, torch.int16), reward=self._empty(self.N, torch.int8),
                       done=self._empty(self.N, torch.uint8), ply=self._empty(self.N, torch.int16),
                       mask=self._empty((self.N, MASK_BYTES), torch.uint8) if want_mask else None)
        N = self.N
        self._launch(lib().st_env_step, self._h, _ptr(actions, torch.int16, "actions", N),
                     _ptr(out["action"], torch.int16, "action", N), _ptr(out["reward"], torch.int8, "reward", N),
                     _ptr(out["done"], torch.uint8, "done", N), _ptr(out["ply"], torch.int16, "ply", N),
                     _ptr(out.get("mask"), torch.uint8, "mask", N * MASK_BYTES))
        return out

    def run(self, n_steps, ring_steps=None, want=("action", "reward", "done", "ply", "mask"), out=None):
        ring_steps = int(ring_steps or n_steps)
        if out is None:
            shp = (ring_steps, self.N)
            out = dict(action=self._empty(shp, torch.int16) if "action" in want else None,
                       reward=self._empty(shp, torch.int8) if "reward" in want else None,
                       done=self._empty(shp, torch.uint8) if "done" in want else None,
                       ply=self._empty(shp, torch.int16) if "ply" in want else None,
                       mask=self._empty(shp + (MASK_BYTES,), torch.uint8) if "mask" in want else None)
        n = ring_steps * self.N
        self._launch(lib().st_env_run, self._h, int(n_steps), ring_steps, _ptr(out["action"], torch.int16, "action", n),
                     _ptr(out["reward"], torch.int8, "reward", n), _ptr(out["done"], torch.uint8, "done", n),
                     _ptr(out["ply"], torch.int16, "ply", n), _ptr(out["mask"], torch.uint8, "mask", n * MASK_BYTES))
        return out

    def set_launch(self, warps_per_block, blocks_per_sm=0, games_per_fetch=1, games_per_warp=1):
        _check(lib().st_env_set_launch(self._h, int(warps_per_block), int(blocks_per_sm), int(games_per_warp),
                                       int(games_per_fetch)))

    def launch_shape(self):
        """The shape st_env_run uses now: {warps_per_block, blocks_per_sm
        (resident, after clamping to the occupancy limit), games_per_warp,
        games_per_fetch}."""
        v = (ctypes.c_int32 * 4)()
        _check(lib().st_env_get_launch(self._h, v))
        return {"warps_per_block": v[0], "blocks_per_sm": v[1], "games_per_warp": v[2], "games_per_fetch": v[3]}

    def reset(self, setups=None, which=None):
        self._launch(lib().st_env_reset, self._h, _ptr(setups, torch.uint8, "setups", self.N * 80),
                     _ptr(which, torch.uint8, "which", self.N))

    def sync(self):
        _check(lib().st_env_sync(self._h))

    def stats(self):
        out = self._empty((self.N, 8), torch.int32)
        self._launch(lib().st_env_stats, self._h, _ptr(out))
        return out

    def export(self, idx):
        idx = idx.to(device=self.device, dtype=torch.int32).contiguous()
        out = self._empty((idx.numel(), POS_BYTES), torch.uint8)
        self._launch(lib().st_env_export, self._h, _ptr(idx), idx.numel(), _ptr(out))
        return out

    def import_(self, idx, pos):
        idx = idx.to(device=self.device, dtype=torch.int32).contiguous()
        self._launch(lib().st_env_import, self._h, _ptr(idx), idx.numel(),
                     _ptr(pos, torch.uint8, "positions", idx.numel() * POS_BYTES))

    def set_setup_pool(self, pool, mirror=False):
        """New games take their setups from pool [2, M, 40] uint8 (None: off)."""
        if pool is None:
            self._launch(lib().st_env_set_setup_pool, self._h, None, 0, 0)
            return
        pool = pool.to(device=self.device, dtype=torch.uint8).contiguous()
        if pool.dim() != 3 or pool.shape[0] != 2 or pool.shape[2] != 40:
            raise ValueError("pool must be [2, M, 40]")
        self._launch(lib().st_env_set_setup_pool, self._h, _ptr(pool), pool.shape[1], POOL_MIRROR if mirror else 0)

    def sample_actions(self):
        """The random policy's next action per slot, not played (-1: none)."""
        out = self._empty(self.N, torch.int16)
        self._launch(lib().st_env_sample_actions, self._h, _ptr(out))
        return out

    def enable_history(self, H):
        """Keep a record of each of the last H steps (0: off)."""
        self._launch(lib().st_env_enable_history, self._h, int(H))

    def current_step(self):
        v = ctypes.c_int64()
        _check(lib().st_env_current_step(self._h, ctypes.byref(v)))
        return v.value

    def history_positions(self, t):
        """Positions at step t: dict(pos [N, 784], status, ended, since)."""
        out = dict(pos=self._empty((self.N, POS_BYTES), torch.uint8), status=self._empty(self.N, torch.uint8),
                   ended=self._empty(self.N, torch.uint8), since=self._empty(self.N, torch.int32))
        self._launch(lib().st_env_history_positions, self._h, int(t), _ptr(out["pos"]), _ptr(out["status"]),
                     _ptr(out["ended"]), _ptr(out["since"]))
        return out

    def history_steps(self, t):
        """The record of step t: dict(action, done, reward, start)."""
        out = dict(action=self._empty(self.N, torch.int16), done=self._empty(self.N, torch.uint8),
                   reward=self._empty(self.N, torch.int8), start=self._empty(self.N, torch.uint8))
        self._launch(lib().st_env_history_steps, self._h, int(t), _ptr(out["action"]), _ptr(out["done"]),
                     _ptr(out["reward"]), _ptr(out["start"]))
        return out

    def history_logs(self, t, L):
        """Setups [N, 80], logs [N, L], plies [N], status [N] of the games at step t."""
        out = dict(setups=self._empty((self.N, 80), torch.uint8), logs=self._empty((self.N, int(L)), torch.int16),
                   plies=self._empty(self.N, torch.int16), status=self._empty(self.N, torch.uint8))
        self._launch(lib().st_env_history_logs, self._h, int(t), int(L), _ptr(out["setups"]), _ptr(out["logs"]),
                     _ptr(out["plies"]), _ptr(out["status"]))
        return out

    def pin(self, idx=None, states=None):
        """Slots idx restart from states [n, 784] whenever their games end
        (replaces the previous pin set; no arguments: clear it)."""
        if idx is None:
            self._launch(lib().st_env_pin, self._h, None, 0, None)
            return
        idx = idx.to(device=self.device, dtype=torch.int32).contiguous()
        self._launch(lib().st_env_pin, self._h, _ptr(idx), idx.numel(),
                     _ptr(states, torch.uint8, "states", idx.numel() * POS_BYTES))


def _dev(t, dtype, device):
    return t.to(device=device, dtype=dtype).contiguous()


def replay_positions(setups, actions, game, ply, k=100, cap=1000, flags=RULES_ALL, stream=None):
    dev = setups.device
    B = game.numel()
    out = torch.empty((B, POS_BYTES), dtype=torch.uint8, device=dev)
    status = torch.empty(B, dtype=torch.uint8, device=dev)
    r = make_rules(k, cap, flags)
    _check(lib().st_replay_positions(_ptr(setups, torch.uint8, "setups", actions.shape[0] * 80),
                                     _ptr(actions, torch.int16, "actions"), actions.shape[1], actions.shape[0],
                                     _ptr(game, torch.int32, "game"), _ptr(ply, torch.int16, "ply", B), B,
                                     ctypes.byref(r), _ptr(out), _ptr(status), _stream(stream)))
    return out, status


def obs_encode(setups, actions, game, ply, player=None, k=100, cap=1000, flags=RULES_ALL, want_u8=True,
               want_bf16=True, want_mask=True, out=None, stream=None):
    dev = setups.device
    B = game.numel()
    if out is None:
        out = dict(planes=torch.empty((B, NCHAN, 100), dtype=torch.uint8, device=dev) if want_u8 else None,
                   planes_bf16=torch.empty((B, NCHAN, 100), dtype=torch.bfloat16, device=dev) if want_bf16 else None,
                   mask=torch.empty((B, MASK_BYTES), dtype=torch.uint8, device=dev) if want_mask else None,
                   status=torch.empty(B, dtype=torch.uint8, device=dev))
    r = make_rules(k, cap, flags)
    _check(lib().st_obs_encode(_ptr(setups, torch.uint8, "setups", actions.shape[0] * 80),
                               _ptr(actions, torch.int16, "actions"), actions.shape[1], actions.shape[0],
                               _ptr(game, torch.int32, "game"), _ptr(ply, torch.int16, "ply", B),
                               _ptr(player, torch.int8, "player", B), B, ctypes.byref(r),
                               _ptr(out["planes"], torch.uint8, "planes", B * NCHAN * 100),
                               _ptr(out["planes_bf16"], torch.bfloat16, "planes_bf16", B * NCHAN * 100),
                               _ptr(out["mask"], torch.uint8, "mask", B * MASK_BYTES),
                               _ptr(out["status"], torch.uint8, "status", B), _stream(stream)))
    return out


def belief_sample(pos, K, seed, stream_ids=None, stream=None):
    P = pos.shape[0]
    types = torch.empty((P, K, 40), dtype=torch.uint8, device=pos.device)
    status = torch.empty(P, dtype=torch.uint8, device=pos.device)
    _check(lib().st_belief_sample(_ptr(pos, torch.uint8, "pos", P * POS_BYTES), P, int(K),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(stream_ids, torch.int32, "stream_ids", P),
                                  _ptr(types), _ptr(status), _stream(stream)))
    return types, status


def rollout(pos, K, depth, seed, stream_ids=None, types=None, k=100, cap=1000, flags=RULES_ALL, out=None,
            stream=None):
    P = pos.shape[0]
    tallies = out if out is not None else torch.empty((P, 4), dtype=torch.int32, device=pos.device)
    status = torch.empty(P, dtype=torch.uint8, device=pos.device)
    r = make_rules(k, cap, flags)
    _check(lib().st_rollout(_ptr(pos, torch.uint8, "pos", P * POS_BYTES), P, int(K), int(depth),
                            int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(stream_ids, torch.int32, "stream_ids", P),
                            _ptr(types, torch.uint8, "types", P * max(int(K), 0) * 40), ctypes.byref(r),
                            _ptr(tallies, torch.int32, "tallies", P * 4), _ptr(status), _stream(stream)))
    return tallies, status


_TYPE_CHARS = "S23456789MFB"   # Spy, Scout .. General, Marshal, Flag, Bomb
_LAKES = {42, 43, 46, 47, 52, 53, 56, 57}


def board_string(pos):
    """A text picture of one 784-byte snapshot for debugging (App. B.1
    BoardStrs): rank 10 on top, two characters per square -- 'r'/'b' and the
    piece's type for red and blue pieces (upper case once revealed), '~~'
    for lakes, '..' for empty squares."""
    import numpy as np
    p = np.asarray(pos.cpu() if isinstance(pos, torch.Tensor) else pos, dtype=np.uint8).reshape(-1)
    if p.size != POS_BYTES:
        raise ValueError("a position is %d bytes" % POS_BYTES)
    cells = [".." if s not in _LAKES else "~~" for s in range(100)]
    for pid in range(80):
        fl = int(p[160 + pid])
        if fl & 1:
            side = "r" if pid < 40 else "b"
            if fl & 2:
                side = side.upper()
            cells[int(p[80 + pid])] = side + _TYPE_CHARS[int(p[pid])]
    ply = int(np.frombuffer(p[240:242].tobytes(), np.int16)[0])
    rows = [" ".join(cells[10 * r:10 * r + 10]) for r in range(9, -1, -1)]
    return "\n".join(rows + ["ply %d, %s to move" % (ply, "red" if ply % 2 == 0 else "blue")])


def positions_mask(pos, k=100, cap=1000, flags=RULES_ALL, stream=None):
    """Legal masks [P, 1264], move counts, two-square flags and status of snapshots."""
    P = pos.shape[0]
    dev = pos.device
    out = dict(mask=torch.empty((P, MASK_BYTES), dtype=torch.uint8, device=dev),
               n_legal=torch.empty(P, dtype=torch.int32, device=dev),
               two_square=torch.empty(P, dtype=torch.uint8, device=dev),
               status=torch.empty(P, dtype=torch.uint8, device=dev))
    r = make_rules(k, cap, flags)
    _check(lib().st_positions_mask(_ptr(pos, torch.uint8, "pos", P * POS_BYTES), P, ctypes.byref(r), _ptr(out["mask"]),
                                   _ptr(out["n_legal"]), _ptr(out["two_square"]), _ptr(out["status"]),
                                   _stream(stream)))
    return out


SEARCH_MAX_MOVES = 256
SEARCH_ALPHA, SEARCH_BETA = 0.002, 0.02   # App. E


def search(pos, S, depth, seed, stream_ids=None, pi_theta=None, alpha=SEARCH_ALPHA, beta=SEARCH_BETA, k=100,
           cap=1000, flags=RULES_ALL, stream=None, q_values=None):
    """Per-candidate-move search with the tabular MMD update (st_search).

    pos: [P, 784] uint8 CUDA tensor; pi_theta: optional [P, 10000] float32
    CUDA tensor of move probabilities by action; q_values: optional
    [P, 10000] float32 per-move values by action, used instead of the
    rollouts.  Returns a dict of CUDA
    tensors: n_moves [P] int32, actions [P, 256] int16, tallies [P, 256, 4]
    int32, q and pi [P, 256] float64, chosen [P] int16, status [P] uint8."""
    P = pos.shape[0]
    dev = pos.device
    out = {
        "n_moves": torch.empty(P, dtype=torch.int32, device=dev),
        "actions": torch.empty((P, SEARCH_MAX_MOVES), dtype=torch.int16, device=dev),
        "tallies": torch.empty((P, SEARCH_MAX_MOVES, 4), dtype=torch.int32, device=dev),
        "q": torch.empty((P, SEARCH_MAX_MOVES), dtype=torch.float64, device=dev),
        "pi": torch.empty((P, SEARCH_MAX_MOVES), dtype=torch.float64, device=dev),
        "chosen": torch.empty(P, dtype=torch.int16, device=dev),
        "status": torch.empty(P, dtype=torch.uint8, device=dev),
    }
    r = make_rules(k, cap, flags)
    _check(lib().st_search(_ptr(pos, torch.uint8, "pos", P * POS_BYTES), P, int(S), int(depth),
                           int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(stream_ids, torch.int32, "stream_ids", P),
                           _ptr(pi_theta, torch.float32, "pi_theta", P * 10000),
                           _ptr(q_values, torch.float32, "q_values", P * 10000), float(alpha), float(beta),
                           ctypes.byref(r), _ptr(out["n_moves"]), _ptr(out["actions"]), _ptr(out["tallies"]),
                           _ptr(out["q"]), _ptr(out["pi"]), _ptr(out["chosen"]), _ptr(out["status"]),
                           _stream(stream)))
    return out


class Server:
    """Search-request server with continuous batching (st_serve_*).

    submit() takes a host position (784 uint8 numpy array or bytes) and
    returns a ticket; poll()/wait() return (tallies[4] numpy int32, timing)
    or raise StrategoError (NOT_READY, TIMEOUT, BAD_POSITION)."""

    def __init__(self, device=0, max_requests=256, sample_slots=1 << 16, max_batches=8, k=100, cap=1000,
                 flags=RULES_ALL):
        import numpy as np  # noqa: F401
        cfg = st_serve_config(int(device), int(max_requests), int(sample_slots), int(max_batches),
                              make_rules(k, cap, flags))
        h = ctypes.c_void_p()
        _check(lib().st_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, pos, K, depth, seed, stream_id=0):
        import numpy as np
        req = st_request()
        buf = np.ascontiguousarray(np.frombuffer(bytes(pos), dtype=np.uint8) if isinstance(pos, (bytes, bytearray))
                                   else np.asarray(pos, dtype=np.uint8))
        if buf.size != POS_BYTES:
            raise ValueError("position must be %d bytes" % POS_BYTES)
        ctypes.memmove(ctypes.addressof(req.pos), buf.ctypes.data, POS_BYTES)
        req.K, req.depth = int(K), int(depth)
        req.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        req.stream_id = int(stream_id) & 0xFFFFFFFF
        t = ctypes.c_uint64()
        _check(lib().st_serve_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def _result(self, fn, *a):
        import numpy as np
        tallies = np.zeros(4, np.int32)
        tm = st_timing()
        _check(fn(self._h, *a, tallies.ctypes.data_as(ctypes.c_void_p), ctypes.byref(tm)))
        return tallies, (tm.submit_ns, tm.admit_ns, tm.done_ns)

    def poll(self, ticket):
        return self._result(lib().st_serve_poll, ctypes.c_uint64(ticket))

    def wait(self, ticket, timeout_ms=60000):
        return self._result(lib().st_serve_wait, ctypes.c_uint64(ticket), int(timeout_ms))

    def stats(self):
        s = st_serve_stats()
        _check(lib().st_serve_get_stats(self._h, ctypes.byref(s)))
        return {n: getattr(s, n) for n, _ in st_serve_stats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().st_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
