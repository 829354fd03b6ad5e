"""The Python binding's extent checks, on CPU.

The C entry points take bare device pointers, so the binding refuses a
tensor smaller than what the call reads or writes.  Here the library is
replaced by a recorder: every wrapper is called with CPU tensors of exactly
the documented shapes, and each checked argument must need exactly the
elements such a tensor holds (a larger requirement would refuse valid
input, a smaller one would let a short tensor through).  _ptr itself is
checked for refusing a short tensor before it looks at the device."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
import paper_2511_07312_gb300 as st  # noqa: E402


class _Recorder:
    def __init__(self):
        self.checked = []

    def ptr(self, t, dtype=None, name="tensor", numel=None):
        if t is None:
            return None
        assert isinstance(t, torch.Tensor)
        if dtype is not None:
            assert t.dtype == dtype, (name, t.dtype, dtype)
        if numel is not None:
            self.checked.append((name, numel, t.numel()))
        return ctypes.c_void_p(0)


class _FakeLib:
    def __getattr__(self, name):
        return lambda *a: 0


@pytest.fixture
def rec(monkeypatch):
    r = _Recorder()
    monkeypatch.setattr(st, "_ptr", r.ptr)
    monkeypatch.setattr(st, "lib", lambda: _FakeLib())
    monkeypatch.setattr(st, "_stream", lambda stream=None: None)
    return r


def _exact(rec, names):
    got = {n: (need, have) for n, need, have in rec.checked}
    for n in names:
        assert n in got, (n, sorted(got))
        need, have = got[n]
        assert need == have, (n, need, have)


def _u8(*shape):
    return torch.zeros(shape, dtype=torch.uint8)


def test_module_functions_need_exactly_the_documented_shapes(rec):
    P, K, B, logs, L = 3, 5, 7, 4, 50
    pos = _u8(P, st.POS_BYTES)
    sid = torch.zeros(P, dtype=torch.int32)
    st.belief_sample(pos, K, 1, stream_ids=sid)
    _exact(rec, ["pos", "stream_ids"])
    rec.checked.clear()
    st.rollout(pos, K, 8, 1, stream_ids=sid, types=_u8(P, K, 40), out=torch.zeros((P, 4), dtype=torch.int32))
    _exact(rec, ["pos", "stream_ids", "types", "tallies"])
    rec.checked.clear()
    st.search(pos, 4, 8, 1, stream_ids=sid, pi_theta=torch.zeros((P, 10000)),
              q_values=torch.zeros((P, 10000)))
    _exact(rec, ["pos", "stream_ids", "pi_theta", "q_values"])
    rec.checked.clear()
    st.positions_mask(pos)
    _exact(rec, ["pos"])
    rec.checked.clear()
    setups = _u8(logs, 80)
    actions = torch.zeros((logs, L), dtype=torch.int16)
    game = torch.zeros(B, dtype=torch.int32)
    ply = torch.zeros(B, dtype=torch.int16)
    st.replay_positions(setups, actions, game, ply)
    _exact(rec, ["setups", "ply"])
    rec.checked.clear()
    out = dict(planes=_u8(B, st.NCHAN, 100), planes_bf16=torch.zeros((B, st.NCHAN, 100), dtype=torch.bfloat16),
               mask=_u8(B, st.MASK_BYTES), status=_u8(B))
    st.obs_encode(setups, actions, game, ply, player=torch.zeros(B, dtype=torch.int8), out=out)
    _exact(rec, ["setups", "ply", "player", "planes", "planes_bf16", "mask", "status"])


def test_env_methods_need_exactly_the_documented_shapes(rec):
    N, R = 6, 3
    env = st.Env.__new__(st.Env)
    env.N, env._h, env.device = N, None, torch.device("cpu")
    env._launch = lambda fn, *a: fn(*a)
    out = dict(action=torch.zeros(N, dtype=torch.int16), reward=torch.zeros(N, dtype=torch.int8),
               done=_u8(N), ply=torch.zeros(N, dtype=torch.int16), mask=_u8(N, st.MASK_BYTES))
    env.step(actions=torch.zeros(N, dtype=torch.int16), out=out)
    _exact(rec, ["actions", "action", "reward", "done", "ply", "mask"])
    rec.checked.clear()
    ring = dict(action=torch.zeros((R, N), dtype=torch.int16), reward=torch.zeros((R, N), dtype=torch.int8),
                done=_u8(R, N), ply=torch.zeros((R, N), dtype=torch.int16), mask=_u8(R, N, st.MASK_BYTES))
    env.run(10, R, out=ring)
    _exact(rec, ["action", "reward", "done", "ply", "mask"])
    rec.checked.clear()
    env.reset(setups=_u8(N, 80), which=_u8(N))
    _exact(rec, ["setups", "which"])
    rec.checked.clear()
    env.import_(torch.arange(2), _u8(2, st.POS_BYTES))
    _exact(rec, ["positions"])
    rec.checked.clear()
    env.pin(torch.arange(3), _u8(3, st.POS_BYTES))
    _exact(rec, ["states"])


def test_ptr_refuses_a_short_tensor_before_the_device_check():
    with pytest.raises(ValueError, match="holds 10 elements; the call uses 12"):
        st._ptr(torch.zeros(10, dtype=torch.uint8), torch.uint8, "x", 12)
    with pytest.raises(TypeError, match="CUDA"):
        st._ptr(torch.zeros(12, dtype=torch.uint8), torch.uint8, "x", 12)
    with pytest.raises(TypeError, match="must be torch.int16"):
        st._ptr(torch.zeros(12, dtype=torch.uint8), torch.int16, "x", 12)
