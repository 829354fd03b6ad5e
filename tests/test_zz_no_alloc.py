"""The allocation-free observation entry point, st_obs_encode_static.

Some callers cannot allocate device memory once they are running (a loop
whose memory budget is fixed at start-up, or code under a memory manager
that does not see stream-ordered allocations).  st_obs_encode_static serves
them: it computes exactly what st_obs_encode computes, with its scratch in a
fixed array inside the library.  This file checks, through the C ABI, that
two calls in a row give the same planes, masks and status as st_obs_encode
and as the oracle (bit for bit, the tolerance of every parity test here),
that a batch of exactly ST_OBS_STATIC_MAX_ITEMS items (the whole array) does
too, that calls leave the device's free memory and the PyTorch allocator's
counters unchanged, and that batches larger than the fixed array are
refused.  It is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2511_07312_gb300 as st  # noqa: E402


def _vp(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _static_call(setups, actions, games, plies, player=None):
    B = games.numel()
    dev = setups.device
    planes = torch.full((B, st.NCHAN, 100), 0xAB, dtype=torch.uint8, device=dev)
    bf = torch.full((B, st.NCHAN, 100), 7, dtype=torch.int16, device=dev)
    mask = torch.full((B, st.MASK_BYTES), 0xCD, dtype=torch.uint8, device=dev)
    status = torch.full((B,), 0xEE, dtype=torch.uint8, device=dev)
    rules = st.make_rules()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = st.lib().st_obs_encode_static(_vp(setups), _vp(actions), actions.shape[1], actions.shape[0],
                                         _vp(games), _vp(plies), _vp(player), B, ctypes.byref(rules),
                                         _vp(planes), _vp(bf), _vp(mask), _vp(status), stream)
    assert code == 0, st.lib().st_last_error()
    torch.cuda.synchronize()
    return planes, bf, mask, status


def _inputs(seed, n_games, per_game, bad_items=False):
    g = oracle.play_games(seed, n_games)
    rng = np.random.default_rng(seed)
    games = np.repeat(np.arange(n_games), per_game).astype(np.int32)
    plies = np.array([rng.integers(0, min(600, g["lengths"][i] - 1) + 1) for i in games], np.int16)
    order = np.lexsort((plies, games))
    games, plies = games[order], plies[order]
    if bad_items:
        games[3] = n_games + 5          # out of range: status 1, zero outputs
        plies[7] = 1001
    dev = torch.device("cuda", 0)
    return (torch.from_numpy(g["setups"]).to(dev), torch.from_numpy(g["actions"]).to(dev),
            torch.from_numpy(games).to(dev), torch.from_numpy(plies).to(dev))


def test_static_entry_point_matches_allocating_one_twice_in_a_row():
    # two different batches back to back: the second call must not see the first's records
    for seed, n_games, per_game, bad in ((41, 10, 30, False), (43, 7, 11, True)):
        setups, actions, games, plies = _inputs(seed, n_games, per_game, bad)
        player = torch.from_numpy((np.arange(games.numel()) % 3 - 1).astype(np.int8)).cuda()
        p_s, b_s, m_s, s_s = _static_call(setups, actions, games, plies, player)
        ref = st.obs_encode(setups, actions, games, plies, player=player)
        torch.cuda.synchronize()
        assert torch.equal(s_s, ref["status"])
        assert torch.equal(p_s, ref["planes"])
        assert torch.equal(b_s, ref["planes_bf16"].view(torch.int16))
        assert torch.equal(m_s, ref["mask"])
        if bad:
            assert int(s_s[3]) == 1 and int(s_s[7]) == 1
            assert int(p_s[3].sum()) == 0


def test_static_entry_point_matches_the_oracle():
    # a small batch against the oracle directly (uint8 and bf16 planes, masks)
    g = oracle.play_games(53, 4)
    rng = np.random.default_rng(53)
    games = np.repeat(np.arange(4), 5).astype(np.int32)
    plies = np.array([rng.integers(0, min(600, g["lengths"][i] - 1) + 1) for i in games], np.int16)
    order = np.lexsort((plies, games))
    games, plies = games[order], plies[order]
    dev = torch.device("cuda", 0)
    for _ in range(2):
        p_s, b_s, m_s, s_s = _static_call(torch.from_numpy(g["setups"]).to(dev),
                                          torch.from_numpy(g["actions"]).to(dev),
                                          torch.from_numpy(games).to(dev), torch.from_numpy(plies).to(dev))
        u8, bf, mask = oracle.obs_encode(g["setups"], g["actions"], games, plies)
        assert int(s_s.sum()) == 0
        assert np.array_equal(p_s.cpu().numpy(), u8)
        assert np.array_equal(b_s.cpu().numpy().view(np.uint16), bf)
        assert np.array_equal(m_s.cpu().numpy(), mask)


def test_static_entry_point_full_array_and_no_allocation():
    # B = ST_OBS_STATIC_MAX_ITEMS uses the last record of the fixed array
    B = 4096
    setups, actions, games, plies = _inputs(59, 64, B // 64)
    assert games.numel() == B
    ref = st.obs_encode(setups, actions, games, plies)
    _static_call(setups, actions, games, plies)          # first call on the device: its one-time set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    planes = torch.empty((B, st.NCHAN, 100), dtype=torch.uint8, device="cuda")
    bf = torch.empty((B, st.NCHAN, 100), dtype=torch.int16, device="cuda")
    mask = torch.empty((B, st.MASK_BYTES), dtype=torch.uint8, device="cuda")
    status = torch.empty((B,), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    alloc1, reserved1 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    rules = st.make_rules()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        code = st.lib().st_obs_encode_static(_vp(setups), _vp(actions), actions.shape[1], actions.shape[0],
                                             _vp(games), _vp(plies), None, B, ctypes.byref(rules), _vp(planes),
                                             _vp(bf), _vp(mask), _vp(status), stream)
        assert code == 0, st.lib().st_last_error()
        torch.cuda.synchronize()
        # nothing allocated by the call: the device's free memory and the
        # PyTorch allocator's counters are where they were before it
        assert torch.cuda.mem_get_info()[0] == free1
        assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == (alloc1, reserved1)
        assert torch.equal(status, ref["status"])
        assert torch.equal(planes, ref["planes"])
        assert torch.equal(bf, ref["planes_bf16"].view(torch.int16))
        assert torch.equal(mask, ref["mask"])
    assert free1 <= free0 and alloc1 >= alloc0 and reserved1 >= reserved0


def test_static_entry_point_refuses_batches_beyond_its_array():
    setups, actions, games, plies = _inputs(47, 2, 2)
    B = 4096 + 1
    big_g = torch.zeros(B, dtype=torch.int32, device="cuda")
    big_p = torch.zeros(B, dtype=torch.int16, device="cuda")
    out = torch.empty((B, st.NCHAN, 100), dtype=torch.uint8, device="cuda")
    rules = st.make_rules()
    code = st.lib().st_obs_encode_static(_vp(setups), _vp(actions), actions.shape[1], actions.shape[0],
                                         _vp(big_g), _vp(big_p), None, B, ctypes.byref(rules), _vp(out), None, None,
                                         None, None)
    assert code == 1
    assert b"exceed" in st.lib().st_last_error()
