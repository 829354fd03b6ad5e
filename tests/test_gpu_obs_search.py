"""GPU parity of replay, observation planes, belief samples and rollouts with
the oracle, bit for bit, through the C ABI."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2511_07312_gb300 as st  # noqa: E402


def _games(seed, n):
    g = oracle.play_games(seed, n)
    dev = torch.device("cuda", 0)
    return g, torch.from_numpy(g["setups"]).to(dev), torch.from_numpy(g["actions"]).to(dev)


def _items(g, per_game, seed=0, sort=True, upto=600):
    rng = np.random.default_rng(seed)
    n = len(g["lengths"])
    games = np.repeat(np.arange(n), per_game).astype(np.int32)
    plies = np.array([rng.integers(0, min(upto, g["lengths"][i] - 1) + 1) for i in games], np.int16)
    if sort:
        order = np.lexsort((plies, games))
        games, plies = games[order], plies[order]
    else:
        perm = rng.permutation(len(games))
        games, plies = games[perm], plies[perm]
    return games, plies


@pytest.mark.parametrize("sort,chunk", [(True, 4), (False, 4), (True, 1), (True, 33)])
def test_replay_positions_bit_exact(sort, chunk):
    g, S, A = _games(17, 12)
    games, plies = _items(g, 10, sort=sort)
    st.set_replay_chunk(chunk)
    try:
        pos, status = st.replay_positions(S, A, torch.from_numpy(games).cuda(), torch.from_numpy(plies).cuda())
        torch.cuda.synchronize()
    finally:
        st.set_replay_chunk(32)
    assert (status.cpu().numpy() == 0).all()
    ref = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    np.testing.assert_array_equal(pos.cpu().numpy(), ref)


def test_obs_planes_and_mask_bit_exact():
    g, S, A = _games(23, 16)
    games, plies = _items(g, 12, seed=1)
    player = np.where(np.arange(len(games)) % 3 == 0, -1, np.arange(len(games)) % 2).astype(np.int8)
    o = st.obs_encode(S, A, torch.from_numpy(games).cuda(), torch.from_numpy(plies).cuda(),
                      player=torch.from_numpy(player).cuda())
    torch.cuda.synchronize()
    u8, bf, mask = oracle.obs_encode(g["setups"], g["actions"], games, plies, player=player)
    got_u8 = o["planes"].cpu().numpy()
    got_bf = o["planes_bf16"].view(torch.int16).cpu().numpy().view(np.uint16)
    for b in range(len(games)):
        bad = np.argwhere(got_u8[b] != u8[b])
        assert bad.size == 0, "item %d uint8 channel %s differs" % (b, bad[0])
        badf = np.argwhere(got_bf[b] != bf[b])
        assert badf.size == 0, "item %d bf16 channel %s differs" % (b, badf[0])
    np.testing.assert_array_equal(o["mask"].cpu().numpy(), mask)
    assert (o["status"].cpu().numpy() == 0).all()


def test_obs_ragged_edges_and_invalid_items():
    g, S, A = _games(29, 6)
    # ply 0, the last non-terminal ply, the terminal ply, and invalid items
    games = np.array([0, 1, 2, 3, 4, 5, 0, 1, 7, -1], np.int32)
    L = g["lengths"]
    plies = np.array([0, L[1] - 1, L[2], 1, L[4] - 1, 0, L[0] + 1, 0, 0, 0], np.int16)
    o = st.obs_encode(S, A, torch.from_numpy(games).cuda(), torch.from_numpy(plies).cuda())
    torch.cuda.synchronize()
    status = o["status"].cpu().numpy()
    assert list(status) == [0] * 6 + [1, 0, 1, 1]
    ok = np.nonzero(status == 0)[0]
    u8, bf, mask = oracle.obs_encode(g["setups"], g["actions"], games[ok], plies[ok])
    np.testing.assert_array_equal(o["planes"].cpu().numpy()[ok], u8)
    np.testing.assert_array_equal(o["mask"].cpu().numpy()[ok], mask)
    assert (o["planes"].cpu().numpy()[status == 1] == 0).all()


def test_belief_samples_bit_exact():
    g, S, A = _games(31, 8)
    games, plies = _items(g, 4, seed=2)
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    tp = torch.from_numpy(pos).cuda()
    types, status = st.belief_sample(tp, 37, seed=1234)
    torch.cuda.synchronize()
    ref = oracle.belief_sample(pos, 37, 1234)
    np.testing.assert_array_equal(types.cpu().numpy(), ref)
    sid = torch.arange(len(pos), dtype=torch.int32).flip(0).cuda().contiguous()
    types2, _ = st.belief_sample(tp, 5, seed=7, stream_ids=sid)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(types2.cpu().numpy(), oracle.belief_sample(pos, 5, 7, stream_ids=sid.cpu().numpy()))


@pytest.mark.parametrize("depth,magnet", [(0, False), (1, False), (32, False), (200, False), (1, True), (32, True),
                                          (200, True)])
def test_rollout_tallies_bit_exact(depth, magnet):
    g, S, A = _games(37, 8)
    games, plies = _items(g, 3, seed=3)
    pos = oracle.replay_positions(g["setups"], g["actions"], games, plies)
    tp = torch.from_numpy(pos).cuda()
    flags = st.RULES_ALL | (st.ROLLOUT_MAGNET if magnet else 0)
    tallies, status = st.rollout(tp, 19, depth, seed=99, flags=flags)
    torch.cuda.synchronize()
    ref = oracle.rollout(pos, 19, depth, 99, flags=flags)
    np.testing.assert_array_equal(tallies.cpu().numpy(), ref)
    assert (tallies.cpu().numpy().sum(1) == 19).all()
    # with supplied samples
    types = oracle.belief_sample(pos, 19, 5)
    t2, _ = st.rollout(tp, 19, depth, seed=99, types=torch.from_numpy(types).cuda(), flags=flags)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(t2.cpu().numpy(), oracle.rollout(pos, 19, depth, 99, types=types, flags=flags))
