"""GPU parity at the benchmark's full sizes, in the launch configuration the
benchmark times, on outputs the oracle computes one by one: the 16,384
observation items, the 4,096-position x 256-sample x depth-32 rollouts, and
the 16,384-slot history query.  Bit for bit."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2511_07312_gb300 as st  # noqa: E402


def _workload3():
    # 64 games of seed 1 to their end or 1,000 plies; 16,384 items at plies
    # uniform in [0, min(600, length - 1)], sorted by (game, ply)
    g = oracle.play_games(1, 64)
    rng = np.random.default_rng(3)
    games = rng.integers(0, 64, 16384).astype(np.int32)
    plies = np.array([rng.integers(0, min(600, max(1, g["lengths"][k]) - 1) + 1) for k in games], np.int16)
    order = np.lexsort((plies, games))
    return g, games[order], plies[order]


def test_observations_16384_items_sampled():
    g, games, plies = _workload3()
    dev = torch.device("cuda", 0)
    o = st.obs_encode(torch.from_numpy(g["setups"]).to(dev), torch.from_numpy(g["actions"]).to(dev),
                      torch.from_numpy(games).to(dev), torch.from_numpy(plies).to(dev))
    torch.cuda.synchronize()
    pick = np.unique(np.r_[0, 1, 7, 8, np.arange(0, 16384, 409), 16383])
    u8, bf, mask = oracle.obs_encode(g["setups"], g["actions"], games[pick], plies[pick])
    np.testing.assert_array_equal(o["planes"][torch.from_numpy(pick).to(dev)].cpu().numpy(), u8)
    got_bf = o["planes_bf16"].view(torch.int16)[torch.from_numpy(pick).to(dev)].cpu().numpy().view(np.uint16)
    np.testing.assert_array_equal(got_bf, bf)
    np.testing.assert_array_equal(o["mask"][torch.from_numpy(pick).to(dev)].cpu().numpy(), mask)
    assert (o["status"].cpu().numpy() == 0).all()


def test_rollouts_4096_positions_256_samples_depth_32_sampled():
    g, games, plies = _workload3()
    sel = np.linspace(0, 16383, 4096).astype(np.int64)
    pos = oracle.replay_positions(g["setups"], g["actions"], games[sel], plies[sel])
    tallies, status = st.rollout(torch.from_numpy(pos).cuda(), 256, 32, seed=7)
    torch.cuda.synchronize()
    t = tallies.cpu().numpy()
    assert (status.cpu().numpy() == 0).all() and (t.sum(1) == 256).all()
    pick = np.array([0, 1, 511, 512, 2047, 3000, 4094, 4095])
    ref = oracle.rollout(pos[pick], 256, 32, 7, stream_ids=pick.astype(np.uint32))
    np.testing.assert_array_equal(t[pick], ref)


def test_history_16384_slots_sampled():
    N, H = 16384, 1000
    env = st.Env(N, seed=5)
    env.set_launch(4, 0, 1, games_per_warp=4)
    env.enable_history(H)
    env.run(H)
    t = env.current_step() - 300
    hp = env.history_positions(t)
    torch.cuda.synchronize()
    status = hp["status"].cpu().numpy()
    pos = hp["pos"].cpu().numpy()
    assert (status == 0).all()
    for g in (0, 1, 151, 152, 8191, 16383):
        ref = oracle.env_run(5, 1, t, slot0=g, want_mask=False, want_final=True)["final"][0]
        np.testing.assert_array_equal(pos[g], ref)
    env.close()
