"""GPU parity under the online game's rule settings: the 200-move rule (App.
A "Additional rule for online play") with the 4,000-ply length cap of
App. D.1, so that channel 42 carries battleless/200 and channel 41
ply/4000 (the evaluation-time fractions).  Every output is compared with the
oracle bit for bit through the C ABI."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2511_07312_gb300 as st  # noqa: E402

K200, CAP = 200, 4000


def test_env_plain_steps_with_masks():
    env = st.Env(64, seed=3, k=K200, cap=CAP)
    outs = {k: [] for k in ("action", "reward", "done", "ply", "mask")}
    for _ in range(600):
        o = env.step()
        for k in outs:
            outs[k].append(o[k].clone())
    env.stream.synchronize()
    gpu = {k: torch.stack(v).cpu().numpy() for k, v in outs.items()}
    ref = oracle.env_run(3, 64, 600, k=K200, cap=CAP)
    for k in outs:
        np.testing.assert_array_equal(gpu[k], ref[k], err_msg=k)
    env.close()


def test_env_persistent_run_4000_plies():
    env = st.Env(64, seed=4, k=K200, cap=CAP)
    out = env.run(4000, 4000, want=("action", "reward", "done", "ply"))
    env.stream.synchronize()
    stats = env.stats().cpu().numpy()
    ref = oracle.env_run(4, 64, 4000, k=K200, cap=CAP, want_mask=False)
    for k in ("action", "reward", "done", "ply"):
        np.testing.assert_array_equal(out[k].cpu().numpy(), ref[k], err_msg=k)
    np.testing.assert_array_equal(stats, ref["stats"].astype(np.int32))
    # games under the 200-move rule do end by it (done code 4)
    assert (ref["done"] == 4).any()
    env.close()


def test_obs_planes_with_the_evaluation_fractions():
    g = oracle.play_games(61, 8, k=K200, cap=CAP)
    rng = np.random.default_rng(61)
    games = np.repeat(np.arange(8), 6).astype(np.int32)
    plies = np.array([rng.integers(0, min(800, g["lengths"][i] - 1) + 1) for i in games], np.int16)
    order = np.lexsort((plies, games))
    games, plies = games[order], plies[order]
    dev = torch.device("cuda", 0)
    o = st.obs_encode(torch.from_numpy(g["setups"]).to(dev), torch.from_numpy(g["actions"]).to(dev),
                      torch.from_numpy(games).to(dev), torch.from_numpy(plies).to(dev), k=K200, cap=CAP)
    torch.cuda.synchronize()
    u8, bf, mask = oracle.obs_encode(g["setups"], g["actions"], games, plies, k=K200, cap=CAP)
    np.testing.assert_array_equal(o["planes"].cpu().numpy(), u8)
    np.testing.assert_array_equal(o["planes_bf16"].view(torch.int16).cpu().numpy().view(np.uint16), bf)
    np.testing.assert_array_equal(o["mask"].cpu().numpy(), mask)


def test_rollouts_and_search_under_the_200_move_rule():
    g = oracle.play_games(62, 4, k=K200, cap=CAP)
    plies = np.minimum(g["lengths"] - 1, [50, 150, 300, 700]).astype(np.int16)
    pos = oracle.replay_positions(g["setups"], g["actions"], np.arange(4), plies, k=K200, cap=CAP)
    tp = torch.from_numpy(pos).cuda()
    tallies, _ = st.rollout(tp, 16, 250, seed=5, k=K200, cap=CAP)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(tallies.cpu().numpy(), oracle.rollout(pos, 16, 250, 5, k=K200, cap=CAP))
    got = st.search(tp, 3, 30, 6, k=K200, cap=CAP)
    torch.cuda.synchronize()
    ref = oracle.search(pos, 3, 30, 6, k=K200, cap=CAP)
    for key in ("n_moves", "actions", "tallies", "q", "chosen", "status"):
        np.testing.assert_array_equal(got[key].cpu().numpy(), ref[key], err_msg=key)
    np.testing.assert_allclose(got["pi"].cpu().numpy(), ref["pi"], rtol=1e-12, atol=0)
