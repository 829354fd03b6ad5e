"""The launch-shape autotuner: picks a shape that exists, caches it, and the
chosen shape gives the same results as any other (parity is shape-free)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_2511_07312_gb300 as st  # noqa: E402
from paper_2511_07312_gb300 import autotune  # noqa: E402


def test_autotune_picks_and_caches_a_valid_shape(tmp_path, monkeypatch):
    monkeypatch.setenv("STRATEGO_GB300_CACHE", str(tmp_path))
    best = autotune.tune(2048, plies=20, reps=1)
    assert best["warps_per_block"] in autotune.WARPS_PER_BLOCK
    assert best["games_per_warp"] in autotune.GAMES_PER_WARP
    assert best["games_per_fetch"] in autotune.GAMES_PER_FETCH
    assert best["blocks_per_sm"] >= 1   # resident blocks per SM: the request clamped to what fits
    assert autotune.load(2048, plies=20) == best
    env = st.Env(64, seed=1)
    env.set_launch(best["warps_per_block"], best["blocks_per_sm"], best["games_per_fetch"],
                   games_per_warp=best["games_per_warp"])
    assert env.launch_shape() == {k: best[k] for k in ("warps_per_block", "blocks_per_sm", "games_per_warp",
                                                       "games_per_fetch")}
    out = env.run(300)
    env.sync()
    ref = oracle.env_run(1, 64, 300)
    for k in ("action", "reward", "done", "ply", "mask"):
        assert np.array_equal(out[k].cpu().numpy(), ref[k]), k
