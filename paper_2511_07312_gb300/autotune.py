"""Launch-shape autotuner of the persistent environment step (st_env_run).

Times short runs of every candidate shape -- warps per block x games per
warp (1, 2, 4 or 8 games side by side in one warp) x slots per queue fetch
x resident blocks per SM (the most that fit, or fewer: with fewer resident
games the last wave of slots can be fuller) -- on a scratch env of the
caller's size and picks the fastest.  Results are cached in a JSON file
keyed by (device name, number of games, library version), so a shape is
tuned once per machine and size.
"""
import json
import os
import time

import torch

from . import Env, version

WARPS_PER_BLOCK = (1, 2, 4, 8)
GAMES_PER_WARP = (1, 2, 4, 8)
GAMES_PER_FETCH = (1, 4)
# 0: as many as fit; the others cap it (tried for 4 and 8 games per warp)
BLOCKS_PER_SM = (0, 4, 5)


def _cache_path():
    base = os.environ.get("STRATEGO_GB300_CACHE") or os.path.join(
        os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")), "stratego_gb300")
    os.makedirs(base, exist_ok=True)
    return os.path.join(base, "launch_shapes.json")


def _key(num_games, device, plies):
    return "%s|%d|%d|%s" % (torch.cuda.get_device_name(device), num_games, plies, version())


def load(num_games, device=0, plies=400):
    """The cached shape for this device, size and launch length (plies per slot), if any."""
    try:
        return json.load(open(_cache_path())).get(_key(num_games, device, plies))
    except (OSError, ValueError):
        return None


def tune(num_games, device=0, plies=400, reps=3, force=False, verbose=False, final_plies=None, finalists=4):
    """Return {"warps_per_block", "games_per_warp", "games_per_fetch",
    "blocks_per_sm" (resident: a request above what fits on an SM is
    clamped, and shapes that clamp to one already timed are skipped),
    "env_steps_per_s"} of the fastest shape, timed with
    CUDA events: every shape on runs of `plies` plies, then (final_plies)
    the `finalists` fastest again on runs of final_plies plies, the length
    the caller will launch (how full the last wave of slots is depends on
    it)."""
    key_plies = final_plies or plies
    if not force:
        hit = load(num_games, device, key_plies)
        if hit:
            return hit
    env = Env(num_games, seed=12345, device=device)
    ring = env.run(1, 4)
    results = []
    seen = set()
    def timed(wpb, gpw, gpf, bps, n_plies, n_reps):
        env.set_launch(wpb, bps, gpf, games_per_warp=gpw)
        env.run(n_plies, 4, out=ring)        # warm-up, captures the graph
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(env.stream)
        for _ in range(n_reps):
            env.run(n_plies, 4, out=ring)
        end.record(env.stream)
        end.synchronize()
        return num_games * n_plies * n_reps / (start.elapsed_time(end) / 1000.0)

    for wpb in WARPS_PER_BLOCK:
        for gpw in GAMES_PER_WARP:
            for gpf in GAMES_PER_FETCH:
                for bps in (BLOCKS_PER_SM if gpw >= 4 else (0,)):
                    try:
                        env.set_launch(wpb, bps, gpf, games_per_warp=gpw)
                    except RuntimeError:
                        continue
                    bps = env.launch_shape()["blocks_per_sm"]   # a request above the occupancy limit is clamped
                    if (wpb, gpw, gpf, bps) in seen:
                        continue
                    seen.add((wpb, gpw, gpf, bps))
                    try:
                        rate = timed(wpb, gpw, gpf, bps, plies, reps)
                    except RuntimeError:
                        continue
                    results.append((rate, wpb, gpw, gpf, bps))
                    if verbose:
                        print("wpb %2d gpw %d gpf %d bps %d: %.3e env-steps/s" % (wpb, gpw, gpf, bps, rate), flush=True)
    if final_plies and final_plies != plies:
        final = []
        for _, wpb, gpw, gpf, bps in sorted(results, reverse=True)[:finalists]:
            rate = timed(wpb, gpw, gpf, bps, final_plies, 2)
            final.append((rate, wpb, gpw, gpf, bps))
            if verbose:
                print("final wpb %2d gpw %d gpf %d bps %d: %.3e env-steps/s" % (wpb, gpw, gpf, bps, rate), flush=True)
        results = final
        plies = final_plies
    env.close()
    rate, wpb, gpw, gpf, bps = max(results)
    best = {"warps_per_block": wpb, "games_per_warp": gpw, "games_per_fetch": gpf, "blocks_per_sm": bps,
            "env_steps_per_s": rate, "plies": plies, "tuned_at": time.strftime("%Y-%m-%dT%H:%M:%S")}
    path = _cache_path()
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        data = {}
    data[_key(num_games, device, key_plies)] = best
    tmp = path + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1)
    os.replace(tmp, path)
    return best
