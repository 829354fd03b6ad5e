"""The launch-shape autotuner's host logic, on the CPU: a fake env stands in
for the library (its own occupancy limits, a shape it refuses, and a
simulated throughput per shape) and a fake CUDA event reads that throughput
back as elapsed time.  Checked: a shape the library refuses is skipped, a
blocks-per-SM request that the occupancy limit clamps to a shape already
timed is not timed again, the finalists are re-timed at the caller's launch
length, the fastest shape wins with its resident blocks per SM, and the
result is cached."""
import pytest

torch = pytest.importorskip("torch")

from paper_2511_07312_gb300 import autotune  # noqa: E402

N = 4096


def _occupancy(wpb, gpw):
    # resident blocks per SM the fake library allows for a shape
    return max(1, 24 // (wpb * max(1, gpw // 2)))


def _rate(wpb, gpw, gpf, bps, plies):
    # simulated env-steps/s; the launch length changes the order of the top two
    base = 1e9 + 1e7 * wpb + 3e7 * gpw - 1e6 * gpf + 2e6 * bps
    if plies >= 1000 and (wpb, gpw) == (2, 8):
        base += 5e8
    return base


class FakeEnv:
    instances = []

    def __init__(self, num_games, seed=0, device=0):
        self.N = num_games
        self.shape = None
        self.work = 0.0          # simulated seconds of device work so far
        self.stream = self
        self.timed = []          # (shape, plies) of every run
        self.closed = False
        FakeEnv.instances.append(self)

    def set_launch(self, wpb, bps, gpf, games_per_warp=1):
        if wpb == 8 and games_per_warp == 8:
            raise RuntimeError("does not fit")
        occ = _occupancy(wpb, games_per_warp)
        self.shape = (wpb, games_per_warp, gpf, occ if bps == 0 else min(bps, occ))

    def launch_shape(self):
        wpb, gpw, gpf, bps = self.shape
        return {"warps_per_block": wpb, "blocks_per_sm": bps, "games_per_warp": gpw, "games_per_fetch": gpf}

    def run(self, n_plies, ring_steps, out=None):
        if self.shape is not None:
            self.timed.append((self.shape, n_plies))
            self.work += self.N * n_plies / _rate(*self.shape, n_plies)
        return {}

    def close(self):
        self.closed = True


class FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream):
        self.t = stream.work

    def synchronize(self):
        pass

    def elapsed_time(self, end):
        return (end.t - self.t) * 1000.0


@pytest.fixture
def fake(monkeypatch, tmp_path):
    FakeEnv.instances.clear()
    monkeypatch.setenv("STRATEGO_GB300_CACHE", str(tmp_path))
    monkeypatch.setattr(autotune, "Env", FakeEnv)
    monkeypatch.setattr(autotune.torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(autotune, "_key", lambda n, d, p: "fake|%d|%d" % (n, p))
    return FakeEnv


def test_each_resident_shape_is_timed_once_and_refused_shapes_are_skipped(fake):
    best = autotune.tune(N, plies=20, reps=2, force=True)
    env = fake.instances[-1]
    assert env.closed
    first = [shape for shape, plies in env.timed if plies == 20]
    # each timing is one warm-up run plus `reps` timed runs of the same shape
    counts = {}
    for shape in first:
        counts[shape] = counts.get(shape, 0) + 1
    assert all(c == 3 for c in counts.values()), counts
    expected = set()
    for wpb in autotune.WARPS_PER_BLOCK:
        for gpw in autotune.GAMES_PER_WARP:
            if wpb == 8 and gpw == 8:
                continue
            for gpf in autotune.GAMES_PER_FETCH:
                occ = _occupancy(wpb, gpw)
                for bps in (autotune.BLOCKS_PER_SM if gpw >= 4 else (0,)):
                    expected.add((wpb, gpw, gpf, occ if bps == 0 else min(bps, occ)))
    assert set(counts) == expected
    assert all(s[0] != 8 or s[1] != 8 for s in counts)
    # the fastest at 20 plies, reported with its resident blocks per SM
    top = max(expected, key=lambda s: _rate(*s, 20))
    assert (best["warps_per_block"], best["games_per_warp"], best["games_per_fetch"],
            best["blocks_per_sm"]) == top
    assert best["plies"] == 20


def test_finalists_are_retimed_at_the_launch_length_and_cached(fake):
    best = autotune.tune(N, plies=20, reps=1, force=True, final_plies=2000, finalists=3)
    env = fake.instances[-1]
    final = [shape for shape, plies in env.timed if plies == 2000]
    assert len(set(final)) == 3
    # the launch length reorders the shapes: 2 warps x 8 games, second at 20
    # plies behind 4 x 8, wins at 2,000
    short = max(set(s for s, p in env.timed if p == 20), key=lambda s: _rate(*s, 20))
    assert short[:2] == (4, 8)
    assert (best["warps_per_block"], best["games_per_warp"], best["games_per_fetch"]) == (2, 8, 1)
    assert best["plies"] == 2000
    assert autotune.load(N, plies=2000) == best
    # a second call is served from the cache without a new env
    n_envs = len(fake.instances)
    assert autotune.tune(N, plies=20, final_plies=2000) == best
    assert len(fake.instances) == n_envs
