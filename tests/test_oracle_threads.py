"""The oracle on several host threads, as the benchmark's CPU baseline runs it.

The C oracle keeps no state between calls and its ctypes binding releases
the GIL, so threads that step disjoint slots must reproduce, slot for slot,
what one call over all the slots gives.  The benchmark's thread helpers are
checked for covering every slot or item exactly once."""
import threading

import numpy as np

import bench
import oracle


def test_threaded_slots_equal_one_sequential_call():
    seed, n, plies = 9, 8, 120
    ref = oracle.env_run(seed, n, plies)
    got = [None] * n

    def one(i):
        got[i] = oracle.env_run(seed, 1, plies, slot0=i)

    threads = [threading.Thread(target=one, args=(i,)) for i in range(n)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for key in ("action", "reward", "done", "ply", "mask"):
        whole = ref[key]
        parts = np.concatenate([g[key] for g in got], axis=1)
        np.testing.assert_array_equal(parts, whole, err_msg=key)
    np.testing.assert_array_equal(np.concatenate([g["stats"] for g in got], axis=0), ref["stats"])


def test_oracle_env_slots_covers_each_slot_once(monkeypatch):
    seen = []
    lock = threading.Lock()

    def fake_env_run(seed, n_slots, n_steps, slot0=0, **kw):
        with lock:
            seen.extend(range(slot0, slot0 + n_slots))

    monkeypatch.setattr(oracle, "env_run", fake_env_run)
    bench.oracle_env_slots(1, 5, 37, 10, threads=4, chunk=3)
    assert sorted(seen) == list(range(5, 42))


def test_timed_items_stops_at_the_item_count():
    done = []
    lock = threading.Lock()

    def fn(i):
        with lock:
            done.append(i)

    n, secs = bench.timed_items(fn, 50, 3, budget_s=60.0)
    assert n == 50 and sorted(done) == list(range(50)) and secs >= 0
