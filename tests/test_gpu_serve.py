"""Serving with continuous batching: each request's result alone equals its
result in a mix of concurrent requests of uneven size, and both equal
st_rollout and the oracle bit for bit (tolerance zero: the tallies are
integers)."""
import threading
import time

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2511_07312_gb300 as st  # noqa: E402


def _positions(seed, n):
    g = oracle.play_games(seed, n)
    rng = np.random.default_rng(seed)
    games = np.arange(n, dtype=np.int32)
    plies = np.array([rng.integers(0, min(600, g["lengths"][i] - 1) + 1) for i in games], np.int16)
    return oracle.replay_positions(g["setups"], g["actions"], games, plies)


def _requests(pos, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(len(pos)):
        K = int(rng.integers(1, 200))
        D = int(rng.integers(0, 40))
        reqs.append((pos[i], K, D, 1000 + i, int(rng.integers(0, 2**32))))
    return reqs


def test_each_request_alone_equals_rollout_and_oracle():
    pos = _positions(51, 6)
    srv = st.Server(max_requests=8, sample_slots=4096, max_batches=2)
    try:
        for p, K, D, seed, sid in _requests(pos, 1):
            t = srv.submit(p, K, D, seed, sid)
            tallies, timing = srv.wait(t, 60000)
            assert timing[0] <= timing[1] <= timing[2]
            ref = oracle.rollout(p[None], K, D, seed, stream_ids=[sid])[0]
            np.testing.assert_array_equal(tallies, ref)
            got, _ = st.rollout(torch.from_numpy(p[None].copy()).cuda(), K, D, seed,
                                stream_ids=torch.tensor([sid], dtype=torch.int64).to(torch.int32).cuda())
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got.cpu().numpy()[0], ref)
    finally:
        srv.close()


def test_mix_of_concurrent_requests_equals_alone_results():
    pos = _positions(53, 24)
    reqs = _requests(pos, 2)
    alone = [oracle.rollout(p[None], K, D, seed, stream_ids=[sid])[0] for p, K, D, seed, sid in reqs]
    # a small sample pool forces admission to wait for memory; several batches in flight
    srv = st.Server(max_requests=6, sample_slots=400, max_batches=3)
    try:
        tickets = []
        for i, (p, K, D, seed, sid) in enumerate(reqs):
            tickets.append(srv.submit(p, K, D, seed, sid))
            if i % 5 == 4:
                time.sleep(0.002)   # some requests arrive while others run
        for t, ref in zip(tickets, alone):
            tallies, _ = srv.wait(t, 60000)
            np.testing.assert_array_equal(tallies, ref)
        stats = srv.stats()
        assert stats["completed"] == len(reqs) and stats["queued"] == 0 and stats["running"] == 0
        assert stats["batches"] >= 2
    finally:
        srv.close()


def test_submissions_from_several_threads():
    pos = _positions(55, 12)
    reqs = _requests(pos, 3)
    srv = st.Server(max_requests=16, sample_slots=8192, max_batches=4)
    results = {}
    try:
        def client(idx):
            for i in idx:
                p, K, D, seed, sid = reqs[i]
                t = srv.submit(p, K, D, seed, sid)
                results[i] = srv.wait(t, 60000)[0]
        ths = [threading.Thread(target=client, args=(list(range(j, len(reqs), 3)),)) for j in range(3)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        for i, (p, K, D, seed, sid) in enumerate(reqs):
            np.testing.assert_array_equal(results[i], oracle.rollout(p[None], K, D, seed, stream_ids=[sid])[0])
    finally:
        srv.close()


def test_edge_requests():
    pos = _positions(57, 2)
    srv = st.Server(max_requests=4, sample_slots=64, max_batches=2)
    try:
        # K = 0: empty tallies
        t = srv.submit(pos[0], 0, 10, 1, 0)
        tallies, _ = srv.wait(t, 10000)
        assert tallies.tolist() == [0, 0, 0, 0]
        # depth 0: every rollout is unfinished
        t = srv.submit(pos[0], 7, 0, 1, 0)
        assert srv.wait(t, 10000)[0].tolist() == [0, 0, 0, 7]
        # an invalid root is reported, not run
        bad = pos[1].copy()
        bad[0] = 99
        t = srv.submit(bad, 5, 5, 1, 0)
        with pytest.raises(st.StrategoError) as ei:
            srv.wait(t, 10000)
        assert ei.value.code == 8
        # K beyond the sample pool is refused at submit
        with pytest.raises(st.StrategoError) as ei:
            srv.submit(pos[0], 65, 5, 1, 0)
        assert ei.value.code == 1
        # unknown ticket
        with pytest.raises(st.StrategoError) as ei:
            srv.poll(123456789)
        assert ei.value.code == 1
        # a wait that runs out reports a timeout and the result stays available
        t = srv.submit(pos[0], 64, 400, 1, 0)
        try:
            srv.wait(t, 0)
        except st.StrategoError as e:
            assert e.code in (5, 7)
        tallies, _ = srv.wait(t, 60000)
        assert tallies.sum() == 64
    finally:
        srv.close()


def test_server_with_the_magnet_rollout_policy():
    pos = _positions(57, 4)
    flags = st.RULES_ALL | st.ROLLOUT_MAGNET
    srv = st.Server(max_requests=4, sample_slots=2048, max_batches=2, flags=flags)
    try:
        for p, K, D, seed, sid in _requests(pos, 4):
            tallies, _ = srv.wait(srv.submit(p, K, D, seed, sid), 60000)
            np.testing.assert_array_equal(tallies, oracle.rollout(p[None], K, D, seed, stream_ids=[sid],
                                                                  flags=flags)[0])
    finally:
        srv.close()


def test_burst_from_several_threads_and_immediate_polls():
    # submissions return before the scheduler has seen them; a ticket polled
    # at once is not ready (never unknown), and every result is exact
    pos = _positions(59, 8)
    reqs = _requests(pos, 6) * 4
    srv = st.Server(max_requests=32, sample_slots=4096, max_batches=4)
    tickets = [None] * len(reqs)
    early = {}
    try:
        def client(j):
            for i in range(j, len(reqs), 4):
                p, K, D, seed, sid = reqs[i]
                tickets[i] = srv.submit(p, K, D, seed, sid)
                try:
                    early[i] = srv.poll(tickets[i])[0]     # done already: the result is taken here
                except st.StrategoError as e:
                    assert e.code == 7, str(e)           # not ready; never unknown
        ths = [threading.Thread(target=client, args=(j,)) for j in range(4)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        want = {}
        for i, (p, K, D, seed, sid) in enumerate(reqs):
            key = (i % len(pos), K, D, seed, sid)
            if key not in want:
                want[key] = oracle.rollout(p[None], K, D, seed, stream_ids=[sid])[0]
            tallies = early[i] if i in early else srv.wait(tickets[i], 60000)[0]
            np.testing.assert_array_equal(tallies, want[key])
        with pytest.raises(st.StrategoError, match="invalid argument"):
            srv.poll(tickets[0])                      # already taken: unknown now
    finally:
        srv.close()
