"""GPU parity of the per-candidate-move search (App. E "Search", steps 1-4)
with the oracle, through the C ABI.

Move lists, tallies and values are compared bit for bit.  The updated
policy is compared within 1e-12 relative: both sides round every product,
sum and quotient of the update one at a time in the same order in double,
and only the library log and exp may differ, by an ulp or two, which the
division by alpha + beta = 0.022 amplifies about 50-fold at most.  The
played move is compared exactly unless the oracle's uniform draw lies
within 1e-10 of a boundary of the cumulative policy, where that ulp-level
difference can decide it."""
import numpy as np
import pytest

import oracle
from tests.helpers import FLAG, MARSHAL, SERGEANT, F_MOVED, make_position, sq

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2511_07312_gb300 as st  # noqa: E402

PI_RTOL = 1e-12


def _positions(seed, n, per_game, upto=400):
    g = oracle.play_games(seed, n)
    rng = np.random.default_rng(seed)
    games = np.repeat(np.arange(n), per_game).astype(np.int32)
    plies = np.array([rng.integers(0, min(upto, g["lengths"][i] - 1) + 1) for i in games], np.int16)
    return oracle.replay_positions(g["setups"], g["actions"], games, plies)


def _uniform_draw(seed, stream):
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    w = oracle.philox(np.array([[stream, 0, 0, 6 << 24]], np.uint32), key)[0]
    return ((int(w[0]) >> 5) * 67108864.0 + (int(w[1]) >> 6)) / 9007199254740992.0


def _compare(got, ref, seed, stream_ids=None):
    g = {k: v.cpu().numpy() for k, v in got.items()}
    np.testing.assert_array_equal(g["status"], ref["status"])
    np.testing.assert_array_equal(g["n_moves"], ref["n_moves"])
    np.testing.assert_array_equal(g["actions"], ref["actions"])
    np.testing.assert_array_equal(g["tallies"], ref["tallies"])
    np.testing.assert_array_equal(g["q"], ref["q"])
    np.testing.assert_allclose(g["pi"], ref["pi"], rtol=PI_RTOL, atol=0)
    for p in range(len(ref["chosen"])):
        if g["chosen"][p] == ref["chosen"][p]:
            continue
        n = ref["n_moves"][p]
        stream = p if stream_ids is None else int(stream_ids[p])
        u = _uniform_draw(seed, stream)
        edge = np.abs(np.cumsum(ref["pi"][p, :n]) - u).min()
        assert edge < 1e-10, "position %d: chosen %d, oracle %d (draw %.17g, %.3g from a boundary)" % (
            p, g["chosen"][p], ref["chosen"][p], u, edge)


@pytest.mark.parametrize("S,depth,magnet", [(5, 1, False), (7, 9, False), (3, 80, False), (4, 9, True),
                                            (3, 80, True)])
def test_search_matches_oracle(S, depth, magnet):
    pos = _positions(41, 6, 2)   # 12 positions: not a multiple of the warps per block
    seed = 1000 + depth
    flags = st.RULES_ALL | (st.ROLLOUT_MAGNET if magnet else 0)
    got = st.search(torch.from_numpy(pos).cuda(), S, depth, seed, flags=flags)
    torch.cuda.synchronize()
    ref = oracle.search(pos, S, depth, seed, flags=flags)
    assert (ref["status"] == 0).all() and (ref["n_moves"] > 0).all()
    _compare(got, ref, seed)
    t = got["tallies"].cpu().numpy()
    n = ref["n_moves"]
    for p in range(len(pos)):
        assert (t[p, :n[p]].sum(-1) == S).all() and (t[p, n[p]:] == 0).all()


def test_search_with_a_move_prior_and_stream_ids():
    pos = _positions(43, 5, 3)
    ref0 = oracle.search(pos, 0, 1, 0)
    rng = np.random.default_rng(5)
    pt = np.zeros((len(pos), 10000), np.float32)
    for p in range(len(pos)):
        n = ref0["n_moves"][p]
        vals = rng.dirichlet(np.ones(n)).astype(np.float32)
        vals[rng.random(n) < 0.2] = 0.0          # some legal moves excluded by the prior
        if vals.sum() == 0:
            vals[0] = 1.0
        pt[p, ref0["actions"][p, :n]] = vals
    pt[:, 9999] = 0.5                             # an illegal action's entry is never read
    sid = (np.arange(len(pos), dtype=np.uint32) * 7919 + 3).astype(np.int32)
    seed = 0xDEADBEEF12345
    got = st.search(torch.from_numpy(pos).cuda(), 6, 12, seed, stream_ids=torch.from_numpy(sid).cuda(),
                    pi_theta=torch.from_numpy(pt).cuda(), alpha=0.01, beta=0.05)
    torch.cuda.synchronize()
    ref = oracle.search(pos, 6, 12, seed, stream_ids=sid.view(np.uint32), pi_theta=pt, alpha=0.01, beta=0.05)
    _compare(got, ref, seed, stream_ids=sid.view(np.uint32))
    pi = got["pi"].cpu().numpy()
    acts = got["actions"].cpu().numpy()
    for p in range(len(pos)):
        n = ref["n_moves"][p]
        assert (pi[p, :n][pt[p, acts[p, :n]] == 0] == 0).all()
        assert abs(pi[p, :n].sum() - 1.0) < 1e-12


def test_search_degenerate_inputs():
    live = make_position([(0, MARSHAL, sq("e4"), F_MOVED), (0, SERGEANT, sq("a1"), 0), (0, FLAG, sq("j1"), 0),
                          (1, FLAG, sq("j10"), 0), (1, SERGEANT, sq("a10"), 0)])
    stuck = make_position([(0, FLAG, sq("a1"), 0), (1, FLAG, sq("j10"), 0), (1, SERGEANT, sq("a10"), 0)])
    bad = live.copy()
    bad[0] = 99
    pos = np.stack([live, stuck, bad, live, live])
    pt = np.zeros((5, 10000), np.float32)
    pt[0] = 1.0 / 10000
    pt[4] = 1.0 / 10000                           # position 3: zero on every legal move
    for S in (0, 4):
        got = st.search(torch.from_numpy(pos).cuda(), S, 6, 77, pi_theta=torch.from_numpy(pt).cuda())
        torch.cuda.synchronize()
        ref = oracle.search(pos, S, 6, 77, pi_theta=pt)
        assert ref["status"].tolist() == [0, 0, 1, 2, 0]
        assert ref["n_moves"][1] == 0 and ref["chosen"][1] == -1 and ref["chosen"][3] == -1
        _compare(got, ref, 77)
    # no positions: nothing to do
    empty = torch.empty((0, oracle.POS_BYTES), dtype=torch.uint8, device="cuda")
    out = st.search(empty, 4, 4, 1)
    assert out["n_moves"].numel() == 0
    # argument errors are reported before anything is enqueued
    for kw in (dict(depth=0), dict(S=-1), dict(alpha=0.0, beta=0.0), dict(alpha=-1.0)):
        args = dict(S=4, depth=4, alpha=0.002, beta=0.02)
        args.update(kw)
        with pytest.raises(st.StrategoError):
            st.search(torch.from_numpy(pos).cuda(), args["S"], args["depth"], 1, alpha=args["alpha"],
                      beta=args["beta"])


def test_search_full_size_all_positions():
    # the benchmark's search workload (256 positions, 16 configurations,
    # depth 40), every position against the oracle; position p's stream id
    # is p on both sides, so a sample keeps its own results as well
    pos = _positions(47, 64, 4, upto=600)
    S, depth, seed = 16, 40, 2024
    got = st.search(torch.from_numpy(pos).cuda(), S, depth, seed)
    torch.cuda.synchronize()
    _compare(got, oracle.search(pos, S, depth, seed), seed)
    pick = np.array([0, 1, 63, 128, 200, 255])
    ref = oracle.search(pos[pick], S, depth, seed, stream_ids=pick.astype(np.uint32))
    sub = {k: v[torch.from_numpy(pick).cuda()] for k, v in got.items()}
    _compare(sub, ref, seed, stream_ids=pick)
    t = got["tallies"].cpu().numpy()
    n = got["n_moves"].cpu().numpy()
    assert (got["status"].cpu().numpy() == 0).all()
    for p in range(len(pos)):
        assert (t[p, :n[p]].sum(-1) == S).all()


def test_search_with_given_values():
    pos = _positions(49, 4, 3)
    ref0 = oracle.search(pos, 0, 1, 0)
    rng = np.random.default_rng(9)
    qv = rng.uniform(-1, 1, size=(len(pos), 10000)).astype(np.float32)
    for magnet in (False, True):
        flags = st.RULES_ALL | (st.ROLLOUT_MAGNET if magnet else 0)
        got = st.search(torch.from_numpy(pos).cuda(), 5, 30, 17, q_values=torch.from_numpy(qv).cuda(), flags=flags)
        torch.cuda.synchronize()
        ref = oracle.search(pos, 5, 30, 17, q_values=qv, flags=flags)
        _compare(got, ref, 17)
        assert (got["tallies"].cpu().numpy() == 0).all()
        for p in range(len(pos)):
            n = ref0["n_moves"][p]
            np.testing.assert_array_equal(got["q"].cpu().numpy()[p, :n],
                                          qv[p, ref0["actions"][p, :n]].astype(np.float64))
