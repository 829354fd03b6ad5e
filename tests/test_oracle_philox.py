"""Pins of the oracle's Philox4x32-10 against two independent library
implementations that run on the CPU: cuRAND's host-side Philox generator and
Triton's interpreter-mode tl.philox.  (The Random123 known-answer file is not
available here, so these stand in for it.)"""
import ctypes
import ctypes.util
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and os.path.exists(cand) if cand.startswith("/") else cand:
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not found")
    gen = ctypes.c_void_p()
    if cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        nblocks = 65536 + 512      # spans the first two values of counter word 0
        buf = np.zeros(4 * nblocks, np.uint32)
        assert cr.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(buf.size)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    # The host generator emits block j from counter (j // 65536, 0, j % 65536, 0).
    j = np.concatenate([np.arange(0, 2048), np.arange(65536 - 64, nblocks)])
    ctr = np.stack([j // 65536, np.zeros_like(j), j % 65536, np.zeros_like(j)], 1).astype(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    ours = oracle.philox(ctr, key)
    np.testing.assert_array_equal(ours, buf.reshape(-1, 4)[j])


TRITON_SCRIPT = textwrap.dedent(r"""
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(c_ptr, out_ptr, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        c0 = tl.load(c_ptr + 4 * i); c1 = tl.load(c_ptr + 4 * i + 1)
        c2 = tl.load(c_ptr + 4 * i + 2); c3 = tl.load(c_ptr + 4 * i + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out_ptr + 4 * i, a); tl.store(out_ptr + 4 * i + 1, b)
        tl.store(out_ptr + 4 * i + 2, c); tl.store(out_ptr + 4 * i + 3, d)

    ctr = np.load(sys.argv[1]); seed = int(sys.argv[2])
    out = torch.zeros(ctr.size, dtype=torch.int32)
    k[(1,)](torch.from_numpy(ctr.view(np.int32).reshape(-1).copy()), out, seed, ctr.shape[0])
    np.save(sys.argv[3], out.numpy().view(np.uint32).reshape(-1, 4))
""")


def test_philox_matches_triton_interpreter(tmp_path):
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2**32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    seed = 0x9E3779B97F4A7C15
    cpath, opath = tmp_path / "c.npy", tmp_path / "o.npy"
    spath = tmp_path / "t.py"
    np.save(cpath, ctr)
    spath.write_text(TRITON_SCRIPT)
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, str(spath), str(cpath), str(seed), str(opath)], env=env,
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    theirs = np.load(opath)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    np.testing.assert_array_equal(oracle.philox(ctr, key), theirs)


def test_uniform_draw_range_and_balance():
    # floor(r*n/2^32) covers [0,n) with every value hit about equally often
    key = np.array([5, 6], np.uint32)
    ctr = np.stack([np.arange(20000), np.zeros(20000), np.zeros(20000), np.zeros(20000)], 1).astype(np.uint32)
    w = oracle.philox(ctr, key)[:, 0].astype(np.uint64)
    for n in (1, 2, 7, 40, 101):
        v = (w * n) >> 32
        assert v.min() >= 0 and v.max() < n
        counts = np.bincount(v.astype(np.int64), minlength=n)
        expected = len(v) / n
        chi2 = ((counts - expected) ** 2 / expected).sum()
        assert chi2 < n + 6 * np.sqrt(2 * n) + 10
