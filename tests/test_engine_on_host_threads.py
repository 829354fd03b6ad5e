"""The engine's CUDA source run on host threads under sanitizers.

compute-sanitizer is not available to this project, so the device code of
the environment (csrc/engine.cuh and the kernels of csrc/env.cu) is also
compiled with g++ against a host stand-in for the CUDA features it uses
(tests/simt_host: one std::thread per lane, warp collectives as
rendezvous of the lanes in their mask, bulk copies performed at their
wait) and run under ThreadSanitizer (data races between the lanes of a
team, between teams and between blocks sharing the work queue) and under
AddressSanitizer with UndefinedBehaviorSanitizer.  Every ply's action,
reward, ending, ply counter and legal mask and every slot's counters must
equal the oracle's, for teams of 4, 8, 16 and 32 lanes.  Only the inline
assembly of the bulk copies is rewritten for the host."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_07312_gb300", "csrc")
HARNESS = os.path.join(ROOT, "tests", "simt_host")


def _host_source(text):
    """The CUDA source with its shared-memory declaration and its bulk-copy
    inline assembly replaced by the harness's host equivalents."""
    text = text.replace("extern __shared__ __align__(16) unsigned char smem[];",
                        "unsigned char* const smem = emu::block_smem();")
    text = text.replace('asm volatile("fence.proxy.async.shared::cta;" ::: "memory");', ";")
    text = re.sub(r'const uint32_t src = static_cast<uint32_t>\(__cvta_generic_to_shared\(G->mask\)\);\s*'
                  r'asm volatile\("cp\.async\.bulk\.global\.shared::cta\.bulk_group \[%0\], \[%1\], %2;"\s*'
                  r'::\s*"l"\(dst\), "r"\(src\), "r"\(\(uint32_t\)kMaskBytes\) : "memory"\);\s*'
                  r'asm volatile\("cp\.async\.bulk\.commit_group;" ::: "memory"\);',
                  "emu::bulk_copy(dst, G->mask, kMaskBytes);", text)
    text = text.replace('asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");', "emu::bulk_wait();")
    text = text.replace('asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");', "emu::bulk_wait();")
    assert "asm" not in re.sub(r"//.*", "", text), "inline assembly the harness does not know"
    return text


def _prepare(dst, edit=None):
    for f in ("engine.cuh", "snapshot.cuh", "rollout.cuh", "features.cuh"):
        text = _host_source(open(os.path.join(CSRC, f)).read())
        if edit is not None:
            text = edit(f, text)
        with open(os.path.join(dst, f), "w") as o:
            o.write(text)
    lines = open(os.path.join(CSRC, "env.cu")).read().split("\n")
    start = next(i for i, l in enumerate(lines) if l.startswith("namespace {"))
    end = next(i for i, l in enumerate(lines) if l.startswith("// ") and "snapshots" in l and "-----" in l)
    pre = [l for l in lines[:start] if (l.startswith("#include") or l.startswith("using namespace"))
           and "host_common.h" not in l]
    with open(os.path.join(dst, "env_dev.cu"), "w") as o:
        o.write(_host_source("\n".join(pre + lines[start:end]) + "\n}  // namespace\n"))


def _build(tmp, flags, name, edit=None):
    src = os.path.join(tmp, "src")
    os.makedirs(src, exist_ok=True)
    _prepare(src, edit)
    exe = os.path.join(tmp, name)
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-pthread", "-w", "-I", os.path.join(HARNESS, "include"),
           "-I", src, "-I", os.path.join(ROOT, "include"), os.path.join(HARNESS, "env_on_host.cpp"), "-o", exe] + flags
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        if "sanitize" in r.stderr or "cannot find" in r.stderr:
            pytest.skip("sanitizer runtime unavailable: %s" % r.stderr[-300:])
        raise AssertionError(r.stderr[-4000:])
    return exe


def _run_and_compare(exe, tmp, N, S, L, wpb, gpf, blocks, seed, env=None):
    out = os.path.join(tmp, "o_%d_%d_%d_%d" % (L, wpb, gpf, blocks))
    r = subprocess.run([exe, str(N), str(S), str(L), str(wpb), str(gpf), str(blocks), str(seed), out],
                       capture_output=True, text=True, timeout=900, env=dict(os.environ, **(env or {})))
    report = r.stdout + r.stderr
    if r.returncode != 0 and "FATAL: ThreadSanitizer" in report and "memory" in report:
        pytest.skip("ThreadSanitizer cannot start here: %s" % report[-300:])
    assert r.returncode == 0, report[-6000:]
    assert "WARNING: ThreadSanitizer" not in report, report[-6000:]
    assert "runtime error" not in report and "ERROR: AddressSanitizer" not in report, report[-6000:]
    assert "status 0 " in r.stdout, report[-2000:]
    ref = oracle.env_run(seed, N, S)
    for k, dt in (("action", np.int16), ("reward", np.int8), ("done", np.uint8), ("ply", np.int16)):
        got = np.fromfile(out + "." + k, dtype=dt).reshape(S, N)
        bad = np.argwhere(got != ref[k])
        assert bad.size == 0, "%s differs first at (ply, slot) %s" % (k, bad[0])
    mask = np.fromfile(out + ".mask", dtype=np.uint8).reshape(S, N, oracle.MASK_BYTES)
    bad = np.argwhere((mask != ref["mask"]).any(-1))
    assert bad.size == 0, "mask differs first at (ply, slot) %s" % bad[0]
    stats = np.fromfile(out + ".stats", dtype=np.uint32).reshape(N, 8)
    np.testing.assert_array_equal(stats, ref["stats"])


@pytest.fixture(scope="module")
def tsan_exe(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("tsan"))
    return _build(tmp, ["-fsanitize=thread"], "env_tsan"), tmp


@pytest.mark.parametrize("L,wpb,gpf,blocks", [(8, 1, 1, 1), (4, 1, 2, 1), (16, 2, 1, 2), (32, 2, 1, 1)])
def test_step_kernel_under_threadsanitizer(tsan_exe, L, wpb, gpf, blocks):
    exe, tmp = tsan_exe
    _run_and_compare(exe, tmp, 12, 160, L, wpb, gpf, blocks, 7,
                     env={"TSAN_OPTIONS": "halt_on_error=1:second_deadlock_stack=1"})


def test_step_kernel_under_address_and_ub_sanitizers(tmp_path):
    exe = _build(str(tmp_path), ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined"], "env_asan")
    for L, wpb, gpf, blocks in ((8, 2, 1, 2), (4, 1, 1, 1)):
        _run_and_compare(exe, str(tmp_path), 16, 300, L, wpb, gpf, blocks, 11,
                         env={"ASAN_OPTIONS": "detect_leaks=0"})


def test_harness_reports_a_planted_missing_sync(tmp_path):
    # the check itself: without the team barrier between clearing the board
    # and placing the pieces, ThreadSanitizer must report a race
    sync = ("    for (int s = T.tl; s < 112; s += L) G->board[s] = (s < 100 && is_lake(s)) ? kLake : kEmpty;\n"
            "    T.sync();")

    def drop_sync(name, text):
        if name != "engine.cuh":
            return text
        assert sync in text
        return text.replace(sync, sync.split("\n")[0])

    exe = _build(str(tmp_path), ["-fsanitize=thread"], "env_race", edit=drop_sync)
    r = subprocess.run([exe, "4", "20", "8", "1", "1", "1", "7", str(tmp_path / "o")], capture_output=True,
                       text=True, timeout=600, env=dict(os.environ, TSAN_OPTIONS="halt_on_error=1"))
    report = r.stdout + r.stderr
    if r.returncode != 0 and "FATAL: ThreadSanitizer" in report and "memory" in report:
        pytest.skip("ThreadSanitizer cannot start here")
    assert "WARNING: ThreadSanitizer: data race" in report and "build_board" in report, report[-3000:]
