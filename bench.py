"""Benchmark of the GB300 Stratego engine.

Default workload (the headline): 65,536 parallel game slots, random legal
policy, auto-reset, 2,000 plies per slot per step through the persistent
launch (st_env_run), every ply's 1,264-byte legal mask, action, reward, done
flag and ply counter written to a 16-row output ring (1.3 GB, larger than L2).
Reported: env-steps/s, the HBM roofline of the step kernel, the plain
per-ply launch path beside it, an end-to-end number through the public API
with host buffers, and the oracle on the host cores.  Secondary workloads:
observation planes for 16,384 replayed positions and belief-sample rollouts
for 4,096 positions x 256 samples x depth 32.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MASK_BYTES = 1264
BYTES_PER_ENV_STEP = MASK_BYTES + 2 + 1 + 1 + 2   # mask + action + reward + done + ply


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--games", type=int, default=65536)
    p.add_argument("--plies", type=int, default=2000, help="plies per slot per step")
    p.add_argument("--ring", type=int, default=16)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--wpb", type=int, default=0, help="warps per block (0 = tuned default)")
    p.add_argument("--gpf", type=int, default=0, help="games per queue fetch (0 = tuned default)")
    p.add_argument("--gpw", type=int, default=0, help="games per warp, 1, 2, 4 or 8 (0 = tuned default)")
    p.add_argument("--bps", type=int, default=0, help="resident blocks per SM with --wpb/--gpw (0 = as many as fit)")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--profile", nargs="?", const="step", default=None, choices=["step", "rollout", "obs"],
                   help="for profiler captures: time one workload only -- the persistent step launch "
                        "(step, the default), the belief-sample rollouts of 4,096 positions (rollout) or "
                        "the observation planes of 16,384 replayed positions (obs); no plain path, "
                        "end-to-end, other workloads or CPU baseline")
    return p.parse_args()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def workload_config(games, plies, ring):
    """The config object both arms print for the env-step workload."""
    return {"workload": "%s random-policy Stratego games, auto-reset, %s plies per slot per step" % (
                "{:,}".format(games), "{:,}".format(plies)),
            "games_per_gpu": games, "plies_per_step": plies, "ring_rows": ring,
            "l2": "output ring %.2f GB > L2 (inputs larger than L2, no flush)" % (ring * games * MASK_BYTES / 1e9)}


def job_rate(units_per_rank, ms_local, world, dist=None, device="cpu"):
    """Whole-job throughput of a weak-scaling run: the units all ranks
    processed divided by the slowest rank's time (max over ranks).  Returns
    (units per second, that time in ms)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return float(units_per_rank) * world / (ms / 1000.0), ms


# The sources the step kernel is compiled from (env.cu and what it includes).
STEP_KERNEL_SOURCES = ("paper_2511_07312_gb300/csrc/env.cu", "paper_2511_07312_gb300/csrc/engine.cuh",
                       "paper_2511_07312_gb300/csrc/snapshot.cuh", "paper_2511_07312_gb300/csrc/rollout.cuh",
                       "paper_2511_07312_gb300/csrc/host_common.h", "include/stratego.h")


def _code_only(text):
    """Source text without comments and with whitespace runs collapsed, so
    that editing a comment does not count as changing the kernel."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for rel in STEP_KERNEL_SOURCES:
        h.update(os.path.basename(rel).encode())
        h.update(_code_only(open(os.path.join(ROOT, rel), encoding="utf-8").read()).encode())
    return h.hexdigest()


def profile_value(name, key):
    """A machine-readable line `key: value` of a committed ncu summary under
    profiles/, or None when the step kernel's code changed since the capture
    (the summary's sources_sha256 line no longer matches)."""
    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        parts = line.strip().split(":", 1)
        if len(parts) == 2:
            vals[parts[0].strip()] = parts[1].strip()
    if vals.get("sources_sha256") != kernel_sources_sha256() or key not in vals:
        return None
    return float(vals[key])


def measured_traffic_per_env_step():
    """DRAM bytes per env-step of the step kernel from the committed ncu
    summary, or None when the kernel sources changed since that capture."""
    return profile_value("k_env_run_traffic.md", "traffic_bytes_per_env_step")


# Issue slots of one GB300: 152 SMs x 4 schedulers x one warp instruction a
# cycle at the 2,070 MHz maximum SM clock.
ISSUE_PEAK_WARP_INST_PER_S = 152 * 4 * 2.07e9


def issue_view(env_steps_per_s_per_gpu, hbm_peak_gbs):
    ipe = profile_value("k_env_run_16384games_100plies.md", "warp_inst_per_env_step")
    lanes = profile_value("k_env_run_16384games_100plies.md", "active_lanes_per_warp_inst")
    if ipe is None:
        return None
    achieved = env_steps_per_s_per_gpu * ipe
    return {"achieved": achieved, "peak": ISSUE_PEAK_WARP_INST_PER_S, "unit": "warp-inst/s",
            "frac": achieved / ISSUE_PEAK_WARP_INST_PER_S, "warp_inst_per_env_step": ipe,
            "active_lanes_per_warp_inst": lanes,
            "note": "instructions per env-step from profiles/k_env_run_16384games_100plies.md; the step's "
                    "binding ceiling: issue allows %.2e env-steps/s, HBM %.2e" %
                    (ISSUE_PEAK_WARP_INST_PER_S / ipe, hbm_peak_gbs * 1e9 / BYTES_PER_ENV_STEP)}


# ---------------------------------------------------------------- oracle on the host

def host_threads():
    """Host threads for the oracle: the cores this process may run on."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_env_slots(seed, slot0, n_slots, plies, threads, chunk):
    """Run the oracle environment over slots slot0 .. slot0+n_slots-1 on
    `threads` host threads, each taking `chunk` slots at a time (the C oracle
    runs with the GIL released, and slots are independent).  Returns the
    wall time in seconds."""
    import oracle
    oracle.lib()   # load the library once, before the threads
    nxt = [slot0]
    lock = threading.Lock()

    def worker():
        while True:
            with lock:
                s = nxt[0]
                if s >= slot0 + n_slots:
                    return
                n = min(chunk, slot0 + n_slots - s)
                nxt[0] = s + n
            oracle.env_run(seed, n, plies, slot0=s)

    t0 = time.perf_counter()
    pool = [threading.Thread(target=worker) for _ in range(threads)]
    for t in pool:
        t.start()
    for t in pool:
        t.join()
    return time.perf_counter() - t0


def oracle_env_rate(seed, plies, budget_s=12.0, chunk=16, threads=1):
    """Oracle env-steps/s over a bounded sample of slots: rounds of
    `threads` x `chunk` slots until about budget_s seconds have passed."""
    t_all = 0.0
    slot = 0
    while t_all < budget_s:
        n = threads * chunk
        t_all += oracle_env_slots(seed, slot, n, plies, threads, chunk)
        slot += n
    return slot * plies / t_all, "%d slots x %d plies (masks written), slots 0..%d, %d host threads" % (
        slot, plies, slot - 1, threads), t_all


def timed_items(fn, n_items, threads, budget_s):
    """Call fn(i) for i = 0, 1, ... on `threads` host threads until about
    budget_s seconds have passed or all n_items are done; returns the items
    done and the wall time in seconds."""
    nxt = [0]
    lock = threading.Lock()
    t0 = time.perf_counter()

    def worker():
        while True:
            with lock:
                i = nxt[0]
                if i >= n_items or time.perf_counter() - t0 >= budget_s:
                    return
                nxt[0] = i + 1
            fn(i)

    pool = [threading.Thread(target=worker) for _ in range(threads)]
    for t in pool:
        t.start()
    for t in pool:
        t.join()
    return nxt[0], time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.lib()
    plies = args.plies
    chunk = 8
    threads = host_threads()
    for _ in range(args.warmup):
        oracle_env_slots(args.seed, 0, threads * 4, 100, threads, 4)
    times = []
    per_step = threads * chunk
    for k in range(args.steps):
        times.append(oracle_env_slots(args.seed, k * per_step, per_step, plies, threads, chunk))
    total = sum(times)
    value = args.steps * per_step * plies / total
    sample = "%d steps x (%d slots x %d plies) of the %d-slot workload, masks written, %d host threads" % (
        args.steps, per_step, plies, args.games, threads)
    line = {"impl": "reference", "metric": "env steps/s at 65,536 games", "value": value, "unit": "env-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(args.games, plies, args.ring),
            "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    import paper_2511_07312_gb300 as st

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    if args.profile in ("rollout", "obs"):
        if rank == 0:
            (profile_rollouts if args.profile == "rollout" else profile_obs)(st, torch, dev, args)
        if world > 1:
            dist.destroy_process_group()
        return
    N, S, R = args.games, args.plies, args.ring
    env = st.Env(N, seed=args.seed + rank, device=local)
    tuned = None
    if args.wpb and args.gpw:
        wpb, gpw, gpf, bps = args.wpb, args.gpw, args.gpf or 1, args.bps
    else:
        from paper_2511_07312_gb300 import autotune
        tuned = autotune.tune(N, device=local, final_plies=S)
        wpb, gpw, gpf = tuned["warps_per_block"], tuned["games_per_warp"], tuned["games_per_fetch"]
        bps = tuned.get("blocks_per_sm", 0)
    env.set_launch(wpb, bps, gpf, games_per_warp=gpw)
    bps = env.launch_shape()["blocks_per_sm"]   # resident blocks per SM after the occupancy clamp
    ring = env.run(1, R)   # allocates the ring; later calls reuse it
    env.sync()

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up (also captures the CUDA graph)
    for _ in range(args.warmup):
        env.run(S, R, out=ring)
    env.sync()

    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(env.stream)
        for _ in range(args.steps):
            env.run(S, R, out=ring)
        end.record(env.stream)
        end.synchronize()
    torch.cuda.synchronize()
    barrier()
    value, ms = job_rate(float(N) * S * args.steps, start.elapsed_time(end), world, dist, dev)
    env.sync()
    per_launch_s = ms / 1000.0 / args.steps
    bytes_per_launch = float(N) * S * BYTES_PER_ENV_STEP
    peak, peak_kind = peaks()
    achieved = bytes_per_launch / per_launch_s / 1e9
    clocks = clk.summary()

    if args.profile:
        if rank == 0:
            print(json.dumps({"profile": True, "games": N, "plies": S, "ms_per_launch": ms / args.steps,
                              "env_steps_per_s": value, "achieved_GBps": achieved}), flush=True)
        env.close()
        if world > 1:
            dist.destroy_process_group()
        return

    extras = {}
    # plain per-ply launch path on the same workload shape (fewer plies)
    plain_plies = 50
    out = env.step()
    env.sync()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(env.stream)
    for _ in range(plain_plies):
        env.step(out=out)
    s1.record(env.stream)
    s1.synchronize()
    plain_ms = s0.elapsed_time(s1)
    extras["plain_path"] = {"value": N * plain_plies / (plain_ms / 1000.0), "unit": "env-steps/s",
                            "plies": plain_plies, "note": "one st_env_step launch per ply, same outputs"}

    # end to end through the public API with host buffers: H2D of the
    # per-slot restart requests, the run, D2H of the per-slot counters
    which_h = torch.zeros(N, dtype=torch.uint8).pin_memory()
    stats_h = torch.empty((N, 8), dtype=torch.int32).pin_memory()
    which_d = torch.empty(N, dtype=torch.uint8, device=dev)
    e2e_steps = max(2, args.steps // 2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(env.stream):
        e0.record(env.stream)
        for _ in range(e2e_steps):
            which_d.copy_(which_h, non_blocking=True)
            env.reset(which=which_d)
            env.run(S, R, out=ring)
            stats_h.copy_(env.stats(), non_blocking=True)
        e1.record(env.stream)
    e1.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e = {"value": float(N) * S * e2e_steps * world / (e2e_ms / 1000.0), "unit": "env-steps/s",
           "h2d_bytes_per_step": N, "d2h_bytes_per_step": N * 8 * 4}

    if not args.no_extras and rank == 0:
        try:
            extras.update(secondary(st, torch, dev, args))
        except Exception as exc:  # secondary workloads never hide the headline
            extras["secondary_error"] = repr(exc)

    cpu = None
    if rank == 0:
        # all host threads (the figure of record), then one thread beside it
        threads = host_threads()
        rate, sample, secs = oracle_env_rate(args.seed, S, budget_s=10.0, chunk=4, threads=threads)
        rate1, sample1, secs1 = oracle_env_rate(args.seed, S, budget_s=5.0, chunk=4, threads=1)
        cpu = {"value": rate, "unit": "env-steps/s", "cores": threads, "kind": "oracle", "sample": sample,
               "seconds": round(secs, 1),
               "single_thread": {"value": rate1, "sample": sample1, "seconds": round(secs1, 1)}}

    if rank == 0:
        line = {"metric": "env steps/s at 65,536 games", "value": value, "unit": "env-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic",
                "config": dict(workload_config(N, S, R),
                               launch={"warps_per_block": wpb, "games_per_warp": gpw, "games_per_fetch": gpf,
                                       "blocks_per_sm": bps,
                                       "chosen_by": "autotuner" if tuned else "command line"}),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak,
                             "traffic": (None if measured_traffic_per_env_step() is None
                                         else measured_traffic_per_env_step() * float(N) * S),
                             "traffic_note": "ncu dram__bytes_read.sum+dram__bytes_write.sum per launch, scaled "
                                             "from a 16,384 x 400 capture (profiles/k_env_run_traffic.md)",
                             "peak_kind": peak_kind + " hbm_gbs (copy, burst)",
                             "algorithmic_bytes_per_env_step": BYTES_PER_ENV_STEP, "kernel": "k_env_run"},
                # the same launch against the issue-slot ceiling, side by side
                # (instructions per env-step from the committed ncu capture)
                "issue": issue_view(value / max(1, world), peak),
                "clocks": clocks, "e2e": e2e, "gpu_launches": args.steps,
                "cpu_baseline": cpu, "extras": extras}
        print(json.dumps(line), flush=True)
    env.close()
    if world > 1:
        dist.destroy_process_group()


def game_positions(st, torch, dev, B=16384):
    """64 random-policy games (seed 1) played on the GPU to their end or the
    1,000-ply cap, and B (game, ply) items at plies uniform in [0, min(600,
    length - 1)], sorted by (game, ply)."""
    import numpy as np
    G = 64
    env = st.Env(G, seed=1, autoreset=False, device=dev.index)
    setups = env.export(torch.arange(G))[:, :80].contiguous()
    traj = env.run(1000, 1000, want=("action",))
    env.sync()
    acts = traj["action"].t().contiguous()
    lengths = (acts >= 0).sum(1).cpu().numpy()
    env.close()
    rng = np.random.default_rng(3)
    games = rng.integers(0, G, B).astype(np.int32)
    plies = np.array([rng.integers(0, min(600, max(1, lengths[g]) - 1) + 1) for g in games], np.int16)
    order = np.lexsort((plies, games))
    games, plies = games[order], plies[order]
    return setups, acts, torch.from_numpy(games).to(dev), torch.from_numpy(plies).to(dev)


def rollout_positions(st, torch, dev, setups, acts, gi, pl, P=4096):
    """P of the items, evenly spaced, as snapshots."""
    import numpy as np
    sel = torch.from_numpy(np.linspace(0, gi.numel() - 1, P).astype(np.int64)).to(dev)
    pos, _ = st.replay_positions(setups, acts, gi[sel].contiguous(), pl[sel].contiguous())
    return pos


def profile_rollouts(st, torch, dev, args):
    """The belief-sample rollout workload alone (4,096 positions x 256
    samples x depth 32), for profiler captures."""
    pos = rollout_positions(st, torch, dev, *game_positions(st, torch, dev))
    K, D = 256, 32
    tallies, _ = st.rollout(pos, K, D, seed=7)
    for _ in range(args.warmup):
        st.rollout(pos, K, D, seed=7, out=tallies)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    for _ in range(args.steps):
        st.rollout(pos, K, D, seed=7, out=tallies)
    t1.record()
    t1.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    print(json.dumps({"profile": "rollout", "positions": pos.shape[0], "K": K, "depth": D, "ms_per_call": ms,
                      "samples_per_s": pos.shape[0] * K / (ms / 1000)}), flush=True)


def profile_obs(st, torch, dev, args):
    """The observation workload alone (planes, bf16 copy and masks of 16,384
    replayed positions), for profiler captures."""
    setups, acts, gi, pl = game_positions(st, torch, dev)
    o = st.obs_encode(setups, acts, gi, pl)
    for _ in range(args.warmup):
        st.obs_encode(setups, acts, gi, pl, out=o)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    for _ in range(args.steps):
        st.obs_encode(setups, acts, gi, pl, out=o)
    t1.record()
    t1.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    B = gi.numel()
    print(json.dumps({"profile": "obs", "positions": B, "ms_per_call": ms, "positions_per_s": B / (ms / 1000),
                      "status_ok": int((o["status"] == 0).sum().item())}), flush=True)


def secondary(st, torch, dev, args):
    """Observation planes of 16,384 replayed positions, belief-sample
    rollouts of 4,096 positions, the per-move search of 256 positions, and
    the serving workload."""
    import numpy as np
    out = {}
    setups, acts, gi, pl = game_positions(st, torch, dev)
    B = gi.numel()
    o = st.obs_encode(setups, acts, gi, pl)
    torch.cuda.synchronize()
    reps = 5
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        st.obs_encode(setups, acts, gi, pl, out=o)
    t1.record()
    t1.synchronize()
    ms = t0.elapsed_time(t1) / reps
    byts = B * (487 * 100 * 3 + MASK_BYTES)
    peak, peak_kind = peaks()
    gbs = byts / (ms / 1000) / 1e9
    out["obs_encode"] = {"positions_per_s": B / (ms / 1000), "ms": ms, "GB_per_s_written": gbs,
                         "positions": B, "bytes_written_per_position": 487 * 100 * 3 + MASK_BYTES,
                         "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                      "frac": gbs / peak, "peak_kind": peak_kind + " hbm_gbs (copy, burst)",
                                      "algorithmic_bytes_per_position": 487 * 100 * 3 + MASK_BYTES,
                                      "kernels": "k_replay + k_obs_emit, one call"}}
    # the oracle beside it: the same items, one per call, on all host threads
    # for about 5 seconds (each item replayed from its game's start)
    import oracle
    oracle.lib()
    threads = host_threads()
    setups_h, acts_h = setups.cpu().numpy(), acts.cpu().numpy()
    gi_h, pl_h = gi.cpu().numpy(), pl.cpu().numpy()
    done_o, dt = timed_items(lambda i: oracle.obs_encode(setups_h, acts_h, gi_h[i:i + 1], pl_h[i:i + 1]), B, threads,
                             5.0)
    out["obs_encode"]["cpu_baseline"] = {"value": done_o / dt, "unit": "positions/s", "cores": threads,
                                         "kind": "oracle", "sample": "items 0..%d of the %d (uint8 and bf16 planes, "
                                         "masks), one item per call" % (done_o - 1, B)}
    # belief-sample rollouts: 4,096 positions x 256 samples x depth 32
    P, K, D = 4096, 256, 32
    pos = rollout_positions(st, torch, dev, setups, acts, gi, pl, P)
    tallies, _ = st.rollout(pos, K, D, seed=7)
    torch.cuda.synchronize()
    t0.record()
    reps = 3
    for _ in range(reps):
        st.rollout(pos, K, D, seed=7, out=tallies)
    t1.record()
    t1.synchronize()
    ms = t0.elapsed_time(t1) / reps
    tl = tallies.sum(0).cpu().numpy().tolist()
    out["belief_rollout"] = {"samples_per_s": P * K / (ms / 1000), "ms": ms, "positions": P, "K": K, "depth": D,
                             "ply_steps_per_s_upper": P * K * D / (ms / 1000),
                             "tallies_win_loss_draw_unfinished": tl}
    # the oracle beside it: one position (all K samples) per call, on all host
    # threads for about 5 seconds
    pos_h = pos.cpu().numpy()
    done_r, dt = timed_items(lambda i: oracle.rollout(pos_h[i:i + 1], K, D, 7, stream_ids=np.array([i], np.uint32)),
                             P, threads, 5.0)
    out["belief_rollout"]["cpu_baseline"] = {"value": done_r * K / dt, "unit": "samples/s", "cores": threads,
                                             "kind": "oracle", "sample": "positions 0..%d of the %d, K=%d, depth %d"
                                             % (done_r - 1, P, K, D)}
    # the same rollouts with the magnet policy as the rollout policy
    mflags = st.RULES_ALL | st.ROLLOUT_MAGNET
    st.rollout(pos, K, D, seed=7, out=tallies, flags=mflags)
    torch.cuda.synchronize()
    t0.record()
    for _ in range(reps):
        st.rollout(pos, K, D, seed=7, out=tallies, flags=mflags)
    t1.record()
    t1.synchronize()
    ms = t0.elapsed_time(t1) / reps
    out["belief_rollout_magnet"] = {"samples_per_s": P * K / (ms / 1000), "ms": ms, "positions": P, "K": K,
                                    "depth": D, "tallies_win_loss_draw_unfinished": tallies.sum(0).cpu().tolist()}
    # per-move search (App. E steps 1-4): 256 positions x every legal move x
    # 16 configurations x depth 40, then the tabular update and the sampled move
    Ps, Ss, Ds = 256, 16, 40
    spos = pos[::P // Ps][:Ps].contiguous()
    res = st.search(spos, Ss, Ds, seed=11)
    torch.cuda.synchronize()
    reps = 5
    t0.record()
    for _ in range(reps):
        st.search(spos, Ss, Ds, seed=11)
    t1.record()
    t1.synchronize()
    ms = t0.elapsed_time(t1) / reps
    n_roll = int(res["n_moves"].sum().item()) * Ss
    out["search"] = {"positions_per_s": Ps / (ms / 1000), "rollouts_per_s": n_roll / (ms / 1000), "ms": ms,
                     "positions": Ps, "S": Ss, "depth": Ds, "rollouts": n_roll,
                     "mean_legal_moves": n_roll / Ss / Ps}
    # the oracle beside it: the same positions, one per call, on all host
    # threads for about 5 seconds
    spos_h = spos.cpu().numpy()
    done_p, dt = timed_items(lambda i: oracle.search(spos_h[i:i + 1], Ss, Ds, 11,
                                                     stream_ids=np.array([i], np.uint32)), Ps, threads, 5.0)
    out["search"]["cpu_baseline"] = {"value": done_p / dt, "unit": "positions/s", "cores": threads,
                                     "kind": "oracle", "sample": "the first %d of the %d positions" % (done_p, Ps)}
    # historical queries: 16,384 slots recording 1,000 steps; positions at
    # step now - 300 rebuilt by replay
    Nh, Hh = 16384, 1000
    henv = st.Env(Nh, seed=5, device=dev.index)
    henv.set_launch(4, 0, 1, games_per_warp=4)
    henv.enable_history(Hh)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(henv.stream)
    henv.run(Hh)
    ev1.record(henv.stream)
    henv.sync()
    rec_ms = ev0.elapsed_time(ev1)
    th = henv.current_step() - 300
    hp = henv.history_positions(th)
    torch.cuda.synchronize()
    t0.record()
    reps = 3
    for _ in range(reps):
        hp = henv.history_positions(th)
    t1.record()
    t1.synchronize()
    ms = t0.elapsed_time(t1) / reps
    rebuilt = int((hp["status"] == 0).sum().item())
    out["history_positions"] = {"slots": Nh, "H": Hh, "step": th, "rebuilt": rebuilt, "ms": ms,
                                "positions_per_s": rebuilt / (ms / 1000)}
    # the oracle beside it: a slot's position at step th is its environment
    # run for th steps; one slot per call on all host threads, ~3 seconds
    done_g, dt = timed_items(lambda i: oracle.env_run(5, 1, th, slot0=i, want_mask=False, want_final=True),
                             Nh, threads, 3.0)
    out["history_positions"]["cpu_baseline"] = {"value": done_g / dt, "unit": "positions/s", "cores": threads,
                                                "kind": "oracle", "sample": "slots 0..%d" % (done_g - 1)}
    # the same env stepping with and without recording (one launch each, first one includes graph capture)
    henv.enable_history(0)
    henv.run(Hh)
    henv.sync()
    ev0.record(henv.stream)
    henv.run(Hh)
    ev1.record(henv.stream)
    henv.sync()
    plain_ms = ev0.elapsed_time(ev1)
    henv.enable_history(Hh)
    henv.run(Hh)
    henv.sync()
    ev0.record(henv.stream)
    henv.run(Hh)
    ev1.record(henv.stream)
    henv.sync()
    rec_ms = ev0.elapsed_time(ev1)
    out["history_recording"] = {"slots": Nh, "steps": Hh, "env_steps_per_s_recording": Nh * Hh / (rec_ms / 1000),
                                "env_steps_per_s_not_recording": Nh * Hh / (plain_ms / 1000)}
    henv.close()
    out["serving"] = serving(st, torch, dev, pos.cpu().numpy(), args)
    # the same request mix at ten times the arrival rate, where requests
    # arrive while others run and batches of several requests form
    out["serving"]["high_rate"] = serving(st, torch, dev, pos.cpu().numpy(), args, duration_s=2.0, rate=20000.0,
                                          compare=False)
    return out


def serving(st, torch, dev, positions, args, duration_s=10.0, rate=2000.0, compare=True):
    """Serving: Poisson arrivals (mean 2,000/s) of search requests, K ~
    U{16..1024}, depth ~ U{8..64}, from positions of the 64 replayed games; the
    continuous-batching server against one launch + sync per request, and a
    burst of heavy requests for capacity (compare=False: the server alone)."""
    import numpy as np
    rng = np.random.default_rng(5)
    n = int(duration_s * rate)
    gaps = rng.exponential(1.0 / rate, n)
    arrive = np.cumsum(gaps)
    Ks = rng.integers(16, 1025, n)
    Ds = rng.integers(8, 65, n)
    which = rng.integers(0, len(positions), n)
    seed = 11

    def pct(lat):
        return {"p50_ms": float(np.percentile(lat, 50)) * 1e3, "p99_ms": float(np.percentile(lat, 99)) * 1e3,
                "mean_ms": float(np.mean(lat)) * 1e3}

    # served
    srv = st.Server(device=dev.index, max_requests=512, sample_slots=1 << 18, max_batches=8)
    tickets = [0] * n
    t0 = time.perf_counter() + 0.05

    def submitter():
        for i in range(n):
            while time.perf_counter() < t0 + arrive[i]:
                pass
            tickets[i] = srv.submit(positions[which[i]], int(Ks[i]), int(Ds[i]), seed, i)

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat = np.zeros(n)
    first, last = None, 0
    for i in range(n):
        _, (sub, adm, done) = srv.wait(tickets[i], 120000)
        lat[i] = (done - sub) / 1e9
        first = sub if first is None else min(first, sub)
        last = max(last, done)
    span = (last - first) / 1e9
    stats = srv.stats()
    srv.close()
    served = dict(pct(lat), requests_per_s=n / span, samples_per_s=float(Ks.sum()) / span,
                  batches=stats["batches"], max_batch_requests=stats["max_batch_requests"],
                  mean_batch_requests=n / max(1, stats["batches"]))
    if not compare:
        return {"requests": n, "arrival_rate_per_s": rate, "K_range": [16, 1024], "depth_range": [8, 64],
                "served": served}
    # plain: one launch + sync per request, in arrival order
    pos_h = torch.from_numpy(positions).pin_memory()
    pos_d = torch.empty((1, positions.shape[1]), dtype=torch.uint8, device=dev)
    tall = torch.empty((1, 4), dtype=torch.int32, device=dev)
    tall_h = torch.empty((1, 4), dtype=torch.int32).pin_memory()
    sid = torch.zeros(1, dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(device=dev)
    lat2 = np.zeros(n)
    t0 = time.perf_counter() + 0.05
    with torch.cuda.stream(s):
        for i in range(n):
            while time.perf_counter() < t0 + arrive[i]:
                pass
            pos_d.copy_(pos_h[which[i]:which[i] + 1], non_blocking=True)
            sid.fill_(i)
            st.rollout(pos_d, int(Ks[i]), int(Ds[i]), seed, stream_ids=sid, out=tall, stream=s)
            tall_h.copy_(tall, non_blocking=True)
            s.synchronize()
            lat2[i] = time.perf_counter() - (t0 + arrive[i])
    span2 = time.perf_counter() - t0
    plain = dict(pct(lat2), requests_per_s=n / span2, samples_per_s=float(Ks.sum()) / span2)
    # capacity: a burst of 2,000 heavy requests (K ~ U{1024..4096}, depth
    # 64) submitted at once, timed from the first submit to the last completion
    nb = 2000
    Kb = rng.integers(1024, 4097, nb)
    srv = st.Server(device=dev.index, max_requests=512, sample_slots=1 << 18, max_batches=8)
    tb = [srv.submit(positions[which[i]], int(Kb[i]), 64, seed, i) for i in range(nb)]
    first, last = None, 0
    for t in tb:
        _, (sub, adm, done) = srv.wait(t, 120000)
        first = sub if first is None else min(first, sub)
        last = max(last, done)
    srv.close()
    spanb = (last - first) / 1e9
    burst = {"requests": nb, "K_range": [1024, 4096], "depth": 64, "requests_per_s": nb / spanb,
             "samples_per_s": float(Kb.sum()) / spanb, "ms": spanb * 1e3}
    return {"requests": n, "arrival_rate_per_s": rate, "K_range": [16, 1024], "depth_range": [8, 64],
            "served": served, "plain_per_request": plain, "burst_capacity": burst}


if __name__ == "__main__":
    main()
