"""Benchmark: pair-interactions/s of the element-model leap-frog step.

One step = the whole hot path of one kick-drift-kick step of a binary system:
opening kick + drift (FP64) with the FP32 copy and contact-grid binning, the
O(N^2) FP32 pair term, the FP64 contact term, the closing kick.  Default
workload: the 1,048,576-element binary (786,432 donor + 262,144 accretor
elements, q = 0.2, uniform spheres of 0.95 r_L and 0.4 r_L), synthetic
initial conditions from the library's seeded recipe.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload binary_1m|binary_64k|binary_1k|binary_256k]

Under torchrun each rank runs its own copy of the workload (weak scaling, no
data-path collective); rank 0 prints one JSON line.  ``--impl reference``
times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# name: (n_donor, n_accretor, q, f_donor, f_accretor, eps, dt, expand_rate, expand_steps)
WORKLOADS = {
    "binary_1k": (512, 512, 0.5, 0.8, 0.5, 0.01, 1e-3, 0.0, -1),
    "binary_64k": (49152, 16384, 0.3, 0.9, 0.5, 0.005, 5e-4, 0.25 / 10000, 10000),
    "binary_1m": (786432, 262144, 0.2, 0.95, 0.4, 0.005, 2.5e-4, 0.0, -1),
    # the 1M binary at a quarter of the elements: profiling captures that
    # must stay a few GB on the device (not a bench line)
    "binary_256k": (196608, 65536, 0.2, 0.95, 0.4, 0.005, 2.5e-4, 0.0, -1),
}
METRIC = "pair-interactions/s"
L2_BYTES = 129e6
# ALU roofline of one pair (Eq. 4) on an SM: 128 FP32 lanes and 16 MUFU
# (special-function) results per clock (the latter measured).  A pair costs 12
# FP32 operations (dx, dy, dz, 3 for d2, r + eps, 2 for the denominator, 3
# accumulations) and 2 MUFU (square root, reciprocal); sharing one reciprocal
# between two pairs trades 0.5 MUFU for 1.5 FP32 per pair.  The bound is the
# best split between the two pipes.
# With each unordered pair evaluated once (Newton's third law), one
# evaluation (15 FP32: 3 more accumulations for the second element; 2 MUFU)
# serves two pair interactions.
FP32_PER_SM_CLK = 128
MUFU_PER_SM_CLK = 16
FP32_PER_PAIR = 12.0
FP32_PER_PAIR_SYM = 15.0
MUFU_PER_PAIR = 2.0
SHARED_RCP_FP32, SHARED_RCP_MUFU = 1.5, 0.5
PAIR_CFG_KEYS = ("tile", "i_per_thread", "threads", "min_blocks", "nr_slots", "i_packed",
                 "shared_rcp", "symmetric")


def pairs_per_sm_clk(symmetric: bool = False, rates=None):
    """Pair interactions per clock per SM at the best split x of shared
    reciprocals: max over x in [0, 1] of 1 / max(FP32 time, MUFU time) per
    evaluation, times the interactions one evaluation serves.  rates: issue
    rates per clock per SM (measured: unit_rates_per_clk), else the nominal
    128 FP32 lanes and 16 MUFU results."""
    fp32_rate = rates["fp32_lanes_per_clk_sm"] if rates else FP32_PER_SM_CLK
    sqrt_rate = rates["mufu_sqrt_per_clk_sm"] if rates else MUFU_PER_SM_CLK
    rcp_rate = rates["mufu_rcp_per_clk_sm"] if rates else MUFU_PER_SM_CLK
    fp32 = FP32_PER_PAIR_SYM if symmetric else FP32_PER_PAIR
    best, x_best = 0.0, 0.0
    for k in range(1001):
        x = k / 1000.0
        t_fp32 = (fp32 + SHARED_RCP_FP32 * x) / fp32_rate
        t_mufu = 1.0 / sqrt_rate + (1.0 - SHARED_RCP_MUFU * x) / rcp_rate
        per_eval = 1.0 / max(t_fp32, t_mufu)
        if per_eval > best:
            best, x_best = per_eval, x
    return (2.0 if symmetric else 1.0) * best, x_best


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# the pair kernels, and the host functions that cut their work into items
PAIR_SOURCES = ("nb_pair_common.cuh", "nb_pair.cu", "nb_pair_sym.cu")
PAIR_PLAN_FUNCTIONS = ("nb_status Batch::plan_pairs_()", "int64_t onesided_chunks(")


def _function_text(src, head):
    """The text of the function whose definition starts with `head` (up to
    the closing brace at the start of a line)."""
    i = src.index(head)
    return src[i:src.index("\n}\n", i) + 3]


def pair_sources_sha():
    """Hash of the pair kernels' sources and of the plan functions (comments
    and whitespace removed): the traffic record is void once they change."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2303_12166_gb300", "csrc")
    texts = []
    for f in PAIR_SOURCES:
        with open(os.path.join(csrc, f)) as fh:
            texts.append(fh.read())
    with open(os.path.join(csrc, "nb_batch.cpp")) as fh:
        plan = fh.read()
    texts += [_function_text(plan, head) for head in PAIR_PLAN_FUNCTIONS]
    for src in texts:
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def _pair_traffic(workload, cfg):
    """DRAM bytes per launch of the pair kernel from the committed ncu capture,
    if it was taken on this workload and launch shape with the current kernel
    sources; otherwise None."""
    p = os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    key = ",".join(str(cfg[k]) for k in PAIR_CFG_KEYS)
    if rec.get("workload") != workload or key not in rec.get("applies_to", [rec.get("pair_cfg")]) \
            or rec.get("sources_sha256_16") != pair_sources_sha():
        return None
    return float(rec["dram_bytes_per_launch"])


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        uu = {r[0] for r in rows}
        if self.uuid and any(self.uuid in u for u in uu):
            rows = [r for r in rows if self.uuid in r[0]]
        elif len(uu) > 1:
            rows = rows  # all GPUs of the host
        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[1]) for r in rows])
        smax = np.nanmax([num(r[2]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = []
        for k, name in enumerate(names):
            if any(r[5 + k].lower().startswith("active") for r in rows):
                reasons.append(name)
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(smax),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": float(np.nanmax([num(r[3]) for r in rows]))}


def _workload(name):
    nd, na, q, fd, fa, eps, dt, rate, cap = WORKLOADS[name]
    return dict(n_donor=nd, n_accretor=na, q=q, f_donor=fd, f_accretor=fa, eps=eps, dt=dt,
                expand_rate=rate, expand_steps=cap, sigma_v=1e-3, seed=0)


def _config(name, w, extra=None):
    n = w["n_donor"] + w["n_accretor"]
    cfg = {"workload": name, "n": n, "n_donor": w["n_donor"], "n_accretor": w["n_accretor"],
           "q": w["q"], "f_donor": w["f_donor"], "f_accretor": w["f_accretor"], "eps": w["eps"],
           "dt": w["dt"], "beta": 0.5, "pairs_per_step": n * n}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ error against the oracle
def _rms_rel(a, ref):
    """sqrt(sum |a - ref|^2 / sum |ref|^2) over elements (the per-step force
    metric of the parity tests)."""
    num = float(np.sum((np.asarray(a) - np.asarray(ref)) ** 2))
    den = float(np.sum(np.asarray(ref) ** 2))
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))


def _oracle_ic(desc, params=None):
    """(m, R0, gamma) of a description from the oracle's own recipe."""
    from oracle import oracle
    _, _, m, R, g = oracle.make_ic(desc["n_donor"], desc["n_accretor"], desc["q"],
                                   f_donor=desc["f_donor"], f_accretor=desc["f_accretor"],
                                   sigma_v=desc.get("sigma_v", 1e-3), seed=desc.get("seed", 0),
                                   stream=desc.get("stream", 0))
    return m, R, g


def _sample_rows(n, n_donor, nrows, seed):
    """Sampled rows plus the ends of the donor and accretor ranges."""
    import synth
    edge = [0, n_donor - 1, n_donor, n - 1]
    rnd = (synth.u01(seed, 77, nrows) * n).astype(np.int64)
    return np.unique(np.clip(np.concatenate([edge, rnd]), 0, n - 1))


def force_error(desc, eps, beta, x, v, a_gpu, rows, k, ic=None):
    """Error of the library's accelerations a_gpu (n x 3) on `rows` against
    the FP64 oracle's direct sum (Eqs. 4-6) at the same state (x, v) with the
    element radii of step k (donor growth law)."""
    from oracle import oracle
    m, R0, g = ic if ic is not None else _oracle_ic(desc)
    R = np.array(R0, dtype=np.float64)
    nd = desc["n_donor"]
    rate = desc.get("expand_rate", 0.0)
    if rate:
        R[:nd] *= oracle.donor_scale(k, desc["f_donor"], rate, desc.get("expand_steps", -1))
    ref = oracle.forces_rows(rows, x, v, m, R, g, G=1.0, eps=eps, beta=beta)
    got = np.asarray(a_gpu)[rows]
    return {"force_rms_rel": _rms_rel(got, ref),
            "force_max_abs_rel": float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)),
            "rows": int(len(rows)), "step": int(k), "vs": "oracle (FP64 direct sum)"}


# ------------------------------------------------------------------ CPU oracle timing
def _oracle_sample(w, target_s=10.0, seed_rows=11):
    """Time the FP64 oracle's direct sum on a bounded sample of rows of the
    workload (all j for each sampled i).  Returns pairs/s, cores, sample text."""
    from oracle import oracle
    import synth
    x, v, m, R, g = oracle.make_ic(w["n_donor"], w["n_accretor"], w["q"], f_donor=w["f_donor"],
                                   f_accretor=w["f_accretor"], sigma_v=w["sigma_v"],
                                   seed=w["seed"])
    n = len(m)
    # calibrate on a small sample, then size the timed sample to ~target_s
    rows = (synth.u01(seed_rows, 1, 64) * n).astype(np.int64)
    t0 = time.perf_counter()
    oracle.forces_rows(rows, x, v, m, R, g, G=1.0, eps=w["eps"], beta=0.5)
    dt = max(time.perf_counter() - t0, 1e-6)
    nrows = int(min(n, max(64, 64 * target_s / dt)))
    rows = (synth.u01(seed_rows, 2, nrows) * n).astype(np.int64)
    t0 = time.perf_counter()
    ref = oracle.forces_rows(rows, x, v, m, R, g, G=1.0, eps=w["eps"], beta=0.5)
    el = time.perf_counter() - t0
    pairs = float(nrows) * n
    return pairs / el, oracle.num_threads(), (
        f"FP64 oracle direct sum (Eqs. 4-6) for {nrows} sampled elements against all {n} "
        f"elements ({pairs:.3e} pairs, {el:.1f} s)"), (x, v, m, R, g), el, rows, ref


def _oracle_configs():
    """The FP64 oracle as it stands on the host cores for the other
    workloads: the 1,024-element binary run in full (100 steps), one step of
    the 65,536-element growing donor, and 8 systems of the 256-system sweep
    for 2 steps each, the last extrapolated to the whole sweep per pair."""
    from oracle import oracle
    import synth
    out = {}

    def timed_run(nd, na, q, fd, fa, eps, dt, steps, rate=0.0, cap=-1, seed=0, stream=0):
        x, v, m, R, g = oracle.make_ic(nd, na, q, f_donor=fd, f_accretor=fa, sigma_v=1e-3,
                                       seed=seed, stream=stream)
        t0 = time.perf_counter()
        oracle.run(x, v, m, R, g, G=1.0, eps=eps, beta=0.5, dt=dt, nsteps=steps, n_donor=nd,
                   grow_f0=fd, grow_rate=rate, grow_cap=cap)
        el = time.perf_counter() - t0
        n = nd + na
        return el, float(n) * n * (steps + 1)  # a^0 and one pass per step

    el, pairs = timed_run(512, 512, 0.5, 0.8, 0.5, 0.01, 1e-3, 100)
    out["binary_1k"] = {"steps": 100, "seconds": el, "pairs_per_s": pairs / el,
                        "steps_per_s": 100 / el, "sample": "the whole run, 101 force passes"}
    w = WORKLOADS["binary_64k"]
    el, pairs = timed_run(w[0], w[1], w[2], w[3], w[4], w[5], w[6], 1, w[7], w[8])
    out["binary_64k"] = {"steps": 1, "seconds": el, "pairs_per_s": pairs / el,
                         "sample": "one step of the 10,000 (2 force passes)"}
    systems = synth.sweep_systems(256, seed=0)
    pick = systems[::32]
    el = pairs = 0.0
    for d in pick:
        e, p_ = timed_run(d["n_donor"], d["n_accretor"], d["q"], d["f_donor"], d["f_accretor"],
                          SWEEP_PARAMS["eps"], SWEEP_PARAMS["dt"], 2, d["expand_rate"],
                          d["expand_steps"], d["seed"], d["stream"])
        el += e
        pairs += p_
    mean_pairs = float(np.mean([(d["n_donor"] + d["n_accretor"]) ** 2 for d in systems]))
    out["sweep_256"] = {"systems_timed": len(pick), "steps_each": 2, "seconds": el,
                        "pairs_per_s": pairs / el,
                        "system_steps_per_s": pairs / el / mean_pairs,
                        "sample": "every 32nd system of the sweep, 2 steps each (3 force "
                                  "passes); system-steps/s extrapolated per pair to the "
                                  "whole sweep"}
    out["cores"] = oracle.num_threads()
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    w = _workload(args.workload)
    n = w["n_donor"] + w["n_accretor"]
    from oracle import oracle
    import synth
    x, v, m, R, g = oracle.make_ic(w["n_donor"], w["n_accretor"], w["q"], f_donor=w["f_donor"],
                                   f_accretor=w["f_accretor"], sigma_v=w["sigma_v"],
                                   seed=w["seed"])
    # rows per step: about 10 s of CPU work per step on the host cores, capped
    rows = (synth.u01(3, 1, 32) * n).astype(np.int64)
    t0 = time.perf_counter()
    oracle.forces_rows(rows, x, v, m, R, g, G=1.0, eps=w["eps"], beta=0.5)
    per_row = max((time.perf_counter() - t0) / 32, 1e-9)
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    nrows = int(min(n, max(32, budget / per_row)))
    times = []
    for s in range(args.warmup + args.steps):
        rows = (synth.u01(3, 10 + s, nrows) * n).astype(np.int64)
        t0 = time.perf_counter()
        oracle.forces_rows(rows, x, v, m, R, g, G=1.0, eps=w["eps"], beta=0.5)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    el = float(np.sum(times))
    pairs = float(nrows) * n * args.steps
    value = pairs / el
    sample = (f"each step: FP64 oracle direct sum (Eqs. 4-6) for {nrows} sampled elements "
              f"against all {n}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args.workload, w, {"sample_rows_per_step": nrows}),
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ batched / served
SWEEP_PARAMS = dict(eps=0.005, dt=5e-4, beta=0.5)


def measure_batched(nbm, torch, dev, stream, args, ws, rank):
    """Parameter sweep of independent binaries (element counts log-uniform in
    [2,048, 65,536]) advanced in one batch: one persistent pair-kernel launch
    per step for all systems.  Systems are dealt to ranks (no exchange).
    Compared with the same systems advanced one at a time through the
    single-system API, with and without FP64 diagnostics every step, each
    system timed on its own (no rescaling)."""
    import synth
    from paper_2303_12166_gb300.dist import max_over_ranks, shard, sum_over_ranks
    systems = synth.sweep_systems(args.sweep_systems, seed=0)
    mine = shard(len(systems), ws, rank)
    descs = [nbm.nb_desc_default(**systems[s]) for s in mine]
    params = [nbm.nb_params_default(**SWEEP_PARAMS) for _ in mine]
    b = nbm.Batch(descs, params, stream=stream)
    tuned = b.autotune(3)
    lanes = b.contact_lanes()
    b.step(3)
    b.sync()
    b.profile(True)
    b.profile_read(reset=True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    b.step(args.batched_steps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    b.sync()
    prof = b.profile_read(reset=True)
    # error against the oracle of three systems (smallest, median, largest)
    # at their state after the timed steps
    acc = []
    if rank == 0:
        order = sorted(range(len(mine)), key=lambda i: descs[i].n_donor + descs[i].n_accretor)
        for i in sorted({order[0], order[len(order) // 2], order[-1]}):
            xv, _, meta = b.get_state(i, with_acc=False)
            a = b.forces(i)
            d = systems[mine[i]]
            n_i = d["n_donor"] + d["n_accretor"]
            e = force_error(d, SWEEP_PARAMS["eps"], SWEEP_PARAMS["beta"], xv[:, :3], xv[:, 3:],
                            a, _sample_rows(n_i, d["n_donor"], 256, 4 + i), int(meta.step))
            acc.append(dict(e, system=int(mine[i]), n=int(n_i)))
    b.close()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    pairs_mine = float(sum((d.n_donor + d.n_accretor) ** 2 for d in descs))
    pairs = sum_over_ranks(pairs_mine, dev)
    el = ms * 1e-3
    out = {"workload": f"sweep_{len(systems)}", "systems": len(systems),
           "n_range": [2048, 65536], "steps": args.batched_steps,
           "value": len(systems) * args.batched_steps / el, "unit": "system-steps/s",
           "pairs_per_s": pairs * args.batched_steps / el,
           "ms_per_step": ms / args.batched_steps,
           "pair_cfg": {k: tuned[k] for k in PAIR_CFG_KEYS}, "contact_lanes": lanes,
           "phase_ms": {"pair": prof["pair_ms"], "contact": prof["contact_ms"],
                        "update": prof["update_ms"]},
           "gpu_launches": int(prof["kernels"]),
           "accuracy": {"systems": acc,
                        "max_force_rms_rel": max((a["force_rms_rel"] for a in acc), default=None),
                        "tolerance": 1e-5}}
    if rank == 0 and ws == 1 and args.per_system_steps > 0:
        # the same systems one at a time through the single-system API, each
        # timed on its own: plain stepping (nb_step), and stepping with the
        # FP64 diagnostics (nb_step(1) + nb_diagnostics) every step
        k = args.per_system_steps
        t_plain = t_diag = 0.0
        for d in systems:
            with nbm.System(nbm.nb_desc_default(**d), nbm.nb_params_default(**SWEEP_PARAMS),
                            stream=stream) as sy:
                sy.step(1)
                sy.diagnostics()
                sy.sync()
                t0 = time.perf_counter()
                sy.step(k)
                sy.sync()
                t_plain += time.perf_counter() - t0
                t0 = time.perf_counter()
                for _ in range(k):
                    sy.step(1)
                    sy.diagnostics()
                t_diag += time.perf_counter() - t0
        out["per_system_path"] = {
            "systems": len(systems), "steps_each": k,
            "plain_system_steps_per_s": len(systems) * k / t_plain,
            "fp64_diag_system_steps_per_s": len(systems) * k / t_diag,
            "note": "every system of the sweep, one at a time through nb_step / "
                    "nb_diagnostics, host wall clock per system (no rescaling); the batched "
                    "form's results equal these runs bit for bit (tested), so both forms have "
                    "the same error against the oracle"}
        out["speedup_vs_per_system_fp64_diag"] = out["value"] / \
            out["per_system_path"]["fp64_diag_system_steps_per_s"]
        out["speedup_vs_per_system_plain"] = out["value"] / \
            out["per_system_path"]["plain_system_steps_per_s"]
    return out


def measure_fp64_path(nbm, torch, dev, stream, args):
    """The FP64-force path (FP64 pair kernel) against the FP32 path on the
    65,536-element binary: one force pass each, CUDA events."""
    w = _workload("binary_64k")
    out = {"workload": "binary_64k"}
    for prec in (32, 64):
        desc = nbm.nb_desc_default(n_donor=w["n_donor"], n_accretor=w["n_accretor"], q=w["q"],
                                   f_donor=w["f_donor"], f_accretor=w["f_accretor"],
                                   sigma_v=w["sigma_v"], seed=w["seed"])
        params = nbm.nb_params_default(eps=w["eps"], dt=w["dt"], beta=0.5, force_prec=prec)
        with nbm.System(desc, params, stream=stream) as sy:
            if prec == 32:
                sy.autotune(1)
            a0 = sy.forces()
            xv0 = sy.get_state(with_acc=False)[0]
            n = w["n_donor"] + w["n_accretor"]
            out[f"fp{prec}_accuracy"] = dict(
                force_error(w, w["eps"], 0.5, xv0[:, :3], xv0[:, 3:], a0,
                            _sample_rows(n, w["n_donor"], 512, 3), 0),
                tolerance=1e-5 if prec == 32 else 1e-12)
            sy.step(1)
            sy.sync()
            sy.profile(True)
            sy.profile_read(reset=True)
            sy.step(1)
            sy.sync()
            p = sy.profile_read(reset=True)
        n = w["n_donor"] + w["n_accretor"]
        out[f"fp{prec}_pair_pairs_per_s"] = float(n) * n / (p["pair_ms"] * 1e-3)
    out["fp32_over_fp64"] = out["fp32_pair_pairs_per_s"] / out["fp64_pair_pairs_per_s"]
    return out


def measure_config1_run(nbm, torch, dev, stream, args):
    """The 65,536-element binary run as configured: 10,000 steps with the
    donor growing from 0.9 to 1.15 r_L (L1 overflow), in chunks of 500
    steps, CUDA events around the whole run; the error against the oracle of
    the accelerations at the final state, and the mass-transfer diagnostics
    there."""
    w = _workload("binary_64k")
    n = w["n_donor"] + w["n_accretor"]
    desc = nbm.nb_desc_default(n_donor=w["n_donor"], n_accretor=w["n_accretor"], q=w["q"],
                               f_donor=w["f_donor"], f_accretor=w["f_accretor"],
                               expand_rate=w["expand_rate"], expand_steps=w["expand_steps"],
                               sigma_v=w["sigma_v"], seed=w["seed"])
    params = nbm.nb_params_default(eps=w["eps"], dt=w["dt"], beta=0.5)
    total, chunk = args.config1_steps, 500
    with nbm.System(desc, params, stream=stream) as sy:
        tuned = sy.autotune(1)
        lanes = sy.contact_lanes()
        d0 = sy.diagnostics()
        torch.cuda.synchronize(dev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        done = 0
        while done < total:
            k = min(chunk, total - done)
            sy.step(k)
            done += k
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        sy.sync()
        ms = ev0.elapsed_time(ev1)
        d1 = sy.diagnostics()
        xv, _, meta = sy.get_state(with_acc=False)
        a = sy.forces()
    acc = force_error(w, w["eps"], 0.5, xv[:, :3], xv[:, 3:], a,
                      _sample_rows(n, w["n_donor"], 1024, 5), int(meta.step))
    return {"workload": "binary_64k", "steps": total, "ms": ms, "ms_per_step": ms / total,
            "value": float(n) * n * total / (ms * 1e-3), "unit": "pairs/s",
            "pair_cfg": {k: tuned[k] for k in PAIR_CFG_KEYS}, "contact_lanes": lanes,
            "r_donor": [float(d0["r_donor"]), float(d1["r_donor"])],
            "donor_past_L1": [int(d0["n_past_L1"]), int(d1["n_past_L1"])],
            "donor_in_accretor_lobe": [int(d0["n_in_accretor_lobe"]),
                                       int(d1["n_in_accretor_lobe"])],
            "mass_in_accretor_lobe": float(d1["m_in_accretor_lobe"]),
            "unbound": int(d1["n_unbound"]),
            "e_tot": [float(d0["e_tot"]), float(d1["e_tot"])],
            "l_z": [float(d0["l"][2]), float(d1["l"][2])],
            "accuracy": dict(acc, tolerance=1e-5),
            "note": "timed in chunks of 500 steps (one CUDA graph each); the donor radius "
                    "reaches 1.15 r_L at step 10,000"}


def _serve(nbm, stream, trace, budget):
    """One served run of `trace` (arrivals replayed in real time) under an
    HBM budget of `budget` bytes; returns the results, the admission
    statistics, the server's shape and its pair configuration."""
    srv = nbm.nb_server_create(budget, 64, 262144, 32, stream)
    try:
        info = nbm.nb_server_info(srv)
        scfg = nbm.nb_server_pair_cfg(srv)
        t0 = time.perf_counter()
        tickets = []
        for r in trace:
            wait = r["t_arrival"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            tickets.append(nbm.nb_submit(srv, nbm.nb_desc_default(**r["desc"]),
                                         nbm.nb_params_default(**SWEEP_PARAMS), r["nsteps"]))
        nbm.nb_server_drain(srv, 3600.0)
        res = [nbm.nb_poll(srv, t) for t in tickets]
        adm = nbm.nb_server_stats_read(srv)
    finally:
        nbm.nb_server_destroy(srv)
    return res, adm, info, scfg


def _served_figures(res):
    lat = np.array([r["t_finish"] - r["t_submit"] for r in res])
    span = max(r["t_finish"] for r in res) - min(r["t_submit"] for r in res)
    pairs = float(sum(r["n"] ** 2 * r["steps"] for r in res))
    steps = float(sum(r["steps"] for r in res))
    return lat, span, pairs, steps


def measure_served(nbm, stream, args):
    """Poisson arrivals (20/s) of sweep runs: element count log-uniform in
    [4,096, 262,144], donor expansion rate in [0.5, 2]e-5 r_L per step, steps
    uniform in [1,000, 20,000] divided by --served-steps-div; served by
    continuous batching (nb_server) under the 150 GB budget.  Compared with
    the same requests run one at a time through the single-system API with
    the FP64 diagnostics every step (and without them), each request timed
    alone for a few steps and charged its full step count."""
    import synth
    trace = synth.served_trace(args.served_requests, seed=0, steps_div=args.served_steps_div)
    res, adm, info, scfg = _serve(nbm, stream, trace, int(150e9))
    bad = [r for r in res if r["status"] != 0]
    lat, span, pairs, steps = _served_figures(res)
    mix_elems = sum(r["desc"]["n_donor"] + r["desc"]["n_accretor"] for r in trace)

    # the same requests one at a time (single-system API, the library's
    # default configuration), each timed for k steps plain and k steps with
    # the FP64 diagnostics after every step, charged its full step count
    k = max(1, args.per_request_steps)
    t_plain = t_diag = 0.0
    for r in trace:
        with nbm.System(nbm.nb_desc_default(**r["desc"]), nbm.nb_params_default(**SWEEP_PARAMS),
                        stream=stream) as sy:
            sy.step(1)
            sy.diagnostics()
            sy.sync()
            c0 = time.perf_counter()
            sy.step(k)
            sy.sync()
            t_plain += (time.perf_counter() - c0) / k * r["nsteps"]
            c0 = time.perf_counter()
            for _ in range(k):
                sy.step(1)
                sy.diagnostics()
            t_diag += (time.perf_counter() - c0) / k * r["nsteps"]

    # three requests (the least work) run again alone with the server's pair
    # configuration: the same diagnostics bit for bit, and the error against
    # the oracle of the accelerations at their final state
    acc = []
    cheap = sorted(range(len(trace)), key=lambda r: (trace[r]["desc"]["n_donor"] +
                                                      trace[r]["desc"]["n_accretor"]) ** 2 *
                   trace[r]["nsteps"])[:3]
    for r in cheap:
        d = dict(trace[r]["desc"])
        with nbm.System(nbm.nb_desc_default(**d), nbm.nb_params_default(**SWEEP_PARAMS),
                        stream=stream) as sy:
            sy.set_pair_cfg(*[scfg[k] for k in PAIR_CFG_KEYS])
            xv, _, meta = sy.get_state(with_acc=False)
            sy.set_state(xv, None, meta)  # a^0 with the server's configuration
            sy.step(trace[r]["nsteps"])
            sy.sync()
            dg = sy.diagnostics()
            xv, _, meta = sy.get_state(with_acc=False)
            a = sy.forces()
        served_d = res[r]["diag"]
        same = all(np.array_equal(np.asarray(dg[k]), np.asarray(served_d[k]))
                   for k in ("step", "e_kin", "p", "l", "com", "separation", "n_past_L1",
                             "n_in_accretor_lobe", "n_unbound"))
        n_r = d["n_donor"] + d["n_accretor"]
        e = force_error(d, SWEEP_PARAMS["eps"], SWEEP_PARAMS["beta"], xv[:, :3], xv[:, 3:], a,
                        _sample_rows(n_r, d["n_donor"], 256, 40 + r), int(meta.step))
        acc.append(dict(e, request=int(r), n=int(n_r), alone_equals_served=bool(same)))

    div = args.served_steps_div
    out = {"workload": f"served_{len(trace)}", "requests": len(trace), "arrival_hz": 20.0,
           "n_range": [4096, 262144],
           "steps_range": [max(1, 1000 // div), max(1, 20000 // div)],
           "steps_scaled": f"config steps [1000, 20000] / {div}" if div != 1 else None,
           "slots": info["nslots"], "failed": len(bad),
           "pair_cfg": {k: scfg[k] for k in PAIR_CFG_KEYS},
           "p50_latency_s": float(np.percentile(lat, 50)),
           "p99_latency_s": float(np.percentile(lat, 99)),
           "makespan_s": span, "value": pairs / span, "unit": "pairs/s",
           "system_steps_per_s": steps / span,
           "admission": {"budget_bytes": adm["budget_bytes"],
                         "arena_elements": adm["capacity_elements"],
                         "mix_elements": int(mix_elems),
                         "peak_requests_in_flight": adm["peak_requests"],
                         "peak_bytes_in_flight": adm["peak_bytes"],
                         "admissions_deferred": adm["admissions_deferred"],
                         "device_bytes": adm["device_bytes"]},
           "per_system_path": {
               "plain_system_steps_per_s": steps / t_plain,
               "fp64_diag_system_steps_per_s": steps / t_diag,
               "note": f"every request alone through nb_step (plain) or nb_step(1) + "
                       f"nb_diagnostics (FP64 diagnostics every step), back to back with no "
                       f"arrival gaps, each timed for {k} steps and charged its step count"},
           "speedup_vs_per_system_fp64_diag": (steps / span) / (steps / t_diag),
           "speedup_vs_per_system_plain": (steps / span) / (steps / t_plain),
           "accuracy": {"requests": acc,
                        "max_force_rms_rel": max((a["force_rms_rel"] for a in acc), default=None),
                        "tolerance": 1e-5}}

    # the same arrivals with steps / 100 under a budget of two of the largest
    # runs, well below what the mix holds at once: admission binds, queued
    # runs wait for retirements, and every run still completes
    if args.served_bound:
        trace_b = synth.served_trace(args.served_requests, seed=0, steps_div=100)
        budget_b = 2 * int(adm["max_request_bytes"])
        res_b, adm_b, _, _ = _serve(nbm, stream, trace_b, budget_b)
        lat_b, span_b, pairs_b, steps_b = _served_figures(res_b)
        out["budget_bound"] = {
            "requests": len(trace_b), "steps_range": [10, 200],
            "steps_scaled": "config steps [1000, 20000] / 100",
            "budget_bytes": budget_b,
            "failed": sum(1 for r in res_b if r["status"] != 0),
            "p50_latency_s": float(np.percentile(lat_b, 50)),
            "p99_latency_s": float(np.percentile(lat_b, 99)),
            "makespan_s": span_b, "value": pairs_b / span_b, "unit": "pairs/s",
            "system_steps_per_s": steps_b / span_b,
            "peak_requests_in_flight": adm_b["peak_requests"],
            "peak_bytes_in_flight": adm_b["peak_bytes"],
            "admissions_deferred": adm_b["admissions_deferred"]}
    return out


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    ws, rank, local = _dist()
    from paper_2303_12166_gb300 import build as b
    b.build()
    from paper_2303_12166_gb300 import nbody as nbm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w = _workload(args.workload)
    n = w["n_donor"] + w["n_accretor"]
    stream = torch.cuda.Stream(device=dev)
    desc = nbm.nb_desc_default(n_donor=w["n_donor"], n_accretor=w["n_accretor"], q=w["q"],
                               f_donor=w["f_donor"], f_accretor=w["f_accretor"],
                               expand_rate=w["expand_rate"], expand_steps=w["expand_steps"],
                               sigma_v=w["sigma_v"], seed=w["seed"], stream=rank)
    params = nbm.nb_params_default(eps=w["eps"], dt=w["dt"], beta=0.5,
                                   force_prec=64 if args.fp64 else 32)
    sysm = nbm.System(desc, params, stream=stream)
    if args.pair_cfg:
        sysm.set_pair_cfg(*[int(v) for v in args.pair_cfg.split(",")])
        tuned = sysm.pair_cfg()
    else:
        tuned = sysm.autotune(2) if not args.fp64 else sysm.pair_cfg()
    if args.contact_lanes:
        sysm.set_contact_lanes(args.contact_lanes)
    contact_lanes = sysm.contact_lanes()
    # accelerations at the initial state with the configuration timed below
    # (compared with the oracle after the timed region)
    a_initial = sysm.forces()

    sysm.step(args.warmup)
    sysm.sync()
    sysm.profile(True)
    sysm.profile_read(reset=True)

    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    # a working set that L2 could hold: flush L2 (write a buffer of twice its
    # size on the library's stream) before every timed step, each step timed
    # on its own; otherwise the steps run back to back in one call
    working_set = sysm.info.device_bytes
    flush = None
    if working_set < 2 * L2_BYTES:
        flush = torch.empty(int(2 * L2_BYTES) // 4, dtype=torch.float32, device=dev)
    with ClockSampler(uuid if rank == 0 else None) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        if flush is None:
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            sysm.step(args.steps)
            ev1.record(stream)
            events = [(ev0, ev1)]
        else:
            events = []
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sysm.step(1)
                e1.record(stream)
                events.append((e0, e1))
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
    sysm.sync()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in events)
    prof = sysm.profile_read(reset=True)
    sysm.profile(False)
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    pairs_step = float(n) * float(n)
    value = pairs_step * args.steps * ws / (ms_max * 1e-3)

    # roofline of the pair kernel: ALU-bound pairs/s of the device
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_src = _measured_peaks()
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sym = bool(tuned.get("symmetric", 0)) and not args.fp64
    clocks = clk.summary()
    rates = None
    try:
        # the pipes' issue rates, measured on this device now (per second per
        # SM), per clock at the SM clock sampled during the timed steps
        r = nbm.nb_measure_unit_rates(stream)
        mhz = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") == clocks.get("sm_mhz") \
            else sm_max_mhz
        rates = {"sm_mhz": mhz,
                 "fp32_lanes_per_clk_sm": r["fp32_lanes_per_s_sm"] / (mhz * 1e6),
                 "mufu_sqrt_per_clk_sm": r["mufu_sqrt_per_s_sm"] / (mhz * 1e6),
                 "mufu_rcp_per_clk_sm": r["mufu_rcp_per_s_sm"] / (mhz * 1e6),
                 "pair_mix_evals_per_clk_sm": r["pair_mix_evals_per_s_sm"] / (mhz * 1e6)}
        pair_mix_per_s = r["pair_mix_evals_per_s_sm"] * r["sm_count"]
    except nbm.NbError:
        rates = None
        pair_mix_per_s = None
    ppc, x_opt = pairs_per_sm_clk(sym, rates)
    peak_pairs = props.multi_processor_count * sm_max_mhz * 1e6 * ppc
    pair_ms = prof["pair_ms"] / max(prof["pair_launches"], 1)
    achieved = pairs_step / (pair_ms * 1e-3)

    # end to end through the public API with host buffers: per step, upload
    # the state, one step, read the state back
    e2e = None
    if not args.no_e2e:
        # page-locked host arrays (the state a caller keeps on the host)
        xv = torch.empty((n, 6), dtype=torch.float64, pin_memory=True).numpy()
        a = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
        _, _, meta = sysm.get_state(out=(xv, a))
        steps_e2e = max(1, min(args.steps, 3))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            sysm.set_state(xv, a, meta)
            sysm.step(1)
            _, _, meta = sysm.get_state(out=(xv, a))
        el = time.perf_counter() - t0
        e2e = {"value": pairs_step * steps_e2e * ws / el, "unit": "pairs/s",
               "h2d_bytes_per_step": int(n * (48 + 24)), "d2h_bytes_per_step": int(n * (48 + 24)),
               "steps": steps_e2e, "host_buffers": "page-locked"}

    # the state after every timed and end-to-end step, and its accelerations
    xv_f, _, meta_f = sysm.get_state(with_acc=False)
    a_final = sysm.forces()

    cpu = None
    accuracy = None
    oracle_configs = None
    if rank == 0:
        eps, beta = w["eps"], 0.5
        ic = None
        if ws == 1 and not args.no_cpu_baseline:
            rate, cores, sample, full_ic, _, rows0, ref0 = _oracle_sample(
                w, target_s=args.cpu_seconds)
            cpu = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                   "sample": sample}
            if not args.no_extras:
                oracle_configs = _oracle_configs()
            ic = full_ic[2:]
            initial = {"force_rms_rel": _rms_rel(a_initial[rows0], ref0),
                       "force_max_abs_rel": float(np.abs(a_initial[rows0] - ref0).max() /
                                                  np.abs(ref0).max()),
                       "rows": int(len(rows0)), "step": 0,
                       "vs": "oracle (FP64 direct sum), the cpu_baseline sample's rows"}
        else:
            from oracle import oracle
            x0, v0, m0, R0, g0 = oracle.make_ic(
                w["n_donor"], w["n_accretor"], w["q"], f_donor=w["f_donor"],
                f_accretor=w["f_accretor"], sigma_v=w["sigma_v"], seed=w["seed"])
            ic = (m0, R0, g0)
            initial = force_error(w, eps, beta, x0, v0, a_initial,
                                  _sample_rows(n, w["n_donor"], 1024, 1), 0, ic)
        final = force_error(w, eps, beta, xv_f[:, :3], xv_f[:, 3:], a_final,
                            _sample_rows(n, w["n_donor"], 1024, 2), int(meta_f.step), ic)
        accuracy = {"initial": initial, "final": final,
                    "tolerance": 1e-12 if args.fp64 else 1e-5,
                    "metric": "RMS-relative acceleration error on the sampled rows, at the "
                              "library's own state and the radii of that step"}

    sysm.close()
    batched = served = fp64_path = config1 = None
    if not args.no_extras:
        batched = measure_batched(nbm, torch, dev, stream, args, ws, rank)
        if rank == 0 and ws == 1:
            if args.served_requests > 0:
                served = measure_served(nbm, stream, args)
            fp64_path = measure_fp64_path(nbm, torch, dev, stream, args)
            if args.config1_steps > 0:
                config1 = measure_config1_run(nbm, torch, dev, stream, args)
    if rank == 0:
        cfg = _config(args.workload, w, {
            "force_prec": 64 if args.fp64 else 32,
            "pair_cfg": {k: tuned[k] for k in PAIR_CFG_KEYS},
            "contact_lanes": contact_lanes,
            "l2": f"no flush: per-step working set {working_set / 1e6:.0f} MB > 2 x L2 (129 MB)"
            if flush is None else
            f"L2 flushed (a {2 * L2_BYTES / 1e6:.0f} MB write) before every timed step, each "
            f"step timed alone: working set {working_set / 1e6:.0f} MB",
            "parallelism": f"replicas x{ws}"})
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.fp64 else "f32", "data": "synthetic", "config": cfg,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_pairs,
                         "unit": "pairs/s", "frac": achieved / peak_pairs,
                         "traffic": None if args.fp64 else _pair_traffic(args.workload, tuned),
                         "peak_basis": f"{props.multi_processor_count} SMs x {sm_max_mhz:.0f} MHz "
                                       f"({peak_src} sm_max_mhz) x {ppc:.3f} pairs/clk/SM: "
                                       + (f"{rates['fp32_lanes_per_clk_sm']:.1f} FP32 lanes, "
                                          f"{rates['mufu_sqrt_per_clk_sm']:.2f} MUFU sqrt and "
                                          f"{rates['mufu_rcp_per_clk_sm']:.2f} MUFU rcp per clk "
                                          f"per SM measured in this run"
                                          if rates else
                                          f"{FP32_PER_SM_CLK} FP32 lanes and {MUFU_PER_SM_CLK} MUFU "
                                          f"per clk per SM (nominal)")
                                       + f"; {FP32_PER_PAIR_SYM if sym else FP32_PER_PAIR:g} FP32 + "
                                       f"{MUFU_PER_PAIR:g} MUFU per evaluation, "
                                       f"{'2 interactions (i and j sides)' if sym else '1 interaction'}"
                                       f" per evaluation, a fraction {x_opt:.3f} of reciprocals shared",
                         "unit_rates": rates,
                         # the symmetric kernel's own instruction mix run from
                         # registers (no memory traffic) at its launch shape
                         "mix_ceiling": None if (pair_mix_per_s is None or not sym) else {
                             "value": 2.0 * pair_mix_per_s, "unit": "pairs/s",
                             "frac": achieved / (2.0 * pair_mix_per_s),
                             "basis": "pair_mix_kernel: the rotating step of the symmetric "
                                      "kernel (12 i-elements x 2 j per thread, 15 packed FP32 + "
                                      "4 MUFU per i-element, 3 shuffles) from registers, 2 x 128 "
                                      "threads per SM, measured in this run; 2 interactions per "
                                      "evaluation"},
                         "kernel": "pair_sym_kernel" if sym else "pair_f32_kernel",
                         "kernel_ms": pair_ms},
            "cpu_baseline": cpu,
            "oracle_other_workloads": oracle_configs,
            "accuracy": accuracy,
            "e2e": e2e,
            "gpu_launches": int(prof["kernels"]),
            "phase_ms": {"pair": prof["pair_ms"], "contact": prof["contact_ms"],
                         "update": prof["update_ms"]},
            "clocks": clocks,
            "batched": batched,
            "served": served,
            "fp64_path": fp64_path,
            "config1_run": config1,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="binary_1m", choices=sorted(WORKLOADS))
    ap.add_argument("--fp64", action="store_true", help="FP64 pair term (comparison path)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-sweep and served measurements")
    ap.add_argument("--sweep-systems", type=int, default=256)
    ap.add_argument("--batched-steps", type=int, default=100)
    ap.add_argument("--per-system-steps", type=int, default=5,
                    help="steps each sweep system is timed for alone (0: skip)")
    ap.add_argument("--served-requests", type=int, default=64)
    ap.add_argument("--config1-steps", type=int, default=10000,
                    help="steps of the 65,536-element growing-donor run (0: skip)")
    ap.add_argument("--served-steps-div", type=int, default=10)
    ap.add_argument("--no-served-bound", dest="served_bound", action="store_false",
                    help="skip the served run under a budget that makes admission bind")
    ap.add_argument("--per-request-steps", type=int, default=3,
                    help="steps each served request is timed for alone")
    ap.add_argument("--contact-lanes", type=int, default=0, choices=[0, 1, 3],
                    help="contact kernel threads per element (0: the tuner's or the default)")
    ap.add_argument("--pair-cfg", default="",
                    help="tile,i_per_thread,threads,min_blocks,nr_slots,i_packed,shared_rcp[,symmetric] (skips the "
                         "autotuner)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
