#!/usr/bin/env python
"""SNAP energy + force benchmark on GB300 (atom-steps/s).

One step = one full snap_compute: device neighbour build, Cayley-Klein
geometry, compute_U, compute_Y, fused dU + dE and the force/virial gather, on
a synthetic BCC configuration resident in HBM.  The headline workload is the
paper's benchmark shape (2000 atoms, 26 neighbours, 2J = 8) in mixed
precision; FP64 and 2J = 14 (2000 and 16000 atoms) are reported as variants.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (under torchrun) runs independent replicas, one per GPU (the SNAP
evaluation of one configuration does not shard here), weak scaling.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SNAP energy+force atom-steps/s at 2J=8/14: mixed vs FP64 on 1 GB300"
UNIT = "atom-steps/s"
FLUSH_BYTES = 256 << 20          # > 129 MB L2
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.5: SMs x FP32 lanes x FMA x max clock
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12         # 1.26: SMs x 2 DFMA/clk x FMA x max clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant-seconds", type=float, default=1.0)
    ap.add_argument("--workload", default="bcc10_2j8",
                    help="headline workload (bcc4_2j8, bcc10_2j8, bcc10_2j14, bcc20_2j14)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--neighbors", default="built", choices=["built", "supplied"],
                    help="supplied: the headline takes the neighbour list from the caller")
    ap.add_argument("--row", choices=["batch", "bispectrum", "force_matching"],
                    help="only this widened row (one JSON line, no headline)")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="only measure the FP32 and FP64 FMA peaks (snap_probe_fma) with clocks")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        time.sleep(0.05)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                smax = max(smax, float(r[1]))
            except ValueError:
                continue
            for name, v in zip(names, r[4:]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(pg, x: float, dev) -> float:
    """The largest x over the ranks of process group module `pg` (x itself
    without one): the job's time is its slowest rank's."""
    if not pg:
        return x
    import torch
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, natoms: int, ms: float) -> float:
    """Atom-steps/s of the whole job: every rank evaluates its own replica of
    `natoms` atoms per step, and a step lasts `ms` (the slowest rank's)."""
    return world * natoms / (ms * 1e-3)


def read_traffic(kernel: str, workload: str, precision: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary (a line 'traffic <kernel> <workload> <precision> <bytes>'), else
    None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        p = line.split()
        if len(p) == 5 and p[0] == "traffic" and p[1] == kernel and p[2] == workload and p[3] == precision:
            return float(p[4])
    return None


def cpu_baseline(w, seconds=10.0):
    """The FP64 oracle, as it stands, on the host cores: whole evaluations of
    the workload (energy, forces, virial) repeated for about `seconds`."""
    from oracle import snap_oracle as O
    cfg, beta = w.config(), w.beta()
    p = O.Params(w.twojmax)
    pairs = O.build_neighbors(cfg.pos, cfg.box, p.rcut)
    n = cfg.natoms
    if w.twojmax > 8:
        # 2J = 14: evaluate a fixed subset of centre atoms per step
        import numpy as np
        need = np.zeros(n, dtype=bool)
        need[: min(n, 256)] = True
        sample = f"oracle E+dE/dr for the first {int(need.sum())} of {n} atoms per step"
        units = int(need.sum())
    else:
        need = None
        sample = f"oracle full E+F+virial of all {n} atoms per step (neighbour list built once)"
        units = n
    t0 = time.perf_counter()
    steps = 0
    while True:
        O.compute(p, beta, n, pairs, need=need)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 50:
            break
    return {"value": units * steps / el, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "sample": f"{sample}; {steps} steps in {el:.1f} s, workload {w.name}"}


def accuracy_vs_oracle(torch, snap, inputs, dev):
    """The GPU results, mixed and FP64, against the FP64 oracle (part of the
    cpu_baseline leg, the bench step that runs the oracle), per 2J: every atom
    of the 2000-atom BCC configuration of the benchmark (+-0.1 A, the
    benchmark's beta draw for that 2J) at 2J = 2, 4, ..., 14.  Errors are
    relative to the largest magnitude of each quantity (E_i, F, virial), plus
    the largest absolute force error (eV/A for beta in eV)."""
    import numpy as np
    from oracle import snap_oracle as O

    def gpu(J, beta, cfg, prec):
        s = snap.Snap(J, beta, precision=prec)
        E, F, W = [x.cpu().numpy() for x in s.compute(torch.tensor(cfg.pos, device=dev), cfg.box)]
        s.close()
        return E, F, W

    def err(a, b):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

    out = {}
    cfg = inputs.WORKLOADS["bcc10_2j8"].config()
    pairs = O.build_neighbors(cfg.pos, cfg.box, inputs.RCUT)
    for J in (2, 4, 6, 8, 10, 12, 14):
        beta = inputs.beta(J)
        ref = O.compute(O.Params(J), beta, cfg.natoms, pairs)
        for prec, tag in ((snap.MIXED, "mixed"), (snap.FP64, "fp64")):
            E, F, W = gpu(J, beta, cfg, prec)
            out[f"2j{J}_{tag}"] = {"E": err(E, ref.E), "F": err(F, ref.F), "W": err(W, ref.W),
                                   "F_max_abs": float(np.abs(F - ref.F).max())}
    return out


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on the host cores, each step
    a bounded sample (a fixed subset of centre atoms) of the workload."""
    import numpy as np
    from oracle import snap_oracle as O
    from paper_2011_12875_gb300 import inputs
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    w = inputs.WORKLOADS[args.workload]
    cfg, beta = w.config(), w.beta()
    p = O.Params(w.twojmax)
    pairs = O.build_neighbors(cfg.pos, cfg.box, p.rcut)
    n = cfg.natoms
    # calibrate: time per centre atom
    need = np.zeros(n, dtype=bool)
    need[:64] = True
    t0 = time.perf_counter()
    O.compute(p, beta, n, pairs, need=need)
    per_atom = (time.perf_counter() - t0) / 64
    budget = 120.0 / max(1, args.steps + args.warmup)
    m = int(max(1, min(n, budget / max(per_atom, 1e-9))))
    if m >= n:
        need = None     # the whole step: E, dE/dr, forces and virial of every atom
        sample = f"oracle E, F and virial of all {n} atoms per step ({w.name})"
    else:
        need = np.zeros(n, dtype=bool)
        need[:m] = True
        sample = f"oracle E + dE/dr of {m} of {n} centre atoms per step ({w.name})"
    for _ in range(args.warmup):
        O.compute(p, beta, n, pairs, need=need)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.compute(p, beta, n, pairs, need=need)
    el = time.perf_counter() - t0
    value = m * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "natoms": n, "twojmax": w.twojmax,
                                        "sample_atoms": m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_variant(torch, snap, w, precision, steps, warmup, flush, dev, profile=False, supplied=False):
    """Device time of `steps` evaluations (CUDA events on the compute stream,
    L2 flushed between steps outside the events).  supplied: the neighbour
    list is the caller's (the library's own list of the configuration, read
    back once and passed in, as an MD code passes its list), so a step is
    compute_U from the stored separations instead of the build."""
    import numpy as np
    cfg, beta = w.config(), w.beta()
    s = snap.Snap(w.twojmax, beta, precision=precision)
    pos = torch.tensor(cfg.pos, dtype=torch.float64, device=dev)
    n = cfg.natoms
    E = torch.empty(n, dtype=torch.float64, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    W = torch.empty(6, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    nb = {}
    if supplied:
        s.compute(pos, cfg.box, E, F, W)
        idx = s.get_buffer(snap.BUF_NBR_IDX)
        K = idx.size // n
        nb = {"neighbors": (torch.tensor(s.get_buffer(snap.BUF_NBR_CNT), device=dev),
                            torch.tensor(idx.reshape(n, K), device=dev),
                            torch.tensor(s.get_buffer(snap.BUF_NBR_IMG).reshape(n, K, 3), device=dev))}
    for _ in range(warmup):
        s.compute(pos, cfg.box, E, F, W, wait=False, **nb)
    s.sync()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(steps):
        flush.fill_(k & 0xff)
        evs[k][0].record(stream)
        s.compute(pos, cfg.box, E, F, W, wait=False, **nb)
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    s.sync()
    ms = [a.elapsed_time(b) for a, b in evs]
    prof = None
    if profile:
        # stage times from a separate pass with events between the stages
        # (they would otherwise perturb the timed steps above)
        s.profile(True)
        for k in range(min(steps, 20)):
            flush.fill_(k & 0xff)
            s.compute(pos, cfg.box, E, F, W, wait=False, **nb)
        s.sync()
        prof = s.profile_read()
        s.profile(False)
    launches = s.launches_per_call()
    cnt = s.get_buffer(snap.BUF_NBR_CNT)
    npairs = int(cnt.sum())
    hist = {int(k): int(v) for k, v in enumerate(np.bincount(cnt)) if v}
    s.close()
    return {"ms": ms, "wall": wall, "prof": prof, "launches": launches, "npairs": npairs,
            "natoms": n, "neighbor_hist": hist}


def e2e_host(snap, torch, w, precision, steps):
    """Same metric through snap_compute_host with pinned host buffers: every
    step moves the positions host -> device and the energies, forces and
    virial device -> host inside the call (the library reads and writes them
    through the host mapping of the pinned buffers), wall clock per call."""
    import numpy as np
    cfg, beta = w.config(), w.beta()
    n = cfg.natoms
    s = snap.Snap(w.twojmax, beta, precision=precision)
    pin = lambda shape: torch.empty(shape, dtype=torch.float64).pin_memory().numpy()
    pos = pin((n, 3))
    pos[:] = cfg.pos
    out = (pin((n,)), pin((n, 3)), pin((6,)))
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(3):
        s.compute_host(pos, cfg.box, stream=stream, out=out)
    t0 = time.perf_counter()
    for _ in range(steps):
        s.compute_host(pos, cfg.box, stream=stream, out=out)
    el = time.perf_counter() - t0
    s.close()
    return {"value": n * steps / el, "unit": UNIT, "h2d_bytes_per_step": n * 3 * 8,
            "d2h_bytes_per_step": n * 8 + n * 3 * 8 + 6 * 8, "steps": steps,
            "ms_per_step": 1e3 * el / steps}


def _events_time(torch, fn, steps, flush, dev):
    """Mean device milliseconds of fn() over `steps` calls (events around each
    call on the current stream, L2 flushed between calls)."""
    stream = torch.cuda.current_stream(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    torch.cuda.synchronize(dev)
    for k in range(steps):
        flush.fill_(k & 0xff)
        evs[k][0].record(stream)
        fn()
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    return statistics.mean(a.elapsed_time(b) for a, b in evs)


def row_batch(torch, snap, inputs, flush, dev, args):
    """Batched evaluation of 64 uneven configurations (graph replay vs a
    per-configuration loop, after the autotuner), and compute_Y's two
    layouts on the headline workload."""
    import numpy as np
    out = {}
    # --- batch: 64 configurations, 54..2000 atoms, +-2% strain, 2J = 8, mixed
    cfgs = inputs.batch(64)
    natoms = np.array([c.natoms for c in cfgs])
    boxes = np.array([c.box for c in cfgs])
    pos = torch.tensor(np.concatenate([c.pos for c in cfgs]), device=dev)
    total = int(natoms.sum())
    beta = inputs.beta(8)
    s = snap.Snap(8, beta, precision=snap.MIXED)
    E = torch.empty(total, dtype=torch.float64, device=dev)
    F = torch.empty((total, 3), dtype=torch.float64, device=dev)
    W = torch.empty((len(cfgs), 6), dtype=torch.float64, device=dev)
    steps = max(5, min(args.steps, 50))
    default_tuning = s.get_tuning()
    s.compute_batch(pos, natoms, boxes, E, F, W, use_graph=True)
    t_default = _events_time(torch, lambda: s.compute_batch(pos, natoms, boxes, E, F, W, use_graph=True,
                                                            wait=False), steps, flush, dev)
    best_ms = s.autotune(pos, natoms, boxes, reps=5)
    tuned = s.get_tuning()
    tuned_persist = s.get_knob(snap.KNOB_PERSIST)
    tuned_de_atoms = s.get_knob(snap.KNOB_DE_ATOMS)
    s.compute_batch(pos, natoms, boxes, E, F, W, use_graph=True)
    t_graph = _events_time(torch, lambda: s.compute_batch(pos, natoms, boxes, E, F, W, use_graph=True,
                                                          wait=False), steps, flush, dev)
    t_nograph = _events_time(torch, lambda: s.compute_batch(pos, natoms, boxes, E, F, W, use_graph=False,
                                                            wait=False), steps, flush, dev)
    # the persistent work-queue launches at the tuned shape, graph replay
    per_persist = {}
    for p_ in (0, 1, 2, 3):
        s.set_knob(snap.KNOB_PERSIST, p_)
        s.compute_batch(pos, natoms, boxes, E, F, W, use_graph=True)
        per_persist[p_] = _events_time(torch, lambda: s.compute_batch(pos, natoms, boxes, E, F, W, use_graph=True,
                                                                      wait=False), steps, flush, dev)
    s.set_knob(snap.KNOB_PERSIST, tuned_persist)
    s.sync()
    singles = [torch.tensor(c.pos, device=dev) for c in cfgs]
    outs = [(torch.empty(c.natoms, dtype=torch.float64, device=dev),
             torch.empty((c.natoms, 3), dtype=torch.float64, device=dev),
             torch.empty(6, dtype=torch.float64, device=dev)) for c in cfgs]

    def loop():
        for c, p_, (e_, f_, w_) in zip(cfgs, singles, outs):
            s.compute(p_, c.box, e_, f_, w_, wait=False)
    loop()
    s.sync()
    t_loop = _events_time(torch, loop, max(3, steps // 5), flush, dev)
    s.sync()
    s.close()
    out["batch_64_configs_2j8_mixed"] = {
        "natoms_total": total, "atom_counts": sorted(set(int(n) for n in natoms)),
        "graph_atom_steps_per_s": total / (t_graph * 1e-3), "graph_ms": t_graph,
        "batched_no_graph_ms": t_nograph, "per_config_loop_ms": t_loop,
        "per_config_loop_atom_steps_per_s": total / (t_loop * 1e-3),
        "speedup_vs_loop": t_loop / t_graph,
        "graph_ms_by_persist": per_persist,
        "default_tuning": {"col_warps": default_tuning[0], "yi_waves": default_tuning[1],
                           "yi_layout": default_tuning[2], "graph_ms": t_default},
        "autotuned": {"col_warps": tuned[0], "yi_waves": tuned[1], "yi_layout": tuned[2],
                      "persist": tuned_persist, "de_atoms": tuned_de_atoms, "autotune_median_ms": best_ms}}
    # --- compute_Y layouts on the headline workload: warp of 32 atoms (AoSoA)
    # vs warp per atom, stage time and whole step
    w = inputs.WORKLOADS["bcc10_2j8"]
    cfg = w.config()
    lay = {}
    for layout, tag in ((0, "warp_of_32_atoms"), (1, "warp_per_atom")):
        s = snap.Snap(8, w.beta(), precision=snap.MIXED)
        s.set_tuning(4, 2, layout)
        p_ = torch.tensor(cfg.pos, device=dev)
        for _ in range(3):
            s.compute(p_, cfg.box, wait=False)
        t = _events_time(torch, lambda: s.compute(p_, cfg.box, wait=False), 10, flush, dev)
        s.profile(True)
        for _ in range(10):
            s.compute(p_, cfg.box, wait=False)
        pr = s.profile_read()
        s.profile(False)
        s.close()
        lay[tag] = {"step_ms": t, "compute_yi_ms": pr["compute_yi"][0] / max(pr["compute_yi"][1], 1)}
    out["compute_y_layout_2000_2j8_mixed"] = lay
    return out


def row_bispectrum(torch, snap, inputs, flush, dev, args):
    """Bispectrum output, 2000 atoms, 2J = 8, both precisions."""
    out = {}
    w = inputs.WORKLOADS["bcc10_2j8"]
    cfg = w.config()
    for prec, tag in ((snap.MIXED, "mixed"), (snap.FP64, "fp64")):
        s = snap.Snap(8, w.beta(), precision=prec)
        p_ = torch.tensor(cfg.pos, device=dev)
        Bout = torch.empty((cfg.natoms, snap.num_coeff(8)), dtype=torch.float64, device=dev)
        s.bispectrum(p_, cfg.box, out=Bout)
        t = _events_time(torch, lambda: s.bispectrum(p_, cfg.box, out=Bout, wait=False), 30, flush, dev)
        s.sync()
        t_sync = _events_time(torch, lambda: s.bispectrum(p_, cfg.box, out=Bout), 30, flush, dev)
        out[f"bispectrum_2000_2j8_{tag}"] = {"atom_steps_per_s": cfg.natoms / (t * 1e-3), "ms": t,
                                             "ms_with_host_wait": t_sync,
                                             "includes": "neighbour list, geometry, compute_U, B"}
        s.close()
    return out


def row_force_matching(torch, snap, inputs, flush, dev, args):
    """Force-matching loss + gradient over 32 configurations, 2J = 8 and 14."""
    import numpy as np
    out = {}
    from paper_2011_12875_gb300 import autograd as AG
    fit = inputs.fitting_set(32)
    rng = np.random.Generator(np.random.PCG64(99))
    natoms_f = np.array([c.natoms for c in fit])
    boxes_f = np.array([c.box for c in fit])
    pos_f = torch.tensor(np.concatenate([c.pos for c in fit]), device=dev)
    fref_f = torch.tensor(rng.normal(size=(int(natoms_f.sum()), 3)), device=dev)
    for J in (8, 14):
        s = snap.Snap(J, inputs.beta(J), precision=snap.MIXED)

        def fm_step():
            return AG.force_matching_grad_batch(s, pos_f, natoms_f, boxes_f, fref_f)[1]
        fm_step()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        reps = 10
        for _ in range(reps):
            fm_step()
        torch.cuda.synchronize(dev)
        el = (time.perf_counter() - t0) / reps
        na = sum(c.natoms for c in fit)
        out[f"force_matching_step_2j{J}_mixed"] = {
            "configs": len(fit), "natoms_total": na, "seconds_per_step": el,
            "atom_steps_per_s": na / el,
            "step": "all 32 configurations batched: E, F (snap_compute_batch); loss sum|F-F_ref|^2; "
                    "dL/dbeta via snap_bispectrum_deriv_batch"}
        s.close()
    return out


ROWS = {"batch": row_batch, "bispectrum": row_bispectrum, "force_matching": row_force_matching}


def next_rows(torch, snap, inputs, flush, dev, args):
    """Measurements of the widened rows: batched evaluation, bispectrum
    output, and the force-matching loss + gradient."""
    out = {}
    for fn in ROWS.values():
        out.update(fn(torch, snap, inputs, flush, dev, args))
    return out


def probe_peaks():
    """FP32 and FP64 FMA peaks of this GPU (best of 5 timed launches each,
    snap_probe_fma), with the SM clocks sampled while they ran."""
    import torch
    from paper_2011_12875_gb300 import build, snap
    build.build()
    snap.load()
    torch.cuda.set_device(0)
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    out = {}
    for prec, tag, iters in ((snap.MIXED, "fp32", 1 << 18), (snap.FP64, "fp64", 1 << 13)):
        sampler = ClockSampler(int(cvd) if cvd.isdigit() else 0)
        sampler.start()
        t0 = time.perf_counter()
        vals = []
        while len(vals) < 5 or time.perf_counter() - t0 < 1.0:
            vals.append(snap.probe_fma(prec, iters))
        out[tag] = {"tflops": max(vals), "median_tflops": statistics.median(vals), "runs": len(vals),
                    "clocks": sampler.stop()}
    out["derived_tflops"] = {"fp32": FP32_PEAK_TFLOPS, "fp64": FP64_PEAK_TFLOPS}
    print(json.dumps({"fma_peaks": out}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.probe_peaks:
        probe_peaks()
        return
    import torch
    world, rank, local = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_2011_12875_gb300 import build, flops, inputs, snap
    build.build()
    snap.load()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    if args.row:
        if rank == 0:
            print(json.dumps({"row": args.row, **ROWS[args.row](torch, snap, inputs, flush, dev, args)}), flush=True)
        if pg:
            pg.barrier()
            pg.destroy_process_group()
        return

    head = inputs.WORKLOADS[args.workload]
    hprec = snap.MIXED if args.precision == "mixed" else snap.FP64
    hpeak = FP32_PEAK_TFLOPS if hprec == snap.MIXED else FP64_PEAK_TFLOPS
    # measured FMA peak of the headline's working precision (context beside
    # the derived peak the roofline fraction uses)
    try:
        measured_peak = snap.probe_fma(hprec, 1 << 16 if hprec == snap.MIXED else 1 << 12)
    except snap.SnapError:
        measured_peak = None
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    sampler = ClockSampler(int(cvd) if cvd.isdigit() else local)
    if pg:
        pg.barrier()
    sampler.start()
    r = time_variant(torch, snap, head, hprec, args.steps, args.warmup, flush, dev,
                     profile=True, supplied=args.neighbors == "supplied")
    clocks = sampler.stop()
    ms_mean = statistics.mean(r["ms"])
    ms_med = statistics.median(r["ms"])
    t_max = max_over_ranks(pg, ms_mean, dev)
    value = job_throughput(world, r["natoms"], t_max)

    # roofline of the dominant kernel (largest share of the step)
    prof = r["prof"]
    dom = max(prof, key=lambda k: prof[k][0])
    fl = flops.step(head.twojmax, r["natoms"], r["npairs"])
    dom_ms = prof[dom][0] / max(prof[dom][1], 1)
    achieved = fl.get(dom, 0) / (dom_ms * 1e-3) / 1e12
    stages = {k: {"ms_per_call": v[0] / max(v[1], 1),
                  "share": v[0] / sum(x[0] for x in prof.values())} for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 recursions, f64 geometry and sums" if hprec == snap.MIXED else "f64",
        "data": "synthetic BCC, +-0.1 A, seeded beta",
        "config": {"workload": head.name, "natoms": r["natoms"], "twojmax": head.twojmax,
                   "precision": args.precision, "l2": "flushed between steps",
                   "neighbors": args.neighbors, "parallelism": f"replicas x{world}"},
        "gpu_launches": r["launches"] * args.steps,
        "roofline": {"kernel": dom, "bound": "alu", "achieved": round(achieved, 3),
                     "peak": round(hpeak, 2), "unit": "TFLOP/s", "frac": round(achieved / hpeak, 4),
                     "peak_measured": round(measured_peak, 2) if measured_peak else None,
                     "traffic": read_traffic(dom, head.name, args.precision)},
        "clocks": clocks,
    }
    detail = {"ms_per_step_median": ms_med, "neighbors": r["npairs"] / r["natoms"],
              "neighbor_hist": r["neighbor_hist"], "stages": stages,
              "flops_per_launch": fl.get(dom, 0),
              "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"
                              if hprec == snap.MIXED else "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz"),
              "peak_measured_source": "snap_probe_fma (8 FMA chains per thread, 8 CTAs of 256 per SM)"}
    # end to end through host buffers, on every rank; the job's step is the
    # slowest rank's
    if pg:
        pg.barrier()
    e2e = e2e_host(snap, torch, head, hprec, min(args.steps, 300))
    e2e["ms_per_step"] = max_over_ranks(pg, e2e["ms_per_step"], dev)
    e2e["value"] = job_throughput(world, r["natoms"], e2e["ms_per_step"])
    if rank == 0:
        line["e2e"] = {k: (round(v, 5) if isinstance(v, float) else v) for k, v in e2e.items()}
        variants = {}
        if not args.no_variants:
            for name, prec, tag in (("bcc10_2j8", snap.FP64, "fp64_2j8_2000"),
                                    ("bcc10_2j14", snap.MIXED, "mixed_2j14_2000"),
                                    ("bcc10_2j14", snap.FP64, "fp64_2j14_2000"),
                                    ("bcc20_2j14", snap.MIXED, "mixed_2j14_16000"),
                                    ("bcc20_2j14", snap.FP64, "fp64_2j14_16000")):
                w = inputs.WORKLOADS[name]
                probe = time_variant(torch, snap, w, prec, 2, 1, flush, dev)
                est = statistics.mean(probe["ms"]) * 1e-3
                k = int(max(3, min(args.steps, args.variant_seconds / max(est, 1e-6))))
                v = time_variant(torch, snap, w, prec, k, 2, flush, dev, profile=True)
                vm = statistics.mean(v["ms"])
                vp = v["prof"]
                vdom = max(vp, key=lambda x: vp[x][0])
                vfl = flops.step(w.twojmax, v["natoms"], v["npairs"])
                vdom_ms = vp[vdom][0] / max(vp[vdom][1], 1)
                peak = FP32_PEAK_TFLOPS if prec == snap.MIXED else FP64_PEAK_TFLOPS
                ach = vfl.get(vdom, 0) / (vdom_ms * 1e-3) / 1e12
                variants[tag] = {"value": round(v["natoms"] / (vm * 1e-3)), "ms": round(vm, 4),
                                 "kernel": vdom, "frac": round(ach / peak, 4)}
                detail.setdefault("variants", {})[tag] = {
                    "steps": k, "dominant_share": vp[vdom][0] / sum(x[0] for x in vp.values()),
                    "achieved_tflops": ach, "peak_tflops": peak,
                    "stages_ms": {x: vp[x][0] / max(vp[x][1], 1) for x in vp}}
            # the headline workload with the caller's neighbour list (an MD
            # code's list): compute_U from stored separations, no build
            w = inputs.WORKLOADS["bcc10_2j8"]
            v = time_variant(torch, snap, w, snap.MIXED, max(3, min(args.steps, 300)), 3, flush, dev,
                             profile=True, supplied=True)
            vm = statistics.mean(v["ms"])
            detail["supplied_list_2j8_2000_mixed"] = {
                "value": round(v["natoms"] / (vm * 1e-3)), "ms": round(vm, 4),
                "stages_ms": {x: v["prof"][x][0] / max(v["prof"][x][1], 1) for x in v["prof"]}}
            detail["next"] = next_rows(torch, snap, inputs, flush, dev, args)
        variants["mixed_2j8_2000"] = {"value": round(value / world), "ms": round(ms_mean, 4),
                                      "kernel": dom, "frac": round(achieved / hpeak, 4)}
        acc = None
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(head)
            acc = accuracy_vs_oracle(torch, snap, inputs, dev)
            detail["accuracy_vs_oracle"] = acc
            # the unreduced method's flops (counted in the oracle's loops)
            # beside the library's reduced algorithm (flops.py), per unit
            from oracle import snap_oracle as O
            detail["flops_per_unit"] = {}
            for J in (8, 14):
                o = O.flops(J)
                detail["flops_per_unit"][f"2j{J}"] = {
                    "oracle": o, "library": {"compute_u_pair": flops.ui_pair(J), "y_atom": flops.yi_atom(J),
                                             "de_pair": flops.de_pair(J)}}
        # the detail first (its own line, no "metric" key), then the bench
        # line itself, short, with the variants and the per-2J force error
        # last so that a short tail of the output still holds them
        print(json.dumps({"bench_detail": detail}), flush=True)
        line["variants"] = variants
        if acc:
            line["force_err_vs_oracle"] = {k: float(f"{v['F']:.2g}") for k, v in acc.items()}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
