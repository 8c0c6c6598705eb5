"""Benchmark of the SPH hot path on GB300: one time step = bin -> AoS->SoA
(U o N o C) -> density with 5 Newton h steps -> force -> kick/drift ->
SoA->AoS, on the 1,072,476-particle Sod shock tube (FP64 AoS master, FP32
SoA storage and arithmetic).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is SPH pair interactions per second (ordered
pairs j != i inside the support, summed over every density pass and the force
pass, counted by the kernels), whole job over all ranks.  Each step is timed
with CUDA events on the library's stream; the L2 is flushed (a 512 MiB write)
between steps, outside the timed intervals.  `--impl reference` times the FP64
CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import sph_inputs  # noqa: E402

METRIC = "SPH pair-interactions/s (density+force)"
UNIT = "pairs/s"
# flops per interacting pair (FMA 2; add, mul, compare, rsqrt 1): density 29 =
# distance 8 + r and q 3 + spline and derivative 11 + compensated sum 4 + dh
# sum 3; force 50 = distance 8 + r, mean h and q 6 + spline derivative 3 +
# gradient 4 + v.r 8 + viscosity 13 + accumulation 8
FLOPS_PER_PAIR = {"density": 29, "force": 50}
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lattice", type=int, default=124, help="Sod lattice (124 -> 1,072,476 particles)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time eager steps instead of graph replays")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="fp32", help="SoA storage of v, m, h, u (fp32|bf16|fp16|m16|m10)")
    ap.add_argument("--no-long-run", action="store_true", help="skip the 33.5M-particle memory-bound rows")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes instead of the autotuner's")
    ap.add_argument("--no-uneven", action="store_true", help="skip the 16.7M-particle clustered batching rows")
    ap.add_argument("--no-vs-plain", action="store_true", help="skip the plain FP32 SoA comparison")
    ap.add_argument("--no-streaming", action="store_true", help="skip the host-resident AoS comparison")
    ap.add_argument("--no-buffers", action="store_true", help="skip the 64-particle-buffer AoS/SoA comparison")
    ap.add_argument("--no-placement", action="store_true", help="skip the host-vs-GPU conversion placement rows")
    ap.add_argument("--no-levels", action="store_true", help="skip the per-particle-h level hierarchy rows")
    ap.add_argument("--levels-only", action="store_true", help="print only the level hierarchy rows")
    ap.add_argument("--profile-n", type=int, default=2_097_152,
                    help="particles of the levels profile case")
    ap.add_argument("--profile-case", choices=["pairs", "memory", "buffers", "levels"], default=None,
                    help="run one small fixed workload for an ncu capture and exit")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- workload
def workload(args):
    return sph_inputs.sod(n_lattice=args.lattice)


def prec_of(args):
    if args.prec == "fp32":
        return None
    return {"v": args.prec, "m": args.prec, "h": args.prec, "u": args.prec}


def kernel_sources_sha256(paths) -> str:
    """SHA-256 over the concatenated bytes of a kernel's source files."""
    h = hashlib.sha256()
    for p in paths:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_from_profile(kernel_srcs, kernel: str):
    """DRAM bytes per launch of a pair kernel from the committed ncu summary,
    if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "k_pairs_sod1m.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_src = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    m_tr = re.search(re.escape(kernel) + r"\.dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m_src or not m_tr:
        return None
    return float(m_tr.group(1)) if kernel_sources_sha256(kernel_srcs) == m_src.group(1) else None


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


# ----------------------------------------------------------------- ours
def run_ours(args, rank, world):
    import torch
    import paper_2512_05516_gb300 as sph

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    wl = workload(args)
    n = wl.n
    stream = torch.cuda.Stream(dev)
    aos_host = torch.from_numpy(wl.aos.copy())
    aos = aos_host.to(dev)
    nc = [int(math.floor(b / max(wl.cell_edge, 2 * wl.h_cap))) for b in wl.box]
    params = sph.make_params(wl.box, gamma=wl.gamma, alpha=wl.alpha_av, beta=wl.beta_av,
                             eps=wl.eps_av, eta=wl.eta, h_max=wl.h_cap)
    s = sph.Sph(aos, sph.layout_112(), params, int(np.prod(nc)), 0, stream=stream)
    prec = prec_of(args)
    # launch shapes from the project's autotuner (searched once per kind of
    # workload and device, then cached)
    tuned = {"tuning": s.tuning(), "cached": None}
    if not args.no_autotune:
        from paper_2512_05516_gb300 import autotune
        with torch.cuda.stream(stream):
            tuned = autotune.tune(s, wl.cell_edge, prec, wl.newton_steps)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    names = ["bin", "aos_to_soa", "density", "force", "kick_drift_writeback"]

    def step(ev=None):
        calls = [lambda: s.bin_cells(wl.cell_edge, drift_keys=True),
                 lambda: s.aos_to_soa(sph.FIELDS_FORCE, prec),
                 lambda: s.density(wl.newton_steps),
                 lambda: s.force(),
                 lambda: s.kick_drift_writeback(wl.dt, wl.dt, sph.FIELDS_OUTPUT)]
        for i, fn in enumerate(calls):
            if ev is not None:
                ev[i][0].record(stream)
            fn()
            if ev is not None:
                ev[i][1].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        s.reset_stats()
        launches0 = s.stats()["launches"]
        K = args.steps
        ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        ev_k = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in names]
                for _ in range(K)]
        # the library records these around the pair kernels themselves (after
        # their pack passes): the roofline's launch durations
        ev_pk = [{w: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for w in (sph.KEV_DENSITY, sph.KEV_FORCE)} for _ in range(K)]
        clocks = ClockSampler(dev.index)
        clocks.start()
        time.sleep(0.3)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)
        for k in range(K):
            flush.fill_(k & 0xFF)                    # evict the L2 between steps
            for w, (e0, e1) in ev_pk[k].items():
                s.set_kernel_events(w, e0, e1)
            ev_step[k][0].record(stream)
            step(ev_k[k])
            ev_step[k][1].record(stream)
        torch.cuda.synchronize(dev)
        for w in (sph.KEV_DENSITY, sph.KEV_FORCE):
            s.set_kernel_events(w, None, None)
        pk_ms = {nm: [ev_pk[k][w][0].elapsed_time(ev_pk[k][w][1]) for k in range(K)]
                 for nm, w in (("density", sph.KEV_DENSITY), ("force", sph.KEV_FORCE))}
        if world > 1:
            dist.barrier()
        st = s.stats()
        launches = st["launches"] - launches0
        step_ms = [a.elapsed_time(b) for a, b in ev_step]
        step_ms_eager = step_ms
        kern_ms = {nm: [ev_k[k][i][0].elapsed_time(ev_k[k][i][1]) for k in range(K)] for i, nm in enumerate(names)}
        if not args.no_graph:
            # the same step captured once as a CUDA graph and replayed K times
            # (L2 flushed between replays): the timed steps of the result
            l0 = s.stats()["launches"]
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                step()
            per_step = s.stats()["launches"] - l0
            s.reset_stats()
            ev_g = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize(dev)
            for k in range(K):
                flush.fill_(k & 0xFF)
                ev_g[k][0].record(stream)
                g.replay()
                ev_g[k][1].record(stream)
            torch.cuda.synchronize(dev)
            if world > 1:
                dist.barrier()
            st = s.stats()
            launches = per_step * K
            step_ms = [a.elapsed_time(b) for a, b in ev_g]
            del g
        clk = clocks.stop()

    total_s = sum(step_ms) / 1e3
    pairs = st["pairs_density"] + st["pairs_force"]
    if st["error_bits"] & (sph.ERR_NONFINITE | sph.ERR_OUTSIDE):
        raise RuntimeError(f"device error bits {st['error_bits']}")

    # e2e: the same step through the C ABI with the AoS in pinned host memory,
    # host->device and device->host copies inside the timed region
    e2e = None
    if not args.no_e2e:
        host = torch.empty_like(aos_host).pin_memory()
        with torch.cuda.stream(stream):
            sph.sph_aos_download(s.ctx, host.data_ptr(), n * 112)
            s.reset_stats()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            e2e_ms = 0.0

            def upload_and_step():
                sph._check(sph.sph_aos_upload(s.ctx, host.data_ptr(), n * 112), "upload")
                step()

            run = upload_and_step
            if not args.no_graph:
                # the upload and the step as one graph, as the headline (the
                # download synchronises, so it stays a call of its own)
                ge = torch.cuda.CUDAGraph()
                with torch.cuda.graph(ge, stream=stream):
                    upload_and_step()
                run = ge.replay
                s.reset_stats()
            for k in range(max(1, K // 2)):
                flush.fill_(k & 0xFF)
                t0.record(stream)
                run()
                sph._check(sph.sph_aos_download(s.ctx, host.data_ptr(), n * 112), "download")
                t1.record(stream)
                t1.synchronize()
                e2e_ms += t0.elapsed_time(t1)
            st2 = s.stats()
        e2e = {"value": (st2["pairs_density"] + st2["pairs_force"]) / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": n * 112, "d2h_bytes_per_step": n * 112,
               "steps": max(1, K // 2), "ms_per_step": e2e_ms / max(1, K // 2)}

    dens_pairs_per_launch = st["pairs_density"] / K
    force_pairs_per_launch = st["pairs_force"] / K
    t_den = statistics.mean(pk_ms["density"]) / 1e3          # k_density launches alone
    t_for = statistics.mean(pk_ms["force"]) / 1e3
    dominant = "density" if t_den >= t_for else "force"
    t_dom = t_den if dominant == "density" else t_for
    flops = (dens_pairs_per_launch if dominant == "density" else force_pairs_per_launch) * FLOPS_PER_PAIR[dominant]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp32_peak_tflops(sms, clk.get("sm_max_mhz") or 2070.0)
    achieved = flops / t_dom / 1e12
    kernel_src = [os.path.join(ROOT, "paper_2512_05516_gb300", "csrc", f) for f in ("k_pairs.cu", "k_pair_math.cuh")]
    roofline = {"bound": "alu", "kernel": f"k_{dominant}", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic_from_profile(kernel_src, f"k_{dominant}"),
                "peak_basis": "FP32 FMA pipe: SMs x 128 lanes x 2 flops x max SM clock",
                "flops_per_pair": FLOPS_PER_PAIR[dominant]}
    hbm = 6753.1
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        pass
    pb = PREC_BYTES[args.prec]
    bytes_pp = algorithmic_bytes(pb, 4)
    kernels = {}
    for nm in names:
        ms = statistics.mean(kern_ms[nm])
        row = {"ms": ms}
        if nm in bytes_pp:
            gbs = bytes_pp[nm] * n / (ms / 1e3) / 1e9
            row.update({"algorithmic_bytes_per_particle": bytes_pp[nm], "GB_s": gbs,
                        "frac_of_measured_hbm": gbs / hbm, "frac_of_nominal_hbm": gbs / HBM_NOMINAL_GBS})
        kernels[nm] = row
    kernels["density"]["pairs"] = dens_pairs_per_launch
    kernels["force"]["pairs"] = force_pairs_per_launch
    kernels["density"]["pair_kernel_ms"] = statistics.mean(pk_ms["density"])   # without the pack pass
    kernels["force"]["pair_kernel_ms"] = statistics.mean(pk_ms["force"])
    kernels["density"]["tests"] = st["tests_density"] / K
    kernels["force"]["tests"] = st["tests_force"] / K
    s.close()
    return {"total_s": total_s, "pairs": pairs, "step_ms": step_ms, "step_ms_eager": step_ms_eager,
            "clocks": clk, "e2e": e2e,
            "roofline": roofline, "kernels": kernels, "launches": launches, "n": n,
            "tuning": tuned["tuning"], "tuning_source": ("default" if tuned["cached"] is None else
                                                         "autotuner cache" if tuned["cached"] else "autotuner search")}


# ----------------------------------------------------------------- long run (HBM-bound rows)
PREC_BYTES = {"fp32": 4, "bf16": 2, "fp16": 2, "m16": 25 / 8, "m10": 19 / 8}
HBM_NOMINAL_GBS = 8000.0          # GB300 HBM3e, nominal (the measured copy peak is the other denominator)


def algorithmic_bytes(prec_bytes: float, pos_bytes: float):
    """Minimum bytes per particle of the memory-bound calls (112-byte FP64
    record; v, m, h, u stored in `prec_bytes`, positions in `pos_bytes`;
    a, du/dt, rho, P FP32; 4-byte permutation and 4-byte key per slot).
      aos_to_soa            read x, v, m, h, u (72 B) + perm, key; write the SoA
      kick_drift            read x (AoS), v, a, u, du/dt, perm; write x, v, u
      soa_to_aos            read v, a, h, rho, u, P, perm; write them (80 B)
      kick_drift_writeback  read x, v, a, u, du/dt, h, rho, P, perm; write x,
                            v, a, h, rho, u, P (104 B) to the AoS"""
    p = prec_bytes
    conv = (72 + 8) + 3 * pos_bytes + 3 * p + 3 * p
    kick = (24 + 3 * p + 12 + p + 4 + 4) + (24 + 3 * p + p)
    back = (3 * p + 12 + p + 4 + p + 4 + 4) + 80
    fused = (24 + 3 * p + 12 + p + 4 + p + 4 + 4 + 4) + 104
    return {"aos_to_soa": conv, "kick_drift": kick, "soa_to_aos": back, "kick_drift_writeback": fused}


def run_long_run(steps: int = 3, graph_steps: int = 100):
    """Memory-bound rows on the 33,554,432-particle long-run lattice (box
    2x1x1, FP64 AoS master, FP16 storage of x, v, m, h, u): per-call CUDA-event
    times of the conversion, kick/drift and write-back kernels against the
    HBM peak, and 100 whole steps captured in one CUDA graph and replayed."""
    import torch
    import paper_2512_05516_gb300 as sph
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    wl = sph_inputs.long_run()
    n = wl.n
    stream = torch.cuda.Stream(dev)
    aos = torch.from_numpy(wl.aos).to(dev)
    del wl.aos
    nc = [int(math.floor(b / max(wl.cell_edge, 2 * wl.h_cap))) for b in wl.box]
    params = sph.make_params(wl.box, gamma=wl.gamma, alpha=wl.alpha_av, beta=wl.beta_av,
                             eps=wl.eps_av, eta=wl.eta, h_max=wl.h_cap)
    s = sph.Sph(aos, sph.layout_112(), params, int(np.prod(nc)), sph.WS_REORDER, stream=stream)
    prec = {"x": "fp16", "v": "fp16", "m": "fp16", "h": "fp16", "u": "fp16"}
    from paper_2512_05516_gb300 import autotune
    with torch.cuda.stream(stream):
        tuned = autotune.tune(s, wl.cell_edge, prec, 0)
    names = ["bin", "aos_to_soa", "density", "force", "kick_drift_writeback"]
    calls = [lambda: s.bin_cells(wl.cell_edge, drift_keys=True), lambda: s.aos_to_soa(sph.FIELDS_FORCE, prec),
             lambda: s.density(0), lambda: s.force(),
             lambda: s.kick_drift_writeback(wl.dt, wl.dt, sph.FIELDS_OUTPUT)]
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in names]
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        # warm-up step; its binning also sorts the AoS records into cell order
        # once, so later steps see an almost sequential permutation
        s.bin_cells(wl.cell_edge, reorder=True)
        for fn in calls[1:]:
            fn()
        for k in range(steps):
            for i, fn in enumerate(calls):
                ev[k][i][0].record(stream)
                fn()
                ev[k][i][1].record(stream)
        stream.synchronize()
        ms = {nm: statistics.mean(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(steps))
              for i, nm in enumerate(names)}
        # S6 and S7 as separate calls (kick/drift alone, then the write-back),
        # timed at the same distance from the reorder as the rows above
        sep = ["kick_drift", "soa_to_aos"]
        ev_sep = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in sep]
                  for _ in range(steps)]
        for k in range(steps):
            for fn in calls[:4]:
                fn()
            for i, fn in enumerate([lambda: s.kick_drift(wl.dt, wl.dt), lambda: s.soa_to_aos(sph.FIELDS_OUTPUT)]):
                ev_sep[k][i][0].record(stream)
                fn()
                ev_sep[k][i][1].record(stream)
        stream.synchronize()
        for i, nm in enumerate(sep):
            ms[nm] = statistics.mean(ev_sep[k][i][0].elapsed_time(ev_sep[k][i][1]) for k in range(steps))
        # whole steps as one CUDA graph
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(graph_steps):
                for fn in calls:
                    fn()
        s.reset_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        e1.synchronize()
        graph_ms = e0.elapsed_time(e1) / graph_steps
    st = s.stats()
    if st["error_bits"] & (sph.ERR_NONFINITE | sph.ERR_OUTSIDE):
        raise RuntimeError(f"long run: device error bits {st['error_bits']}")
    pairs = (st["pairs_density"] + st["pairs_force"]) / graph_steps
    # the comparison: an FP32 SoA kept across steps needs no conversion or
    # write-back; its step is binning + density + force + kick/drift on FP32
    # storage (timed per call; the FP32 conversion that refreshes the SoA
    # here between those calls is not counted)
    names32 = ["bin", "density", "force", "kick_drift"]
    ev32 = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in names32]
            for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps + 1):
            for i, fn in enumerate([lambda: s.bin_cells(wl.cell_edge, drift_keys=True), None, lambda: s.density(0),
                                    lambda: s.force(), lambda: s.kick_drift(wl.dt, wl.dt)]):
                if fn is None:
                    s.aos_to_soa(sph.FIELDS_FORCE)          # FP32, untimed
                    continue
                j = i if i == 0 else i - 1
                if k > 0:
                    ev32[k - 1][j][0].record(stream)
                fn()
                if k > 0:
                    ev32[k - 1][j][1].record(stream)
            s.soa_to_aos(sph.FIELDS_OUTPUT)                  # keeps the AoS state current, untimed
        stream.synchronize()
    ms32 = {nm: statistics.mean(ev32[k][i][0].elapsed_time(ev32[k][i][1]) for k in range(steps))
            for i, nm in enumerate(names32)}
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6753.1
    bpp = algorithmic_bytes(2, 2)
    kern = {}
    for nm in names + sep:
        row = {"ms": ms[nm]}
        if nm in bpp:
            gbs = bpp[nm] * n / (ms[nm] / 1e3) / 1e9
            row.update({"algorithmic_bytes_per_particle": bpp[nm], "GB_s": gbs,
                        "frac_of_measured_hbm": gbs / hbm, "frac_of_nominal_hbm": gbs / HBM_NOMINAL_GBS})
        kern[nm] = row
    s.close()
    del aos
    torch.cuda.empty_cache()
    fp16_step = sum(ms[nm] for nm in names)
    fp32_step = sum(ms32.values())
    return {"workload": "long_run_33554432", "particles": n, "storage": "fp16 (x, v, m, h, u)",
            "tuning": tuned["tuning"],
            "ms_per_step_graph": graph_ms, "graph_steps": graph_steps, "pairs_per_s": pairs / (graph_ms / 1e3),
            "kernels": kern, "hbm_peak_gbs": hbm,
            "vs_fp32_soa": {"fp16_with_conversion_ms": fp16_step,
                            "fp32_soa_no_conversion_ms": fp32_step,
                            "fp32_kernels_ms": ms32, "speedup": fp32_step / fp16_step}}


def run_vs_plain(lattice: int = 124, steps: int = 3):
    """The reduced-precision batched step against the plain FP32 SoA step on
    the same Sod set: bin, convert, density (5 Newton steps), force,
    kick/drift + write-back.  Reduced: v, m, h, u stored in FP16 under
    power-of-two storage scales, batched kernels with the autotuner's shapes.
    Plain: FP32 storage, one thread per particle over the 27 neighbour
    cells."""
    import torch
    import paper_2512_05516_gb300 as sph
    from paper_2512_05516_gb300 import autotune
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    wl = sph_inputs.sod(n_lattice=lattice)
    stream = torch.cuda.Stream(dev)
    nc = [int(math.floor(b / max(wl.cell_edge, 2 * wl.h_cap))) for b in wl.box]
    params = sph.make_params(wl.box, gamma=wl.gamma, alpha=wl.alpha_av, beta=wl.beta_av,
                             eps=wl.eps_av, eta=wl.eta, h_max=wl.h_cap)
    rows = {}
    for name in ("plain_fp32", "batched_fp16_scaled"):
        aos = torch.from_numpy(wl.aos.copy()).to(dev)
        s = sph.Sph(aos, sph.layout_112(), params, int(np.prod(nc)), 0, stream=stream)
        prec = None
        with torch.cuda.stream(stream):
            if name == "plain_fp32":
                s.set_tuning(pair_kernel=1)
            else:
                prec = {"v": "fp16", "m": "fp16", "h": "fp16", "u": "fp16"}
                s.set_scale({f: sph.suggest_scale(float(np.abs(wl.col(f)).max()), "fp16") for f in ("v", "m", "h", "u")})
                autotune.tune(s, wl.cell_edge, prec, wl.newton_steps)
            s.step(wl.dt, wl.newton_steps, prec=prec, cell_edge=wl.cell_edge)
            s.reset_stats()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                s.step(wl.dt, wl.newton_steps, prec=prec, cell_edge=wl.cell_edge)
            e1.record(stream)
            e1.synchronize()
        st = s.stats()
        ms = e0.elapsed_time(e1) / steps
        rows[name] = {"ms_per_step": ms,
                      "pairs_per_s": (st["pairs_density"] + st["pairs_force"]) / steps / (ms / 1e3),
                      "tests_per_pair": (st["tests_density"] + st["tests_force"]) /
                      max(1, st["pairs_density"] + st["pairs_force"])}
        s.close()
        del aos
    rows["speedup"] = rows["plain_fp32"]["ms_per_step"] / rows["batched_fp16_scaled"]["ms_per_step"]
    rows["workload"] = f"sod_{wl.n}"
    rows["density_error_note"] = ("FP16 storage under power-of-two scales: density relative RMSE "
                                  "3.1e-4, max 4.5e-4 against FP64 after one step (tests/precision_report.py)")
    return rows


def run_streaming(steps: int = 5):
    """The paper's two GPU variants (Section 6.3) on the Sod set, FP32
    storage, default launch shapes: in-place (the AoS master in device
    memory) against streaming (the same records in pinned host memory,
    which the binning, conversion and kick/drift + write-back kernels read
    and write over the host link; nothing is staged by copies)."""
    import torch
    import paper_2512_05516_gb300 as sph
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    wl = sph_inputs.sod()
    stream = torch.cuda.Stream(dev)
    nc = [int(math.floor(b / max(wl.cell_edge, 2 * wl.h_cap))) for b in wl.box]
    params = sph.make_params(wl.box, gamma=wl.gamma, alpha=wl.alpha_av, beta=wl.beta_av,
                             eps=wl.eps_av, eta=wl.eta, h_max=wl.h_cap)
    names = ["bin", "aos_to_soa", "density", "force", "kick_drift_writeback"]
    rows = {}
    for where in ("in_place", "streaming"):
        t = torch.from_numpy(wl.aos.copy())
        aos = t.to(dev) if where == "in_place" else t.pin_memory()
        s = sph.Sph(aos, sph.layout_112(), params, int(np.prod(nc)), 0, stream=stream)
        calls = [lambda: s.bin_cells(wl.cell_edge, drift_keys=True), lambda: s.aos_to_soa(sph.FIELDS_FORCE),
                 lambda: s.density(wl.newton_steps), lambda: s.force(),
                 lambda: s.kick_drift_writeback(wl.dt, wl.dt, sph.FIELDS_OUTPUT)]
        ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in names]
              for _ in range(steps)]
        with torch.cuda.stream(stream):
            for fn in calls:
                fn()
            for k in range(steps):
                for i, fn in enumerate(calls):
                    ev[k][i][0].record(stream)
                    fn()
                    ev[k][i][1].record(stream)
            stream.synchronize()
        ms = {nm: statistics.mean(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(steps))
              for i, nm in enumerate(names)}
        rows[where] = {"ms_per_step": sum(ms.values()), "kernels_ms": ms}
        s.close()
        del aos
    rows["streaming_over_in_place"] = rows["streaming"]["ms_per_step"] / rows["in_place"]["ms_per_step"]
    rows["workload"] = f"sod_{wl.n}"
    return rows


def _records_144(wl, seed: int = 9):
    """The paper's 144-byte benchmark record (ID, FP64 x, FP32 fields) for a
    workload, with random accelerations and du/dt for the kick."""
    import paper_2512_05516_gb300 as sph
    offs = {k: v for k, v in sph.RECORD_144.items() if k not in ("cs", "dudt")}
    raw = sph_inputs.pack_records(wl, offs, 144, f32_fields=sph.F32_144)
    raw[:, 0:8] = np.arange(wl.n, dtype=np.int64).view(np.uint8).reshape(-1, 8)
    raw[:, 76:80] = 0
    rng = np.random.Generator(np.random.PCG64(seed))
    raw[:, 44:56] = rng.uniform(-1, 1, (wl.n, 3)).astype(np.float32).view(np.uint8).reshape(-1, 12)
    raw[:, 80:84] = rng.uniform(-1, 1, wl.n).astype(np.float32).view(np.uint8).reshape(-1, 4)
    return raw


def run_buffers(nb=(64, 64, 32), reps: int = 5):
    """The paper's benchmark shape (Section 6, Fig. 2): 4x4x4 lattice blocks,
    each a contiguous buffer of 64 records in the paper's 144-byte record;
    density and force over every pair of a buffer, kick and drift per
    particle.  Each kernel reads the records directly (AoS) or the converted
    SoA (FP32, and 16-bit: v, m, h, u in FP16 under power-of-two scales,
    positions FP32 offsets); the pair kernels in two forms, partners staged
    in shared memory (the default) and read from global memory (the
    structure of the paper's kernels).  CUDA-event mean over `reps` calls
    after one warm-up, inputs larger than L2.  Also the conversion and
    write-back that the SoA variants need around the kernels, for a whole
    step."""
    import torch
    import paper_2512_05516_gb300 as sph
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    wl = sph_inputs.buffer_blocks(nb=nb)
    B = wl.meta["B"]
    raw = _records_144(wl)
    stream = torch.cuda.Stream(dev)
    nc = [int(math.floor(b / (2 * wl.h_cap))) for b in wl.box]
    params = sph.make_params(wl.box, gamma=wl.gamma, alpha=wl.alpha_av, beta=wl.beta_av,
                             eps=wl.eps_av, eta=wl.eta, h_max=wl.h_cap)
    aos = torch.from_numpy(raw.reshape(-1)).to(dev)
    del raw
    s = sph.Sph(aos, sph.layout_144(), params, max(int(np.prod(nc)), 27), 0, stream=stream)
    s.bin_buffers(B)
    col = lambda name: wl.col(name)
    scale16 = {k: sph.suggest_scale(float(np.abs(col(k)).max()), "fp16") for k in ("v", "m", "h", "u")}

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    kernels = ["density", "force", "kick", "drift"]
    calls = {"density": lambda src: s.buffer_density(src), "force": lambda src: s.buffer_force(src),
             "kick": lambda src: s.buffer_kick(1e-6, src), "drift": lambda src: s.buffer_drift(1e-6, src)}
    inputs = sph.mask("x", "v", "a", "m", "h", "u", "dudt")
    outputs = sph.mask("x", "v", "a", "rho", "P", "cs", "u", "dudt")
    rows = {}
    with torch.cuda.stream(stream):
        s.reset_stats()
        s.buffer_density("aos")
        s.buffer_force("aos")
        st = s.stats()
        rows["aos"] = {k: timed(lambda k=k: calls[k]("aos")) for k in kernels}
        s.set_tuning(pair_kernel=1)
        rows["aos"].update({k + "_plain": timed(lambda k=k: calls[k]("aos")) for k in ("density", "force")})
        s.set_tuning(pair_kernel=0)
        for name, prec, scale in (("soa_fp32", None, {}),
                                  ("soa_16bit", {"v": "fp16", "m": "fp16", "h": "fp16", "u": "fp16"}, scale16)):
            s.set_scale(scale)
            conv = timed(lambda: s.aos_to_soa(inputs, prec))
            r = {k: timed(lambda k=k: calls[k]("soa")) for k in kernels}
            s.set_tuning(pair_kernel=1)
            r.update({k + "_plain": timed(lambda k=k: calls[k]("soa")) for k in ("density", "force")})
            s.set_tuning(pair_kernel=0)
            r["aos_to_soa"] = conv
            r["soa_to_aos"] = timed(lambda: s.soa_to_aos(outputs))
            rows[name] = r
        s.set_scale({})
    out = {"workload": f"buffer_blocks_{wl.n}", "buffer": B, "record_bytes": 144, "n": wl.n,
           "pairs_per_step": {"density": st["pairs_density"], "force": st["pairs_force"]},
           "ms": rows, "soa_16bit_scales": scale16}
    speed = {}
    for name in ("soa_fp32", "soa_16bit"):
        speed[name] = {k: rows["aos"][k] / rows[name][k] for k in kernels + ["density_plain", "force_plain"]}
        step_aos = sum(rows["aos"][k] for k in kernels)
        step_soa = sum(rows[name][k] for k in kernels) + rows[name]["aos_to_soa"] + rows[name]["soa_to_aos"]
        speed[name]["step_with_conversions"] = step_aos / step_soa
        # the paper's kernel structure (partners read from global memory): its
        # end-to-end in-place comparison (conversions included) against the
        # AoS baseline
        plain_aos = rows["aos"]["density_plain"] + rows["aos"]["force_plain"] + rows["aos"]["kick"] + rows["aos"]["drift"]
        plain_soa = (rows[name]["density_plain"] + rows[name]["force_plain"] + rows[name]["kick"] + rows[name]["drift"]
                     + rows[name]["aos_to_soa"] + rows[name]["soa_to_aos"])
        speed[name]["plain_step_with_conversions"] = plain_aos / plain_soa
    out["soa_speedup_over_aos"] = speed
    out["pairs_per_s"] = {src: {"density": st["pairs_density"] / (rows[src]["density"] * 1e-3),
                                "force": st["pairs_force"] / (rows[src]["force"] * 1e-3)}
                          for src in ("aos", "soa_fp32", "soa_16bit")}
    s.close()
    return out


def run_placement(reps: int = 5):
    """Where the conversion runs (Section 6.3, Fig. 1): the Sod records in
    pinned host memory end up as SoA in device memory either by moving the
    AoS and converting on the GPU (one upload, then sph_aos_to_soa), or by
    converting on the host cores and moving the narrowed SoA
    (sph_aos_to_soa_host: the permutation comes down, the SoA goes up), or by
    GPU kernels reading the host records in place (no copy).  Per kernel's
    field set (density, force, kick, drift, full record) in 32-bit storage
    and in 16-bit storage (FP16 under power-of-two scales; a stays FP32).
    Times: CUDA events for the GPU placements, the host clock around the
    synchronised host call for the CPU one; mean over `reps` after a
    warm-up."""
    import torch
    import paper_2512_05516_gb300 as sph
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    wl = sph_inputs.sod()
    n = wl.n
    stream = torch.cuda.Stream(dev)
    nc = [int(math.floor(b / max(wl.cell_edge, 2 * wl.h_cap))) for b in wl.box]
    params = sph.make_params(wl.box, gamma=wl.gamma, alpha=wl.alpha_av, beta=wl.beta_av,
                             eps=wl.eps_av, eta=wl.eta, h_max=wl.h_cap)
    host = torch.from_numpy(np.ascontiguousarray(wl.aos)).pin_memory()
    s = sph.Sph(host.to(dev), sph.layout_112(), params, int(np.prod(nc)), 0, stream=stream)
    sh = sph.Sph(host, sph.layout_112(), params, int(np.prod(nc)), 0, stream=stream)   # kernels on host records
    sets = {"density": sph.FIELDS_DENSITY, "force": sph.FIELDS_FORCE, "kick": sph.mask("v", "a", "u"),
            "drift": sph.mask("x", "v"), "full": sph.mask("x", "v", "a", "m", "h", "rho", "u", "P")}
    half = {"x": "fp16", "v": "fp16", "m": "fp16", "h": "fp16", "u": "fp16", "rho": "fp16", "P": "fp16"}
    scale16 = {k: sph.suggest_scale(float(np.abs(wl.col(k)).max()), "fp16") for k in ("v", "m", "h", "u", "rho", "P")}
    cores = os.cpu_count() or 1

    def ev_time(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        stream.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def wall_time(fn):
        fn()
        stream.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
            stream.synchronize()
        return (time.perf_counter() - t0) / reps * 1e3

    rows = {}
    with torch.cuda.stream(stream):
        for ctx in (s, sh):
            ctx.bin_cells(wl.cell_edge)
        for bits, prec, scale in (("32", None, {}), ("16", half, scale16)):
            for ctx in (s, sh):
                ctx.set_scale(scale)
            for name, fields in sets.items():
                pr = None if prec is None else {k: v for k, v in prec.items() if fields & sph.mask(k)}
                gpu = ev_time(lambda: (sph._check(sph.sph_aos_upload(s.ctx, host.data_ptr(), n * 112), "upload"),
                                       s.aos_to_soa(fields, pr)))
                in_place = ev_time(lambda: sh.aos_to_soa(fields, pr))
                cpu = wall_time(lambda: s.aos_to_soa_host(host, fields, pr))
                rows[f"{name}_{bits}bit"] = {"gpu_move_then_convert_ms": gpu, "gpu_kernels_on_host_records_ms": in_place,
                                            "cpu_convert_then_move_ms": cpu, "gpu_speedup_over_cpu": cpu / gpu}
            # the way back (C^T N^T U^T): the step's outputs to the host records
            out = sph.FIELDS_OUTPUT
            pr = None if prec is None else {k: v for k, v in prec.items() if out & sph.mask(k)}
            s.aos_to_soa(out, pr)
            back = host.clone().pin_memory()
            gpu = ev_time(lambda: (s.soa_to_aos(out),
                                   sph._check(sph.sph_aos_download(s.ctx, back.data_ptr(), n * 112), "download")))
            cpu = wall_time(lambda: s.soa_to_aos_host(back, out))
            rows[f"write_back_{bits}bit"] = {"gpu_convert_then_move_ms": gpu, "cpu_move_then_convert_ms": cpu,
                                             "gpu_speedup_over_cpu": cpu / gpu}
        for ctx in (s, sh):
            ctx.set_scale({})
    s.close()
    sh.close()
    return {"workload": f"sod_{n}", "host_threads": cores, "rows": rows,
            "note": "paper, Fig. 1 (other hardware, context): GPU conversion up to 35x faster than the CPU's "
                    "in 32-bit and up to 500x in 16-bit on GH200 and MI300A"}


def run_uneven(n: int = 16_777_216):
    """Uneven occupancy (the clustered Gaussian mixture, one global h, up to
    ~65,000 particles in a cell), BF16 storage of v, m, h, u: one density
    (fixed h) and one force call per work-queue variant -- one persistent
    launch over the queue in cell order, the same with the costliest items
    first, and one launch per power-of-two cost class."""
    import torch
    import paper_2512_05516_gb300 as sph
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    wl = sph_inputs.gaussian_mixture(n=n)
    stream = torch.cuda.Stream(dev)
    aos = torch.from_numpy(wl.aos).to(dev)
    nc = [int(math.floor(b / max(wl.cell_edge, 2 * wl.h_cap))) for b in wl.box]
    params = sph.make_params(wl.box, eta=wl.eta, h_max=wl.h_cap)
    s = sph.Sph(aos, sph.layout_112(), params, int(np.prod(nc)), 0, stream=stream)
    prec = {"v": "bf16", "m": "bf16", "h": "bf16", "u": "bf16"}
    rows = []
    with torch.cuda.stream(stream):
        for order, per in [(0, 0), (1, 0), (1, 1)]:
            s.set_tuning(item_order=order, class_launches=per)
            s.bin_cells(wl.cell_edge)
            s.aos_to_soa(sph.FIELDS_FORCE, prec)
            s.density(0)                                  # warm-up
            s.force()
            s.reset_stats()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            s.density(0)
            ev[1].record(stream)
            s.force()
            ev[2].record(stream)
            ev[2].synchronize()
            st = s.stats()
            td, tf = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
            rows.append({"queue": "costliest first" if order else "cell order",
                         "launches": "one per cost class" if per else "one persistent",
                         "density_ms": td, "force_ms": tf,
                         "density_pairs_per_s": st["pairs_density"] / (td / 1e3),
                         "force_pairs_per_s": st["pairs_force"] / (tf / 1e3),
                         "pairs_per_s": (st["pairs_density"] + st["pairs_force"]) / ((td + tf) / 1e3),
                         "max_occupancy": st["max_occupancy"]})
    s.close()
    del aos
    torch.cuda.empty_cache()
    return {"workload": f"gaussian_mixture_{n}", "storage": "bf16 (v, m, h, u)", "h": wl.meta["h"],
            "cells_per_axis": nc[0], "variants": rows}


def _levels_density(sph, wl, dev, stream, margin, reps, force=True):
    """Bin for the hierarchy, convert, and time the density with 5 Newton
    steps and the force over it (reps timed runs after one warm-up; counters
    of the last)."""
    import torch
    lo, hi = wl.meta["levels"]
    aos = torch.from_numpy(wl.aos).to(dev)
    params = sph.make_params(wl.box, eta=wl.eta, h_max=wl.h_cap)
    s = sph.Sph(aos, sph.layout_112(), params, 27, sph.WS_LEVELS, stream=stream)
    ms_bin, ms_den, ms_frc = [], [], []
    with torch.cuda.stream(stream):
        for r in range(reps + 1):
            s.reset_stats()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            s.bin_levels(lo, hi, margin)
            s.aos_to_soa(sph.FIELDS_FORCE)
            ev[1].record(stream)
            s.density_levels(5)
            ev[2].record(stream)
            if force:
                s.force_levels()
            ev[3].record(stream)
            ev[3].synchronize()
            if r:
                ms_bin.append(ev[0].elapsed_time(ev[1]))
                ms_den.append(ev[1].elapsed_time(ev[2]))
                ms_frc.append(ev[2].elapsed_time(ev[3]))
        st = s.stats()
        done, prom = s.level_counts()
        fl = s.density_flags()
        flags = {"newton": int(((fl & sph.PFLAG_NEWTON) != 0).sum().item()),
                 "hcap": int(((fl & sph.PFLAG_HCAP) != 0).sum().item()),
                 "nonfinite": int(((fl & sph.PFLAG_NONFINITE) != 0).sum().item())}
    s.close()
    del aos
    torch.cuda.empty_cache()
    td = statistics.median(ms_den)
    out = {"margin": margin, "bin_and_convert_ms": statistics.median(ms_bin), "density_ms": td,
            "density_pairs_per_s": st["pairs_density"] / (ms_den[-1] / 1e3),
            "tests_per_pair": st["tests_density"] / max(st["pairs_density"], 1),
            "particles_per_level": {str(l): done[l] for l in range(lo, hi + 1)},
            "promoted_per_level": {str(l): prom[l] for l in range(lo, hi + 1)},
            "error_bits": st["error_bits"],
            # particles whose Newton step met f'(h) <= 0 and kept their h (the
            # FP64 oracle flags the same ones: tests/test_gpu_levels.py)
            "particles_flagged": flags}
    if force:
        out.update({"force_ms": statistics.median(ms_frc),
                    "force_pairs_per_s": st["pairs_force"] / (ms_frc[-1] / 1e3),
                    "force_tests_per_pair": st["tests_force"] / max(st["pairs_force"], 1)})
    return out


def run_levels(n: int = 16_777_216, n_compare=(262_144, 1_048_576), reps: int = 3):
    """Per-particle h on the clustered set (h from the mixture's local number
    density, 48 neighbours; 5 Newton steps): the density and the force over
    the level hierarchy at full size for three level margins, and at smaller
    sizes the density next to one grid sized for the largest h (the only grid the
    single-level path can use: its cells hold the whole support of the
    background particles, so the dense cores share a handful of cells)."""
    import torch
    import paper_2512_05516_gb300 as sph
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream(dev)
    wl = sph_inputs.gaussian_mixture_adaptive(n)
    rows = [_levels_density(sph, wl, dev, stream, m, reps) for m in (0.0, 0.1, 0.25)]
    out = {"workload": f"gaussian_mixture_adaptive_{n}", "storage": "fp32", "newton_steps": 5,
           "levels": list(wl.meta["levels"]), "h_range": [wl.meta["h_min"], wl.meta["h_max"]],
           "hierarchy": rows, "vs_single_grid": []}
    del wl
    for nc_ in n_compare:
        w = sph_inputs.gaussian_mixture_adaptive(nc_)
        lv = _levels_density(sph, w, dev, stream, 0.1, 1, force=False)
        aos = torch.from_numpy(w.aos).to(dev)
        nc = int(math.floor(1.0 / (2.0 * w.h_cap)))
        params = sph.make_params(w.box, eta=w.eta, h_max=w.h_cap)
        s = sph.Sph(aos, sph.layout_112(), params, nc ** 3, 0, stream=stream)
        with torch.cuda.stream(stream):
            s.bin_cells(2.0 * w.h_cap)
            s.aos_to_soa(sph.FIELDS_DENSITY)
            s.reset_stats()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            s.density(5)
            ev[1].record(stream)
            ev[1].synchronize()
            st = s.stats()
        s.close()
        del aos
        torch.cuda.empty_cache()
        t1 = ev[0].elapsed_time(ev[1])
        out["vs_single_grid"].append({
            "n": nc_, "levels": list(w.meta["levels"]), "single_grid_cells_per_axis": nc,
            "single_grid_max_occupancy": st["max_occupancy"], "single_grid_density_ms": t1,
            "single_grid_tests_per_pair": st["tests_density"] / max(st["pairs_density"], 1),
            "hierarchy_density_ms": lv["density_ms"], "speedup": t1 / lv["density_ms"]})
    return out


# ----------------------------------------------------------------- oracle
def run_oracle_sample(n_targets: int, seed: int = 1):
    """The FP64 oracle (as it stands) on a sample of the same workload: the
    density with 5 Newton steps, EOS and force of `n_targets` random particles
    (the density of every particle their forces need is evaluated too)."""
    import oracle
    wl = sph_inputs.sod()
    rng = np.random.default_rng(seed)
    targets = np.sort(rng.choice(wl.n, n_targets, replace=False))
    oracle.lib()
    t0 = time.perf_counter()
    x, m = wl.col("x"), wl.col("m")
    d = oracle.density(x, m, wl.col("h"), wl.box, wl.eta, wl.h_cap, wl.newton_steps, targets=targets)
    P, c = oracle.eos(d["rho"], wl.col("u")[targets], wl.gamma)
    # forces among the sampled particles use their own h, rho, P, c
    sub_rho = np.ones(wl.n)
    sub_h = np.array(wl.col("h"))
    sub_P = np.zeros(wl.n)
    sub_c = np.zeros(wl.n)
    sub_rho[targets] = d["rho"]
    sub_h[targets] = d["h"]
    sub_P[targets] = P
    sub_c[targets] = c
    f = oracle.force(x, wl.col("v"), m, sub_h, sub_rho, sub_P, sub_c, wl.box, wl.alpha_av,
                     wl.beta_av, wl.eps_av, targets=targets)
    dt = time.perf_counter() - t0
    # pairs the oracle evaluated: every Newton pass and the final density
    # pass, plus the force pairs
    pairs = float(np.sum(d["pairs_all"]) + np.sum(f["nngb"]))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return pairs, dt, cores


def cpu_baseline():
    n_t = 600000
    pairs, dt, cores = run_oracle_sample(n_t)
    return {"value": pairs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_t} random particles of the 1,072,476-particle Sod step "
                      f"(density with 5 Newton steps + EOS + force), {dt:.1f} s"}


def combine_ranks(total_s: float, pairs: float, e2e_value: float, device: str):
    """Whole-job figures of N independent replicas (the path has no exchange
    step): the slowest rank's timed seconds, the pairs all ranks processed,
    and the sum of the ranks' end-to-end rates.  Every rank calls it."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_s], dtype=torch.float64, device=device)
    p = torch.tensor([pairs, e2e_value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t[0].item()), float(p[0].item()), float(p[1].item())


def profile_buffers():
    """'buffers': 4x4x4 lattice blocks, 2,097,152 particles in 144-byte
    records (302 MB > L2), buffers of 64: density and force from the records
    and from FP32 SoA, staged and plain, then kick and drift from the SoA and
    from the records."""
    import torch
    import paper_2512_05516_gb300 as sph
    wl = sph_inputs.buffer_blocks(nb=(32, 32, 32))
    raw = _records_144(wl)
    nc = [int(math.floor(b / (2 * wl.h_cap))) for b in wl.box]
    params = sph.make_params(wl.box, gamma=wl.gamma, alpha=wl.alpha_av, beta=wl.beta_av,
                             eps=wl.eps_av, eta=wl.eta, h_max=wl.h_cap)
    aos = torch.from_numpy(raw.reshape(-1)).cuda()
    s = sph.Sph(aos, sph.layout_144(), params, max(int(np.prod(nc)), 27), 0)
    s.bin_buffers(wl.meta["B"])
    s.aos_to_soa(sph.mask("x", "v", "a", "m", "h", "u", "dudt"))
    for plain in (0, 1):
        s.set_tuning(pair_kernel=plain)
        for src in ("aos", "soa"):
            s.buffer_density(src)
            s.buffer_force(src)
    for src in ("soa", "aos"):              # an AoS call leaves the SoA copies of its outputs stale
        s.buffer_kick(1e-6, src)
        s.buffer_drift(1e-6, src)
    torch.cuda.synchronize()
    st = s.stats()
    print(json.dumps({"profile_case": "buffers", "n": wl.n, "error_bits": st["error_bits"],
                      "pairs_density": st["pairs_density"], "pairs_force": st["pairs_force"]}))
    if st["error_bits"] & (sph.ERR_NONFINITE | sph.ERR_OUTSIDE):
        raise SystemExit(1)


def profile_levels(n: int = 2_097_152):
    """'levels': the adaptive-h clustered set at n particles (2,097,152 by
    default: AoS 235 MB > L2), levels from the set, margin 0.1: bin, convert,
    the density with 5 Newton steps and the force over the hierarchy, twice."""
    import torch
    import paper_2512_05516_gb300 as sph
    wl = sph_inputs.gaussian_mixture_adaptive(n)
    lo, hi = wl.meta["levels"]
    params = sph.make_params(wl.box, eta=wl.eta, h_max=wl.h_cap)
    aos = torch.from_numpy(wl.aos).cuda()
    s = sph.Sph(aos, sph.layout_112(), params, 27, sph.WS_LEVELS)
    for _ in range(2):
        s.bin_levels(lo, hi, 0.1)
        s.aos_to_soa(sph.FIELDS_FORCE)
        s.density_levels(5)
        s.force_levels()
    torch.cuda.synchronize()
    st = s.stats()
    done, prom = s.level_counts()
    print(json.dumps({"profile_case": "levels", "n": wl.n, "levels": [lo, hi], "error_bits": st["error_bits"],
                      "pairs_density": st["pairs_density"], "pairs_force": st["pairs_force"],
                      "done": done[lo:hi + 1],
                      "promoted": prom[lo:hi + 1]}))
    if st["error_bits"] & (sph.ERR_NONFINITE | sph.ERR_OUTSIDE):
        raise SystemExit(1)


def profile_case(which: str, n_levels: int = 2_097_152):
    """Small fixed workloads for ncu captures (profiles/ summaries name the
    command).  'pairs': the 1,072,476-particle Sod step twice (the second is
    the one to capture), default launch shapes.  'memory': the long-run
    lattice at 256 x 128 x 128 (4,194,304 particles, AoS 470 MB > L2), FP16
    storage, cell-ordered records; step 1 with separate kick/drift and
    write-back, step 2 with the fused call."""
    import torch
    import paper_2512_05516_gb300 as sph
    if which == "buffers":
        profile_buffers()
        return
    if which == "levels":
        profile_levels(n_levels)
        return
    if which == "pairs":
        wl = sph_inputs.sod()
        prec, ws, steps = None, 0, 2
    else:
        wl = sph_inputs.long_run(nx=256, ny=128, nz=128)
        prec, ws, steps = {"x": "fp16", "v": "fp16", "m": "fp16", "h": "fp16", "u": "fp16"}, sph.WS_REORDER, 2
    aos = torch.from_numpy(wl.aos).cuda()
    nc = [int(math.floor(b / max(wl.cell_edge, 2 * wl.h_cap))) for b in wl.box]
    params = sph.make_params(wl.box, gamma=wl.gamma, alpha=wl.alpha_av, beta=wl.beta_av,
                             eps=wl.eps_av, eta=wl.eta, h_max=wl.h_cap)
    s = sph.Sph(aos, sph.layout_112(), params, int(np.prod(nc)), ws)
    ns = wl.newton_steps if which == "pairs" else 0
    for k in range(steps):
        s.bin_cells(wl.cell_edge, reorder=(which == "memory" and k == 0))
        s.aos_to_soa(sph.FIELDS_FORCE, prec)
        s.density(ns)
        s.force()
        if which == "memory" and k == 0:
            s.kick_drift(wl.dt, wl.dt)
            s.soa_to_aos(sph.FIELDS_OUTPUT)
        else:
            s.kick_drift_writeback(wl.dt, wl.dt, sph.FIELDS_OUTPUT)
    torch.cuda.synchronize()
    st = s.stats()
    print(json.dumps({"profile_case": which, "n": wl.n, "error_bits": st["error_bits"],
                      "tuning": s.tuning()}))
    if st["error_bits"] & (sph.ERR_NONFINITE | sph.ERR_OUTSIDE):
        raise SystemExit(1)


def main():
    args = parse()
    if args.profile_case:
        profile_case(args.profile_case, args.profile_n)
        return
    if args.levels_only:
        print(json.dumps({"adaptive_h_levels": run_levels()}))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        if rank != 0:
            return
        n_t = 20000
        times, pairs_l = [], []
        cores = 1
        for _ in range(args.warmup):
            run_oracle_sample(n_t, seed=7)
        for k in range(args.steps):
            p, dt, cores = run_oracle_sample(n_t, seed=100 + k)
            times.append(dt)
            pairs_l.append(p)
        value = sum(pairs_l) / sum(times)
        sample = (f"{n_t} random particles per step of the 1,072,476-particle Sod step "
                  "(density with 5 Newton steps + EOS + force)")
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "sod_1072476", "sample_particles_per_step": n_t},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    r = run_ours(args, rank, world)

    total_s, pairs = r["total_s"], r["pairs"]
    if world > 1:
        e2e_in = r["e2e"]["value"] if r["e2e"] else 0.0
        total_s, pairs, e2e_v = combine_ranks(total_s, pairs, e2e_in, "cuda")
        if r["e2e"]:
            r["e2e"]["value"] = e2e_v
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline()
    long = None if args.no_long_run or world > 1 else run_long_run()
    uneven = None if args.no_uneven or world > 1 else run_uneven()
    vs_plain = None if args.no_vs_plain or world > 1 else run_vs_plain()
    streaming = None if args.no_streaming or world > 1 else run_streaming()
    buffers = None if args.no_buffers or world > 1 else run_buffers()
    placement = None if args.no_placement or world > 1 else run_placement()
    levels = None if args.no_levels or world > 1 else run_levels()
    out = {
        "metric": METRIC, "value": pairs / total_s, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "sod_1072476" if args.lattice == 124 else f"sod_lattice{args.lattice}",
                   "particles_per_gpu": r["n"], "newton_steps": 5, "storage": args.prec,
                   "aos_record_bytes": 112, "parallelism": f"replicas{world}",
                   "l2": "flushed between steps (512 MiB write)",
                   "timed": "one captured CUDA graph of the step, replayed" if not args.no_graph else "eager calls",
                   "ms_per_step_eager": statistics.mean(r["step_ms_eager"]),
                   "tuning": r["tuning"], "tuning_source": r["tuning_source"]},
        "roofline": r["roofline"], "cpu_baseline": cpu, "e2e": r["e2e"],
        "gpu_launches": r["launches"], "clocks": r["clocks"], "kernels": r["kernels"],
        "memory_bound_rows": long, "uneven_batching": uneven, "vs_plain_fp32_soa": vs_plain,
        "streaming_vs_in_place": streaming,
        "buffers_aos_vs_soa": buffers,
        "conversion_placement": placement,
        "adaptive_h_levels": levels,
    }
    print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
