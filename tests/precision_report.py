"""Storage-precision report: the error every storage format leaves in the
step's results, against the FP64 oracle without quantisation (mode T), after
1 step and after 100 steps (the paper's Section 7 error study: relative RMSE,
i.e. RMSE over the mean magnitude of the quantity, per field).

Formats: v, m, h, u stored in FP32 (the plain SoA baseline), BF16, FP16,
FP16 under a power-of-two storage scale, FP32-m16 and FP32-m10 (truncated
mantissas, packed), each with positions stored as FP32 or FP16 cell offsets.
The kernels compute in FP32 whatever the storage.

Workloads: the 1,072,476-particle Sod tube (1 and 100 steps), the
8,388,608-particle Sedov blast (1 step) and the 1,048,576-particle Sedov
blast (100 steps).  1-step errors use the oracle on sampled targets (every
particle within reach of a target is evaluated); 100-step errors use the
oracle trajectories that tests/golden/make_trajectories.py stores.  Beyond
the first step the trajectories diverge chaotically: those errors are
reported, not gated.  Step times are CUDA-event means over 10 steps without
L2 flushing (indicative; bench.py times the benchmark).

With --sweep: the truncated family at every width instead, v, m, h, u stored
with 23 down to 1 mantissa bits (32 down to 10 total bits), one Sod step.

With --oracle-sweep (CPU only, no GPU): the paper's own study on the FP64
oracle, one force call in FP64 arithmetic over inputs stored in 64 down to 10
total bits of Table 2's family.

Usage (GPU):  python tests/precision_report.py [--json out.json] [--quick | --sweep]
Usage (CPU):  python tests/precision_report.py --oracle-sweep [--json out.json]
"""
import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import sph_inputs  # noqa: E402

FORMATS = ["fp32", "bf16", "fp16", "fp16s", "m16", "m10"]
POSITIONS = ["fp32", "fp16"]
N_TARGETS = 512


def make(wl, torch, sph):
    aos = torch.from_numpy(np.ascontiguousarray(wl.aos)).cuda()
    nc = [int(math.floor(b / max(wl.cell_edge, 2 * wl.h_cap))) for b in wl.box]
    params = sph.make_params(wl.box, gamma=wl.gamma, alpha=wl.alpha_av, beta=wl.beta_av,
                             eps=wl.eps_av, eta=wl.eta, h_max=wl.h_cap)
    return sph.Sph(aos, sph.layout_112(), params, max(int(np.prod(nc)), 27))


def config(wl, fmt, pos, sph):
    """Per-field storage formats and scales of one report row."""
    base = "fp16" if fmt == "fp16s" else fmt
    prec = {"x": pos, "v": base, "m": base, "h": base, "u": base}
    scale = {}
    if fmt == "fp16s":
        for name in ("v", "m", "h", "u"):
            scale[name] = sph.suggest_scale(float(np.abs(wl.col(name)).max()), "fp16")
    return prec, scale


def errors(got, ref, vector=False):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if vector:
        d = np.linalg.norm(got - ref, axis=1)
        mag = np.mean(np.linalg.norm(ref, axis=1))
    else:
        d = np.abs(got - ref)
        mag = np.mean(np.abs(ref))
    if not np.all(np.isfinite(got)):
        return {"rel_rmse": float("inf"), "max_rel": float("inf")}
    return {"rel_rmse": float(np.sqrt(np.mean(d * d)) / mag), "max_rel": float(d.max() / mag)}


def min_image(dx, box):
    b = np.asarray(box)
    return dx - b * np.round(dx / b)


def run_steps(wl, fmt, pos, nsteps, torch, sph, time_it=False):
    s = make(wl, torch, sph)
    prec, scale = config(wl, fmt, pos, sph)
    s.set_scale(scale)
    for _ in range(nsteps):
        s.step(wl.dt, wl.newton_steps, prec=prec, cell_edge=wl.cell_edge)
    torch.cuda.synchronize()
    out = s.aos.cpu().numpy()
    st = s.stats()
    ms = None
    if time_it:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            s.step(wl.dt, wl.newton_steps, prec=prec, cell_edge=wl.cell_edge)
        e0.record()
        for _ in range(10):
            s.step(wl.dt, wl.newton_steps, prec=prec, cell_edge=wl.cell_edge)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
    s.close()
    return out, st, ms, scale


def one_step_report(wl, torch, sph, time_it):
    rng = np.random.default_rng(11)
    tgt = np.sort(rng.choice(wl.n, N_TARGETS, replace=False))
    t0 = time.time()
    o = oracle.step(wl, targets=tgt)
    t_orc = time.time() - t0
    rows = []
    for pos in POSITIONS:
        for fmt in FORMATS:
            out, st, ms, scale = run_steps(wl, fmt, pos, 1, torch, sph, time_it)
            r = {"workload": wl.name, "n": wl.n, "steps": 1, "storage": fmt, "positions": pos,
                 "scale": scale, "error_bits": st["error_bits"], "ms_per_step": ms,
                 "rho": errors(out[tgt, 11], o["rho"]), "h": errors(out[tgt, 10], o["h"]),
                 "P": errors(out[tgt, 13], o["P"]), "a": errors(out[tgt, 6:9], o["a"], True)}
            rows.append(r)
            print(json.dumps(r), flush=True)
    return rows, t_orc


def sweep_report(wl, torch, sph):
    """The truncated family at every width (the paper's error-against-bits
    study, Section 7 and Table 2): v, m, h, u stored as FP32 with n mantissa
    bits, n = 23 (FP32 itself) down to 1, i.e. 32 down to 10 total bits;
    positions FP32; one step against FP64 on sampled targets."""
    rng = np.random.default_rng(11)
    tgt = np.sort(rng.choice(wl.n, N_TARGETS, replace=False))
    o = oracle.step(wl, targets=tgt)
    rows = []
    for n in range(23, 0, -1):
        fmt = "fp32" if n == 23 else f"m{n}"
        out, st, _, _ = run_steps(wl, fmt, "fp32", 1, torch, sph)
        r = {"workload": wl.name, "n": wl.n, "steps": 1, "storage": fmt, "total_bits": 9 + n,
             "positions": "fp32", "error_bits": st["error_bits"],
             "rho": errors(out[tgt, 11], o["rho"]), "h": errors(out[tgt, 10], o["h"]),
             "P": errors(out[tgt, 13], o["P"]), "a": errors(out[tgt, 6:9], o["a"], True)}
        rows.append(r)
        print(json.dumps(r), flush=True)
    return rows


def oracle_sweep_report():
    """The paper's error-against-bits study (Section 7, Fig. 5) on the FP64
    oracle alone, CPU only: the Sod set at 62,208 particles (the paper's
    ~65,000) with small random velocities, its FP64 density (5 Newton steps)
    and EOS as the state; then one force call in FP64 arithmetic whose inputs
    (x, v, m, h, rho, P, c) are stored in t bits of Table 2's family, for every
    t from 64 down to 10, against the same call on the untruncated inputs.
    Also with the positions kept in FP64 and only the other inputs truncated.
    Error: relative RMSE of the acceleration (RMSE over the mean |a|) and the
    maximum over the mean."""
    wl = sph_inputs.sod(n_lattice=48, seed=sph_inputs.SEED_BASE + 40)
    wl.col("v")[:] = np.random.default_rng(40).uniform(-0.1, 0.1, (wl.n, 3))
    x, v, m, u = wl.col("x"), wl.col("v"), wl.col("m"), wl.col("u")
    d = oracle.density(x, m, wl.col("h"), wl.box, wl.eta, wl.h_cap, wl.newton_steps)
    P, c = oracle.eos(d["rho"], u, wl.gamma)
    inputs = {"x": x, "v": v, "m": m, "h": d["h"], "rho": d["rho"], "P": P, "c": c}

    def force(q):
        return oracle.force(q["x"], q["v"], q["m"], q["h"], q["rho"], q["P"], q["c"], wl.box,
                            wl.alpha_av, wl.beta_av, wl.eps_av)["a"]

    ref = force(inputs)
    rows = []
    for t in range(64, 9, -1):
        tr = {k: oracle.truncate_bits(a, t) for k, a in inputs.items()}
        keep_x = dict(tr, x=x)
        r = {"workload": "sod", "n": wl.n, "total_bits": t,
             "a_all": errors(force(tr), ref, True), "a_x_fp64": errors(force(keep_x), ref, True)}
        rows.append(r)
        print(json.dumps(r), flush=True)
    return rows


def hundred_step_report(name, wl, torch, sph):
    path = os.path.join(ROOT, "tests", "golden", f"trajectory_{name}.npz")
    if not os.path.exists(path):
        print(f"# {path} missing: run tests/golden/make_trajectories.py {name}", flush=True)
        return []
    z = np.load(path)
    assert int(z["n"]) == wl.n and int(z["steps"]) > 1
    tgt = z["targets"]
    rows = []
    for pos in POSITIONS:
        for fmt in FORMATS:
            out, st, _, scale = run_steps(wl, fmt, pos, int(z["steps"]), torch, sph)
            dx = min_image(out[tgt, 0:3] - z["x"], wl.box)
            spacing = float(np.mean(wl.col("m")) ** (1.0 / 3.0))
            r = {"workload": wl.name, "n": wl.n, "steps": int(z["steps"]), "storage": fmt,
                 "positions": pos, "scale": scale, "error_bits": st["error_bits"],
                 "rho": errors(out[tgt, 11], z["rho"]), "h": errors(out[tgt, 10], z["h"]),
                 "P": errors(out[tgt, 13], z["P"]), "u": errors(out[tgt, 12], z["u"]),
                 "v": errors(out[tgt, 3:6], z["v"], True), "a": errors(out[tgt, 6:9], z["a"], True),
                 "x_rms_over_spacing": float(np.sqrt(np.mean(np.sum(dx * dx, axis=1))) / spacing)}
            rows.append(r)
            print(json.dumps(r), flush=True)
    return rows


def table(rows, fields):
    head = "| workload | steps | storage | positions | " + " | ".join(fields) + " | ms/step |"
    sep = "|" + "---|" * (5 + len(fields))
    lines = [head, sep]
    for r in rows:
        cells = []
        for f in fields:
            v = r.get(f)
            cells.append(f"{v:.2e}" if isinstance(v, float) else
                         (f"{v['rel_rmse']:.2e} / {v['max_rel']:.1e}" if v else "-"))
        ms = r.get("ms_per_step")
        lines.append(f"| {r['workload']} {r['n']} | {r['steps']} | {r['storage']} | {r['positions']} | "
                     + " | ".join(cells) + f" | {ms:.3f} |" if ms else
                     f"| {r['workload']} {r['n']} | {r['steps']} | {r['storage']} | {r['positions']} | "
                     + " | ".join(cells) + " | - |")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--json", default=None)
    ap.add_argument("--quick", action="store_true", help="1-step rows only")
    ap.add_argument("--sweep", action="store_true",
                    help="only the truncated-mantissa sweep (32 down to 10 total bits) on the Sod set")
    ap.add_argument("--oracle-sweep", action="store_true",
                    help="CPU only: the FP64 oracle's force error against total storage bits "
                         "(64 down to 10, Table 2's family)")
    args = ap.parse_args()
    if args.oracle_sweep:
        rows = oracle_sweep_report()
        print()
        print("| total bits | layout | a: all inputs truncated | a: positions kept in FP64 |")
        print("|---|---|---|---|")
        for r in rows:
            t = r["total_bits"]
            lay = ("double" if t == 64 else f"double, {t - 12} mantissa bits" if t >= 33 else
                   "single" if t == 32 else f"single, {t - 9} mantissa bits" if t >= 17 else
                   "half" if t == 16 else f"half, {t - 6} mantissa bits")
            print(f"| {t} | {lay} | " + " | ".join(
                f"{r[f]['rel_rmse']:.2e} / {r[f]['max_rel']:.1e}" for f in ("a_all", "a_x_fp64")) + " |")
        if args.json:
            with open(args.json, "w") as f:
                json.dump(rows, f, indent=1)
        return
    import torch
    import paper_2512_05516_gb300 as sph
    if not torch.cuda.is_available():
        raise SystemExit("the precision report runs the CUDA path: no GPU here")
    if args.sweep:
        rows = sweep_report(sph_inputs.sod(), torch, sph)
        print()
        print("| total bits | storage | rho | h | P | a |")
        print("|---|---|---|---|---|---|")
        for r in rows:
            print(f"| {r['total_bits']} | {r['storage']} | " +
                  " | ".join(f"{r[f]['rel_rmse']:.2e} / {r[f]['max_rel']:.1e}" for f in ("rho", "h", "P", "a")) + " |")
        if args.json:
            with open(args.json, "w") as f:
                json.dump(rows, f, indent=1)
        return
    rows = []
    sod = sph_inputs.sod()
    r1, _ = one_step_report(sod, torch, sph, time_it=True)
    rows += r1
    sed = sph_inputs.sedov()
    r1, _ = one_step_report(sed, torch, sph, time_it=True)
    rows += r1
    if not args.quick:
        rows += hundred_step_report("sod", sph_inputs.sod(), torch, sph)
        rows += hundred_step_report("sedov", sph_inputs.sedov(128, 128, 64), torch, sph)
    print()
    print("relative RMSE / max relative error (both over the mean magnitude), mode T")
    print(table([r for r in rows if r["steps"] == 1], ["rho", "h", "P", "a"]))
    print()
    print(table([r for r in rows if r["steps"] > 1], ["rho", "h", "P", "u", "v", "a", "x_rms_over_spacing"]))
    if args.json:
        with open(args.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
