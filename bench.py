"""Benchmark of the compressed-patch time step (one JSON line on stdout).

Workload: D2Q9 BGK, 2048^2 periodic, folded BL5/3 patches of 64 cells
(65^2 nodes), 4 levels, FP32 compute, BF16 details with per-band scale,
shear wave u_x = 0.05 sin(2 pi y/2048) + N(0, 1e-4), tau = 0.6.

  1. quality pass: for eps in {1e-5, 1e-4, 1e-3}, the full 2000-step run,
     compressed vs the uncompressed FP32 run on the same GPU; relative L2 of
     u and rho at the end (rho - <rho> is reported too: in this nearly
     incompressible flow it is ~1e-7 and relative errors of it are noise),
     compression ratio;
  2. the headline eps is the largest whose errors are <= 1e-3;
  3. timing: W warm-up steps, then K steps each timed with CUDA events on the
     simulation's stream, the 129 MB L2 flushed (a 512 MB write) before each
     timed step; MLUPS = 2048^2 * K / sum of step times;
  4. the uncompressed baseline timed the same way, the C-ABI end to end with
     host buffers, nvidia-smi clocks during the timed region, and the CPU
     oracle on a bounded sample (--impl reference times only the oracle);
  5. side sections: the 2-D Euler workload (4096^2 cells, outflow) under
     "euler", the batch of 96 D2Q9 grids under "batch", learned against
     uniform eps under "learned_eps", D3Q19 (quality on 256^3, timing on
     1024^3, and the 42-input network) under "d3q19".

--gpus N (under torchrun) runs N independent replicas (weak scaling); rank 0
prints the line with the max time over ranks.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2302_09883_gb300 import inputs  # noqa: E402

WORKLOAD = "d2q9_bl53_2048"
METRIC = "MLUPS & compression ratio, compressed vs uncompressed, at rel. L2 err ≤1e-3"
EPS_SWEEP = (1e-7, 1e-6, 1e-5, 1e-4, 1e-3)
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quality-steps", type=int, default=None)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-euler", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-d3q19", action="store_true")
    ap.add_argument("--no-transport", action="store_true")
    ap.add_argument("--no-swe", action="store_true")
    ap.add_argument("--no-hilo", action="store_true")
    ap.add_argument("--d3q19-n", type=int, default=1024, help="D3Q19 timing grid (cells per axis)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(torch, ms, device):
    """The slowest replica's time, on every rank (the job's time at N > 1)."""
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def macro_fields(w, n=None):
    return inputs.initial_fields(w, n=n, seed=0)


def velocity_rho(F):
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], np.float64)[:, None, None]
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], np.float64)[:, None, None]
    rho = F.sum(0)
    return rho, (cx * F).sum(0) / rho, (cy * F).sum(0) / rho


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.out = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()  # nvidia-smi takes a while to start: the timed region begins after its first sample
            while not self.out and time.time() - t0 < 5.0:
                time.sleep(0.01)
            self.first = len(self.out)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # the samples taken while the timed region ran (the one before it
        # only if the region was shorter than the sampling interval)
        lines = self.out[getattr(self, "first", 0):] or self.out[-1:]
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def reruns(obj):
    """Steps a simulation has re-run after an arena overflow (0 for the dense
    baselines); read outside timed regions."""
    return obj.stats().get("arena_reruns", 0) if hasattr(obj, "resident_bytes") else 0


def timed_steps(torch, obj, s, K, flush, _again=True):
    """Sum of per-step CUDA-event times (ms) on stream s, with an L2 flush
    before each step (outside the timed interval).  A step whose records
    overflowed an automatic arena returns at once and is re-run by the next
    synchronising call, outside the events: such a measurement is taken
    again (the arena has grown by then)."""
    r0 = reruns(obj)
    ms = _timed_steps(torch, obj, s, K, flush)
    if reruns(obj) != r0:
        if not _again:
            raise RuntimeError("arena overflow inside the timed steps")
        return timed_steps(torch, obj, s, K, flush, _again=False)
    return ms


def _timed_steps(torch, obj, s, K, flush):
    total = 0.0
    evs = []
    for _ in range(K):
        with torch.cuda.stream(s):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
        obj.step(1)
        with torch.cuda.stream(s):
            b.record(s)
        evs.append((a, b))
    s.synchronize()
    for a, b in evs:
        total += a.elapsed_time(b)
    return total


def quality_pass(torch, w, steps, eps_list, timing=None):
    """Full-length compressed runs (automatic arenas) against the uncompressed
    FP32 run: per eps the relative L2 of u and rho at the end, the record
    and resident compression ratios, survivors, FP64 mass drift; with
    timing = (K, flush, stream), K more steps timed from the state the run
    ended in (the one its survivors describe)."""
    from paper_2302_09883_gb300 import Dense, Sim
    n = w["n"]
    f = macro_fields(w)
    d = Dense("d2q9", n, n, tau=w["tau"])
    d.init_macro(f)
    d.step(steps)
    Fd = np.stack([d.export_field(i) for i in range(9)])
    rho_d, ux_d, uy_d = velocity_rho(Fd)
    m0 = float(np.sum(f[0]))
    dense_drift = (float(Fd.sum()) - m0) / m0
    dense_bytes = d.nbytes()
    d.close()
    res = []
    for eps in eps_list:
        s = Sim("d2q9", w["wavelet"], n, n, w["P"], w["L"], eps, prec=w["prec"], store=w["store"], tau=w["tau"],
                stream=timing[2] if timing else None)
        s.init_macro(f)
        s.step(steps)
        s.sync()
        Fc = s.export_field(-1)
        rho_c, ux_c, uy_c = velocity_rho(Fc)
        st = s.stats()
        cb = s.compressed_bytes()
        u_err = rel_l2(np.stack([ux_c, uy_c]), np.stack([ux_d, uy_d]))
        r_err = rel_l2(rho_c, rho_d)
        res.append({"eps": eps, "rel_l2_u": u_err, "rel_l2_rho": r_err,
                    "rel_l2_rho_dev": rel_l2(rho_c - rho_c.mean(), rho_d - rho_d.mean()),
                    "rel_l2_pop_max": max(rel_l2(Fc[i], Fd[i]) for i in range(9)),
                    "compression_ratio": st["uncompressed_bytes"] / cb, "compressed_bytes": cb,
                    "entropy_coded_bytes": len(s.entropy_code()), "record_bytes": st["live_bytes"],
                    "survivors_per_patch": s.survivors() / s.npatch,
                    "resident_bytes": st["resident_bytes"],
                    "resident_ratio": st["uncompressed_bytes"] / st["resident_bytes"],
                    "resident_ratio_vs_dense_run": dense_bytes / st["resident_bytes"],
                    "arena_reruns": st["arena_reruns"],
                    "mass_drift": (st["mass"] - m0) / m0, "dense_mass_drift": dense_drift})
        if timing:
            K, flush, bs = timing
            ms = timed_steps(torch, s, bs, K, flush)
            s.sync()
            res[-1]["ms_per_step"] = ms / K
            res[-1]["mlups"] = n * n * K / (ms * 1e-3) / 1e6
            res[-1]["timed_from_step"] = steps
        # the compression's own mass drift: one encode and decode of the
        # uncompressed run's final state (FP64 sums of its FP32 nodes before
        # and after), apart from the collision's FP32 drift that mass_drift
        # and dense_mass_drift carry (re-encoding a decoded state would give
        # it back unchanged)
        m1 = float(Fd.astype(np.float64).sum())
        s.import_field(-1, Fd)
        res[-1]["encode_mass_drift"] = (float(s.export_field(-1).astype(np.float64).sum()) - m1) / m1
        s.close()
    return res


def euler_section(torch, K, W, flush, bs, qsteps=None, eps_sweep=(1e-5, 3e-5, 1e-4, 3e-4, 1e-3), stores=("i8", "bf16")):
    """2-D Euler (Rusanov), 4096 cells (4097 nodes) per axis, outflow, BL5/3
    P = 64, L = 4, FP32 compute, four-quadrant Riemann data, CFL 0.4.
    Quality: every (storage, eps) against the uncompressed FP32 run for the
    workload's 1500 steps at the fixed dt/h that CFL 0.4 gives on the
    initial state (so both runs are compared at the same times); timing:
    the adaptive CFL 0.4 step."""
    from paper_2302_09883_gb300 import Dense, Sim
    from paper_2302_09883_gb300._lib import WcsError
    w = dict(inputs.WORKLOADS["euler_bl53_4096"])
    n, qs = w["n"], qsteps or w["steps"]
    f = macro_fields(w)
    # quality at a fixed dt/h = CFL / (largest signal speed of the initial
    # state): CFL 0.4 at the start, and both runs compared at the same times
    rho, u, v, p = f
    c = np.sqrt(w["gamma"] * p / rho)
    dth = w["cfl"] / float(np.max(np.maximum(np.abs(u) + c, np.abs(v) + c)))
    kw = dict(periodic=(False, False), cfl=-dth, gamma=w["gamma"], stream=bs)
    kwt = dict(periodic=(False, False), cfl=w["cfl"], gamma=w["gamma"], stream=bs)
    d = Dense("euler2d", n, n, **kw)
    d.init_macro(f)
    d.step(qs)
    Wd = [d.export_field(q) for q in range(4)]
    d.close()
    sweep, heads = [], {}
    for store in stores:
        good = []
        for eps in eps_sweep:
            s = Sim("euler2d", "bl53", n, n, w["P"], w["L"], eps, prec=w["prec"], store=store, **kw)
            s.init_macro(f)
            s.step(qs)
            try:
                s.sync()
            except WcsError as ex:  # the lossy state lost positivity: the step reported non-finite values
                sweep.append({"store": store, "eps": eps, "failed": str(ex)})
                s.close()
                continue
            Wc = s.export_field(-1)
            st = s.stats()
            q = {"store": store, "eps": eps, "rel_l2": [rel_l2(Wc[k], Wd[k]) for k in range(4)],
                 "compression_ratio": st["uncompressed_bytes"] / s.compressed_bytes(),
                 "resident_ratio": st["uncompressed_bytes"] / st["resident_bytes"],
                 "survivors_per_patch": s.survivors() / s.npatch, "time": st["time"]}
            sweep.append(q)
            good.append(q)
            s.close()
        ok = [q for q in good if max(q["rel_l2"]) <= 1e-3]
        if good:
            heads[store] = max(ok, key=lambda q: q["eps"]) if ok else min(good, key=lambda q: q["eps"])
    out = {"workload": "euler_bl53_4096", "grid_nodes": [n + 1, n + 1], "P": w["P"], "levels": w["L"],
           "cfl": w["cfl"], "quality_dt_over_h": dth, "quality_steps": qs, "sweep": sweep}
    lu = (n + 1) * (n + 1)
    for store, head in heads.items():
        s = Sim("euler2d", "bl53", n, n, w["P"], w["L"], head["eps"], prec=w["prec"], store=store, **kwt)
        s.init_macro(f)
        s.step(W)
        s.sync()
        ms = timed_steps(torch, s, bs, K, flush)
        s.sync()
        s.close()
        out[store] = {"eps": head["eps"], "mlups": lu * K / (ms * 1e-3) / 1e6, "ms_per_step": ms / K,
                      "compression_ratio": head["compression_ratio"], "resident_ratio": head["resident_ratio"],
                      "rel_l2_rho_rhou_rhov_E": head["rel_l2"], "meets_1e-3": max(head["rel_l2"]) <= 1e-3}
    d = Dense("euler2d", n, n, **kwt)
    d.init_macro(f)
    d.step(W)
    dms = timed_steps(torch, d, bs, K, flush)
    d.close()
    out["uncompressed_mlups"] = lu * K / (dms * 1e-3) / 1e6
    return out


def transport_section(torch, K, W, flush, bs, levels=(1, 2, 3, 4, 5), thresholds=(0.0, 0.0025, 0.005, 0.01, 0.02, 0.04),
                      rules=("const", "accum", "capped")):
    """The paper's transport workload (Sec. 3.1.2, 3.2.1-3.2.3): 128^2 on
    [-1, 1]^2, 2 x 2 patches of 64 cells, outflow, velocity (0.9, 0.9), CFL
    0.45, to t = 0.5 (64 steps), FP32 with FP32 details.  Per (level,
    threshold, rule): the compression ratio averaged over the steps (stored
    bytes of an uncompressed FP32 state / live record bytes of each step),
    the paper's L2 error against the exact translated Gaussian (eq.
    L2_error) and the relative L2 difference from the uncompressed run.
    Then per rule the threshold giving a fixed compression error (relative
    L2 against the uncompressed run) at level 4, found by bisection in log
    c, and its ratio (the paper's test of the rules, Sec. 2.2).  Timing: the
    level-4 capped step at c = 0.01 on the paper's grid and on 4096^2."""
    from paper_2302_09883_gb300 import Dense, Sim
    w = dict(inputs.WORKLOADS["transport_128"])
    n = w["n"]
    kw = dict(periodic=(False, False), cfl=w["cfl"], velocity=w["velocity"], length=w["length"], stream=bs)
    f = inputs.transport_gaussian(n)
    steps = int(round(w["t_end"] / (w["cfl"] * (w["length"] / n) / max(w["velocity"]))))
    exact = inputs.transport_gaussian(n, t=w["t_end"])[0]
    d = Dense("transport", n, n, **kw)
    d.init_macro(f)
    d.step(steps)
    Wd = d.export_field(0)
    d.close()
    unc = (n + 1) ** 2 * 4
    area = (w["length"] ** 2) / (n + 1) ** 2

    def run(L, c, rule):
        s = Sim("transport", "bl53", n, n, w["P"], L, c, prec="f32", store="f32", rule=rule, **kw)
        s.init_macro(f)
        rs, rr, re, rv = [], [], [], []
        ncoarse = s.npatch * ((w["P"] >> L) + 1) ** 2
        for k in range(steps):
            s.step(1)
            rs.append(unc / s.stats()["live_bytes"])
            rr.append(unc / s.compressed_bytes())
            rv.append((n + 1) ** 2 / (ncoarse + s.survivors()))  # stored values against the grid's values
            if L == 4 and k % 8 == 7:  # the entropy stage on top, every 8th step
                re.append(unc / len(s.entropy_code()))
        Wc = s.export_field(0)
        t = s.stats()["time"]
        s.close()
        return {"level": L, "threshold": c, "rule": rule, "mean_ratio": float(np.mean(rs)),
                "mean_ratio_with_ring": float(np.mean(rr)),
                "mean_ratio_entropy_coded": float(np.mean(re)) if re else None,
                "mean_value_count_ratio": float(np.mean(rv)),
                "final_ratio": rs[-1], "l2_error_vs_exact": float(area * np.sum((Wc - exact) ** 2)),
                "rel_l2_vs_uncompressed": rel_l2(Wc - 1.0, Wd - 1.0), "time": t}

    sweep = [run(L, c, r) for L in levels for c in thresholds for r in rules]
    equal_error = {}
    for target in (1e-3, 1e-2):
        row = {}
        for rule in rules:
            lo, hi, best = -7.0, 0.0, None
            for _ in range(22):
                mid = 0.5 * (lo + hi)
                q = run(4, 10 ** mid, rule)
                if q["rel_l2_vs_uncompressed"] <= target:
                    lo, best = mid, q
                else:
                    hi = mid
            row[rule] = {"threshold": best["threshold"], "mean_ratio": best["mean_ratio"],
                         "rel_l2_vs_uncompressed": best["rel_l2_vs_uncompressed"]} if best else None
        ok = {r: v for r, v in row.items() if v}
        row["best_rule"] = max(ok, key=lambda r: ok[r]["mean_ratio"]) if ok else None
        equal_error["%.0e" % target] = row
    timing = {}
    for nt in (n, 4096):
        ft = inputs.transport_gaussian(nt)
        kt = dict(kw)
        s = Sim("transport", "bl53", nt, nt, w["P"], 4, 0.01, prec="f32", store="f32", rule="capped", **kt)
        s.init_macro(ft)
        s.step(W)
        s.sync()
        ms = timed_steps(torch, s, bs, K, flush)
        ratio = (nt + 1) ** 2 * 4 / s.stats()["live_bytes"]
        s.close()
        dd = Dense("transport", nt, nt, **kt)
        dd.init_macro(ft)
        dd.step(W)
        dms = timed_steps(torch, dd, bs, K, flush)
        dd.close()
        lu = (nt + 1) ** 2
        timing[str(nt)] = {"mlups": lu * K / (ms * 1e-3) / 1e6, "ms_per_step": ms / K, "compression_ratio": ratio,
                           "uncompressed_mlups": lu * K / (dms * 1e-3) / 1e6, "uncompressed_ms_per_step": dms / K}
    return {"workload": "transport_128", "steps": steps, "sweep": sweep, "equal_error_level4": equal_error,
            "timing_level4_capped_c0.01": timing,
            "note": "mean_ratio = uncompressed FP32 bytes of the unique nodes / record bytes (bitmask codec, not "
                    "the paper's CSR or LZ4); mean_ratio_with_ring also counts the patch table (BL5/3 patches "
                    "keep no ghost ring); mean_value_count_ratio = values of the grid / stored values (coarse "
                    "samples + kept details)"}


def swe_section(torch, bs, patches=(64, 32)):
    """The paper's cost study (Sec. 3.2.4, Table 1): shallow water with the
    Godunov flux on 129^2 nodes, the raised square, 38245 steps of dt =
    10 s / 38245, level 4, c = 5e-4, FP32 with FP32 details, compressed
    (decode, step and encode fused in one launch per step) against the
    uncompressed FP32 step on the same GPU: total GPU time of each (CUDA
    events around the whole run), the compression's overhead, the average
    compression ratio over the first simulated second and over the run, and
    the relative L2 difference of h at t = 10 s."""
    from paper_2302_09883_gb300 import Dense, Sim
    w = dict(inputs.WORKLOADS["swe_129"])
    n, steps = w["n"], w["steps"]
    dth = w["dt"] * n / w["length"]
    kw = dict(periodic=(False, False), cfl=-dth, gravity=w["gravity"], length=w["length"], stream=bs)
    f = inputs.swe_square(n)
    unc = (n + 1) ** 2 * 3 * 4

    def total_ms(obj, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        r0 = reruns(obj)
        with torch.cuda.stream(bs):
            a.record(bs)
        obj.step(k)
        with torch.cuda.stream(bs):
            b.record(bs)
        bs.synchronize()
        if reruns(obj) != r0:
            raise RuntimeError("arena overflow inside the timed run")
        return a.elapsed_time(b)

    d = Dense("swe", n, n, **kw)
    d.init_macro(f)
    d_ms = total_ms(d, steps)
    hd = d.export_field(0)
    d.close()
    runs = {}
    for P in patches:
        # a fixed arena of the whole uncompressed state: the run's records
        # always fit, so no step is re-run outside the timed region
        s = Sim("swe", "bl53", n, n, P, w["L"], w["eps"], prec="f32", store="f32", rule=w["rule"],
                arena_factor=1.0, **kw)
        s.init_macro(f)
        s_ms = total_ms(s, steps)
        s.sync()
        hc = s.export_field(0)
        t_end = s.stats()["time"]
        s.close()
        # compression ratio per step over the first simulated second
        # (synchronising after every step, so not timed) and every 100th step
        s = Sim("swe", "bl53", n, n, P, w["L"], w["eps"], prec="f32", store="f32", rule=w["rule"], **kw)
        s.init_macro(f)
        first, every, firstc = [], [], []
        k1 = int(round(1.0 / w["dt"]))
        # the count of stored values (coarse samples + kept details) against
        # the grid's values, the measure closest to the paper's CSR count
        ncoarse = s.npatch * 3 * ((P >> w["L"]) + 1) ** 2
        for k in range(steps):
            s.step(1)
            if k < k1:
                first.append(unc / s.stats()["live_bytes"])
                firstc.append(3 * (n + 1) ** 2 / (ncoarse + s.survivors()))
            elif k % 100 == 0:
                every.append(unc / s.stats()["live_bytes"])
        s.close()
        runs["P%d" % P] = {"patches": (n // P) ** 2, "compressed_total_ms": s_ms, "t_end": t_end,
                           "overhead_pct": 100.0 * (s_ms - d_ms) / d_ms,
                           "mean_ratio_first_second": float(np.mean(first)),
                           "mean_ratio_run": float(np.mean(first + every)),
                           "mean_value_count_ratio_first_second": float(np.mean(firstc)),
                           "rel_l2_h_vs_uncompressed": rel_l2(hc, hd)}
    return {"workload": "swe_129", "steps": steps, "eps": w["eps"], "levels": w["L"],
            "rule": w["rule"], "uncompressed_total_ms": d_ms, "compressed": runs,
            "paper_context": "V100, CUDA, CSR: 95.67 s uncompressed, 114.13 s with wavelets + CSR (+17.41 %), "
                             "x73.51 average ratio over the first second"}


def _velocity_rho_dev(torch, F):
    cx = torch.tensor([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=F.dtype, device=F.device)[:, None, None]
    cy = torch.tensor([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=F.dtype, device=F.device)[:, None, None]
    rho = F.sum(0)
    return rho, (cx * F).sum(0) / rho, (cy * F).sum(0) / rho


def _rel_dev(torch, a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def batch_section(torch, K, W, flush, bs, nsims=96, quality_steps=500, store="f32",
                  eps_ladder=(1e-4, 3e-5, 1e-5, 3e-6, 1e-6, 3e-7, 1e-7, 3e-8, 1e-8, 3e-9, 1e-9, 0.0)):
    """96 independent D2Q9 runs, sides drawn from {256,512,1024,2048} (seeded),
    Gaussian bumps with amplitude U(0.01,0.1) and width U(4,32), FP32 compute
    with FP32 details (BF16's 2^-9 relative rounding alone exceeds 1e-3 of
    the small velocities of the weaker bumps), P chosen per side by the
    library's autotuner among (64,4) and (32,3).
    Each simulation gets its own eps: the largest of a ladder (down to 0,
    which keeps every coefficient) whose 500-step run keeps the relative L2
    error of u and rho <= 1e-3 against its own uncompressed run, found by
    bisection over the ladder (the error grows with eps); where even eps = 0
    errs by more (the FP32 rounding of the lifting against velocities of
    order 1e-4), the gate is 1.1 x that floor.  The batch steps both patch sizes in one persistent
    launch per step (launch shape tuned), six steps per CUDA-graph replay;
    each replay is one timed unit with the L2 flushed before it."""
    from paper_2302_09883_gb300 import Batch, Dense, Sim, autotune
    specs = inputs.batch_specs(nsims, seed=0)
    tau = 0.6
    reps_by_side = {}
    for sp in specs:
        reps_by_side.setdefault(sp["side"], sp)
    dev = lambda sp: inputs.gaussian_bump_device(sp["side"], sp["amp"], sp["sigma"], sp["cx"], sp["cy"])
    choice = {}
    for n, sp in sorted(reps_by_side.items()):
        best, ms = autotune("d2q9", "bl53", n, n, 1e-5, dev(sp), candidates=((64, 4), (32, 3)), tau=tau, store=store,
                            stream=bs)
        choice[n] = ({0: (64, 4), 1: (32, 3)}[best], ms)
    # per-simulation eps at the gate
    eps_of, err_of = [], []
    for sp in specs:
        n = sp["side"]
        (P, L), _ = choice[n]
        d = Dense("d2q9", n, n, tau=tau, stream=bs)
        d.init_macro(dev(sp))
        d.step(quality_steps)
        Fd = torch.stack([torch.from_numpy(d.export_field(i)).cuda() for i in range(9)])
        d.close()
        rd, uxd, uyd = _velocity_rho_dev(torch, Fd)
        ud = torch.stack([uxd, uyd])
        def trial(eps):
            c = Sim("d2q9", "bl53", n, n, P, L, eps, prec="f32", store=store, tau=tau, stream=bs)
            c.init_macro(dev(sp))
            c.step(quality_steps)
            Fc = torch.empty((9, n, n), dtype=torch.float64, device="cuda")
            c.export_field(-1, out=Fc)
            c.close()
            rc, uxc, uyc = _velocity_rho_dev(torch, Fc)
            return _rel_dev(torch, torch.stack([uxc, uyc]), ud), _rel_dev(torch, rc, rd)
        # the FP32 floor: eps = 0 keeps every coefficient, and what error
        # remains is the rounding of the FP32 lifting against the FP32
        # uncompressed run; where that floor is above 1e-3 (weak bumps whose
        # velocities are tiny) the gate is 1.1 x the floor
        res = {len(eps_ladder) - 1: trial(eps_ladder[-1])}
        gate = (max(1e-3, 1.1 * res[len(eps_ladder) - 1][0]), max(1e-3, 1.1 * res[len(eps_ladder) - 1][1]))
        lo, hi = 0, len(eps_ladder) - 1  # find the first index that passes
        while lo < hi:
            mid = (lo + hi) // 2
            if mid not in res:
                res[mid] = trial(eps_ladder[mid])
            if res[mid][0] <= gate[0] and res[mid][1] <= gate[1]:
                hi = mid
            else:
                lo = mid + 1
        eps_of.append(eps_ladder[lo])
        err_of.append({"u": res[lo][0], "rho": res[lo][1], "floor_u": res[len(eps_ladder) - 1][0],
                       "gate_u": gate[0], "gate_rho": gate[1]})
    sims = []
    for sp, eps in zip(specs, eps_of):
        n = sp["side"]
        (P, L), _ = choice[n]
        s = Sim("d2q9", "bl53", n, n, P, L, eps, prec="f32", store=store, tau=tau, stream=bs)
        s.init_macro(dev(sp))
        sims.append(s)
    b = Batch(sims)
    launches, grid = b.launches_per_step()
    nitems = sum(s.npatch for s in sims)
    tune = None
    if launches == 1:
        nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        cands = [nsm, nitems]
        tune = {"grids": cands, "ms_per_step": b.tune_launch(cands, steps=6)}
        launches, grid = b.launches_per_step()
    b.step(max(6, (W + 5) // 6 * 6))
    b.sync()
    reps = max(1, (K + 5) // 6)

    def timed():
        evs = []
        for _ in range(reps):
            with torch.cuda.stream(bs):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(bs)
            b.step(6)
            with torch.cuda.stream(bs):
                e1.record(bs)
            evs.append((e0, e1))
        bs.synchronize()
        return sum(e0.elapsed_time(e1) for e0, e1 in evs)

    # a simulation whose records outgrew its arenas inside the timed steps
    # froze and caught up in b.sync(): those steps did not run in the timed
    # launches, so the timing is taken again (the arenas have grown by then)
    retimed = 0
    while True:
        r0 = sum(reruns(s) for s in sims)
        ms = timed()
        b.sync()
        if sum(reruns(s) for s in sims) == r0:
            break
        retimed += 1  # the arenas doubled; records still grow as the waves spread
        if retimed > 4:
            raise RuntimeError("batch: arena overflow inside the timed steps five times")
    lu = sum(sp["side"] ** 2 for sp in specs)
    unc = sum(s.stats()["uncompressed_bytes"] for s in sims)
    comp = sum(s.compressed_bytes() for s in sims)
    res = sum(s.resident_bytes() for s in sims)
    nrerun = sum(reruns(s) for s in sims)
    b.close()
    for s in sims:
        s.close()
    eps_hist = {("%.0e" % e): eps_of.count(e) for e in sorted(set(eps_of), reverse=True)}
    return {"workload": "d2q9_batch_96", "nsims": nsims, "lattice_updates_per_step": lu,
            "eps_per_simulation": eps_hist, "max_rel_l2_u": max(e["u"] for e in err_of),
            "max_rel_l2_rho": max(e["rho"] for e in err_of), "all_meet_1e-3": all(
                e["u"] <= 1e-3 and e["rho"] <= 1e-3 for e in err_of),
            "n_meet_1e-3": sum(e["u"] <= 1e-3 and e["rho"] <= 1e-3 for e in err_of),
            "n_at_fp32_floor_gate": sum(e["gate_u"] > 1e-3 for e in err_of),
            "max_fp32_floor_u": max(e["floor_u"] for e in err_of),
            "all_meet_gate": all(e["u"] <= e["gate_u"] and e["rho"] <= e["gate_rho"] for e in err_of),
            "autotune": {str(k): {"P": v[0][0], "levels": v[0][1], "ms_per_step_P64_P32": v[1]} for k, v in choice.items()},
            "launches_per_step": launches, "launch_grid": grid, "launch_tuning": tune,
            "mlups": lu * 6 * reps / (ms * 1e-3) / 1e6, "ms_per_step": ms / (6 * reps), "timed_steps": 6 * reps,
            "compression_ratio": unc / comp, "resident_ratio": unc / res, "quality_steps": quality_steps,
            "arena_reruns": nrerun, "retimed_after_overflow": retimed}


def learned_section(torch, K, W, flush, bs, n_eval=1024, steps=1000, deltas=(3e-6, 1e-5, 3e-5),
                    eps_sweep=(1e-6, 3e-6, 1e-5, 3e-5, 1e-4, 3e-4)):
    """Per-patch eps from the network against one uniform eps, D2Q9 FP32/BF16,
    BL5/3 P = 64, L = 4, tau 0.6.  Training data: dense FP32 snapshots
    (t = 0, 100, 300, 600) of 512^2 runs from eight seeded initial states
    (Gaussian bumps, amplitude U(0.01, 0.1), width U(4, 32), random centre;
    shear waves with N(0, 1e-4) noise), features and labels by the library's
    kernels for every delta.  Evaluation: a 1024^2 Gaussian bump (amplitude
    0.05, width 40, centred) for `steps` steps against the uncompressed run;
    the uniform sweep's ratio is interpolated (log-log) at the learned run's
    error of u, and both step times are measured like the headline."""
    from paper_2302_09883_gb300 import Dense, Sim, learned
    P, L, tau = 64, 4, 0.6
    rng = np.random.default_rng(123)
    snaps = []
    for k in range(8):
        n = 512
        if k % 2 == 0:
            f = inputs.gaussian_bump_device(n, rng.uniform(0.01, 0.1), rng.uniform(4, 32), rng.uniform(0, n),
                                            rng.uniform(0, n))
        else:
            f = inputs.shear_wave(n, seed=100 + k)
        d = Dense("d2q9", n, n, tau=tau, stream=bs)
        d.init_macro(f)
        done = 0
        for t in (0, 100, 300, 600):
            d.step(t - done)
            done = t
            snaps.append(torch.from_numpy(np.stack([d.export_field(i) for i in range(9)]).astype(np.float32)).cuda())
        d.close()
    fe = lambda sp: inputs.gaussian_bump_device(n_eval, 0.05, 40.0, n_eval / 2, n_eval / 2)
    d = Dense("d2q9", n_eval, n_eval, tau=tau, stream=bs)
    d.init_macro(fe(None))
    d.step(steps)
    rd, uxd, uyd = velocity_rho(np.stack([d.export_field(i) for i in range(9)]))
    d.close()

    def evaluate(sim):
        sim.init_macro(fe(None))
        sim.step(steps)
        sim.sync()
        rc, uxc, uyc = velocity_rho(sim.export_field(-1))
        st = sim.stats()
        return {"rel_l2_u": rel_l2(np.stack([uxc, uyc]), np.stack([uxd, uyd])), "rel_l2_rho": rel_l2(rc, rd),
                "compression_ratio": st["uncompressed_bytes"] / sim.compressed_bytes(),
                "record_ratio": st["uncompressed_bytes"] / st["live_bytes"]}

    uniform = []
    for eps in eps_sweep:
        c = Sim("d2q9", "bl53", n_eval, n_eval, P, L, eps, prec="f32", store="bf16", tau=tau, arena_factor=0.5,
                stream=bs)
        uniform.append(dict(eps=eps, **evaluate(c)))
        c.close()
    def uniform_ratio_at(err, key):
        pts = sorted((q["rel_l2_u"], q[key]) for q in uniform)
        xs = np.log([p[0] for p in pts])
        ys = np.log([p[1] for p in pts])
        if not (xs[0] <= np.log(err) <= xs[-1]):
            return None
        return float(np.exp(np.interp(np.log(err), xs, ys)))

    runs = []
    for delta in deltas:
        X, T = [], []
        for u in snaps:
            f_, l_ = learned.features_labels(u, P, L, delta)
            X.append(f_)
            T.append(l_)
        X, T = torch.cat(X), torch.cat(T)
        m, hist = learned.fit(X, T, epochs=200, batch=128, lr=2e-3, seed=1)
        c = Sim("d2q9", "bl53", n_eval, n_eval, P, L, 1e-5, prec="f32", store="bf16", tau=tau, arena_factor=0.5,
                stream=bs)
        learned.use_mlp(c, m, 1e-7, 1e-2)
        r = evaluate(c)
        _, eps_p = learned.patch_data(c, L)
        c.close()
        ur = uniform_ratio_at(r["rel_l2_u"], "compression_ratio")
        urr = uniform_ratio_at(r["rel_l2_u"], "record_ratio")
        runs.append(dict(delta=delta, n_train=int(X.shape[0]), label_mean=float(T.mean()), label_std=float(T.std()),
                         train_loss_first=float(hist[0]), train_loss_last=float(hist[-1]),
                         eps_patch_log10_min=float(np.log10(eps_p.min())),
                         eps_patch_log10_max=float(np.log10(eps_p.max())),
                         uniform_ratio_at_same_error=ur, ratio_gain=(r["compression_ratio"] / ur) if ur else None,
                         uniform_record_ratio_at_same_error=urr,
                         record_ratio_gain=(r["record_ratio"] / urr) if urr else None, **r))
        keep = m
    # step time: learned mode (features + inference) vs uniform at the same size
    times = {}
    for mode in ("uniform", "learned"):
        c = Sim("d2q9", "bl53", n_eval, n_eval, P, L, 1e-5, prec="f32", store="bf16", tau=tau, arena_factor=0.5,
                stream=bs)
        if mode == "learned":
            learned.use_mlp(c, keep, 1e-7, 1e-2)
        c.init_macro(fe(None))
        c.step(W)
        c.sync()
        torch.cuda.synchronize()
        ms = timed_steps(torch, c, bs, K, flush)
        c.sync()
        c.close()
        times[mode] = ms / K
    return {"workload": "d2q9_bl53_bump_1024_learned_eps", "steps": steps, "P": P, "levels": L,
            "network": "6L=24 -> 64 -> 64 -> 1 GELU FP32", "uniform": uniform, "learned": runs,
            "ms_per_step_uniform": times["uniform"], "ms_per_step_learned": times["learned"],
            "mlups_learned": n_eval * n_eval / (times["learned"] * 1e-3) / 1e6}


def hilo_section(torch, K, W, flush, bs, w, eps, steps=100):
    """hi + lo coarse storage on the headline configuration (Sec. 2.1.2, eq.
    conservation).  A state of the headline run (steps steps from its
    initial fields, decoded to dense FP32 populations) is imported into a
    simulation with the option on: Check A compares the FP64 coarse-domain
    mass after that encode (field_sum + field_sum_lo) with the FP64 sum of
    the imported values, and the FP32 coarse samples alone with the same.
    Then the step is timed with the option on (W warm-up, K steps, L2
    flushed before each)."""
    from paper_2302_09883_gb300 import Sim
    n = w["n"]
    s = Sim("d2q9", "bl53", n, n, w["P"], w["L"], eps, prec="f32", store="bf16", tau=w["tau"], stream=bs,
            coarse_hilo=True)
    s.init_macro(macro_fields(w))
    s.step(steps)
    Fd = torch.empty((9, n, n), dtype=torch.float32, device="cuda")
    s.export_field(-1, out=Fd, dtype=np.float32)
    want = Fd.double().sum(dim=(1, 2))
    scale = Fd.double().abs().sum(dim=(1, 2))
    s.import_field(-1, Fd)
    st = s.stats()
    fs = torch.tensor(st["field_sum"], dtype=torch.float64, device="cuda")
    fl = torch.tensor(st["field_sum_lo"], dtype=torch.float64, device="cuda")
    rel = float(((fs + fl - want).abs() / scale).max())
    rel_hi = float(((fs - want).abs() / scale).max())
    del Fd
    s.step(W)
    torch.cuda.synchronize()
    ms = timed_steps(torch, s, bs, K, flush) / K
    s.sync()
    st = s.stats()
    out = {"workload": "d2q9_bl53_%d" % n, "eps": eps, "state": "headline run after %d steps, imported" % steps,
           "check_a_rel": rel, "check_a_rel_hi_only": rel_hi, "check_a_bound": 1e-12,
           "ms_per_step": ms, "mlups": n * n / (ms * 1e-3) / 1e6,
           "compression_ratio": st["uncompressed_bytes"] / s.compressed_bytes(),
           "lo_bytes": s.npatch * 9 * ((w["P"] >> w["L"]) + 1) ** 2 * 4}
    s.close()
    out["d3q19"] = _hilo_d3q19(torch, K, W, flush, bs)
    return out


def _hilo_d3q19(torch, K, W, flush, bs, n=256, steps=20, P=32, L=3, eps=1e-7):
    """The same for D3Q19 (Taylor-Green vortex, n^3, P 32, L 3, BF16):
    Check A on an imported state of the run, and the step time with the
    option on and off."""
    from paper_2302_09883_gb300 import Sim3
    res = {"workload": "d3q19_bl53_tgv_%d" % n, "eps": eps}
    for on in (True, False):
        s = Sim3(n, n, n, P, L, eps, store="bf16", tau=0.55, stream=bs, coarse_hilo=on)
        s.init_macro(_tgv_device(torch, n))
        s.step(steps)
        if on:
            Fd = torch.empty((19, n, n, n), dtype=torch.float32, device="cuda")
            s.export_field(-1, out=Fd, dtype=np.float32)
            want = Fd.double().sum(dim=(1, 2, 3))
            scale = Fd.double().abs().sum(dim=(1, 2, 3))
            s.import_field(-1, Fd)
            del Fd
            st = s.stats()
            fs = torch.tensor(st["field_sum"], dtype=torch.float64, device="cuda")
            fl = torch.tensor(st["field_sum_lo"], dtype=torch.float64, device="cuda")
            res["check_a_rel"] = float(((fs + fl - want).abs() / scale).max())
            res["check_a_rel_hi_only"] = float(((fs - want).abs() / scale).max())
        s.step(W)
        torch.cuda.synchronize()
        res["ms_per_step_hilo" if on else "ms_per_step"] = timed_steps(torch, s, bs, K, flush) / K
        s.close()
        torch.cuda.empty_cache()
    return res


def _tgv_device(torch, n, u0=0.04):
    return inputs.taylor_green_3d_device(n, u0=u0)


def d3q19_section(torch, K, W, flush, bs, n_quality=256, quality_steps=1000, n_time=1024,
                  eps_sweep=(1e-7, 1e-6, 1e-5)):
    """D3Q19 BGK, decaying Taylor-Green vortex u0 = 0.04, tau = 0.55, periodic,
    BL5/3 P = 32, L = 3, FP32 compute, BF16 details.  Quality: n_quality^3
    for quality_steps steps against the uncompressed FP32 run (rel. L2 of u
    and rho on the device).  Timing: n_time^3, compressed and uncompressed,
    W warm-up then K steps, each timed with CUDA events and the L2 flushed
    before it."""
    from paper_2302_09883_gb300 import Dense3, Sim3
    P, L, tau = 32, 3, 0.55
    cx = torch.tensor([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0], dtype=torch.float64, device="cuda")
    cy = torch.tensor([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1], dtype=torch.float64, device="cuda")
    cz = torch.tensor([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1], dtype=torch.float64, device="cuda")

    def moments(Fd):
        rho = Fd.sum(0)
        u = torch.stack([torch.tensordot(c, Fd, dims=([0], [0])) / rho for c in (cx, cy, cz)])
        return rho, u

    n = n_quality
    d = Dense3(n, n, n, tau=tau, stream=bs)
    d.init_macro(_tgv_device(torch, n))
    d.step(quality_steps)
    Fd = torch.empty((19, n, n, n), dtype=torch.float32, device="cuda")
    for i in range(19):
        d.export_field(i, out=Fd[i], dtype=np.float32)
    d.close()
    rho_d, u_d = moments(Fd.double())
    m0 = float(_tgv_device(torch, n)[0].sum())
    dense_drift = (float(Fd.double().sum()) - m0) / m0
    del Fd
    quality = []
    for eps in eps_sweep:
        c = Sim3(n, n, n, P, L, eps, store="bf16", tau=tau, arena_factor=0.3, stream=bs)
        c.init_macro(_tgv_device(torch, n))
        c.step(quality_steps)
        c.sync()
        Fc = torch.empty((19, n, n, n), dtype=torch.float32, device="cuda")
        c.export_field(-1, out=Fc, dtype=np.float32)
        rho_c, u_c = moments(Fc.double())
        st = c.stats()
        quality.append({"eps": eps, "rel_l2_u": float((u_c - u_d).norm() / u_d.norm()),
                        "rel_l2_rho": float((rho_c - rho_d).norm() / rho_d.norm()),
                        "compression_ratio": st["uncompressed_bytes"] / c.compressed_bytes(),
                        "record_ratio": st["uncompressed_bytes"] / st["live_bytes"],
                        "mass_drift": (st["mass"] - m0) / m0, "dense_mass_drift": dense_drift})
        c.close()
        del Fc
    torch.cuda.empty_cache()
    ok = [q for q in quality if q["rel_l2_u"] <= 1e-3 and q["rel_l2_rho"] <= 1e-3]
    head = max(ok, key=lambda q: q["eps"]) if ok else quality[0]

    # learned eps (config 5's network, 42 inputs): trained on dense snapshots
    # of 128^3 vortices (u0 0.02 / 0.04 / 0.06, with and without N(0, 1e-5)
    # velocity noise, t = 0 and 300), compared with the uniform sweep at the
    # same error of u on the quality grid
    from paper_2302_09883_gb300 import learned
    snaps = []
    gen = torch.Generator(device="cuda").manual_seed(5)
    for u0 in (0.02, 0.04, 0.06):
        for noise in (0.0, 1e-5):
            m3 = 128
            fm = _tgv_device(torch, m3, u0)
            if noise:
                fm[1] = fm[1] + noise * torch.randn(fm[1].shape, generator=gen, device="cuda", dtype=torch.float64)
            d = Dense3(m3, m3, m3, tau=tau, stream=bs)
            d.init_macro(fm)
            done = 0
            for t in (0, 300):
                d.step(t - done)
                done = t
                Fs = torch.empty((19, m3, m3, m3), dtype=torch.float32, device="cuda")
                for i in range(19):
                    d.export_field(i, out=Fs[i], dtype=np.float32)
                snaps.append(Fs)
            d.close()
    pts = sorted((q["rel_l2_u"], q["compression_ratio"]) for q in quality)

    def uniform_ratio_at(err):
        xs, ys = np.log([p[0] for p in pts]), np.log([p[1] for p in pts])
        if not (xs[0] <= np.log(err) <= xs[-1]):
            return None
        return float(np.exp(np.interp(np.log(err), xs, ys)))

    learned_runs = []
    for delta in (3e-7, 3e-6):
        X, T = [], []
        for Fs in snaps:
            f_, l_ = learned.features_labels3(Fs, P, L, delta)
            X.append(f_)
            T.append(l_)
        X, T = torch.cat(X), torch.cat(T)
        mdl, hist = learned.fit(X, T, epochs=300, batch=64, lr=2e-3, seed=3)
        c = Sim3(n, n, n, P, L, 1e-6, store="bf16", tau=tau, arena_factor=0.3, stream=bs)
        learned.use_mlp(c, mdl, 1e-8, 1e-2)
        c.init_macro(_tgv_device(torch, n))
        c.step(quality_steps)
        c.sync()
        Fc = torch.empty((19, n, n, n), dtype=torch.float32, device="cuda")
        c.export_field(-1, out=Fc, dtype=np.float32)
        rho_c, u_c = moments(Fc.double())
        st = c.stats()
        _, eps_p = learned.patch_data(c, L)
        r = {"delta": delta, "n_train": int(X.shape[0]), "label_mean": float(T.mean()), "label_std": float(T.std()),
             "train_loss_first": float(hist[0]), "train_loss_last": float(hist[-1]),
             "rel_l2_u": float((u_c - u_d).norm() / u_d.norm()), "rel_l2_rho": float((rho_c - rho_d).norm() / rho_d.norm()),
             "compression_ratio": st["uncompressed_bytes"] / c.compressed_bytes(),
             "eps_patch_log10_min": float(np.log10(eps_p.min())), "eps_patch_log10_max": float(np.log10(eps_p.max()))}
        ur = uniform_ratio_at(r["rel_l2_u"])
        r["uniform_ratio_at_same_error"] = ur
        r["ratio_gain"] = r["compression_ratio"] / ur if ur else None
        learned_runs.append(r)
        c.close()
        del Fc
    del snaps
    torch.cuda.empty_cache()

    def timed(obj):
        obj.step(W)
        torch.cuda.synchronize()
        return timed_steps(torch, obj, bs, K, flush) / K

    n = n_time
    c = Sim3(n, n, n, P, L, head["eps"], store="bf16", tau=tau, stream=bs)  # automatic arenas
    f = _tgv_device(torch, n)
    c.init_macro(f)
    del f
    torch.cuda.empty_cache()
    ms_c = timed(c)
    c.sync()
    st = c.stats()
    ratio_big = st["uncompressed_bytes"] / c.compressed_bytes()
    resident_c = st["resident_bytes"]
    c.close()
    d = Dense3(n, n, n, tau=tau, stream=bs)
    f = _tgv_device(torch, n)
    d.init_macro(f)
    del f
    torch.cuda.empty_cache()
    ms_d = timed(d)
    dense_bytes = d.nbytes()
    d.close()
    lu = n ** 3
    return {"workload": "d3q19_bl53_tgv_%d" % n, "P": P, "levels": L, "store": "bf16", "tau": tau, "u0": 0.04,
            "eps": head["eps"], "quality_grid": n_quality, "quality_steps": quality_steps, "quality": quality,
            "mlups": lu / (ms_c * 1e-3) / 1e6, "ms_per_step": ms_c, "uncompressed_mlups": lu / (ms_d * 1e-3) / 1e6,
            "uncompressed_ms_per_step": ms_d, "uncompressed_gbs": 152.0 * lu / (ms_d * 1e-3) / 1e9,
            "compression_ratio": ratio_big, "resident_bytes": resident_c, "uncompressed_resident_bytes": dense_bytes,
            "learned": learned_runs}


def roofline_bytes(sim, w):
    """Algorithmic bytes of one step launch.  Compulsory (what has to cross
    HBM): the records of state n read, the records of state n+1 written
    (about as many), the patch tables (8 B read and 8 B written per patch),
    the FP64 coarse-block sums (8 B per field and patch); the ring kernels
    also read and write their ghost rings.  With L2 reuse (D2Q9 on BL5/3):
    plus the eight neighbours' records of state n each patch reads for its
    ghosts, which mostly hit L2."""
    st = sim.stats()
    npatch = sim.npatch
    live = st["live_bytes"]
    base = 2 * live + 2 * npatch * 8 + npatch * 9 * 8
    if w["scheme"] == "d2q9" and w["wavelet"] == "bl53":
        return {"compulsory": base, "with_l2_reuse": base + 8 * live}
    ring = 2 * npatch * (12 * (w["P"] + 1) + 4) * 4
    return {"compulsory": base + ring, "with_l2_reuse": base + ring}


def lifting_flops_per_line(P, L):
    """FP32 operations of one BL5/3 line of P+1 nodes over L levels, counting
    each add/sub/mul separately: predict 3 (add, mul, sub) per detail, update
    4 (2 mul, 2 add) per interior sample (Sec. 2.1.2)."""
    ops = 0
    for lev in range(1, L + 1):
        K = (P >> (lev - 1)) // 2
        ops += 3 * K + 4 * (K - 1)
    return ops


def algorithmic_flops_per_lu(P, L, F=9):
    """Per lattice update of the D2Q9 compressed step: one inverse and one
    forward 2-D transform of every field (2 passes of E lines each), the BGK
    collision (135 operations, counted from the formula), the threshold test
    (|d| and a compare per coefficient)."""
    E = P + 1
    dwt = 2 * (2 * E * lifting_flops_per_line(P, L)) * F / (P * P)
    return dwt + 135 + 2 * F * E * E / (P * P)


def kernel_src_hash():
    """sha256 (first 16 hex) of the step kernel's sources with comments and
    blank lines removed: comment edits do not invalidate a profile."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ["common.cuh", "patch2d.cuh", "launch.cuh"]:
        src = open(os.path.join(ROOT, "paper_2302_09883_gb300", "csrc", f)).read()
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(md_name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    try:
        txt = open(os.path.join(ROOT, "profiles", md_name)).read()
    except OSError:
        return None
    tr, hs = None, None
    for line in txt.splitlines():
        if line.startswith("DRAM traffic per launch"):
            tr = int(line.split(":")[1].split()[0])
        if line.startswith("Kernel source hash"):
            hs = line.split(":")[-1].strip()
    return tr if hs == kernel_src_hash() else None


def cpu_oracle_mlups(w, seconds_target=10.0, prec=None, threads=0, n=512):
    """The oracle as it stands (OpenMP over patches) on a bounded sample of
    the workload: an n^2 periodic sub-problem with the same patch size,
    levels, storage and eps, stepped for about seconds_target.  prec: the
    oracle's arithmetic ("f32": the instantiation the GPU matches bit for
    bit; "f64": FP64 arithmetic and storage); threads: 0 = all host cores."""
    import oracle as O
    prec = prec or w["prec"]
    store = w["store"] if prec == "f32" else "f64"
    f = macro_fields(w, n=n)
    used = O.set_threads(threads)
    try:
        o = O.OracleSim("d2q9", w["wavelet"], n, n, w["P"], w["L"], w["eps"], prec=prec, store=store, tau=w["tau"])
        o.init_macro(f)
        t0 = time.perf_counter()
        o.step(1)
        per = time.perf_counter() - t0
        k = max(1, min(200, int(seconds_target / max(per, 1e-6))))
        t0 = time.perf_counter()
        o.step(k)
        dt = time.perf_counter() - t0
    finally:
        O.set_threads(0)
    return {"value": n * n * k / dt / 1e6, "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": "%d steps of a %dx%d periodic sub-problem (same P, L, eps), %s oracle%s" %
                      (k, n, n, prec.upper(), "" if prec == "f32" else " with F64 storage")}


def headline_config(w, eps):
    return {"workload": WORKLOAD, "grid": [w["n"], w["n"]], "P": w["P"], "levels": w["L"], "wavelet": "bl5/3",
            "store": w["store"], "eps": eps, "tau": w["tau"],
            "l2": "flushed (512 MB write) before each timed step", "parallelism": "single"}


def run_reference(args):
    """The oracle as it stands on the host cores, each step a bounded sample
    of the workload (a 512^2 periodic sub-problem, same P, L, storage and
    eps); rank 0 only."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = dict(inputs.WORKLOADS[WORKLOAD])
    import oracle as O
    n = 512
    f = macro_fields(w, n=n)
    o = O.OracleSim("d2q9", w["wavelet"], n, n, w["P"], w["L"], w["eps"], prec=w["prec"], store=w["store"],
                    tau=w["tau"])
    o.init_macro(f)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = n * n * args.steps / dt / 1e6
    cores = O.set_threads(0)
    sample = "each step: one FP32 oracle step of a %dx%d periodic sub-problem of the workload (same P, L, " \
             "storage, eps)" % (n, n)
    cfg = headline_config(w, w["eps"])
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                      "data": "synthetic", "config": cfg,
                      "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2302_09883_gb300 import Dense, Sim

    w = dict(inputs.WORKLOADS[WORKLOAD])
    n = w["n"]
    K, W = args.steps, max(3, args.warmup)
    lu = n * n
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    flops_lu = algorithmic_flops_per_lu(w["P"], w["L"])

    # 1-2. quality pass over the eps sweep; the headline eps is the
    # workload's (1e-3) when its errors are <= 1e-3, else the largest that passes
    flush = torch.empty(4 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    f = macro_fields(w)
    bs = torch.cuda.Stream()
    qsteps = args.quality_steps or w["steps"]
    # every eps of the sweep is timed for K steps from the state its quality
    # run ended in: the survivor-bearing points show the codec's cost
    sweep = quality_pass(torch, w, qsteps, EPS_SWEEP, timing=(K, flush, bs))
    ok = [q for q in sweep if q["rel_l2_u"] <= 1e-3 and q["rel_l2_rho"] <= 1e-3]
    head = next((q for q in ok if q["eps"] == w["eps"]), None) or \
        (max(ok, key=lambda q: q["eps"]) if ok else min(sweep, key=lambda q: q["rel_l2_u"]))
    eps = head["eps"]

    # 3. the headline: W warm-up steps from the initial state, then K timed
    # steps with the clocks sampled
    head_ms = None
    for q in [head]:
        sim = Sim("d2q9", w["wavelet"], n, n, w["P"], w["L"], q["eps"], prec=w["prec"], store=w["store"],
                  tau=w["tau"], stream=bs)
        sim.init_macro(f)
        sim.step(W)
        sim.sync()
        if q["eps"] == eps:
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            with ClockSampler(local) as clk:
                ms = timed_steps(torch, sim, bs, K, flush)
            clk_summary = clk.summary()
            sim.sync()
            torch.cuda.synchronize()
            if world > 1:
                ms = max_over_ranks(torch, ms, "cuda")
            head_ms = ms
            rb = roofline_bytes(sim, w)
            st = sim.stats()
            comp_bytes = sim.compressed_bytes()
            head_res = sim.resident_bytes()
            head_surv = sim.survivors()
            # warm (L2-resident, back-to-back launches) rate for context
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(bs):
                a.record(bs)
            sim.step(K)
            with torch.cuda.stream(bs):
                b.record(bs)
            bs.synchronize()
            warm_ms = a.elapsed_time(b)
        sim.sync()
        sim.close()
    ms = head_ms

    # uncompressed baseline, same timing rules
    d = Dense("d2q9", n, n, tau=w["tau"], stream=bs)
    d.init_macro(f)
    d.step(W)
    torch.cuda.synchronize()
    dms = timed_steps(torch, d, bs, K, flush)
    dense_bytes = d.nbytes()
    d.close()

    # e2e through the C-ABI with host buffers: host init (h2d), K steps with
    # the FP64 step statistics of every step read back (queued into pinned
    # memory behind the step and collected while the next step runs), final
    # field export (d2h); the simulation's device memory is set up before
    # the timed region
    host_f = [np.ascontiguousarray(x) for x in f]
    out = np.empty((9, n, n), np.float32)
    e = Sim("d2q9", w["wavelet"], n, n, w["P"], w["L"], eps, prec=w["prec"], store=w["store"], tau=w["tau"],
            stream=bs)
    e.init_macro(host_f)
    e.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e.init_macro(host_f)
    masses = []
    for k in range(K):
        e.step(1)
        e.stats_enqueue(k % 2)
        if k > 0:
            masses.append(e.stats_collect((k - 1) % 2)["mass"])
    masses.append(e.stats_collect((K - 1) % 2)["mass"])
    e.export_field(-1, out=out, dtype=np.float32)
    e2e_s = time.perf_counter() - t0
    e.close()
    assert len(masses) == K and all(np.isfinite(masses))
    h2d = sum(x.nbytes for x in host_f)
    d2h = out.nbytes + K * ((n // w["P"]) ** 2 * 9 * 8 + 88)

    def side(fn, *a, **kw):
        # a side section that fails reports its error in its own key (the
        # traceback goes to stderr) instead of taking the headline line down
        try:
            return fn(*a, **kw)
        except Exception as exc:  # noqa: BLE001
            import traceback
            traceback.print_exc()
            torch.cuda.synchronize()
            return {"error": "%s: %s" % (type(exc).__name__, exc)}

    euler = None
    if not args.no_euler:
        euler = side(euler_section, torch, K, W, flush, bs,
                     qsteps=None if args.quality_steps is None else args.quality_steps)

    batch = None
    if not args.no_batch:
        batch = side(batch_section, torch, K, W, flush, bs)

    learned_eps = None
    if not args.no_learned:
        learned_eps = side(learned_section, torch, K, W, flush, bs)

    transport = None
    if not args.no_transport:
        transport = side(transport_section, torch, K, W, flush, bs)

    swe = None
    if not args.no_swe:
        swe = side(swe_section, torch, bs)

    hilo = None
    if not args.no_hilo:
        hilo = side(hilo_section, torch, K, W, flush, bs, w, eps)

    d3q19 = None
    if not args.no_d3q19:
        d3q19 = side(d3q19_section, torch, min(K, 10), W, flush, bs, n_time=args.d3q19_n,
                     quality_steps=args.quality_steps or 1000)

    mlups = lu * K * world / (ms * 1e-3) / 1e6
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    launch_s = ms * 1e-3 / K
    clk = clk_summary
    sm_mhz = clk["sm_mhz"] or float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = nsm * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s, 128 FP32 lanes per SM, FMA = 2
    alu_achieved = flops_lu * lu / launch_s / 1e12
    traffic = profiled_traffic("patch_kernel_d2q9_bl53_2048.md")
    for q in sweep:  # ALU fraction against the clock sampled during the headline's timed steps
        q["alu_frac"] = flops_lu * lu / (q["ms_per_step"] * 1e-3) / 1e12 / fp32_peak
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cpu = cpu_oracle_mlups(dict(w, eps=eps))
            cpu["fp64_all_cores"] = cpu_oracle_mlups(dict(w, eps=eps), prec="f64")
            cpu["fp32_one_thread"] = cpu_oracle_mlups(dict(w, eps=eps), threads=1, n=256, seconds_target=8.0)
        except Exception as ex:
            cpu = {"value": None, "unit": "MLUPS", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "failed: %s" % ex}
    if rank == 0:
        cfg = headline_config(w, eps)
        cfg["parallelism"] = "replicas" if world > 1 else "single"
        line = {
            "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg,
            "compression_ratio": head["compression_ratio"],
            "resident_bytes": head_res, "resident_ratio": st["uncompressed_bytes"] / head_res,
            "resident_ratio_vs_dense_run": dense_bytes / head_res,
            "survivors_per_patch": head_surv / ((n // w["P"]) ** 2),
            "rel_l2": {"u": head["rel_l2_u"], "rho": head["rel_l2_rho"], "pop_max": head["rel_l2_pop_max"],
                       "steps": qsteps},
            "uncompressed_mlups": lu * K / (dms * 1e-3) / 1e6,
            # the dense step moves 72 B per update (9 populations read and written)
            "uncompressed_hbm": {"gbs": 72.0 * lu * K / (dms * 1e-3) / 1e9, "peak": hbm_peak,
                                 "frac": 72.0 * lu * K / (dms * 1e-3) / 1e9 / hbm_peak},
            "speed_vs_uncompressed": dms / ms,
            "warm_mlups": lu * K / (warm_ms * 1e-3) / 1e6,
            "sweep": sweep,
            "compressed_bytes": comp_bytes, "uncompressed_bytes": st["uncompressed_bytes"],
            "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": alu_achieved / fp32_peak, "traffic": traffic,
                         "traffic_source": ("ncu DRAM bytes per launch from profiles/patch_kernel_d2q9_bl53_2048.md "
                                            "(taken on the same kernel source)") if traffic else
                                           "none: the committed profile predates the current kernel source",
                         "flops_per_lu": flops_lu, "bytes_per_launch": rb["compulsory"],
                         "kernel": "patch_kernel<D2Q9,BL53,f32,BF16,64,4,STEP>",
                         "peak_source": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (median SM clock sampled "
                                        "during the timed steps)" % (nsm, sm_mhz),
                         "hbm": {"achieved": rb["compulsory"] / launch_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": rb["compulsory"] / launch_s / 1e9 / hbm_peak,
                                 "bytes": "compulsory: records read and written, tables, FP64 sums",
                                 "with_l2_reuse_bytes": rb["with_l2_reuse"],
                                 "with_l2_reuse_gbs": rb["with_l2_reuse"] / launch_s / 1e9,
                                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}},
            "clocks": clk_summary,
            "e2e": {"value": lu * K / e2e_s / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d / K,
                    "d2h_bytes_per_step": d2h / K,
                    "result_read": "FP64 mass of every step, collected while the next step runs"},
            "gpu_launches": K,
            "euler": euler,
            "batch": batch,
            "learned_eps": learned_eps,
            "d3q19": d3q19,
            "transport": transport,
            "swe": swe,
            "hilo": hilo,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
