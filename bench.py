#!/usr/bin/env python3
"""Benchmark of the GRFFE DG-FD hybrid step on GB300.

Workload: the FFE breakdown / current-sheet problem, box [-2,2]x[-0.25,0.25]^2,
64x8x8 elements at P=5 (884,736 LGL nodes; troubled elements on 11^3 subcells),
eta = 1e3, FP64.  A step is one IMEX-SSP3(4,3,3) step of the whole hybrid path:
3 right-hand sides + 4 stage solves, filter, indicator, rollback and FD<->DG
switching.  Metric: element-node updates per second (one DG node or FD cell
advanced through one explicit RHS and its stage update).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun every rank advances its own
replica (weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ffe_workloads as W  # noqa: E402

METRIC = "RHS element-node updates/s FP64 at 1 GB300, % roofline; adjoint/forward time"
UNIT = "element-node updates/s"
# DRAM bytes (read + write) of k_fd_flux per FD element it processes, from an
# ncu capture of the kernel on the 8x8x8 breakdown box: a launch moves this
# many bytes for each element of its chunk (scaled to a launch of this run by
# its FD element count)
DRAM_BYTES_PER_FD_ELEMENT = {"fd_flux": 5.535e5}
TRAFFIC_SOURCE = ("scaled: 553.5 KB of DRAM traffic per FD element (ncu dram__bytes_read.sum + "
                  "dram__bytes_write.sum of k_fd_flux on the 8x8x8 breakdown box) x FD elements per launch")

RECON = {"weno5z": 0, "mp5": 1}

CPU_SAMPLE = dict(nx=16, ny=2, nz=2, x_half=0.5)
CPU_SAMPLE_TEXT = ("oracle (numpy fp64, 1 thread) on a 16x2x2-element slab of the breakdown "
                   "workload (same element width, order and current sheet), whole hybrid steps")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_ranks(ms, units, dist, device):
    """Whole-job timing over the replicas: the slowest rank's time and the sum of
    the units every rank advanced (one replica per rank, no exchange)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.item(), u.item()


def cpu_oracle_rate(steps, budget_s=None):
    """Time the oracle, as it stands, on the bounded sample (1 thread)."""
    from oracle.problem import Problem
    from oracle.stepper import Stepper
    import numpy as np
    cfg = W.breakdown(**CPU_SAMPLE)
    pr = Problem(cfg)
    st = pr.initial_state()
    S = Stepper(pr)
    nn, nc = (cfg["P"] + 1) ** 3, (2 * cfg["P"] + 1) ** 3
    units, t0, done = 0, time.perf_counter(), 0
    for _ in range(steps):
        fd = int(st["mask"].sum())
        st = S.step(st)
        units += 3 * ((pr.disc.E - fd) * nn + fd * nc)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return units / dt, dt, done


def _oracle_procs(n_proc, steps, budget_s):
    """Start n_proc fresh single-threaded interpreters (no CUDA), each timing
    the oracle on its own copy of the sample."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "r, dt, n = bench.cpu_oracle_rate(%d, %r); print(json.dumps([r, dt, n]))" % (ROOT, steps, budget_s))
    return [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                             text=True) for _ in range(n_proc)]


def _collect(procs):
    res = []
    for p in procs:
        out, err = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError(err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    return res


def cpu_baseline_subprocess(steps, budget_s):
    """Run the oracle timing in a fresh single-threaded interpreter (spawned, no CUDA)."""
    r, dt, n = _collect(_oracle_procs(1, steps, budget_s))[0]
    return r, dt, n


def cpu_baseline_all_cores(steps, budget_s):
    """The oracle on every host core: one single-threaded interpreter per core
    (os.cpu_count()), each advancing its own copy of the sample (independent
    slabs, like elements split over cores); rate = all their element-node
    updates / the longest wall time."""
    n = os.cpu_count() or 1
    res = _collect(_oracle_procs(n, steps, budget_s))
    units = sum(r * dt for r, dt, _ in res)
    wall = max(dt for _, dt, _ in res)
    return units / wall, wall, min(k for _, _, k in res), n


class Clocks:
    """nvidia-smi sampler for the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nme, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(nme)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    per_step_budget = None
    for _ in range(args.warmup):
        pass
    r, dt, n = cpu_baseline_subprocess(args.steps + args.warmup, per_step_budget)
    line = {"impl": "reference", "metric": METRIC, "value": r, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "breakdown 16x2x2 slab (oracle sample)", "P": 5},
            "cpu_baseline": {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": CPU_SAMPLE_TEXT + f", {n} steps in {dt:.1f} s"},
            "e2e": {"value": r, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_wald(args):
    """The Wald workload (Kerr-Schild a = 0.9, 6 wedges x 8x8x16, P = 5,
    r in [1.5, 50], exact Wald field, Dirichlet at both ends) for 1000 steps
    with the troubled-cell indicator on: step time and rate, the paper's L2
    error of B~ against the exact field (Sec. IV.B.1) at steps 100, 500 and
    1000, the RMS of the divergence-cleaning fields psi~, phi~ (constraint
    monitors) and the FD population."""
    import torch
    from paper_2404_01531_gb300 import ffe
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg = W.wald()
    cfg["params"]["tci_on"] = 1
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows, done, ms_total, u0 = [], 0, 0.0, ctx.info().node_updates
    for target in (100, 500, 1000):
        torch.cuda.synchronize()
        e0.record(st)
        ctx.step(target - done)
        e1.record(st)
        torch.cuda.synchronize()
        ms_total += e0.elapsed_time(e1)
        done = target
        l2, n = ctx.diagnostic("l2_err")
        rows.append({"step": target, "t": ctx.info().t, "l2_B": l2, "rms_psi": ctx.diagnostic("l2_err", (6, 1))[0],
                     "rms_phi": ctx.diagnostic("l2_err", (7, 1))[0], "fd_elements": ctx.info().n_fd_elem})
    units = ctx.info().node_updates - u0
    line = {"metric": METRIC, "value": units / (ms_total / 1e3), "unit": UNIT, "n_gpus": 1, "steps": done,
            "warmup": 0, "ms_per_step": ms_total / done, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Wald field, Kerr-Schild M=1 a=0.9, 6 wedges x 8x8x16, P=5, r in [1.5, 50], eta=0, "
                                   "indicator on", "elements": ctx.n_elem},
            "wald": rows, "status_bits": ctx.status()}
    ctx.close()
    print(json.dumps(line), flush=True)


def run_wald_vacuum(args):
    """The paper's vacuum Wald problem (Sec. IV.B.2) at its grid (16 x 96
    elements, P = 5, spherical Kerr-Schild radius r in [M, 125 M]): Wald's
    magnetic field with E~ = 0 at t = 0, eta = 0, evolved to t = 125 M for
    several spins; the flux of B~ through the upper half of the outer horizon
    (FFE_DIAG_BFLUX_UPPER on the coordinate surface r = r+) at t = 25, 50, 75,
    100, 125 M against the closed form pi r+^2 B0 (1 - a^4/r+^4) of the
    stationary state (King et al.), and the RMS of psi~ and phi~."""
    import math
    import torch
    from paper_2404_01531_gb300 import ffe
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rows = []
    for a in args.spins:
        cfg = W.wald_vacuum(spin=a)
        ctx = ffe.Context(cfg)
        ctx.set_initial()
        dt = ctx.dt
        rp = 1.0 + math.sqrt(1.0 - a * a)
        king = math.pi * rp * rp * (1.0 - a ** 4 / rp ** 4)
        flux0 = ctx.diagnostic("bflux_upper", (rp,))[0]
        series, done = [], 0
        t0 = time.perf_counter()
        for tt in (25.0, 50.0, 75.0, 100.0, cfg["t_end"]):
            n = int(round(tt / dt))
            ctx.step(n - done)
            done = n
            series.append({"t": n * dt, "flux": ctx.diagnostic("bflux_upper", (rp,))[0],
                           "rms_psi": ctx.diagnostic("l2_err", (6, 1))[0],
                           "rms_phi": ctx.diagnostic("l2_err", (7, 1))[0]})
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        rows.append({"spin": a, "r_plus": rp, "dt": dt, "steps": done, "king": king, "flux_t0": flux0,
                     "series": series, "rel_err_end": series[-1]["flux"] / king - 1.0, "wall_s": wall,
                     "status_bits": ctx.status()})
        ctx.close()
    line = {"metric": "horizon magnetic flux / closed form, vacuum Wald (Sec. IV.B.2)",
            "value": max(abs(r["rel_err_end"]) for r in rows), "unit": "max relative deviation at t_end",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "vacuum Wald: Kerr-Schild M=1, Wald B with E=0 at t=0, eta=0, 6 wedges x 4x4x16, "
                                   "P=5, spherical Kerr-Schild r in [1, 125], outflow between the horizons, no "
                                   "incoming Poynting flux outside, t_end = 125"},
            "runs": rows}
    print(json.dumps(line), flush=True)


def run_inclination(args):
    """The oblique rotator's spin-down luminosity against inclination (Sec.
    IV.C.2): rotating conducting star of radius R = 1 with the regularised
    dipole (mu = 1, delta = 0.1 R), Omega = 1/(5 R), eta = 1e5 / R, on a
    6-wedge shell r in [R, 20 R] (n_ang x n_ang x n_rad per wedge, P = 5, CFL
    0.25, indicator on unless --no-tci); one context per inclination chi, all advanced
    together on their own CUDA streams, for two rotation periods; L through
    r = 6 R (FFE_DIAG_LUMINOSITY) every eighth of a period.  Fits
    L = L0 (k1 + k2 sin^2 chi) with L0 = L(chi = 0) (least squares over the
    inclinations, on the mean of L over the last half period) and reports
    L0 / (4 pi mu^2 Omega^4): the equations are in Heaviside-Lorentz units
    (energy density (E^2 + B^2)/2, Poynting flux E x B), where the dipole
    moment mu is the Gaussian one over sqrt(4 pi), so the force-free aligned
    rotator's mu_G^2 Omega^4 (c = 1) reads 4 pi mu^2 Omega^4 here."""
    import math
    import numpy as np
    import torch
    from paper_2404_01531_gb300 import ffe
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    r_lc, mu, r_L = 5.0, 1.0, 6.0
    period = 2.0 * math.pi * r_lc
    cfgs = []
    for chi in args.chis:
        cfg = W.pulsar(r_lc=r_lc, chi=math.radians(chi), n_ang=args.n_ang, n_rad=args.n_rad, P=5, mu=mu,
                       r_out=4.0 * r_lc)
        if args.no_tci:
            cfg["params"]["tci_on"] = 0
        cfgs.append(cfg)
    ctxs, streams = [], []
    if args.batch:
        # every inclination an instance of one batched context: one launch per
        # kernel and substep for all of them
        b = ffe.BatchContext(cfgs, fd_capacity=1 if args.no_tci else 0)
        b.set_initial()
        b.step(1)
        torch.cuda.synchronize()
        ctxs.append(b)
        streams.append(b.stream)
        first = b.layout()[3]

        def sample(i):
            L_i = b.diagnostic("luminosity", (r_L, i))[0]   # synchronises the batch's stream
            m = b.mask().cpu().numpy()
            return L_i, int(m[first[i]:first[i + 1]].sum())
    else:
        for cfg in cfgs:
            s = torch.cuda.Stream()
            ctx = ffe.Context(cfg, stream=s)
            ctx.set_initial()
            ctx.step(1)            # first step: launch-shape tuning, alone on the GPU
            torch.cuda.synchronize()
            ctxs.append(ctx)
            streams.append(s)

        def sample(i):
            return ctxs[i].diagnostic("luminosity", (r_L,))[0], ctxs[i].info().n_fd_elem
    dt = ctxs[0].dt   # the instances differ only in chi: one grid, one time step
    n_total = int(round(args.periods * period / dt))
    marks = [int(round(k * period / 8 / dt)) for k in range(1, int(round(8 * args.periods)) + 1)]
    series = [[] for _ in cfgs]
    done, t0 = 1, time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(torch.cuda.current_stream())
    for m in marks:
        # interleave the contexts in short runs of steps so that every stream
        # has work queued while the host enqueues the others
        for k in range(done, m, 16):
            for ctx in ctxs:
                ctx.step(min(16, m - k))
        done = m
        t_now = ctxs[0].info().t
        for i in range(len(cfgs)):
            L_i, nfd_i = sample(i)
            series[i].append({"t": t_now, "L": L_i, "fd_elements": nfd_i})
        el = time.perf_counter() - t0
        print(json.dumps({"progress_t": series[0][-1]["t"], "wall_s": round(el, 1),
                          "L": [ser[-1]["L"] for ser in series],
                          "fd_elements": [ser[-1]["fd_elements"] for ser in series]}), file=sys.stderr, flush=True)
        if el > args.wall_budget:
            break
    for s in streams:
        torch.cuda.current_stream().wait_stream(s)
    e1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    wall = time.perf_counter() - t0
    rows = []
    reached = series[0][-1]["t"] / period
    status = [c.status() for c in ctxs]
    for i, (chi, ser) in enumerate(zip(args.chis, series)):
        tail = [p["L"] for p in ser if p["t"] >= (reached - 0.5) * period - 1e-9]
        rows.append({"chi_deg": chi, "L_end": ser[-1]["L"], "L_mean_last_half_period": float(np.mean(tail)),
                     "fd_elements_end": ser[-1]["fd_elements"],
                     "status_bits": status[0] if args.batch else status[i], "series": ser})
    L = np.array([r["L_mean_last_half_period"] for r in rows])
    chis = np.radians(np.array(args.chis))
    i0 = int(np.argmin(np.abs(chis)))
    A = np.stack([np.ones_like(chis), np.sin(chis) ** 2], axis=1)
    k1, k2 = np.linalg.lstsq(A, L / L[i0], rcond=None)[0]
    units = sum(c.info().node_updates for c in ctxs)
    line = {"metric": "oblique rotator spin-down luminosity vs inclination (Sec. IV.C.2)",
            "value": float(k2), "unit": "k2 of L = L0 (k1 + k2 sin^2 chi)", "k1": float(k1), "k2": float(k2),
            "L0_over_4pi_mu2_omega4": float(L[i0] / (4.0 * math.pi * mu ** 2 * (1.0 / r_lc) ** 4)),
            "n_gpus": 1, "higher_is_better": None, "dtype": "f64", "data": "synthetic",
            "steps": done, "steps_planned": n_total, "periods_reached": reached, "dt": dt,
            "ms_per_step_all_contexts": ms / max(done - 1, 1), "wall_s": wall,
            "node_updates_per_s": units / (ms / 1e3),
            "config": {"workload": f"oblique rotator: star R=1, mu=1, delta=0.1, Omega=1/5, eta=1e5, 6 wedges x "
                                   f"{args.n_ang}x{args.n_ang}x{args.n_rad}, P=5, r in [1, 20], CFL 0.25, "
                                   f"indicator {'off (DG and filter only)' if args.no_tci else 'on'}, "
                                   f"{args.periods} periods, L at r=6",
                       "inclinations_deg": args.chis,
                       "contexts": "one batched context, an instance per inclination" if args.batch
                       else "one per inclination, concurrent streams"},
            "runs": rows}
    for c in ctxs:
        c.close()
    print(json.dumps(line), flush=True)


def run_shell(args):
    """The neutron-star shell (6 wedges x 6x6x12, P=5, eta=1e5) with its three
    innermost radial layers on FD subcells and the mask frozen: an FD-heavy
    curved-mesh step (subcell fluxes of every physical component at every face)."""
    import torch
    from paper_2404_01531_gb300 import ffe
    from paper_2404_01531_gb300.roofline import FP64_PEAK_TFLOPS, fd_faces_per_element, fd_flux_flops
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg = W.adjoint_pulsar(steps=args.steps)
    cfg["params"].update(tci_on=0, recon=RECON[args.recon])
    ctx = ffe.Context(cfg)
    U, m = ctx.state()
    e = torch.arange(ctx.n_elem, device=m.device)
    na, nr = cfg["n_ang"], cfg["n_rad"]
    mask = ((e // (na * na)) % nr < 3).to(torch.uint8)
    ctx.set_state(U.clone(), mask)
    ctx.set_initial(keep_mask=True)
    ctx.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    i0 = ctx.info()
    e0.record(st)
    ctx.step(args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    i1 = ctx.info()
    ctx.set_profiling(True)
    j0 = ctx.info()
    ctx.step(args.steps)
    j1 = ctx.info()
    ctx.set_profiling(False)
    prof = ctx.profile_read()
    n_fd = j1.fd_elem_updates - j0.fd_elem_updates
    fl = n_fd * fd_faces_per_element(ctx.P) * fd_flux_flops(RECON[args.recon])
    ach = fl / (prof["fd_flux"][1] / 1e3) / 1e12
    line = {"metric": METRIC, "value": (i1.node_updates - i0.node_updates) / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "neutron-star shell 6 wedges x 6x6x12 P=5, eta=1e5, three inner radial layers "
                                   "on FD (frozen mask)", "elements": ctx.n_elem, "fd_elements": int(mask.sum()),
                       "recon": args.recon},
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_PEAK_TFLOPS, "kernel": "fd_flux (k_fd_flux_curved)",
                         "units": {"fd_elem_updates": n_fd}},
            "kernel_ms": {k: v[1] / max(v[0], 1) for k, v in prof.items()},
            "kernel_max_ms": {k: v[2] for k, v in prof.items()}, "status_bits": ctx.status()}
    ctx.close()
    print(json.dumps(line), flush=True)


def _oned_profile(test, x):
    """Exact or reference profile b(x) of the paper's 1-D data (App. A)."""
    import numpy as np
    if test == "fast_wave_kink":
        return np.where(x < -0.1, 1.0, np.where(x > 0.1, 0.7, 0.85 - 1.5 * x))
    if test == "alfven":
        return np.where(x < -0.1, 1.0, np.where(x > 0.1, 1.3, 1.15 + 0.15 * np.sin(5.0 * np.pi * x)))
    raise ValueError(test)


def _oned_points(ctx, U, mask):
    """Values [9][n] and x [n] of the representation each element uses (DG nodes
    of DG elements, subcell centres of FD elements)."""
    import numpy as np
    xd, xf = ctx.coords()
    dg, fd = ctx.split(U)
    xd = xd.cpu().numpy().reshape(3, ctx.n_elem, -1)[0]
    xf = xf.cpu().numpy().reshape(3, ctx.n_elem, -1)[0]
    dg = dg.reshape(9, ctx.n_elem, -1)
    fd = fd.reshape(9, ctx.n_elem, -1)
    on_dg, on_fd = mask == 0, mask == 1
    vals = np.concatenate([dg[:, on_dg].reshape(9, -1), fd[:, on_fd].reshape(9, -1)], axis=1)
    xs = np.concatenate([xd[on_dg].reshape(-1), xf[on_fd].reshape(-1)])
    return vals, xs


def oned_measure(levels=(0, 1, 2, 3)):
    """The paper's 1-D tests (Sec. IV.A, Table I, App. A) to their end times at
    resolution levels n (32 2^n elements): step time, element-node update rate
    and the errors the paper plots -- fast wave against its exact translation,
    Alfven wave against the stationary profile, breakdown through B^2 - E^2 and
    E.B -- plus the fast wave from the FD start."""
    import numpy as np
    import torch
    from paper_2404_01531_gb300 import ffe
    out = []
    runs = [(t, n, False) for t in W.ONED for n in levels] + [("fast_wave_kink", 0, True)]
    for test, n, via in runs:
        cfg = W.oned(test, n, via_fd=via)
        ctx = ffe.Context(cfg)
        ctx.set_initial()
        fd0 = int(ctx.download()[1].sum())
        ctx.step(2)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        i0 = ctx.info()
        e0.record(st)
        ctx.step(cfg["steps"] - 2)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        i1 = ctx.info()
        U, mask = ctx.download()
        vals, xs = _oned_points(ctx, U, mask)
        t = cfg["steps"] * cfg["params"]["dt"]
        r = {"test": test, "level": n, "elements_x": cfg["n"][0], "steps": cfg["steps"], "t_end": t,
             "fd_start": via, "fd_elements_start": fd0, "fd_elements_end": int(mask.sum()),
             "ms_per_step": ms / (cfg["steps"] - 2),
             "node_updates_per_s": (i1.node_updates - i0.node_updates) / (ms / 1e3), "status_bits": ctx.status()}
        if test == "fast_wave_kink":
            b = _oned_profile(test, xs - t)
            err = np.abs(vals[2] + b)
            far = (np.abs(xs - t - 0.1) > 0.15) & (np.abs(xs - t + 0.1) > 0.15)
            r.update(err_Ez_max=float(err.max()), err_Ez_mean=float(err.mean()), err_Ez_max_far_from_kinks=float(err[far].max()))
        elif test == "alfven":
            b = _oned_profile(test, xs)
            r.update(dev_Bz_max=float(np.abs(vals[5] - b).max()), dev_Bz_mean=float(np.abs(vals[5] - b).mean()),
                     dev_Ex_max=float(np.abs(vals[0] + b).max()))
        else:
            E, B = vals[0:3], vals[3:6]
            r.update(min_B2_minus_E2=float(((B * B).sum(0) - (E * E).sum(0)).min()),
                     max_abs_EdotB=float(np.abs((E * B).sum(0)).max()))
        ctx.close()
        out.append(r)
    return out


def split_measure(steps=20, warmup=3):
    """The paper's efficiency experiment (Sec. IV.A.4): the stationary Alfven
    wave on (8, 32, 8) elements with the elements below a y row forced onto FD
    and the rest on DG (indicator off, mask frozen); step time against the FD
    fraction x, the speedup over all-FD and the factor f of the model
    1 / (x + (1 - x)/f) fitted to the mixed runs."""
    import torch
    from paper_2404_01531_gb300 import ffe
    h = 3.0 / 8
    cfg = W.oned("alfven", 0)
    cfg.update(lo=(-1.5, -16 * h, -4 * h), hi=(1.5, 16 * h, 4 * h), n=(8, 32, 8))
    cfg["params"].update(tci_on=0)
    ctx = ffe.Context(cfg)
    U, m = ctx.state()
    E = ctx.n_elem
    yc = ctx.coords()[0].view(3, E, -1)[1].mean(1)   # element centres in y
    rows = []
    for k in (32, 16, 6, 3, 2, 1, 0):
        mask = (yc < -16 * h + k * h).to(torch.uint8)
        ctx.set_state(U.clone(), mask)
        ctx.set_initial(keep_mask=True)
        ctx.step(warmup)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        i0 = ctx.info()
        e0.record(st)
        ctx.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        i1 = ctx.info()
        rows.append({"fd_rows": k, "fd_fraction": k / 32, "ms_per_step": ms,
                     "node_updates_per_s": (i1.node_updates - i0.node_updates) / (ms * steps / 1e3),
                     "status_bits": ctx.status()})
        U, m = ctx.state()
    ctx.close()
    t_fd = rows[0]["ms_per_step"]
    for r in rows:
        r["speedup_over_all_fd"] = t_fd / r["ms_per_step"]
    mixed = [r for r in rows if 0 < r["fd_fraction"] < 1]
    # 1/s - x = (1 - x)/f, least squares in 1/f
    num = sum((1 - r["fd_fraction"]) * (1 / r["speedup_over_all_fd"] - r["fd_fraction"]) for r in mixed)
    den = sum((1 - r["fd_fraction"]) ** 2 for r in mixed)
    return {"elements": E, "rows": rows, "f_all_dg": t_fd / rows[-1]["ms_per_step"], "f_fit_mixed": den / num}


def run_dg_phases(args):
    """Cost of the optional phases of the box DG substep kernel: the smooth fast
    wave on 16^3 elements (all DG, nothing flagged), the kernel's average launch
    time with the filter, the indicator and the driver current each switched
    off through ffe_params (physics changed; timing only)."""
    import torch
    from paper_2404_01531_gb300 import ffe
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rows = {}
    for label, prm in (("all_on", {}), ("indicator_off", dict(tci_on=0)), ("filter_off", dict(filter_on=0)),
                       ("eta_0", dict(eta=0.0)), ("all_off", dict(tci_on=0, filter_on=0, eta=0.0))):
        cfg = W.fast_wave(n=16)
        cfg["params"].update(prm)
        ctx = ffe.Context(cfg)
        ctx.set_initial()
        ctx.step(max(args.warmup, 3))
        torch.cuda.synchronize()
        ctx.set_profiling(True)
        ctx.step(6)
        ctx.set_profiling(False)
        p = ctx.profile_read()
        rows[label] = p["dg_substep"][1] / p["dg_substep"][0]
        ctx.close()
    line = {"metric": "k_dg_substep average launch time", "value": rows["all_on"], "unit": "ms",
            "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fast wave, periodic 16^3 elements, P=5, all DG"}, "dg_substep_ms": rows}
    print(json.dumps(line), flush=True)


def run_oned(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    o = oned_measure()
    sp = split_measure(steps=args.steps if args.steps != 50 else 20, warmup=max(args.warmup, 3))
    ten = min(sp["rows"], key=lambda r: abs(r["fd_fraction"] - 0.1))
    line = {"metric": METRIC, "value": ten["node_updates_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ten["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper's 1-D tests (Table I, levels 0-3, to their end times) and the Alfven "
                                   "DG/FD split on (8,32,8) elements (value: the run nearest 10% FD)",
                       "fd_fraction": ten["fd_fraction"]},
            "oned": o, "split": sp}
    print(json.dumps(line), flush=True)


def run_pulsars(args):
    """Batched shells: one launch per kernel and substep for every instance,
    against the same instances advanced one context at a time.  Under
    torchrun the batch is split by whole instances over the ranks
    (partition.assign_instances; no exchange on the data path): each rank
    advances its own batched context, the timing is the slowest rank's and the
    units are summed (fixed total work: strong scaling)."""
    import torch
    from paper_2404_01531_gb300 import ffe
    from paper_2404_01531_gb300.partition import instances_of
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfgs_all = W.pulsars(n_inst=args.n_inst)
    mine = instances_of(cfgs_all, ws, rank)
    cfgs = [cfgs_all[i] for i in mine]
    E = sum(6 * c["n_ang"] ** 2 * c["n_rad"] for c in cfgs)
    E_all = sum(6 * c["n_ang"] ** 2 * c["n_rad"] for c in cfgs_all)
    b = ffe.BatchContext(cfgs, fd_capacity=int(args.fd_capacity * E))
    b.set_initial()
    b.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    u0 = b.info().node_updates
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(st)
    b.step(args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_b = e0.elapsed_time(e1)
    inf = b.info()
    units_b = inf.node_updates - u0
    ms_max, units_all = combine_ranks(ms_b, units_b, dist, "cuda")
    fd_end = inf.n_fd_elem
    status = b.status()
    b.set_profiling(True)
    b.step(2)
    b.set_profiling(False)
    prof = b.profile_read()
    b.close()
    vb = units_all / (ms_max / 1e3)
    single = None
    if ws == 1:
        # one context per instance, same steps, timed one after the other
        ms_s, units_s = 0.0, 0
        for c in cfgs:
            s1 = ffe.Context(c)
            s1.set_initial()
            s1.step(max(args.warmup, 3))
            torch.cuda.synchronize()
            u0 = s1.info().node_updates
            e0.record(st)
            s1.step(args.steps)
            e1.record(st)
            torch.cuda.synchronize()
            ms_s += e0.elapsed_time(e1)
            units_s += s1.info().node_updates - u0
            s1.close()
        vs = units_s / (ms_s / 1e3)
        single = {"value": vs, "ms_per_step": ms_s / args.steps}
    if rank == 0:
        line = {"metric": METRIC, "value": vb, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"pulsars: {len(cfgs_all)} rotating-dipole shells (seed 1531), P in {{4,5}}",
                           "elements": E_all, "fd_elements_end_rank0": fd_end,
                           "fd_capacity": int(args.fd_capacity * E),
                           "parallelism": f"whole instances over {ws} ranks" if ws > 1 else "one batched context"},
                "one_instance_per_launch": single,
                "batched_over_single": vb / single["value"] if single else None,
                "kernel_ms": {k: v[1] / max(v[0], 1) for k, v in prof.items()}, "status_bits": status}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def batch_measure(n_inst=32, steps=3, warmup=2, fd_capacity=0.5):
    """The batched workload (n_inst rotating-dipole shells, seed 1531) for a
    few steps: one batched context (one launch per kernel and substep for every
    instance) against one context per instance advanced one after the other;
    node updates per second of each and their ratio."""
    import torch
    from paper_2404_01531_gb300 import ffe
    cfgs = W.pulsars(n_inst=n_inst)
    E = sum(6 * c["n_ang"] ** 2 * c["n_rad"] for c in cfgs)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b = ffe.BatchContext(cfgs, fd_capacity=int(fd_capacity * E))
    b.set_initial()
    b.step(warmup)
    torch.cuda.synchronize()
    u0 = b.info().node_updates
    e0.record(st)
    b.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    units_b = b.info().node_updates - u0
    tuned = list(b.info().dg_ctas_per_sm)
    status = b.status()
    b.close()
    ms_s, units_s = 0.0, 0
    for c in cfgs:
        s1 = ffe.Context(c)
        s1.set_initial()
        s1.step(warmup)
        torch.cuda.synchronize()
        u0 = s1.info().node_updates
        e0.record(st)
        s1.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        ms_s += e0.elapsed_time(e1)
        units_s += s1.info().node_updates - u0
        s1.close()
    vb, vs = units_b / (ms_b / 1e3), units_s / (ms_s / 1e3)
    return {"workload": f"{n_inst} rotating-dipole shells (seed 1531), {E} elements, P in {{4,5}}, {steps} steps",
            "batched_value": vb, "batched_ms_per_step": ms_b / steps, "single_value": vs,
            "single_ms_per_step": ms_s / steps, "batched_over_single": vb / vs,
            "dg_ctas_per_sm_by_order": dict(zip(("P5", "P4", "P3"), tuned)), "status_bits": status}


def adjoint_measure(steps=500, every=25, r_L=20.0, fd_check=False):
    """Neutron-star shell 6 wedges x 6x6x12 at P=5: time of `steps` forward steps
    (graph replays) against the checkpointed gradient of the time-averaged
    luminosity through r = r_L w.r.t. (mu, chi, Omega); optionally the gradient
    against central differences of the forward run (relative step 1e-6)."""
    import torch
    from paper_2404_01531_gb300 import ffe
    from paper_2404_01531_gb300.adjoint import lbar_forward, luminosity_gradient
    from paper_2404_01531_gb300.adjoint import freeze_union_mask
    cfg = W.adjoint_pulsar(steps=steps)
    cfg["params"].update(tci_on=1)
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    t_m = time.perf_counter()
    union = freeze_union_mask(ctx, steps)      # mask frozen from the indicator-on forward pass
    torch.cuda.synchronize()
    t_m = time.perf_counter() - t_m
    U0, m0 = (t.clone() for t in ctx.state())
    st = torch.cuda.current_stream()
    ctx.step(3)
    ctx.set_state(U0, m0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    ctx.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    # one adjoint step alone (stage recomputation + reverse), same state
    lam = torch.randn(U0.shape, dtype=torch.float64, device="cuda")
    out = torch.empty_like(lam)
    for _ in range(3):
        ctx.adjoint_step(U0, lam, out)
    k = 20
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(k):
        ctx.adjoint_step(U0, lam, out)
    e1.record(st)
    torch.cuda.synchronize()
    adj_ms = e0.elapsed_time(e1) / k
    # the backward sweep alone, with the step's stages kept in device memory
    stages = torch.empty(5 * U0.numel(), dtype=U0.dtype, device=U0.device)
    ctx.adjoint_forward(U0, stages, None)
    for _ in range(3):
        ctx.adjoint_reverse(U0, stages, lam, out)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(k):
        ctx.adjoint_reverse(U0, stages, lam, out)
    e1.record(st)
    torch.cuda.synchronize()
    rev_ms = e0.elapsed_time(e1) / k
    # where the backward sweep's time goes (eager, per-kernel events)
    ctx.set_profiling(True)
    ctx.adjoint_reverse(U0, stages, lam, out)
    ctx.set_profiling(False)
    rev_prof = {kk: v[1] for kk, v in ctx.profile_read().items()}
    del stages
    ctx.set_state(U0, m0)
    L, g, tm = luminosity_gradient(ctx, steps, r_L=r_L, every=every)
    ctx.close()
    res = {"workload": f"rotating dipole (mu, chi, Omega) = (1, 45 deg, 1/6), shell r in [1, 24], "
                       f"6 wedges x 6x6x12 elements P=5, eta=1e5, {steps} steps, checkpoint every {every}, "
                       f"mask frozen as the union of the indicator's masks over a forward pass",
           "fd_elements": int(union.sum()), "mask_pass_s": t_m,
           "forward_ms_per_step": fwd_ms / steps, "adjoint_step_ms": adj_ms,
           "adjoint_step_over_forward_step": adj_ms / (fwd_ms / steps),
           "adjoint_reverse_ms": rev_ms, "adjoint_reverse_over_forward_step": rev_ms / (fwd_ms / steps),
           "reverse_kernel_ms": rev_prof,
           "gradient_s": tm["forward_s"] + tm["adjoint_s"], "forward_s": fwd_ms / 1e3,
           "gradient_over_forward": (tm["forward_s"] + tm["adjoint_s"]) / (fwd_ms / 1e3),
           "Lbar": L, "grad": g}
    if fd_check:
        kind, kw = cfg["initial"]
        base = {"mu": kw["mu"], "chi": kw["chi"], "omega": cfg["params"]["omega_star"]}
        fd = []
        for name in ("mu", "chi", "omega"):
            h = 1e-6 * base[name]
            vals = []
            for sgn in (1, -1):
                c = dict(cfg)
                c["params"] = dict(cfg["params"])
                kw2 = dict(kw)
                if name == "omega":
                    c["params"]["omega_star"] = base[name] + sgn * h
                else:
                    kw2[name] = base[name] + sgn * h
                c["initial"] = (kind, kw2)
                cx = ffe.Context(c)
                cx.set_state(cx.state()[0].clone(), union)
                cx.set_initial(keep_mask=True)
                cx.freeze_mask(True)
                vals.append(lbar_forward(cx, steps, r_L))
                cx.close()
            fd.append((vals[0] - vals[1]) / (2 * h))
        res["grad_central_differences"] = fd
        res["max_rel_err_vs_fd"] = max(abs(a - b) / abs(b) for a, b in zip(g, fd))
    return res


def run_adjoint(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    r = adjoint_measure(steps=args.steps, every=25, fd_check=True)
    line = {"metric": METRIC, "value": r["adjoint_reverse_over_forward_step"],
            "unit": "adjoint step (stages kept in HBM) / forward step",
            "n_gpus": 1, "steps": args.steps, "warmup": 3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": r.pop("workload")},
            "adjoint": r}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nx", type=int, default=64,
                    help="elements along x (same width 4/64; smaller values for profiler captures)")
    ap.add_argument("--workload", default="breakdown",
                    choices=["breakdown", "pulsars", "adjoint", "shell", "oned", "dgphases", "wald", "wald_vacuum",
                             "inclination"],
                    help="pulsars: the 32-shell batch, batched launch vs one context per instance; "
                         "adjoint: luminosity gradient of one neutron-star shell (--steps steps); "
                         "shell: that shell with three FD layers, frozen mask (curved FD kernels); "
                         "oned: the paper's 1-D tests and its DG/FD split experiment; "
                         "dgphases: cost of the DG kernel's filter, indicator and stiff-current phases; "
                         "wald: the Kerr-Schild Wald shell, 1000 steps, indicator on; "
                         "wald_vacuum: horizon flux against spin (Sec. IV.B.2); "
                         "inclination: oblique rotator luminosity against inclination (Sec. IV.C.2)")
    ap.add_argument("--no-adjoint", action="store_true", help="breakdown: skip the adjoint/forward timing")
    ap.add_argument("--no-batch", action="store_true",
                    help="breakdown: skip the batched-against-single timing of the 32-shell batch")
    ap.add_argument("--no-split", action="store_true",
                    help="breakdown: skip the DG/FD split experiment (Alfven wave on (8,32,8) elements)")
    ap.add_argument("--recon", default="weno5z", choices=list(RECON),
                    help="breakdown and shell: FD reconstruction (the paper's WENO5-Z, or MP5)")
    ap.add_argument("--n-inst", type=int, default=32)
    ap.add_argument("--spins", type=float, nargs="+", default=[0.0, 0.5, 0.7, 0.9, 0.999],
                    help="wald_vacuum: black-hole spins")
    ap.add_argument("--chis", type=float, nargs="+", default=[0.0, 30.0, 60.0, 90.0],
                    help="inclination: magnetic inclinations in degrees")
    ap.add_argument("--periods", type=float, default=2.0, help="inclination: rotation periods to evolve")
    ap.add_argument("--batch", action="store_true",
                    help="inclination: all inclinations as instances of one batched context")
    ap.add_argument("--no-tci", action="store_true",
                    help="inclination: indicator off, every element on DG (with the filter)")
    ap.add_argument("--wall-budget", type=float, default=900.0,
                    help="inclination: stop at the first eighth of a period after this many seconds")
    ap.add_argument("--n-ang", type=int, default=4, help="inclination: angular elements per wedge side")
    ap.add_argument("--n-rad", type=int, default=12, help="inclination: radial elements per wedge")
    ap.add_argument("--fd-capacity", type=float, default=0.5, help="pulsars: FD slots as a fraction of elements")
    ap.add_argument("--fd-slots", type=float, default=0.25,
                    help="breakdown: FD slot pool as a fraction of the elements (1 = one FD block per element)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "pulsars":
        return run_pulsars(args)
    if args.workload == "shell":
        return run_shell(args)
    if args.workload == "wald":
        return run_wald(args)
    if args.workload == "wald_vacuum":
        return run_wald_vacuum(args)
    if args.workload == "inclination":
        return run_inclination(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "oned":
        return run_oned(args)
    if args.workload == "dgphases":
        return run_dg_phases(args)

    import numpy as np
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2404_01531_gb300 import ffe
    from paper_2404_01531_gb300.roofline import (fp64_peak_tflops, fd_flux_flops, dg_flops_per_node,
                                                 fd_faces_per_element)

    cfg = W.breakdown(nx=args.nx, x_half=2.0 * args.nx / 64)
    cfg["params"]["recon"] = RECON[args.recon]
    n_elem = args.nx * 8 * 8
    fd_slots = min(n_elem, max(1, int(round(args.fd_slots * n_elem))))
    cfg["params"]["fd_capacity"] = fd_slots
    stream = torch.cuda.current_stream()
    ctx = ffe.Context(cfg, stream=stream)
    ctx.set_initial()
    ctx.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    # the state before the timed window: the profiled pass below replays the
    # same steps from it
    ckpt = ctx.save()

    # ---- timed region: graph replays, inputs resident in HBM (working set >> L2)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    i_t0 = ctx.info()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    inf = ctx.info()
    units = inf.node_updates - i_t0.node_updates
    n_fd_end = inf.n_fd_elem
    ms_max, units_all = combine_ranks(ms, units, dist, "cuda")
    value = units_all / (ms_max / 1e3)
    n0 = ctx.launch_count()
    ctx.step(1)
    torch.cuda.synchronize()
    per_step_launches = ctx.launch_count() - n0
    launches = per_step_launches * args.steps

    # ---- per-kernel event timing of the same steps (eager launches) from the
    # same starting state; algorithmic work of the window from the library's
    # element-update counters (every FD element update is one pass of fd_flux
    # over it, every DG element update one pass of dg_substep)
    ctx.load_checkpoint(ckpt)
    i0 = ctx.info()
    ctx.set_profiling(True)
    ctx.step(args.steps)
    ctx.set_profiling(False)
    i1 = ctx.info()
    prof = ctx.profile_read()
    same_window = (i1.node_updates - i0.node_updates == units and
                   i1.fd_elem_updates - i0.fd_elem_updates == inf.fd_elem_updates - i_t0.fd_elem_updates)
    total_ms = sum(v[1] for v in prof.values())
    E, P = ctx.n_elem, ctx.P
    nn = (P + 1) ** 3
    n_fd_upd = i1.fd_elem_updates - i0.fd_elem_updates
    n_dg_upd = i1.dg_elem_updates - i0.dg_elem_updates
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    f_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = fp64_peak_tflops(props.multi_processor_count, f_max)
    peak_src = (f"derived: 2 FP64 FMA lanes/clk/SM x {props.multi_processor_count} SMs (device) x "
                f"{f_max / 1e3:.3f} GHz (max SM clock, nvidia-smi)")
    fma_measured = ffe.fp64_fma_rate(stream)

    def kernel_roof(name, flops):
        if name not in prof or flops is None:
            return None
        launches_k, ms_k, max_k = prof[name]
        ach = flops / (ms_k / 1e3) / 1e12
        r = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
             "traffic": (DRAM_BYTES_PER_FD_ELEMENT[name] * n_fd_upd / launches_k
                         if DRAM_BYTES_PER_FD_ELEMENT.get(name) else None),
             "kernel": name, "peak_source": peak_src, "peak_measured_fma": fma_measured,
             "frac_of_measured_fma": ach / fma_measured, "share": ms_k / total_ms, "launches": launches_k,
             "ms_per_step": ms_k / args.steps, "max_launch_ms": max_k,
             "profiled_window": "the timed steps replayed from the same state" if same_window else "differs",
             "units": {"fd_elem_updates": n_fd_upd, "dg_elem_updates": n_dg_upd}}
        if r["traffic"] is not None:
            r["traffic_source"] = TRAFFIC_SOURCE
        return r
    dg_fl = n_dg_upd * nn * sum(dg_flops_per_node(P, s) for s in range(3)) / 3.0
    fd_fl = n_fd_upd * fd_faces_per_element(P) * fd_flux_flops(RECON[args.recon])
    roofs = {"fd_flux": kernel_roof("fd_flux", fd_fl), "dg_substep": kernel_roof("dg_substep", dg_fl)}
    dom = max((k for k in roofs if roofs[k]), key=lambda k: prof[k][1])
    roof = roofs[dom]
    roof_dg = roofs["dg_substep"]

    # ---- end to end through the C ABI with host buffers
    pin = torch.empty(ctx.n_state, dtype=torch.float64, pin_memory=True)
    pmask = torch.empty(ctx.n_elem, dtype=torch.uint8, pin_memory=True)
    ctx.download_into(pin.data_ptr(), pmask.data_ptr())
    ke = max(3, args.steps // 5)
    u0 = ctx.info().node_updates
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(ke):
        ctx.upload_from(pin.data_ptr(), pmask.data_ptr())
        ctx.step(1)
        ctx.download_into(pin.data_ptr(), pmask.data_ptr())
    w1 = time.perf_counter()
    ue = ctx.info().node_updates - u0
    e2e = {"value": ue * ws / (w1 - w0), "unit": UNIT, "h2d_bytes_per_step": ctx.n_state * 8 + ctx.n_elem,
           "d2h_bytes_per_step": ctx.n_state * 8 + ctx.n_elem}
    status = ctx.status()
    ctx.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    adj = None
    if not args.no_adjoint:
        try:
            adj = adjoint_measure()
        except Exception as ex:  # reported, not fatal
            adj = {"failed": str(ex)}
    batched = None
    if not args.no_batch and ws == 1:
        try:
            batched = batch_measure(args.n_inst, 3, 2, args.fd_capacity)
        except Exception as ex:  # reported, not fatal
            batched = {"failed": str(ex)}
    split = None
    if not args.no_split and ws == 1:
        try:
            split = split_measure(steps=5, warmup=3)
        except Exception as ex:  # reported, not fatal
            split = {"failed": str(ex)}
    cpu = None
    if not args.no_cpu_baseline:
        try:
            r1, dt1, n1 = cpu_baseline_subprocess(40, 15.0)
            ra, dta, na, ncores = cpu_baseline_all_cores(40, 15.0)
            cpu = {"value": ra, "unit": UNIT, "cores": ncores, "kind": "oracle",
                   "sample": (f"oracle (numpy fp64) on a 16x2x2-element slab of the breakdown workload (same "
                              f"element width, order and current sheet), whole hybrid steps: {ncores} "
                              f"single-threaded processes, one per host core, each on its own copy of the slab, "
                              f"at least {na} steps each in {dta:.1f} s"),
                   "one_core": {"value": r1, "cores": 1, "sample": CPU_SAMPLE_TEXT + f", {n1} steps in {dt1:.1f} s"}}
        except Exception as ex:  # reported, not fatal
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"breakdown {args.nx}x8x8 P=5 (FFE breakdown / current sheet, eta=1e3)",
                       "elements": E, "P": P, "dg_nodes": E * nn, "fd_elements_end": n_fd_end,
                       "parallelism": f"replicas x{ws}", "l2": "working set > L2 (no flush needed)",
                       "recon": args.recon, "fd_slots": fd_slots},
            "roofline": roof, "roofline_dg": roof_dg, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "kernel_ms": {k: v[1] / max(v[0], 1) for k, v in prof.items()},
            "adjoint": adj, "batched_over_single": (batched or {}).get("batched_over_single"),
            "batch": batched, "split": split, "status_bits": status}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
