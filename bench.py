"""Benchmark: SSP-RK3 time steps of the modal DG Euler residual on one GB300.

One step = one SSP-RK3 step = 3 fused residual + stage-update launches over
the whole mesh (every row of the hot path: interpolation, fluxes, Riemann
solver, lift, inverse mass, RK axpy).  Metric: residual DOF-updates per
second = 3 * N_e * 5 * N_b / t_step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3]
                    [--precision auto|mixed|mixed-bf16|fp64|fp32] [--impl ours|reference]

Workloads (seeded, synthetic; they stand in for the paper's 2D grids):
  c1  6^3 x 6 periodic cube, P1, jitter 10%   (1,296 tets)
  c2  48^3 x 6 periodic cube, P2, jitter 10%  (663,552 tets), vortex + 1% noise
  c3  64^3 x 6 periodic cube, P3, jitter 15%  (1,572,864 tets), vortex, Roe
  c4  32^3 x 6 periodic cube, P2              (196,608 tets)
  c5  96x48x48 x 6 box channel, P3, walls + far field (1,327,104 tets), pulse
The default is c3 (the P3 workload the HBM-roofline target refers to).

Multi-GPU (torchrun): every rank runs its own copy of the workload on its
own GPU (replicas; the residual needs no exchange for independent meshes);
value = all ranks' DOF-updates / the slowest rank's time.
"""
from __future__ import annotations

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

WORKLOADS = {
    "c1": dict(n=6, p=1, jitter=0.10, flux="rusanov", field="vortex", box=False, order="morton"),
    "c2": dict(n=48, p=2, jitter=0.10, flux="rusanov", field="vortex_noise", box=False, order="rcm"),
    "c3": dict(n=64, p=3, jitter=0.15, flux="roe", field="vortex", box=False, order="morton"),
    "c4": dict(n=32, p=2, jitter=0.10, flux="rusanov", field="vortex", box=False, order="morton"),
    "c5": dict(dims=(96, 48, 48), p=3, jitter=0.15, flux="roe", field="pulse", box=True, order="morton"),
    # small case of the c3 kernel for profiler captures (state 157 MB > L2)
    "c3s": dict(n=32, p=3, jitter=0.15, flux="roe", field="vortex", box=False, order="morton"),
}
ORDER_NAMES = ("morton", "hilbert", "rcm", "asis")
NB = {1: 4, 2: 10, 3: 20}
NQ = {1: 4, 2: 14, 3: 24}
NQF = {1: 3, 2: 6, 3: 12}
# FP64 flops of one Riemann solve per face point (counted from the formulas, divisions and
# square roots as one flop each)
RIEMANN_FLOPS = {"rusanov": 70, "roe": 160}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def replica_value(work_per_rank, t_local, world, device=None):
    """Whole-job throughput of independent replicas: every rank did
    ``work_per_rank`` units; the job time is the slowest rank's (all-reduce MAX
    over the process group when world > 1)."""
    t = t_local
    if world > 1:
        import torch
        x = torch.tensor([t_local], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
        t = float(x.item())
    return t, world * work_per_rank / t


def flux_of(args):
    """Numerical flux of the run: --flux, else the workload's."""
    return getattr(args, "flux", None) or WORKLOADS[args.workload]["flux"]


def order_of(args):
    """Element order of the run: --order, else the workload's (RCM where the workload names it,
    a Morton space-filling curve otherwise)."""
    return getattr(args, "order", None) or WORKLOADS[args.workload]["order"]


def make_workload(name):
    from paper_2209_01877_gb300 import inputs as I
    w = WORKLOADS[name]
    if w["box"]:
        mesh = I.make_box_channel(*w["dims"], jitter=w["jitter"])
    else:
        mesh = I.make_periodic_cube(w["n"], jitter=w["jitter"])
    if w["field"] == "pulse":
        c = I.pulse_centre()
        field = lambda x: I.gaussian_pulse(x, c)
    else:
        field = lambda x: I.isentropic_vortex(x)
    return mesh, field, w


def algorithmic_model(p, ne, flux, s_state, stage):
    """Bytes and flops of one fused residual + RK-stage launch (the minimum the
    method needs): the state read once, the RK base state read (stages 2, 3),
    the new state written, 32 B of connectivity/geometry per element; flops
    with every interior face's traces and Riemann solve counted once."""
    nb, nq, nqf = NB[p], NQ[p], NQF[p]
    nv = 5 * nb
    reads = 2 if stage > 1 else 1
    bytes_ = ne * (nv * s_state * (reads + 1) + 32)
    per_elem = (2 * 2 * nqf * 5 * nb * 2          # traces: 2 faces/elem x 2 sides
                + 2 * nqf * RIEMANN_FLOPS[flux]   # Riemann: 2 faces/elem
                + nq * 5 * nb * 2                 # volume interpolation
                + nq * (25 + 45 * 2)              # Euler flux + contravariant transform
                + 5 * nb * 3 * nq * 2             # projection on the basis gradients
                + 5 * nb * 4 * nqf * 2            # lift of the 4 face fluxes
                + nv * 4)                         # RK stage
    return bytes_, ne * per_elem


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the fused stage kernel from one
# ncu capture of the 32^3 x 6 P3 Roe vortex case (three consecutive stage launches, mean bytes
# per element per launch; Morton order for the mixed kernel, RCM for FP64), with the hash of the
# device sources the kernel was built from (its kernel file, the device headers it includes and
# dg_device.h, which holds every declaration of the shared headers that device code uses).  Traffic
# grows in proportion to the element count (one pass over the element-ordered state), so the
# bench scales it to the workload's tets; it reports null when the sources changed since.
MEASURED_TRAFFIC = {
    # (precision, p, flux): (bytes per element per launch, source files, sha256[:16] of them)
    ("mixed", 3, "roe"): (2036.8, ("kernels_mixed.cu", "mixed_common.cuh", "tc_ops.cuh", "euler_device.cuh",
                                   "dg_device.h"), "83821532acbe6d04"),
    # the FP64 stage is three kernels (traces, one flux per face, residual): their sum per stage
    ("f64", 3, "roe"): (10170.3, ("kernels_simt.cu", "euler_device.cuh", "dg_device.h"), "7c8c5ce929f70147"),
}


def kernel_source_hash(files):
    """sha256[:16] of the sources' code: comments and whitespace are left out, so that an edit
    of the commentary alone keeps a measured figure valid; any change of the code voids it."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2209_01877_gb300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", "", src).encode())
    return h.hexdigest()[:16]


def measured_traffic(precision_name, p, flux, ne):
    """Per-launch DRAM bytes for this kernel and workload, or None."""
    key = ("mixed" if precision_name.startswith("f16") else precision_name, p, flux)
    if key not in MEASURED_TRAFFIC:
        return None
    per_elem, files, digest = MEASURED_TRAFFIC[key]
    if kernel_source_hash(files) != digest:
        return None
    return per_elem * ne


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def fp64_peak_tflops(sm_mhz=2070.0):
    """FP64 FMA peak of GB300: 152 SMs x 2 FP64 FMA/clk/SM (4 flop/clk/SM) x clock."""
    return 152 * 4 * sm_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------------------------
def run_ours(args, rank, world, device):
    import torch
    from paper_2209_01877_gb300 import dg

    mesh, field, w = make_workload(args.workload)
    p, flux = w["p"], flux_of(args)
    precision = {"auto": dg.DG_MIXED_FP16, "mixed": dg.DG_MIXED_FP16, "mixed-bf16": dg.DG_MIXED_BF16,
                 "fp64": dg.DG_FP64, "fp32": dg.DG_FP32}[args.precision]
    fs = (0, 0, 0, 0, 0)
    if w["box"]:
        from paper_2209_01877_gb300 import inputs as I
        fs = tuple(I.freestream_state(0.3))
    t0 = time.time()
    ren = {"morton": dg.DG_ORDER_MORTON, "hilbert": dg.DG_ORDER_HILBERT, "rcm": dg.DG_ORDER_RCM,
           "asis": dg.DG_ORDER_ASIS}[order_of(args)]
    M = dg.Mesh(mesh.tet_vid, mesh.tet_xyz, None if not w["box"] else mesh.bc_tag, order=p, precision=precision,
                flux=dg.DG_ROE if flux == "roe" else dg.DG_RUSANOV, renumber=ren, freestream=fs)
    U0 = M.project(field)
    if w["field"] == "vortex_noise":
        from paper_2209_01877_gb300 import inputs as I
        U0 = I.perturb_coefficients(U0)
    log(f"[rank {rank}] mesh + state ready in {time.time() - t0:.1f}s: ne={mesh.ne} p={p} {flux}")
    stream = torch.cuda.current_stream(device)
    dg.dg_set_state(M.handle, U0, stream)
    dt = dg.dg_stable_dt(M.handle, 0.1, stream)
    ne, nb = mesh.ne, NB[p]
    dofs = ne * 5 * nb

    for _ in range(args.warmup):
        dg.dg_rk3_step(M.handle, dt, 1, stream)
    torch.cuda.synchronize(device)
    dg.dg_sync_status(M.handle, stream)

    # timed region: K steps, events around every stage launch
    nev = 3 * args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nev)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(device.index if device.index is not None else 0)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(device)
    clocks.start()
    time.sleep(0.3)
    start.record(stream)
    k = 0
    for _ in range(args.steps):
        for st in (1, 2, 3):
            ev[k][0].record(stream)
            dg.dg_rk_stage(M.handle, st, dt, stream)
            ev[k][1].record(stream)
            k += 1
    stop.record(stream)
    torch.cuda.synchronize(device)
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    dg.dg_sync_status(M.handle, stream)
    t_total = start.elapsed_time(stop) / 1e3
    stage_ms = [[], [], []]
    for i, (a, b) in enumerate(ev):
        stage_ms[i % 3].append(a.elapsed_time(b))
    t_local = t_total
    t_total, value = replica_value(3 * dofs * args.steps, t_local, world, device)
    ms_per_step = t_total / args.steps * 1e3

    # roofline of the dominant kernel (the fused residual + RK-stage kernel)
    s_state = 4 if precision == dg.DG_FP32 else 8     # FP64, or the float-float pair of the mixed form
    peaks, peak_src = measured_peaks()
    tot_bytes = tot_flops = tot_ms = 0.0
    for st in (1, 2, 3):
        b, f = algorithmic_model(p, ne, flux, s_state, st)
        tot_bytes += b * len(stage_ms[st - 1])
        tot_flops += f * len(stage_ms[st - 1])
        tot_ms += sum(stage_ms[st - 1])
    nlaunch = sum(len(x) for x in stage_ms)
    avg_ms = tot_ms / nlaunch
    bytes_per_launch = tot_bytes / nlaunch
    flops_per_launch = tot_flops / nlaunch
    hbm_achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    if precision == dg.DG_FP64:
        peak_alu = fp64_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
        achieved = flops_per_launch / (avg_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
                "frac": achieved / peak_alu, "traffic": None,
                "peak_source": "FP64 FMA pipe: 152 SMs x 4 flop/clk x max SM clock (recipe unit counts and clock)",
                "hbm_achieved_gbs": hbm_achieved, "hbm_frac": hbm_achieved / peaks["hbm_gbs"],
                "kernel": "FP64 stage: k_traces, k_faces, k_residual<double,P,FLUX,RK,FB> (time and DRAM "
                          "traffic of the three per stage)", "algorithmic_bytes_per_launch": bytes_per_launch,
                "algorithmic_flops_per_launch": flops_per_launch, "avg_launch_ms": avg_ms}
    else:
        kname = "k_residual<float,P,FLUX,RK>" if precision == dg.DG_FP32 else "k_stage_mixed<P,FLUX,BF16>"
        roof = {"bound": "hbm", "achieved": hbm_achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": hbm_achieved / peaks["hbm_gbs"], "traffic": None,
                "peak_source": f"hbm_gbs of {peak_src} peaks", "kernel": kname,
                "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        Uh = torch.empty((ne, 5, nb), dtype=torch.float64, pin_memory=True).numpy()
        Uh[...] = U0
        nrep = max(1, min(args.steps, 5))
        dg.dg_rk3_step(M.handle, dt, 1, stream)
        torch.cuda.synchronize(device)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(nrep):
            dg.dg_set_state(M.handle, Uh, stream)
            dg.dg_rk3_step(M.handle, dt, 1, stream)
            dg.dg_get_state(M.handle, Uh, stream)
        b.record(stream)
        torch.cuda.synchronize(device)
        te = a.elapsed_time(b) / 1e3
        e2e = {"value": world * 3 * dofs * nrep / te, "unit": "DOF-updates/s", "h2d_bytes_per_step": dofs * 8,
               "d2h_bytes_per_step": dofs * 8, "steps": nrep}
    M.close()
    pname = {dg.DG_FP64: "f64", dg.DG_FP32: "f32", dg.DG_MIXED_FP16: "f16x2-tc/f32/ff32",
             dg.DG_MIXED_BF16: "bf16x2-tc/f32/ff32"}[precision]
    roof["traffic"] = measured_traffic(pname, p, flux, ne)
    return dict(value=value, ms_per_step=ms_per_step, roofline=roof, clocks=clk, e2e=e2e, t_local=t_local,
                precision=pname, ne=ne, p=p, flux=flux,
                stage_ms=[float(np.mean(x)) for x in stage_ms], nlaunch=nlaunch)


# ---------------------------------------------------------------------------------------------
def _field_of(name, w):
    """The workload's pointwise initial field (the 1% noise of c2 acts on coefficients, not on
    the field, and does not change the oracle's work)."""
    from paper_2209_01877_gb300 import inputs as I
    if name == "pulse":
        c = I.pulse_centre()
        return lambda x: I.gaussian_pulse(x, c)
    return lambda x: I.isentropic_vortex(x)


def _oracle_worker(conn, vid, xyz, tag, rows, p, flux, fs, field_name):
    """One host core: the oracle's residual of `rows` of a sub-mesh (the rows and their face
    neighbours; faces that lose their partner there get a wall tag -- their elements' residuals
    are not evaluated).  Answers each message k with the seconds of k back-to-back evaluations."""
    from oracle.dg import Problem
    P = Problem(vid, xyz, tag, p=p, flux=flux, freestream=fs)
    U = P.project(_field_of(field_name, None), rule="volume")
    P.residual(U, rows[:16])
    conn.send("ready")
    while True:
        k = conn.recv()
        if k is None:
            break
        t0 = time.perf_counter()
        for _ in range(k):
            P.residual(U, rows)
        conn.send(time.perf_counter() - t0)
    conn.close()


class OraclePool:
    """`cores` processes (spawn), each holding an equal share of a seeded sample of the workload's
    elements; `run(k)` has every process evaluate its share k times at once and returns the wall
    time until the last one is done."""

    def __init__(self, workload, nsample, cores, flux=None, seed=11):
        import multiprocessing as mp
        from oracle.mesh import match_faces
        mesh, _, w = make_workload(workload)
        tag = mesh.bc_tag if w["box"] else None
        nbr, _, _ = match_faces(mesh.tet_vid, tag)
        rng = np.random.default_rng(seed)
        rows = np.sort(rng.choice(mesh.ne, size=min(nsample, mesh.ne), replace=False))
        fs = None
        if w["box"]:
            from paper_2209_01877_gb300 import inputs as I
            fs = I.freestream_state(0.3)
        self.nrows, self.nb, self.cores = len(rows), NB[w["p"]], cores
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for chunk in np.array_split(rows, cores):
            need = np.unique(np.concatenate([chunk, nbr[chunk].ravel()]))
            need = need[need >= 0]
            t = np.ones((len(need), 4), dtype=np.int8)
            if w["box"]:
                t = np.where(mesh.bc_tag[need] > 0, mesh.bc_tag[need], 1).astype(np.int8)
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, mesh.tet_vid[need], mesh.tet_xyz[need], t,
                                                          np.searchsorted(need, chunk), w["p"],
                                                          flux or w["flux"], fs, w["field"]))
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        for c in self.conns:
            assert c.recv() == "ready"

    def run(self, k):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(k)
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0

    def dual_phase_rate(self):
        """DOF-updates/s from the dual-phase timing (K1 = 1 and K2 = 3 evaluations, subtracted):
        per-evaluation time without the fixed costs of a call."""
        t1 = self.run(1)
        t3 = self.run(3)
        per = max((t3 - t1) / 2.0, 1e-9)
        return self.nrows * 5 * self.nb / per, per

    def close(self):
        for c in self.conns:
            c.send(None)
        for pr in self.procs:
            pr.join(timeout=30)


def _oracle_child(mode, workload, nsample, steps=1, warmup=0, flux=None):
    """Run the oracle timing in a child process (no CUDA device, one BLAS thread per process)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_timing(%r, %r, %d, %d, %d, %r)))"
            % (ROOT, mode, workload, nsample, steps, warmup, flux))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_timing(mode, workload, nsample, steps=1, warmup=0, flux=None):
    """mode "baseline": dual-phase rates of the oracle on one core and on every host core;
    mode "steps": `warmup` untimed and `steps` timed evaluations of the sample on every core."""
    cores = os.cpu_count() or 1
    if mode == "baseline":
        one = OraclePool(workload, nsample, 1, flux)
        r1, s1 = one.dual_phase_rate()
        one.close()
        pool = OraclePool(workload, nsample, cores, flux)
        rn, sn = pool.dual_phase_rate()
        pool.close()
        return {"single": r1, "single_s": s1, "all": rn, "all_s": sn, "cores": cores, "rows": pool.nrows}
    pool = OraclePool(workload, nsample, cores, flux)
    for _ in range(warmup):
        pool.run(1)
    ts = [pool.run(1) for _ in range(steps)]
    pool.close()
    return {"rates": [pool.nrows * 5 * pool.nb / t for t in ts], "seconds": ts, "cores": cores,
            "rows": pool.nrows}


def cpu_baseline_subprocess(workload, nsample, flux=None):
    r = _oracle_child("baseline", workload, nsample, flux=flux)
    return {"value": r["all"], "unit": "DOF-updates/s", "cores": r["cores"], "kind": "oracle",
            "sample": f"FP64 oracle residual on {r['rows']} seeded elements of {workload} (each host process "
                      f"holds its share and their face neighbours), split over {r['cores']} processes with one "
                      f"BLAS thread each, dual-phase timing (K1 = 1, K2 = 3 evaluations): {r['all_s']:.2f} s "
                      f"per evaluation",
            "single_core": {"value": r["single"], "cores": 1,
                            "sample": f"the same sample in one process, dual-phase: {r['single_s']:.1f} s per "
                                      f"evaluation"}}


SAMPLE = {"c1": 1296, "c2": 120000, "c3": 60000, "c4": 120000, "c5": 60000, "c3s": 60000}


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores (one process per core, one BLAS
    thread each), each step one residual evaluation of a bounded seeded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = config_of(args)
    n = SAMPLE.get(args.workload, 2000)
    r = _oracle_child("steps", args.workload, n, args.steps, args.warmup, flux_of(args))
    rate = float(np.mean(r["rates"]))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "DOF-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(r["seconds"])) * 1e3,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": rate, "unit": "DOF-updates/s", "cores": r["cores"], "kind": "oracle",
                             "sample": f"FP64 oracle residual on {r['rows']} seeded elements of {args.workload} "
                                       f"per step, split over {r['cores']} processes with one BLAS thread each"},
            "e2e": {"value": rate, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = "DG residual DOF-updates/s (P1-P3 tets), mixed vs FP64; % of HBM roofline"


def config_of(args):
    w = WORKLOADS[args.workload]
    from paper_2209_01877_gb300 import inputs as I
    ne = 6 * (w["n"] ** 3 if not w["box"] else int(np.prod(w["dims"])))
    desc = {"c1": "6^3x6 periodic cube", "c2": "48^3x6 periodic cube", "c3": "64^3x6 periodic cube",
            "c4": "32^3x6 periodic cube", "c5": "96x48x48x6 box channel", "c3s": "32^3x6 periodic cube"}
    oname = {"morton": "Morton order", "hilbert": "Hilbert order", "rcm": "RCM order",
             "asis": "input (random) order"}[order_of(args)]
    return {"workload": f"{args.workload}: {desc[args.workload]}, P{w['p']}, {ne} tets, {flux_of(args)} flux, "
                        f"jitter {w['jitter']}, {oname}, field {w['field']}",
            "tets": ne, "order": w["p"], "flux": flux_of(args), "dofs": ne * 5 * I.n_basis(w["p"]),
            "step": "one SSP-RK3 step = 3 fused residual+stage launches",
            "l2": "inputs larger than L2 (state >= 157 MB vs 129 MB L2)" if w["p"] >= 2 and ne > 100000
            else "state fits in L2 (small case)"}


def run_study(args):
    """Studies of the paper's two optimisations, printed as one JSON object.

    temporal-mp  (Sec. III-B, Tab. 2): n steps with the first k in FP32 and the
                 rest in FP64, k = 0, 20%, 50%, 80%, 100% of n; device time and
                 the RMS coefficient difference from the all-FP64 run.
    renumbering  (Sec. III-B, Tab. 1): element-adjacency bandwidth and RK-step
                 throughput for the input (random) order, RCM, Morton and Hilbert.
    adjoint      residual VJP and RK-step VJP throughput, and the checkpointed
                 multi-step adjoint (steps = --steps, checkpoints every 10).
    aux          the time-step reduction and the conservation / kinetic-energy
                 sums (device time per call).
    ns           (periodic workloads, FP64) device time of the Navier-Stokes residual
                 (BR1 gradient and viscous lines added) against the Euler residual.
    launch       device time per RK3 step of dg_rk3_step (a replayed CUDA graph on
                 small meshes) against one dg_rk_stage launch per stage.
    conservation change of the conserved totals over --steps SSP-RK3 steps
                 for FP64 and both mixed forms, minus what the boundary flux
                 carried out (Eq. 11's boundary-face line integrated over the
                 RK stages): the discrete conservation drift."""
    import torch
    from paper_2209_01877_gb300 import dg
    from paper_2209_01877_gb300.temporal import run_temporal_mp
    torch.cuda.set_device(0)
    mesh, field, w = make_workload(args.workload)
    p, flux = w["p"], flux_of(args)
    fl = dg.DG_ROE if flux == "roe" else dg.DG_RUSANOV
    tag = mesh.bc_tag if w["box"] else None
    fs = (0, 0, 0, 0, 0)
    if w["box"]:
        from paper_2209_01877_gb300 import inputs as I
        fs = tuple(I.freestream_state(0.3))
    out = {"study": args.study, "workload": config_of(args)["workload"]}
    if args.study == "temporal-mp":
        m64 = dg.Mesh(mesh.tet_vid, mesh.tet_xyz, tag, order=p, precision=dg.DG_FP64, flux=fl, freestream=fs)
        m32 = dg.Mesh(mesh.tet_vid, mesh.tet_xyz, tag, order=p, precision=dg.DG_FP32, flux=fl, freestream=fs)
        U0 = torch.from_numpy(m64.project(field)).cuda()
        dg.dg_set_state(m64.handle, U0)
        dt = dg.dg_stable_dt(m64.handle, 0.1)
        n = args.steps
        run_temporal_mp(m32, m64, U0, dt, 1, 1)          # warm-up of both paths
        run_temporal_mp(m32, m64, U0, dt, 1, 0)
        ref, _, t_ref = run_temporal_mp(m32, m64, U0, dt, n, 0)
        rows = []
        for frac in (0.0, 0.2, 0.5, 0.8, 1.0):
            k = int(round(frac * n))
            U, t_sp, t_dp = run_temporal_mp(m32, m64, U0, dt, n, k)
            rows.append({"sp_steps": k, "dp_steps": n - k, "seconds": t_sp + t_dp,
                         "rms_diff_vs_dp": float(((U - ref) ** 2).mean().sqrt())})
        out.update({"steps": n, "dt": dt, "rows": rows})
    elif args.study == "adjoint":
        from paper_2209_01877_gb300.adjoint import rk3_adjoint
        prec = {"fp32": dg.DG_FP32}.get(args.precision, dg.DG_FP64)
        M = dg.Mesh(mesh.tet_vid, mesh.tet_xyz, tag, order=p, precision=prec, flux=fl, freestream=fs)
        U0 = torch.from_numpy(M.project(field)).cuda()
        dg.dg_set_state(M.handle, U0)
        dt = dg.dg_stable_dt(M.handle, 0.1)
        lam = torch.ones_like(U0)
        out_t = torch.empty_like(U0)
        dofs = mesh.ne * 5 * NB[p]

        def timed(fn, reps):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / 1e3 / reps

        t_res = timed(lambda: dg.dg_residual(M.handle, U0, out_t), 5)
        t_vjp = timed(lambda: dg.dg_residual_vjp(M.handle, U0, lam, out_t), 5)
        t_svjp = timed(lambda: dg.dg_rk3_step_vjp(M.handle, U0, dt, lam, out_t), 3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, g, peak = rk3_adjoint(M, U0, dt, args.steps, ckpt_every=10)
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        out.update({"precision": "f32" if prec == dg.DG_FP32 else "f64", "dofs": dofs,
                    "residual_ms": t_res * 1e3, "residual_vjp_ms": t_vjp * 1e3,
                    "residual_vjp_dof_per_s": dofs / t_vjp, "rk3_step_vjp_ms": t_svjp * 1e3,
                    "adjoint_steps": args.steps, "adjoint_seconds": t_adj, "adjoint_peak_states": peak,
                    "kinetic_energy": J})
    elif args.study == "aux":
        prec = {"fp64": dg.DG_FP64, "fp32": dg.DG_FP32}.get(args.precision, dg.DG_MIXED_FP16)
        M = dg.Mesh(mesh.tet_vid, mesh.tet_xyz, tag, order=p, precision=prec, flux=fl, freestream=fs)
        dg.dg_set_state(M.handle, M.project(field))
        for _ in range(3):
            dg.dg_stable_dt(M.handle, 0.1)
            dg.dg_integrals(M.handle)
        n = max(args.steps, 5)
        t0 = time.perf_counter()
        for _ in range(n):
            dg.dg_stable_dt(M.handle, 0.1)
        t_dt = (time.perf_counter() - t0) / n
        t0 = time.perf_counter()
        for _ in range(n):
            dg.dg_integrals(M.handle)
        t_int = (time.perf_counter() - t0) / n
        out.update({"stable_dt_ms_incl_sync": t_dt * 1e3, "integrals_ms_incl_sync": t_int * 1e3,
                    "tets": mesh.ne})
    elif args.study == "ns":
        prec = {"fp32": dg.DG_FP32, "mixed": dg.DG_MIXED_FP16, "mixed-bf16": dg.DG_MIXED_BF16}.get(args.precision,
                                                                                                  dg.DG_FP64)
        M = dg.Mesh(mesh.tet_vid, mesh.tet_xyz, tag, order=p, precision=prec, flux=fl, freestream=fs)
        U = torch.from_numpy(M.project(field)).cuda()
        R = torch.empty_like(U)
        n = max(args.steps, 3)
        res = {}
        dg.dg_set_state(M.handle, U)
        dt_ns = 0.1 * dg.dg_stable_dt(M.handle, 0.1)
        calls = (("dg_residual (Euler)", lambda: dg.dg_residual(M.handle, U, R)),
                 ("dg_ns_residual (mu 1e-3, Pr 0.72)", lambda: dg.dg_ns_residual(M.handle, U, R, 1e-3, 0.72)),
                 ("dg_rk3_step (Euler, one step)", lambda: dg.dg_rk3_step(M.handle, dt_ns, 1)),
                 ("dg_ns_rk3_step (one step, mu 1e-3, Pr 0.72)",
                  lambda: dg.dg_ns_rk3_step(M.handle, dt_ns, 1, 1e-3, 0.72)))
        for name, call in calls:
            call()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(n):
                call()
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3 / n
            stages = 3 if "step" in name else 1          # one RK3 step = three residual evaluations
            res[name] = {"ms": t * 1e3, "dof_updates_per_s": stages * mesh.ne * 5 * NB[p] / t}
        dg.dg_sync_status(M.handle)
        M.close()
        out.update({"precision": {dg.DG_FP64: "f64", dg.DG_FP32: "f32", dg.DG_MIXED_FP16: "f16x2-tc/f32/ff32",
                                  dg.DG_MIXED_BF16: "bf16x2-tc/f32/ff32"}[prec], "tets": mesh.ne, "calls": n,
                    "rows": res})
    elif args.study == "launch":
        prec = {"fp64": dg.DG_FP64, "fp32": dg.DG_FP32, "mixed-bf16": dg.DG_MIXED_BF16}.get(args.precision,
                                                                                         dg.DG_MIXED_FP16)
        M = dg.Mesh(mesh.tet_vid, mesh.tet_xyz, tag, order=p, precision=prec, flux=fl, freestream=fs)
        dg.dg_set_state(M.handle, M.project(field))
        dt = dg.dg_stable_dt(M.handle, 0.1)
        n = max(args.steps, 8)
        dg.dg_rk3_step(M.handle, dt, 8)
        for st in (1, 2, 3):
            dg.dg_rk_stage(M.handle, st, dt)
        torch.cuda.synchronize()
        res = {}
        for name in ("dg_rk3_step", "dg_rk_stage x 3", "dg_rk3_step, new dt every call"):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            a.record()
            if name == "dg_rk3_step":
                dg.dg_rk3_step(M.handle, dt, n)
            elif name == "dg_rk_stage x 3":
                for _ in range(n):
                    for st in (1, 2, 3):
                        dg.dg_rk_stage(M.handle, st, dt)
            else:
                # a loop that recomputes dt before every call: 8 steps per call, the captured graph
                # updated in place for each new dt
                for i in range(n // 8):
                    dg.dg_rk3_step(M.handle, dt * (1.0 - 1e-3 * (i % 7)), 8)
            b.record()
            torch.cuda.synchronize()
            res[name] = a.elapsed_time(b) * 1e3 / n
            res[name + " (host wall)"] = (time.perf_counter() - t0) * 1e6 / n
        dg.dg_sync_status(M.handle)
        M.close()
        out.update({"steps": n, "tets": mesh.ne, "us_per_step": res,
                    "note": "dg_rk3_step replays a CUDA graph of 8 captured steps on meshes of <= 65536 tets"})
    elif args.study == "conservation":
        ren = {"morton": dg.DG_ORDER_MORTON, "hilbert": dg.DG_ORDER_HILBERT, "rcm": dg.DG_ORDER_RCM,
               "asis": dg.DG_ORDER_ASIS}[order_of(args)]
        rows = []
        for pname, prec, cons in (("f64", dg.DG_FP64, False), ("f16x2-tc/f32/ff32", dg.DG_MIXED_FP16, False),
                                  ("f16x2-tc/f32/ff32, conservative mode 0", dg.DG_MIXED_FP16, True),
                                  ("bf16x2-tc/f32/ff32", dg.DG_MIXED_BF16, False),
                                  ("bf16x2-tc/f32/ff32, conservative mode 0", dg.DG_MIXED_BF16, True)):
            nsteps = args.steps
            M = dg.Mesh(mesh.tet_vid, mesh.tet_xyz, tag, order=p, precision=prec, flux=fl, renumber=ren,
                        freestream=fs)
            if cons:
                dg.dg_set_conservative(M.handle, True)
            U0 = M.project(field)
            dg.dg_set_state(M.handle, U0)
            dt = dg.dg_stable_dt(M.handle, 0.1)
            # stage time of this form (CUDA events over 5 steps after 2), then the drift run from U0
            dg.dg_rk3_step(M.handle, dt, 2)
            torch.cuda.synchronize()
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record()
            dg.dg_rk3_step(M.handle, dt, 5)
            eb.record()
            torch.cuda.synchronize()
            ms_step = ea.elapsed_time(eb) / 5
            dg.dg_set_state(M.handle, U0)
            t0, _ = dg.dg_integrals(M.handle)
            acc = np.zeros(5)
            t_start = time.perf_counter()
            for _ in range(nsteps):
                if w["box"] and cons:
                    # the boundary flux each stage applied: the totals move by -dt (B1/6 + B2/6 + 2 B3/3)
                    B = []
                    for st in (1, 2, 3):
                        dg.dg_rk_stage(M.handle, st, dt)
                        B.append(dg.dg_applied_boundary_flux(M.handle))
                    acc += dt * (B[0] / 6.0 + B[1] / 6.0 + 2.0 * B[2] / 3.0)
                elif w["box"]:
                    # B at the three stage states: the totals move by -dt (B0/6 + B1/6 + 2 B2/3)
                    b0 = dg.dg_boundary_flux(M.handle)
                    dg.dg_rk_stage(M.handle, 1, dt)
                    b1 = dg.dg_boundary_flux(M.handle, None, 1)
                    dg.dg_rk_stage(M.handle, 2, dt)
                    b2 = dg.dg_boundary_flux(M.handle, None, 2)
                    dg.dg_rk_stage(M.handle, 3, dt)
                    acc += dt * (b0 / 6.0 + b1 / 6.0 + 2.0 * b2 / 3.0)
                else:
                    dg.dg_rk3_step(M.handle, dt, 1)
            t1, _ = dg.dg_integrals(M.handle)
            dg.dg_sync_status(M.handle)
            M.close()
            d = t1 - t0 + acc
            rows.append({"precision": pname, "steps": nsteps, "dt": dt, "seconds": time.perf_counter() - t_start,
                         "ms_per_step": ms_step,
                         "totals_start": t0.tolist(), "boundary_flux_integral": (-acc).tolist(),
                         "drift": d.tolist(),
                         "rel_drift_mass": abs(d[0]) / abs(t0[0]),
                         "rel_drift_momentum": float(np.linalg.norm(d[1:4]) / np.linalg.norm(t0[1:4])),
                         "rel_drift_energy": abs(d[4]) / abs(t0[4])})
        out.update({"rows": rows,
                    "note": "drift = change of the totals + dt sum over steps of the boundary flux (0 on periodic "
                            "meshes): B0/6 + B1/6 + 2 B2/3 at the stage states, re-evaluated in FP64 "
                            "(dg_boundary_flux), or for the conservative mode the flux each stage applied "
                            "(dg_applied_boundary_flux); ms_per_step from CUDA events over 5 steps"})
    else:
        rows = []
        for name, order in (("input (random)", dg.DG_ORDER_ASIS), ("RCM", dg.DG_ORDER_RCM),
                            ("Morton", dg.DG_ORDER_MORTON), ("Hilbert", dg.DG_ORDER_HILBERT)):
            prec = {"fp64": dg.DG_FP64, "fp32": dg.DG_FP32}.get(args.precision, dg.DG_MIXED_FP16)
            M = dg.Mesh(mesh.tet_vid, mesh.tet_xyz, tag, order=p, precision=prec, flux=fl, renumber=order,
                        freestream=fs)
            info = M.info()
            U0 = M.project(field)
            dg.dg_set_state(M.handle, U0)
            dt = dg.dg_stable_dt(M.handle, 0.1)
            dg.dg_rk3_step(M.handle, dt, 3)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dg.dg_rk3_step(M.handle, dt, args.steps)
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3
            rows.append({"order": name, "bandwidth": info["bandwidth_after"],
                         "dof_updates_per_s": 3 * mesh.ne * 5 * NB[p] * args.steps / t,
                         "ms_per_step": t / args.steps * 1e3})
            M.close()
        out.update({"precision": args.precision, "rows": rows})
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="auto", choices=["auto", "mixed", "mixed-bf16", "fp64", "fp32"])
    ap.add_argument("--flux", default=None, choices=["roe", "rusanov"],
                    help="numerical flux (default: the workload's; Roe for c3 and c5)")
    ap.add_argument("--order", default=None, choices=ORDER_NAMES,
                    help="element order (default: the workload's; RCM for c2, Morton otherwise)")
    ap.add_argument("--no-fp64-leg", action="store_true", help="skip the FP64 comparison leg of a mixed run")
    ap.add_argument("--study", choices=["temporal-mp", "renumbering", "adjoint", "aux", "conservation", "launch", "ns"],
                    default=None,
                    help="print a study table instead of the benchmark line")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        log("warmup raised to 3 (timing rule)")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    if args.study:
        run_study(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu_base = cpu_baseline_subprocess(args.workload, SAMPLE.get(args.workload, 20000), flux=flux_of(args))
        except Exception as e:  # reported, not fatal
            cpu_base = {"value": None, "error": str(e)[-300:]}
    r = run_ours(args, rank, world, device)
    fp64_leg = None
    if r["precision"].startswith("f16") and not args.no_fp64_leg:
        import copy
        a64 = copy.copy(args)
        a64.precision, a64.steps, a64.no_e2e = "fp64", 2, True
        r64 = run_ours(a64, rank, world, device)
        fp64_leg = {"value": r64["value"], "unit": "DOF-updates/s", "ms_per_step": r64["ms_per_step"], "steps": 2,
                    "warmup": a64.warmup, "roofline": r64["roofline"],
                    "mixed_over_fp64": r["value"] / r64["value"]}
    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": "DOF-updates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": r["precision"],
                "data": "synthetic", "config": config_of(args), "roofline": r["roofline"],
                "cpu_baseline": cpu_base, "e2e": r["e2e"], "clocks": r["clocks"],
                "gpu_launches": r["nlaunch"], "stage_ms": r["stage_ms"], "fp64": fp64_leg}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
