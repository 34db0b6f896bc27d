"""Benchmark of rapid Kriging prediction on GB300 (one JSON line on rank 0).

Workload (default "pred1024"): the 1024 x 1024 grid on [0,1]^2 with n = 20000
uniform sites and 16 data fields, Matern nu = 5/2, range 0.08, sigma^2 = 1,
tau^2 = 1e-3, L = 3 (M = 36; torus 2187^2).  One step is the rapid
prediction of the 16 fields from (sites, coefficients) resident in HBM: box
assignment and weights (steps 3-4), the exact low-frequency block, the
scatter c* = A^T c (step 5) and the FFT convolution and crop (steps 6-7),
replayed as a CUDA graph.  The coefficients c = M^{-1} z come from the
library's FP64 Cholesky at set-up, like the fitted model of the paper's
timing; z are seeded smooth fields at the sites (synth.smooth_field).

"paper350" runs the paper-scale configuration instead (n = 1368 clustered
sites, 350^2 grid on [0,1.6] x [0,1], range 0.15, tau^2 = 1e-3, nine cells
nu in {1/2, 3/2, 5/2} x L in {1, 2, 3}); by default it is measured as a
secondary, with conditional simulation (512^2, R = 256), the three-grid
simulation call (128^2, 256^2, 512^2, R = 64 each) and the 1024^2 adjoint.

The oracle (FP64, numpy, host cores) runs only in the cpu_baseline leg: its
rate on a bounded sample, and its values at seeded grid nodes, against which
the GPU outputs saved by the GPU arm are compared (the "error" entries).

--impl reference times the oracle on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "grid-point predictions/s (N x realizations)"
NODE_SAMPLE = 128          # seeded grid nodes per checked field


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pred1024", choices=["pred1024", "paper350"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU path")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the CPU oracle leg (rate and errors)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary measurements")
    ap.add_argument("--backward-n", type=int, default=None,
                    help="sites for the adjoint measurement (default: the workload's 20000)")
    ap.add_argument("--secondary-only", default=None,
                    choices=["paper350", "cs512", "cs_mixed", "table2", "factorial",
                             "grad1024_backward"],
                    help="run one secondary measurement alone and print it (for profiling)")
    return ap.parse_args()


# ------------------------------------------------------------------ workloads --

def workload_cells(name):
    """The workload's sites and [(cell name, plan kwargs, fields)]."""
    key = "grad1024" if name == "pred1024" else name
    w = synth.WORKLOADS[key]
    seed = synth.seed_for(w["config"])
    xy = synth.sites(w["sites"], w["n"], w["extent"], seed)
    cells = []
    if name == "paper350":
        for nu in w["nus"]:
            for L in w["Ls"]:
                cells.append((f"nu{nu}_L{L}", dict(nx=w["nx"], ny=w["ny"], extent=w["extent"],
                                                   nu=nu, rho=w["rho"], sigma2=w["sigma2"],
                                                   tau2=w["tau2"], L=L), w["B"]))
    else:
        cells.append((name, dict(nx=w["nx"], ny=w["ny"], extent=w["extent"], nu=w["nu"],
                                 rho=w["rho"], sigma2=w["sigma2"], tau2=w["tau2"],
                                 L=w["L"]), w["B"]))
    return w, xy, cells


def workload_data(name):
    """The data fields z (B x n): seeded smooth fields at the sites."""
    w, xy, cells = workload_cells(name)
    return synth.smooth_field(xy, cells[0][2], synth.seed_for(w["config"], 1))


def max_over_ranks(x, device):
    """MAX of x over the ranks of the default process group (x when alone):
    the replicas' timed region ends when the slowest one does."""
    import torch
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(name, world=1):
    """The workload part of the JSON line's config (both arms)."""
    w, xy, cells = workload_cells(name)
    kw = cells[0][1]
    cfg = {"workload": name, "grid": f"{kw['nx']}x{kw['ny']}", "n": int(xy.shape[0]),
           "fields_per_cell": cells[0][2], "parallelism": f"replicas x{world}",
           "data": "seeded smooth fields at the sites (synth.smooth_field); c = M^-1 z "
                   "by the library's FP64 Cholesky at set-up"}
    if name == "paper350":
        cfg["cells"] = [c[0] for c in cells]
        cfg["sites"] = "1368 clustered (60% jittered lattice, 40% in 5 Gaussian blobs)"
    else:
        cfg.update(nu=kw["nu"], range=kw["rho"], tau2=kw["tau2"], L=kw["L"])
    return cfg


def sample_nodes(nx, ny, seed=7, k=NODE_SAMPLE):
    rs = np.random.default_rng(seed)
    return rs.integers(0, nx, k), rs.integers(0, ny, k)


# -------------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- roofline --

def _load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# GB300's FP64 peak from its unit counts and clock: 152 SMs x 2070 MHz x
# 4 FP64 operations per clock per SM (two fused multiply-adds) = 1.26 TFLOP/s,
# NVIDIA's nominal 1.25 TFLOP/s
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12
# double-float on the FP32 pipe: 152 SMs x 128 lanes x 2070 MHz FP32
# instructions per second, 12 of them per double-float multiply-add of an
# unnormalised pair sum (product, its error, two cross terms, TwoSum, one
# add), 2 operations per multiply-add = 6.7 TFLOP/s of FP64-class work
DF_PEAK_TFLOPS = 152 * 128 * 2.070e9 / 12 * 2 / 1e12

# DRAM bytes (read + write) per launch from one ncu capture of the kernel (its
# summary file under profiles/ gives the command), the workload it was taken
# on and a digest of the sources it was built from; reported only while the
# sources are unchanged
TRAFFIC = {
    # ncu --set full of rcols<float, 2187, 9, 1, 4, 0> on this workload: one launch, 16 fields
    ("cols", "pred1024"): {"bytes_per_launch": 169529344 + 100468480,
                           "sources": ["k_fftr.cu", "fftr.cuh", "fft.cuh", "common.cuh"],
                           "digest": "a29201f8358c997c"},
}


def _sources_digest(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2605_29284_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload):
    t = TRAFFIC.get((kernel, workload))
    if not t:
        return None
    try:
        return t["bytes_per_launch"] if _sources_digest(t["sources"]) == t["digest"] else None
    except OSError:
        return None


def roofline(prof, steps, peaks, workload=None):
    """The dominant kernel's roofline (by time): HBM-bound passes as algorithmic
    bytes per second against the measured copy bandwidth, FP64 and
    double-float passes as algorithmic FP64-class operations per second."""
    hbm = peaks.get("hbm_gbs")
    src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    dname, (dl, dms, dbytes, dflops, dpipe) = max(prof.items(), key=lambda kv: kv[1][1])
    kernels = {}
    for k, v in prof.items():
        e = {"launches": v[0], "ms_per_step": v[1] / steps,
             "GBps": v[2] / (v[1] / 1e3) / 1e9 if v[1] > 0 else None,
             "bytes_per_launch": v[2] / v[0]}
        if v[3] > 0:
            key = "fp64_TFLOPs" if v[4] == 64 else "double_float_TFLOPs"
            e[key] = v[3] / (v[1] / 1e3) / 1e12 if v[1] > 0 else None
        kernels[k] = e
    traffic = _traffic(dname, workload)
    if dflops > 0:
        achieved = dflops / (dms / 1e3) / 1e12
        if dpipe == 64:
            peak, psrc = FP64_PEAK_TFLOPS, "nominal FP64 (152 SMs x 2070 MHz x 4)"
        else:
            peak, psrc = DF_PEAK_TFLOPS, ("double-float on the FP32 pipe (152 SMs x 128 lanes x "
                                          "2070 MHz / 12 instructions x 2)")
        roof = {"bound": "alu", "kernel": dname, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": psrc}
    else:
        achieved = dbytes / dl / (dms / dl / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                "peak_source": src + " copy bandwidth"}
    return roof, kernels


def transform_model_bytes(nx, ny, L, P):
    """Algorithmic bytes per FP32 field of the FFT convolution (steps 6-7) in the
    two-pass model: c* in, the row spectra out and in, the needed column results
    out and in, the window out: 4 P1^2 + 8 P1 H + 8 m H + 8 m H + 4 m^2 for a
    square grid (m = nx = ny, P1 = m + 2 (L - 1), H = P / 2 + 1)."""
    p1y, p1x, H = ny + 2 * (L - 1), nx + 2 * (L - 1), P // 2 + 1
    return 4.0 * p1y * p1x + 8.0 * p1y * H + 16.0 * ny * H + 4.0 * ny * nx


# ------------------------------------------------------------------ the arm --

class Arm:
    """One workload on one device: plans, resident inputs and a timed step."""

    def __init__(self, workload, precision, dev):
        import torch
        import paper_2605_29284_gb300 as rk
        self.torch, self.rk, self.dev = torch, rk, dev
        self.name = workload
        self.w, self.xy_np, self.cells = workload_cells(workload)
        self.z_np = workload_data(workload)
        self.xy = torch.from_numpy(self.xy_np).to(dev)
        self.st = []
        for name, kw, B in self.cells:
            p = rk.Plan(kw["nx"], kw["ny"], kw["extent"], kw["nu"], kw["rho"], kw["sigma2"],
                        kw["tau2"], kw["L"], precision=precision)
            # coefficients from the library's FP64 Cholesky (untimed set-up)
            p.set_obs(self.xy, torch.from_numpy(self.z_np[:B]).to(dev))
            c = p.debug_copy("coef").clone()
            out = torch.empty((B, kw["ny"], kw["nx"]), dtype=p.dtype, device=dev)
            self.st.append((p, c, out))
        self.points = sum(kw["nx"] * kw["ny"] * B for _, kw, B in self.cells)
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.streams = [torch.cuda.Stream(device=dev) for _ in self.st]
        tori = {(p.info()["px"], p.info()["py"]) for p, _, _ in self.st}
        self.grouped = len(tori) == 1 and len(self.st) <= 16
        self.graph = None
        torch.cuda.synchronize()

    def _issue(self):
        """One step: every cell's weights (site update), coefficients and
        prediction.  Cells sharing a torus go as groups (rk_set_sites_group:
        one weights launch per L; rk_set_coef_group: one copy launch;
        rk_predict_group: one launch per pass); otherwise one stream per cell."""
        torch = self.torch
        if self.grouped:
            plans = [p for p, _, _ in self.st]
            self.rk.set_sites_group(plans, [self.xy] * len(plans))
            self.rk.set_coef_group(plans, [c for _, c, _ in self.st])
            self.rk.predict_group(plans, [o for _, _, o in self.st])
            return
        cur = torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(cur)
        joins = []
        for (p, c, out), s in zip(self.st, self.streams):
            s.wait_event(fork)
            with torch.cuda.stream(s):
                p.set_sites_async(self.xy)
                p.set_coef(c)
                p.predict(out)
                e = torch.cuda.Event()
                e.record(s)
            joins.append(e)
        for e in joins:
            cur.wait_event(e)

    def capture(self):
        """Capture one step in a CUDA graph."""
        torch = self.torch
        for _ in range(2):
            self._issue()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._issue()
        torch.cuda.synchronize()

    def step(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._issue()

    def check(self):
        for p, _, _ in self.st:
            p.check_sites()

    def timed(self, steps, warmup, world=1, profile=False):
        torch, rk = self.torch, self.rk
        for _ in range(warmup):
            self.step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        total = 0.0
        if profile:
            rk.profile_read()
            rk.profile_enable(True)
        for _ in range(steps):
            self.flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            self.step()
            b.record()
            b.synchronize()
            total += a.elapsed_time(b)
            self.check()
        prof = None
        if profile:
            rk.profile_enable(False)
            prof = rk.profile_read()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return max_over_ranks(total, self.dev), prof

    def samples(self):
        """The last step's outputs at seeded nodes of the first and last field
        of every cell: {cell: [(field, jx, jy, values)]} (host arrays)."""
        self.torch.cuda.synchronize()
        res = {}
        for (name, kw, B), (p, c, out) in zip(self.cells, self.st):
            jx, jy = sample_nodes(kw["nx"], kw["ny"])
            o = out.double().cpu().numpy()
            res[name] = [(f, jx, jy, o[f][jy, jx]) for f in sorted({0, B - 1})]
        return res

    def e2e(self, steps, warmup):
        """The same step through the host-buffer API (a prepared
        rk_predict_host_group call, or rk_predict_host per cell): sites and
        coefficients in from pinned host memory, the grids back to it, inside
        the timed region (the kernels read and write the pinned buffers over
        NVLink-C2C)."""
        torch = self.torch
        xy = torch.from_numpy(self.xy_np).pin_memory().numpy()
        cs = [c.cpu().pin_memory().numpy() for _, c, _ in self.st]
        outs = [torch.empty(tuple(o.shape), dtype=o.dtype, pin_memory=True).numpy()
                for _, _, o in self.st]
        plans = [p for p, _, _ in self.st]
        call = self.rk.HostGroupCall(plans, [xy] * len(plans), cs, outs) if self.grouped else None

        def once():
            if call is not None:
                call.run()
            else:
                for p, c, o in zip(plans, cs, outs):
                    p.predict_host(xy, c, o)

        for _ in range(warmup):
            once()
        acc = 0.0
        for _ in range(steps):
            self.flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            once()
            acc += time.perf_counter() - t1
        n = self.xy_np.shape[0]
        esz = 4 if self.st[0][0].dtype == torch.float32 else 8
        h2d = sum(n * 2 * 8 + B * n * 8 for _, kw, B in self.cells)
        d2h = sum(B * kw["nx"] * kw["ny"] * esz for _, kw, B in self.cells)
        return self.points * steps / acc, h2d, d2h

    def launches_per_step(self):
        """Our kernels per step: per L one weights launch (grouped), the scatter
        order for n >= 4096 (scan, fill), for FP32 plans the block factors, the
        coefficient split and the block GEMM; the coefficient copy; a zeroing
        pass when a cell scatters with atomics (n < 4096); scatter, rows_fwd,
        cols, rows_inv."""
        f32 = self.st[0][0].dtype == self.torch.float32
        ncell = len(self.cells)
        nsite = int(self.xy_np.shape[0])
        order = 2 if nsite >= 4096 else 0
        zero = 0 if nsite >= 4096 else 1
        blk = 3 if f32 else 0
        if self.grouped:
            nL = len({kw["L"] for _, kw, _ in self.cells})
            return nL + ncell * order + blk + 1 + zero + 4
        return ncell * (1 + order + blk + 1 + zero + 4)

    def close(self):
        for p, _, _ in self.st:
            p.close()


# ------------------------------------------------------------ secondaries --

def measure_paper350(dev, steps, peaks, world):
    """The paper-scale step (nine cells) in FP32 and FP64, with outputs sampled
    for the oracle leg."""
    a = Arm("paper350", "fp32", dev)
    ms_p, prof = a.timed(steps, 2, world, profile=True)
    a.capture()
    ms, _ = a.timed(steps, 2, world)
    roof, kernels = roofline(prof, steps, peaks, "paper350")
    res = {"value": a.points * steps * world / (ms / 1e3), "unit": "grid-point predictions/s",
           "ms_per_step": ms / steps, "roofline": roof, "kernels": kernels,
           "config": workload_config("paper350", world)}
    samples = {"fp32": a.samples()}
    a.close()
    a64 = Arm("paper350", "fp64", dev)
    a64.capture()
    ms64, _ = a64.timed(max(2, steps // 2), 2, world)
    res["fp64_path"] = {"value": a64.points * max(2, steps // 2) * world / (ms64 / 1e3),
                        "ms_per_step": ms64 / max(2, steps // 2)}
    samples["fp64"] = a64.samples()
    a64.close()
    return res, samples


def _cs_plan(rk, torch, dev, name, nx, R=None):
    w = synth.WORKLOADS[name]
    xy = synth.sites(w["sites"], w["n"], w["extent"], synth.seed_for(w["config"]))
    z = synth.smooth_field(xy, 1, synth.seed_for(w["config"], 1))
    p = rk.Plan(nx, nx, w["extent"], w["nu"], w["rho"], w["sigma2"], w["tau2"], w["L"])
    p.set_obs(torch.from_numpy(xy).to(dev), torch.from_numpy(z).to(dev))
    return p, w, xy, z


def measure_cs(dev, steps, peaks, R=None):
    """Conditional simulation, 512 x 512 grid, n = 5000 sites, R realisations per
    call; realisations 0 and 1 of seed 1 are sampled for the oracle leg."""
    import torch
    import paper_2605_29284_gb300 as rk
    w = synth.WORKLOADS["cs512"]
    R = R or w["R"]
    t0 = time.perf_counter()
    p, _, _, _ = _cs_plan(rk, torch, dev, "cs512", w["nx"])
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    out = torch.empty((1, R, w["ny"], w["nx"]), dtype=torch.float32, device=dev)
    p.simulate(R, 1, out)
    torch.cuda.synchronize()
    jx, jy = sample_nodes(w["nx"], w["ny"])
    o = out[0, :2].double().cpu().numpy()
    sample = [(t, jx, jy, o[t][jy, jx]) for t in range(2)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    total = 0.0
    rk.profile_read()
    rk.profile_enable(True)
    for i in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        p.simulate(R, 100 + i, out)
        b.record()
        b.synchronize()
        total += a.elapsed_time(b)
    rk.profile_enable(False)
    prof = rk.profile_read()
    roof, kernels = roofline(prof, steps, peaks, "cs512")
    info = p.info()
    p.close()
    sec = total / steps / 1e3
    return {"realisations_per_s": R / sec,
            "value": R * w["nx"] * w["ny"] / sec, "unit": "grid-point predictions/s",
            "ms_per_call": sec * 1e3, "setup_cholesky_s": setup_s, "kernels": kernels,
            "roofline": roof,
            "config": {"grid": "512x512", "n": w["n"], "R": R, "nu": w["nu"], "range": w["rho"],
                       "L": w["L"], "tau2": w["tau2"], "ce_torus": [info["qx"], info["qy"]]}}, \
        sample


def measure_cs_mixed(dev, steps, peaks):
    """One rk_simulate_group call: the 128^2, 256^2 and 512^2 grids of one data
    set (n = 5000 sites, nu = 3/2, range 0.1, L = 2), R = 64 realisations
    each; realisations 0 and 1 of every grid are sampled for the oracle leg."""
    import torch
    import paper_2605_29284_gb300 as rk
    w = synth.WORKLOADS["cs_mixed"]
    R = w["R"]
    xy = synth.sites(w["sites"], w["n"], w["extent"], synth.seed_for(w["config"]))
    z = synth.smooth_field(xy, 1, synth.seed_for(w["config"], 1))
    plans = []
    for m in w["grids"]:
        p = rk.Plan(m, m, w["extent"], w["nu"], w["rho"], w["sigma2"], w["tau2"], w["L"])
        p.set_obs(torch.from_numpy(xy).to(dev), torch.from_numpy(z).to(dev))
        plans.append(p)
    outs = rk.simulate_group(plans, R, 1)
    torch.cuda.synchronize()
    sample = {}
    for m, o in zip(w["grids"], outs):
        jx, jy = sample_nodes(m, m)
        oo = o[0, :2].double().cpu().numpy()
        sample[m] = [(t, jx, jy, oo[t][jy, jx]) for t in range(2)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    total = 0.0
    for i in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        rk.simulate_group(plans, R, 100 + i, outs)
        b.record()
        b.synchronize()
        total += a.elapsed_time(b)
    qs = [p.info()["qx"] for p in plans]
    for p in plans:
        p.close()
    sec = total / steps / 1e3
    nreal = R * len(w["grids"])
    points = R * sum(m * m for m in w["grids"])
    return {"realisations_per_s": nreal / sec, "value": points / sec,
            "unit": "grid-point predictions/s", "ms_per_call": sec * 1e3,
            "config": {"grids": list(w["grids"]), "R_each": R, "n": w["n"], "nu": w["nu"],
                       "range": w["rho"], "L": w["L"], "tau2": w["tau2"], "ce_tori": qs,
                       "issue": "one rk_simulate_group call: one shared triangular solve "
                                "for the three grids' 192 right-hand sides"}}, sample


def _range_for_correlation(rk, nu, dist, corr=0.7):
    """range rho with phi(dist / rho) = corr, phi from the library's table
    (host evaluation, rk_matern_eval) by bisection in t = dist / rho."""
    lo, hi = 1e-6, 50.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if rk.matern_eval(nu, 0, [mid])[0] > corr else (lo, mid)
    return dist / (0.5 * (lo + hi))


def measure_factorial(dev, sets=5):
    """The factorial study of Section 3.1 on the GPU: mean absolute error of the
    rapid prediction against exact Kriging at five grid nodes (centre, quarter
    point, corner, two edge points) over `sets` seeded uniform site sets per
    cell, data drawn from the model (rk_draw_obs), sigma^2 = 1, on [0,1]^2.
    Levels: n 200/500/1500; range with correlation 0.7 at 0.2/0.4/0.8; nu
    0.5/1/1.5; tau^2 0.01/0.1/0.5; L 2/4 (the paper's L = 8, M = 256, is past
    this library's M <= 64); grids 100^2/350^2/500^2.  Reports the mean of
    log10(mean abs error) per level of each factor, and the worst cell."""
    import itertools
    import torch
    import paper_2605_29284_gb300 as rk
    levels = {"n": (200, 500, 1500), "dist": (0.2, 0.4, 0.8), "nu": (0.5, 1.0, 1.5),
              "tau2": (0.01, 0.1, 0.5), "L": (2, 4), "grid": (100, 350, 500)}
    ext = (0.0, 1.0, 0.0, 1.0)
    t0 = time.perf_counter()
    cells = []
    for nu, dist, tau2, L, m in itertools.product(levels["nu"], levels["dist"], levels["tau2"],
                                                  levels["L"], levels["grid"]):
        rho = _range_for_correlation(rk, nu, dist)
        nodes = [(m // 2, m // 2), (m // 4, m // 4), (0, 0), (0, m // 2), (m // 2, m - 1)]
        pts = torch.tensor([[i / (m - 1), j / (m - 1)] for i, j in nodes], dtype=torch.float64,
                           device=dev)
        jx = torch.tensor([i for i, _ in nodes], device=dev)
        jy = torch.tensor([j for _, j in nodes], device=dev)
        with rk.Plan(m, m, ext, nu, rho, 1.0, tau2, L, precision="fp64") as p:
            for n in levels["n"]:
                errs = []
                for k in range(sets):
                    seed = synth.seed_for(2, 1000 + 10 * k) + n
                    xy = torch.from_numpy(synth.sites_uniform(n, ext, seed)).to(dev)
                    p.set_sites(xy)
                    z = p.draw_obs(torch.from_numpy(synth.normals((1, n), seed + 1)).to(dev))
                    p.solve_coef(z)
                    exact = p.exact_predict(pts)[0]
                    rapid = p.predict()[0][jy, jx]
                    errs.append((rapid - exact).abs())
                e = torch.stack(errs).mean().item()
                cells.append({"nu": nu, "dist": dist, "tau2": tau2, "L": L, "grid": m, "n": n,
                              "range": rho, "mean_abs_error": e})
    torch.cuda.synchronize()
    effects = {}
    for f, lv in levels.items():
        effects[f] = {str(v): float(np.mean([np.log10(c["mean_abs_error"]) for c in cells
                                             if c[f] == v])) for v in lv}
    worst = max(cells, key=lambda c: c["mean_abs_error"])
    return {"cells": len(cells), "sets_per_cell": sets, "seconds": time.perf_counter() - t0,
            "mean_log10_error_by_level": effects, "worst_cell": worst,
            "paper": "worst case nu = 0.5, tau^2 = 0.01, L = 2: mean log10 error below -2; "
                     "error falls with nu, L, grid size and tau^2 (Table 1 / A2)"}


def measure_table2(dev):
    """Lambda(Omega, s*) of Section 3.2 on the GPU over Table 2's grids
    (range 0.25, L = 2, m in 20 .. 200, mesh h / 2) and the fitted orders."""
    import torch
    import paper_2605_29284_gb300 as rk
    ms = [20, 40, 60, 80, 100, 140, 200]
    res, t0 = {}, time.perf_counter()
    for nu in (0.5, 1.0, 1.5, 2.5):
        lam = []
        for m in ms:
            with rk.Plan(m, m, (0.0, 1.0, 0.0, 1.0), nu, 0.25, 1.0, 1e-3, 2,
                         precision="fp64") as p:
                lam.append(p.kernel_error(2))
        use = [i for i, m in enumerate(ms) if nu != 2.5 or m <= 140]
        slope = -np.polyfit(np.log10([ms[i] for i in use]), np.log10([lam[i] for i in use]),
                            1)[0]
        res[str(nu)] = {"lambda": lam, "order": float(slope)}
    torch.cuda.synchronize()
    return {"grids": ms, "by_nu": res, "seconds": time.perf_counter() - t0,
            "paper_orders": {"0.5": 1.00, "1.0": 1.99, "1.5": 2.00, "2.5 (<= 140^2)": 2.99}}


def measure_backward(dev, steps, peaks, n=None):
    """Forward and adjoint on the 1024 x 1024 grid, 16 fields, nu = 5/2, L = 3,
    and the FP32 theta-gradients against central differences of the FP64 map
    (4-point stencil, step 0.03 in log range and log sigma^2; fields 0, 15)."""
    import torch
    import paper_2605_29284_gb300 as rk
    w = synth.WORKLOADS["grad1024"]
    n = n or w["n"]
    xy_np = synth.sites(w["sites"], n, w["extent"], synth.seed_for(w["config"]))
    xy = torch.from_numpy(xy_np).to(dev)
    z = torch.from_numpy(synth.smooth_field(xy_np, w["B"], synth.seed_for(w["config"], 1))).to(dev)
    gbar = torch.from_numpy(synth.normals((w["B"], w["ny"], w["nx"]),
                                          synth.seed_for(w["config"], 2))).float().to(dev)
    args = (w["nx"], w["ny"], w["extent"], w["nu"], w["rho"], w["sigma2"], w["tau2"], w["L"])
    p = rk.Plan(*args)
    t0 = time.perf_counter()
    p.set_obs(xy, z)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    y = p.predict()
    p.backward(gbar)
    torch.cuda.synchronize()
    fwd = bwd = 0.0
    for _ in range(steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        c = torch.cuda.Event(enable_timing=True)
        a.record()
        p.predict(y)
        b.record()
        p.backward(gbar)
        c.record()
        c.synchronize()
        fwd += a.elapsed_time(b)
        bwd += b.elapsed_time(c)
    # one more adjoint with per-pass events (apart from the timed calls)
    rk.profile_read()
    rk.profile_enable(True)
    p.backward(gbar)
    torch.cuda.synchronize()
    rk.profile_enable(False)
    roof, kernels = roofline(rk.profile_read(), 1, peaks, "grad1024_backward")
    _, g_rho, g_s2 = (t.cpu().numpy() if t is not None else None for t in p.backward(gbar))
    p.close()
    # central differences of sum(gbar * g_hat) in FP64 plans
    fields = [0, w["B"] - 1]
    gb64 = gbar.double()[fields]
    z2 = z[fields].contiguous()

    def loss(rho, s2):
        a2 = list(args)
        a2[4], a2[5] = rho, s2
        with rk.Plan(*a2, precision="fp64") as q:
            q.set_obs(xy, z2)
            return (q.predict() * gb64).sum(dim=(1, 2)).cpu().numpy()
    # a 4-point stencil at h = 0.03 (error O(h^4)): the weights of each
    # re-created plan carry the rounding of the neighbourhood solve (cond K_N
    # ~ 1e12 at nu = 5/2, L = 3), which swamps quotients of steps near 1e-4
    h = 0.03
    r0, s0 = w["rho"], w["sigma2"]

    def d4(f):
        return (8.0 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12.0 * h)
    fd_rho = d4(lambda t: loss(r0 * np.exp(t), s0))
    fd_s2 = d4(lambda t: loss(r0, s0 * np.exp(t)))
    err = max(float(np.abs(g_rho[fields] - fd_rho).max() / np.abs(fd_rho).max()),
              float(np.abs(g_s2[fields] - fd_s2).max() / np.abs(fd_s2).max()))
    with rk.Plan(*args, precision="fp64") as q:
        q.set_obs(xy, z2)
        _, r64, s64 = (t.cpu().numpy() for t in q.backward(gb64))
    detail = {"fd_rho": fd_rho.tolist(), "fd_s2": fd_s2.tolist(),
              "fp32_rho": g_rho[fields].tolist(), "fp32_s2": g_s2[fields].tolist(),
              "fp64_rho": r64.tolist(), "fp64_s2": s64.tolist()}
    return {"forward_ms": fwd / steps, "backward_ms": bwd / steps,
            "value": w["B"] * w["nx"] * w["ny"] / ((fwd + bwd) / steps / 1e3),
            "unit": "grid-point predictions/s (forward + adjoint)", "setup_cholesky_s": setup_s,
            "kernels": kernels, "roofline": roof,
            "gradient_error_vs_fd": {"value": err, "fields": fields, "step": h,
                                     "stencil": "4-point", "detail": detail,
                                     "what": "max over log range and log sigma^2 of |FP32 "
                                             "adjoint - central difference of the FP64 map| / "
                                             "max |difference|"},
            "config": {"grid": "1024x1024", "n": n, "fields": w["B"], "nu": w["nu"],
                       "range": w["rho"], "L": w["L"], "tau2": w["tau2"]}}


# ------------------------------------------------------------ CPU oracle --

def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def oracle_setup(workload):
    """The oracle's coefficients c = M^{-1} z for every cell (dense FP64
    Cholesky of K_xx + tau^2 I), timed as set-up."""
    from oracle import kriging
    w, xy, cells = workload_cells(workload)
    z = workload_data(workload)
    t0 = time.perf_counter()
    coef = {}
    for name, kw, B in cells:
        coef[name] = kriging.coef(xy, z[:B].T, kw["nu"], kw["rho"], kw["sigma2"], kw["tau2"]).T
    return xy, cells, coef, time.perf_counter() - t0


def oracle_rate(workload, setup, budget_s=15.0, steps=1):
    """Oracle predictions/s: weights, scatter and direct Eq. (9) sums at batches
    of 256 seeded grid nodes of the middle cell, for about budget_s."""
    from oracle import rapid
    xy, cells, coef, setup_s = setup
    name, kw, B = cells[len(cells) // 2]
    g = rapid.Grid(kw["nx"], kw["ny"], kw["extent"], kw["L"])
    c = coef[name][:1]
    rs = np.random.default_rng(7)
    nodes = 256
    total_pts, total_t = 0, 0.0
    for _ in range(steps):
        t0 = time.perf_counter()
        while True:
            jx = rs.integers(0, g.nx, nodes)
            jy = rs.integers(0, g.ny, nodes)
            ix, iy, W = rapid.weights(xy, g, kw["nu"], kw["rho"], kw["sigma2"])
            cs = rapid.scatter(ix, iy, W, c, g)
            rapid.bttb_predict(cs, g, kw["nu"], kw["rho"], kw["sigma2"], jx=jx, jy=jy, chunk=32)
            total_pts += nodes
            if time.perf_counter() - t0 > budget_s / steps:
                break
        total_t += time.perf_counter() - t0
    return {"value": total_pts / total_t, "unit": "grid-point predictions/s", "cores": _cores(),
            "kind": "oracle", "setup_s": setup_s,
            "sample": f"{workload} cell {name}, one field: weights, scatter and direct Eq. (9) "
                      f"sums at batches of {nodes} seeded grid nodes for ~{budget_s:.0f} s "
                      "(numpy FP64, BLAS threads = host cores); the set-up (the dense Cholesky "
                      "of K_xx + tau^2 I for every cell and field) is timed apart"}


def oracle_errors(setup, samples):
    """max |GPU - oracle| / max |oracle| over the sampled nodes of every cell,
    per precision; the oracle sums Eq. (9) directly with its own weights and
    coefficients."""
    from oracle import rapid
    xy, cells, coef, _ = setup
    res = {}
    for prec, by_cell in samples.items():
        worst = 0.0
        per = {}
        for name, kw, B in cells:
            g = rapid.Grid(kw["nx"], kw["ny"], kw["extent"], kw["L"])
            ix, iy, W = rapid.weights(xy, g, kw["nu"], kw["rho"], kw["sigma2"])
            e = 0.0
            for f, jx, jy, vals in by_cell[name]:
                cs = rapid.scatter(ix, iy, W, coef[name][f], g)
                ref = rapid.bttb_predict(cs, g, kw["nu"], kw["rho"], kw["sigma2"], jx=jx,
                                         jy=jy, chunk=32)[0]
                e = max(e, float(np.abs(vals - ref).max() / np.abs(ref).max()))
            per[name] = e
            worst = max(worst, e)
        res[prec] = worst
        if len(per) > 1:
            res[prec + "_per_cell"] = per
    res["nodes_per_field"] = NODE_SAMPLE
    res["what"] = ("max |GPU - oracle| / max |oracle| at seeded grid nodes of the first and "
                   "last field, oracle = direct Eq. (9) sums with its own weights and "
                   "Cholesky coefficients (FP64 CPU)")
    return res


def oracle_cs_error(sample):
    """Realisations 0 and 1 of the 512^2 simulation (seed 1) against the oracle's
    own conditional simulation (same Philox streams), at the sampled nodes."""
    from oracle import cs, rapid
    w = synth.WORKLOADS["cs512"]
    xy = synth.sites(w["sites"], w["n"], w["extent"], synth.seed_for(w["config"]))
    z = synth.smooth_field(xy, 1, synth.seed_for(w["config"], 1))
    g = rapid.Grid(w["nx"], w["ny"], w["extent"], w["L"])
    ref = cs.simulate(xy, z, g, w["nu"], w["rho"], w["sigma2"], w["tau2"], 2, 1)[0]
    e = 0.0
    for t, jx, jy, vals in sample:
        r = ref[t][jy, jx]
        e = max(e, float(np.abs(vals - r).max() / np.abs(r).max()))
    return {"fp32": e, "what": "realisations 0, 1 at seeded nodes against the oracle's "
                               "simulation with the same counter-based noise"}


def oracle_cs_mixed_error(sample):
    """Realisations 0 and 1 of each grid of the group call against the oracle's
    simulation of that grid alone (same seed, same noise)."""
    from oracle import cs, rapid
    w = synth.WORKLOADS["cs_mixed"]
    xy = synth.sites(w["sites"], w["n"], w["extent"], synth.seed_for(w["config"]))
    z = synth.smooth_field(xy, 1, synth.seed_for(w["config"], 1))
    e = 0.0
    for m, rows in sample.items():
        g = rapid.Grid(m, m, w["extent"], w["L"])
        ref = cs.simulate(xy, z, g, w["nu"], w["rho"], w["sigma2"], w["tau2"], 2, 1)[0]
        for t, jx, jy, vals in rows:
            r = ref[t][jy, jx]
            e = max(e, float(np.abs(vals - r).max() / np.abs(r).max()))
    return {"fp32": e, "what": "realisations 0, 1 of every grid at seeded nodes against "
                               "the oracle's simulation of that grid"}


def cpu_leg(workload, samples, secondary_samples, budget_s=15.0):
    """Everything that runs the oracle: its rate (cpu_baseline) and the errors
    of the GPU outputs sampled by the GPU arm."""
    setup = oracle_setup(workload)
    cb = oracle_rate(workload, setup, budget_s)
    errors = {workload: oracle_errors(setup, samples)} if samples else {}
    if "paper350" in secondary_samples:
        errors["paper350"] = oracle_errors(oracle_setup("paper350"),
                                           secondary_samples["paper350"])
    if "cs512" in secondary_samples:
        errors["cs512"] = oracle_cs_error(secondary_samples["cs512"])
    if "cs_mixed" in secondary_samples:
        errors["cs_mixed"] = oracle_cs_mixed_error(secondary_samples["cs_mixed"])
    return cb, errors


# --------------------------------------------------------------- our arm --

def run_ours(args, rank, world):
    import torch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    peaks = _load_peaks()
    main = Arm(args.workload, args.precision, dev)
    sampler = ClockSampler(dev.index)
    sampler.start()
    # timed region 1: the step issued from the host with per-kernel CUDA events
    # (the roofline's kernel durations); timed region 2: the same step replayed
    # from a CUDA graph (the headline value)
    prof_ms, prof = main.timed(args.steps, args.warmup, world, profile=True)
    main.capture()
    total_ms, _ = main.timed(args.steps, args.warmup, world)
    clocks = sampler.stop()
    samples = {args.precision: main.samples()}
    value = main.points * args.steps * world / (total_ms / 1e3)
    value_nograph = main.points * args.steps * world / (prof_ms / 1e3)
    roof, kernels = roofline(prof, args.steps, peaks, args.workload)
    ms_step = total_ms / args.steps
    hbm = peaks.get("hbm_gbs") or 6800.0
    _, _, cells = workload_cells(args.workload)
    model = 0.0
    for (_, kw, B), (p, _, _) in zip(cells, main.st):
        model += B * transform_model_bytes(kw["nx"], kw["ny"], kw["L"], p.info()["px"])
    step_roof = {"model_bytes_per_step": model, "achieved_GBps": model / (ms_step / 1e3) / 1e9,
                 "peak_GBps": hbm, "frac": model / (ms_step / 1e3) / 1e9 / hbm,
                 "what": "the FFT convolution's algorithmic bytes (4 P1^2 + 8 P1 H + 16 m H + "
                         "4 m^2 per FP32 field) over the whole step's time, weights and "
                         "scatter included"}
    main.graph = None
    e2e_value, h2d, d2h = main.e2e(max(3, args.steps // 2), 2)
    launches = main.launches_per_step()
    main.close()
    fp64 = None
    if not args.no_fp64 and args.precision == "fp32":
        a64 = Arm(args.workload, "fp64", dev)
        k64 = max(2, args.steps // 5)
        a64.capture()
        ms64, _ = a64.timed(k64, 2, world)
        v64 = a64.points * k64 * world / (ms64 / 1e3)
        fp64 = {"value": v64, "unit": "grid-point predictions/s", "ms_per_step": ms64 / k64,
                "speedup_fp32_over_fp64": value / v64}
        samples["fp64"] = a64.samples()
        a64.close()
    secondary, sec_samples = {}, {}
    if not args.no_secondary:
        k = max(3, args.steps // 2)
        if args.workload != "paper350":
            secondary["paper350"], sec_samples["paper350"] = measure_paper350(dev, k, peaks,
                                                                              world)
        secondary["cs512_simulate"], sec_samples["cs512"] = measure_cs(dev, max(2, args.steps // 5),
                                                                       peaks)
        secondary["cs_mixed_simulate"], sec_samples["cs_mixed"] = measure_cs_mixed(
            dev, max(2, args.steps // 5), peaks)
        secondary["grad1024_backward"] = measure_backward(dev, max(2, args.steps // 5), peaks,
                                                          n=args.backward_n)
        secondary["table2_kernel_error"] = measure_table2(dev)
        secondary["factorial"] = measure_factorial(dev)
    res = {
        "metric": METRIC, "value": value, "unit": "grid-point predictions/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic (seeded sites and smooth data fields)",
        "config": {**workload_config(args.workload, world),
                   "l2": "flushed between timed steps (256 MB write)",
                   "issue": ("the cells' site updates grouped (rk_set_sites_group), their "
                             "predictions grouped (rk_predict_group: one launch per pass), "
                             "the step replayed from a CUDA graph"),
                   "value_without_graph": value_nograph},
        "roofline": roof,
        "step_roofline": step_roof,
        "kernels": kernels,
        "e2e": {"value": e2e_value, "unit": "grid-point predictions/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
        "fp64_path": fp64,
        "secondary": secondary,
    }
    return res, samples, sec_samples


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        setup = oracle_setup(args.workload)
        cb = oracle_rate(args.workload, setup, budget_s=max(10.0, 2.0 * args.steps),
                         steps=args.steps)
        cfg = workload_config(args.workload, 1)
        w, _, cells = workload_cells(args.workload)
        points = sum(kw["nx"] * kw["ny"] * B for _, kw, B in cells)
        res = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": cb["unit"],
               "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": points / cb["value"] * 1e3,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic (seeded sites and smooth data fields)",
               "config": {**cfg, "issue": "the FP64 CPU oracle on the host cores (sampled)"},
               "cpu_baseline": cb,
               "e2e": {"value": cb["value"], "unit": cb["unit"], "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(res))
        return 0
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.secondary_only:
        import torch
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
        torch.cuda.set_device(dev)
        peaks = _load_peaks()
        if args.secondary_only == "paper350":
            out = measure_paper350(dev, args.steps, peaks, 1)[0]
        elif args.secondary_only == "cs512":
            out = measure_cs(dev, args.steps, peaks)[0]
        elif args.secondary_only == "cs_mixed":
            out = measure_cs_mixed(dev, args.steps, peaks)[0]
        elif args.secondary_only == "table2":
            out = measure_table2(dev)
        elif args.secondary_only == "factorial":
            out = measure_factorial(dev)
        else:
            out = measure_backward(dev, args.steps, peaks, n=args.backward_n)
        if rank == 0:
            print(json.dumps({"secondary": args.secondary_only, **out}))
        return 0
    res, samples, sec_samples = run_ours(args, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu:
        res["cpu_baseline"], res["error"] = cpu_leg(args.workload, samples, sec_samples)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
