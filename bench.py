"""Benchmark of the plain FV rollout: decaying turbulence, 256^2, batch 16, FP32.

One bench step is one call of the library's rollout over the whole workload:
16 trajectories of 2D incompressible decaying turbulence on a periodic 2 pi box,
256 x 256 cells, nu = 1e-3 (Re = 1000), dt = 1.75e-3, 2000 time steps of four RK4
stages each, every stage projected with the spectral Poisson solve. The metric
is cell-updates/s = 256^2 x 16 x 2000 / (time of one bench step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own 16 trajectories (replicas, weak
scaling, no collective on the data path); rank 0 prints one JSON line.
``--impl reference`` times the FP64 oracle on the host cores on a bounded
sample of the same workload (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, BATCH, STEPS_PER_ROLLOUT = 256, 16, 2000
NU, DT = 1e-3, 1.75e-3
METRIC = "cell-updates/s"
UNIT = "cell-updates/s"
WORKLOAD = "decaying NS 256^2, batch 16, 2000-step RK4 rollout (FP32, spectral projection)"
# algorithmic FP32 flops per cell and time step, per RK stage: 8 face operators x 4 taps x 2 (64),
# flux assembly (24), RK combination (8), divergence (4), gradient (4), spectral multiply (2) and a
# real-to-complex plus complex-to-real 2D FFT pair (2 x 2.5 log2(N^2) = 10 log2 N per cell)
FLOP_PER_CELL_STEP = 4 * (64 + 24 + 8 + 4 + 4 + 2 + 10 * math.log2(N))
SMS, FP32_LANES = 152, 128


def _sample_clocks(stop: threading.Event, out: list):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return
    try:
        while not stop.is_set():
            line = p.stdout.readline()
            if not line:
                break
            out.append(line.strip())
    finally:
        p.terminate()
        try:
            p.wait(timeout=2)
        except Exception:
            p.kill()


def _clock_summary(lines, dev: int):
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9 or not f[0].isdigit() or int(f[0]) != dev:
            continue
        try:
            sm.append(float(f[1]))
            mx = max(mx, float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons)}


# DRAM bytes (read + write) of one launch of the on-chip rollout kernel on the
# 256^2 workload with 15 trajectories on chip, from an ncu capture of the
# current kernel: the 7.86 MB state read plus a little; the launch's final
# 7.86 MB write drains after the kernel ends and is not counted. None until a
# capture of the current kernel exists.
ONCHIP_DRAM_BYTES_PER_LAUNCH = 7.95e6


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# the profiling recipe's fallback denominators, used only when no measured
# peaks file is present on the box
_FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def _peak(key: str):
    """(value, basis) of a roofline denominator: measured on this machine when the
    driver's peaks file exists, else the recipe's fallback."""
    v = _measured_peaks().get(key)
    if isinstance(v, (int, float)) and v > 0:
        return float(v), "of measured"
    return _FALLBACK_PEAKS[key], "of fallback"


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.processor() or platform.machine()


def _oracle_job(args):
    """One oracle trajectory on one core (runs in a spawn-started worker):
    ('c2', seed, steps) decaying 256^2; ('c1', seed, steps) Burgers 32^2 FP64
    with 2nd-order operators; ('c3', seed, steps) learned 64^2 Kolmogorov.
    Returns (cell-updates, seconds)."""
    import oracle as O
    from paper_2507_01975_gb300 import inputs as I

    kind, seed, steps = args
    if kind == "c2":
        p = O.Problem(nx=N, ny=N, nu=NU, dt=DT)
        U = I.decaying_ic(N, seed)
        step = lambda U: O.rk4_step(U, p)  # noqa: E731
    elif kind == "c1":
        p = O.Problem(nx=32, ny=32, nu=0.01, dt=1e-3, flow=O.FLOW_BURGERS, deriv_order=2)
        U = I.burgers_ic(32, seed)
        step = lambda U: O.rk4_step(U, p)  # noqa: E731
    else:
        p = O.Problem(nx=64, ny=64, nu=1e-3, dt=1.75e-3, forcing_kind=1)
        st = I.random_conv_stack(1, 2, 64, 160, last_scale=0.05)
        model = O.LearnedModel(W_L=I.random_wl(3, 1e-2), stencil=st)
        U = I.kolmogorov_ic(64, seed)
        step = lambda U: O.learned_step(U, p, model)  # noqa: E731
    t0 = time.perf_counter()
    for _ in range(steps):
        U = step(U)
    el = time.perf_counter() - t0
    return U.shape[1] * U.shape[2] * steps, el


def _pool(procs):
    import multiprocessing as mp

    pool = mp.get_context("spawn").Pool(procs)
    pool.map(_oracle_job, [("c1", k, 1) for k in range(procs)])  # start and import in every worker
    return pool


def _rate_all_cores(pool, procs, kind, steps):
    t0 = time.perf_counter()
    res = pool.map(_oracle_job, [(kind, k, steps) for k in range(procs)], chunksize=1)
    wall = time.perf_counter() - t0
    return sum(r[0] for r in res) / wall, wall


def run_reference(args):
    """FP64 oracle on all host cores (one trajectory per core), bounded sample of
    the same workload: each bench step advances nproc trajectories of the 256^2
    decaying flow by one time step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    procs = os.cpu_count() or 1
    pool = _pool(procs)
    for _ in range(args.warmup):
        _rate_all_cores(pool, procs, "c2", 1)
    t = []
    for _ in range(args.steps):
        t.append(_rate_all_cores(pool, procs, "c2", 1)[1])
    pool.close()
    pool.join()
    cells = N * N * procs
    value = cells * args.steps / sum(t)
    sample = (f"{procs} trajectories x 1 time step of the 256^2 decaying flow per bench step, one trajectory per "
              f"host core (FP64 numpy oracle, {_cpu_model()})")
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(t) / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline():
    """Time the oracle as it stands on the host cores (about 20 s of CPU work):
    one core, and every core with one trajectory each, on the headline workload
    (decaying 256^2) and on the Burgers 32^2 FP64 and learned 64^2 Kolmogorov
    workloads. The line's value is the all-core rate on the headline workload."""
    procs = os.cpu_count() or 1
    pool = _pool(procs)
    per = {}
    for kind, steps_one, steps_all, what in (
            ("c2", 30, 30, "decaying NS 256^2 (FP64)"),
            ("c1", 200, 200, "Burgers 32^2, 200 steps (FP64, 2nd-order operators)"),
            ("c3", 1, 1, "learned 64^2 Kolmogorov step (stencil network in FP64 loops)")):
        cells, el = _oracle_job((kind, 0, steps_one))
        all_rate, wall = _rate_all_cores(pool, procs, kind, steps_all)
        per[kind] = {"workload": what, "one_core": cells / el, "all_cores": all_rate,
                     "one_core_sample": f"1 trajectory x {steps_one} steps ({el:.1f} s)",
                     "all_cores_sample": f"{procs} trajectories x {steps_all} steps ({wall:.1f} s)"}
    pool.close()
    pool.join()
    return {
        "value": per["c2"]["all_cores"],
        "unit": UNIT,
        "cores": procs,
        "kind": "oracle",
        "cpu_model": _cpu_model(),
        "nproc": procs,
        "sample": per["c2"]["all_cores_sample"] + " of the 256^2 decaying flow, one trajectory per core "
                                                  "(FP64 numpy, 1 thread per process)",
        "per_workload": per,
    }


def learned_measurement(fd, I, steps: int = 60):
    """Learned-stencil inference (Kolmogorov 64^2, batch 128, BF16 network on the
    tensor cores, temporal correction every 4 steps): cell-updates/s and the
    tensor-core rate of the stencil network, timed with CUDA events."""
    import torch

    n, b, kc = 64, 128, 4
    st = I.random_conv_stack(1, 2, 64, 160, last_scale=0.05)
    tc = I.random_conv_stack(2, 2 * kc, 64, 2, last_scale=0.02)
    s = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", nu=1e-3, dt=1.75e-3, forcing="kolmogorov",
                            learned=True, k_c=kc))
    s.set_params(I.pack_params(I.random_wl(3, 1e-2), st, tc))
    U0 = np.stack([I.kolmogorov_ic(n, k) for k in range(b)]).astype(np.float32)
    u = torch.tensor(U0, device="cuda")
    o = torch.empty_like(u)
    coef = torch.empty((b, 160, n, n), device="cuda")
    for _ in range(2):
        s.rollout(u, o, 8)
        s.network_forward(u, coef)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.rollout(u, o, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / steps
    reps = 10
    s.network_forward(u)
    e0.record(stream)
    for _ in range(reps):
        s.network_forward(u)  # input packing + the 7 convolution launches, no FP32 unpacking
    e1.record(stream)
    torch.cuda.synchronize()
    ms_net = e0.elapsed_time(e1) / reps
    flop_net = 481_536 * n * n * b  # one stencil-network evaluation (6 conv3x3 layers)
    flop_step = (4 * 481_536 + (2 * kc * 64 * 9 * 2 + 4 * 64 * 64 * 9 * 2 + 64 * 2 * 9 * 2) / kc) * n * n * b
    # the network is timed on its own (a short burst of launches): burst peak
    peak, basis = _peak("bf16_tflops")
    peak_sus, _ = _peak("bf16_tflops_sustained")
    achieved = flop_net / (ms_net * 1e-3) / 1e12
    # the same step with the Fourier operators of the forced-flow configuration
    # (Table S3): O_F (6 layers, 32 modes, width 16) in the flux block and the
    # temporal correction as an FNO (4 layers, 32 modes, width 8), FP32 on the CUDA cores
    fno = I.random_fno(4, 16, 32, 6, out_scale=0.01)
    tcf = I.random_fno(5, 8, 32, 4, out_scale=0.01, cin=2 * kc, cout=2)
    sf = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", nu=1e-3, dt=1.75e-3, forcing="kolmogorov",
                             learned=True, k_c=kc, fno_layers=6, fno_modes=32, fno_width=16,
                             tc_fno_layers=4, tc_fno_modes=32, tc_fno_width=8))
    sf.set_params(I.pack_params(I.random_wl(3, 1e-2), st, tcf, fno))
    for _ in range(2):
        sf.rollout(u, o, 8)
    torch.cuda.synchronize()
    e0.record(stream)
    sf.rollout(u, o, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fno = e0.elapsed_time(e1) / steps
    fno_ok = bool(sf.check_finite(o))
    sf.close()
    return {
        "workload": "Kolmogorov 64^2, batch 128, learned stencil network (6 conv3x3, 64 ch, BF16) + temporal correction k_c=4",
        "with_frequency_operator": {"fno": "O_F 6 Fourier layers, 32 modes, width 16; FNO temporal correction "
                                           "4 layers, 32 modes, width 8 (FP32)",
                                    "ms_per_time_step": ms_fno, "value": n * n * b / (ms_fno * 1e-3),
                                    "finite": fno_ok},
        "value": n * n * b / (ms_step * 1e-3),
        "unit": "cell-updates/s",
        "ms_per_time_step": ms_step,
        "step_tflops": flop_step / (ms_step * 1e-3) / 1e12,
        "finite": bool(s.check_finite(o)),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "stencil network forward (input packing + 7 conv3x3_tc_kernel launches per evaluation)",
                     "peak_basis": f"cuBLAS bf16 burst ({basis}): the network is timed alone",
                     "frac_of_sustained": achieved / peak_sus},
    }


def training_measurement(fd, I, iters: int = 5):
    """Differentiable training (shear layer 64^2, batch 32, 32-step unrolled
    rollouts through the hand-written adjoint, checkpoints every 8 steps, MSE,
    Adam): milliseconds per training iteration and the rollout cell-updates per
    second it sustains, timed with CUDA events."""
    import torch

    from paper_2507_01975_gb300.train import TrainConfig, Trainer

    n, b, unroll, ckpt = 64, 32, 32, 8
    nu, dt = 1e-3, 7e-3
    st = I.random_conv_stack(4, 2, 64, 160, last_scale=0.05)
    params = I.pack_params(I.random_wl(5, 1e-2), st)
    s = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", nu=nu, dt=dt, learned=True))
    plain = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", nu=nu, dt=dt))
    u0 = torch.tensor(np.stack([I.shear_ic(n)] * b).astype(np.float32), device="cuda")
    # labels: the plain coarse solver's rollout (stand-in for coarse-grained fine-grid states)
    tgt = torch.empty((unroll, b, 2, n, n), device="cuda")
    last = torch.empty_like(u0)
    plain.rollout(u0, last, unroll, traj=tgt, save_every=1)
    tr = Trainer(s, params, TrainConfig(unroll=unroll, ckpt_every=ckpt, lr=1e-4))
    for _ in range(2):
        tr.step(u0, tgt)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(iters):
        loss = tr.step(u0, tgt)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_iter = e0.elapsed_time(e1) / iters
    # one step's reverse mode alone
    lam = torch.ones_like(u0)
    dp = torch.zeros(s.param_count(), device="cuda")
    s.step_adjoint(u0, lam, lam, dp)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(iters):
        s.step_adjoint(u0, lam, lam, dp)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_adj = e0.elapsed_time(e1) / iters
    return {
        "workload": "shear layer 64^2, batch 32, 32-step unrolled rollouts, checkpoints every 8 steps, MSE, Adam "
                    "(labels: plain coarse rollout)",
        "ms_per_iteration": ms_iter,
        "value": n * n * b * unroll / (ms_iter * 1e-3),
        "unit": "rollout cell-updates/s (forward + reverse mode + Adam)",
        "ms_per_step_adjoint": ms_adj,
        "loss": float(loss.item()),
        "paper_grids": paper_grid_training(fd, I, iters),
    }


def paper_grid_training(fd, I, iters: int):
    """Training iterations of the models on the paper's own coarse grids, which
    run on the generic-grid path (CUDA-core network, FP32 reverse mode): the
    Burgers LDSolver on 25^2 over [0, 1]^2 and the shear-flow LDSolver on 128 x 64
    over [0, 8] x [0, 4], both at dt = 1e-2 with the stencil network and a CNN
    temporal correction every k_c = 4 steps; labels are the plain coarse rollout."""
    import torch

    from paper_2507_01975_gb300.train import TrainConfig, Trainer

    out = {}
    kc = 4
    cases = (("burgers_25x25", dict(n=25, flow="burgers", nu=0.002, lx=1.0, ly=1.0), 16, 16,
              lambda: I.burgers_ic(25, 1, lx=1.0)),
             ("shear_128x64", dict(n=128, ny=64, nu=1e-3, lx=8.0, ly=4.0), 4, 8,
              lambda: I.shear_scalar_ic(128, 64)[0]))
    for name, geo, b, unroll, ic in cases:
        cfg = dict(batch=b, dtype="f32", dt=1e-2, **geo)
        s = fd.Solver(fd.Config(learned=True, k_c=kc, **cfg))
        plain = fd.Solver(fd.Config(**cfg))
        st = I.random_conv_stack(4, 2, 64, 160, last_scale=0.05)
        tc = I.random_conv_stack(6, 2 * kc, 64, 2, last_scale=0.02)
        u0 = torch.tensor(np.stack([ic()] * b).astype(np.float32), device="cuda")
        tgt = torch.empty((unroll,) + tuple(u0.shape), device="cuda")
        plain.rollout(u0, torch.empty_like(u0), unroll, traj=tgt, save_every=1)
        tr = Trainer(s, I.pack_params(I.random_wl(5, 1e-2), st, tc), TrainConfig(unroll=unroll, ckpt_every=kc, lr=1e-4))
        tr.step(u0, tgt)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(iters):
            loss = tr.step(u0, tgt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / iters
        out[name] = {"batch": b, "unroll": unroll, "ckpt_every": kc, "k_c": kc, "ms_per_iteration": ms,
                     "rollout_cell_updates_per_s": s.state_shape[2] * s.state_shape[3] * b * unroll / (ms * 1e-3),
                     "loss": float(loss.item())}
        s.close()
        plain.close()
    out["shear_128x64_with_scalar"] = joint_training(fd, I, iters)
    return out


def joint_training(fd, I, iters: int, b: int = 4, unroll: int = 8, kc: int = 4, D: float = 2e-3):
    """Training iterations of the shear-flow model that learns the passive scalar
    (network on (u, v, s), CNN temporal correction every k_c steps) on 128 x 64 at
    dt = 1e-2: fd_train_step_scalar (checkpointed joint rollout, MSE over velocity
    and scalar) and an Adam update; labels are the plain coarse joint rollout."""
    import torch

    nx, ny = 128, 64
    cfg = dict(n=nx, ny=ny, batch=b, dtype="f32", nu=1e-3, dt=1e-2, lx=8.0, ly=4.0)
    s = fd.Solver(fd.Config(learned=True, k_c=kc, scalar_learned=True, **cfg))
    plain = fd.Solver(fd.Config(**cfg))
    st = I.random_conv_stack(4, 3, 64, 240, last_scale=0.05)
    tc = I.random_conv_stack(6, 2 * kc, 64, 2, last_scale=0.02)
    theta = torch.tensor(I.pack_params(I.random_wl(5, 1e-2), st, tc, W_Ls=I.random_wl(8, 1e-2)), device="cuda")
    grad, m, v = torch.zeros_like(theta), torch.zeros_like(theta), torch.zeros_like(theta)
    s.set_params_device(theta)
    ics = [I.shear_scalar_ic(nx, ny, seed=k) for k in range(b)]
    u0 = torch.tensor(np.stack([x for x, _ in ics]).astype(np.float32), device="cuda")
    s0 = torch.tensor(np.stack([y for _, y in ics]).astype(np.float32), device="cuda")
    tu = torch.empty((unroll,) + tuple(u0.shape), device="cuda")
    ts = torch.empty((unroll,) + tuple(s0.shape), device="cuda")
    uu, ss = u0.clone(), s0.clone()
    for k in range(unroll):  # labels one step at a time: the plain joint rollout
        plain.rollout_scalar(uu, ss, tu[k], ts[k], 1, D)
        uu, ss = tu[k], ts[k]
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def it(t):
        s.train_step_scalar(D, u0, s0, tu, ts, unroll, kc, grad, loss)
        fd.adam_step(theta, grad, m, v, t, 1e-4, 0.9, 0.999, 1e-8, zero_grads=True)
        s.set_params_device(theta)

    it(1)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for t in range(iters):
        it(t + 2)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    s.close()
    plain.close()
    return {"batch": b, "unroll": unroll, "ckpt_every": kc, "k_c": kc, "diffusivity": D, "ms_per_iteration": ms,
            "rollout_cell_updates_per_s": nx * ny * b * unroll / (ms * 1e-3), "loss": float(loss.item())}


# algorithmic minimum per cell and time step: read and write the FP32 state (u, v)
ALGO_BYTES_PER_CELL_STEP = 16
# HBM bytes per cell and time step that the streaming path's kernels move (FP32):
# stage kernels 32 + 44 + 44 + 36, projections 4 x (12 + 8 + 8), final 20
STREAM_BYTES_PER_CELL_STEP = 288


def fine_measurement(fd, I, steps: int = 40):
    """Plain FV 2048^2 FP32, one trajectory, streaming path (the fine-grid
    reference): cell-updates/s and the whole step's effective HBM bandwidth
    against the measured copy bandwidth."""
    import torch

    n = 2048
    s = fd.Solver(fd.Config(n=n, batch=1, dtype="f32", nu=1e-3, dt=2.19e-4))
    u = torch.tensor(I.decaying_ic(n, 0)[None].astype(np.float32), device="cuda")
    o = torch.empty_like(u)
    s.rollout(u, o, 4)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.rollout(u, o, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    gbs = ALGO_BYTES_PER_CELL_STEP * n * n / (ms * 1e-3) / 1e9
    gbs_model = STREAM_BYTES_PER_CELL_STEP * n * n / (ms * 1e-3) / 1e9
    peak, basis = _peak("hbm_gbs")
    # energy spectrum of the final state (analysis kernels: row and column FFTs of
    # u + iv, shell sums); algorithmic traffic 24 B per cell (state in, complex
    # scratch out and back in)
    spec = torch.empty((1, n // 2 + 1), dtype=torch.float64, device="cuda")
    s.energy_spectrum(o, spec)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        s.energy_spectrum(o, spec)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_spec = e0.elapsed_time(e1) / reps
    return {
        "workload": "decaying NS 2048^2, batch 1, FP32, streaming path (17 launches per step, CUDA graph)",
        "value": n * n / (ms * 1e-3),
        "unit": "cell-updates/s",
        "ms_per_time_step": ms,
        "finite": bool(s.check_finite(o)),
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                     "traffic": None, "kernel": "whole step (stage, FFT and final kernels)",
                     "algorithmic_bytes_per_cell_step": ALGO_BYTES_PER_CELL_STEP,
                     "peak_basis": f"copy bandwidth ({basis})",
                     "implementation_model": {
                         "bytes_per_cell_step": STREAM_BYTES_PER_CELL_STEP,
                         "note": "HBM traffic of this implementation's 17 launches per step (each RK stage "
                                 "reads and writes the state, accumulator and stage result, and every "
                                 "projection passes its field through three FFT kernels)",
                         "achieved_gbs": gbs_model, "frac": gbs_model / peak}},
        "energy_spectrum": {"ms": ms_spec, "kmax": n // 2,
                            "gbs_at_24_bytes_per_cell": 24 * n * n / (ms_spec * 1e-3) / 1e9,
                            "energy": float(spec.sum().item())},
    }


def corr_measurement(fd, I, n_fine: int = 2048, n_train: int = 8, n_test: int = 4, warm: float = 4.0,
                     horizon: float = 4.0, iters: int = 300, unroll: int = 16, lr: float = 1e-3, rt: int = 32,
                     kc: int = 4):
    """Wall time to a 0.95 vorticity correlation, learned vs plain FV (forced flow, Re = 1000).

    A fine plain-FV reference (n_fine^2, streaming path) is warmed up from random
    fields, then coarse-grained (face averages to 64^2, every rt fine steps: the
    coarse step is 32 fine 2048^2 steps, Table S2) into labels. The learned 64^2
    solver (stencil network + temporal-correction head every kc steps, both last
    layers zero-initialised so training starts from the plain solver) is trained
    here with Adam on the first n_train trajectories: unrolled MSE through the
    hand-written adjoint (fd_train_step). Plain solvers at 64 .. n_fine/2 (same
    CFL number) and the learned solver start from the coarse-grained state of the
    test trajectories; their vorticity correlation with the labels (min over the
    test trajectories) is tracked to the horizon. H = the time the learned
    solver keeps the correlation >= 0.95 (the horizon if it never drops); the
    cheapest plain solver that keeps it >= 0.95 through H is the match, and the
    reported ratio is its wall time to H over the learned solver's (same GPU,
    same batch, CUDA events).
    """
    import torch

    from paper_2507_01975_gb300.train import TrainConfig, Trainer

    nc, nu = 64, 1e-3
    dt_f = 2.19e-4 * 2048 / n_fine
    rt = rt * n_fine // 2048
    dt_c = rt * dt_f
    B = n_train + n_test
    kt = int(round(horizon / dt_c))
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn):
        e0, e1 = ev(), ev()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    t0 = time.perf_counter()
    fine = fd.Solver(fd.Config(n=n_fine, batch=B, dtype="f32", nu=nu, dt=dt_f, forcing="kolmogorov"))
    u = torch.tensor(np.stack([I.kolmogorov_ic(n_fine, 200 + k) for k in range(B)]).astype(np.float32), device="cuda")
    fine.rollout(u, u, int(round(warm / dt_f)))
    labels = torch.empty((kt + 1, B, 2, nc, nc), device="cuda")
    fd.downsample(u, labels[0], n_fine // nc)
    u_fine0 = u.clone()
    for k in range(kt):
        fine.rollout(u, u, rt)
        fd.downsample(u, labels[k + 1], n_fine // nc)
    torch.cuda.synchronize()
    fine.close()
    t_ref = time.perf_counter() - t0
    lt = labels[:, :n_train].contiguous()
    lv = labels[:, n_train:].contiguous()
    test0 = u_fine0[n_train:].contiguous()
    del u, u_fine0
    corr = torch.zeros(n_test, dtype=torch.float64, device="cuda")
    scorer = fd.Solver(fd.Config(n=nc, batch=n_test, dtype="f32"))

    def curve_of(solver, n, steps_per_coarse):
        u0 = torch.empty((n_test, 2, n, n), device="cuda")
        fd.downsample(test0, u0, n_fine // n)
        traj = torch.empty((kt, n_test, 2, n, n), device="cuda")
        last = torch.empty_like(u0)
        solver.rollout(u0, last, kt * steps_per_coarse, traj=traj, save_every=steps_per_coarse)
        coarse = torch.empty((n_test, 2, nc, nc), device="cuda")
        curve = []
        for k in range(kt):
            fd.downsample(traj[k], coarse, n // nc)
            scorer.vorticity_pcc(coarse, lv[k + 1], corr)
            curve.append(float(corr.min().item()))
        t95 = next(((k + 1) * dt_c for k, c in enumerate(curve) if c < 0.95), None)
        return u0, curve, t95

    def wall_to(solver, u0, t, dt):
        steps = max(1, int(round(t / dt)))
        last = torch.empty_like(u0)
        solver.rollout(u0, last, steps)  # warm (graphs, plans)
        return min(timed(lambda: solver.rollout(u0, last, steps)) for _ in range(2)), steps

    # learned 64^2 with the temporal correction: zero-initialised last layers
    st = I.random_conv_stack(11, 2, 64, 160, last_scale=0.0)
    tc = I.random_conv_stack(12, 2 * kc, 64, 2, last_scale=0.0)
    params = I.pack_params(np.zeros((2, 2, 5, 4)), st, tc)
    ls = fd.Solver(fd.Config(n=nc, batch=n_train, dtype="f32", nu=nu, dt=dt_c, forcing="kolmogorov", learned=True,
                             k_c=kc))
    tr = Trainer(ls, params, TrainConfig(unroll=unroll, ckpt_every=8, lr=lr))
    rng = np.random.default_rng(0)
    losses = []
    t_train = 0.0
    for it in range(iters):
        s0 = int(rng.integers(0, kt - unroll + 1))
        t_train += timed(lambda: tr.step(lt[s0], lt[s0 + 1:s0 + 1 + unroll]))
        if it % 25 == 0 or it == iters - 1:
            losses.append(float(tr.loss.item()))
    le = fd.Solver(fd.Config(n=nc, batch=n_test, dtype="f32", nu=nu, dt=dt_c, forcing="kolmogorov", learned=True,
                             k_c=kc))
    le.set_params_device(tr.theta)
    u0l, curve_l, t95_l = curve_of(le, nc, 1)
    H = t95_l if t95_l is not None else kt * dt_c
    wall_l, steps_l = wall_to(le, u0l, H, dt_c)
    out = {"workload": f"forced NS (Re 1000): {n_fine}^2 plain-FV reference (warm-up {warm} time units from random "
                       f"fields) face-averaged to 64^2 every {rt} fine steps; learned 64^2 solver (stencil network + "
                       f"temporal correction every {kc} steps, dt {dt_c:.3g}) trained here on {n_train} trajectories; "
                       f"{n_test} test trajectories, horizon {horizon} time units",
           "H_learned": H,
           "solvers": {"learned64": {"t_corr_095": t95_l, "corr_at_horizon": curve_l[-1],
                                     "corr_curve_every_20": curve_l[::20], "wall_ms_to_H": wall_l, "steps_to_H": steps_l,
                                     "ms_per_step": wall_l / steps_l}},
           "training": {"iterations": iters, "unroll": unroll, "lr": lr, "loss_every_25": losses,
                        "seconds": t_train / 1e3},
           "reference_seconds": t_ref}
    for n in [m for m in (64, 128, 256, 512, 1024) if m < n_fine]:
        dt_n = dt_f * n_fine / n
        s = fd.Solver(fd.Config(n=n, batch=n_test, dtype="f32", nu=nu, dt=dt_n, forcing="kolmogorov"))
        u0, curve, t95 = curve_of(s, n, rt * n // n_fine)
        wall, steps = wall_to(s, u0, H, dt_n)
        out["solvers"][f"plain{n}"] = {"t_corr_095": t95, "corr_at_horizon": curve[-1],
                                       "corr_curve_every_20": curve[::20], "wall_ms_to_H": wall, "steps_to_H": steps,
                                       "ms_per_step": wall / steps,
                                       "holds_095_through_H": t95 is None or t95 > H}
        s.close()
    matches = [(k, v) for k, v in out["solvers"].items() if k.startswith("plain") and v["holds_095_through_H"]]
    if matches:
        k, v = min(matches, key=lambda kv: kv[1]["wall_ms_to_H"])
        out["cheapest_plain_matching_learned"] = k
        out["wall_time_ratio_plain_over_learned"] = v["wall_ms_to_H"] / wall_l
    else:
        out["cheapest_plain_matching_learned"] = None
        out["wall_time_ratio_plain_over_learned"] = None
    return out


def resweep_measurement(fd, I, train_re: float = 1000.0, res=(200.0, 500.0, 1000.0, 1500.0, 2000.0),
                        n_fine: int = 1024, n_train: int = 8, n_test: int = 4, warm: float = 2.0,
                        horizon: float = 3.0, iters: int = 300, unroll: int = 16, lr: float = 1e-3, kc: int = 4):
    """Generalisation over the Reynolds number (the paper's Re sweep, Sec. 4): the
    learned 64^2 solver (stencil network + temporal-correction head) is trained once,
    on forced-flow labels at Re = train_re (an n_fine^2 plain-FV reference
    face-averaged to 64^2), then evaluated, unchanged, at every Re of the sweep (the
    context's viscosity is 1/Re; the network is the same) against a fresh reference
    at that Re. Reported per Re: the time the vorticity correlation (min over the
    test trajectories) stays >= 0.95 for the learned solver and for plain FV at
    64^2, and the correlation at the horizon."""
    import torch

    from paper_2507_01975_gb300.train import TrainConfig, Trainer

    nc = 64
    dt_f = 2.19e-4 * 2048 / n_fine
    rt = 32 * n_fine // 2048
    dt_c = rt * dt_f
    kt = int(round(horizon / dt_c))

    def reference(nu, batch, seed0):
        fine = fd.Solver(fd.Config(n=n_fine, batch=batch, dtype="f32", nu=nu, dt=dt_f, forcing="kolmogorov"))
        u = torch.tensor(np.stack([I.kolmogorov_ic(n_fine, seed0 + k) for k in range(batch)]).astype(np.float32),
                         device="cuda")
        fine.rollout(u, u, int(round(warm / dt_f)))
        labels = torch.empty((kt + 1, batch, 2, nc, nc), device="cuda")
        fd.downsample(u, labels[0], n_fine // nc)
        for k in range(kt):
            fine.rollout(u, u, rt)
            fd.downsample(u, labels[k + 1], n_fine // nc)
        torch.cuda.synchronize()
        fine.close()
        return labels

    t0 = time.perf_counter()
    lt = reference(1.0 / train_re, n_train, 500)
    st = I.random_conv_stack(21, 2, 64, 160, last_scale=0.0)
    tc = I.random_conv_stack(22, 2 * kc, 64, 2, last_scale=0.0)
    ls = fd.Solver(fd.Config(n=nc, batch=n_train, dtype="f32", nu=1.0 / train_re, dt=dt_c, forcing="kolmogorov",
                             learned=True, k_c=kc))
    tr = Trainer(ls, I.pack_params(np.zeros((2, 2, 5, 4)), st, tc), TrainConfig(unroll=unroll, ckpt_every=8, lr=lr))
    rng = np.random.default_rng(1)
    for _ in range(iters):
        s0 = int(rng.integers(0, kt - unroll + 1))
        tr.step(lt[s0], lt[s0 + 1:s0 + 1 + unroll])
    torch.cuda.synchronize()
    final_loss = float(tr.loss.item())
    corr = torch.zeros(n_test, dtype=torch.float64, device="cuda")
    scorer = fd.Solver(fd.Config(n=nc, batch=n_test, dtype="f32"))

    def horizon_of(solver, labels):
        u0 = labels[0].clone()
        traj = torch.empty((kt, n_test, 2, nc, nc), device="cuda")
        last = torch.empty_like(u0)
        solver.rollout(u0, last, kt, traj=traj, save_every=1)
        curve = []
        for k in range(kt):
            scorer.vorticity_pcc(traj[k], labels[k + 1], corr)
            curve.append(float(corr.min().item()))
        t95 = next(((k + 1) * dt_c for k, c in enumerate(curve) if c < 0.95), None)
        return {"t_corr_095": t95, "corr_at_horizon": curve[-1]}

    rows = {}
    for re_ in res:
        nu = 1.0 / re_
        lv = reference(nu, n_test, 900)
        le = fd.Solver(fd.Config(n=nc, batch=n_test, dtype="f32", nu=nu, dt=dt_c, forcing="kolmogorov", learned=True,
                                 k_c=kc))
        le.set_params_device(tr.theta)
        pl = fd.Solver(fd.Config(n=nc, batch=n_test, dtype="f32", nu=nu, dt=dt_c, forcing="kolmogorov"))
        rows[f"Re{int(re_)}"] = {"learned64": horizon_of(le, lv), "plain64": horizon_of(pl, lv)}
        le.close()
        pl.close()
    return {"workload": f"forced NS, learned 64^2 (stencil network + temporal correction every {kc} steps, "
                        f"dt {dt_c:.3g}) trained at Re {int(train_re)} on {n_train} trajectories of a {n_fine}^2 "
                        f"reference ({iters} Adam iterations), evaluated unchanged at each Re against a fresh "
                        f"{n_fine}^2 reference ({n_test} test trajectories, horizon {horizon})",
            "final_training_loss": final_loss, "per_re": rows, "seconds": time.perf_counter() - t0}


def batch_measurement(fd, I, T: float = 0.5, reps: int = 3):
    """Mixed batch (512 trajectories): plain FP32 32^2 Burgers, 64^2 decaying, 128^2
    Kolmogorov, 256^2 shear (64 each) and learned BF16-network 32^2 Kolmogorov and 64^2
    decaying (128 each), every group advanced by the same physical time T with the
    CFL-matched step dt(N) = 1.75e-3 * 256 / N, all in one graph (fd_batch: the plain
    32^2 and 64^2 trajectories in one persistent launch, the other groups as branches).
    Reported: cell-updates/s of the graph, the graph without the persistent launch, and
    the same rollouts run one after another."""
    import torch

    st = I.random_conv_stack(12, 2, 64, 160, last_scale=0.05)
    params = I.pack_params(I.random_wl(13, 1e-2), st)
    groups = [(32, 64, "burgers", False), (64, 64, "decaying", False), (128, 64, "kolmogorov", False),
              (256, 64, "shear", False), (32, 128, "kolmogorov", True), (64, 128, "decaying", True)]
    batch, tuned = fd.Batch(), fd.Batch()
    runs = []
    cells = 0
    for n, b, kind, learned in groups:
        dt = 1.75e-3 * 256 / n
        steps = int(round(T / dt))
        cfg = fd.Config(n=n, batch=b, dtype="f32", nu=1e-2 if kind == "burgers" else 1e-3, dt=dt,
                        flow="burgers" if kind == "burgers" else "ns",
                        forcing="kolmogorov" if kind == "kolmogorov" else None, learned=learned)
        s = fd.Solver(cfg)
        if learned:
            s.set_params(params)
        u0 = torch.tensor(I.ic_batch(kind, n, b, seed0=300).astype(np.float32), device="cuda")
        out = torch.empty_like(u0)
        batch.add(s, u0, out, steps)
        runs.append((s, u0, out, steps))
        cells += b * n * n * steps
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_batch(bt):
        bt.run()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            bt.run()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = timed_batch(batch)
    persistent = batch.persistent_count()
    batch.set_persistent(False)  # every context its own branch of the graph
    ms_branches = timed_batch(batch)
    batch.close()
    # the same batch after each context's autotuner picked its plan (timed alone)
    plans = []
    for s, u0, out, steps in runs:
        s.autotune(probe_steps=16)
        plans.append(s.plan())
        tuned.add(s, u0, out, steps)
    ms_tuned = timed_batch(tuned)
    tuned_launches = tuned.launch_count()
    tuned.close()
    for s, u0, out, steps in runs:  # warm every solver's own path
        s.rollout(u0, out, steps)
    e0.record(stream)
    for s, u0, out, steps in runs:
        s.rollout(u0, out, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    return {"workload": "512 trajectories: plain FP32 32^2 Burgers, 64^2 decaying, 128^2 Kolmogorov, 256^2 shear "
                        "(64 each) + learned 32^2 Kolmogorov, 64^2 decaying (128 each), physical time 0.5 each",
            "value": cells / (min(ms, ms_tuned) * 1e-3), "unit": "cell-updates/s",
            "ms_per_batch_default_plans": ms, "ms_per_batch_autotuned_plans": ms_tuned,
            "persistent_trajectories": persistent, "ms_per_batch_without_persistent_launch": ms_branches,
            "autotuned_plans": [{k: p[k] for k in ("path", "cluster", "n_onchip", "n_stream")} for p in plans],
            "ms_one_after_another": ms_seq, "graph_kernel_launches_autotuned": tuned_launches,
            "finite": all(bool(s.check_finite(out)) for s, _, out, _ in runs)}


# FLOPs per pixel of one stencil-network evaluation on the generic-grid path for a
# model that learns the scalar: six 3x3 layers 3 -> 64 x 5 -> 240, 2 per multiply-add
GEN_NET_FLOP_PER_PIXEL = 2 * 9 * (3 * 64 + 4 * 64 * 64 + 64 * 240)


def generic_learned_measurement(fd, I, steps: int = 20):
    """The generic-grid path's learned joint step on the shear flow's model grid
    (128 x 64 on [0, 8] x [0, 4], batch 16, dt = 1e-2, D = 2e-3): a model that
    learns the scalar (network on (u, v, s), 240 channels) with a CNN temporal
    correction every 4 steps, through fd_rollout_scalar (graph-replayed groups).
    The CUDA-core network dominates; its roofline is the FP32 FMA peak."""
    import torch

    nx, ny, b, kc = 128, 64, 16, 4
    cfg = fd.Config(n=nx, ny=ny, batch=b, dtype="f32", nu=1e-3, dt=1e-2, lx=8.0, ly=4.0, learned=True, k_c=kc,
                    scalar_learned=True)
    s = fd.Solver(cfg)
    st = I.random_conv_stack(1, 3, 64, 240, last_scale=0.05)
    tc = I.random_conv_stack(6, 2 * kc, 64, 2, last_scale=0.02)
    s.set_params(I.pack_params(I.random_wl(3, 1e-2), st, tc, W_Ls=I.random_wl(7, 1e-2)))
    ics = [I.shear_scalar_ic(nx, ny, seed=k) for k in range(b)]
    u = torch.tensor(np.stack([x for x, _ in ics]).astype(np.float32), device="cuda")
    sc = torch.tensor(np.stack([y for _, y in ics]).astype(np.float32), device="cuda")
    uo, so = torch.empty_like(u), torch.empty_like(sc)
    s.rollout_scalar(u, sc, uo, so, steps, 2e-3)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    stop, lines = threading.Event(), []
    sampler = threading.Thread(target=_sample_clocks, args=(stop, lines), daemon=True)
    sampler.start()
    for _ in range(3):
        e0.record(stream)
        s.rollout_scalar(u, sc, uo, so, steps, 2e-3)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / steps)
    stop.set()
    sampler.join(timeout=5)
    clocks = _clock_summary(lines, torch.cuda.current_device())
    finite = bool(s.check_finite(uo))
    s.close()
    flop_step = 4 * GEN_NET_FLOP_PER_PIXEL * nx * ny * b
    peak = SMS * FP32_LANES * 2 * (clocks.get("sm_mhz") or 2070.0) * 1e6 / 1e12
    return {"workload": "shear flow 128 x 64, batch 16, learned joint step (network on (u, v, s), 240 channels, "
                        "CNN temporal correction k_c = 4), dt 1e-2, D 2e-3, generic-grid path",
            "ms_per_step": best, "value": nx * ny * b / (best * 1e-3), "unit": "cell-updates/s", "finite": finite,
            "clocks": clocks,
            "network_roofline": {"bound": "alu", "achieved": flop_step / (best * 1e-3) / 1e12,
                                 "peak": peak, "unit": "TFLOP/s",
                                 "frac": flop_step / (best * 1e-3) / 1e12 / peak,
                                 "note": "stencil-network FLOPs of the whole step over the whole step's time "
                                         "(FP32 on the CUDA cores; the face, flux, projection and correction "
                                         "kernels count as zero FLOPs)",
                                 "peak_basis": "FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x the median SM clock "
                                               "sampled during the timed rollouts"}}


def adjoint_measurement(fd, I, iters: int = 5):
    """Reverse mode of one learned step (shear layer 64^2, batch 32) alone."""
    import torch

    n, b = 64, 32
    st = I.random_conv_stack(4, 2, 64, 160, last_scale=0.05)
    s = fd.Solver(fd.Config(n=n, batch=b, dtype="f32", nu=1e-3, dt=7e-3, learned=True))
    s.set_params(I.pack_params(I.random_wl(5, 1e-2), st))
    u0 = torch.tensor(np.stack([I.shear_ic(n)] * b).astype(np.float32), device="cuda")
    lam = torch.ones_like(u0)
    dp = torch.zeros(s.param_count(), device="cuda")
    s.step_adjoint(u0, lam, lam, dp)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(iters):
        s.step_adjoint(u0, lam, lam, dp)
    e1.record(stream)
    torch.cuda.synchronize()
    return {"workload": "reverse mode of one learned step, shear layer 64^2, batch 32",
            "ms_per_step_adjoint": e0.elapsed_time(e1) / iters, "launches_per_call": s.last_launch_count()}


def speed_measurement(fd, I, reps: int = 3):
    """GPU seconds per simulated physical second, batch 1: the only speed figure the
    paper reports (Table 4, on an A100), on its grids. DNS rows run the plain solver:
    Burgers 100^2 on [0, 1]^2 with dt = 1e-3 (Table S2) on the generic-grid path;
    decaying and forced Navier-Stokes 1024^2 with dt = 2.19e-4 (the fine step of
    Table S2; the paper does not give the 1024^2 one) on the streaming path; the
    shear layer 1024 x 512 on [0, 8] x [0, 4] with dt = 3.125e-4 on the generic-grid
    path. Model rows (random weights): the learned 64^2 solver with the paper's
    forced-flow learnable module (stencil network, O_F of 6 layers / 32 modes / width
    16, FNO temporal correction of 4 layers / 32 modes / width 8, k_c = 4) at
    dt = 32 x 2.19e-4 on the tensor-core path; Burgers 25^2 at dt = 1e-2 and the
    shear layer 128 x 64 at dt = 1e-2 with the stencil network and a CNN temporal
    correction (k_c = 4) on the generic-grid path, whose learned module has no
    Fourier operators. The plain 25^2 Burgers solver is reported beside its model.
    Both shear rows advance the passive scalar with the velocity (D = 2e-3): the DNS
    with the physics kernels, the model with its learned scalar operators (network on
    (u, v, s), 240 channels)."""
    import torch

    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def per_physical_second(s, U0, dt, S0=None, D=2e-3):
        u = torch.tensor(U0, device="cuda")
        o = torch.empty_like(u)
        steps = int(round(1.0 / dt))
        if S0 is None:
            run = lambda: s.rollout(u, o, steps)
        else:
            sc = torch.tensor(S0, device="cuda")
            so = torch.empty_like(sc)
            run = lambda: s.rollout_scalar(u, sc, o, so, steps, D)
        run()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0.record(stream)
            run()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        finite = bool(s.check_finite(o))
        s.close()
        return {"seconds": best, "steps": steps, "finite": finite}

    paper = {"burgers": (2.3067, 0.9800), "decaying": (29.2402, 2.3773), "forced": (32.8061, 3.8036),
             "shear": (29.1428, 2.7857)}
    rows = {}
    st = I.random_conv_stack(1, 2, 64, 160, last_scale=0.05)
    dt_f, kc = 2.19e-4, 4
    tcc = I.random_conv_stack(6, 2 * kc, 64, 2, last_scale=0.02)
    dns = fd.Solver(fd.Config(n=100, batch=1, dtype="f32", flow="burgers", nu=0.002, dt=1e-3, lx=1.0, ly=1.0))
    coarse = fd.Solver(fd.Config(n=25, batch=1, dtype="f32", flow="burgers", nu=0.002, dt=1e-2, lx=1.0, ly=1.0))
    lrn25 = fd.Solver(fd.Config(n=25, batch=1, dtype="f32", flow="burgers", nu=0.002, dt=1e-2, lx=1.0, ly=1.0,
                                learned=True, k_c=kc))
    lrn25.set_params(I.pack_params(I.random_wl(3, 1e-2), st, tcc))
    b25 = I.burgers_ic(25, 1, lx=1.0)[None].astype(np.float32)
    rows["burgers"] = {"dns_100x100": per_physical_second(dns, I.burgers_ic(100, 1, lx=1.0)[None].astype(np.float32),
                                                          1e-3),
                       "plain_25x25": per_physical_second(coarse, b25, 1e-2),
                       "learned_25x25": per_physical_second(lrn25, b25, 1e-2)}
    fno = I.random_fno(4, 16, 32, 6, out_scale=0.01)
    tcf = I.random_fno(5, 8, 32, 4, out_scale=0.01, cin=2 * kc, cout=2)
    for flow, forcing, ic in (("decaying", None, I.decaying_ic), ("forced", "kolmogorov", I.kolmogorov_ic)):
        dns = fd.Solver(fd.Config(n=1024, batch=1, dtype="f32", nu=1e-3, dt=dt_f, forcing=forcing))
        lrn = fd.Solver(fd.Config(n=64, batch=1, dtype="f32", nu=1e-3, dt=32 * dt_f, forcing=forcing, learned=True,
                                  k_c=kc, fno_layers=6, fno_modes=32, fno_width=16, tc_fno_layers=4,
                                  tc_fno_modes=32, tc_fno_width=8))
        lrn.set_params(I.pack_params(I.random_wl(3, 1e-2), st, tcf, fno))
        rows[flow] = {"dns_1024x1024": per_physical_second(dns, ic(1024, 0)[None].astype(np.float32), dt_f),
                      "learned_64x64": per_physical_second(lrn, ic(64, 0)[None].astype(np.float32), 32 * dt_f)}
    dns = fd.Solver(fd.Config(n=1024, ny=512, batch=1, dtype="f32", nu=1e-3, dt=3.125e-4, lx=8.0, ly=4.0))
    lrn = fd.Solver(fd.Config(n=128, ny=64, batch=1, dtype="f32", nu=1e-3, dt=1e-2, lx=8.0, ly=4.0, learned=True,
                              k_c=kc, scalar_learned=True))
    st_s = I.random_conv_stack(1, 3, 64, 240, last_scale=0.05)
    lrn.set_params(I.pack_params(I.random_wl(3, 1e-2), st_s, tcc, W_Ls=I.random_wl(7, 1e-2)))
    (uf, sf), (uc, sc) = I.shear_scalar_ic(1024, 512), I.shear_scalar_ic(128, 64)
    f32 = lambda a: a[None].astype(np.float32)
    rows["shear"] = {"dns_1024x512_with_scalar": per_physical_second(dns, f32(uf), 3.125e-4, f32(sf)),
                     "learned_128x64_with_scalar": per_physical_second(lrn, f32(uc), 1e-2, f32(sc))}
    for k, (p_dns, p_model) in paper.items():
        rows[k]["paper_a100"] = {"dns": p_dns, "ldsolver": p_model}
    return {"unit": "GPU seconds per simulated physical second, batch 1 (min of %d runs)" % reps, **rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-stencil inference measurement")
    ap.add_argument("--no-training", action="store_true", help="skip the training-step measurement")
    ap.add_argument("--no-fine", action="store_true", help="skip the 2048^2 streaming-path measurement")
    ap.add_argument("--no-resweep", action="store_true",
                    help="skip the Reynolds-number generalisation sweep of the learned solver")
    ap.add_argument("--no-corr", action="store_true",
                    help="skip the wall-time-to-0.95-correlation measurement (learned vs plain FV)")
    ap.add_argument("--no-speed", action="store_true",
                    help="skip the GPU-seconds-per-physical-second measurement on the paper's grids")
    ap.add_argument("--only", choices=["learned", "training", "adjoint", "fine", "corr", "batch", "speed", "resweep",
                                       "glearned"],
                    help="run one side measurement alone and print its JSON (for profiling)")
    ap.add_argument("--iters", type=int, default=5, help="iterations of the side measurement (--only)")
    ap.add_argument("--plan", default=None,
                    help="cluster,n_onchip,n_stream: fix the launch plan instead of autotuning it (profiling "
                         "under ncu, which serialises kernels and so changes the autotuner's ranking)")
    ap.add_argument("--time-steps", type=int, default=STEPS_PER_ROLLOUT,
                    help="time steps per rollout (the workload's 2000 by default; smaller only for ncu captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_2507_01975_gb300 import build as B
    from paper_2507_01975_gb300 import fd
    from paper_2507_01975_gb300 import inputs as I

    if args.only:
        torch.cuda.set_device(0)
        B.build()
        fd.load()
        fn = {"learned": lambda: learned_measurement(fd, I, steps=max(args.iters, 4)),
              "training": lambda: training_measurement(fd, I, iters=args.iters),
              "adjoint": lambda: adjoint_measurement(fd, I, iters=args.iters),
              "fine": lambda: fine_measurement(fd, I, steps=max(args.iters, 2)),
              "corr": lambda: corr_measurement(fd, I, iters=max(args.iters, 300)),
              "batch": lambda: batch_measurement(fd, I),
              "speed": lambda: speed_measurement(fd, I),
              "resweep": lambda: resweep_measurement(fd, I),
              "glearned": lambda: generic_learned_measurement(fd, I, steps=max(args.iters, 4))}[args.only]
        print(json.dumps(fn()), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    fd.load()

    cfg = fd.Config(n=N, batch=BATCH, dtype="f32", nu=NU, dt=DT)
    solver = fd.Solver(cfg)
    # launch plan: the library's autotuner times the cluster shapes and the
    # on-chip / streaming splits of this batch and keeps the fastest
    if args.plan:
        cl, on, stv = (int(x) for x in args.plan.split(","))
        solver.set_plan(cl, on, stv)
        candidates = []
    else:
        candidates = solver.autotune(probe_steps=32)
    plan = solver.plan()
    seed0 = rank * BATCH
    U0 = np.stack([I.decaying_ic(N, seed0 + b) for b in range(BATCH)]).astype(np.float32)
    u0 = torch.tensor(U0, device="cuda")
    out = torch.empty_like(u0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        solver.rollout(u0, out, args.time_steps)
    torch.cuda.synchronize()
    if not solver.check_finite(out):
        raise RuntimeError("rollout produced non-finite values")

    clock_lines, stop = [], threading.Event()
    th = threading.Thread(target=_sample_clocks, args=(stop, clock_lines), daemon=True)
    th.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        solver.rollout(u0, out, args.time_steps)
        ends[k].record(stream)
        launches += solver.last_launch_count()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    stop.set()
    th.join(timeout=5)
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(ms)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    units = N * N * BATCH * args.time_steps
    value = units * args.steps * world / (total_ms * 1e-3)
    clocks = _clock_summary(clock_lines, dev)

    # end to end through the host-buffer entry point: H2D copy, rollout, D2H copy
    hin = torch.tensor(U0).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    solver.rollout_host(hin, hout, args.time_steps)
    e2e_t = []
    for _ in range(max(3, min(args.steps, 5))):
        t0 = time.perf_counter()
        solver.rollout_host(hin, hout, args.time_steps)
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = units * world / (sum(e2e_t) / len(e2e_t))

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    avg_launch_s = statistics.mean(ms) * 1e-3
    # the dominant kernel is the on-chip rollout kernel; it processes the plan's
    # n_onchip trajectories, and the call (which also waits for the concurrent
    # streaming part) bounds its duration from above
    flops = FLOP_PER_CELL_STEP * N * N * plan["n_onchip"] * args.time_steps
    achieved = flops / avg_launch_s / 1e12
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    roofline = {
        "bound": "alu",
        "achieved": achieved,
        "peak": peak,
        "unit": "TFLOP/s",
        "frac": achieved / peak,
        # dram__bytes_read.sum + dram__bytes_write.sum of one launch of this kernel
        # (15 on-chip trajectories; ncu capture of the unchanged kernel): the state
        # is read once and written once per launch, whatever its number of steps
        "traffic": ONCHIP_DRAM_BYTES_PER_LAUNCH if plan["n_onchip"] == 15 else None,
        "traffic_unit": "bytes per launch",
        "traffic_note": "ncu dram read+write of one launch; the final state write drains after the kernel",
        "kernel": f"fv_rollout_kernel<float, 8, {plan['cluster']}, 512, 4> ({plan['n_onchip']} of {BATCH} "
                  f"trajectories; {plan['n_stream']} on the streaming kernels concurrently)",
        "peak_basis": "FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x median sampled SM clock",
        "achieved_all_trajectories": FLOP_PER_CELL_STEP * units / avg_launch_s / 1e12,
        "hbm_gbs": _peak("hbm_gbs")[0],
        "hbm_gbs_basis": _peak("hbm_gbs")[1],
    }
    cpu = None if args.no_cpu_baseline else cpu_baseline()
    learned = None if args.no_learned else learned_measurement(fd, I)
    training = None if args.no_training else training_measurement(fd, I)
    fine = None if args.no_fine else fine_measurement(fd, I)
    speed = None if args.no_speed else speed_measurement(fd, I)
    glearned = None if args.no_speed else generic_learned_measurement(fd, I)
    corr = None if args.no_corr else corr_measurement(fd, I)
    resweep = None if args.no_resweep else resweep_measurement(fd, I)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD,
            "grid": N,
            "batch_per_gpu": BATCH,
            "time_steps_per_bench_step": args.time_steps,
            "l2": "flushed (256 MB write) between timed bench steps; state resident on chip within a rollout",
            "parallelism": f"replicas x{world}",
            "plan": plan,
            "autotune_candidates": [{k: c[k] for k in ("cluster", "n_onchip", "n_stream", "resident", "us_per_step")}
                                    for c in candidates],
        },
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(U0.nbytes),
                "d2h_bytes_per_step": int(U0.nbytes)},
        "gpu_launches": launches,
        "clocks": clocks,
        "learned": learned,
        "training": training,
        "fine_grid": fine,
        "paper_speed_table": speed,
        "generic_learned": glearned,
        "wall_time_to_corr_095": corr,
        "re_generalisation": resweep,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
