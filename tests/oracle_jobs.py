"""Oracle calls run in worker processes (spawn start method) by the GPU parity
tests at full batch sizes. Imports only numpy and the oracle, so a worker never
touches CUDA. Test infrastructure only."""

import numpy as np

import oracle as O
from oracle import adjoint as A


def step_vjp_job(args):
    """(U, problem, lam, model) -> oracle.adjoint.step_vjp(U, problem, lam, model)."""
    U, p, lam, model = args
    return A.step_vjp(U, p, lam, model)


def learned_step_job(args):
    """(U, problem, model) -> oracle.learned_step(U, problem, model)."""
    U, p, model = args
    return O.learned_step(U, p, model)


def run_pool(fn, jobs, max_procs=16):
    """Map ``fn`` over ``jobs`` in a spawn-started pool (safe after CUDA use)."""
    import multiprocessing as mp
    import os

    procs = max(1, min(max_procs, os.cpu_count() or 1, len(jobs)))
    if procs == 1:
        return [fn(j) for j in jobs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(fn, jobs, chunksize=1)


def rollout_vjp_job(args):
    """(U0, problem, n, lam_traj, model) -> (lam0, flat parameter gradient) of
    oracle.train.rollout_vjp_full."""
    from oracle import train as T

    U0, p, n, lam_traj, model = args
    lam0, g = T.rollout_vjp_full(U0, p, n, lam_traj, model)
    return lam0, (None if g is None else T.flat_grads(g, model))


def tc_vjp_job(args):
    """(U, hist, problem, model, gbar) -> oracle.adjoint.temporal_correction_vjp(...)."""
    U, hist, p, model, gbar = args
    return A.temporal_correction_vjp(U, hist, p, model, gbar)
