"""Training data for the learned cost model: timings the planner generates.

For each network, the planner's candidate contraction orders
(:func:`tqc.plan_candidates`) are planned and timed on the GPU with CUDA
events; each timing is paired with the plan's features.  The model
(:class:`tqc.CostModel`) is then trained on the log of the measured over
the analytic seconds (a correction to the planner's own model) and used by
``Plan(..., planner=tqc.PLANNER_LEARNED, costmodel_path=...)`` to rank
candidates.  All device work goes through libtqc."""
from __future__ import annotations

import math

import numpy as np

from . import tqc


def time_plan(plan: "tqc.Plan", out, reps: int = 3, warmup: int = 1) -> float:
    """Median seconds of ``plan.contract(out)`` over ``reps`` runs."""
    import torch
    for _ in range(warmup):
        plan.contract(out)
    ts = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        plan.contract(out)
        e.record()
        e.synchronize()
        ts.append(s.elapsed_time(e) / 1e3)
    return float(np.median(ts))


def collect(handle: "tqc.Network", precision="auto", free_qubits=None, max_candidates: int = 10, reps: int = 3,
            mem_budget: int = 0, window: float = 10.0):
    """Time the candidate plans of one network.

    Returns a list of records ``{"order", "features", "seconds",
    "predicted_s", "flops"}`` (``predicted_s`` is the analytic model's
    estimate, the planner's own model).  ``mem_budget`` (device bytes, 0 =
    unlimited) slices every candidate as tqc_plan would.  Candidates whose
    analytic estimate exceeds ``window`` times the best one are not timed:
    the learned planner never ranks them either (see tqc_plan)."""
    import torch
    recs = []
    orders = tqc.plan_candidates(handle, max_candidates, precision=precision, free_qubits=free_qubits)
    n_out = 1 << (handle.n_qubits if free_qubits is None else len(free_qubits))
    out = torch.empty(n_out, dtype=torch.float32, device="cuda")
    plans = [tqc.Plan(handle, precision=precision, order=od, free_qubits=free_qubits, mem_budget=mem_budget)
             for od in orders]
    best = min(p.describe()["predicted_s"] for p in plans)
    for od, p in zip(orders, plans):
        d = p.describe()
        if d["predicted_s"] <= window * best:
            secs = time_plan(p, out, reps=reps)
            recs.append({"order": od, "features": p.features(), "seconds": secs, "predicted_s": d["predicted_s"],
                         "flops": d["flops"]})
        p.close()
    return recs


def dataset(records):
    """(features, targets): the target is log(measured / analytic seconds),
    the correction the network learns on top of the analytic model (with no
    data it predicts 0, i.e. the analytic estimate)."""
    X = np.stack([r["features"] for r in records]).astype(np.float32)
    y = np.array([math.log(max(r["seconds"], 1e-9)) - math.log(max(r["predicted_s"], 1e-12)) for r in records],
                 np.float32)
    return X, y


def predicted_log_seconds(model: "tqc.CostModel", records):
    """The learned estimate of log seconds for each record: analytic log
    time plus the network's correction (what the learned planner ranks)."""
    X, _ = dataset(records)
    return model.predict(X) + np.log([max(r["predicted_s"], 1e-12) for r in records])
