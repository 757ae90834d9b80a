#!/usr/bin/env python
"""Reconstruction throughput on one GB300 (or N, one process per GPU).

Workload: the 30-qubit grid shape -- 4 subcircuits of width 10, 10 cuts,
pseudo-physical FP64 tensors, every qubit free (the full 2^30 FP32
probability vector).  One step = one tqc_contract of the whole path (ingest,
the pairwise steps, renormalisation by the total mass Z) with the inputs
resident in HBM.  Z depends on the tensors only: the first contract after
they change computes it (an FP64 scalar network, under 0.2 ms) and later
ones reuse it, so the timed steps do not recompute it; the e2e leg uploads
the tensors every step and so recomputes Z every step.  Metric:
reconstructed probabilities per second, for the chosen form (tensor-core
steps, FP32 accumulate) and, beside it, the plain FP32 CUDA-core form.

At one GPU the same JSON line also carries two sub-records, each with its
own CUDA-event timing, roofline, clock samples and sampled oracle error:
``tensor_bound`` (one 2^24-state bin of the 48-qubit QAOA network per step,
tensor-core bound) and ``batched`` (256 independent networks in one
persistent launch replayed from a CUDA graph, against sequential calls).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload qaoa48|grid64   (tensor-bound bins, one JSON line)
  python bench.py --batch 256                 (the batched launch, one JSON line)
  python bench.py --hss | --planner-eval      (heavy state selection; learned planner)
  python bench.py --smallk all                (small-K CUDA-core steps, both tile forms)

Under torchrun each rank reconstructs its own network instance (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
`--impl reference` times the CPU FP64 oracle on the host cores instead."""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reconstructed probs/s & % of roofline, chosen vs plain FP32 form at <=1e-5 err"
PLAN_FIELDS = ["log2_m", "log2_n", "log2_k", "class", "tile", "ksplit", "kblk"]
UNIT = "probs/s"
WORKLOAD = "grid30: 30 qubits, 4 subcircuits of width 10, 10 cuts, full 2^30 output"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--free-qubits", type=int, default=30,
                    help="reconstruct the bin of the lowest N qubits (others fixed to 0); 30 = full output")
    ap.add_argument("--no-clocks", action="store_true", help="skip the clock sampler and its load loop")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead: time the batched persistent launch over this many networks")
    ap.add_argument("--batch-n-lo", type=int, default=16)
    ap.add_argument("--batch-n-hi", type=int, default=28)
    ap.add_argument("--workload", default="grid30", choices=["grid30", "qaoa48", "grid64"],
                    help="qaoa48 / grid64: time one bin of 2^24 states of the tensor-bound networks instead")
    ap.add_argument("--mem-budget-gb", type=float, default=32.0,
                    help="device memory budget of the qaoa48 / grid64 plans (forces slicing)")
    ap.add_argument("--hss", action="store_true",
                    help="instead: heavy state selection on GHZ / W / Regular / Supremacy circuits (n = 20)")
    ap.add_argument("--hss-states", type=int, default=256)
    ap.add_argument("--planner-eval", action="store_true",
                    help="instead: learned vs greedy vs exhaustive planner on 48-qubit QAOA bins")
    ap.add_argument("--pe-train", type=int, default=40)
    ap.add_argument("--pe-test", type=int, default=12)
    ap.add_argument("--pe-candidates", type=int, default=6)
    ap.add_argument("--states", type=int, default=0,
                    help="instead: time tqc_contract_states on this many grid30 states")
    ap.add_argument("--cuts", action="store_true", help="instead: the cut finder on the 48-qubit QAOA circuit")
    ap.add_argument("--smallk", default="",
                    help="instead: one small-K CUDA-core final step (a gen.workloads.SMALLK_CASES name, or all), "
                         "the small-K tile against the general tiles")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the tensor_bound and batched sub-records of the default line")
    ap.add_argument("--sub-steps", type=int, default=5, help="timed steps of each sub-record")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p["bf16_tflops"], p.get("bf16_tflops_sustained"), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "reasons": reasons}


def step_dtypes(desc):
    """The operand types the plan's steps compute in, e.g. "bf16x3+tf32"."""
    return "+".join(sorted({s_["prec"] for s_ in desc["steps"]})) or "f64"


def step_bytes(st, out_bytes):
    """Algorithmic HBM bytes of one pairwise step: operands read once, the
    result written once."""
    m, n, k = 2 ** st["log2_m"], 2 ** st["log2_n"], 2 ** st["log2_k"]
    ein = {"bf16": 2, "bf16x3": 4, "tf32": 4}.get(st["prec"], 4) if st["class"] == "tcgen05" else 4
    return ein * (m * k + n * k) + out_bytes * m * n


def step_flops(st):
    m, n, k = 2 ** st["log2_m"], 2 ** st["log2_n"], 2 ** st["log2_k"]
    mult = 3 if (st["class"] == "tcgen05" and st["prec"] == "bf16x3") else 1
    return 2.0 * m * n * k * mult


def traffic_record(kernel):
    """dram read+write bytes per launch from the committed ncu summary, or
    None when the kernel's sources (its .cu file and the shared epilogue
    header) changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.md")
    csrc = os.path.join(ROOT, "paper_2502_03445_gb300", "csrc")
    srcs = [os.path.join(csrc, "umma.cu" if kernel.startswith("umma") else "simt.cu"),
            os.path.join(csrc, "device_common.cuh"), os.path.join(csrc, "tc_ptx.cuh")]
    try:
        rec = {}
        with open(path) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    rec[k.strip()] = v.strip()
        h = hashlib.sha256(b"".join(open(f, "rb").read() for f in srcs)).hexdigest()[:16]
        if rec.get("source_sha256_16") != h:
            return None
        return float(rec["dram_bytes_per_full_launch"])
    except Exception:
        return None


def cpu_oracle_sample(net, target_s=12.0, seed=7, n_free=None):
    """Oracle A on uniformly drawn entries of the bin of the lowest n_free
    qubits (other qubits 0), so entry index = state index."""
    import oracle
    rng = np.random.Generator(np.random.PCG64(seed))
    n = net.n_qubits if n_free is None else n_free
    calib = [int(x) for x in rng.integers(0, 1 << n, size=16, dtype=np.int64)]
    _, t = oracle.timed_sample(net, calib)
    per = max(t / len(calib), 1e-6)
    cnt = int(min(max(target_s / per, 16), 1 << 16))
    states = [int(x) for x in rng.integers(0, 1 << n, size=cnt, dtype=np.int64)]
    p, t = oracle.timed_sample(net, states)
    return {"value": len(states) / t, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{len(states)} uniformly drawn states of the grid30 network, oracle A "
                      f"(4^10 cut assignments x 4 subcircuits per state), {t:.1f} s"}, states, p


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    from gen import workloads
    net = workloads.grid30(0)
    rng = np.random.Generator(np.random.PCG64(11))
    per_step = 512
    n = net.n_qubits
    for _ in range(args.warmup):
        oracle.recon_states(net, [int(x) for x in rng.integers(0, 1 << n, size=32, dtype=np.int64)])
    times = []
    for _ in range(args.steps):
        st = [int(x) for x in rng.integers(0, 1 << n, size=per_step, dtype=np.int64)]
        t0 = time.perf_counter()
        oracle.recon_states(net, st)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = per_step * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "step": f"{per_step} sampled states"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"{per_step} random states per step, oracle A (FP64 brute force over "
                                       f"4^10 cut assignments)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def leaf_bytes(desc, m, src_bytes):
    """Algorithmic bytes of a plan's ingest: every leaf operand element read
    once from the node tensor and written once as a 4-byte operand."""
    tot = 0
    for lay in desc["layouts"][:m]:
        bits = sum(2 if x.startswith("c") else 1 for x in lay)
        tot += (src_bytes + 4) * (1 << bits)
    return tot


def measure_batched(args, count=256, steps=None, warmup=None):
    """Batched persistent launch: ``count`` independent networks of uneven
    sizes (n 16-28, 2-8 subcircuits, 2-12 cuts, full 2^n outputs each), with
    tile configurations from the autotuner, reconstructed by one
    tqc_contract_batch call (the persistent kernel runs every small step;
    steps predicted to take 16 us or more follow as their own launches)
    replayed from a CUDA graph, against contracting them one after the
    other.  Raw probabilities
    (the Gaussian FP32 test tensors can have a total mass near zero)."""
    import torch
    import oracle
    from gen import Network as GNet, Node as GNode, workloads
    from paper_2502_03445_gb300 import tqc
    steps = steps or args.steps
    warmup = max(3, warmup or args.warmup)
    nets, redraws = workloads.batch_recipe(count, args.batch_n_lo, args.batch_n_hi)
    hs, plans, outs = [], [], []
    for net in nets:
        h = tqc.Network(net, dtype=tqc.F32)
        # tile configurations from the autotuner (its choices are cached by step shape)
        p = tqc.Plan(h, precision=args.precision, flags=tqc.FLAG_NO_RENORM, autotune=1)
        o = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
        p.contract(o)
        hs.append(h)
        plans.append(p)
        outs.append(o)
    units = sum(o.numel() for o in outs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        tqc.contract_batch(plans, outs, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        tqc.contract_batch(plans, outs, stream=s)
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if not args.no_clocks else None
    t_end = time.time() + (0.0 if args.no_clocks else 0.6)
    while time.time() < t_end:
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    tqc.batch_status()
    ms = e0.elapsed_time(e1) / steps
    # the same work as separate tqc_contract calls
    for _ in range(2):
        for p, o in zip(plans, outs):
            p.contract(o)
    torch.cuda.synchronize()
    n_seq = max(2, steps // 2)
    e0.record()
    for _ in range(n_seq):
        for p, o in zip(plans, outs):
            p.contract(o)
    e1.record()
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1) / n_seq
    g.replay()
    torch.cuda.synchronize()
    tqc.batch_status()
    launches, tail_steps = tqc.batch_launches()
    classes, alg_bytes = {}, 0
    descs = [p.describe() for p in plans]
    for net, d in zip(nets, descs):
        for i, st in enumerate(d["steps"]):
            classes[st["class"]] = classes.get(st["class"], 0) + 1
            alg_bytes += step_bytes(st, 4)
        alg_bytes += leaf_bytes(d, len(net.nodes), 4) if d["steps"] else 8 * (1 << net.n_qubits)
    hbm = peaks()[0]
    achieved = alg_bytes / (ms / 1e3) / 1e9
    # sampled check: two states of every fourth network against oracle A,
    # against the bound of the plan's arithmetic (n_steps 2^-12 of the mean
    # absolute term mass per state)
    rng = np.random.Generator(np.random.PCG64(21))
    worst, max_abs, n_chk = 0.0, 0.0, 0
    for k in range(0, len(nets), 4):
        net, p, o = nets[k], plans[k], outs[k]
        idx = sorted(set(int(i) for i in rng.integers(0, 1 << net.n_qubits, size=2)))
        want = oracle.recon_states(net, idx)
        got = o[torch.tensor(idx, device="cuda")].double().cpu().numpy()
        a = GNet(net.n_qubits, net.n_cuts,
                 [GNode(nd.out_qubits, nd.cut_ids, nd.cut_role, np.abs(nd.data)) for nd in net.nodes])
        scale = oracle.total_mass(a) / float(1 << net.n_qubits)
        n_steps = max(len(descs[k]["steps"]), 1)
        err = float(np.abs(got - want).max())
        worst = max(worst, err / (n_steps * 2.0 ** -12 * scale))
        max_abs = max(max_abs, err)
        n_chk += len(idx)
    for p in plans:
        p.close()
    for h in hs:
        h.close()
    del outs, g
    torch.cuda.empty_cache()
    return {"workload": f"batch: {len(nets)} networks, n ~ U{{{args.batch_n_lo}..{args.batch_n_hi}}}, "
                        f"m ~ U{{2..8}}, |E| ~ U{{max(2,m-1)..12}}, full 2^n outputs (raw, FP32 Gaussian "
                        f"tensors), one persistent kernel (small steps) plus the large steps' own "
                        f"launches, replayed from a CUDA graph",
            "value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "outputs": units, "redraws": redraws, "step_classes": classes, "gpu_launches": steps * launches,
            "steps_after_persistent_kernel": tail_steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None,
                         "kernel": "the batched launch (persistent kernel and large steps)",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "peak_kind": f"{peaks()[3]} copy bandwidth"},
            "clocks": clocks,
            "sequential_contracts": {"ms_per_step": ms_seq, "value": units / (ms_seq / 1e3),
                                     "speedup_of_batched": ms_seq / ms},
            "error_vs_oracle": {"states": n_chk, "oracle": "A", "max_abs": max_abs,
                                "max_err_over_bound": worst,
                                "bound": "n_steps * 2^-12 * mean |term| mass per state"}}


def run_batch(args):
    import torch
    torch.cuda.set_device(0)
    r = measure_batched(args, count=args.batch)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["steps"],
            "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic (Gaussian tensors)",
            "config": {"workload": r["workload"], "outputs": r["outputs"], "redraws": r["redraws"],
                       "step_classes": r["step_classes"],
                       "steps_after_persistent_kernel": r["steps_after_persistent_kernel"]},
            "roofline": r["roofline"], "clocks": r["clocks"], "gpu_launches": r["gpu_launches"],
            "sequential_contracts": r["sequential_contracts"], "error_vs_oracle": r["error_vs_oracle"]}
    print(json.dumps(line), flush=True)
    return 0


def fp32_alu_peak():
    """FP32 CUDA-core peak of the part in TFLOP/s: 152 SMs x 128 FP32 lanes x
    2 flop per FMA x the maximum SM clock (2070 MHz) = 80.5."""
    return 152 * 128 * 2 * 2.070e9 / 1e12


def measure_states(args, count=1_000_000, steps=None, warmup=None):
    """Arbitrary state lists (§VII-C reconstructs one million arbitrary
    states): ``count`` uniformly drawn states of the grid30 network through
    tqc_contract_states (the fused single-state kernel), device-timed, the
    list's host-to-device copy included in each call."""
    import torch
    import oracle
    from gen import workloads
    from paper_2502_03445_gb300 import tqc
    steps = steps or args.steps
    warmup = max(3, warmup or args.warmup)
    net = workloads.grid30(0)
    h = tqc.Network(net)
    p = tqc.Plan(h, free_qubits=[])
    d = p.describe()
    st = np.random.Generator(np.random.PCG64(17)).integers(0, 1 << net.n_qubits, size=count, dtype=np.uint64)
    out = torch.empty(count, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        p.contract_states(st, out)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if not args.no_clocks else None
    t_end = time.time() + (0.0 if args.no_clocks else 0.6)
    while time.time() < t_end:
        p.contract_states(st, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        p.contract_states(st, out)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1) / steps
    macs = sum(2 ** (s_["log2_m"] + s_["log2_n"] + s_["log2_k"]) for s_ in d["steps"])
    achieved = 2.0 * macs * count / (ms / 1e3) / 1e12
    pk = fp32_alu_peak()
    k = 2048
    z = oracle.total_mass(net)
    want = oracle.recon_states(net, st[:k]) / z
    err = np.abs(out[:k].double().cpu().numpy() - want)
    p.close()
    h.close()
    del out
    torch.cuda.empty_cache()
    return {"workload": f"grid30: {count} uniformly drawn states of 2^30, one tqc_contract_states call per step "
                        f"(the list's 8-byte states copied host to device inside the call)",
            "value": count / (ms / 1e3), "unit": "states/s", "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "form": d["states_form"], "macs_per_state": macs,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                         "traffic": None, "kernel": "states_kernel",
                         "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                         "algorithmic_flops_per_launch": 2.0 * macs * count},
            "clocks": clocks, "gpu_launches": steps,
            "error_vs_oracle": {"states": k, "oracle": "A", "max_abs": float(err.max()),
                                "max_abs_rel_to_max_p": float(err.max() / np.abs(want).max())}}


def measure_bin_stream(args, n_bins=16):
    """Reuse of intermediates across bins: grid30 bins of 2^26 states whose
    four fixed qubits all belong to the subcircuit that enters the last
    step, so consecutive bins differ only in that subcircuit's fixed bits;
    ms per bin with TQC_FLAG_REUSE and without it."""
    import torch
    from gen import workloads
    from paper_2502_03445_gb300 import tqc
    net = workloads.grid30(0)
    h = tqc.Network(net)
    probe = tqc.Plan(h)
    last = probe.describe()["steps"][-1]
    m = len(net.nodes)
    leaf = last["b"] if last["b"] < m else last["a"]
    probe.close()
    if leaf >= m:
        h.close()
        return {"skipped": "the last step joins two intermediates"}
    fixed_q = net.nodes[leaf].out_qubits[:4]
    free = [q for q in range(net.n_qubits) if q not in fixed_q]
    res = {}
    for name, flags in (("reuse", tqc.FLAG_REUSE), ("no_reuse", 0)):
        p = tqc.Plan(h, free_qubits=free, flags=flags)
        out = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
        fbs = []
        for b in range(n_bins):
            fb = np.zeros(net.n_qubits, np.uint8)
            fb[fixed_q] = [(b >> i) & 1 for i in range(4)]
            fbs.append(fb)
        for fb in fbs[:3]:
            p.contract(out, fixed_bits=fb)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for fb in fbs:
            p.contract(out, fixed_bits=fb)
        e1.record()
        torch.cuda.synchronize()
        d = p.describe()
        res[name] = {"ms_per_bin": e0.elapsed_time(e1) / n_bins, "reused_leaves": d["reused_leaves"],
                     "reused_steps": d["reused_steps"]}
        p.close()
        del out
    h.close()
    torch.cuda.empty_cache()
    res["workload"] = (f"grid30: {n_bins} bins of 2^26 states; fixed qubits {fixed_q} all in subcircuit {leaf}, "
                       f"which enters the last step")
    res["speedup_of_reuse"] = res["no_reuse"]["ms_per_bin"] / res["reuse"]["ms_per_bin"]
    return res


def measure_learned_planner(args, n_train=16, n_small=12, n_test=8):
    """The learned planner against the planners without it: the MLP cost
    model (3 x 128, the library's own GPU kernels) is trained on the
    planner's timings of the candidate plans of 28-30-qubit networks (4-6
    subcircuits) and smaller ones; on held-out 28-30-qubit networks the plans
    chosen by the learned planner, the analytic ranking of the same
    candidates, TQC_PLANNER_AUTO and the greedy planner are timed against the
    fastest candidate (geometric means)."""
    import math
    import torch
    from gen import workloads
    from paper_2502_03445_gb300 import costmodel, tqc
    t0 = time.perf_counter()
    train, test = [], []
    for kind, seed in [("g30", 9800 + i) for i in range(n_train + n_test)] + \
                      [("small", 9000 + i) for i in range(n_small)]:
        net = workloads.planner_network(seed, kind)
        h = tqc.Network(net, dtype=tqc.F32)
        recs = costmodel.collect(h, precision=args.precision, max_candidates=8, reps=5)
        (test.append((net, recs)) if kind == "g30" and seed >= 9800 + n_train else train.extend(recs))
        h.close()
    X, y = costmodel.dataset(train)
    cm = tqc.CostModel(X.shape[1], seed=0)
    t1 = time.perf_counter()
    cm.train(X, y, epochs=400, batch=32, lr=1e-3, seed=1)
    t_train = time.perf_counter() - t1
    path = os.path.join(tempfile.mkdtemp(), "costmodel.bin")
    cm.save(path)
    ratios = {"learned": [], "analytic_ranking": [], "auto": [], "greedy": []}
    err = {"mlp": [], "analytic": []}
    for net, recs in test:
        meas = np.array([r["seconds"] for r in recs])
        best = meas.min()
        ana = np.log([r["predicted_s"] for r in recs])
        pred = costmodel.predicted_log_seconds(cm, recs)
        err["mlp"].append(float(np.mean(np.abs(pred - np.log(meas)))))
        err["analytic"].append(float(np.mean(np.abs(ana - np.log(meas)))))
        ratios["analytic_ranking"].append(meas[int(np.argmin(ana))] / best)
        h = tqc.Network(net, dtype=tqc.F32)
        out = torch.empty(1 << net.n_qubits, dtype=torch.float32, device="cuda")
        for name, pl in (("learned", tqc.PLANNER_LEARNED), ("auto", tqc.PLANNER_AUTO), ("greedy", tqc.PLANNER_GREEDY)):
            p = tqc.Plan(h, precision=args.precision, planner=pl,
                         costmodel_path=path if pl == tqc.PLANNER_LEARNED else None)
            ratios[name].append(costmodel.time_plan(p, out, reps=5) / best)
            p.close()
        del out
        h.close()
    cm.close()
    torch.cuda.empty_cache()
    gm = {k: float(math.exp(np.mean(np.log(v)))) for k, v in ratios.items()}
    return {"workload": f"held-out networks: {n_test} of 27-30 qubits, 4-6 subcircuits (Gaussian values, timing "
                        f"only); trained on {n_train} such and {n_small} of 20-24 qubits",
            "plan_time_over_best_candidate": gm, "learned_speedup_over_auto": gm["auto"] / gm["learned"],
            "learned_speedup_over_analytic_ranking": gm["analytic_ranking"] / gm["learned"],
            "held_out_mean_abs_log_error": {k: float(np.mean(v)) for k, v in err.items()},
            "train_records": len(train), "collect_and_eval_s": time.perf_counter() - t0, "train_s": t_train,
            "model": "MLP 32-128-128-128-1 (ReLU), MSE on log(measured / analytic seconds), own GPU kernels"}


def measure_cut_finder():
    """The cut finder (§VI, Alg. 2/3) on the 48-qubit QAOA p=1 circuit:
    subcircuits of at most 16 qubits and half the circuit's two-qubit gates,
    K_t swept 1..16, T_QPU by Eq. qpu_runtime (10 QPUs), T_classical the
    planner's estimate for a 2^20-state bin."""
    from gen import circuits
    from paper_2502_03445_gb300 import tqc
    n, gates = circuits.qaoa_regular(48, 4000)
    gq = [tuple(qs) for _, qs, _ in gates]
    n2q = sum(1 for q in gq if len(q) == 2)
    t0 = time.perf_counter()
    part, r = tqc.find_cuts(n, gq, w_max=16, s_max=max(1, n2q // 2), k_t=0, k_sweep_max=16, cost_free_qubits=20)
    r["find_s"] = time.perf_counter() - t0
    r["circuit"] = f"QAOA p=1, random 3-regular graph, n = {n}, {n2q} two-qubit gates"
    r["cost_ratio_cutqc_over_tensorqc"] = r["cutqc_mults"] / r["tensorqc_mults"] if r["tensorqc_mults"] else None
    return r


def tensor_peak(prec, bf16):
    """(peak in algorithmic TFLOP/s, how it is derived) of a tensor-core step."""
    if prec == "bf16x3":
        return bf16 / 3.0, "measured bf16 burst / 3 (split BF16 issues three MMAs per product)"
    if prec == "tf32":
        return bf16 * 1.1 / 2.25, "measured bf16 burst x 1.1/2.25 (nominal TF32/BF16 ratio)"
    return bf16, "measured bf16 burst"


def path_roofline(steps, n_slices, hbm, bf16):
    """Roofline time of the whole plan in ms: for every step the larger of
    its algorithmic bytes over HBM bandwidth and its algorithmic flops over
    the tensor peak of its precision (CUDA-core steps: bytes only), summed
    over the steps and repeated per slice.  Intermediates count 4 bytes per
    element; the final step writes FP32 once, or reads and writes the FP64
    accumulator once per slice when the plan is sliced."""
    t = 0.0
    for i, st in enumerate(steps):
        if st.get("fuse") == 2:      # counted with the step before it
            continue
        last = i == len(steps) - 1
        tb = step_bytes(st, (16 if n_slices > 1 else 4) if last else 4) / (hbm * 1e9)
        tf = 0.0
        if st["class"] == "tcgen05":
            pk, _ = tensor_peak(st["prec"], bf16)
            tf = 2.0 * 2 ** (st["log2_m"] + st["log2_n"] + st["log2_k"]) / (pk * 1e12)
        if st.get("fuse") == 1:      # a fused pair: the intermediate is neither written nor read
            nx = steps[i + 1]
            m, n, k = 2 ** nx["log2_m"], 2 ** nx["log2_n"], 2 ** nx["log2_k"]
            tb = (step_bytes(st, 0) + 4 * n * k + 4 * m * n) / (hbm * 1e9)
            pk, _ = tensor_peak(nx["prec"], bf16)
            tf += 2.0 * m * n * k / (pk * 1e12)
        t += max(tb, tf)
    return t * n_slices * 1e3


def measure_tensor_bound(args, workload="qaoa48", steps=None, warmup=None):
    """One 2^24-state bin of the 48-qubit QAOA network (or of the 64-qubit
    grid shape) per step, sliced to the memory budget: these plans end in
    tensor-bound steps (K = 4^7..4^9 after slicing), so the roofline is the
    tensor pipe of the dominant step, quoted against the peak of its own
    precision and against the raw measured BF16 burst."""
    import torch
    from gen import workloads
    from paper_2502_03445_gb300 import tqc
    import oracle
    steps = steps or args.steps
    warmup = max(3, warmup or args.warmup)
    net = workloads.qaoa48(0) if workload == "qaoa48" else workloads.grid64_bin(0, 0)
    spec = ("gen.workloads", "qaoa48", (0,)) if workload == "qaoa48" else ("gen.workloads", "grid64_bin", (0, 0))
    h = tqc.Network(net)
    plan = tqc.Plan(h, precision=args.precision, mem_budget=int(args.mem_budget_gb * (1 << 30)))
    out = torch.empty(plan.out_elems, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        plan.contract(out)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if not args.no_clocks else None
    t_end = time.time() + (0.0 if args.no_clocks else 0.6)
    while time.time() < t_end:
        plan.contract(out)
    torch.cuda.synchronize()
    ms = time_plan(torch, plan, out, steps, 0, profile=True)
    clocks = sampler.stop() if sampler else None
    desc = plan.describe()
    info = plan.info()
    step_ms = [plan.step_time(i)[0] for i in range(len(desc["steps"]))]
    plan.profile(False)
    top = int(np.argmax(step_ms))
    st = desc["steps"][top]
    alg = 2.0 * 2 ** (st["log2_m"] + st["log2_n"] + st["log2_k"])
    hbm, bf16, bf16_sus, peak_kind = peaks()
    pk, how = tensor_peak(st["prec"], bf16)
    achieved = alg / (step_ms[top] / 1e3) / 1e12
    roof = {"bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
            "traffic": None, "peak_kind": f"{peak_kind}: {how}",
            "kernel": f"umma_step (step {top}: log2 M,N,K = {st['log2_m']},{st['log2_n']},{st['log2_k']}, "
                      f"{st['prec']}, tile {st['tile']}, ksplit {st['ksplit']})",
            "algorithmic_flops_per_launch": alg, "mean_launch_ms": step_ms[top], "step_ms": step_ms,
            "frac_of_bf16_burst": achieved / bf16,
            "tensor_pipe_issue_frac_of_bf16": achieved * (3 if st["prec"] == "bf16x3" else 1) / bf16}
    if bf16_sus:
        roof["frac_of_bf16_sustained"] = achieved / bf16_sus
    roof["path_roofline_ms"] = path_roofline(desc["steps"], info["n_slices"], hbm, bf16)
    roof["path_frac"] = roof["path_roofline_ms"] / ms
    got = out.double().cpu().numpy()
    # sampled check: a sub-bin of 2^8 states by oracle C, and four uniformly
    # drawn states by oracle B
    z = oracle.total_mass(net)
    rng = np.random.Generator(np.random.PCG64(5))
    sub_free = sorted(int(q) for q in rng.choice(net.n_qubits, size=8, replace=False))
    fixed = rng.integers(0, 2, size=net.n_qubits).astype(np.uint8)
    idx_c = np.array(oracle.bin_states(net.n_qubits, sub_free, fixed, np.arange(256)), dtype=np.int64)
    t0 = time.perf_counter()
    want_c = oracle.recon_bin_pairwise(net, sub_free, fixed) / z
    t_c = time.perf_counter() - t0
    idx_b = [int(x) for x in rng.integers(0, 1 << net.n_qubits, size=4)]
    t0 = time.perf_counter()
    want_b = oracle.recon_states_elim(net, idx_b) / z
    t_b = time.perf_counter() - t0
    want = np.concatenate([want_c, want_b])
    err = np.abs(got[np.concatenate([idx_c, np.array(idx_b, dtype=np.int64)])] - want)
    plan.close()
    h.close()
    del out
    torch.cuda.empty_cache()
    return {"workload": f"{workload}: bin of 2^24 states, {net.n_cuts} cuts, {len(net.nodes)} subcircuits, "
                        f"node tensors drawn bin-restricted",
            "value": (1 << net.n_qubits) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "dtype": step_dtypes(desc),
            "slices": info["n_slices"], "sliced": desc["sliced"],
            "plan": [[s_["log2_m"], s_["log2_n"], s_["log2_k"], s_["class"], s_["prec"], s_["tile"],
                      s_["ksplit"], s_["kblk"]] for s_ in desc["steps"]],
            "plan_fields": PLAN_FIELDS[:4] + ["prec"] + PLAN_FIELDS[4:],
            "flops_per_step": info["flops"], "tflops_per_step": info["flops"] / (ms / 1e3) / 1e12,
            "mem_budget_gb": args.mem_budget_gb,
            "roofline": roof, "clocks": clocks, "gpu_launches": desc["launches_per_contract"] * steps,
            "error_vs_oracle": {"states": int(len(want)), "max_abs": float(err.max()),
                                "tv_over_checked": float(0.5 * err.sum() / np.abs(want).sum()),
                                "sample": "a 2^8-state sub-bin (oracle C) and 4 uniformly drawn states (oracle B)"},
            "cpu_baseline": {"value": (256 + len(idx_b)) / (t_c + t_b), "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"256 states of a sub-bin by oracle C ({t_c:.1f} s) and {len(idx_b)} states "
                                       f"by oracle B ({t_b:.1f} s), numpy FP64, BLAS threads up to the host's cores"},
            "_spec": spec}


def run_workload(args):
    import torch
    torch.cuda.set_device(0)
    r = measure_tensor_bound(args, args.workload)
    r.pop("_spec")
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["steps"],
            "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": r["dtype"], "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "slices", "sliced", "plan", "plan_fields", "flops_per_step",
                                         "mem_budget_gb")},
            "tflops_per_step": r["tflops_per_step"], "roofline": r["roofline"], "clocks": r["clocks"],
            "gpu_launches": r["gpu_launches"], "error_vs_oracle": r["error_vs_oracle"],
            "cpu_baseline": r["cpu_baseline"]}
    print(json.dumps(line), flush=True)
    return 0


def run_hss(args):
    """Heavy state selection (§IV) on the circuit families of §VII (n = 20,
    3 subcircuits, exact tensors): device norms and selection, the selected
    network gathered on the device, then the ordinary contraction of the
    product states.  Reports the paper's metrics (P_HSS, r_{P,HSS},
    r_|HSS|, eta_HSS) against the uncut circuit's statevector."""
    import torch
    from gen import statevector as sv, workloads
    from paper_2502_03445_gb300 import tqc
    torch.cuda.set_device(0)
    rows = {}
    for fam in workloads.HSS_FAMILIES:
        net, (n, gates) = workloads.hss_circuit(fam, 20)
        psi = sv.simulate(n, gates)
        p_true = np.abs(psi) ** 2
        h = tqc.Network(net)
        zp = tqc.Plan(h, free_qubits=[])               # total mass of the full network
        z = zp.contract(torch.empty(1, dtype=torch.float64, device="cuda"), want_z=True)
        zp.close()
        times = []
        for rep in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sel, n_states = h.hss_select(args.hss_states)
            sub = h.select(sel)
            plan = tqc.Plan(sub, precision=args.precision, flags=tqc.FLAG_NO_RENORM)
            out = torch.empty(plan.out_elems, dtype=torch.float64, device="cuda")
            plan.contract(out)
            p_hss = float(out.sum().item()) / z
            t = time.perf_counter() - t0
            if rep >= args.warmup:
                times.append(t)
            plan.close()
            sub.close()
        h.close()
        top = np.sort(p_true)[::-1][:n_states]
        r_size = n_states / float(1 << n)
        rows[fam] = {"cuts": net.n_cuts, "n_states": n_states, "selected_per_subcircuit": [len(x) for x in sel],
                     "P_HSS": p_hss, "P_HSS_max": float(top.sum()), "r_P_HSS": p_hss / float(top.sum()),
                     "r_size": r_size, "eta_HSS": p_hss / r_size, "ms": 1e3 * float(np.median(times))}
    ms = sum(r["ms"] for r in rows.values())
    line = {"metric": "heavy-state reconstruction: selected states per second (norms, selection, gather, contract)",
            "value": sum(r["n_states"] for r in rows.values()) / (ms / 1e3), "unit": "states/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": args.precision, "data": "synthetic (seeded circuits, exact subcircuit tensors)",
            "config": {"workload": f"GHZ / W / Regular / Supremacy, n = 20, 3 subcircuits, s_max = {args.hss_states}"},
            "families": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_planner_eval(args):
    """The learned planner on its configuration: 48-qubit QAOA p=1 bins of
    2^24 states (16-24 cuts, subcircuits <= 16 qubits, sliced to the memory
    budget).  The MLP cost model (3 x 128) is trained on the GPU on the
    planner's own timings of every candidate plan of the training instances;
    on held-out instances the plans chosen by the greedy, exhaustive (DP on
    the analytic model) and learned planners are timed against the fastest
    candidate."""
    import math
    import torch
    from gen import workloads
    from paper_2502_03445_gb300 import costmodel, tqc
    torch.cuda.set_device(0)
    budget = int(args.mem_budget_gb * (1 << 30))
    t0 = time.perf_counter()
    train, test, skipped = [], [], []
    k = 0
    while len(test) < args.pe_test:
        try:
            net = workloads.qaoa48_timing(k)
        except RuntimeError:      # no 16-24 cut partition within the width cap
            skipped.append(k)
            k += 1
            continue
        h = tqc.Network(net, dtype=tqc.F32)
        recs = costmodel.collect(h, precision=args.precision, max_candidates=args.pe_candidates, reps=2,
                                 mem_budget=budget)
        if k - len(skipped) < args.pe_train:
            train.extend(recs)
        else:
            test.append((k, recs))
        h.close()
        k += 1
    t_collect = time.perf_counter() - t0
    X, y = costmodel.dataset(train)
    cm = tqc.CostModel(X.shape[1], seed=0)
    t1 = time.perf_counter()
    cm.train(X, y, epochs=400, batch=32, lr=1e-3, seed=1)
    t_train = time.perf_counter() - t1
    path = os.path.join(tempfile.mkdtemp(), "costmodel.bin")
    cm.save(path)
    out = torch.empty(1 << 24, dtype=torch.float32, device="cuda")
    ratios = {"greedy": [], "exhaustive": [], "learned": []}
    err_mlp, err_ana = [], []
    for k, recs in test:
        yt = np.log([r["seconds"] for r in recs])
        pred = costmodel.predicted_log_seconds(cm, recs)
        err_mlp.append(float(np.mean(np.abs(pred - yt))))
        err_ana.append(float(np.mean(np.abs(np.log([r["predicted_s"] for r in recs]) - yt))))
        best = min(r["seconds"] for r in recs)
        h = tqc.Network(workloads.qaoa48_timing(k), dtype=tqc.F32)
        for name, pl in (("greedy", tqc.PLANNER_GREEDY), ("exhaustive", tqc.PLANNER_EXHAUSTIVE),
                         ("learned", tqc.PLANNER_LEARNED)):
            p = tqc.Plan(h, precision=args.precision, planner=pl, mem_budget=budget,
                         costmodel_path=path if pl == tqc.PLANNER_LEARNED else None)
            assert pl != tqc.PLANNER_LEARNED or p.describe()["planner"] == "learned"
            secs = costmodel.time_plan(p, out, reps=2)
            ratios[name].append(secs / best)
            p.close()
        h.close()
    cm.close()
    gm = {k: float(math.exp(np.mean(np.log(v)))) for k, v in ratios.items()}
    line = {"metric": "plan time / fastest candidate (geometric mean over held-out instances)",
            "value": gm["learned"], "unit": "ratio", "n_gpus": 1, "higher_is_better": False,
            "data": "synthetic (QAOA-48 shapes, Gaussian values: timing only)",
            "config": {"workload": "48-qubit QAOA p=1 on 3-regular graphs, 5-6 subcircuits <= 16 qubits, "
                                   "16-24 cuts, bin of 2^24 states", "train_instances": args.pe_train,
                       "test_instances": args.pe_test, "candidates_per_instance": args.pe_candidates,
                       "mem_budget_gb": args.mem_budget_gb, "precision": args.precision,
                       "model": "MLP 32-128-128-128-1 (ReLU), MSE on log(measured / analytic seconds), own GPU kernels"},
            "planner_time_over_best": gm,
            "learned_vs_greedy_speedup": gm["greedy"] / gm["learned"],
            "held_out_mean_abs_log_error": {"mlp": float(np.mean(err_mlp)), "analytic": float(np.mean(err_ana))},
            "train_records": len(train), "skipped_instances": skipped, "collect_s": t_collect,
            "train_s": t_train}
    print(json.dumps(line), flush=True)
    return 0


def time_plan(torch, plan, out, steps, warmup, profile=False):
    for _ in range(warmup):
        plan.contract(out)
    torch.cuda.synchronize()
    if profile:
        plan.profile(True)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(steps):
        plan.contract(out)
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / steps


def measure_smallk(args, case):
    """One small-K final step (two subcircuits sharing one or two cut edges,
    2^27-2^28 FP32 results): the step's CUDA-event time with the small-K tile
    and with the general tiles (TQC_FLAG_NO_SMALLK), against the measured copy
    bandwidth over its algorithmic bytes, and sampled states against oracle A."""
    import torch
    import oracle
    from gen import workloads
    from paper_2502_03445_gb300 import tqc
    net = workloads.smallk_network(case)
    h = tqc.Network(net, dtype=tqc.F32)
    hbm = peaks()[0]
    res = {}
    for tag, flags in (("smallk", 0), ("general", tqc.FLAG_NO_SMALLK)):
        p = tqc.Plan(h, precision="fp32", flags=tqc.FLAG_NO_RENORM | flags)
        o = torch.empty(p.out_elems, dtype=torch.float32, device="cuda")
        for _ in range(max(3, args.warmup)):
            p.contract(o)
        torch.cuda.synchronize()
        p.profile(True)
        for _ in range(args.steps):
            p.contract(o)
        torch.cuda.synchronize()
        d = p.describe()
        last = len(d["steps"]) - 1
        st = d["steps"][last]
        ms = p.step_time(last)[0]
        p.profile(False)
        m, n, k = st["log2_m"], st["log2_n"], st["log2_k"]
        alg = 4.0 * (2 ** (m + n) + 2 ** (m + k) + 2 ** (n + k))
        gbs = alg / (ms / 1e3) / 1e9
        res[tag] = {"ms": ms, "GB/s": gbs, "frac": gbs / hbm, "tile": st["tile"]}
        if tag == "smallk":
            rng = np.random.Generator(np.random.PCG64(5))
            idx = sorted(set(int(i) for i in rng.integers(0, 1 << net.n_qubits, size=4)))
            want = oracle.recon_states(net, idx)
            got = o[torch.tensor(idx, device="cuda")].double().cpu().numpy()
            res["max_abs_err_vs_oracle"] = float(np.abs(got - want).max())
            res["max_abs_p"] = float(np.abs(want).max())
            res["step"] = {"log2_m": m, "log2_n": n, "log2_k": k, "mask_r": hex(st["mask_r"]),
                           "mask_c": hex(st["mask_c"])}
            res["algorithmic_bytes"] = alg
        p.close()
        del o
    h.close()
    res["speedup_of_smallk"] = res["general"]["ms"] / res["smallk"]["ms"]
    return res


def run_smallk(args):
    import torch
    torch.cuda.set_device(0)
    from gen import workloads
    cases = list(workloads.SMALLK_CASES) if args.smallk == "all" else [args.smallk]
    out = {c: measure_smallk(args, c) for c in cases}
    print(json.dumps({"metric": "small-K CUDA-core final step, GB/s over algorithmic bytes", "unit": "GB/s",
                      "peak": peaks()[0], "peak_kind": f"{peaks()[3]} copy bandwidth", "steps": args.steps,
                      "cases": out}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch > 0:
        return run_batch(args)
    if args.smallk:
        return run_smallk(args)
    if args.planner_eval:
        return run_planner_eval(args)
    if args.hss:
        return run_hss(args)
    if args.states:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(measure_states(args, args.states)), flush=True)
        return 0
    if args.cuts:
        print(json.dumps(measure_cut_finder()), flush=True)
        return 0
    if args.workload != "grid30":
        return run_workload(args)
    ws, rank, local = dist_env()
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from gen import workloads
    from paper_2502_03445_gb300 import shard, tqc

    net = workloads.grid30(rank)          # weak scaling: one independent network per rank
    # upload (tensors to HBM) and planning (host only) are timed apart from the steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = tqc.Network(net)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    free = None if args.free_qubits >= net.n_qubits else list(range(args.free_qubits))
    plan = tqc.Plan(h, precision=args.precision, free_qubits=free)
    t2 = time.perf_counter()
    setup = {"upload_ms": 1e3 * (t1 - t0), "upload_bytes": int(sum(nd.data.nbytes for nd in net.nodes)),
             "planning_ms": 1e3 * (t2 - t1)}
    desc = plan.describe()
    cost = plan.cost_report()
    out = torch.empty(plan.out_elems, dtype=torch.float32, device="cuda")
    probs_per_step = plan.out_elems

    # warm up (allocates the workspace), then sample clocks around the timed region
    for _ in range(max(args.warmup, 3)):
        plan.contract(out)
    torch.cuda.synchronize()
    desc = plan.describe()                # tiles and K splits as the first contract set them
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 and not args.no_clocks else None
    t_end = time.time() + (0.0 if args.no_clocks else 0.6)   # load the GPU so the sampler sees it
    while time.time() < t_end:
        plan.contract(out)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    plan.profile(True)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(args.steps):
        plan.contract(out)
    e.record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = s.elapsed_time(e) / args.steps
    clocks = sampler.stop() if sampler else None
    # whole job: probabilities of every rank over the slowest rank's time
    total_probs, sec = shard.aggregate(float(probs_per_step), ms / 1e3, dist if ws > 1 else None, "cuda")
    ms = sec * 1e3
    value = total_probs / sec

    # dominant kernel: the step with the largest mean duration over the timed region
    hbm, bf16, bf16_sus, peak_kind = peaks()
    step_ms = [plan.step_time(i)[0] for i in range(len(desc["steps"]))]
    plan.profile(False)
    top = int(np.argmax(step_ms))
    st = desc["steps"][top]
    out_b = 4
    byt, fl = step_bytes(st, out_b), step_flops(st)
    t_top = step_ms[top] / 1e3
    ridge = bf16 * 1e12 / (hbm * 1e9)
    kern = "umma_step" if st["class"] == "tcgen05" else "simt_step"
    if fl / byt < ridge or st["class"] != "tcgen05":
        roof = {"bound": "hbm", "achieved": byt / t_top / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_kind": f"{peak_kind} copy bandwidth"}
    else:
        roof = {"bound": "tensor", "achieved": fl / t_top / 1e12, "peak": bf16, "unit": "TFLOP/s",
                "peak_kind": f"{peak_kind} bf16 burst"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = traffic_record(f"{kern}_grid30") if top == len(desc["steps"]) - 1 else None
    roof["kernel"] = f"{kern} (step {top}: log2 M,N,K = {st['log2_m']},{st['log2_n']},{st['log2_k']})"
    roof["algorithmic_bytes_per_launch"] = byt
    roof["mean_launch_ms"] = step_ms[top]
    roof["step_ms"] = step_ms
    # the whole plan against its roofline, and the plan-independent floor
    # (the FP32 output written once and the FP64 node tensors read once)
    roof["path_roofline_ms"] = path_roofline(desc["steps"], 1, hbm, bf16)
    roof["path_frac"] = roof["path_roofline_ms"] / ms
    in_bytes = sum(8 * nd.tensor().size for nd in net.nodes)
    roof["floor_ms"] = (4 * plan.out_elems + in_bytes) / (hbm * 1e9) * 1e3

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": step_dtypes(desc), "data": "synthetic",
            "config": {"workload": WORKLOAD if free is None else
                       WORKLOAD.replace("full 2^30 output", f"bin of the lowest {args.free_qubits} qubits"),
                       "plan": [[s_["log2_m"], s_["log2_n"], s_["log2_k"], s_["class"], s_["tile"],
                                 s_["ksplit"], s_["kblk"]] for s_ in desc["steps"]],
                       "plan_fields": PLAN_FIELDS,
                       "order": desc["order"], "instance_seed": "2000 + rank",
                       "l2": "working set 4.6 GB > 129 MB L2, no flush needed",
                       "parallelism": f"weak x{ws}, one network per GPU"},
            "roofline": roof, "gpu_launches": desc["launches_per_contract"] * args.steps,
            "clocks": clocks, "setup": setup, "cost_report": cost}

    # plain FP32 CUDA-core form on the same network
    if not args.no_plain:
        pplan = tqc.Plan(h, precision="fp32", free_qubits=free)
        pms = time_plan(torch, pplan, out, max(2, min(args.steps, 5)), 2)
        line["plain_fp32"] = {"value": probs_per_step / (pms / 1e3), "ms_per_step": pms,
                              "speedup_of_chosen": pms / ms}
        plain_out = out.clone()
        plan.contract(out)
        torch.cuda.synchronize()
        tv = 0.5 * (out.double() - plain_out.double()).abs().sum().item()
        line["plain_fp32"]["tv_chosen_vs_plain_full_vector"] = tv
        del plain_out
        pplan.close()
    else:
        plan.contract(out)
        torch.cuda.synchronize()

    # accuracy of the chosen form against the oracle on sampled states (rank 0)
    if rank == 0 and not args.no_cpu_baseline:
        cpu, states, want = cpu_oracle_sample(net, n_free=min(args.free_qubits, net.n_qubits))
        line["cpu_baseline"] = cpu
        got = out.cpu().numpy()[np.array(states, dtype=np.int64)].astype(np.float64)
        err = np.abs(got - want)
        line["error_vs_oracle"] = {"states": len(states), "max_abs": float(err.max()),
                                   "max_abs_rel_to_max_p": float(err.max() / np.abs(want).max()),
                                   "tv_estimate": float(0.5 * err.mean() * probs_per_step)}

    # end to end through the C ABI with host buffers: H2D of the tensors, D2H of the bin
    if not args.no_e2e:
        hin = [torch.from_numpy(np.ascontiguousarray(nd.data)).pin_memory() for nd in net.nodes]
        hout = torch.empty(plan.out_elems, dtype=torch.float32).pin_memory()
        plan.contract_host(hin, hout)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            plan.contract_host(hin, hout)
        t_e2e = (time.perf_counter() - t0) / args.e2e_steps
        e2e_probs, t_e2e = shard.aggregate(float(probs_per_step), t_e2e, dist if ws > 1 else None, "cuda")
        line["e2e"] = {"value": e2e_probs / t_e2e, "unit": UNIT,
                       "h2d_bytes_per_step": int(sum(x.numel() * 8 for x in hin)),
                       "d2h_bytes_per_step": int(hout.numel() * 4), "ms_per_step": 1e3 * t_e2e}
    plan.close()
    h.close()
    del out
    torch.cuda.empty_cache()
    # sub-records at one GPU: the tensor-bound bin, the batched launch, state
    # lists, reuse across bins, the cut finder
    if ws == 1 and not args.no_sub:
        tb = measure_tensor_bound(args, "qaoa48", steps=args.sub_steps, warmup=args.warmup)
        tb.pop("_spec")
        line["tensor_bound"] = tb
        line["batched"] = measure_batched(args, 256, steps=args.sub_steps, warmup=args.warmup)
        line["states"] = measure_states(args, 1_000_000, steps=args.sub_steps, warmup=args.warmup)
        line["bin_stream"] = measure_bin_stream(args)
        line["cut_finder"] = measure_cut_finder()
        line["learned_planner"] = measure_learned_planner(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
