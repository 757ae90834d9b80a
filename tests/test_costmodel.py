"""Learned cost model: the FP64 oracle pinned by finite differences, the GPU
forward/backward against it, training, and what the trained model gains
over the analytic FLOP/byte model that the planner uses without it."""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from gen import tensors
from paper_2502_03445_gb300 import tqc

F = tqc.PLAN_FEATURES


def seeded_problem(seed, n=48):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.standard_normal((n, F))
    t = np.sin(X[:, 0]) + 0.5 * X[:, 1] ** 2 - 0.3 * X[:, 2] * X[:, 3]
    theta = rng.standard_normal(omlp.n_params(F)) * 0.1
    return X, t, theta


# ---------------------------------------------------------------- CPU: pin the oracle
@pytest.mark.parametrize("seed", [0, 1])
def test_oracle_backprop_matches_finite_differences(seed):
    X, t, theta = seeded_problem(seed, n=12)
    g = omlp.grad(theta, X, t)
    rng = np.random.Generator(np.random.PCG64(seed + 10))
    idx = rng.choice(len(theta), size=60, replace=False)
    # every layer's weights and biases are represented
    sh = omlp.shapes(F)
    starts = np.cumsum([0] + [int(np.prod(s)) for s in sh])[:-1]
    idx = np.concatenate([idx, starts, np.minimum(starts + 1, len(theta) - 1), [len(theta) - 1]])
    fd = omlp.finite_difference_grad(theta, X, t, idx)
    np.testing.assert_allclose(g[idx], fd, rtol=1e-6, atol=1e-9)


def test_oracle_planted_mistake_is_caught():
    """Dropping the ReLU mask in backprop breaks the finite-difference pin."""
    X, t, theta = seeded_problem(3, n=12)
    W1, b1, W2, b2, W3, b3, W4, b4 = omlp.unpack(theta, F)
    y, (A0, Z1, A1, Z2, A2, Z3, A3) = omlp.forward(theta, X)
    dy = (2.0 / len(t)) * (y - t)[:, None]
    wrong_gW3 = A2.T @ (dy @ W4.T)          # mask (Z3 > 0) left out
    k0 = sum(int(np.prod(s)) for s in omlp.shapes(F)[:4])
    idx = list(range(k0, k0 + 40))
    fd = omlp.finite_difference_grad(theta, X, t, idx)
    assert np.abs(wrong_gW3.reshape(-1)[:40] - fd).max() > 1e-3


def test_adam_matches_its_definition_on_a_quadratic():
    theta = np.array([3.0, -2.0])
    m = v = np.zeros(2)
    for step in range(1, 2001):
        theta, m, v = omlp.adam_step(theta, 2 * theta, m, v, step, lr=0.05)
    assert np.abs(theta).max() < 1e-2


# ---------------------------------------------------------------- host: candidates and features
def test_candidates_and_features_on_shape_only_network():
    net = tensors.sample_shape  # noqa: F841 (keeps the import used by name)
    n = tensors.random_shape_network(20, 6, 10, 10, seed=5)
    h = tqc.Network(n, shape_only=True)
    cands = tqc.plan_candidates(h, 12)
    assert len(cands) >= 4
    keys = set()
    for od in cands:
        p = tqc.Plan(h, order=od)
        f = p.features()
        assert f.shape == (F,) and np.all(np.isfinite(f))
        keys.add(tuple(map(tuple, od)))
        p.close()
    assert len(keys) == len(cands)
    # without a model file the learned planner falls back to the analytic one
    p = tqc.Plan(h, planner=tqc.PLANNER_LEARNED, costmodel_path="/nonexistent/model.bin")
    assert p.describe()["planner"].startswith("fallback")


# ---------------------------------------------------------------- GPU
torch = pytest.importorskip("torch")


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [0, 1])
def test_gpu_gradient_matches_fp64_oracle(seed):
    _cuda()
    X, t, _ = seeded_problem(seed, n=64)
    cm = tqc.CostModel(F, seed=seed)
    theta = cm.params().astype(np.float64)
    loss_gpu, g_gpu = cm.grad(X.astype(np.float32), t.astype(np.float32))
    # the oracle sees the FP32-rounded inputs the GPU sees
    Xr, tr = X.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64)
    g_or = omlp.grad(theta, Xr, tr)
    assert abs(loss_gpu - omlp.loss(theta, Xr, tr)) <= 1e-4 * abs(omlp.loss(theta, Xr, tr))
    rel = np.linalg.norm(g_gpu - g_or) / np.linalg.norm(g_or)
    assert rel <= 1e-4, rel
    assert np.abs(g_gpu - g_or).max() <= 1e-4 * np.abs(g_or).max()
    cm.close()


@pytest.mark.gpu
def test_gpu_training_fits_a_smooth_function():
    _cuda()
    X, t, _ = seeded_problem(7, n=2048)
    cm = tqc.CostModel(F, seed=1)
    first = cm.train(X, t, epochs=1, batch=128, lr=1e-3, seed=2)
    last = cm.train(X, t, epochs=150, batch=128, lr=1e-3, seed=3)
    assert last < 0.1 and last < 0.2 * first, (first, last)
    pred = cm.predict(X[:256])
    assert np.corrcoef(pred, t[:256])[0, 1] > 0.95
    cm.close()


@pytest.mark.gpu
def test_learned_model_beats_the_analytic_estimate(tmp_path):
    """Train on the planner's own timings of training networks (27-30-qubit
    networks of 4-6 subcircuits plus smaller ones); on held-out 27-30-qubit
    networks the model predicts measured time better than the analytic
    FLOP/byte estimate (the paper's Eq. classical_runtime, which it finds
    consistently high), and the learned planner's plans are within 3% of the
    fastest timed candidate and of the default planner's (TQC_PLANNER_AUTO).
    Its plans are not faster here: with the small-K CUDA-core tile (whose
    slower predecessor the analytic model priced wrong, which the learned
    correction used to win by) the analytic ranking already picks plans
    within 1% of the fastest candidate on this family."""
    _cuda()
    from gen import workloads
    from paper_2502_03445_gb300 import costmodel
    train_recs, test_sets = [], []
    nets = [("g30", 9800 + i) for i in range(24)] + [("small", 9000 + i) for i in range(12)]
    for kind, seed in nets:
        net = workloads.planner_network(seed, kind)
        h = tqc.Network(net, dtype=tqc.F32)
        recs = costmodel.collect(h, precision="auto", max_candidates=8, reps=5)
        if kind == "g30" and seed >= 9816:
            test_sets.append((net, recs))
        else:
            train_recs.extend(recs)
        h.close()
    X, y = costmodel.dataset(train_recs)
    cm = tqc.CostModel(F, seed=0)
    cm.train(X, y, epochs=400, batch=32, lr=1e-3, seed=1)
    path = str(tmp_path / "costmodel.bin")
    cm.save(path)
    err_mlp, err_flop, r_learned, r_analytic, r_auto = [], [], [], [], []
    for net, recs in test_sets:
        yt = np.log([r["seconds"] for r in recs])
        pred = costmodel.predicted_log_seconds(cm, recs)
        ana = np.log([r["predicted_s"] for r in recs])
        err_mlp.append(np.mean(np.abs(pred - yt)))
        err_flop.append(np.mean(np.abs(ana - yt)))
        meas = np.array([r["seconds"] for r in recs])
        best = meas.min()
        r_analytic.append(meas[int(np.argmin(ana))] / best)
        # the plans tqc_plan picks with the learned and the default planner, timed
        h = tqc.Network(net, dtype=tqc.F32)
        out = torch.empty(1 << net.n_qubits, dtype=torch.float32, device="cuda")
        for planner, dst in ((tqc.PLANNER_LEARNED, r_learned), (tqc.PLANNER_AUTO, r_auto)):
            p = tqc.Plan(h, planner=planner, costmodel_path=path if planner == tqc.PLANNER_LEARNED else None)
            assert planner != tqc.PLANNER_LEARNED or p.describe()["planner"] == "learned"
            dst.append(costmodel.time_plan(p, out, reps=5) / best)
            p.close()
        del out
        h.close()
    gm = lambda x: float(np.exp(np.mean(np.log(x))))
    print("mean |log err| mlp", np.mean(err_mlp), "analytic", np.mean(err_flop))
    print("plan time / best candidate: learned", gm(r_learned), "analytic ranking", gm(r_analytic), "auto", gm(r_auto))
    assert np.mean(err_mlp) < np.mean(err_flop)
    assert gm(r_learned) <= 1.03 and gm(r_learned) <= 1.03 * gm(r_auto)
    cm.close()
