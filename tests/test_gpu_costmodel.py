"""GPU kernels of the learned path cost model against the FP64 oracle, and what
the trained model gains over FLOP-count ranking.

The GPU forward pass uses BF16 copies of the weight matrices (biases FP32) and
FP32 accumulation; the oracle is given the same BF16-rounded weights in FP64,
so the comparison isolates the FP32 arithmetic (bound: 1e-4 relative per
gradient tensor).
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

D, H = 16, 64


@pytest.fixture(scope="module")
def T():
    from paper_2104_10523_gb300 import build, tnq
    build.build()
    tnq.load()
    return tnq


def flat(P):
    return np.concatenate([P[k].reshape(-1) for k in omlp.PARAMS]).astype(np.float32)


def unflat(v):
    out, o = {}, 0
    for k, shape in (("W1", (D, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, 1)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def oracle_view(P32):
    """The parameters as the GPU forward sees them: BF16 weights, FP32 biases."""
    P = unflat(P32)
    for k in ("W1", "W2", "W3"):
        P[k] = omlp.bf16_round(P[k])
    return P


def data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, size=(n, D)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    return X, t


def model(T, max_batch=512):
    ctx = T.Context(0, "fp32")
    m = T.CostModel(ctx, hidden=H, max_batch=max_batch, seed=3)
    P = omlp.init_params(D, H, seed=5)
    rng = np.random.default_rng(6)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.standard_normal(P[k].shape) * 0.1
    m.set_params(flat(P))
    return ctx, m


def test_gradients_match_oracle(T):
    ctx, m = model(T)
    X, t = data(1, 256)
    g, loss = m.gradients(X, t)
    P = oracle_view(m.get_params())
    Xo, to = X.astype(np.float64), t.astype(np.float64)
    G = omlp.gradients(P, Xo, to)
    Gg = unflat(g)
    for k in omlp.PARAMS:
        err = np.linalg.norm(Gg[k] - G[k]) / max(np.linalg.norm(G[k]), 1e-30)
        assert err <= 1e-4, (k, err)
    assert abs(loss - omlp.loss(P, Xo, to)) <= 1e-5 * omlp.loss(P, Xo, to)


def test_adam_step_matches_oracle(T):
    ctx, m = model(T)
    X, t = data(2, 256)
    before = m.get_params()
    m.train(X, t, epochs=1, batch=256, lr=1e-3)
    after = m.get_params()
    P = oracle_view(before)
    G = omlp.gradients(P, X.astype(np.float64), t.astype(np.float64))
    P0 = unflat(before)
    P1 = {k: v.copy() for k, v in P0.items()}
    omlp.adam_step(P1, G, {}, lr=1e-3, step=1)
    want = flat(P1).astype(np.float64) - before
    got = after.astype(np.float64) - before
    # the first Adam step is lr * g / (|g| + eps): entries with gradients at the FP32
    # noise level may flip sign, so require agreement on nearly all entries
    close = np.abs(got - want) <= 2e-5
    assert close.mean() >= 0.99, close.mean()


def test_training_fits_synthetic_step_times(T):
    """On rows whose target is a smooth function of the features the loss falls
    far below the target variance."""
    ctx, m = model(T, max_batch=1024)
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, size=(8192, D)).astype(np.float32)
    t = (3 * X[:, 4] + np.log1p(5 * X[:, 7]) + 0.5 * X[:, 10]).astype(np.float32)
    m.train(X, t, epochs=30, batch=512, lr=2e-3)
    pred = m.predict(X[:2048])
    mse = float(np.mean((pred - t[:2048]) ** 2))
    assert mse < 0.05 * float(np.var(t)), (mse, np.var(t))


def test_learned_ranking_vs_flop_ranking(T):
    """Collect step timings on executed plans, train the model on the GPU, then
    rank the candidate trees of held-out circuits by predicted time and compare
    the measured time of the learned pick with the FLOP-minimal pick."""
    from paper_2104_10523_gb300 import costmodel
    from workloads import cost_model_circuit
    ctx = T.Context(0, "bf16x3")
    train_c = costmodel.pick_circuits(range(0, 40), 5e9, cost_model_circuit)[:12]
    eval_c = costmodel.pick_circuits(range(2000, 2040), 5e9, cost_model_circuit)[:8]
    X, t = costmodel.collect(ctx, train_c, 4, "bf16x3")
    assert X.shape[0] == t.shape[0] > 500
    m = T.CostModel(ctx, hidden=256, max_batch=4096, seed=1)
    m.train(X, t, epochs=40, batch=512, lr=1e-3)
    resid = m.predict(X) - t
    assert float(np.mean(resid ** 2)) < 0.5 * float(np.var(t))
    rows = costmodel.evaluate(ctx, m, eval_c, n_candidates=16)
    s = costmodel.summarize(rows)
    print("learned vs FLOP-minimal ranking:", s)
    assert s["n"] == len(eval_c)
    # the learned pick is not systematically slower than the FLOP-minimal one
    assert s["geomean_ratio"] <= 1.10, s


def test_learned_ranking_gain_at_workload_scale(T):
    """The cost-model workload at its own scale: the model is trained on step
    timings of the training circuits (seeds 0-1999 up to 1e12 flops, about
    1,500 circuits) and ranks 32 candidate trees of each held-out circuit
    (seeds 2000-2199); the measured time of its pick is compared with the
    FLOP-minimal pick's.  The learned ranking must gain: geometric-mean time
    ratio below 0.95, and more wins than losses."""
    from paper_2104_10523_gb300 import costmodel
    ctx = T.Context(0, "tf32x3")
    out = costmodel.run_config5(ctx, "tf32x3", 1e12, epochs=30)
    s = out["eval"]
    print("config-5 learned vs FLOP-minimal:", {k: out[k] for k in out if k != "rows"})
    assert out["train_circuits"] >= 1000 and s["n"] >= 100
    assert out["final_loss"] < 0.2 * out["target_variance"]
    assert s["geomean_ratio"] < 0.95, s
    assert s["wins"] > s["losses"], s

