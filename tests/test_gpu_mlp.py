"""The cost model's CUDA forward, gradient and training kernels against the float64 reference
network (oracle/mlp.py), and what the trained network gains over the closed-form bound.

Tolerance: FP32 evaluation of dot products of at most 64 terms and gradient sums over at most a
few hundred samples carry relative errors of order (64 + n) * 2^-24 ~ 3e-5 of the summed
magnitudes; 1e-3 of the largest magnitude is used, far below what a wrong term would cause."""

import numpy as np
import pytest

import paper_1501_02237_gb300 as bd
from oracle import mlp
from workloads import batch_systems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield


def close(a, b, rel=1e-3):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b)) <= rel * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("seed", range(3))
def test_forward_and_gradient_match_reference(seed):
    rng = np.random.default_rng(seed)
    m = bd.CostModel(seed)
    p = rng.normal(0, 0.2, mlp.NPARAM).astype(np.float32)
    mean = rng.normal(0, 1, mlp.F).astype(np.float32)
    std = rng.uniform(0.5, 2.0, mlp.F).astype(np.float32)
    m.set_params(p, np.concatenate([mean, std]))
    X = rng.normal(0, 2, (300, mlp.F)).astype(np.float32)
    y = rng.normal(0, 1, 300).astype(np.float32)
    f_ref, _ = mlp.forward(p.astype(np.float64), X, mean, std)
    assert close(m.predict(X), f_ref)
    g, loss = m.gradient(X, y)
    g_ref = mlp.gradient(p.astype(np.float64), X, y, mean, std)
    assert close(g, g_ref)
    assert abs(loss - mlp.loss(p.astype(np.float64), X, y, mean, std)) <= 1e-3 * max(1.0, loss)


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (4000, mlp.F)).astype(np.float32)
    y = (X @ rng.normal(0, 1, mlp.F) + 0.5 * np.abs(X[:, 0])).astype(np.float32)
    m = bd.CostModel(3)
    base = float(np.mean((y - y.mean()) ** 2))
    final = m.train(X, y, epochs=40, batch=128, lr=3e-3, seed=5)
    assert final < 0.05 * base
    assert float(np.mean((m.predict(X) - y) ** 2)) < 0.05 * base


@pytest.fixture(scope="module")
def trained():
    # training data made by the method itself: per-system SM cycles of a batched run
    systems = batch_systems(700, first_seed=20000)
    b = bd.Batch()
    for s in systems:
        b.add(s.A, seed=0)
    b.prepare()
    b.run(mode=0)
    cyc = np.array([r["cycles"] for r in b.results()], dtype=np.float64)
    X = b.features()
    b.close()
    keep = cyc > 0
    X, y, cyc = X[keep], np.log2(cyc[keep]).astype(np.float32), cyc[keep]
    n_train = int(0.7 * len(y))
    m = bd.CostModel(0)
    m.train(X[:n_train], y[:n_train], epochs=300, batch=64, lr=2e-3, seed=1)
    # the method without the network: log2 of the closed-form bound, calibrated by least squares
    cf = X[:, 3].astype(np.float64)
    A = np.stack([np.ones(n_train), cf[:n_train]], 1)
    coef, *_ = np.linalg.lstsq(A, y[:n_train], rcond=None)
    return dict(m=m, X=X, y=y, cyc=cyc, n=n_train, cf=coef[0] + coef[1] * cf)


def test_trained_model_beats_closed_form_bound(trained):
    t, n = trained, trained["n"]
    err_mlp = np.mean(np.abs(t["m"].predict(t["X"][n:]) - t["y"][n:]))
    err_cf = np.mean(np.abs(t["cf"][n:] - t["y"][n:]))
    assert err_mlp < 0.8 * err_cf, (err_mlp, err_cf)


def mean_completion(costs, order):
    """Mean completion time of the held-out systems run one after another in `order`."""
    return float(np.mean(np.cumsum(costs[order])))


def test_trained_model_improves_the_shortest_first_schedule(trained):
    # Schedule quality on the held-out systems, each weighed by its measured cost (SM cycles of
    # its work in the batched run): admitting the shortest predicted first, the network's
    # predictions give a lower mean completion time than the closed-form bound's, and both beat
    # arrival order; the order by the measured costs themselves is the lower limit.
    t, n = trained, trained["n"]
    c = t["cyc"][n:]
    mct = dict(fifo=mean_completion(c, np.arange(len(c))),
               closed_form=mean_completion(c, np.argsort(t["cf"][n:], kind="stable")),
               network=mean_completion(c, np.argsort(t["m"].predict(t["X"][n:]), kind="stable")),
               measured=mean_completion(c, np.argsort(c, kind="stable")))
    assert mct["measured"] <= mct["network"] < mct["closed_form"] < mct["fifo"], mct
    # the network closes a good part of the gap that the closed form leaves to the best order
    # (measured on a GB300: about 45 % of it)
    gap_cf = mct["closed_form"] - mct["measured"]
    gap_net = mct["network"] - mct["measured"]
    assert gap_net < 0.8 * gap_cf, mct


def serve_burst(systems, order, costs, slots=4):
    """Submit every system at once to a server with few slots, so that admission order decides
    who waits; (mean latency ms, degrees in submission order)."""
    srv = bd.Server(slots=slots, order=order)
    got = {}
    try:
        tickets = [srv.submit(s.A, seed=5, predicted_cost=float(costs[i]) if costs is not None else 0.0)
                   for i, s in enumerate(systems)]
        while len(got) < len(tickets):
            r = srv.poll(wait_ms=5000)
            assert r is not None, "server stalled"
            got[r[0]] = (r[1]["degree"], r[2])
    finally:
        srv.stop()
    return float(np.mean([got[t][1] for t in tickets])), [got[t][0] for t in tickets]


def test_cost_ordered_admission_lowers_latency_under_load(trained):
    # Serving under load (a burst of systems large enough that the GPU, not the submitting thread,
    # sets the pace, into 4 slots): admitting the smallest predicted cost first, with the network's
    # predictions, gives a lower mean latency than arrival order on held-out systems, and every
    # degree is the same whatever the order.
    systems = batch_systems(120, first_seed=21000, n_range=(20, 28), k_range=(6, 9))
    b = bd.Batch()
    for s in systems:
        b.add(s.A, seed=5)
    b.prepare()
    pred = np.exp2(trained["m"].predict(b.features()))
    b.run(mode=0)
    want = [r["degree"] for r in b.results()]
    b.close()
    fifo, d_fifo = serve_burst(systems, 0, None)
    net, d_net = serve_burst(systems, 1, pred)
    closed, d_cf = serve_burst(systems, 1, None)
    assert d_fifo == d_net == d_cf == want
    assert net < 0.8 * fifo, dict(fifo=fifo, network=net, closed_form=closed)
