"""Gradients and replay on the GPU: CUDA-graph replays equal direct launches;
the score-function gradients (density, Bragg scale, radius with the interface
term) agree with central finite differences on common random numbers; and
TransportFn's backward equals the contraction of the accumulators."""
import numpy as np
import pytest

import workloads as W
from stats import stats

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as G
    G.build()
    from paper_2304_06226_gb300 import engine
    return engine


def test_graph_replay_equals_direct_launch(eng):
    n = 30_000
    desc = W.slab(g=3.0, n_histories=n, precision="f64")
    direct = eng.Scene(desc)
    graphed = eng.Scene(desc)
    for first in (0, n, 5 * n):          # same launch key: one capture, replays
        direct.run(n, first=first, kernel=1)
        graphed.run(n, first=first, kernel=1, graph=True)
    graphed.run(n // 3, first=9 * n, kernel=1, graph=True)   # new total: captured again
    direct.run(n // 3, first=9 * n, kernel=1)
    torch.cuda.synchronize()
    a, b = direct.raw(0), graphed.raw(0)
    assert np.allclose(a["sum"], b["sum"], rtol=1e-12, atol=1e-14)
    assert np.allclose(a["sumsq"], b["sumsq"], rtol=1e-12, atol=1e-14)
    assert graphed.counters()["histories"] == 3 * n + n // 3


def one_instance(radius=0.5, scale=1.0, density=1.0, precision="f32"):
    d = W.batched(n_instances=1, count_lo=1e6, count_hi=1e6, precision=precision)
    d["instances"]["params"] = np.array([[radius, scale, density]])
    return d


def total_and_grad(eng, params, n, nbatch, want_grad):
    """Integrated detector total per batch (and its LR gradient per unit of
    each parameter), over the same history ids for every call."""
    desc = one_instance(*params)
    sc = eng.Scene(desc)
    tot, grad = [], []
    for b in range(nbatch):
        sc.reset()
        sc.run(n, first=b * n, want_grad=want_grad, kernel=1)
        torch.cuda.synchronize()
        raw = sc.raw(0)
        tot.append(raw["sum"].sum() / n)
        if want_grad:
            g = raw["J"].sum(axis=1) / n
            g[1] /= params[1]     # scale: accumulators are per log-parameter
            g[2] /= params[2]     # density
            grad.append(g)
    sc.close()
    return np.array(tot), (np.array(grad) if want_grad else None)


@pytest.mark.parametrize("p,h,nsig", [(1, 0.05, 4.0), (2, 0.05, 4.0), (0, 0.02, 5.0)])
def test_gradient_matches_crn_finite_differences(eng, p, h, nsig):
    base = [0.5, 1.0, 1.0]
    n, nb = 1_000_000, 16
    _, lr = total_and_grad(eng, base, n, nb, True)
    up = list(base); up[p] += h
    dn = list(base); dn[p] -= h
    tp, _ = total_and_grad(eng, up, n, nb, False)
    tm, _ = total_and_grad(eng, dn, n, nb, False)
    fd = (tp - tm) / (2 * h)
    diff = lr[:, p] - fd
    err = diff.std(ddof=1) / np.sqrt(nb)
    assert abs(diff.mean()) < nsig * err + 1e-3 * abs(fd.mean()), (p, lr[:, p].mean(), fd.mean(), err)
    assert abs(fd.mean()) > 3 * fd.std(ddof=1) / np.sqrt(nb)   # a non-trivial derivative


def test_transportfn_backward_is_the_accumulator_contraction(eng):
    desc = W.batched(n_instances=3, count_lo=2e5, count_hi=2e5)
    sc = eng.Scene(desc)
    params = torch.tensor(desc["instances"]["params"], dtype=torch.float64, requires_grad=True)
    means = eng.TransportFn.apply(params, sc)
    w = torch.linspace(0.0, 1.0, means.shape[1], dtype=torch.float64, device=means.device)
    loss = (means * w).sum()
    loss.backward()
    got = params.grad.cpu().numpy()
    for q in range(3):
        raw = sc.raw(q)
        n = float(desc["instances"]["counts"][q])
        expect = raw["J"] @ w.cpu().numpy() / n
        expect[1] /= desc["instances"]["params"][q][1]
        expect[2] /= desc["instances"]["params"][q][2]
        assert np.allclose(got[q], expect, rtol=1e-9, atol=1e-12)
    # the forward really ran with these parameters
    m0 = means[0].sum().item()
    assert 0.3 < m0 < 1.0
