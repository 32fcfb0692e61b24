"""Batched cylinders (cyl_plan_batch / cyl_heat_step_batch): every problem of
a batch must equal its own single-problem run, for every launch
configuration the autotuner may pick, inside a CUDA graph too, and match the
oracle."""
import numpy as np
import pytest

from oracle import heat as oheat
from paper_2206_04827_gb300 import inputs

torch = pytest.importorskip('torch')
pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def cyl():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_2206_04827_gb300 import cyl as C
    return C


def _batch(rng, k, lo, hi, thetas):
    n_r = rng.integers(lo, hi + 1, size=k)
    n_z = rng.integers(lo, hi + 1, size=k)
    n_t = rng.choice(thetas, size=k)
    alpha = rng.uniform(0.01, 1.0, size=k)
    return n_r, n_z, n_t, alpha


def _fields(rng, shapes):
    return [inputs.smooth_coeffs(p, m, n, 1.25, rng) for p, m, n in shapes]


def _run_batch(bp, T0s, gs, steps):
    T = torch.cat([torch.as_tensor(x, device='cuda').reshape(-1) for x in T0s])
    g = torch.cat([torch.as_tensor(x, device='cuda').reshape(-1) for x in gs])
    bp.heat_step(T, g, steps)
    bp.sync()
    return [bp.view(T, i).cpu().numpy() for i in range(len(T0s))]


def _run_plain(cyl, shapes, alpha, dt, T0s, gs, steps, twisted=False):
    """Per-problem runs; plain LU sweeps unless twisted (the batch kernel's
    arithmetic, so equal bit for bit)."""
    out = []
    for (p, m, n), a, x, gg in zip(shapes, alpha, T0s, gs):
        pl = cyl.Plan(m, n, p, a, dt, 1e-14, poisson=False, heat=True,
                      extra_flags=0 if twisted else cyl.PLAIN_SWEEPS)
        T = torch.as_tensor(x, device='cuda').clone()
        pl.heat_step(T, torch.as_tensor(gg, device='cuda'), steps)
        pl.sync()
        out.append(T.cpu().numpy())
        pl.close()
    return out


def test_batch_equals_single_problem_runs_for_every_config(cyl):
    rng = np.random.default_rng(31)
    n_r, n_z, n_t, alpha = _batch(rng, 7, 6, 72, [4, 8, 16])
    dt, steps = 1e-3, 4
    bp = cyl.BatchPlan(n_r, n_z, n_t, alpha, dt, 1e-14, plain_sweeps=True)
    T0s = _fields(rng, bp.shapes)
    gs = _fields(rng, bp.shapes)
    plain = _run_plain(cyl, bp.shapes, alpha, dt, T0s, gs, steps)
    configs = [(63, 4), (0, 1), (31, 2), (15, 4), (95, 1), (47, 2)]
    # one-sided sweeps in both forms: the same arithmetic, bit for bit, with one or two chains per thread
    for thr, G in configs:
        for cpt in (1, 2):
            bp.set_config(thr, G, chains_per_thread=cpt)
            got = _run_batch(bp, T0s, gs, steps)
            for a, b in zip(got, plain):
                assert np.abs(a - b).max() <= 1e-15 * np.abs(b).max()
    # the default batch (twisted solves per slice) and the per-problem default agree to rounding
    tw = cyl.BatchPlan(n_r, n_z, n_t, alpha, dt, 1e-14)
    for thr, G in configs:
        try:
            tw.set_config(thr, G)
        except cyl.CylError:
            continue          # a twisted class may not fit this (threshold, groups) setting
        for a, b in zip(_run_batch(tw, T0s, gs, steps), plain):
            assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    for a, b in zip(_run_plain(cyl, bp.shapes, alpha, dt, T0s, gs, steps, twisted=True), plain):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_batch_matches_oracle(cyl):
    rng = np.random.default_rng(32)
    n_r, n_z, n_t, alpha = _batch(rng, 4, 8, 30, [4, 8])
    dt, steps = 2e-3, 3
    bp = cyl.BatchPlan(n_r, n_z, n_t, alpha, dt, 1e-14)
    T0s = _fields(rng, bp.shapes)
    gs = _fields(rng, bp.shapes)
    got = _run_batch(bp, T0s, gs, steps)
    for a, x, gg, out in zip(alpha, T0s, gs, got):
        want = oheat.heat_steps(x, gg, a, dt, steps)
        assert np.abs(out - want).max() <= 1e-12 * np.abs(want).max()


def test_batch_autotune_and_graph_capture(cyl):
    rng = np.random.default_rng(33)
    n_r, n_z, n_t, alpha = _batch(rng, 24, 32, 160, [32, 64, 128])
    dt, steps = 1e-3, 3
    bp = cyl.BatchPlan(n_r, n_z, n_t, alpha, dt, 1e-14)
    T0s = _fields(rng, bp.shapes)
    gs = _fields(rng, bp.shapes)
    T0 = torch.cat([torch.as_tensor(x, device='cuda').reshape(-1) for x in T0s])
    g = torch.cat([torch.as_tensor(x, device='cuda').reshape(-1) for x in gs])
    ms = bp.autotune(T0, g, 1)
    assert ms > 0
    thr, G, counts = bp.config()
    assert G in (1, 2, 4) and sum(counts) > 0
    ref = T0.clone()
    bp.heat_step(ref, g, steps)
    # the batch step captured in a CUDA graph and replayed
    s = torch.cuda.Stream()
    T = T0.clone()
    with torch.cuda.stream(s):
        gb = cyl.BatchPlan(n_r, n_z, n_t, alpha, dt, 1e-14, stream=s.cuda_stream)
        gb.set_config(thr, G)
        gb.heat_step(T, g, 1)          # warm-up outside the capture
        torch.cuda.synchronize()
        T.copy_(T0)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            gb.heat_step(T, g, steps)
    T.copy_(T0)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(T, ref)
    gb.sync()
