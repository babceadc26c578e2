"""Captured-graph replay of repeated evaluations.

snap_compute / snap_compute_async / snap_compute_host capture the whole
evaluation into a CUDA graph the second time the same call (sizes, box,
buffers, tunables) is seen in a row and replay it afterwards; batches do the
same with use_graph.  A replay must give the bits of a direct evaluation, and
anything that moves a device buffer the graph refers to (workspace growth,
new coefficients) must not leave a stale graph behind.
"""
import numpy as np
import pytest

from paper_2011_12875_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snapmod():
    from paper_2011_12875_gb300 import build, snap
    build.build()
    snap.load()
    return snap


def run(s, cfg, reps):
    pos = torch.tensor(cfg.pos, device="cuda:0")
    n = cfg.natoms
    E = torch.empty(n, dtype=torch.float64, device="cuda:0")
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda:0")
    W = torch.empty(6, dtype=torch.float64, device="cuda:0")
    out = []
    for _ in range(reps):
        s.compute(pos, cfg.box, E, F, W)
        out.append([x.cpu().numpy().copy() for x in (E, F, W)])
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_replay_is_bitwise(snapmod, prec):
    """Direct run, capture, replays: identical E, F, W."""
    cfg = inputs.bcc(3, disp=0.1, seed=51)
    s = snapmod.Snap(8, inputs.beta(8), precision=prec)
    res = run(s, cfg, 5)
    for r in res[1:]:
        for x, y in zip(r, res[0]):
            assert np.array_equal(x, y)
    s.close()


def test_replay_follows_new_beta_and_workspace_growth(snapmod):
    """set_beta between replays, and a larger configuration that reallocates
    the workspace in between: each result equals a fresh context's."""
    small, big = inputs.bcc(3, disp=0.1, seed=52), inputs.bcc(5, disp=0.1, seed=53)
    b1, b2 = inputs.beta(8, seed=1), inputs.beta(8, seed=2)
    s = snapmod.Snap(8, b1, precision=1)
    run(s, small, 3)                 # captured and replayed
    s.set_beta(b2)
    after_beta = run(s, small, 3)[-1]
    run(s, big, 3)                   # workspace grows: buffers move
    after_growth = run(s, small, 3)[-1]
    s.close()
    ref = snapmod.Snap(8, b2, precision=1)
    want = run(ref, small, 1)[0]
    ref.close()
    for got in (after_beta, after_growth):
        for x, y in zip(got, want):
            assert np.array_equal(x, y)


def test_batch_graph_follows_new_beta(snapmod):
    cfgs = [inputs.bcc(nc, disp=0.1, seed=60 + k) for k, nc in enumerate([3, 2, 4])]
    pos = torch.tensor(np.concatenate([c.pos for c in cfgs]), device="cuda:0")
    natoms = np.array([c.natoms for c in cfgs])
    boxes = np.array([c.box for c in cfgs])
    s = snapmod.Snap(8, inputs.beta(8, seed=1), precision=1)
    for _ in range(2):
        s.compute_batch(pos, natoms, boxes, use_graph=True)
    s.set_beta(inputs.beta(8, seed=2))
    Eg, Fg, _ = [x.cpu().numpy().copy() for x in s.compute_batch(pos, natoms, boxes, use_graph=True)]
    En, Fn, _ = [x.cpu().numpy().copy() for x in s.compute_batch(pos, natoms, boxes, use_graph=False)]
    s.close()
    assert np.array_equal(Eg, En) and np.array_equal(Fg, Fn)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_entry_replay(snapmod, pinned):
    """snap_compute_host with pinned buffers (captured) and pageable ones
    (never captured): same bits as the device entry point."""
    cfg = inputs.bcc(3, disp=0.1, seed=54)
    s = snapmod.Snap(8, inputs.beta(8), precision=1)
    n = cfg.natoms
    if pinned:
        alloc = lambda shape: torch.empty(shape, dtype=torch.float64).pin_memory().numpy()
    else:
        alloc = lambda shape: np.empty(shape)
    pos = alloc((n, 3))
    pos[:] = cfg.pos
    out = (alloc((n,)), alloc((n, 3)), alloc((6,)))
    got = []
    for _ in range(4):
        s.compute_host(pos, cfg.box, out=out)
        got.append([x.copy() for x in out])
    want = run(s, cfg, 1)[0]
    s.close()
    for g in got:
        for x, y in zip(g, want):
            assert np.array_equal(x, y)
