"""Host logic of the checkpointed adjoint (``adjoint.Simulation``), on the CPU with the
library calls replaced by a recorder: the forward pass checkpoints every ``checkpoint_every``
steps and records s^1 .. s^N in order; the backward pass visits the adjoint steps
m = N .. 2 exactly once, in decreasing order, each with G^m and the displacements
u^{m-2}, u^{m-1}, u^m (the pairing that sem_adjoint_segment documents), recomputed from the
right checkpoint with the step counter restored."""
import numpy as np
import pytest
import torch

from paper_2606_12850_gb300 import adjoint


class FakeLibrary:
    """Stands for the sem_* calls adjoint.py makes; the 'state' is just the step number n,
    written into every array the library would fill."""

    def __init__(self):
        self.n = 0
        self.visits = []  # (m, G value, (u indices)) per adjoint step, in call order

    def sem_sync(self, ctx):
        pass

    def sem_set_moduli(self, ctx, *a):
        pass

    def sem_set_dt(self, ctx, dt):
        pass

    def sem_set_state(self, ctx, *a):
        self.n = 0

    def sem_get_state_dev(self, ctx, u, v, a):
        for t in (u, v, a):
            t.fill_(self.n)

    def sem_run_dev(self, ctx, k, chunk):
        for j in range(k):
            chunk[:, :, j] = self.n + 1 + j  # s^{n+1+j}
        self.n += k

    def sem_set_state_dev(self, ctx, u, v, a):
        self.n = int(u[0].item())

    def sem_set_step(self, ctx, step):
        assert step == self.n, "step counter differs from the restored checkpoint"

    def sem_run_snapshots(self, ctx, k, out):
        for j in range(k):
            out[j].fill_(self.n + 1 + j)
        self.n += k

    def sem_run_record_snapshots(self, ctx, k, seis, out):
        for j in range(k):
            seis[:, :, j] = self.n + 1 + j
            out[j].fill_(self.n + 1 + j)
        self.n += k

    def sem_adjoint_begin(self, ctx):
        self.visits = []

    def sem_adjoint_segment(self, ctx, count, G, U):
        n0 = int(U[0, 0].item())
        for j in range(count, 0, -1):
            self.visits.append((n0 + j + 1, float(G[j - 1, 0, 0]),
                                (int(U[j - 1, 0]), int(U[j, 0]), int(U[j + 1, 0]))))

    def sem_adjoint_gradients(self, ctx):
        return (np.zeros(1),) * 3


def _run(monkeypatch, nsteps, every, keep_all=False):
    fake = FakeLibrary()
    for name in dir(fake):
        if name.startswith("sem_"):
            monkeypatch.setattr(adjoint.sem, name, getattr(fake, name))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)

    class Ctx:
        shots, nglob, nrec = 1, 4, 2

    sim = adjoint.Simulation.__new__(adjoint.Simulation)  # the initialiser wants a CUDA device
    sim.ctx, sim.dt, sim.nsteps, sim.every = Ctx(), 1e-3, nsteps, every
    sim.device, sim.nglob, sim.nrec, sim.checkpoints = torch.device("cpu"), 4, 2, []
    sim.keep_all, sim.snapshots = keep_all, None
    seis = sim.forward(np.ones(1), np.ones(1), np.ones(1))
    if keep_all:
        assert sim.checkpoints == [] and sim.snapshots.shape[0] == nsteps + 1
    else:
        assert [c[0] for c in sim.checkpoints] == list(range(0, nsteps, every))
    assert np.array_equal(seis[0, 0].numpy(), np.arange(1, nsteps + 1))
    G = torch.arange(1, nsteps + 1, dtype=torch.float32).expand(2, 3, nsteps)  # G^m = m
    sim.gradient(G)
    return seis, fake.visits


def _schedule_ok(visits, nsteps):
    return [v[0] for v in visits] == list(range(nsteps, 1, -1)) and all(
        g == m and us == (m - 2, m - 1, m) for m, g, us in visits)


@pytest.mark.parametrize("nsteps,every", [(50, 7), (60, 60), (61, 60), (10, 1), (200, 50), (3, 5)])
def test_checkpoint_schedule(monkeypatch, nsteps, every):
    _, visits = _run(monkeypatch, nsteps, every)
    assert _schedule_ok(visits, nsteps)


@pytest.mark.parametrize("nsteps", [50, 2, 1])
def test_kept_snapshots_schedule(monkeypatch, nsteps):
    """Every displacement kept from the forward run: one segment visits m = N .. 2 with G^m
    and u^{m-2}, u^{m-1}, u^m."""
    seis, visits = _run(monkeypatch, nsteps, 7, keep_all=True)
    assert np.array_equal(seis[0, 0].numpy(), np.arange(1, nsteps + 1))
    assert _schedule_ok(visits, nsteps)


@pytest.mark.parametrize("old,new", [
    ("count = min(self.every, N - 1 - n0)", "count = min(self.every, N - n0)"),
    ("Gt[n0 + 1:n0 + count + 1]", "Gt[n0:n0 + count]"),
    ("self._segment_displacements(n0, n0 + count + 1)", "self._segment_displacements(n0, n0 + count)"),
])
def test_planted_schedule_mistake_is_caught(monkeypatch, old, new):
    """An extra adjoint step, G shifted by one step, or a segment one snapshot short (in a
    copy of Simulation.gradient) breaks the schedule check."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(adjoint.Simulation.gradient))
    assert old in src
    ns = dict(adjoint.__dict__)
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    monkeypatch.setattr(adjoint.Simulation, "gradient", ns["gradient"])
    try:
        _, visits = _run(monkeypatch, 50, 7)
    except (IndexError, RuntimeError, AssertionError, ValueError):
        return
    assert not _schedule_ok(visits, 50)
