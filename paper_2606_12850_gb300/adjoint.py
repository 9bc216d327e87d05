"""Seismograms as a differentiable function of the material (rho, kappa, mu per local point).

When the displacement of every step fits in device memory (by default: in half of what is
free), the forward pass keeps all of them and the backward pass runs the discrete adjoint of
the explicit scheme over the whole run in one call, with no recomputation. Otherwise the
forward pass keeps a checkpoint of the complete state every ``checkpoint_every`` steps, and
the backward pass walks the checkpoints in reverse, recomputes the displacements of one
segment from its checkpoint and runs the adjoint backward through it (see
``sem_adjoint_begin`` in include/sem.h). All arithmetic runs in the CUDA library; this
module only orders the calls and holds the device buffers (PyTorch tensors).
"""
from __future__ import annotations

import numpy as np
import torch

from . import sem


class Simulation:
    """One model, one shot: forward seismograms and their material gradients.

    ``ctx`` is a context with its mesh, sources and receivers set; ``dt`` the time step. The
    material is given per call as float tensors/arrays [nspec][ngll^3] (rho, kappa, mu).
    The simulation sets the context's SEM_OPT_NODE_ORDER to the internal order.
    """

    def __init__(self, ctx: sem.Ctx, dt: float, nsteps: int, checkpoint_every: int = 50, device: int = 0,
                 keep_all="auto"):
        """keep_all: True keeps every step's displacement from the forward run (no
        recomputation in the backward run), False checkpoints, "auto" keeps all when they
        take at most half of the free device memory."""
        if ctx.shots != 1:
            raise ValueError("one shot per simulation")
        self.keep_all = keep_all
        self.snapshots = None  # [nsteps + 1][nglob*3] when every displacement is kept
        self.ctx = ctx
        self.dt = float(dt)
        self.nsteps = int(nsteps)
        self.every = max(1, int(checkpoint_every))
        self.device = torch.device("cuda", device)
        self.nglob = self.ctx.nglob
        self.nrec = self.ctx.nrec
        self.checkpoints = []  # (step, u, v, a) device tensors [nglob*3], solver node order
        # checkpoints and snapshots only travel between library calls: keep them in the
        # solver's internal node order (no permutation on every copy)
        sem.sem_set_option(self.ctx, sem.SEM_OPT_NODE_ORDER, 1)

    def _state(self):
        n3 = 3 * self.nglob
        u, v, a = (torch.empty(n3, device=self.device) for _ in range(3))
        sem.sem_sync(self.ctx)
        torch.cuda.synchronize(self.device)
        sem.sem_get_state_dev(self.ctx, u, v, a)
        sem.sem_sync(self.ctx)
        return u, v, a

    def set_material(self, rho, kappa, mu):
        mats = (rho, kappa, mu)
        if all(torch.is_tensor(x) and x.is_cuda for x in mats):
            mats = [x.detach().to(self.device, torch.float32).contiguous() for x in mats]
            torch.cuda.synchronize(self.device)
            sem.sem_set_moduli_dev(self.ctx, *mats)
        else:
            to_np = lambda x: x.detach().cpu().numpy() if torch.is_tensor(x) else np.asarray(x)  # noqa: E731
            sem.sem_set_moduli(self.ctx, *(to_np(x) for x in mats))
        sem.sem_set_dt(self.ctx, self.dt)

    def keeps_all(self) -> bool:
        if self.keep_all == "auto":
            need = (self.nsteps + 1) * 3 * self.nglob * 4
            free, _ = torch.cuda.mem_get_info(self.device)
            return need <= free // 2
        return bool(self.keep_all)

    def forward(self, rho, kappa, mu) -> torch.Tensor:
        """Seismograms [nrec][3][nsteps] (s^1 .. s^N) on the device."""
        self.set_material(rho, kappa, mu)
        sem.sem_set_state(self.ctx)
        N = self.nsteps
        seis = torch.empty((self.nrec, 3, N), device=self.device)
        self.checkpoints = []
        self.snapshots = None
        if self.keeps_all():
            U = torch.empty((N + 1, 3 * self.nglob), device=self.device)
            U[0].copy_(self._state()[0])
            torch.cuda.synchronize(self.device)
            sem.sem_run_record_snapshots(self.ctx, N, seis, U[1:])
            sem.sem_sync(self.ctx)
            self.snapshots = U
            return seis
        n = 0
        while n < N:
            self.checkpoints.append((n,) + self._state())
            k = min(self.every, N - n)
            chunk = torch.empty((self.nrec, 3, k), device=self.device)
            sem.sem_run_dev(self.ctx, k, chunk)
            sem.sem_sync(self.ctx)
            seis[:, :, n:n + k] = chunk
            n += k
        return seis

    def _segment_displacements(self, n0: int, n1: int) -> torch.Tensor:
        """u^{n0} .. u^{n1} recomputed from the checkpoint at n0: [n1 - n0 + 1][nglob*3]."""
        _, u0, v0, a0 = next(c for c in self.checkpoints if c[0] == n0)
        out = torch.empty((n1 - n0 + 1, 3 * self.nglob), device=self.device)
        out[0].copy_(u0)
        torch.cuda.synchronize(self.device)
        sem.sem_set_state_dev(self.ctx, u0, v0, a0)
        sem.sem_set_step(self.ctx, n0)
        sem.sem_run_snapshots(self.ctx, n1 - n0, out[1:])
        return out

    def gradient(self, G: torch.Tensor):
        """dL/d(rho, kappa, mu) for dL/ds = G [nrec][3][nsteps]; float64 numpy [nspec][ngll^3]."""
        N = self.nsteps
        # Gt[m - 1] = G^m as a contiguous [nrec][3] block
        Gt = G.detach().to(self.device, torch.float32).permute(2, 0, 1).contiguous()
        torch.cuda.synchronize(self.device)
        sem.sem_adjoint_begin(self.ctx)
        if self.snapshots is not None:  # the terms n = 1 .. N - 1 read u^0 .. u^N
            if N > 1:
                sem.sem_adjoint_segment(self.ctx, N - 1, Gt[1:N], self.snapshots)
            sem.sem_sync(self.ctx)
            return sem.sem_adjoint_gradients(self.ctx)
        for n0 in reversed([c[0] for c in self.checkpoints]):
            # the terms n = n0 + 1 .. n0 + count, which read u^{n0} .. u^{n0 + count + 1}
            count = min(self.every, N - 1 - n0)
            if count <= 0:
                continue
            U = self._segment_displacements(n0, n0 + count + 1)
            sem.sem_adjoint_segment(self.ctx, count, Gt[n0 + 1:n0 + count + 1], U)
            sem.sem_sync(self.ctx)  # U is released (or reused) after this
        return sem.sem_adjoint_gradients(self.ctx)


class Seismograms(torch.autograd.Function):
    """seis = Seismograms.apply(rho, kappa, mu, simulation): differentiable in the three
    per-point material tensors (gradients through the discrete adjoint)."""

    @staticmethod
    def forward(ctx, rho, kappa, mu, sim: Simulation):
        ctx.sim = sim
        ctx.device = rho.device
        return sim.forward(rho, kappa, mu)

    @staticmethod
    def backward(ctx, grad_seis):
        g_rho, g_kappa, g_mu = ctx.sim.gradient(grad_seis)
        as_t = lambda g: torch.from_numpy(g.astype(np.float32)).to(ctx.device)  # noqa: E731
        return as_t(g_rho), as_t(g_kappa), as_t(g_mu), None
