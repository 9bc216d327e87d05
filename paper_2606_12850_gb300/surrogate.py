"""Binding of the learned seismogram surrogate (include/surrogate.h) and the host code
around it: training data from solver runs, the training loop and the solver fallback.

Every arithmetic step of the network (forward, backward, loss, Adam) runs in libsemgb's
CUDA kernels; the training data come from the spectral-element solver (moment-tensor
sources, many shots per launch). This module marshals arguments, draws the seeded random
numbers the method uses (initial weights, minibatch order) and orders the calls.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import inputs, sem

_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
SG_OPT_PRODUCT = 1  # product kernel: 1 tcgen05 (default), 0 warp mma.sync
SG_OPT_STALL_TEST = 2  # tests only: tcgen05 products wait until their limit runs out

# name: (restype, argtypes) for every symbol declared in include/surrogate.h
SIGNATURES = {
    "sg_create": (_I, [_P, _I, _P, _I, _I, _I, _I, _I, _P, _P, _I, _I]),
    "sg_destroy": (_I, [_P]),
    "sg_info": (_I, [_P, _P]),
    "sg_set_params": (_I, [_P, _P]),
    "sg_get_params": (_I, [_P, _P]),
    "sg_forward": (_I, [_P, _I, _P, _P]),
    "sg_loss_grad": (_I, [_P, _I, _P, _P, _P]),
    "sg_get_grads": (_I, [_P, _P]),
    "sg_adam_step": (_I, [_P, _F, _F, _F, _F]),
    "sg_sync": (_I, [_P]),
    "sg_set_option": (_I, [_P, _I, _I]),
    "sg_get_option": (_I, [_P, _I, _P]),
    "sg_last_error": (ctypes.c_char_p, [_P]),
}

_bound = False


def lib() -> ctypes.CDLL:
    global _bound
    handle = sem.lib()
    if not _bound:
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _bound = True
    return handle


def _check(code: int, where: str, model=None):
    if code != 0:
        msg = lib().sg_last_error(model.handle if model is not None else None)
        raise sem.SemError(code, where, (msg or b"").decode(errors="replace"))


@dataclass
class Spec:
    """Network sizes. The default is the surrogate of the 16^3 layered medium: 9 inputs
    (position, six moment-tensor entries), two hidden layers of 512, a [64][125] seed, three
    x2 upsampling stages to 1000 time samples, and a last stage of 6 x 192 channels that the
    six moment entries combine into 64 receivers x 3 components (seismograms are linear in
    the moment tensor)."""

    in_dim: int = 9
    hidden: int = 512
    c0: int = 64
    l0: int = 125
    stage_cout: tuple = (96, 96, 96, 6 * 192)
    stage_up: tuple = (2, 2, 2, 1)
    contract: int = 6

    @property
    def out_c(self) -> int:
        return self.stage_cout[-1] // self.contract if self.contract else self.stage_cout[-1]

    @property
    def out_l(self) -> int:
        return self.l0 * int(np.prod(self.stage_up))

    def shapes(self) -> list:
        """(name, shape) of every parameter tensor in the library's order."""
        out = [("W1", (self.hidden, self.in_dim)), ("b1", (self.hidden,)),
               ("W2", (self.hidden, self.hidden)), ("b2", (self.hidden,)),
               ("W3", (self.c0 * self.l0, self.hidden)), ("b3", (self.c0 * self.l0,))]
        cin = self.c0
        for s, co in enumerate(self.stage_cout):
            out += [(f"C{s}", (co, cin, 3)), (f"c{s}", (co,))]
            cin = co
        return out

    def split(self, flat) -> dict:
        out, o = {}, 0
        for name, shape in self.shapes():
            n = int(np.prod(shape))
            out[name] = np.asarray(flat[o:o + n]).reshape(shape)
            o += n
        return out

    def init_params(self, seed: int) -> np.ndarray:
        """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, seeded; float32."""
        parts = []
        for i, (name, shape) in enumerate(self.shapes()):
            if name[0] in "bc":
                parts.append(np.zeros(int(np.prod(shape))))
            else:
                fan_in = int(np.prod(shape[1:]))
                bound = np.sqrt(6.0 / fan_in)
                parts.append(inputs.uniform(seed, (int(np.prod(shape)),), -bound, bound, stream=40 + i))
        return np.concatenate(parts).astype(np.float32)


class Model:
    """A network on one GPU (see include/surrogate.h)."""

    def __init__(self, spec: Spec, max_batch: int = 256, device: int = 0, stream=None):
        self.spec = spec
        out = _P()
        co = np.asarray(spec.stage_cout, dtype=np.int32)
        up = np.asarray(spec.stage_up, dtype=np.int32)
        s = None if stream is None else _P(stream if isinstance(stream, int) else stream.cuda_stream)
        _check(lib().sg_create(ctypes.byref(out), device, s, spec.in_dim, spec.hidden, spec.c0, spec.l0, len(co),
                               co.ctypes.data_as(_P), up.ctypes.data_as(_P), int(spec.contract), int(max_batch)),
               "sg_create")
        self.handle = out.value
        self.device = int(device)
        self.max_batch = int(max_batch)
        info = self.info()
        self.nparams = info["params"]

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib().sg_destroy(self.handle)
            except Exception:
                pass
            self.handle = None

    def info(self) -> dict:
        out = np.zeros(4, dtype=np.int64)
        _check(lib().sg_info(self.handle, out.ctypes.data_as(_P)), "sg_info", self)
        return dict(zip(("params", "out_c", "out_l", "device_bytes"), (int(v) for v in out)))

    def set_params(self, flat):
        arr = np.ascontiguousarray(flat, dtype=np.float32)
        if arr.size != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters, got {arr.size}")
        _check(lib().sg_set_params(self.handle, arr.ctypes.data_as(_P)), "sg_set_params", self)

    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        _check(lib().sg_get_params(self.handle, out.ctypes.data_as(_P)), "sg_get_params", self)
        return out

    def get_grads(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        _check(lib().sg_get_grads(self.handle, out.ctypes.data_as(_P)), "sg_get_grads", self)
        return out

    def forward(self, x_dev, y_dev):
        b = x_dev.shape[0]
        _check(lib().sg_forward(self.handle, b, sem._dev(x_dev, b * self.spec.in_dim, self),
                                sem._dev(y_dev, b * self.spec.out_c * self.spec.out_l, self)), "sg_forward", self)

    def loss_grad(self, x_dev, t_dev) -> float:
        b = x_dev.shape[0]
        loss = ctypes.c_double(0.0)
        _check(lib().sg_loss_grad(self.handle, b, sem._dev(x_dev, b * self.spec.in_dim, self),
                                  sem._dev(t_dev, b * self.spec.out_c * self.spec.out_l, self), ctypes.byref(loss)),
               "sg_loss_grad", self)
        return loss.value

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        _check(lib().sg_adam_step(self.handle, float(lr), float(beta1), float(beta2), float(eps)), "sg_adam_step",
               self)

    def sync(self):
        _check(lib().sg_sync(self.handle), "sg_sync", self)

    @property
    def product(self) -> int:
        """Product kernel: 1 = tcgen05 with TMEM accumulators (default), 0 = warp mma.sync."""
        out = ctypes.c_int(0)
        _check(lib().sg_get_option(self.handle, SG_OPT_PRODUCT, ctypes.byref(out)), "sg_get_option", self)
        return out.value

    @product.setter
    def product(self, kind: int):
        _check(lib().sg_set_option(self.handle, SG_OPT_PRODUCT, int(kind)), "sg_set_option", self)

    def set_option(self, option: int, value: int):
        _check(lib().sg_set_option(self.handle, int(option), int(value)), "sg_set_option", self)


# ---- training data, training, fallback ---------------------------------------------------------

def features(xyz, moments, side: float) -> np.ndarray:
    """Network inputs: the source position scaled to [-1, 1]^3 and the unit-norm moment
    tensor (Mxx, Myy, Mzz, Mxy, Mxz, Myz); float32 [n][9]."""
    xyz = np.atleast_2d(xyz)
    return np.concatenate([2.0 * xyz / side - 1.0, np.atleast_2d(moments)], axis=1).astype(np.float32)


class AmplitudeModel:
    """Expected trace size of a source, fitted to training runs: log rms(traces) ~ a
    cubic in the scaled depth plus a multiple of log max(r, r0), r the distance to the
    nearest receiver (the layers' impedance contrast and geometric spreading). Dividing the
    targets by it gives runs of comparable size, so that the unweighted mean squared error
    treats deep and shallow sources alike; predictions are multiplied back."""

    def __init__(self, side: float, rec_xyz, coef=None, r0: float = 200.0):
        self.side = float(side)
        self.rec_xyz = np.asarray(rec_xyz, dtype=np.float64)
        self.coef = None if coef is None else np.asarray(coef, dtype=np.float64)
        self.r0 = float(r0)

    def design(self, xyz) -> np.ndarray:
        xyz = np.atleast_2d(xyz)
        z = 2.0 * xyz[:, 2] / self.side - 1.0
        r = np.sqrt(((xyz[:, None, :] - self.rec_xyz[None, :, :]) ** 2).sum(-1)).min(axis=1)
        return np.stack([np.ones_like(z), z, z * z, z ** 3, np.log(np.maximum(r, self.r0))], axis=1)

    def fit(self, xyz, rms) -> "AmplitudeModel":
        self.coef, *_ = np.linalg.lstsq(self.design(xyz), np.log(np.asarray(rms, dtype=np.float64)), rcond=None)
        return self

    def __call__(self, xyz) -> np.ndarray:
        return np.exp(self.design(xyz) @ self.coef)


@dataclass
class Runs:
    """Solver runs for the surrogate: features [n][9] (host), traces [n][3 nrec][nsteps]
    (device, float32), and what produced them."""

    x: np.ndarray
    y: object
    node: np.ndarray
    xyz: np.ndarray
    moments: np.ndarray
    seconds: float = 0.0
    info: dict = field(default_factory=dict)


class Solver:
    """The spectral-element solver set up for the surrogate's medium, many shots per launch
    (moment-tensor sources at the nodes nearest the requested positions)."""

    def __init__(self, workload, shots: int = 32, device: int = 0, stream=None, moment_scale: float = 1e16):
        import torch
        self.w = workload
        self.shots = int(shots)
        self.scale = float(moment_scale)
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        self.setup = sem.setup_workload(workload, device=device, stream=self.stream)
        self.ctx = self.setup.ctx
        sem.sem_set_shots(self.ctx, self.shots)
        sem.sem_set_receiver_nodes(self.ctx, self.setup.rec_nodes)
        self.nrec = len(self.setup.rec_nodes)
        self.rec_xyz = sem.sem_node_xyz(self.ctx, self.setup.rec_nodes)

    def amplitude_model(self) -> AmplitudeModel:
        return AmplitudeModel(self.w.mesh.lengths[0], self.rec_xyz)

    def run(self, xyz, moments, out=None):
        """Traces [n][3 nrec][nsteps] (device) of the sources (positions snapped to nodes)."""
        import torch
        xyz = np.atleast_2d(xyz)
        n = len(xyz)
        nodes = sem.sem_locate_nodes(self.ctx, xyz)
        K = self.w.nsteps
        dev = torch.device("cuda", self.device)
        if out is None:
            out = torch.empty((n, 3 * self.nrec, K), device=dev)
        with torch.cuda.stream(self.stream):
            buf = torch.empty((self.shots, self.nrec, 3, K), device=dev)
        for b0 in range(0, n, self.shots):
            b = min(self.shots, n - b0)
            sem.sem_set_shot_moment_sources(self.ctx, np.arange(b), nodes[b0:b0 + b],
                                            self.scale * np.atleast_2d(moments)[b0:b0 + b], self.w.f0, self.w.t0)
            sem.sem_set_state(self.ctx)
            sem.sem_run_dev(self.ctx, K, buf)
            sem.sem_sync(self.ctx)
            out[b0:b0 + b] = buf[:b].reshape(b, 3 * self.nrec, K)
        torch.cuda.synchronize(dev)
        return out, nodes

    def snapped(self, xyz):
        nodes = sem.sem_locate_nodes(self.ctx, np.atleast_2d(xyz))
        return nodes, sem.sem_node_xyz(self.ctx, nodes)


def generate_runs(solver: Solver, count: int, seed: int) -> Runs:
    """``count`` solver runs with seeded random sources; features use the snapped positions."""
    import time

    import torch
    side = solver.w.mesh.lengths[0]
    pos, mom = inputs.surrogate_sources(count, side, seed)
    nodes, xyz = solver.snapped(pos)
    torch.cuda.synchronize()
    t = time.perf_counter()
    y, _ = solver.run(xyz, mom)
    secs = time.perf_counter() - t
    return Runs(features(xyz, mom, side), y, nodes, xyz, mom, secs)


def train(model: Model, x, y_scaled, epochs: int, batch: int, lr: float, seed: int, lr_final: float | None = None,
          log=None) -> list:
    """Minibatch Adam on (x [n][9] device, y_scaled [n][C][L] device) with a seeded
    permutation per epoch and a cosine learning-rate decay to ``lr_final``; returns the mean
    loss per epoch."""
    import torch
    n = x.shape[0]
    lr_final = lr * 0.02 if lr_final is None else lr_final
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    losses = []
    k = 0
    for ep in range(epochs):
        perm = np.argsort(inputs.uniform(seed, (n,), stream=1000 + ep))
        idx = torch.from_numpy(perm.astype(np.int64)).to(x.device)
        acc = 0.0
        for s in range(steps_per_epoch):
            sel = idx[s * batch:(s + 1) * batch]
            xb = x.index_select(0, sel).contiguous()
            yb = y_scaled.index_select(0, sel).contiguous()
            torch.cuda.synchronize()
            acc += model.loss_grad(xb, yb)
            cur = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * k / max(1, total - 1)))
            model.adam_step(cur)
            k += 1
        losses.append(acc / steps_per_epoch)
        if log:
            log(ep, losses[-1])
    model.sync()
    return losses


def nearest_run_baseline(train: Runs, test: Runs):
    """The answer without a network: for every test source, the traces of the training run
    whose features (scaled position and unit moment tensor) lie nearest. Device tensor."""
    import torch
    d = ((test.x[:, None, :].astype(np.float64) - train.x[None, :, :]) ** 2).sum(-1)
    idx = torch.from_numpy(d.argmin(axis=1).astype(np.int64)).to(train.y.device)
    return train.y.index_select(0, idx)


def rel_l2_per_run(pred, ref) -> np.ndarray:
    """Relative L2 error of every run (over its receivers, components and samples)."""
    d = (pred - ref).reshape(pred.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    return (d.norm(dim=1) / r.norm(dim=1)).double().cpu().numpy()


def training_targets(y, amplitude, scale: float):
    """Network targets from solver traces: y / amplitude(source) * scale (device)."""
    import torch
    a = torch.from_numpy(np.asarray(amplitude, dtype=np.float32)).to(y.device)
    return (y / a[:, None, None] * scale).contiguous()


def run_rms(y) -> np.ndarray:
    """RMS of every run's traces, float64 [n]."""
    return y.double().pow(2).mean(dim=(1, 2)).sqrt().cpu().numpy()


class Surrogate:
    """A trained network with the scaling of its targets (a global scale and the fitted
    per-source amplitude), and the solver as fallback."""

    def __init__(self, model: Model, target_scale: float, side: float, amplitude: AmplitudeModel,
                 solver: Solver | None = None):
        self.model = model
        self.scale = float(target_scale)
        self.side = float(side)
        self.amplitude = amplitude
        self.solver = solver

    def predict(self, xyz, moments):
        """Traces [n][C][L] on the device for sources at (snapped) positions xyz."""
        import torch
        x = torch.from_numpy(features(xyz, moments, self.side)).cuda()
        y = torch.empty((x.shape[0], self.model.spec.out_c, self.model.spec.out_l), device=x.device)
        torch.cuda.synchronize()
        self.model.forward(x, y)
        self.model.sync()
        a = torch.from_numpy(self.amplitude(xyz).astype(np.float32)).to(y.device)
        return y * (a[:, None, None] / self.scale)

    def predict_or_solve(self, xyz, moments, tol: float, check: int = 4, seed: int = 0):
        """The surrogate's traces if the solver, run on ``check`` of the sources chosen at
        random, finds them within ``tol`` (relative L2 per run); else the solver's traces for
        all sources. Acceptance is a sample check: the sources not among the ``check`` may
        miss ``tol``. Returns (traces, used_solver, checked errors)."""
        if self.solver is None:
            raise ValueError("predict_or_solve needs a solver to check against (Surrogate(..., solver))")
        xyz = np.atleast_2d(xyz)
        pred = self.predict(xyz, moments)
        pick = np.argsort(inputs.uniform(seed, (len(xyz),), stream=77))[:min(check, len(xyz))]
        ref, _ = self.solver.run(xyz[pick], np.atleast_2d(moments)[pick])
        errs = rel_l2_per_run(pred[pick], ref)
        if np.all(errs <= tol):
            return pred, False, errs
        full, _ = self.solver.run(xyz, moments)
        return full, True, errs
