"""The compiled FP64 CPU baseline (oracle/sem_cpu.c) against the numpy oracle: the same
forces and the same time steps to rounding, whatever the thread count (its colour-by-colour
order is fixed). CPU only."""
import numpy as np
import pytest

from oracle import sem_cpu, sem_oracle
from paper_2606_12850_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("ngll", [2, 4, 5, 7])
def test_cpu_forces_match_numpy_oracle(ngll):
    mesh = inputs.structured_hex_mesh((3, 3, 2), ngll, (900.0, 800.0, 700.0), jitter=0.15, seed=ngll)
    shape = mesh.ibool.shape
    rho = inputs.uniform(1, shape, 2000.0, 3000.0)
    vp = inputs.uniform(2, shape, 3000.0, 5000.0)
    m = sem_oracle.Model(mesh.ibool, mesh.ctrl, mesh.nglob, rho, vp, vp / 1.8, ngll)
    u = inputs.random_field(mesh.nglob, 5).astype(np.float64)
    f_ref = m.forces(u)
    for threads in (1, 3):
        f = sem_cpu.CpuBaseline(m, threads).forces(u)
        assert rel(f, f_ref) <= 1e-13


def test_cpu_run_matches_numpy_oracle_and_threads_agree():
    w = inputs.homogeneous_cube(n=4, ngll=5, nsteps=30)
    m = sem_oracle.build_model(w)
    dt = m.cfl_dt(w.courant)
    src, rec = sem_oracle.locate_workload(m, w)
    _, u_ref, v_ref, _ = sem_oracle.newmark_run(m, dt, 30, src_nodes=src, src_force=w.source_force, f0=w.f0,
                                                t0=w.t0, rec_nodes=rec)
    outs = []
    for threads in (1, 4):
        u, v, _ = sem_cpu.CpuBaseline(m, threads).run(dt, 30, src_node=int(src[0]), src_force=w.source_force[0],
                                                      f0=w.f0, t0=w.t0)
        assert rel(u, u_ref) <= 1e-12 and rel(v, v_ref) <= 1e-12
        outs.append(u)
    assert np.array_equal(outs[0], outs[1])
