"""GPU tests of the cooperative smoothing-phase launch (mg_params.smooth_phase): a whole pre- or
post-smoothing phase of a small level in one launch with grid barriers between the red-black
half sweeps.  Each node's arithmetic and the order of the half sweeps are those of the
one-launch-per-half-sweep path, so every result must be the same bit for bit; that path is
itself checked against the FP64 CPU oracle in test_gpu_parity.py."""
import numpy as np
import pytest

import workloads as W
from oracle import discretization as disc
from oracle.grid import Grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0811_4446_gb300 import build, mg as mgmod
    build.build()
    return mgmod


def _rhs(d, dt):
    g = Grid(d.nr, d.nz, d.R, d.z)
    phys = disc.Physics(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p,
                        D_p=d.D_p, table=d.table, pressure_factor=d.pressure_factor)
    u = np.stack([d.ne0, d.np0, d.V0])
    F = disc.residual(g, u, u * 0.99, d.S_e, d.S_p, dt, phys)
    return u, F


@pytest.mark.parametrize("n,precision", [(64, "fp64"), (128, "fp64"), (128, "mixed")])
def test_phase_linear_solve_equals_half_sweep_launches(mg, n, precision):
    d = W.make_discharge(n, seed=3, V_cathode=-300.0, use_table=True)
    dt = 1e-8
    u, F = _rhs(d, dt)
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    out = []
    for phase in (0, n):
        s = mg.from_discharge(d, precision=prec, smooth_phase=phase)
        s.set_old_state(*[np.ascontiguousarray(a * 0.99) for a in u])
        x, h, rc = s.linear_solve(dt, list(-F), 1e-10, 100)
        assert rc == mg.MG_OK
        out.append((np.stack(x), np.asarray(h)))
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_phase_steady_257_equals_default(mg, precision):
    """The benchmark's workload (257^2 steady solve, two-level continuation): same steps,
    Newton iterations, V-cycles and state."""
    d = W.steady_257()
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    res = []
    for phase in (0, 128):
        s = mg.from_discharge(d, precision=prec, smooth_phase=phase)
        rc, st = s.solve_steady(1e-8)
        assert rc == mg.MG_OK
        res.append((np.stack(s.get_state()), st))
    (u0, s0), (u1, s1) = res
    for k in ("steps_accepted", "steps_rejected", "newton_iterations", "vcycles"):
        assert s0[k] == s1[k], k
    assert np.array_equal(u0, u1)


def test_phase_batched_concurrent_streams(mg):
    """Cooperative launches of several solves on concurrent streams (the batched form): every
    result equals its solve without the phase launches."""
    ds = W.batch_64()
    pick, seen = [], set()
    for d in ds:
        if d.nr not in seen and d.nr <= 256:
            seen.add(d.nr)
            pick.append(d)
    states = []
    for phase in (0, 128):
        solvers = [mg.from_discharge(d, precision=mg.MG_MIXED, smooth_phase=phase, stream=torch.cuda.Stream())
                   for d in pick]
        rc, _, rcs = mg.solve_steady_batch(solvers, 1e-8, workers=3)
        assert rc == mg.MG_OK, rcs
        states.append([np.stack(sv.get_state()) for sv in solvers])
    for a, b in zip(*states):
        assert np.array_equal(a, b)
