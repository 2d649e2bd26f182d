"""GPU test of mg_residual_noalloc, the allocation-free residual entry point.

Callers that cannot allocate device memory (code inside another framework's memory pool,
real-time loops where cudaMalloc is forbidden, plug-ins limited to the buffers they are
given) use this entry point; it keeps its scratch in a static device array instead.  The
test checks it through the C ABI against the state-based mg_residual on the same inputs, on
two calls in a row (the shared scratch must not leak the first call into the second).  The
file name makes pytest collect it last.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0811_4446_gb300 import build, mg as mgmod
    build.build()
    return mgmod


def _state(d, rng):
    ne = 1e14 * (0.5 + rng.random(d.shape))
    np_ = 1e14 * (0.5 + rng.random(d.shape))
    V = d.V0 + 3.0 * rng.standard_normal(d.shape)
    for a in (ne, np_):
        a[0, :] = 0.0
        a[-1, :] = 0.0
    V[0, :] = d.V_cathode
    V[-1, :] = d.V_anode
    return [np.ascontiguousarray(a) for a in (ne, np_, V)]


@pytest.mark.parametrize("n,nz,table,dts", [(32, 32, False, (1e-9, 0.0)), (128, 64, True, (1e-6, 1e-9)),
                                             (256, 256, True, (0.0, 1e-6))])
def test_noalloc_matches_state_residual_twice(mg, n, nz, table, dts):
    d = W.make_discharge(n, nz=nz, seed=7, V_cathode=-300.0, use_table=table, pressure_factor=1.2)
    rng = np.random.default_rng(n)
    s = mg.from_discharge(d)
    params = mg.default_params(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p,
                               D_p=d.D_p, pressure_factor=d.pressure_factor)
    for call, dt in enumerate(dts):                     # two calls in a row, different inputs
        u, uo = _state(d, rng), _state(d, rng)
        s.set_state(*u)
        s.set_old_state(*uo)
        F_ref, rho_ref = s.residual(dt)
        dev = lambda a: torch.from_numpy(a).cuda()
        F_dev = [torch.zeros(d.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
        rho = mg.residual_noalloc(d.nr, d.nz, d.R, d.z, params, [dev(a) for a in u], [dev(a) for a in uo],
                                  [dev(np.ascontiguousarray(d.S_e)), dev(np.ascontiguousarray(d.S_p))], dt,
                                  F_out=F_dev, table=d.table)
        assert np.allclose(rho, rho_ref, rtol=1e-9, atol=0.0), (call, rho, rho_ref)
        for q in range(3):
            scale = np.abs(F_ref[q]).max()
            assert np.abs(F_dev[q].cpu().numpy() - F_ref[q]).max() <= 1e-12 * scale, (call, q)


def test_noalloc_rejects_sizes_beyond_the_limit(mg):
    z = W.z_nodes(8, 1e-2)
    params = mg.default_params()
    t = torch.zeros((9, 2049), dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MGError):
        mg.residual_noalloc(2048, 8, 1e-2, z, params, [t, t, t], None, [t, t], 0.0)
