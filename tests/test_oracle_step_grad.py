"""Pins of the dense differentiable MCTDHF step (`oracle/step_grad.py`), the
oracle of the differentiation form beyond the one-electron limit: its step
equals the numpy oracle's step (`mctdhf.MCTDHF.step`, Sec. 2 and Sec. 3.2:
the same orbitals, CI vector and dipole signal), and its gradient of
J = sum_k g_k d_k with respect to the field amplitudes equals central
differences of its own forward map (h = 1e-3 and the Richardson combination
of h = 1e-3 and 2e-3: the signal is smooth in E, so the truncation error is
far below the bar while rounding stays small)."""
import numpy as np
import pytest
import torch

from oracle import fem, mctdhf, mesh as omesh, step_grad
from paper_2301_02387_gb300 import inputs

CASE = (-6.0, 6.0, 2, 2, [((0.0, 0.0, 0.7), 1.0, 1), ((0.0, 0.0, -0.7), 1.0, 1)], 2.0)


@pytest.fixture(scope="module", params=[(2, 1, 1), (3, 2, 1)], ids=["n2", "n3"])
def system(request):
    n, na, nb = request.param
    om = omesh.Mesh(*CASE)
    op = fem.Operators(om)
    sim = mctdhf.MCTDHF(op, n, na, nb)
    dm = step_grad.DenseMCTDHF(sim, e_dir=(0.3, -0.4, 0.866))
    phi = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, CASE[4], n), op.ML)
    C = inputs.initial_ci(n, na, nb, amp=0.1)
    return sim, dm, phi, C


def test_dense_step_equals_oracle_step(system):
    sim, dm, phi, C = system
    dt, Ea = 0.01, 0.03
    e = np.array([0.3, -0.4, 0.866])
    phi_n, C_n, info = sim.step(phi, C, tuple(Ea * e), dt, 12)
    p1, c1 = dm.step(dm.restrict(phi), torch.from_numpy(C), torch.tensor(Ea, dtype=torch.float64), dt)
    # the oracle's Krylov step reaches the exact exponential within its estimate
    assert np.linalg.norm(p1.numpy() - phi_n[dm.I]) <= 10.0 * info["arnoldi_err"] + 1e-11 * np.linalg.norm(phi_n)
    assert np.linalg.norm(c1.numpy() - C_n) <= 1e-12 * np.linalg.norm(C_n)
    d = float(dm.signal(dm.restrict(phi), torch.from_numpy(C)))
    assert abs(d - float(info["dipole"] @ e)) <= 1e-12 * max(1.0, abs(d))


def test_gradient_matches_central_differences(system):
    sim, dm, phi, C = system
    K, dt = (3 if sim.n == 2 else 2), 0.01
    rng = np.random.default_rng(7)
    E = 0.02 * rng.standard_normal(K)
    g = rng.standard_normal(K + 1)
    p0, c0 = dm.restrict(phi), torch.from_numpy(C)
    J, grad = dm.gradient(p0, c0, E, dt, g)

    def Jof(Ev):
        with torch.no_grad():
            return float(torch.sum(torch.from_numpy(g) * dm.signals(p0, c0, torch.from_numpy(Ev), dt)))

    assert abs(J - Jof(E)) <= 1e-14 * max(1.0, abs(J))

    def cd(h):
        out = np.zeros(K)
        for k in range(K):
            Ep, Em = E.copy(), E.copy()
            Ep[k] += h
            Em[k] -= h
            out[k] = (Jof(Ep) - Jof(Em)) / (2 * h)
        return out

    c1, c2 = cd(1e-3), cd(2e-3)
    scale = np.abs(c1).max()
    assert np.abs(grad - c1).max() <= 1e-6 * scale
    assert np.abs(grad - (4.0 * c1 - c2) / 3.0).max() <= 1e-6 * scale


def test_tangent_dot_product_and_differences(system):
    """The tangent map against the gradient (<g, J v> = <J^T g, v> to 1e-10)
    and against central differences along v (1e-6)."""
    sim, dm, phi, C = system
    K, dt = (2 if sim.n == 2 else 1), 0.01
    rng = np.random.default_rng(9)
    E = 0.02 * rng.standard_normal(K)
    g = rng.standard_normal(K + 1)
    v = rng.standard_normal(K)
    p0, c0 = dm.restrict(phi), torch.from_numpy(C)
    d, dd = dm.tangent(p0, c0, E, dt, v)
    _, grad = dm.gradient(p0, c0, E, dt, g)
    assert dd[0] == 0.0
    assert abs(g @ dd - v @ grad) <= 1e-10 * max(abs(g @ dd), abs(v @ grad))
    with torch.no_grad():
        sp = dm.signals(p0, c0, torch.from_numpy(E + 1e-3 * v), dt).numpy()
        sm = dm.signals(p0, c0, torch.from_numpy(E - 1e-3 * v), dt).numpy()
    np.testing.assert_allclose(d, dm.signals(p0, c0, torch.from_numpy(E), dt).detach().numpy(), rtol=0, atol=1e-14)
    assert np.abs(dd - (sp - sm) / 2e-3).max() <= 1e-6 * np.abs(dd).max()
