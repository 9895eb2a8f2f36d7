"""GPU parity of the differentiation form (one-electron limit of the orbital
step, Sec. 3.2; operators of Sec. 3.1): afem_tdse_forward / _jvp / _vjp
against the oracle's dense propagator, Frechet derivatives and adjoint on a
small hanging-node mesh, plus properties that hold at any size (central
differences, the dot-product identity, checkpoint-interval invariance) and
the autograd Function on a spline-parametrised harmonic-yield objective."""
import numpy as np
import pytest

from oracle import adjoint as oadj, fem, mesh as omesh
from paper_2301_02387_gb300 import inputs
from tests._match import assert_close, coord_permutation

pytestmark = pytest.mark.gpu

CASE = (-6.0, 6.0, 3, 2, [((0.5, 0.5, 0.7), 1.0, 1), ((0.5, 0.5, -0.7), 1.0, 1)], 0.5)
CASE_P3 = (-6.0, 6.0, 3, 3, [((0.3, -0.45, 0.7), 1.0, 1), ((-0.2, 0.4, -0.7), 1.0, 1)], 0.5)
E_DIR = (0.0, 0.0, 1.0)


def _setup(case, e_dir=E_DIR):
    import torch
    import paper_2301_02387_gb300 as pkg
    gm = pkg.Mesh(*case)
    om = omesh.Mesh(*case)
    op = fem.Operators(om)
    X, _, _ = gm.tables()
    perm = coord_permutation(X, om.Xm)
    phi = inputs.lowdin(inputs.molecular_orbitals(om.Xm, ~om.boundary, case[4], 1), op.ML)[:, 0]
    td = oadj.TDSE(op, e_dir=e_dir)
    phi_g = torch.from_numpy(np.ascontiguousarray(phi[perm])).cuda()
    return gm, td, td.restrict(phi), phi_g, perm, om


def _fields(K, seed, amp=0.05):
    return amp * np.random.default_rng(seed).standard_normal(K)


@pytest.mark.parametrize("case,e_dir", [(CASE, E_DIR), (CASE_P3, (0.6, 0.0, 0.8))])
@pytest.mark.parametrize("tol,dt", [(0.0, 0.01), (1e-12, 0.1)])
def test_forward_vjp_jvp_match_oracle(case, e_dir, tol, dt):
    """FP64 bar 1e-10 relative, against dense expm / expm_frechet."""
    from paper_2301_02387_gb300 import adjoint as adj
    gm, td, phi0, phi_g, perm, om = _setup(case, e_dir)
    K, every = 7, 3          # two full checkpoint segments and a ragged one
    E = _fields(K, 11)
    rng = np.random.default_rng(12)
    g = rng.standard_normal(K + 1)
    v = rng.standard_normal(K)
    d_ref, _ = td.forward(phi0, E, dt)
    grad_ref, lam_ref = td.vjp(phi0, E, dt, g)
    _, dd_ref = td.jvp(phi0, E, dt, v)
    d, _, ckpt = adj.tdse_forward(gm, phi_g, E, dt, e_dir, krylov_m=16, tol=tol, ckpt_every=every)
    assert np.max(np.abs(d - d_ref)) <= 1e-10 * np.max(np.abs(d_ref))
    grad, lam0 = adj.tdse_vjp(gm, ckpt, every, E, g, dt, e_dir, krylov_m=16, tol=tol, want_lam0=True)
    assert np.max(np.abs(grad - grad_ref)) <= 1e-10 * np.max(np.abs(grad_ref))
    lam_full = np.zeros(om.N, dtype=np.complex128)
    lam_full[td.I] = lam_ref
    lam_g = lam0.cpu().numpy()
    assert_close(lam_g, lam_full[perm], 1e-10, what="adjoint state")
    dj, dd = adj.tdse_jvp(gm, phi_g, E, v, dt, e_dir, krylov_m=16, tol=tol)
    assert np.max(np.abs(dj - d_ref)) <= 1e-10 * np.max(np.abs(d_ref))
    assert np.max(np.abs(dd - dd_ref)) <= 1e-10 * np.max(np.abs(dd_ref))


def test_checkpoint_interval_invariance_and_edges():
    """The gradient does not depend on the checkpoint interval beyond rounding
    (segments are recomputed; the cell passes add by atomics, so in any
    order); K = 1 and an interval larger than K work."""
    from paper_2301_02387_gb300 import adjoint as adj
    gm, td, phi0, phi_g, perm, om = _setup(CASE)
    K, dt = 9, 0.02
    E = _fields(K, 21)
    g = np.random.default_rng(22).standard_normal(K + 1)
    grads = []
    for every in (1, 4, 9, 50):
        d, _, ckpt = adj.tdse_forward(gm, phi_g, E, dt, E_DIR, ckpt_every=every)
        assert ckpt.shape[0] == adj.n_checkpoints(K, every)
        grads.append(adj.tdse_vjp(gm, ckpt, every, E, g, dt, E_DIR)[0])
    for gr in grads[1:]:
        assert np.max(np.abs(gr - grads[0])) <= 1e-12 * np.max(np.abs(grads[0]))
    d1, _, ck1 = adj.tdse_forward(gm, phi_g, E[:1], dt, E_DIR, ckpt_every=50)
    g1, _ = adj.tdse_vjp(gm, ck1, 50, E[:1], g[:2], dt, E_DIR)
    r1, _ = td.vjp(phi0, E[:1], dt, g[:2])
    assert abs(g1[0] - r1[0]) <= 1e-10 * abs(r1[0])
    d0, end, _ = adj.tdse_forward(gm, phi_g, np.zeros(0), dt, E_DIR, want_end=True)
    assert d0.shape == (1,) and abs(d0[0] - td.dipole(phi0)) <= 1e-12 * max(1.0, abs(td.dipole(phi0)))
    np.testing.assert_array_equal(end.cpu().numpy(), phi_g.cpu().numpy())


def test_dot_product_identity_gpu():
    """<J v, g> = <v, J^T g> between the GPU tangent and adjoint to 1e-10."""
    from paper_2301_02387_gb300 import adjoint as adj
    gm, td, phi0, phi_g, perm, om = _setup(CASE)
    K, dt = 12, 0.01
    E = _fields(K, 31)
    rng = np.random.default_rng(32)
    v = rng.standard_normal(K)
    g = rng.standard_normal(K + 1)
    _, dd = adj.tdse_jvp(gm, phi_g, E, v, dt, E_DIR)
    _, _, ckpt = adj.tdse_forward(gm, phi_g, E, dt, E_DIR, ckpt_every=5)
    grad, _ = adj.tdse_vjp(gm, ckpt, 5, E, g, dt, E_DIR)
    lhs, rhs = g @ dd, v @ grad
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs))


def test_autograd_harmonic_yield_vs_central_differences():
    """dJ/dc of J = harmonic yield of the dipole acceleration for a field given
    by 16 cubic-spline samples c (on this small mesh the band is harmonics
    2..6 of omega0 = 0.35, which holds FFT bins of the 128-step signal):
    torch.autograd through the hand-written adjoint against central
    differences (h = 1e-6) on 8 seeded samples, <= 1e-5 relative."""
    import torch
    from paper_2301_02387_gb300 import adjoint as adj
    gm, td, phi0, phi_g, perm, om = _setup(CASE)
    K, dt, n_c = 128, 0.05, 16
    omega0 = 0.35
    S = torch.from_numpy(adj.spline_matrix(n_c, K))
    c0 = torch.from_numpy(0.05 * np.sin(np.linspace(0.0, 3.0 * np.pi, n_c)))

    def J(c):
        d = adj.dipole_signal(S @ c, gm, phi_g, dt, E_DIR, krylov_m=16, tol=0.0, ckpt_every=10)
        return adj.harmonic_yield(d, dt, omega0, 2, 6)

    c = c0.clone().requires_grad_(True)
    val = J(c)
    val.backward()
    grad = c.grad.numpy()
    idx = np.random.default_rng(41).choice(n_c, 8, replace=False)
    h = 1e-6
    for j in idx:
        cp, cm = c0.clone(), c0.clone()
        cp[j] += h
        cm[j] -= h
        fd = (J(cp).item() - J(cm).item()) / (2 * h)
        assert abs(grad[j] - fd) <= 1e-5 * np.max(np.abs(grad)), (j, grad[j], fd)


def test_mixed_precision_gradient_close_to_fp64():
    """The FP32-operator form of the same adjoint: gradient within 1e-4
    relative (complex64 cell passes; FP64 Krylov arithmetic)."""
    from paper_2301_02387_gb300 import PREC_MIXED
    from paper_2301_02387_gb300 import adjoint as adj
    gm, td, phi0, phi_g, perm, om = _setup(CASE)
    K, dt = 8, 0.02
    E = _fields(K, 51)
    g = np.random.default_rng(52).standard_normal(K + 1)
    grad_ref, _ = td.vjp(phi0, E, dt, g)
    _, _, ckpt = adj.tdse_forward(gm, phi_g, E, dt, E_DIR, ckpt_every=4, precision=PREC_MIXED)
    grad, _ = adj.tdse_vjp(gm, ckpt, 4, E, g, dt, E_DIR, precision=PREC_MIXED)
    assert np.max(np.abs(grad - grad_ref)) <= 1e-4 * np.max(np.abs(grad_ref))


def test_full_size_dot_product_and_checkpoints():
    """On the benchmark mesh (H2, Q4, N = 775,009): a few short steps with one
    fixed-dimension Krylov step each (dt = 2e-4, m = 16, accurate to rounding
    at this mesh's stiffness): the dot-product identity between tangent and
    adjoint to 1e-10, the tangent's signal equal to the forward's, and the
    gradient independent of the checkpoint interval.  (Central differences
    need a window long enough for the field to move the dipole well above its
    rounding; they run on the small meshes above.)"""
    import torch
    import paper_2301_02387_gb300 as pkg
    from paper_2301_02387_gb300 import adjoint as adj
    w = inputs.WORKLOADS["h2_q4"]
    gm = pkg.Mesh(*inputs.mesh_args("h2_q4"))
    X, ml, _ = gm.tables()
    interior = np.arange(gm.N) < gm.n_interior
    phi = inputs.lowdin(inputs.molecular_orbitals(X, interior, w["nuclei"], 1, phase_noise=0.0), ml)[:, 0]
    phi_g = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
    K, dt = 4, 2e-4
    E = np.array([0.05, -0.04, 0.06, 0.02])
    rng = np.random.default_rng(61)
    g = rng.standard_normal(K + 1)
    v = rng.standard_normal(K)
    d, _, ckpt = adj.tdse_forward(gm, phi_g, E, dt, E_DIR, krylov_m=16, tol=0.0, ckpt_every=3)
    grad, _ = adj.tdse_vjp(gm, ckpt, 3, E, g, dt, E_DIR, krylov_m=16, tol=0.0)
    dj, dd = adj.tdse_jvp(gm, phi_g, E, v, dt, E_DIR, krylov_m=16, tol=0.0)
    assert np.max(np.abs(dj - d)) <= 1e-10 * np.max(np.abs(d))
    lhs, rhs = g @ dd, v @ grad
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs))
    _, _, ck1 = adj.tdse_forward(gm, phi_g, E, dt, E_DIR, krylov_m=16, tol=0.0, ckpt_every=1)
    grad1, _ = adj.tdse_vjp(gm, ck1, 1, E, g, dt, E_DIR, krylov_m=16, tol=0.0)
    assert np.max(np.abs(grad1 - grad)) <= 1e-12 * np.max(np.abs(grad))


@pytest.mark.parametrize("tol,dt", [(0.0, 0.01), (1e-12, 0.1)])
def test_force_observable_matches_oracle(tol, dt):
    """The signal <phi_k, M_L^-1 F[e.f] phi_k>_M (f = -grad V, the potential
    part of the Ehrenfest acceleration), its adjoint and tangent against the
    oracle, 1e-10 relative; oblique field direction."""
    from oracle import adjoint as oadj2
    from paper_2301_02387_gb300 import adjoint as adj
    e_dir = (0.3, -0.4, 0.866)
    gm, td, phi0, phi_g, perm, om = _setup(CASE, e_dir)
    tdf = oadj2.TDSE(td.ops, e_dir=e_dir, observable="force")
    K, every = 6, 4
    E = _fields(K, 71)
    rng = np.random.default_rng(72)
    g = rng.standard_normal(K + 1)
    v = rng.standard_normal(K)
    d_ref, _ = tdf.forward(phi0, E, dt)
    grad_ref, _ = tdf.vjp(phi0, E, dt, g)
    _, dd_ref = tdf.jvp(phi0, E, dt, v)
    kw = dict(krylov_m=16, tol=tol, observable="force")
    d, _, ckpt = adj.tdse_forward(gm, phi_g, E, dt, e_dir, ckpt_every=every, **kw)
    assert np.max(np.abs(d - d_ref)) <= 1e-10 * np.max(np.abs(d_ref))
    grad, _ = adj.tdse_vjp(gm, ckpt, every, E, g, dt, e_dir, **kw)
    assert np.max(np.abs(grad - grad_ref)) <= 1e-10 * np.max(np.abs(grad_ref))
    _, dd = adj.tdse_jvp(gm, phi_g, E, v, dt, e_dir, **kw)
    assert np.max(np.abs(dd - dd_ref)) <= 1e-10 * np.max(np.abs(dd_ref))


def test_autograd_ehrenfest_yield_vs_central_differences():
    """J = harmonic yield of the Ehrenfest acceleration a_k = <f.e>_k - E(t_k)
    (the force signal from the hand-written adjoint, the explicit field term
    and the spline by torch) against central differences (h = 1e-6) on 6
    seeded spline samples, <= 1e-5 relative."""
    import torch
    from paper_2301_02387_gb300 import adjoint as adj
    gm, td, phi0, phi_g, perm, om = _setup(CASE)
    K, dt, n_c = 128, 0.05, 16
    S = torch.from_numpy(adj.spline_matrix(n_c, K + 1))   # field at the K + 1 signal times
    c0 = torch.from_numpy(0.05 * np.cos(np.linspace(0.0, 2.5 * np.pi, n_c)))

    def J(c):
        Es = S @ c
        f = adj.dipole_signal(Es[:K], gm, phi_g, dt, E_DIR, krylov_m=16, tol=0.0, ckpt_every=16,
                              observable="force")
        a = adj.ehrenfest_acceleration(f, Es, E_DIR)
        return adj.harmonic_yield(None, dt, 0.35, 2, 6, acceleration=a)

    c = c0.clone().requires_grad_(True)
    J(c).backward()
    grad = c.grad.numpy()
    h = 1e-6
    for j in np.random.default_rng(81).choice(n_c, 6, replace=False):
        cp, cm = c0.clone(), c0.clone()
        cp[j] += h
        cm[j] -= h
        fd = (J(cp).item() - J(cm).item()) / (2 * h)
        assert abs(grad[j] - fd) <= 1e-5 * np.max(np.abs(grad)), (j, grad[j], fd)
