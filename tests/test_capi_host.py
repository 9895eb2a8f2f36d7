"""CPU checks of the C ABI library: it loads, exports every declared symbol,
and its host mesh builder agrees exactly with the oracle's mesh."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import mesh as omesh
from tests._match import coord_permutation

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.filterwarnings("ignore")


def _lib():
    from paper_2301_02387_gb300 import _capi
    if not os.path.exists(_capi.LIB_PATH):
        from paper_2301_02387_gb300 import build
        build.build(verbose=False)
    return _capi.load()


def test_every_declared_symbol_is_exported():
    lib = _lib()
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        txt = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(afem_\w+)\s*\(", txt, re.M))
    assert len(names) >= 6
    from paper_2301_02387_gb300 import _capi
    for n in sorted(names):
        assert hasattr(lib, n), n
        assert n in _capi.SIGNATURES, n


CASES = [
    (-10.0, 10.0, 4, 2, [((0.0, 0.0, 0.0), 1.0, 3)], 2.0),
    (-8.0, 8.0, 4, 3, [((0.3, -0.45, 0.7), 1.0, 2), ((-1.1, 0.2, -0.35), 2.0, 3)], 1.5),
    (-8.0, 8.0, 3, 4, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0),
    (-6.0, 6.0, 2, 1, [((0.5, 0.5, 0.5), 8.0, 3)], 1.0),
]


@pytest.mark.parametrize("case", CASES)
def test_host_mesh_matches_oracle(case):
    from paper_2301_02387_gb300 import Mesh
    lo, hi, nc, p, nuclei, c = case
    lib_mesh = Mesh(lo, hi, nc, p, nuclei, c, host_only=True)
    om = omesh.Mesh(lo, hi, nc, p, nuclei, c)
    X, ml, cells = lib_mesh.tables()
    # identical leaf sets (integer work: bit-exact)
    assert sorted(map(tuple, cells.tolist())) == [tuple(t) for t in om.leaf_tuples()]
    assert lib_mesh.N == om.N and lib_mesh.n_hanging == om.n_hanging
    assert lib_mesh.n_interior == int((~om.boundary).sum())
    assert lib_mesh.n_constraint_entries == om.C.nnz - om.N
    perm = coord_permutation(X, om.Xm)
    # interior-first numbering
    assert not om.boundary[perm[:lib_mesh.n_interior]].any()
    assert om.boundary[perm[lib_mesh.n_interior:]].all()
    from oracle import fem
    op = fem.Operators(om)
    np.testing.assert_allclose(ml, op.ML[perm], rtol=1e-12)


def test_host_mesh_matches_oracle_benchmark_size():
    """The host mesh builder on the H2 Q4 benchmark mesh itself (12,144 cells,
    775,009 masters, 55,200 hanging points): the same leaves, counts, numbering
    and lumped mass as the oracle (whose lumped mass comes from its row-wise
    operators, without global assembly)."""
    from paper_2301_02387_gb300 import Mesh, inputs
    from oracle import rows
    args = inputs.mesh_args("h2_q4")
    lib_mesh = Mesh(*args, host_only=True)
    om = omesh.Mesh(*args)
    X, ml, cells = lib_mesh.tables()
    assert (lib_mesh.N, lib_mesh.n_hanging, len(cells)) == (775009, 55200, 12144)
    assert sorted(map(tuple, cells.tolist())) == [tuple(t) for t in om.leaf_tuples()]
    assert lib_mesh.N == om.N and lib_mesh.n_hanging == om.n_hanging
    assert lib_mesh.n_interior == int((~om.boundary).sum())
    assert lib_mesh.n_constraint_entries == om.C.nnz - om.N
    perm = coord_permutation(X, om.Xm)
    assert not om.boundary[perm[:lib_mesh.n_interior]].any()
    assert om.boundary[perm[lib_mesh.n_interior:]].all()
    np.testing.assert_allclose(ml, rows.RowOperators(om).ML[perm], rtol=1e-12)


def test_bad_descriptions_are_rejected():
    from paper_2301_02387_gb300 import Mesh, AfemError
    with pytest.raises(AfemError):
        Mesh(-1.0, 1.0, 2, 5, [], 2.0, host_only=True)
    with pytest.raises(AfemError):
        Mesh(1.0, -1.0, 2, 2, [], 2.0, host_only=True)
    with pytest.raises(AfemError):
        Mesh(-1.0, 1.0, 0, 2, [], 2.0, host_only=True)


def test_profile_classes_host_side():
    """Kernel-class timing bookkeeping: an unknown class is rejected, a class
    with nothing recorded reads as zero (no device work involved)."""
    import paper_2301_02387_gb300 as pkg
    with pytest.raises(pkg.AfemError):
        pkg.profile_read(pkg.PROF_COUNT)
    with pytest.raises(pkg.AfemError):
        pkg.profile_read(-1)
    pkg.profile_enable(False)
    for c in range(pkg.PROF_COUNT):
        assert pkg.profile_read(c, reset=True) == (0.0, 0, 0.0)


def test_batch_create_rejects_bad_inputs_host_side():
    """afem_batch_create refuses an empty batch and host-only meshes before
    touching a device."""
    import ctypes
    from paper_2301_02387_gb300 import _capi, Mesh
    lib = _capi.load()
    h = ctypes.c_void_p()
    assert lib.afem_batch_create(None, 0, ctypes.byref(h)) == _capi.AFEM_EINVAL
    m = Mesh(-2.0, 2.0, 1, 2, [], 2.0, host_only=True)
    arr = (ctypes.c_void_p * 1)(m.handle)
    assert lib.afem_batch_create(arr, 1, ctypes.byref(h)) == _capi.AFEM_EINVAL and not h.value


def test_new_entry_points_reject_bad_inputs_host_side():
    """The integrals entry, the batch stepper and the G-pass staging option
    check their arguments before touching a device (host-only mesh, null
    pointers, out-of-range values)."""
    import ctypes
    from paper_2301_02387_gb300 import _capi, Mesh, OPT_GCELL_BLOCKS
    lib = _capi.load()
    m = Mesh(-2.0, 2.0, 1, 2, [], 2.0, host_only=True)
    dummy = ctypes.c_void_p(16)
    assert lib.afem_two_electron_integrals(None, dummy, 2, dummy, dummy, 0, None) == _capi.AFEM_EINVAL
    assert lib.afem_two_electron_integrals(m.handle, dummy, 2, dummy, dummy, 0, None) == _capi.AFEM_EINVAL
    assert lib.afem_two_electron_integrals(m.handle, dummy, 2, dummy, dummy, 5, None) == _capi.AFEM_EINVAL
    assert b"precision" in lib.afem_last_error()
    h = ctypes.c_void_p()
    assert lib.afem_batch_stepper_create(None, 0, ctypes.byref(h)) == _capi.AFEM_EINVAL and not h.value
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.afem_batch_stepper_create(arr, 1, None) == _capi.AFEM_EINVAL
    assert lib.afem_batch_stepper_step(None, None, None, None, None, 0.01, 1e-10, 10, None, None) == _capi.AFEM_EINVAL
    assert lib.afem_batch_stepper_tuning(None, None, None, None, None) == _capi.AFEM_EINVAL
    assert lib.afem_mesh_set_option(m.handle, OPT_GCELL_BLOCKS, 3) == _capi.AFEM_EINVAL
    assert lib.afem_mesh_set_option(m.handle, OPT_GCELL_BLOCKS, 0) == _capi.AFEM_OK


def test_tdse_entry_points_reject_bad_inputs_host_side():
    """afem_tdse_* refuse host-only meshes, negative step counts, non-positive
    dt, bad Krylov dimensions and missing checkpoints before any device work."""
    from paper_2301_02387_gb300 import _capi, Mesh
    lib = _capi.load()
    m = Mesh(-2.0, 2.0, 1, 2, [], 2.0, host_only=True)
    e = (ctypes.c_double * 3)(0.0, 0.0, 1.0)
    E = (ctypes.c_double * 2)(0.01, 0.02)
    d = (ctypes.c_double * 3)()
    g = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    x = ctypes.c_void_p(16)   # never dereferenced: every call below fails its checks first
    pos = _capi.OP_POS
    assert lib.afem_tdse_forward(m.handle, e, E, 2, 0.1, 8, 0.0, 0, pos, x, None, d, None, 0,
                                 None) == _capi.AFEM_EINVAL
    assert b"host-only" in lib.afem_last_error()
    assert lib.afem_tdse_forward(m.handle, e, E, 2, 0.1, 8, 0.0, 0, _capi.OP_H1, x, None, d, None, 0,
                                 None) == _capi.AFEM_EINVAL
    assert b"observable" in lib.afem_last_error()
    m2 = Mesh(-2.0, 2.0, 1, 2, [], 2.0, host_only=True)
    for args, why in [((2, -0.1, 8, 0.0, 0), b"dt"), ((2, 0.1, 0, 0.0, 0), b"krylov_m"),
                      ((2, 0.1, 17, 0.0, 0), b"krylov_m"), ((2, 0.1, 8, -1.0, 0), b"tol"),
                      ((2, 0.1, 8, 0.0, 5), b"precision"), ((-1, 0.1, 8, 0.0, 0), b"n_steps")]:
        K, dt, mk, tol, prec = args
        assert lib.afem_tdse_forward(m2.handle, e, E, K, dt, mk, tol, prec, pos, x, None, d, None, 0,
                                     None) == _capi.AFEM_EINVAL
        assert why in lib.afem_last_error(), (args, lib.afem_last_error())
    assert lib.afem_tdse_vjp(m2.handle, e, E, 0, 0.1, 8, 0.0, 0, pos, x, 1, g, d, None, None) == _capi.AFEM_EINVAL
    assert lib.afem_tdse_vjp(m2.handle, e, E, 2, 0.1, 8, 0.0, 0, pos, None, 1, g, d, None,
                             None) == _capi.AFEM_EINVAL
    assert lib.afem_tdse_jvp(None, e, E, 2, 0.1, 8, 0.0, 0, pos, x, E, d, d, None) == _capi.AFEM_EINVAL


def test_spline_and_harmonic_yield_helpers():
    """The cubic-spline field map reproduces linear fields exactly and
    interpolates its samples; the harmonic yield equals the band sum of the
    squared FFT of the second-difference acceleration."""
    import torch
    from paper_2301_02387_gb300 import adjoint as adj
    S = adj.spline_matrix(9, 33)
    assert S.shape == (33, 9)
    t = np.linspace(0.0, 1.0, 9)
    x = np.linspace(0.0, 1.0, 33)
    np.testing.assert_allclose(S @ (2.0 - 3.0 * t), 2.0 - 3.0 * x, atol=1e-13)
    # not-a-knot: a single cubic through the samples is reproduced exactly
    np.testing.assert_allclose(S @ (t ** 3 - t), x ** 3 - x, atol=1e-13)
    np.testing.assert_allclose(S[::4], np.eye(9), atol=1e-13)
    assert adj.n_checkpoints(100, 50) == 2 and adj.n_checkpoints(101, 50) == 3 and adj.n_checkpoints(1, 50) == 1
    rng = np.random.default_rng(0)
    d = rng.standard_normal(64)
    dt, w0 = 0.1, 0.4
    a = np.diff(d, 2) / dt ** 2
    A = np.fft.rfft(a)
    w = 2 * np.pi * np.arange(len(A)) / (len(a) * dt)
    band = (w >= 3 * w0) & (w <= 9 * w0)
    assert band.sum() >= 2
    ref = np.sum(np.abs(A[band]) ** 2)
    got = adj.harmonic_yield(torch.from_numpy(d), dt, w0, 3, 9).item()
    assert abs(got - ref) <= 1e-12 * ref


@pytest.mark.parametrize("case,kelly", [
    ((-8.0, 8.0, 4, 2, [((0.0, 0.0, 0.7), 1.0, 5), ((0.0, 0.0, -0.7), 1.0, 5)], 2.0), (0.3, 4)),
    ((-6.0, 6.0, 3, 3, [((0.3, -0.2, 0.1), 3.0, 5)], 2.0), (0.5, 3)),
    ((-8.0, 8.0, 2, 4, [((0.0, 0.0, 0.0), 8.0, 5), ((1.43, 1.1, 0.0), 1.0, 5), ((-1.43, 1.1, 0.0), 1.0, 5)], 2.0),
     (1.0, 4)),
])
def test_host_kelly_mesh_matches_oracle(case, kelly):
    """Kelly refinement (Sec. 3.1) on the host builder and in the oracle: the
    same leaves, masters and hanging points (threshold decisions in FP64 on
    both sides; a tie at the threshold would show here)."""
    from paper_2301_02387_gb300 import Mesh
    lib_mesh = Mesh(*case, host_only=True, kelly=kelly)
    om = omesh.Mesh(*case, kelly=kelly)
    X, ml, cells = lib_mesh.tables()
    assert sorted(map(tuple, cells.tolist())) == [tuple(t) for t in om.leaf_tuples()]
    assert lib_mesh.N == om.N and lib_mesh.n_hanging == om.n_hanging
