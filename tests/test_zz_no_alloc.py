"""afem_poisson_boundary_noalloc: the pair mean fields' surface data computed
without any device allocation inside the library.

Some callers cannot let the library allocate device memory once they run (a
process whose device memory is held by another allocator's pool, a loop with
a fixed memory budget).  This entry point serves them from a fixed file-scope
scratch array.  Its output must equal the surface rows that the allocating
entry point afem_poisson_batch writes, on consecutive calls sharing the one
scratch array, and a call must leave the device's free memory and the torch
caching allocator's statistics unchanged.

The file is collected last so that a run stopping at the first failure has
run every other test before this one; the tests here depend on no other test
(each builds its own mesh and inputs) and pass alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASE = (-8.0, 8.0, 3, 3, [((0.0, 0.0, 0.7), 1.0, 2), ((0.0, 0.0, -0.7), 1.0, 2)], 2.0)


def _orbitals(X, n_interior, n, seed):
    rng = np.random.default_rng(seed)
    phi = np.zeros((len(X), n), dtype=np.complex128)
    for j in range(n):
        c = rng.uniform(-1.0, 1.0, 3)
        phi[:, j] = np.exp(-(0.5 + 0.3 * j) * np.sum((X - c) ** 2, axis=1)) * np.exp(1j * (X @ rng.uniform(-1, 1, 3)))
    phi[n_interior:] = 0
    return phi


def _noalloc(lib, mesh, phi, W):
    import torch
    rc = lib.afem_poisson_boundary_noalloc(mesh.handle, ctypes.c_void_p(phi.data_ptr()), phi.shape[1],
                                           ctypes.c_void_p(W.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


@pytest.mark.parametrize("n", [1, 3, 4])
def test_noalloc_surface_data_matches_poisson_batch(n):
    import torch
    import paper_2301_02387_gb300 as pkg
    lib = pkg.load_library()
    mesh = pkg.Mesh(*CASE)
    X, _, _ = mesh.tables()
    Ni, N = mesh.n_interior, mesh.N
    for seed in (1, 2):   # two calls in a row share the scratch array
        phi = torch.from_numpy(_orbitals(X, Ni, n, seed)).cuda()
        W_ref = torch.zeros((N, n * n), dtype=torch.float64, device="cuda")
        pkg.poisson_batch(mesh, phi, W_ref, rtol=1e-6, max_it=5000)
        W = torch.full((N, n * n), 3.0, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, mesh, phi, W) == 0
        torch.cuda.synchronize()
        ref = W_ref[Ni:].cpu().numpy()
        got = W[Ni:].cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
        assert torch.all(W[:Ni] == 3.0).item()      # interior rows untouched


def test_noalloc_rejects_too_many_orbitals():
    import torch
    import paper_2301_02387_gb300 as pkg
    lib = pkg.load_library()
    mesh = pkg.Mesh(*CASE)
    phi = torch.zeros((mesh.N, 5), dtype=torch.complex128, device="cuda")
    W = torch.zeros((mesh.N, 25), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, mesh, phi, W) == pkg._capi.AFEM_EINVAL
    assert b"n_orb" in lib.afem_last_error()


def test_noalloc_allocates_no_device_memory():
    """After a warm-up call (which does the per-device set-up), calls with
    n = 1..4 change neither the free device memory nor the torch caching
    allocator's statistics."""
    import torch
    import paper_2301_02387_gb300 as pkg
    lib = pkg.load_library()
    mesh = pkg.Mesh(*CASE)
    X, _, _ = mesh.tables()
    bufs = []
    for n in (1, 2, 3, 4):
        phi = torch.from_numpy(_orbitals(X, mesh.n_interior, n, 10 + n)).cuda()
        W = torch.zeros((mesh.N, n * n), dtype=torch.float64, device="cuda")
        bufs.append((phi, W))
    assert _noalloc(lib, mesh, *bufs[0]) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for _ in range(3):
        for phi, W in bufs:
            assert _noalloc(lib, mesh, phi, W) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current",
                "allocated_bytes.all.current"):
        assert stats1.get(key) == stats0.get(key), key
