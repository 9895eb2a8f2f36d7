"""GB300 (sm_103a) library for MCTDHF on an adaptive finite-element mesh
(Orimo, Sato, Ishikawa, arXiv 2301.02387).

Thin Python binding over the C ABI of ``include/afem_mctdhf.h``: each function
here checks and marshals its arguments (torch CUDA tensors -> device
pointers, the current torch stream) and calls the entry point of the same
name.  Every step of the computation runs in the library's CUDA kernels.
"""
import ctypes

import numpy as np

from . import _capi
from ._capi import (AfemError, OP_H1, OP_STIFF, OP_STIFF_F32, OP_H1_C64, OP_POS, OP_FORCE,  # noqa: F401
                    OP_H1_VG, OP_H1_VG_C64, GAUGE_LENGTH, GAUGE_VELOCITY)

__all__ = ["Mesh", "op_apply", "AfemError", "OP_H1", "OP_STIFF", "load_library"]


def load_library():
    return _capi.load()


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, shape0=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape0 is not None and t.shape[0] != shape0:
        raise ValueError(f"{name} must have leading dimension {shape0}, got {t.shape[0]}")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """Adaptive octree mesh (Sec. 3.1) built on the host and resident on the current GPU.

    nuclei: sequence of (position (3,), charge Z, refinement levels L).
    kelly: None (the geometric rule toward the nuclei) or (threshold,
    max_level) for Kelly refinement on the nuclear Coulomb potential.
    """

    def __init__(self, lo, hi, n_coarse, degree, nuclei, refine_c=2.0, host_only=False, kelly=None):
        lib = _capi.load()
        d = _capi.MeshDesc()
        d.lo, d.hi = float(lo), float(hi)
        d.n_coarse, d.degree = int(n_coarse), int(degree)
        nuclei = list(nuclei)
        if len(nuclei) > _capi.MAX_NUCLEI:
            raise ValueError("too many nuclei")
        d.n_nuclei = len(nuclei)
        for a, (R, Z, L) in enumerate(nuclei):
            for ax in range(3):
                d.nuc_pos[a][ax] = float(R[ax])
            d.nuc_charge[a] = float(Z)
            d.nuc_levels[a] = int(L)
        d.refine_c = float(refine_c)
        if kelly is not None:
            d.refine_mode = 1
            d.kelly_threshold = float(kelly[0])
            d.kelly_max_level = int(kelly[1])
        self.desc = d
        self.nuclei = [(np.asarray(R, dtype=np.float64), float(Z), int(L)) for (R, Z, L) in nuclei]
        h = ctypes.c_void_p()
        flags = _capi.MESH_HOST_ONLY if host_only else 0
        _capi.check(lib.afem_mesh_create_ex(ctypes.byref(d), flags, ctypes.byref(h)))
        self._h = h
        info = _capi.MeshInfo()
        _capi.check(lib.afem_mesh_get_info(h, ctypes.byref(info)))
        self.n_cells = info.n_cells
        self.N = info.n_masters
        self.n_interior = info.n_interior
        self.n_hanging = info.n_hanging
        self.n_constraint_entries = info.n_constraint_entries
        self.degree = info.degree
        self.max_level = info.max_level
        self.h_min, self.h_max = info.h_min, info.h_max

    @property
    def handle(self):
        return self._h

    def tables(self):
        """(coords (N,3), lumped mass (N,), cells (n_cells,4) level,i,j,k) as numpy arrays."""
        X = np.empty((self.N, 3), dtype=np.float64)
        ml = np.empty(self.N, dtype=np.float64)
        cells = np.empty((self.n_cells, 4), dtype=np.int32)
        _capi.check(_capi.load().afem_mesh_tables(
            self._h, X.ctypes.data_as(ctypes.c_void_p), ml.ctypes.data_as(ctypes.c_void_p),
            cells.ctypes.data_as(ctypes.c_void_p)))
        return X, ml, cells

    def close(self):
        if getattr(self, "_h", None):
            _capi.load().afem_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PREC_FP64 = 0
PREC_MIXED = 1


def poisson_batch(mesh, phi, W, rtol=1e-10, max_it=20000, warm_start=False, stream=None,
                  raise_on_maxit=True, precision=PREC_FP64):
    """afem_poisson_batch(_ex): pair mean fields W ([N, n^2] float64) of orbitals phi ([N, n] complex128).

    Returns (iterations, relative residuals per column, status code); with
    precision=PREC_MIXED the iteration count is the float32 inner total.
    """
    import torch
    n = int(phi.shape[1])
    _dev_ptr(phi, torch.complex128, mesh.N, "phi")
    _dev_ptr(W, torch.float64, mesh.N, "W")
    if W.shape[1] != n * n:
        raise ValueError("W must have n_orb^2 columns")
    it = ctypes.c_int(0)
    outer = ctypes.c_int(0)
    rel = np.zeros(n * n, dtype=np.float64)
    rc = _capi.load().afem_poisson_batch_ex(
        mesh.handle, ctypes.c_void_p(phi.data_ptr()), n, ctypes.c_void_p(W.data_ptr()), float(rtol),
        int(max_it), 1 if warm_start else 0, int(precision), ctypes.byref(it), ctypes.byref(outer),
        rel.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream))
    if rc != _capi.AFEM_OK and (raise_on_maxit or rc != _capi.AFEM_ECG_MAXIT):
        _capi.check(rc)
    return it.value, rel, rc


def two_electron_integrals(mesh, phi, W, eri=None, precision=PREC_FP64, stream=None):
    """afem_two_electron_integrals: (pq|rs) as a [n^2, n^2] complex128 tensor,
    eri[p n + q, r n + s], from orbitals phi ([N, n] complex128) and their pair
    mean fields W ([N, n^2] float64, the column layout of poisson_batch)."""
    import torch
    n = int(phi.shape[1])
    _dev_ptr(phi, torch.complex128, mesh.N, "phi")
    _dev_ptr(W, torch.float64, mesh.N, "W")
    if W.shape[1] != n * n:
        raise ValueError("W must have n_orb^2 columns")
    if eri is None:
        eri = torch.empty((n * n, n * n), dtype=torch.complex128, device=phi.device)
    _dev_ptr(eri, torch.complex128, n * n, "eri")
    _capi.check(_capi.load().afem_two_electron_integrals(
        mesh.handle, ctypes.c_void_p(phi.data_ptr()), n, ctypes.c_void_p(W.data_ptr()),
        ctypes.c_void_p(eri.data_ptr()), int(precision), _stream_ptr(stream)))
    return eri


def _E3(E):
    if E is None:
        return None
    return (ctypes.c_double * 3)(*[float(e) for e in E])


def arnoldi_step(mesh, phi, U, krylov_m, dt, E=None, out=None, stream=None, precision=PREC_FP64):
    """afem_arnoldi_step: phi_out = exp(-i G dt) phi by short-iterative Arnoldi.

    phi: [N, n] complex128; U: [N, n, n] complex128 or None.  Returns
    (phi_out, err_est, m_used, breakdown).
    """
    import torch
    n = int(phi.shape[1])
    _dev_ptr(phi, torch.complex128, mesh.N, "phi")
    if U is not None:
        _dev_ptr(U, torch.complex128, mesh.N, "U")
        if tuple(U.shape[1:]) != (n, n):
            raise ValueError("U must be [N, n, n]")
    out = torch.empty_like(phi) if out is None else out
    _dev_ptr(out, torch.complex128, mesh.N, "out")
    err = ctypes.c_double(0.0)
    mu = ctypes.c_int(0)
    brk = ctypes.c_int(0)
    Earr = _E3(E)
    _capi.check(_capi.load().afem_arnoldi_step_ex(
        mesh.handle, ctypes.cast(Earr, ctypes.c_void_p) if Earr is not None else None,
        ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(U.data_ptr()) if U is not None else None,
        n, int(krylov_m), float(dt), int(precision), ctypes.c_void_p(out.data_ptr()), ctypes.byref(err),
        ctypes.byref(mu), ctypes.byref(brk), _stream_ptr(stream)))
    return out, err.value, mu.value, bool(brk.value)


def arnoldi_propagate(mesh, phi, U, krylov_m, dt, tol, E=None, out=None, stream=None, precision=PREC_FP64):
    """afem_arnoldi_propagate: exp(-i G dt) phi with Krylov error control.  Returns (phi_out, err, substeps)."""
    import torch
    n = int(phi.shape[1])
    _dev_ptr(phi, torch.complex128, mesh.N, "phi")
    if U is not None:
        _dev_ptr(U, torch.complex128, mesh.N, "U")
    out = torch.empty_like(phi) if out is None else out
    _dev_ptr(out, torch.complex128, mesh.N, "out")
    err = ctypes.c_double(0.0)
    sub = ctypes.c_int(0)
    Earr = _E3(E)
    _capi.check(_capi.load().afem_arnoldi_propagate(
        mesh.handle, ctypes.cast(Earr, ctypes.c_void_p) if Earr is not None else None,
        ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(U.data_ptr()) if U is not None else None,
        n, int(krylov_m), float(dt), int(precision), float(tol), ctypes.c_void_p(out.data_ptr()),
        ctypes.byref(err), ctypes.byref(sub), _stream_ptr(stream)))
    return out, err.value, sub.value


def arnoldi_adaptive(mesh, phi, U, m_max, dt, steps, tol, E=None, out=None, stream=None, precision=PREC_FP64):
    """afem_arnoldi_adaptive: exp(-i G dt) phi by Sec. 3.2's rule (fixed steps,
    dimension chosen by the estimate).  Returns (phi_out, err, dim_max, dim_sum, unmet)."""
    import torch
    n = int(phi.shape[1])
    _dev_ptr(phi, torch.complex128, mesh.N, "phi")
    if U is not None:
        _dev_ptr(U, torch.complex128, mesh.N, "U")
    out = torch.empty_like(phi) if out is None else out
    _dev_ptr(out, torch.complex128, mesh.N, "out")
    err = ctypes.c_double(0.0)
    dmax, dsum, unmet = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    Earr = _E3(E)
    _capi.check(_capi.load().afem_arnoldi_adaptive(
        mesh.handle, ctypes.cast(Earr, ctypes.c_void_p) if Earr is not None else None,
        ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(U.data_ptr()) if U is not None else None,
        n, int(m_max), float(dt), int(steps), int(precision), float(tol), ctypes.c_void_p(out.data_ptr()),
        ctypes.byref(err), ctypes.byref(dmax), ctypes.byref(dsum), ctypes.byref(unmet), _stream_ptr(stream)))
    return out, err.value, dmax.value, dsum.value, unmet.value


class MCTDHF:
    """afem_mctdhf_*: the MCTDHF time stepper of one mesh (Sec. 2, Sec. 3.2).

    State lives in caller tensors: phi [N, n] complex128, C [ci_dim] complex128,
    W [N, n^2] float64 (zeros before the first step).
    """

    def __init__(self, mesh, n_orb, n_alpha, n_beta, krylov_m):
        self.mesh = mesh
        self.n, self.n_alpha, self.n_beta, self.krylov_m = n_orb, n_alpha, n_beta, krylov_m
        h = ctypes.c_void_p()
        _capi.check(_capi.load().afem_mctdhf_create(mesh.handle, n_orb, n_alpha, n_beta, krylov_m,
                                                    ctypes.byref(h)))
        self._h = h
        d = ctypes.c_int64(0)
        _capi.check(_capi.load().afem_mctdhf_ci_dim(h, ctypes.byref(d)))
        self.ci_dim = d.value

    def set_krylov_tol(self, tol):
        _capi.check(_capi.load().afem_mctdhf_set_krylov_tol(self._h, float(tol)))

    def set_krylov_adaptive(self, steps):
        """Sec. 3.2's rule: `steps` equal Krylov steps per time step, dimension by the estimate (0: off)."""
        _capi.check(_capi.load().afem_mctdhf_set_krylov_adaptive(self._h, int(steps)))

    def set_gauge(self, gauge):
        """GAUGE_LENGTH (the step's E is the field) or GAUGE_VELOCITY (the step's E is A(t))."""
        _capi.check(_capi.load().afem_mctdhf_set_gauge(self._h, int(gauge)))

    def set_imaginary(self, on=True):
        """Imaginary-time steps (ground-state preparation) when on, real time otherwise."""
        _capi.check(_capi.load().afem_mctdhf_set_imaginary(self._h, 1 if on else 0))

    def set_precision(self, precision):
        _capi.check(_capi.load().afem_mctdhf_set_precision(self._h, int(precision)))

    def step(self, phi, C, W, E, dt, cg_rtol=1e-10, cg_max_it=20000, stream=None, raise_on_maxit=True):
        import torch
        _dev_ptr(phi, torch.complex128, self.mesh.N, "phi")
        _dev_ptr(C, torch.complex128, self.ci_dim, "C")
        _dev_ptr(W, torch.float64, self.mesh.N, "W")
        info = _capi.StepInfo()
        Earr = _E3(E)
        rc = _capi.load().afem_mctdhf_step(
            self._h, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(C.data_ptr()),
            ctypes.c_void_p(W.data_ptr()), ctypes.cast(Earr, ctypes.c_void_p) if Earr is not None else None,
            float(dt), float(cg_rtol), int(cg_max_it), ctypes.byref(info), _stream_ptr(stream))
        if rc != _capi.AFEM_OK and (raise_on_maxit or rc != _capi.AFEM_ECG_MAXIT):
            _capi.check(rc)
        return dict(energy=info.energy, arnoldi_err=info.arnoldi_err, cg_relres_max=info.cg_relres_max,
                    krylov_m_used=info.krylov_m_used, breakdown=bool(info.breakdown), cg_iters=info.cg_iters,
                    krylov_substeps=info.krylov_substeps, dipole=tuple(info.dipole),
                    krylov_dim_sum=info.krylov_dim_sum, krylov_unmet=info.krylov_unmet,
                    status=rc)

    def close(self):
        if getattr(self, "_h", None):
            _capi.load().afem_mctdhf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchStepper:
    """afem_batch_stepper_*: one MCTDHF step of every instance per call (the
    batching form at the level of the time step).  solvers: MCTDHF objects
    (kept alive by this object); each instance computes what its own
    MCTDHF.step computes."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        n = len(self.solvers)
        arr = (ctypes.c_void_p * n)(*[s._h.value for s in self.solvers])
        h = ctypes.c_void_p()
        _capi.check(_capi.load().afem_batch_stepper_create(ctypes.cast(arr, ctypes.c_void_p), n, ctypes.byref(h)))
        self._h = h

    def step(self, phis, Cs, Ws, Es, dt, cg_rtol=1e-10, cg_max_it=20000, stream=None, raise_on_maxit=True):
        import torch
        n = len(self.solvers)
        if not (len(phis) == len(Cs) == len(Ws) == n):
            raise ValueError("one phi, C and W per instance")
        for s, phi, C, W in zip(self.solvers, phis, Cs, Ws):
            _dev_ptr(phi, torch.complex128, s.mesh.N, "phi")
            _dev_ptr(C, torch.complex128, s.ci_dim, "C")
            _dev_ptr(W, torch.float64, s.mesh.N, "W")
        P = ctypes.c_void_p * n
        pa = P(*[t.data_ptr() for t in phis])
        ca = P(*[t.data_ptr() for t in Cs])
        wa = P(*[t.data_ptr() for t in Ws])
        Earr = None
        if Es is not None:
            flat = []
            for e in Es:
                flat.extend(float(v) for v in (e if e is not None else (0.0, 0.0, 0.0)))
            Earr = (ctypes.c_double * (3 * n))(*flat)
        infos = (_capi.StepInfo * n)()
        rc = _capi.load().afem_batch_stepper_step(
            self._h, ctypes.cast(pa, ctypes.c_void_p), ctypes.cast(ca, ctypes.c_void_p),
            ctypes.cast(wa, ctypes.c_void_p), ctypes.cast(Earr, ctypes.c_void_p) if Earr is not None else None,
            float(dt), float(cg_rtol), int(cg_max_it), ctypes.cast(infos, ctypes.c_void_p), _stream_ptr(stream))
        if rc != _capi.AFEM_OK and (raise_on_maxit or rc != _capi.AFEM_ECG_MAXIT):
            _capi.check(rc)
        return [dict(energy=i.energy, arnoldi_err=i.arnoldi_err, cg_iters=i.cg_iters,
                     krylov_substeps=i.krylov_substeps, dipole=tuple(i.dipole)) for i in infos]

    def tuning(self):
        streams, nc = ctypes.c_int(0), ctypes.c_int(0)
        cs = (ctypes.c_int * 8)()
        cm = (ctypes.c_double * 8)()
        _capi.check(_capi.load().afem_batch_stepper_tuning(self._h, ctypes.byref(streams), ctypes.byref(nc),
                                                           ctypes.cast(cs, ctypes.c_void_p),
                                                           ctypes.cast(cm, ctypes.c_void_p)))
        return {"streams": streams.value, "candidates": [(cs[i], cm[i]) for i in range(nc.value)]}

    def close(self):
        if getattr(self, "_h", None):
            _capi.load().afem_batch_stepper_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def op_apply(mesh, kind, x, y, E=None, stream=None):
    """afem_op_apply: y = op(x) for all columns of x ([N, n_vec], DoF-major).

    OP_H1: complex128, y = M_L^{-1} H1~ x (Dirichlet); OP_STIFF: float64, y = A x;
    OP_POS: complex128, y = M_L^{-1} F[e.r] x (Dirichlet) with e passed as E;
    OP_FORCE: the same with the nuclear force e.(-grad V) in place of e.r.
    """
    import torch
    dtype = {OP_H1: torch.complex128, OP_STIFF: torch.float64, OP_STIFF_F32: torch.float32,
             OP_H1_C64: torch.complex64, OP_POS: torch.complex128,
             OP_FORCE: torch.complex128, OP_H1_VG: torch.complex128,
             OP_H1_VG_C64: torch.complex64}.get(kind, x.dtype)
    xp = _dev_ptr(x, dtype, mesh.N, "x")
    yp = _dev_ptr(y, dtype, mesh.N, "y")
    if x.shape != y.shape:
        raise ValueError("x and y must have the same shape")
    nvec = 1 if x.dim() == 1 else int(x.shape[1])
    Earr = None
    if E is not None:
        Earr = (ctypes.c_double * 3)(*[float(e) for e in E])
    _capi.check(_capi.load().afem_op_apply(
        mesh.handle, int(kind), ctypes.cast(Earr, ctypes.c_void_p) if Earr is not None else None,
        xp, yp, nvec, _stream_ptr(stream)))
    return y


def convert(x, y, stream=None):
    """afem_convert: y = x rounded to float32 (x float64) or widened to float64
    (x float32) by the library's integer-pipe conversions (same shape, CUDA)."""
    import torch
    if x.dtype == torch.float64:
        direction, ydt = _capi.CONVERT_F64_F32, torch.float32
    elif x.dtype == torch.float32:
        direction, ydt = _capi.CONVERT_F32_F64, torch.float64
    else:
        raise TypeError("x must be float32 or float64")
    xp = _dev_ptr(x, x.dtype, None, "x")
    yp = _dev_ptr(y, ydt, None, "y")
    if x.numel() != y.numel():
        raise ValueError("x and y must have the same number of elements")
    _capi.check(_capi.load().afem_convert(xp, yp, int(x.numel()), direction, _stream_ptr(stream)))
    return y


PEAK_FP64 = 0
PEAK_FP32 = 1


def fma_peak(kind, target_ms=50.0, stream=None):
    """afem_fma_peak: measured FP64 (PEAK_FP64) or FP32 (PEAK_FP32) multiply-add
    throughput of the current device, flop/s."""
    out = ctypes.c_double(0.0)
    _capi.check(_capi.load().afem_fma_peak(int(kind), float(target_ms), ctypes.byref(out), _stream_ptr(stream)))
    return out.value


OPT_CELL32_VARIANT = 1
OPT_POISSON_SOLVER = 2
OPT_GCELL_BLOCKS = 3
POISSON_JACOBI = 0
POISSON_MULTIGRID = 1


def mesh_set_option(mesh, option, value):
    """afem_mesh_set_option (kernel-shape tuning)."""
    _capi.check(_capi.load().afem_mesh_set_option(mesh.handle, int(option), int(value)))


def mesh_set_ecs(mesh, theta, half_width):
    """afem_mesh_set_ecs: exterior complex scaling of the kinetic energy by the
    angle theta outside the box |x_d| <= half_width[d]; theta = 0 removes it."""
    hw = (ctypes.c_double * 3)(*[float(v) for v in half_width])
    _capi.check(_capi.load().afem_mesh_set_ecs(mesh.handle, float(theta), hw))


from ._capi import (PROF_GS, PROF_GCELL32, PROF_STIFF32, PROF_CGVEC32, PROF_CELL64,  # noqa: E402,F401
                    PROF_COUNT)


def profile_enable(on=True):
    """afem_profile_enable: bracket the kernel classes with CUDA events."""
    _capi.check(_capi.load().afem_profile_enable(1 if on else 0))


def profile_read(cls, reset=False):
    """afem_profile_read: (ms, calls, work) of one kernel class."""
    ms, calls, work = ctypes.c_double(0.0), ctypes.c_int64(0), ctypes.c_double(0.0)
    _capi.check(_capi.load().afem_profile_read(int(cls), ctypes.byref(ms), ctypes.byref(calls),
                                               ctypes.byref(work), 1 if reset else 0))
    return ms.value, calls.value, work.value


class Batch:
    """afem_batch_*: the FP32 cell passes of many meshes in one persistent
    launch (batching form), optionally replayed from a captured CUDA graph.

    meshes: list of uploaded Mesh objects (kept alive by the batch)."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        arr = (ctypes.c_void_p * len(self.meshes))(*[m.handle for m in self.meshes])
        h = ctypes.c_void_p()
        _capi.check(_capi.load().afem_batch_create(arr, len(self.meshes), ctypes.byref(h)))
        self.handle = h

    def apply(self, kind, xs, ys, E=None, graph=True, stream=None):
        """y_i = op(x_i) for every instance: kind OP_H1_C64 (complex64 [N_i, n_i],
        n_i even; E: list of 3-vectors or None) or OP_STIFF_F32 (float32 [N_i, k_i],
        k_i % 4 == 0)."""
        import torch
        k = len(self.meshes)
        if len(xs) != k or len(ys) != k:
            raise ValueError("one input and one output per instance")
        dt = torch.complex64 if kind == OP_H1_C64 else torch.float32
        for m, x, y in zip(self.meshes, xs, ys):
            _dev_ptr(x, dt, m.N, "x")
            _dev_ptr(y, dt, m.N, "y")
            if x.shape != y.shape:
                raise ValueError("x and y shapes differ")
        xa = (ctypes.c_void_p * k)(*[x.data_ptr() for x in xs])
        ya = (ctypes.c_void_p * k)(*[y.data_ptr() for y in ys])
        nv = (ctypes.c_int * k)(*[int(x.shape[1]) for x in xs])
        Earr = None
        if E is not None:
            Earr = (ctypes.c_double * (3 * k))(*[float(v) for e in E for v in e])
        _capi.check(_capi.load().afem_batch_op_apply(
            self.handle, int(kind), ctypes.cast(Earr, ctypes.c_void_p) if Earr is not None else None,
            xa, ya, nv, _capi.BATCH_GRAPH if graph else 0, _stream_ptr(stream)))
        return ys

    def tuning(self):
        """The launch shape the autotuner kept and every candidate's time (ms)."""
        t = _capi.BatchTuning()
        _capi.check(_capi.load().afem_batch_get_tuning(self.handle, ctypes.byref(t)))
        cands = [(int(t.cand_block[i]), int(t.cand_grid[i]), float(t.cand_ms[i])) for i in range(t.n_candidates)]
        return {"tuned": bool(t.tuned), "block": t.block, "grid": t.grid, "blocks_per_sm": t.blocks_per_sm,
                "count": t.count, "total_cells": int(t.total_cells), "candidates": cands}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _capi.load().afem_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
