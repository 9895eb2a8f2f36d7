"""Differentiation form: the one-electron limit of the orbital step behind
``torch.autograd.Function``.

The field is held fixed over each step (Sec. 3.2), so the signal
d_k = <phi_k, Z~ phi_k>_M (the dipole along e, k = 0..K) is a function of the
K field amplitudes E_k.  ``DipoleSignal`` maps E -> d on the GPU and its
backward is the hand-written adjoint of ``afem_tdse_vjp`` (checkpoints every
``ckpt_every`` steps, each segment recomputed in the backward sweep); the
tangent map of ``afem_tdse_jvp`` is exposed as ``tdse_jvp``.  The signal is
the dipole or (``observable="force"``) the expectation of the nuclear force
along e, the potential part of the Ehrenfest acceleration.  The objective
around it is ordinary torch code: a cubic-spline map from a few field samples
to the field at the step and signal times, the acceleration (Ehrenfest, with
its explicit field term, or second differences of the dipole) and its
harmonic yield, whose gradients torch forms itself.
"""
import ctypes

import numpy as np

from . import _capi, _dev_ptr, _stream_ptr, PREC_FP64

# the signal: the dipole <phi, Z~ phi> or the potential part of the Ehrenfest
# acceleration <phi, M_L^-1 F[e.(-grad V)] phi>
OBSERVABLES = {"dipole": _capi.OP_POS, "force": _capi.OP_FORCE}


def _host(a, n, name):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if a.shape[0] != n:
        raise ValueError(f"{name} must have {n} entries, got {a.shape[0]}")
    return a


def _dptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None and a.size else None


def n_checkpoints(n_steps, ckpt_every):
    """Slots of the checkpoint buffer: phi_{c ckpt_every} for c ckpt_every < n_steps."""
    return (int(n_steps) + int(ckpt_every) - 1) // int(ckpt_every)


def tdse_forward(mesh, phi0, E, dt, e_dir=(0.0, 0.0, 1.0), krylov_m=16, tol=0.0, precision=PREC_FP64,
                 ckpt_every=0, want_end=False, stream=None, observable="dipole"):
    """afem_tdse_forward.  phi0: complex128 [N] CUDA tensor; E: K host values.

    Returns (d numpy [K+1], phi_end tensor or None, ckpt tensor [n_ckpt, N] or None).
    """
    import torch
    K = int(np.asarray(E).size)
    Eh = _host(E, K, "E")
    _dev_ptr(phi0, torch.complex128, mesh.N, "phi0")
    e = _host(e_dir, 3, "e_dir")
    d = np.zeros(K + 1)
    end = torch.empty_like(phi0) if want_end else None
    ckpt = None
    if ckpt_every and K > 0:
        ckpt = torch.empty((n_checkpoints(K, ckpt_every), mesh.N), dtype=torch.complex128, device=phi0.device)
    _capi.check(_capi.load().afem_tdse_forward(
        mesh.handle, _dptr(e), _dptr(Eh), K, float(dt), int(krylov_m), float(tol), int(precision),
        OBSERVABLES[observable],
        ctypes.c_void_p(phi0.data_ptr()), ctypes.c_void_p(end.data_ptr()) if end is not None else None,
        _dptr(d), ctypes.c_void_p(ckpt.data_ptr()) if ckpt is not None else None, int(ckpt_every or 0),
        _stream_ptr(stream)))
    return d, end, ckpt


def tdse_jvp(mesh, phi0, E, v, dt, e_dir=(0.0, 0.0, 1.0), krylov_m=16, tol=0.0, precision=PREC_FP64,
             stream=None, observable="dipole"):
    """afem_tdse_jvp: returns (d [K+1], dd [K+1]) for the field perturbation v [K]."""
    import torch
    K = int(np.asarray(E).size)
    Eh = _host(E, K, "E")
    vh = _host(v, K, "v")
    _dev_ptr(phi0, torch.complex128, mesh.N, "phi0")
    e = _host(e_dir, 3, "e_dir")
    d = np.zeros(K + 1)
    dd = np.zeros(K + 1)
    _capi.check(_capi.load().afem_tdse_jvp(
        mesh.handle, _dptr(e), _dptr(Eh), K, float(dt), int(krylov_m), float(tol), int(precision),
        OBSERVABLES[observable], ctypes.c_void_p(phi0.data_ptr()), _dptr(vh), _dptr(d), _dptr(dd),
        _stream_ptr(stream)))
    return d, dd


def tdse_vjp(mesh, ckpt, ckpt_every, E, g, dt, e_dir=(0.0, 0.0, 1.0), krylov_m=16, tol=0.0,
             precision=PREC_FP64, want_lam0=False, stream=None, observable="dipole"):
    """afem_tdse_vjp: returns (grad_E [K], lam0 tensor or None) for the cotangent g [K+1]."""
    import torch
    K = int(np.asarray(E).size)
    Eh = _host(E, K, "E")
    gh = _host(g, K + 1, "g")
    e = _host(e_dir, 3, "e_dir")
    if not isinstance(ckpt, torch.Tensor) or ckpt.dim() != 2 or ckpt.shape[0] != n_checkpoints(K, ckpt_every):
        raise ValueError("ckpt must be the [n_checkpoints, N] buffer of tdse_forward")
    _dev_ptr(ckpt, torch.complex128, None, "ckpt")
    if ckpt.shape[1] != mesh.N:
        raise ValueError("ckpt rows must have N entries")
    grad = np.zeros(K)
    lam0 = torch.empty(mesh.N, dtype=torch.complex128, device=ckpt.device) if want_lam0 else None
    _capi.check(_capi.load().afem_tdse_vjp(
        mesh.handle, _dptr(e), _dptr(Eh), K, float(dt), int(krylov_m), float(tol), int(precision),
        OBSERVABLES[observable], ctypes.c_void_p(ckpt.data_ptr()), int(ckpt_every), _dptr(gh), _dptr(grad),
        ctypes.c_void_p(lam0.data_ptr()) if lam0 is not None else None, _stream_ptr(stream)))
    return grad, lam0


def _make_function():
    import torch

    class DipoleSignal(torch.autograd.Function):
        """E [K] (float64, CPU) -> d [K+1] (float64, CPU); backward by the adjoint sweep."""

        @staticmethod
        def forward(ctx, E, mesh, phi0, dt, e_dir, krylov_m, tol, precision, ckpt_every, observable):
            En = E.detach().cpu().numpy().astype(np.float64)
            d, _, ckpt = tdse_forward(mesh, phi0, En, dt, e_dir, krylov_m, tol, precision, ckpt_every,
                                      observable=observable)
            ctx.args = (mesh, En, dt, e_dir, krylov_m, tol, precision, ckpt_every, observable)
            ctx.ckpt = ckpt
            return torch.from_numpy(d).to(E.dtype)

        @staticmethod
        def backward(ctx, g):
            mesh, En, dt, e_dir, krylov_m, tol, precision, every, observable = ctx.args
            if En.size == 0:
                return (torch.zeros(0, dtype=torch.float64),) + (None,) * 9
            grad, _ = tdse_vjp(mesh, ctx.ckpt, every, En, g.detach().cpu().numpy(), dt, e_dir, krylov_m, tol,
                               precision, observable=observable)
            return (torch.from_numpy(grad),) + (None,) * 9

    return DipoleSignal


_FN = None


def dipole_signal(E, mesh, phi0, dt, e_dir=(0.0, 0.0, 1.0), krylov_m=16, tol=0.0, precision=PREC_FP64,
                  ckpt_every=50, observable="dipole"):
    """Differentiable signal s(E): E float64 CPU tensor [K] -> float64 CPU tensor
    [K+1], s_k = <phi_k, O phi_k>_M with O the dipole's (observable="dipole")
    or the nuclear force's along e (observable="force")."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    if observable not in OBSERVABLES:
        raise ValueError("observable must be 'dipole' or 'force'")
    return _FN.apply(E, mesh, phi0, float(dt), tuple(float(x) for x in e_dir), int(krylov_m), float(tol),
                     int(precision), int(ckpt_every), observable)


def spline_matrix(n_samples, n_steps):
    """Not-a-knot cubic spline through n_samples (>= 4) equally spaced values on
    [0, 1], evaluated at the n_steps step points k / (n_steps - 1): a
    [n_steps, n_samples] float64 matrix S, so that E = S c (the window's field
    from its samples; the spline is linear in the samples, so dJ/dc = S^T dJ/dE)."""
    import scipy.interpolate
    t = np.linspace(0.0, 1.0, n_samples)
    x = np.linspace(0.0, 1.0, n_steps) if n_steps > 1 else np.zeros(1)
    S = np.empty((n_steps, n_samples))
    for j in range(n_samples):
        c = np.zeros(n_samples)
        c[j] = 1.0
        S[:, j] = scipy.interpolate.CubicSpline(t, c, bc_type="not-a-knot")(x)
    return S


def ehrenfest_acceleration(force_signal, E_samples, e_dir=(0.0, 0.0, 1.0)):
    """The electron's acceleration along e at the sample times: the force signal
    <-grad V . e> minus (e . e) E(t_k) (torch, differentiable in both).
    E_samples holds the field at the K+1 signal times."""
    ee = float(np.dot(np.asarray(e_dir, dtype=np.float64), np.asarray(e_dir, dtype=np.float64)))
    return force_signal - ee * E_samples


def harmonic_yield(d, dt, omega0, h_lo=15, h_hi=25, acceleration=None):
    """sum over FFT bins with omega in [h_lo omega0, h_hi omega0] of |FFT a|^2: a the
    given acceleration signal, or else the dipole acceleration by central second
    differences of d (torch, differentiable)."""
    import torch
    a = acceleration if acceleration is not None else (d[2:] - 2.0 * d[1:-1] + d[:-2]) / (dt * dt)
    A = torch.fft.rfft(a)
    omega = 2.0 * np.pi * np.arange(A.shape[0]) / (a.shape[0] * dt)
    band = torch.from_numpy((omega >= h_lo * omega0) & (omega <= h_hi * omega0))
    return (A.real ** 2 + A.imag ** 2)[band].sum()
