"""Short-iterative Arnoldi propagator (Sec. 3.2).

With the operator frozen over one step, phi(t + dt) = exp(-i G dt) phi(t)
(Sec. 3.2).  The Krylov space of G started at phi is built by the Arnoldi
process (modified Gram-Schmidt, one pass) in the inner product
<u, v> = sum_p u_p^H M_L v_p over the stacked orbitals; with
G V_m = V_m H_m + h_{m+1,m} v_{m+1} e_m^T the propagated vector is
beta V_m exp(-i dt H_m) e_1, beta = ||phi||.  The error estimate is the
classical one of the Krylov exponential literature that the paper cites
(Park and Light): beta |h_{m+1,m}| |e_m^T exp(-i dt H_m) e_1|.

Test infrastructure only (see the package docstring).
"""
import numpy as np
import scipy.linalg

LADDER = 64          # candidate substep lengths per ladder in arnoldi_propagate
LADDER_LOG2 = 0.125  # candidate c is tau_max 2^(-c LADDER_LOG2)


def _expm(H, dt, imaginary):
    """exp(-i dt H), or exp(-dt H) for an imaginary-time step."""
    return scipy.linalg.expm((-dt if imaginary else -1j * dt) * H)


def arnoldi_expm(apply_G, phi, inner, m, dt, breakdown_tol=1e-14, imaginary=False):
    """Returns (phi_new, err_estimate, H (m+1 x m), m_used, breakdown).

    apply_G: v -> G v; inner: (u, v) -> <u, v> (complex scalar).
    A happy breakdown (h_{j+1,j} < breakdown_tol * beta) stops the process
    early; the result is then exact in exact arithmetic.  imaginary: the
    imaginary-time step beta V_m exp(-dt H_m) e_1 (t -> -i tau), with the
    same estimate formed from exp(-dt H_m).
    """
    beta = np.sqrt(inner(phi, phi).real)
    V = [phi / beta]
    H = np.zeros((m + 1, m), dtype=np.complex128)
    m_used = m
    breakdown = False
    for j in range(m):
        w = apply_G(V[j])
        for i in range(j + 1):
            H[i, j] = inner(V[i], w)
            w = w - H[i, j] * V[i]
        hn = np.sqrt(inner(w, w).real)
        H[j + 1, j] = hn
        if hn < breakdown_tol * beta:
            m_used = j + 1
            breakdown = True
            break
        V.append(w / hn)
    Hm = H[:m_used, :m_used]
    Em = _expm(Hm, dt, imaginary)
    y = beta * Em[:, 0]
    out = sum(y[i] * V[i] for i in range(m_used))
    err = 0.0 if breakdown else beta * abs(H[m_used, m_used - 1]) * abs(Em[m_used - 1, 0])
    return out, err, H, m_used, breakdown


def arnoldi_basis(apply_G, phi, inner, m, breakdown_tol=1e-14):
    """(beta, V list, H (m+1 x m), m_used, breakdown, h_{m_used+1, m_used}) of the Krylov space from phi."""
    beta = np.sqrt(inner(phi, phi).real)
    V = [phi / beta]
    H = np.zeros((m + 1, m), dtype=np.complex128)
    m_used, breakdown = m, False
    for j in range(m):
        w = apply_G(V[j])
        for i in range(j + 1):
            H[i, j] = inner(V[i], w)
            w = w - H[i, j] * V[i]
        hn = np.sqrt(inner(w, w).real)
        H[j + 1, j] = hn
        if hn < breakdown_tol * beta:
            m_used, breakdown = j + 1, True
            break
        V.append(w / hn)
    return beta, V, H, m_used, breakdown, abs(H[m_used, m_used - 1])


def arnoldi_propagate(apply_G, phi, inner, m, dt, tol, max_substeps=4096, return_info=False, stop_after=None,
                      imaginary=False):
    """exp(-i G dt) phi with the Krylov error controlled substep by substep.

    Sec. 3.2 fixes the Krylov accuracy by an a-posteriori estimate (threshold
    1e-10 in the paper) and leaves open how the step adapts (Park and Light
    allow an adaptive step or an adaptive dimension).  Here the dimension m is
    fixed and dt is covered by substeps of the same G, each as long as the
    candidates allow: tau_c = tau_max 2^(-c/8), c = 0..63, with tau_max the
    whole remainder for the first substep and min(remainder, 2 tau_previous)
    after it; the first (longest) candidate whose estimate
    beta |h_{m+1,m}| |e_m^T exp(-i tau_c H_m) e_1| is <= tol beta is taken;
    when none is, the ladder continues below its smallest candidate (at most 8
    more ladders, then the smallest is taken).  A breakdown (invariant Krylov
    space) takes the whole remainder with estimate 0.  tol <= 0: one step over
    dt.  Returns (phi_new, sum of estimates, substeps), and with return_info a
    fourth item: {"taus": substep lengths, "margin": the smallest
    |log(estimate / (tol beta))| over every candidate the decisions compared
    with the threshold, "remaining": the time left} -- a margin near zero marks
    a near-tie, a decision that rounding at the level of the margin could flip.
    stop_after: return after that many substeps (a partial propagation, for
    timing a bounded sample).  imaginary: exp(-G dt) phi (imaginary time),
    the candidates' estimates formed from exp(-tau H_m).
    """
    remaining = dt
    cur = phi
    total, substeps, tau_prev = 0.0, 0, 0.0
    taus, margin = [], np.inf
    while remaining > 0.0:
        if substeps >= max_substeps:
            raise RuntimeError("too many Krylov substeps")
        beta, V, H, mu, brk, hlast = arnoldi_basis(apply_G, cur, inner, m)
        if brk or tol <= 0.0:
            tau = remaining
            Em = _expm(H[:mu, :mu], tau, imaginary)
            err = 0.0 if brk else beta * hlast * abs(Em[mu - 1, 0])
        else:
            tau_max = remaining if substeps == 0 else min(remaining, 2.0 * tau_prev)
            found = False
            for ladder in range(9):
                for c in range(LADDER):
                    tau = tau_max * 2.0 ** (-LADDER_LOG2 * c)
                    Em = _expm(H[:mu, :mu], tau, imaginary)
                    err = beta * hlast * abs(Em[mu - 1, 0])
                    if err > 0.0:
                        margin = min(margin, abs(np.log(err / (tol * beta))))
                    if err <= tol * beta:
                        found = True
                        break
                if found:
                    break
                tau_max *= 2.0 ** (-LADDER_LOG2 * LADDER)
        cur = sum(beta * Em[i, 0] * V[i] for i in range(mu))
        total += err
        substeps += 1
        tau_prev = tau
        taus.append(tau)
        remaining = 0.0 if tau >= remaining else remaining - tau
        if stop_after is not None and substeps >= stop_after:
            break
    if return_info:
        return cur, total, substeps, dict(taus=taus, margin=margin, remaining=remaining)
    return cur, total, substeps


def arnoldi_adaptive(apply_G, phi, inner, m_max, dt, tol, substeps=1, breakdown_tol=1e-14, imaginary=False):
    """exp(-i G dt) phi by the rule of Sec. 3.2: the step is fixed and the Krylov
    dimension is chosen by the estimate.

    dt is split into `substeps` equal steps tau = dt / substeps (the paper fixes
    its time step so that the dimension stays within 10-15).  In each, the
    Arnoldi process (modified Gram-Schmidt, M_L inner product) adds one vector
    at a time; after vector j + 1 the estimate of dimension j + 1,
    beta |h_{j+2,j+1}| |e_{j+1}^T exp(-i tau H_{j+1}) e_1|, is formed, and the
    first dimension whose estimate is <= tol beta is used (a breakdown ends the
    process with the exact projected exponential).  If no dimension up to
    m_max passes, m_max is used and its estimate is reported.  Returns
    (phi_new, sum of estimates, info) with info = {"dims": dimension of each
    step, "margin": the smallest |log(estimate / (tol beta))| over every
    dimension compared with the threshold, "passed": all steps met tol}.
    """
    tau = dt / substeps
    cur = phi
    total, dims, margin, passed = 0.0, [], np.inf, True
    for _ in range(substeps):
        beta = np.sqrt(inner(cur, cur).real)
        V = [cur / beta]
        H = np.zeros((m_max + 1, m_max), dtype=np.complex128)
        for j in range(m_max):
            w = apply_G(V[j])
            for i in range(j + 1):
                H[i, j] = inner(V[i], w)
                w = w - H[i, j] * V[i]
            hn = np.sqrt(inner(w, w).real)
            H[j + 1, j] = hn
            mu = j + 1
            Em = _expm(H[:mu, :mu], tau, imaginary)
            if hn < breakdown_tol * beta:
                err = 0.0
                break
            err = beta * hn * abs(Em[mu - 1, 0])
            if err > 0.0:
                margin = min(margin, abs(np.log(err / (tol * beta))))
            if err <= tol * beta:
                break
            if j + 1 == m_max:
                passed = False
                break
            V.append(w / hn)
        cur = sum(beta * Em[i, 0] * V[i] for i in range(mu))
        total += err
        dims.append(mu)
    return cur, total, dict(dims=dims, margin=margin, passed=passed)
