"""The two reformulations the CUDA gradient path relies on, checked in FP64
with explicit operators on a small 1-D grid (no GPU; the identities do not
depend on the dimension):

1. mu = D lam obeys the forward recurrence backward in time, with the
   residual injected scaled by D (so the forward sweep kernel runs the
   adjoint);
2. the imaging term 2 g (u^{k-1} - u^{k-2}) - c2 L u^{k-1} equals
   -(1+g) [(u^k - c2 S^{k-1}) - 2 u^{k-1} + u^{k-2}] by the forward
   recurrence (so it is computed pointwise from three stored states);

and the gradient assembled from them (in mu) against central finite
differences of the objective.  The recurrence is Eq. 1 with the sponge:
u^k = D L u^{k-1} + B u^{k-1} + C u^{k-2} + M S^{k-1}, D = dt^2/(m + a),
B = 2m/(m + a), C = (a - m)/(m + a), M = dt^2/m, a = eta dt / 2."""
from __future__ import annotations

import numpy as np
import pytest

N, NT, H = 48, 36, 10.0


def problem(seed=3):
    g = np.random.default_rng(seed)
    # centred 4th-order second derivative, zero values outside the grid
    c = np.array([-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0]) / H ** 2
    L = np.zeros((N, N))
    for i in range(N):
        L[i, i] = c[0]
        for k in (1, 2):
            if i - k >= 0:
                L[i, i - k] = c[k]
            if i + k < N:
                L[i, i + k] = c[k]
    vp = g.uniform(1500.0, 3000.0, N)
    m = 1.0 / vp ** 2
    dt = 0.5 * H / vp.max()
    eta = np.zeros(N)
    nbl = 8
    ramp = (np.arange(nbl, 0, -1) / nbl) ** 2 * 400.0
    eta[:nbl] = ramp
    eta[-nbl:] = ramp[::-1]
    a = eta * dt / 2.0
    S = np.zeros((NT, N))  # S^{k-1}, k = 1 .. NT
    w = np.sin(np.linspace(0.0, 3.0 * np.pi, NT)) * np.exp(-np.linspace(0.0, 3.0, NT))
    S[:, 20] = w
    S[:, 3] = 0.5 * w          # one source inside the sponge (g != 0 there)
    P = np.zeros((5, N))
    for j, i in enumerate([2, 11, 25, 33, 45]):
        P[j, i] = 1.0
    r = g.standard_normal((NT, 5))
    return L, m, dt, a, S, P, r


def coeffs(m, dt, a):
    D = dt ** 2 / (m + a)
    B = 2.0 * m / (m + a)
    C = (a - m) / (m + a)
    M = dt ** 2 / m
    return D, B, C, M


def forward(L, m, dt, a, S):
    D, B, C, M = coeffs(m, dt, a)
    u = np.zeros((NT + 2, N))  # u[k + 1] = u^k, k = -1 .. NT
    for k in range(1, NT + 1):
        u[k + 1] = D * (L @ u[k]) + B * u[k] + C * u[k - 1] + M * S[k - 1]
    return u


def objective(L, m, dt, a, S, P, r):
    u = forward(L, m, dt, a, S)
    return sum(float((P @ u[k + 1]) @ r[k - 1]) for k in range(1, NT + 1))


def adjoint_lam(L, m, dt, a, P, r):
    D, B, C, _ = coeffs(m, dt, a)
    lam = np.zeros((NT + 3, N))  # lam[k] = lam^k, k = 1 .. NT + 2
    for k in range(NT, 0, -1):
        lam[k] = L @ (D * lam[k + 1]) + B * lam[k + 1] + C * lam[k + 2] + P.T @ r[k - 1]
    return lam


def adjoint_mu(L, m, dt, a, P, r):
    """The forward recurrence, backward in time, residual scaled by D."""
    D, B, C, _ = coeffs(m, dt, a)
    mu = np.zeros((NT + 3, N))
    for k in range(NT, 0, -1):
        mu[k] = D * (L @ mu[k + 1]) + B * mu[k + 1] + C * mu[k + 2] + D * (P.T @ r[k - 1])
    return mu


def test_lam_recurrence_is_the_transpose():
    """<P u, r> = <S, M lam>: the lam recurrence is the adjoint (the setup the
    other checks build on)."""
    L, m, dt, a, S, P, r = problem()
    _, _, _, M = coeffs(m, dt, a)
    lhs = objective(L, m, dt, a, S, P, r)
    lam = adjoint_lam(L, m, dt, a, P, r)
    rhs = sum(float(S[k - 1] @ (M * lam[k])) for k in range(1, NT + 1))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_mu_is_D_times_lam():
    L, m, dt, a, S, P, r = problem()
    D, _, _, _ = coeffs(m, dt, a)
    lam = adjoint_lam(L, m, dt, a, P, r)
    mu = adjoint_mu(L, m, dt, a, P, r)
    np.testing.assert_allclose(mu, D * lam, rtol=1e-12, atol=1e-12 * np.abs(mu).max())


def test_imaging_term_from_three_states():
    L, m, dt, a, S, P, r = problem()
    c2, g = dt ** 2 / m, a / m
    u = forward(L, m, dt, a, S)
    for k in range(2, NT + 1):
        uk, u1, u2 = u[k + 1], u[k], u[k - 1]
        lhs = 2.0 * g * (u1 - u2) - c2 * (L @ u1)
        rhs = -(1.0 + g) * ((uk - c2 * S[k - 1]) - 2.0 * u1 + u2)
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-10 * max(np.abs(lhs).max(), 1e-300))


def gradient_mu(L, m, dt, a, S, P, r):
    """d J / d m as the CUDA path assembles it: -sum mu^k [(u^k - u^{k-1}) -
    (u^{k-1} - u^{k-2})] / dt^2 - sum mu^k (c2 S^{k-1}) g / dt^2."""
    c2, g = dt ** 2 / m, a / m
    u = forward(L, m, dt, a, S)
    mu = adjoint_mu(L, m, dt, a, P, r)
    gm = np.zeros(N)
    for k in range(1, NT + 1):
        d2 = (u[k + 1] - u[k]) - (u[k] - u[k - 1])
        gm -= mu[k] * d2 / dt ** 2
        gm -= mu[k] * (c2 * S[k - 1]) * g / dt ** 2
    return gm


@pytest.mark.parametrize("p", [3, 11, 20, 30, 44])
def test_gradient_matches_finite_differences(p):
    """Interior points, the point of the source in the sponge (3) and the
    point of the interior source (20)."""
    L, m, dt, a, S, P, r = problem()
    gm = gradient_mu(L, m, dt, a, S, P, r)
    e = 1e-5 * m[p]
    mp, mm = m.copy(), m.copy()
    mp[p] += e
    mm[p] -= e
    fd = (objective(L, mp, dt, a, S, P, r) - objective(L, mm, dt, a, S, P, r)) / (2.0 * e)
    assert gm[p] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(gm).max())
