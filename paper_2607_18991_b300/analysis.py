"""Host-side analysis of the GPU results (FP64).

* ``p_hat``   -- mean n*/L^5 per neighborhood, the finite-size estimate of p_c used to place the
  mass measurements;
* ``fit_df``  -- the fractal dimension from S_max ~ L^{d_f} at p = p_c (eq. M_vs_L): ordinary least
  squares of ln <S_max> on ln L, with the slope's standard error;
* ``delta``   -- the percentage error of d_f against d_f* = d - beta/nu (eq. d_f_star, eq. delta);
* ``extrapolate_pc`` -- p_c from finite-size estimates p_hat(L) = p_c + A L^(-1/nu) (FSS with the
  paper's nu_5), linear least squares in x = L^(-1/nu);
* ``fit_power_zeta`` / ``fit_rational_z`` -- the universality laws p_c = zeta^(-g) (eq.
  pc_zeta-to-gamma, with an optional prefactor a) and p_c = c / (z + b) (eq. pc_const-over-z),
  nonlinear least squares in p_c, with standard errors and the residual sum of squares.
"""
from __future__ import annotations

import numpy as np

DF_STAR_5D = 3.5215  # d_f* for d = 5 with beta_5 = 0.8457 and nu_5 = 0.5720 (eq. d_f_star)
NU_5 = 0.5746        # nu for d = 5 (Finite-size scaling theory section)
# sites of coordination zones 1..7 of the 5D simple cubic lattice (|v|^2 = i; Table I single-zone rows)
ZONE_SIZES = (10, 40, 80, 90, 112, 240, 320)


def mask_z_zeta(mask: int) -> tuple[int, float]:
    """z = sum of the selected zones' sizes z_i (eq. z) and zeta = sum z_i sqrt(i) (eq. zeta)."""
    sel = [i for i in range(1, 8) if mask & (1 << (i - 1))]
    return sum(ZONE_SIZES[i - 1] for i in sel), float(sum(ZONE_SIZES[i - 1] * np.sqrt(i) for i in sel))


def p_hat(L: int, nstar) -> float:
    nstar = np.asarray(nstar, dtype=np.float64)
    return float(np.mean(nstar) / float(L) ** 5)


def fit_df(Ls, mean_mass) -> tuple[float, float]:
    """(d_f, standard error) of the least-squares line ln M = d_f ln L + c."""
    x = np.log(np.asarray(Ls, dtype=np.float64))
    y = np.log(np.asarray(mean_mass, dtype=np.float64))
    A = np.stack([x, np.ones_like(x)], axis=1)
    coef, res, _, _ = np.linalg.lstsq(A, y, rcond=None)
    n = len(x)
    if n > 2:
        resid = y - A @ coef
        s2 = float(resid @ resid) / (n - 2)
        cov = s2 * np.linalg.inv(A.T @ A)
        err = float(np.sqrt(cov[0, 0]))
    else:
        err = float("nan")
    return float(coef[0]), err


def delta(df: float, df_star: float = DF_STAR_5D) -> float:
    """Percentage error (d_f* - d_f) / d_f* * 100 (eq. delta)."""
    return (df_star - df) / df_star * 100.0


def extrapolate_pc(Ls, p_hats, nu: float = NU_5) -> tuple[float, float, float]:
    """(p_c, its standard error, A) from p_hat(L) = p_c + A L^(-1/nu) by linear least squares."""
    x = np.asarray(Ls, dtype=np.float64) ** (-1.0 / nu)
    y = np.asarray(p_hats, dtype=np.float64)
    A = np.stack([np.ones_like(x), x], axis=1)
    coef = np.linalg.lstsq(A, y, rcond=None)[0]
    n = len(x)
    err = float("nan")
    if n > 2:
        r = y - A @ coef
        err = float(np.sqrt(float(r @ r) / (n - 2) * np.linalg.inv(A.T @ A)[0, 0]))
    return float(coef[0]), err, float(coef[1])


def _gauss_newton(resid, jac, p0, iters: int = 200):
    """Least squares min |resid(p)|^2 by Gauss-Newton with step halving; returns (p, J, r)."""
    p = np.asarray(p0, dtype=np.float64)
    r = resid(p)
    for _ in range(iters):
        J = jac(p)
        step = np.linalg.lstsq(J, -r, rcond=None)[0]
        t = 1.0
        while t > 1e-12:
            q = p + t * step
            rq = resid(q)
            if float(rq @ rq) <= float(r @ r):
                break
            t *= 0.5
        if t <= 1e-12 or np.max(np.abs(t * step)) <= 1e-15 * (1.0 + np.max(np.abs(p))):
            break
        p, r = q, rq
    return p, jac(p), r


def _fit_result(p, J, r):
    rss = float(r @ r)
    dof = len(r) - len(p)
    cov = np.linalg.inv(J.T @ J) * (rss / dof if dof > 0 else float("nan"))
    return p, np.sqrt(np.diag(cov)), rss


def fit_power_zeta(zeta, pc, prefactor: bool = False):
    """Least squares of p_c = zeta^(-g) (or a zeta^(-g) with prefactor=True) over the data.
    Returns (params, standard errors, residual sum of squares); params = [g] or [a, g]."""
    zeta = np.asarray(zeta, dtype=np.float64)
    pc = np.asarray(pc, dtype=np.float64)
    lz = np.log(zeta)
    if prefactor:
        resid = lambda p: p[0] * zeta ** (-p[1]) - pc
        jac = lambda p: np.stack([zeta ** (-p[1]), -p[0] * lz * zeta ** (-p[1])], axis=1)
        g0 = -np.polyfit(lz, np.log(pc), 1)[0]
        return _fit_result(*_gauss_newton(resid, jac, [1.0, g0]))
    resid = lambda p: zeta ** (-p[0]) - pc
    jac = lambda p: (-lz * zeta ** (-p[0]))[:, None]
    g0 = float(-np.sum(lz * np.log(pc)) / np.sum(lz * lz))
    return _fit_result(*_gauss_newton(resid, jac, [g0]))


def fit_rational_z(z, pc):
    """Least squares of p_c = c / (z + b).  Returns ([b, c], standard errors, residual sum of squares)."""
    z = np.asarray(z, dtype=np.float64)
    pc = np.asarray(pc, dtype=np.float64)
    resid = lambda p: p[1] / (z + p[0]) - pc
    jac = lambda p: np.stack([-p[1] / (z + p[0]) ** 2, 1.0 / (z + p[0])], axis=1)
    # start from the linear form 1/p_c = z/c + b/c
    s, i = np.polyfit(z, 1.0 / pc, 1)
    return _fit_result(*_gauss_newton(resid, jac, [i / s, 1.0 / s]))
