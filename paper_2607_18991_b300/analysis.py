"""Host-side analysis of the GPU results (FP64).

* ``p_hat``   -- mean n*/L^5 per neighborhood, the finite-size estimate of p_c used to place the
  mass measurements;
* ``fit_df``  -- the fractal dimension from S_max ~ L^{d_f} at p = p_c (eq. M_vs_L): ordinary least
  squares of ln <S_max> on ln L, with the slope's standard error;
* ``delta``   -- the percentage error of d_f against d_f* = d - beta/nu (eq. d_f_star, eq. delta).
"""
from __future__ import annotations

import numpy as np

DF_STAR_5D = 3.5215  # d_f* for d = 5 with beta_5 = 0.8457 and nu_5 = 0.5720 (eq. d_f_star)


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
