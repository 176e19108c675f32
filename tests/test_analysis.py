"""Host analysis: d_f least squares and percentage error (eq. M_vs_L, eq. delta)."""
import numpy as np

from paper_2607_18991_b300 import analysis


def test_fit_recovers_exact_power_law():
    Ls = [8, 12, 16, 20, 24, 32]
    M = [3.7 * L ** 3.5215 for L in Ls]
    df, err = analysis.fit_df(Ls, M)
    assert abs(df - 3.5215) < 1e-12 and err < 1e-10


def test_fit_error_matches_textbook_formula():
    rng = np.random.default_rng(0)
    Ls = np.array([8, 12, 16, 20, 24, 32.0])
    y = 3.5 * np.log(Ls) + 1.0 + rng.normal(0, 0.01, len(Ls))
    df, err = analysis.fit_df(Ls, np.exp(y))
    x = np.log(Ls)
    b = np.sum((x - x.mean()) * (y - y.mean())) / np.sum((x - x.mean()) ** 2)
    a = y.mean() - b * x.mean()
    s2 = np.sum((y - a - b * x) ** 2) / (len(x) - 2)
    assert np.isclose(df, b) and np.isclose(err, np.sqrt(s2 / np.sum((x - x.mean()) ** 2)))


def test_delta_of_table2_rows():
    # the paper's Table II: d_f = 3.5453 for sc(5)-1 gives 0.68 %, 3.5836 for sc(5)-1..7 gives 1.76 %
    assert round(abs(analysis.delta(3.5453)), 2) == 0.68
    assert round(abs(analysis.delta(3.5836)), 2) == 1.76
    assert analysis.p_hat(2, [16, 16]) == 0.5
