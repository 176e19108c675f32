"""Measured runs of the workloads besides the L = 16 benchmark line.

    python -m paper_2607_18991_b300.experiments mass|L24|L40|mixed|all [--quick]

Each run prints one JSON line:

* ``mass``  -- compact neighborhoods {1..k}, k = 1..7: p_hat(k) = mean n*/16^5 over seeds 1..256 at
  L = 16, then S_max at n = floor(p_hat L^5 + 1/2) for L in {8, 12, 16, 20, 24, 32}, seeds 1..512,
  and the d_f least-squares fit (eq. M_vs_L) with its percentage error (eq. delta);
* ``L24``   -- all 127 neighborhoods at L = 24, seeds 1..128: samples/s and passes with the learned
  bracket (network trained at L = 8 and 16 only) and with the plain one;
* ``L40``   -- sc(5)-1,...,7 at L = 40 (102.4M sites), seeds 1..8;
* ``mixed`` -- 4096 samples with L uniform in {10..40} and random masks, plain and learned;
* ``large`` -- the largest lattices: L = 48 (254.8M sites), all 127 neighborhoods, seeds 1..2, and
  L = 64 (1.07G sites), sc(5)-1,...,7, seeds 1..4; samples/s with the plain bracket;
* ``universality`` -- p_hat(k, L) = mean n*/L^5 for all 127 neighborhoods at L in {8, 12, 16, 20, 24},
  extrapolated per neighborhood to L -> infinity (p_hat = p_c + A L^(-1/nu)), compared with Table I,
  and the universality fits p_c = c/(z+b), p_c = zeta^(-g), p_c = a zeta^(-g) on those values and on
  Table I (section "Universality of p_c behavior").

Times are wall-clock with the device synchronised, ranking included.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import analysis, bracket, driver, perc, workloads

L16 = 16
# p_c of the compact neighborhoods as the paper lists them (Table II), for the cross-check fit
PC_TABLE2 = {1: 0.14079633, 3: 0.033794, 7: 0.013190, 15: 0.007850, 31: 0.0051575, 63: 0.002981, 127: 0.001934}


def trained_params(quick: bool = False):
    """Bracket network trained on plain n* of held-out seeds at L = 8 (zone 1) and L = 16."""
    n8, n16 = (200, 8) if quick else (1000, 64)
    wl = np.concatenate([np.array([(8, 1, s) for s in range(1_000_001, 1_000_001 + n8)]),
                         np.array([(L16, m, s) for m in workloads.ALL_MASKS
                                   for s in range(1_000_001, 1_000_001 + n16)])])
    ns, _ = driver.nstar(wl)
    params, _ = bracket.train(wl[:, 0], wl[:, 1], ns, steps=3000, lr=3e-3)
    return params


def _timed(fn):
    torch.cuda.synchronize()
    t = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t


def _mass_fits(p_of_mask: dict, nseeds: int):
    rows, ns = [], []
    for L in workloads.MASS_LS:
        for m in workloads.COMPACT_MASKS:
            for s in range(1, nseeds + 1):
                rows.append((L, m, s))
                ns.append(workloads.mass_n(p_of_mask[m], L))
    wl = np.array(rows, dtype=np.int64)
    mass, dt = _timed(lambda: driver.mass(wl, ns))
    fits = {}
    for m in workloads.COMPACT_MASKS:
        mean = [float(mass[(wl[:, 0] == L) & (wl[:, 1] == m)].mean()) for L in workloads.MASS_LS]
        df, err = analysis.fit_df(workloads.MASS_LS, mean)
        k = bin(m).count("1")
        fits[f"1..{k}"] = {"p": p_of_mask[m], "d_f": df, "err": err, "delta_pct": analysis.delta(df),
                           "mean_mass": mean}
    return wl, dt, fits


def run_mass(quick: bool = False) -> dict:
    seeds16 = range(1, 33 if quick else 257)
    wl16 = workloads.samples(L16, workloads.COMPACT_MASKS, seeds16)
    ns16, _ = driver.nstar(wl16)
    p_hat = {m: analysis.p_hat(L16, ns16[wl16[:, 1] == m]) for m in workloads.COMPACT_MASKS}
    nseeds = 32 if quick else 512
    wl, dt, fits = _mass_fits(p_hat, nseeds)
    _, dt2, fits_t2 = _mass_fits(PC_TABLE2, nseeds)  # physics cross-check at the paper's p_c
    return {"workload": "compact masses", "samples": len(wl), "seconds": dt, "samples_per_s": len(wl) / dt,
            "L": workloads.MASS_LS, "seeds": nseeds, "fits_at_p_hat_L16": fits, "fits_at_table2_pc": fits_t2}


def _learned_vs_plain(wl: np.ndarray, params) -> dict:
    out = {}
    for name, p in (("learned", params), ("plain", None)):
        stats = perc.new_stats()
        (ns, passes), dt = _timed(lambda: driver.nstar(wl, params=p, margin=0.05, stats=stats))
        st = perc.stats_dict(stats)
        out[name] = {"seconds": dt, "samples_per_s": len(wl) / dt, "passes_per_sample": float(passes.mean()),
                     "fallbacks": st["fallbacks"], "verified": st["verified"]}
        out[name + "_nstar"] = ns
    assert np.array_equal(out.pop("learned_nstar"), out.pop("plain_nstar")), "learned and plain n* differ"
    return out


def run_L24(params, quick: bool = False) -> dict:
    wl = workloads.all127_L24(16 if quick else 128)
    res = _learned_vs_plain(wl, params)
    return {"workload": "all 127 masks, L=24", "samples": len(wl), **res}


def run_L40(params, quick: bool = False) -> dict:
    wl = workloads.z892_L40(2 if quick else 8)
    res = _learned_vs_plain(wl, params)
    return {"workload": "sc(5)-1..7, L=40", "samples": len(wl), **res}


def run_mixed(params, quick: bool = False) -> dict:
    wl = workloads.mixed4096(512 if quick else 4096)
    res = _learned_vs_plain(wl, params)
    return {"workload": "mixed L in 10..40, random masks", "samples": len(wl), **res}


UNIV_SEEDS = {8: 512, 12: 256, 16: 128, 20: 64, 24: 32}


def run_large(quick: bool = False) -> dict:
    out = {"workload": "largest lattices, plain bracket, times with the ranking of every seed"}
    for name, wl in (("L48_all127", workloads.samples(48, workloads.ALL_MASKS, range(1, 2 if quick else 3))),
                     ("L64_z892", workloads.samples(64, [127], range(1, 2 if quick else 5)))):
        (ns, passes), dt = _timed(lambda: driver.nstar(wl))
        out[name] = {"samples": len(wl), "seconds": dt, "samples_per_s": len(wl) / dt,
                     "mean_nstar_over_N": float(np.mean(ns / float(wl[0, 0]) ** 5)),
                     "passes_per_sample": float(passes.mean())}
    return out


def _fits(z, zeta, pc) -> dict:
    (b, c), (eb, ec), rss = analysis.fit_rational_z(z, pc)
    (g,), (eg,), rss_g = analysis.fit_power_zeta(zeta, pc)
    (a, g2), (ea, eg2), rss_g2 = analysis.fit_power_zeta(zeta, pc, prefactor=True)
    return {"c_over_z_plus_b": {"b": b, "b_err": eb, "c": c, "c_err": ec, "rss": rss},
            "zeta_power": {"g": g, "g_err": eg, "rss": rss_g},
            "zeta_power_prefactor": {"a": a, "a_err": ea, "g": g2, "g_err": eg2, "rss": rss_g2}}


def run_universality(quick: bool = False) -> dict:
    masks = workloads.ALL_MASKS
    p_hat = {}
    t0 = time.perf_counter()
    for L, ns in UNIV_SEEDS.items():
        wl = workloads.samples(L, masks, range(1, (max(ns // 8, 2) if quick else ns) + 1))
        nst, _ = driver.nstar(wl)
        p_hat[L] = np.array([analysis.p_hat(L, nst[wl[:, 1] == m]) for m in masks])
    dt = time.perf_counter() - t0
    Ls = sorted(p_hat)
    ext = [analysis.extrapolate_pc(Ls, [p_hat[L][k] for L in Ls]) for k in range(len(masks))]
    pc_ext = np.array([e[0] for e in ext])
    z = np.array([analysis.mask_z_zeta(m)[0] for m in masks], dtype=np.float64)
    zeta = np.array([analysis.mask_z_zeta(m)[1] for m in masks], dtype=np.float64)
    pc_t1 = np.array([workloads.TABLE1_PC[m] for m in masks])
    rel = pc_ext / pc_t1 - 1.0
    return {"workload": "universality: n* of all 127 neighborhoods at L = " + ", ".join(map(str, Ls)),
            "seeds": UNIV_SEEDS, "seconds": dt,
            "p_hat_mean_rel_to_table1": {str(L): float(np.mean(p_hat[L] / pc_t1 - 1.0)) for L in Ls},
            "extrapolated_vs_table1": {"mean_rel": float(rel.mean()), "rms_rel": float(np.sqrt(np.mean(rel ** 2))),
                                       "max_abs_rel": float(np.abs(rel).max()),
                                       "sc5_1": [float(pc_ext[0]), float(ext[0][1])],
                                       "sc5_1_7": [float(pc_ext[126]), float(ext[126][1])]},
            "fits_extrapolated": _fits(z, zeta, pc_ext), "fits_table1": _fits(z, zeta, pc_t1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["mass", "L24", "L40", "mixed", "universality", "large", "all"])
    ap.add_argument("--quick", action="store_true")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    params = None if args.which in ("mass", "universality", "large") else trained_params(args.quick)
    todo = ["mass", "L24", "L40", "mixed"] if args.which == "all" else [args.which]
    for w in todo:
        if w == "mass":
            r = run_mass(args.quick)
        elif w == "universality":
            r = run_universality(args.quick)
        elif w == "large":
            r = run_large(args.quick)
        elif w == "L24":
            r = run_L24(params, args.quick)
        elif w == "L40":
            r = run_L40(params, args.quick)
        else:
            r = run_mixed(params, args.quick)
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
