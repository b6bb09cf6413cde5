"""Finite-temperature scan (Sec. 2.2): the Polyakov loop and the
colour-averaged free energy over a range of couplings at fixed Nt, with the
string tension from F(r) = a0 - a1 / r + sigma r at every coupling.

The lattice work runs in the CUDA library through the C ABI: one batched
handle holds every coupling's lattice, `su2_batch_heatbath` thermalises
them and `su2_batch_heatbath_measure` advances them in bins of sweeps,
returning per bin the sums over its sweeps of the Polyakov loop, its
modulus and the correlator C(r).  Everything after that (bin means,
jackknife errors, the fits) is host post-processing of those FP64 sums.

Scale setting is a reading, since the paper does not give its own: the
critical coupling beta_c is where <|L|> first climbs through half of its
largest value in this scan, and T / T_c = a(beta_c) / a(beta) with the
two-loop asymptotic scaling of the SU(2) lattice spacing.

    python -m paper_1104_5432_gb300.scan --out scan.json
"""
from __future__ import annotations

import argparse
import json
import math
import sys
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import analysis

# two-loop coefficients of the SU(N) beta function, N = 2
B0 = 11.0 * 2 / (48.0 * math.pi ** 2)
B1 = (34.0 / 3.0) * 4.0 / (16.0 * math.pi ** 2) ** 2


def lattice_spacing(beta):
    """a Lambda_L at two loops: (b0 g^2)^(-b1 / (2 b0^2)) exp(-1 / (2 b0 g^2)),
    g^2 = 4 / beta."""
    g2 = analysis.g2_of_beta(beta)
    return (B0 * g2) ** (-B1 / (2 * B0 ** 2)) * np.exp(-1.0 / (2 * B0 * g2))


def t_over_tc(beta, beta_c):
    """T / T_c = a(beta_c) / a(beta) at fixed Nt."""
    return lattice_spacing(beta_c) / lattice_spacing(beta)


def jackknife(bins: np.ndarray, f=lambda m: m):
    """Mean and jackknife error of f(bin mean) over the first axis."""
    bins = np.asarray(bins, dtype=np.float64)
    nb = bins.shape[0]
    full = f(bins.mean(0))
    tot = bins.sum(0)
    samples = np.stack([f((tot - bins[k]) / (nb - 1)) for k in range(nb)])
    err = np.sqrt((nb - 1) / nb * np.sum((samples - samples.mean(0)) ** 2, axis=0))
    return full, err, samples


def beta_critical(betas: Sequence[float], abs_L: Sequence[float]) -> float:
    """The coupling where <|L|> first climbs through half of its largest
    value in the scan, by linear interpolation between the two couplings
    around the crossing.  Half the maximum, not the steepest slope, because
    on the deconfined side of a large lattice a hot start can leave Z2
    domain walls that pull single couplings back towards zero."""
    b = np.asarray(betas, dtype=np.float64)
    y = np.asarray(abs_L, dtype=np.float64)
    half = 0.5 * float(y.max())
    k = int(np.argmax(y >= half))
    if k == 0:
        return float(b[0])
    return float(b[k - 1] + (half - y[k - 1]) * (b[k] - b[k - 1]) / (y[k] - y[k - 1]))


def fit_sigma(C_bins: np.ndarray, Nt: int, rmin: int = 2, rel_err_max: float = 0.3,
              min_points: int = 4) -> Optional[Dict]:
    """String tension of one coupling from the binned correlator C(r).

    F(r) = -T ln C(r) - T ln 4 (T = 1/Nt) is fitted with a0 - a1 / r + sigma r
    over r = rmin .. r_hi, r_hi the last r (consecutively from rmin) where
    C(r) is positive in every jackknife sample and its relative error is
    below rel_err_max; the fit is weighted by the jackknife errors of F, and
    the errors of the parameters come from fitting every jackknife sample.
    None when fewer than min_points separations qualify (deconfined
    couplings, where F flattens, or too noisy a correlator)."""
    C_bins = np.asarray(C_bins, dtype=np.float64)
    Cm, Ce, Cs = jackknife(C_bins)
    r_hi = rmin - 1
    for r in range(rmin, C_bins.shape[1]):
        if Cm[r] > 0 and np.all(Cs[:, r] > 0) and Ce[r] < rel_err_max * Cm[r]:
            r_hi = r
        else:
            break
    if r_hi - rmin + 1 < min_points:
        return None
    rs = np.arange(rmin, r_hi + 1, dtype=np.float64)

    def F_of(C):
        return analysis.free_energy(C[rmin:r_hi + 1], Nt)

    F, Fe, Fs = jackknife(C_bins, F_of)
    coef, _ = analysis.fit_string_tension(rs, F, Fe)
    per = np.array([analysis.fit_string_tension(rs, Fs[k], Fe)[0] for k in range(len(Fs))])
    nb = len(Fs)
    err = np.sqrt((nb - 1) / nb * np.sum((per - per.mean(0)) ** 2, axis=0))
    res = F - (coef[0] - coef[1] / rs + coef[2] * rs)
    chi2 = float(np.sum((res / Fe) ** 2))
    return {"a0": coef[0], "a1": coef[1], "sigma": coef[2], "a0_err": err[0],
            "a1_err": err[1], "sigma_err": err[2], "r_range": [rmin, r_hi],
            "chi2_dof": chi2 / max(len(rs) - 3, 1)}


def run_scan(betas: Sequence[float], Ns: int = 48, Nt: int = 4, therm: int = 500,
             meas: int = 2000, bin_sweeps: int = 50, rmax: int = 24,
             seeds: Optional[Sequence[int]] = None, autotune: bool = True,
             start: str = "hot") -> Dict:
    """Thermalise one lattice per coupling from a hot (Haar) or cold (unit)
    start, then measure in bins of bin_sweeps sweeps (the Polyakov loop and
    C(r), r = 0..rmax, after every sweep); returns the per-bin means."""
    import torch

    from . import su2

    n = len(betas)
    seeds = list(seeds) if seeds is not None else [1000 + i for i in range(n)]
    lat = su2.Lattice([Ns] * n, [Nt] * n, su2.F32)
    if autotune:
        lat.autotune(beta=list(betas))
    lat.batch_init(su2.HOT if start == "hot" else su2.COLD, seeds)
    lat.batch_heatbath(betas, therm, seeds, plaq=None)
    nb = meas // bin_sweeps
    L = np.zeros((nb, n))
    L_abs = np.zeros((nb, n))
    C = np.zeros((nb, n, rmax + 1))
    P = np.zeros((nb, n))
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev[0].record()
    for b in range(nb):
        plaq, ps, cs = lat.batch_heatbath_measure(betas, bin_sweeps, seeds, rmax)
        L[b], L_abs[b] = ps[0] / bin_sweeps, ps[1] / bin_sweeps
        C[b] = cs / bin_sweeps
        P[b] = plaq.mean(1)
    ev[1].record()
    torch.cuda.synchronize()
    seconds = ev[0].elapsed_time(ev[1]) / 1e3
    lat.close()
    return {"betas": list(map(float, betas)), "Ns": Ns, "Nt": Nt, "therm": therm, "start": start,
            "meas": nb * bin_sweeps, "bin_sweeps": bin_sweeps, "rmax": rmax, "seeds": seeds,
            "L": L, "L_abs": L_abs, "C": C, "plaquette": P,
            "measure_seconds": seconds,
            "link_updates_per_s": 4 * Ns ** 3 * Nt * n * nb * bin_sweeps / seconds}


def analyse(res: Dict, rmin: int = 2) -> Dict:
    """Jackknife means of the plaquette, L and |L|, beta_c, T / T_c and the
    string tension of every coupling (None where no fit qualifies)."""
    betas = np.asarray(res["betas"])
    Nt = res["Nt"]
    P, Pe, _ = jackknife(res["plaquette"])
    La, Lae, _ = jackknife(res["L_abs"])
    L, Le, _ = jackknife(res["L"])
    bc = beta_critical(betas, La)
    rows: List[Dict] = []
    for i, b in enumerate(betas):
        fit = fit_sigma(res["C"][:, i, :], Nt, rmin=rmin)
        row = {"beta": float(b), "plaquette": float(P[i]), "plaquette_err": float(Pe[i]),
               "L": float(L[i]), "L_err": float(Le[i]), "L_abs": float(La[i]),
               "L_abs_err": float(Lae[i]), "T_over_Tc": float(t_over_tc(b, bc))}
        if fit is not None:
            row.update({k: (float(v) if not isinstance(v, list) else v) for k, v in fit.items()})
            row["sigma_over_T2"] = row["sigma"] * Nt ** 2
            row["sigma_over_T2_err"] = row["sigma_err"] * Nt ** 2
        rows.append(row)
    return {"beta_c": bc, "rows": rows}


def table(an: Dict) -> str:
    """The analysis as a markdown table."""
    out = ["| beta | T/T_c | <P> | <abs L> | sigma a^2 | sigma/T^2 | fit r | chi2/dof |",
           "|---:|---:|---:|---:|---:|---:|---:|---:|"]
    for r in an["rows"]:
        s = (f"{r['sigma']:.4f}({round(r['sigma_err'] * 1e4):d}) | "
             f"{r['sigma_over_T2']:.3f}({round(r['sigma_over_T2_err'] * 1e3):d}) | "
             f"{r['r_range'][0]}..{r['r_range'][1]} | {r['chi2_dof']:.2f}"
             if "sigma" in r else "-- | -- | -- | --")
        out.append(f"| {r['beta']:.2f} | {r['T_over_Tc']:.3f} | {r['plaquette']:.5f} | "
                   f"{r['L_abs']:.4f}({round(r['L_abs_err'] * 1e4):d}) | {s} |")
    return "\n".join(out)


def main(argv=None):
    from . import inputs

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--points", type=int, default=21)
    ap.add_argument("--Ns", type=int, default=48)
    ap.add_argument("--Nt", type=int, default=4)
    ap.add_argument("--therm", type=int, default=500)
    ap.add_argument("--meas", type=int, default=2000)
    ap.add_argument("--bin", type=int, default=50)
    ap.add_argument("--rmax", type=int, default=24)
    ap.add_argument("--start", choices=["hot", "cold"], default="hot",
                    help="hot (Haar) or cold (unit links) start; a cold start avoids Z2 "
                         "domain walls on the deconfined side")
    ap.add_argument("--out", default=None, help="write the raw bins and the analysis as JSON")
    ap.add_argument("--analyse", default=None, metavar="JSON",
                    help="analyse the raw bins of an earlier --out file (no GPU)")
    args = ap.parse_args(argv)
    if args.analyse:
        with open(args.analyse) as f:
            raw = json.load(f)["raw"]
        res = {k: (np.asarray(v) if k in ("L", "L_abs", "C", "plaquette") else v)
               for k, v in raw.items()}
        an = analyse(res)
        print(f"beta_c = {an['beta_c']:.4f}; {res['Ns']}^3x{res['Nt']}, {res['start']} start, "
              f"{res['therm']} + {res['meas']} sweeps, bins of {res['bin_sweeps']}")
        print(table(an))
        return 0
    scan = inputs.temperature_scan(args.points, args.Ns, args.Nt)
    res = run_scan([e["beta"] for e in scan], args.Ns, args.Nt, args.therm, args.meas, args.bin,
                   args.rmax, [e["seed"] for e in scan], start=args.start)
    an = analyse(res)
    print(f"beta_c = {an['beta_c']:.4f}; {res['link_updates_per_s'] / 1e9:.1f} G link "
          f"updates/s over the measured sweeps")
    print(table(an))
    if args.out:
        raw = {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in res.items()}
        with open(args.out, "w") as f:
            json.dump({"raw": raw, "analysis": an}, f)
    return 0


if __name__ == "__main__":
    sys.exit(main())
