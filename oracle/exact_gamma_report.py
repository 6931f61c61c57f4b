"""How the oracle's exact entropic gamma is decided on the 64^3 randomized Taylor-Green
ensemble at Re = 800, Ma = 0.025 (test infrastructure: calls only the oracle).

Runs one or more samples with the exact gamma (Eq. (kbc_entropy), minimised over
0 <= gamma <= 4 / omega) and prints, per window of steps, the share of node updates whose
minimiser is an interior root (the paper's unconstrained argmin), an end point of the
interval (the constraint binds), or kept at the closed form because no gamma keeps every
post-collision population positive, and the share with Dh = 0.

  python oracle/exact_gamma_report.py [--N 64] [--M 1] [--steps 100] [--window 10]
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    import ensemble_inputs as gen
    import oracle
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--M", type=int, default=1)
    ap.add_argument("--Re", type=float, default=800.0)
    ap.add_argument("--Ma", type=float, default=0.025)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--window", type=int, default=10)
    ap.add_argument("--seed", type=int, default=1)
    a = ap.parse_args()
    un = oracle.units(a.N, a.Re, a.Ma)
    f = oracle.init_ensemble(a.N, gen.draw_params(a.seed, a.M), un["ulat"])
    rows = []
    total = dict.fromkeys(("dh_zero", "empty", "lower_end", "upper_end", "interior"), 0)
    for w0 in range(0, a.steps, a.window):
        with oracle.exact_gamma() as ex:
            for _ in range(min(a.window, a.steps - w0)):
                oracle.step(f, un["omega"])
            c = ex.counts()
        n = sum(c.values())
        for k in total:
            total[k] += c[k]
        rows.append({"steps": [w0 + 1, w0 + min(a.window, a.steps - w0)], **{k: v / n for k, v in c.items()}})
    n = sum(total.values())
    print(json.dumps({"config": {"N": a.N, "M": a.M, "Re": a.Re, "Ma": a.Ma, "omega": un["omega"], "steps": a.steps},
                      "windows": rows, "all_steps": {k: v / n for k, v in total.items()}}, indent=1))


if __name__ == "__main__":
    main()
