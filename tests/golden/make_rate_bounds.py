"""Writes rate_bounds.json: iteration counts implied by Eq. (conv_rate).

gamma_FFTH = (rho - 1)/(rho + 1), gamma_CG = (sqrt(rho) - 1)/(sqrt(rho) + 1);
eta_r^m <= gamma^m eta_r^0 reaches eps after ceil(ln eps / ln gamma) steps.
Pure arithmetic on the paper's closed forms (Section 3.2); no solver runs.
"""
import json
import math
import os

RHO = [1e1, 1e2, 1e3, 1e4]
EPS = [1e-4, 1e-6, 1e-8]


def main():
    rows = []
    for rho in RHO:
        gf = (rho - 1.0) / (rho + 1.0)
        gc = (math.sqrt(rho) - 1.0) / (math.sqrt(rho) + 1.0)
        rows.append({
            "ffth": [math.ceil(math.log(e) / math.log(gf)) for e in EPS],
            "cg": [math.ceil(math.log(e) / math.log(gc)) for e in EPS],
        })
    out = {
        "source": "Eq. (conv_rate), Section 3.2: ceil(ln eps / ln gamma)",
        "rho": RHO,
        "eps": EPS,
        "rows": rows,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rate_bounds.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
