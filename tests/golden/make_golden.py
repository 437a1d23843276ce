"""Writes tests/golden/oracle_c1.json from the FP64 oracle only.

The paper prints no worked example that its stated parameters reproduce
(Table I needs scattering lengths, box and noise that Sec. VI.A does not give),
so the stored values are the oracle's own outputs on the seeded C1 workload:
a regression pin that makes any later change of the oracle's arithmetic
visible.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2510_24543_gb300 import inputs as I  # noqa: E402


def c1_case():
    w = I.PRESETS["c1"]
    g = O.Grid(w.n, w.L)
    prm = O.Params(w.g, w.gdd, w.kappa, w.eta_s, w.lhy_nodes, w.trap)
    return w, g, prm, I.gaussian_start(w)


def main():
    w, g, prm, psi = c1_case()
    ev = O.evaluate(g, prm, psi)
    p = O.project(g, psi, I.raw_direction(w.n, w.L, 77))
    E0, Ep, Epp = O.line_coeffs(g, prm, psi, p, ev)
    _, rep = O.ncg_solve(g, prm, psi, O.SolveOpts(precond="kinetic+diagonal", tol_res=1e-10))
    out = dict(
        source="oracle (FP64 NumPy), seeded C1 workload 32^3 on [-8,8]^3, seed 1001",
        initial=dict(E=ev.E, mu=ev.mu.tolist(), terms={k: float(v) for k, v in ev.terms.items()}),
        line_coeffs=dict(direction_seed=77, E0=E0, Ep=Ep, Epp=Epp),
        ground_state=dict(precond="kinetic+diagonal", tol_res=1e-10, E=rep["E"], mu=rep["mu"].tolist(),
                          iters=rep["iters"], status=rep["status"]),
    )
    with open(os.path.join(HERE, "oracle_c1.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
