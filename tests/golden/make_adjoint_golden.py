"""Writes adjoint_256x96.json: the oracle's reference gradient of the two
objectives of oracle/gradient.py (final <n_ee> and log <|n_emu|>) with respect
to the uniform species (n_nu, n_nubar, f_nu, f_nubar) of the 256-cell x
96-direction growth-phase box, after 400 RK4 steps at the fixed step of Eq. 7
for the unperturbed input.  Central differences, h = 1e-6 relative.

Calls only oracle/ (and the seeded input generator).  Run from the repository
root:  python tests/golden/make_adjoint_golden.py  (16 oracle runs of 400
steps; about two minutes on 8 cores).
"""
import json
import os
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parents[1]))

import numpy as np  # noqa: E402

from oracle import gradient, oracle  # noqa: E402
from paper_2101_02745_gb300 import workloads  # noqa: E402


def main():
    wl = workloads.adjoint_box()
    kw = dict(nz=wl.nz, ndir=wl.ndir, Lz=wl.Lz, kappa=wl.kappa, c_light=wl.c_light, cfl_adv=wl.cfl_adv,
              cfl_flavor=wl.cfl_flavor, area=wl.area)
    cfg = oracle.config(**kw)
    parts = oracle.init(cfg, wl.n_nu, wl.n_nubar, wl.f_nu, wl.f_nubar, wl.alpha, wl.seed)
    dt = oracle.timestep(cfg, oracle.deposit(cfg, parts))
    theta = np.concatenate([[wl.n_nu[0], wl.n_nubar[0]], wl.f_nu[0], wl.f_nubar[0]])
    h = 1e-6
    L = gradient.evaluate(kw, theta, wl.alpha, wl.seed, dt, wl.steps)
    g = gradient.fd_gradient(kw, theta, wl.alpha, wl.seed, dt, wl.steps, h=h, processes=os.cpu_count() or 1)
    out = {
        "source": "oracle central differences (oracle/gradient.py), written by tests/golden/make_adjoint_golden.py",
        "workload": wl.name, "config": kw, "alpha": wl.alpha, "seed": wl.seed, "nsteps": wl.steps, "dt": dt,
        "h": h, "params": list(gradient.PARAMS), "theta": theta.tolist(),
        "objectives": ["<n_ee>", "log <|n_emu|>"], "values": L.tolist(), "gradient": g.tolist(),
    }
    (HERE / "adjoint_256x96.json").write_text(json.dumps(out, indent=1) + "\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
