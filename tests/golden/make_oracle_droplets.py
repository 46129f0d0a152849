"""Writes oracle_droplets_100k.json: the FP64 oracle's state after 100000
well-balanced steps of the stationary droplets of the Laplace test (256^2,
R = 40 and 60, W = 4, rho_l = 1, rho_g = 0.1, kappa = 0.01, tau = 1.0,
rho0 = 0): the bulk densities, max|u|, the mu spread, the mass and the
density along the row through the centre.  Calls only the oracle (and the
seeded input generator); the GPU test compares the CUDA path with these
values.  Run: python tests/golden/make_oracle_droplets.py (about 8 minutes
with the all-cores oracle build)."""
import json
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle.oracle import WELL_BALANCED, Oracle, Params  # noqa: E402
from paper_2012_11075_gb300 import workloads as wl  # noqa: E402

STEPS = 100000


def main():
    out = {"steps": STEPS, "scheme": "well_balanced", "cases": {}}
    for radius in (40.0, 60.0):
        pr = wl.droplet(n=256, radius=radius, tau=1.0)
        o = Oracle(Params(pr.nx, pr.ny, pr.tau, pr.kappa, pr.beta, pr.rho_l, pr.rho_g, 0.0,
                          WELL_BALANCED), openmp=True)
        f = o.init(pr.rho)
        o.step(f, STEPS)
        m, st = o.macro(f), o.stats(f)
        out["cases"][f"R{int(radius)}"] = {
            "radius": radius, "rho_in": float(m["rho"][128, 128]),
            "rho_out": float(m["rho"][0, 0]), "umax": st["umax"],
            "mu_spread": st["mu_max"] - st["mu_min"], "mass": st["mass"],
            "rho_row128": [float(v) for v in m["rho"][128, :]],
        }
    path = Path(__file__).resolve().parent / "oracle_droplets_100k.json"
    path.write_text(json.dumps(out, indent=1) + "\n")
    print(f"wrote {path}")


if __name__ == "__main__":
    main()
