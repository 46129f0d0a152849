"""Edge-case workloads run through the library that WBLBE_LIBRARY names (the
bounds-checked build, in test_gpu_bounds.py); prints the number of
out-of-bounds accesses its kernels saw as one JSON line."""
import json

import numpy as np

from paper_2012_11075_gb300 import wblbe
from paper_2012_11075_gb300 import workloads as wl

SHAPES = [(3, 3), (1, 17), (17, 1), (5, 2), (67, 129), (130, 70), (257, 33), (64, 80)]


def main():
    wblbe.debug_bounds_errors(reset=True)
    runs = 0
    for prec in (wblbe.FP64, wblbe.FP32_SHIFTED):
        for sch in (wblbe.STANDARD, wblbe.WELL_BALANCED, wblbe.STANDARD_PRESSURE,
                    wblbe.STANDARD_TEXTBOOK, wblbe.STANDARD_E6):
            if sch == wblbe.STANDARD_E6 and prec != wblbe.FP64:
                continue
            for nx, ny in SHAPES:
                rng = np.random.default_rng(nx * 1000 + ny)
                rho = 0.6 + 0.3 * rng.uniform(-1, 1, (ny, nx))
                s = wblbe.Solver(wblbe.Params(nx, ny, 0.85, 0.0128, 0.01, 1.0, 0.2,
                                              scheme=sch, precision=prec))
                s.init_rho(rho)
                for tile in (32, 64, 128, 256):
                    for rows in (1, 3, 16):
                        s.set_launch(tile, rows)
                        s.step(3)
                s.moments()
                s.moments(device=True)
                s.close()
                runs += 1
    specs = wl.batched_case_specs(count=12, seed=9, side_min=8, side_max=70)
    for prec in (wblbe.FP64, wblbe.FP32_SHIFTED):
        for cfg in ((32, 4, 2), (64, 8, 3), (256, 16, 1)):
            b = wblbe.Batch(scheme=wblbe.WELL_BALANCED, precision=prec, max_cases=len(specs),
                            max_tiles=4096, max_case_nodes=70 * 70, arena_bytes=64 << 20,
                            tile_x=cfg[0], rows_per_tile=cfg[1], steps_per_launch=cfg[2])
            ids = []
            for sp in specs:
                p = wblbe.Params(sp["nx"], sp["ny"], sp["tau"], sp["kappa"], sp["beta"],
                                 sp["rho_l"], sp["rho_g"], scheme=wblbe.WELL_BALANCED,
                                 precision=prec)
                ids.append((b.admit(p, wl.case_field(sp), 0.0, 10 ** 6), sp))
            b.advance(4)
            for cid, sp in ids:
                b.fetch(cid, (sp["ny"], sp["nx"]))
            b.close()
            runs += 1
    print(json.dumps({"errors": wblbe.debug_bounds_errors(), "runs": runs}), flush=True)


if __name__ == "__main__":
    main()
