"""Count the iterations the oracle's plain CG (Sec. 3.2.3, from zero) needs to
reach a relative residual of 1e-8 on the benchmark workloads, and write them
to oracle/plain_cg_iterations.json.

bench.py's reference arm times a bounded sample of the oracle (a few CG
iterations and time steps) and extrapolates the whole pass with these counts,
the oracle's own. Test infrastructure, like the rest of oracle/.

    python oracle/plain_cg_iterations.py            # all three workloads
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as orc  # noqa: E402
from paper_2607_28414_b300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "plain_cg_iterations.json")


def count(w, tol=1e-8):
    t0 = time.time()
    _, _, status, st = orc.project(*w.force, w.dx, tol=tol)
    assert status == "converged", status
    return {"iters": st["iters"], "rel_res": st["rel_res"], "true_rel_res": st["true_rel_res"],
            "grid": [w.nx, w.ny, w.nz], "seconds": round(time.time() - t0, 1)}


def main():
    res = json.load(open(OUT)) if os.path.exists(OUT) else {}
    todo = sys.argv[1:] or ["sweep", "inclusions256", "bone512"]
    for name in todo:
        if name == "inclusions256":
            w = inputs.heterogeneous_inclusions(n=256)
        elif name == "bone512":
            w = inputs.bone_shell()
        else:
            w = inputs.sweep_cases(n_steps=1000)[0]
        res[name] = count(w)
        print(name, res[name], flush=True)
        json.dump(res, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main()
