"""Writes oracle_small_case.json: oracle outputs (Eq. render with Eq. accu,
Eq. loss and the gradient) for one small seeded case.  Calls only the oracle
and the seeded input generators.  Re-run only when a change to the oracle's
arithmetic is justified by a passage of the paper, and say which in the
commit message."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2509_25075_gb300 import synthetic as syn  # noqa: E402


def main():
    w = syn.Workload("golden", d=16, M=12, B=2, apix=1.2)
    params = syn.gaussians(w)
    R, t = syn.views(w)
    prm = syn.ctf_params(w)
    imgs = syn.images(w)
    proj = oracle.project(params, R, t, w.d, w.apix, w.tau)
    H = oracle.ctf_grid_from_params(prm, w.d, w.apix)
    L, _, _, g = oracle.loss(H, proj, imgs)
    G = oracle.grad(params, R, t, w.d, w.apix, w.tau, g)
    out = {
        "case": "d=16 M=12 B=2 apix=1.2 seed=0, tau = workload default, norm_mode 0, CTF from parameters",
        "loss": L,
        "proj_sums": proj.sum(axis=(1, 2)).tolist(),
        "grad": G.tolist(),
    }
    with open(os.path.join(HERE, "oracle_small_case.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
