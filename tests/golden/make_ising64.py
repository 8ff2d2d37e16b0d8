"""Write ising64_chi128.json: oracle values for the 64x64 Ising beta sweep at chi = 128.

Workload: 64 x 64 open square lattice, J = 1, the paper's symmetric W on every
bond (SI "Ising model"), the row-by-row boundary tree with compressions after
each row (Sec. "Bond compression strategies"; boundary contraction), chi = 128,
beta_t = 0.2 + 0.5 t / 255 for a subset of t.  For each beta the oracle
(oracle/approx.py, FP64) is run on the network as built and on copies whose
tensor 0 is scaled by (1 + eps) for eps in +-1e-15, +-3e-15; since scaling one
tensor by c shifts ln|Z| by exactly ln c, the spread of ln|Z| - ln(1 + eps)
over those runs is the rounding sensitivity ("chaos band") of the truncated
contraction at this beta.  Also stored: the smallest relative gap
(s_k - s_{k+1}) / s_1 at any executed cut.

Only the oracle and the seeded input builders are called.  Usage:
    python tests/golden/make_ising64.py [--procs 8]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
L, CHI, N_BETA = 64, 128, 256
T_SUBSET = [0, 61, 110, 123, 184, 255]
EPS = [0.0, 1e-15, -1e-15, 3e-15, -3e-15]


def run_one(args):
    t, eps = args
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from tn_inputs import networks as nw
    from tn_inputs import trees as tr
    from oracle import approx
    beta = float(nw.beta_sweep(N_BETA)[t])
    n, edges = nw.square_lattice(L, L)
    net = nw.ising_network(n, edges, beta)
    net.data[0] = net.data[0] * (1.0 + eps)
    t0 = time.time()
    r = approx.contract(net, tr.boundary_rows(L, L), CHI)
    return t, eps, beta, r.logabs - math.log1p(eps), r.sign, min(g for _, _, g in r.diag), time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    jobs = [(t, e) for t in T_SUBSET for e in EPS]
    with mp.get_context("spawn").Pool(args.procs) as pool:
        res = pool.map(run_one, jobs)
    out = {"workload": f"{L}x{L} open square lattice Ising, J=1, symmetric W, boundary-row tree, chi={CHI}",
           "beta_rule": f"beta_t = 0.2 + 0.5 t / {N_BETA - 1}", "eps": EPS, "entries": []}
    for t in T_SUBSET:
        rows = [r for r in res if r[0] == t]
        base = [r for r in rows if r[1] == 0.0][0]
        vals = [r[3] for r in rows]
        out["entries"].append({"t": t, "beta": base[2], "logabsz": base[3], "sign": base[4],
                               "spread_rel": (max(vals) - min(vals)) / abs(base[3]),
                               "perturbed_logabsz": vals, "min_gap": min(r[5] for r in rows),
                               "oracle_s": base[6]})
    with open(os.path.join(HERE, "ising64_chi128.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
