"""URand lambda sweep on the oracle (Sec. "Hardness transition in random tensor networks").

Tensor entries uniform in [lambda, 1]: with positive entries the approximate
contraction converges quickly in chi, while towards lambda = -1 the sign
structure makes Z essentially impossible to approximate at any moderate chi.
On an 8 x 8 lattice, D = 3, boundary rows, against the exact contraction
(the same tree with no truncation), for three seeds:

  lambda = 0:   |dZ/Z| < 1e-5 at chi = 16 and at least 10x below chi = 4
                (measured 2.6e-7, 4.2e-7, 2.2e-7);
  lambda = -1:  the sign is wrong or |dZ/Z| > 0.1 at chi = 16 as at chi = 4
                (measured: two wrong signs, 0.58).

Median |dZ/Z| over seeds 0..3 at chi = 2, 4, 8, 16 (same lattice) show the
transition between lambda = -0.6 and -0.4:
  -1.0: 2.0, 2.0, 0.77, 1.3      -0.4: 5.2e-2, 5.1e-3, 1.1e-3, 7.1e-4
  -0.6: 2.0, 1.4, 0.10, 0.35      0.0: 1.0e-3, 3.3e-5, 2.3e-6, 3.4e-7
(2.0 = wrong sign).
"""
import math

from oracle import approx
from tn_inputs import networks as nw
from tn_inputs import trees as tr


def _rel_dz(net, tree, chi, exact):
    r = approx.contract(net, tree, chi)
    if r.sign != exact.sign:
        return math.inf
    return abs(math.expm1(r.logabs - exact.logabs))


def test_urand_hardness_transition():
    n, e = nw.square_lattice(8, 8)
    tree = tr.boundary_rows(8, 8)
    for seed in range(3):
        pos = nw.random_network(n, e, 3, seed=seed, dist="uniform", lam=0.0)
        ex = approx.contract(pos, tree, 10 ** 6)
        e4, e16 = _rel_dz(pos, tree, 4, ex), _rel_dz(pos, tree, 16, ex)
        assert e16 < 1e-5 and e16 * 10 < e4, (seed, e4, e16)
        mixed = nw.random_network(n, e, 3, seed=seed, dist="uniform", lam=-1.0)
        ex = approx.contract(mixed, tree, 10 ** 6)
        assert _rel_dz(mixed, tree, 16, ex) > 0.1, seed
