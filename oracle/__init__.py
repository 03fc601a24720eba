"""The oracle: a plain, slow, exact CPU statement of what the degree path computes.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, calls or links
anything in this directory; only the tests, the smoke check of `__graft_entry__`
and the CPU-baseline leg of `bench.py` may use it.  It shares no code with the CUDA
path (different language, different algorithms); the only inputs both sides see
come from `workloads/`, which holds none of the method's arithmetic.

Contents (all arithmetic is exact: Python integers and `fractions.Fraction`):

* `snf`        -- Smith Normal Form with unimodular transforms by Bezout row/column
                  reductions (Sec. 3), rank, torsion |prod d_j| (Prop. 1),
                  consistency b^{Q_0} = 1 (Prop. 2), kernel points P_0 (Prop. 4).
* `volume`     -- normalized volume NVol_k(conv S) = k! Vol_k(conv S) (Sec. 4,
                  Eq. deg-nvol) by two independent exact algorithms:
                  facet-enumeration pyramid decomposition, and a placing
                  (beneath-beyond) triangulation.
* `lower_facet`-- the lower-facet test of one lifted subset written as the inequality
                  system of Eq. lower-face (strict form of Sec. 5), solved in
                  rationals; a brute-force lifting volume built on it for tiny inputs.
* `lifts`      -- the counter-based lift generator (splitmix64, Steele-Lea-Flood 2014)
                  implemented from its published definition.
* `degree`     -- degree = |prod d_j| * NVol_d(conv{0, columns of P_0}) (Props. 1, 4).
* `cells`, `start` -- the cells of the lifting's triangulation with their inner normals
                  and the start solutions of every cell's binomial system (Sec. 6).
* `mixed`      -- the mixed volume of k point sets (the BKK bound that Appendix A names
                  as the general case of the degree): by the polarization formula over
                  Minkowski sums, and by the fine mixed cells of a lifting in rationals.
* `mlp`        -- the cost model's forward and backward passes in float64.

Parity status: every function here is pinned by tests against closed forms, the
paper's worked example and its master-space degree table; see tests/test_oracle_*.py.
"""
