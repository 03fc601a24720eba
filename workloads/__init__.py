"""Seeded synthetic inputs shared by the tests, the oracle scripts and the benchmark.

This package only *draws* inputs: exponent matrices of binomial systems, random
point sets, supports of sparse systems and arrival times.  It holds none of the degree method's arithmetic
(no Smith form, no kernel basis, no volume, no lifting) so that the CUDA path and
the CPU oracle can both consume the same inputs without sharing any code that
could hide a common mistake.
"""

from .generators import (  # noqa: F401
    BinomialSystem,
    random_binomial_system,
    quiver_binomial_system,
    config_system,
    batch_systems,
    master_space_system,
    random_points,
    poisson_arrivals,
    sparse_supports,
    mixed_config,
    CONFIGS,
    MIXED_CONFIGS,
)
