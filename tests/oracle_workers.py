"""Oracle evaluations for process pools (test infrastructure).

Kept apart from the test modules so that a spawned worker imports only the
oracle and the seeded input generator (not torch), and runs single-threaded.
"""
import os


def single_threaded():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")


def lightcone_zz(args):
    """<Z_j Z_k> of (workload name, batch, edge, angle set) by the oracle's
    lightcone contraction."""
    from oracle import lightcone as lc
    from workloads import workload
    name, batch, e, k = args
    n, edges, p, g, b = workload(name, batch=batch)
    return lc.lightcone_zz(n, edges, p, g[k], b[k], e)[0]
