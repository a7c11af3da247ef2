"""The small systems of the solver-level parity tests and the oracle's iteration band on them.

No GPU and no torch here: the CPU pins and the GPU parity tests share this list.
"""
import oracle as O
from paper_2407_15973_gb300 import problems as PB

PROBLEMS = {
    "poisson2d_bs8": lambda: PB.make_problem("poisson2d", bs=8),
    "subcube24_bs32": lambda: PB.make_problem("subcube3d", seed=1, m=24, bs=32),
    "subcube24_bs64": lambda: PB.make_problem("subcube3d", seed=2, m=24, bs=64),
    "aniso27_12_bs64": lambda: PB.make_problem("aniso27", seed=3, m=12, bs=64),
    "voronoi24_uneven": lambda: PB.make_problem("voronoi3d", seed=4, m=24),
    "ragged13_bs32": lambda: PB.make_problem("subcube3d", seed=5, m=13, bs=32),
}

DOT_ORDERS = (O.DOT_SEQUENTIAL, O.DOT_REVERSED, O.DOT_PAIRWISE, O.DOT_STRIDED, O.DOT_COMPENSATED)


def uniform_iteration_band(pr, b, P, tol=1e-10, maxit=3000):
    """(fewest, most) iterations of the oracle's uniform binary64 BJAC-PCG over the five
    summation orders of its dot products. PCG (Section 3.2) fixes no order for a dot product,
    so each order is an equally valid evaluation; a GPU reduction is one more."""
    its = []
    old = O.set_dot_order(O.DOT_SEQUENTIAL)
    try:
        for order in DOT_ORDERS:
            O.set_dot_order(order)
            res = O.pcg(pr.A, P, b, tol=tol, maxit=maxit)
            assert res["converged"]
            its.append(res["iters"])
    finally:
        O.set_dot_order(old)
    return min(its), max(its)
