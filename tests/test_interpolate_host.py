"""Host interpolation of node values on a tree (refine.interpolate), used to measure how well an
output tree resolves u between its nodes: exact for tensor polynomials of degree < k, on CPU."""
import numpy as np

from paper_2305_07165_gb300 import refine as R
import workloads as W


def test_interpolation_is_exact_for_polynomials():
    rng = np.random.default_rng(2)
    for d, k in ((2, 6), (3, 4)):
        tr = W.random_balanced_tree(d, 5, max_level=4 if d == 2 else 3, min_level=1)
        coef = rng.standard_normal((k,) * d) * 0.5

        def poly(X):
            v = np.zeros(X.shape[:-1])
            for alpha in np.ndindex(*coef.shape):
                term = coef[alpha]
                for a in range(d):
                    term = term * X[..., a] ** alpha[a]
                v = v + term
            return v
        u = poly(W.node_positions(tr, k))
        pts = rng.uniform(-0.5, 0.5, size=(500, d))
        got = R.interpolate(tr.level, tr.coord, u, d, k, pts)
        assert np.abs(got - poly(pts)).max() <= 1e-12 * np.abs(poly(pts)).max()
