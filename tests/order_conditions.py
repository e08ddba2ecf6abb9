"""Order conditions of additive (two-part) Runge-Kutta pairs, derived from
rooted trees with two node colours (Butcher series of ARK methods): for every
tree t of order <= p and every colouring, sum_i b^{c(root)}_i Phi_i(t) = 1/gamma(t)."""
import itertools

import numpy as np


def rooted_trees(order):
    """All rooted trees with 1..order nodes as nested tuples of children."""
    memo = {1: [()]}

    def gen(n):
        if n in memo:
            return memo[n]
        out = set()

        def parts(rem, bound):
            if rem == 0:
                yield ()
                return
            for k in range(min(rem, bound[0]), 0, -1):
                for t in gen(k):
                    if (k, t) <= bound:
                        for rest in parts(rem - k, (k, t)):
                            yield ((k, t),) + rest

        for p in parts(n - 1, (n, ())):
            out.add(tuple(t for _, t in p))
        memo[n] = sorted(out)
        return memo[n]

    res = []
    for n in range(1, order + 1):
        res += gen(n)
    return res


def size(t):
    return 1 + sum(size(c) for c in t)


def density(t):
    g = size(t)
    for c in t:
        g *= density(c)
    return g


def max_violation(AE, AI, bE, bI, order):
    A = {"E": np.asarray(AE, float), "I": np.asarray(AI, float)}
    b = {"E": np.asarray(bE, float), "I": np.asarray(bI, float)}
    s = A["E"].shape[0]
    worst = 0.0
    for t in rooted_trees(order):
        for cols in itertools.product("EI", repeat=size(t)):
            it = iter(cols)

            def phi(tree):
                v = np.ones(s)
                for c in tree:
                    col = next(it)
                    v = v * (A[col] @ phi(c))
                return v

            rc = next(it)
            w = b[rc] @ phi(t)
            worst = max(worst, abs(w - 1.0 / density(t)))
    return worst
