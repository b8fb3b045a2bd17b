"""Seeded synthetic inputs (no arithmetic of the method).

A module of its own: the CUDA library and the oracle never import it; tests
and the benchmark draw instances here and pass the same numbers to both.

Random parameters are drawn with splitmix64 (to seed) and xoshiro256**
(Blackman & Vigna, "Scrambled linear pseudorandom number generators", 2018),
written here from their published definitions, so that every consumer of a
seed gets the same numbers.  Both the tests (CPU oracle and GPU library) and the
benchmark take their instances from here.
"""
import math

MASK = (1 << 64) - 1
DEFAULT_SEED = 20190201


def _rotl(x, k):
    return ((x << k) | (x >> (64 - k))) & MASK


class Xoshiro256ss:
    def __init__(self, seed=DEFAULT_SEED):
        s = seed & MASK
        self.s = []
        for _ in range(4):  # splitmix64
            s = (s + 0x9E3779B97F4A7C15) & MASK
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
            self.s.append(z ^ (z >> 31))

    def next(self):
        s = self.s
        r = (_rotl((s[1] * 5) & MASK, 7) * 9) & MASK
        t = (s[1] << 17) & MASK
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return r

    def uniform(self, lo=0.0, hi=1.0):
        return lo + (hi - lo) * ((self.next() >> 11) * (1.0 / (1 << 53)))

    def integer(self, lo, hi):
        """Uniform integer in [lo, hi]."""
        return lo + self.next() % (hi - lo + 1)


def forest_trees(n=64, seed=DEFAULT_SEED):
    """Independent 2D advection instances: Gaussian centre in [0,1)^2, sigma in
    [0.02, 0.1], constant velocity components in [-1, 1], Jmax uniform in 4..8,
    log10 eps uniform in [-5, -3], Jmin 2, 17^2 blocks."""
    g = Xoshiro256ss(seed)
    trees = []
    for _ in range(n):
        cx, cy = g.uniform(), g.uniform()
        sigma = g.uniform(0.02, 0.1)
        u, v = g.uniform(-1.0, 1.0), g.uniform(-1.0, 1.0)
        jmax = g.integer(4, 8)
        eps = 10.0 ** g.uniform(-5.0, -3.0)
        trees.append(dict(Jmin=2, Jmax=jmax, eps=eps, ic="gauss", ic_params=(cx, cy, 0.0, sigma),
                          rhs_params=(u, v, 0.0)))
    return trees


def cfl_dt(tree, Bs=17, cfl=0.5, umax=None):
    """Time step of the harness: cfl * dx at the tree's finest level / max |u|."""
    if umax is None:
        umax = math.hypot(*tree["rhs_params"][:2]) or 1.0
    return cfl * (1.0 / ((Bs - 1) * (1 << tree["Jmax"]))) / umax


def mixing_layer_perturbation(seed=DEFAULT_SEED, modes=8):
    """Amplitudes a_k in [-1, 1] and phases phi_k in [0, 2 pi) of the seeded
    streamwise perturbation modes of the temporal mixing layer."""
    g = Xoshiro256ss(seed)
    a = [g.uniform(-1.0, 1.0) for _ in range(modes)]
    phi = [g.uniform(0.0, 2.0 * math.pi) for _ in range(modes)]
    return a, phi


def cnn_init_params(nparam_shapes, seed=DEFAULT_SEED):
    """He-normal initial weights of the proposal network (biases zero), drawn
    with Box-Muller from the seeded generator.  nparam_shapes: list of shapes in
    packing order; 4-D shapes are convolutions (fan-in = in_channels * 9), the
    last 1-D shape of length > 1 is the linear layer (fan-in = its length)."""
    import numpy as np
    g = Xoshiro256ss(seed)

    def normal(n):
        out = np.empty(n)
        for i in range(0, n, 2):
            u1 = max(g.uniform(), 1e-300)
            u2 = g.uniform()
            r = math.sqrt(-2.0 * math.log(u1))
            out[i] = r * math.cos(2 * math.pi * u2)
            if i + 1 < n:
                out[i + 1] = r * math.sin(2 * math.pi * u2)
        return out
    parts = []
    linear = max(k for k, s in enumerate(nparam_shapes) if len(s) == 1 and s[0] > 1)
    for k, s in enumerate(nparam_shapes):
        n = int(np.prod(s))
        if len(s) == 4:
            parts.append(normal(n) * math.sqrt(2.0 / (s[1] * 9)))
        elif k == linear:
            parts.append(normal(n) * math.sqrt(1.0 / s[0]))
        else:
            parts.append(np.zeros(n))
    return np.concatenate(parts)
