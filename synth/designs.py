"""Counter-based design generator and square-wall load cases.

Design fractions: per element, the n_phase fractions are a Dirichlet(1,...,1)
draw built from normalised Exp(1) variates.  Every variate comes from a
counter-based generator, so the same (seed, mesh, n_phase) gives the same
design in any language:

    u(e, i) = ((splitmix64(seed XOR (e*n_phase + i)) >> 11) + 1) * 2**-53
    g(e, i) = -log(u(e, i))
    x(e, i) = g(e, i) / sum_k g(e, k)

splitmix64 is the output function of Steele, Lea and Flood's SplitMix64
generator ("Fast splittable pseudorandom number generators", OOPSLA 2014):
add the golden-ratio increment 0x9E3779B97F4A7C15, then two xor-shift-multiply
rounds and a final xor-shift.  Applied to a counter it is a stateless hash.

Loads (the square wall, bottom edge clamped):
  * top-edge case: f_y = -1 at every node of the top edge, corners included;
  * right-edge case: f_x = +1 at every node of the right edge.  The
    bottom-right node is clamped, so its load is dropped by the solver.
"""

import numpy as np

BOTTOM, LEFT, RIGHT, TOP = 1, 2, 4, 8

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(z):
    """SplitMix64 output function applied to uint64 counters (vectorised)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed, counters):
    """Uniform variates in (0, 1] with 53 random bits, one per counter."""
    c = np.asarray(counters, dtype=np.uint64) ^ np.uint64(seed)
    bits = splitmix64(c) >> np.uint64(11)
    return (bits.astype(np.float64) + 1.0) * 2.0**-53


def dirichlet_design(nelx, nely, n_phase, seed, chunk=1 << 22):
    """Per-element Dirichlet(1,...,1) phase fractions, float64 [n_phase][nely][nelx]."""
    n_el = nelx * nely
    out = np.empty((n_phase, n_el), dtype=np.float64)
    for s in range(0, n_el, chunk):
        e = np.arange(s, min(n_el, s + chunk), dtype=np.uint64)
        ctr = e[None, :] * np.uint64(n_phase) + np.arange(n_phase, dtype=np.uint64)[:, None]
        g = -np.log(uniform01(seed, ctr))
        out[:, s:s + len(e)] = g / g.sum(axis=0, keepdims=True)
    return out.reshape(n_phase, nely, nelx)


def _signed64(v):
    return v - (1 << 64) if v >= (1 << 63) else v


def dirichlet_design_torch(nelx, nely, n_phase, seed, device, chunk=1 << 22):
    """dirichlet_design computed with torch on `device` (for designs too large
    to build on the host): the same counters and the same 53-bit variates,
    with the uint64 arithmetic done in int64 (products and sums wrap modulo
    2^64 alike; right shifts are made logical by masking).  The logarithm is
    torch's, so fractions may differ from the numpy version in the last bit."""
    import torch

    g_inc, m1, m2 = (_signed64(int(v)) for v in (_GAMMA, _M1, _M2))

    def lsr(z, k):
        return (z >> k) & ((1 << (64 - k)) - 1)

    n_el = nelx * nely
    out = torch.empty((n_phase, n_el), dtype=torch.float64, device=device)
    ph = torch.arange(n_phase, dtype=torch.int64, device=device)[:, None]
    for s in range(0, n_el, chunk):
        e = torch.arange(s, min(n_el, s + chunk), dtype=torch.int64, device=device)
        z = (e[None, :] * n_phase + ph) ^ seed
        z = z + g_inc
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        z = z ^ lsr(z, 31)
        g = -torch.log((lsr(z, 11).to(torch.float64) + 1.0) * 2.0**-53)
        out[:, s:s + e.numel()] = g / g.sum(dim=0, keepdim=True)
    return out.reshape(n_phase, nely, nelx)


def batch_sizes(n, seed, choices=(128, 256, 512, 1024)):
    """n square mesh sizes drawn uniformly from `choices` by the counter-based generator."""
    u = uniform01(seed, np.arange(n, dtype=np.uint64))
    idx = np.minimum((u * len(choices)).astype(np.int64), len(choices) - 1)
    return [int(choices[i]) for i in idx]


def load_top_edge(nelx, nely, value=-1.0):
    """f_y = value at every top-edge node; layout [nely+1][nelx+1][2]."""
    f = np.zeros((nely + 1, nelx + 1, 2), dtype=np.float64)
    f[nely, :, 1] = value
    return f


def load_right_edge(nelx, nely, value=1.0):
    """f_x = value at every right-edge node; layout [nely+1][nelx+1][2]."""
    f = np.zeros((nely + 1, nelx + 1, 2), dtype=np.float64)
    f[:, nelx, 0] = value
    return f
