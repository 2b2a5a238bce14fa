"""The largest mesh of the suite: 16384 x 16384 elements (536,936,450 DOFs),
ten coarsenings to 16 x 16, mixed path, sixteen phases.

The design holds 16 x 268 M = 4.3 G fractions, so every phase-by-element
index passes 2^31 and must be formed in 64 bits; the mesh, its operators and
the test's arrays take about 140 GB of device memory at the peak.  The inputs
are built on the device (the counter-based design generator's torch version,
the square wall's top-edge load) and nothing of full size goes to the host.
Checks, on outputs the oracle computes one by one (Eq. 5, Eq. 7 element sums,
the sensitivity of Sec. 4) and on properties that hold at any size:
  * design: 512 seeded (phase, element) fractions equal the host generator's
    to a few ulps;
  * moduli E_e = sum_i x_{e,i}^3 E_i at 4,096 seeded elements: relative 1e-14;
  * the solve converges and the float64 true residual the GPU reports is at
    most 1.1 tol;
  * the float64 operator K u at 4,096 seeded nodes against the oracle's sums
    of E_e KE u_e over the node's elements: within 1e-12 of the row's
    absolute sum;
  (the oracle's element products act on u_e - t_e, t_e the element's first
  node's displacement at all four nodes: KE annihilates translations, and at
  this size the displacements dwarf the strains, so the plain products would
  lose about seven digits to cancellation;)
  * the compliance equals f.u, and the energy identity
    |f.u - u.Ku| <= ||u|| ||f - K u|| holds over all DOFs;
  * sensitivities -3 x^2 E_i u_e^T KE u_e at 4,096 seeded (phase, element)
    picks: relative 1e-12.
"""

import numpy as np
import pytest
import torch

from oracle import fem
from synth import dirichlet_design_torch, uniform01

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
N, NC, NP, SEED = 16384, 10, 16, 9
EP16 = [0.8 ** p for p in range(NP - 1)] + [1e-9]
TOL = 1e-8


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


def host_fractions(e, p):
    """The host generator's fractions of elements e (all phases), picked phase p."""
    ctr = e[:, None].astype(np.uint64) * np.uint64(NP) + np.arange(NP, dtype=np.uint64)[None, :]
    g = -np.log(uniform01(SEED, ctr))
    return (g / g.sum(axis=1, keepdims=True))[np.arange(len(e)), p]


def test_max_size_sixteen_phases(mto):
    free_b, _ = torch.cuda.mem_get_info(DEV)
    if free_b < 180 * 2**30:
        pytest.skip(f"needs about 180 GB of free device memory, {free_b / 2**30:.0f} GB free")
    KE = fem.element_stiffness(0.3)
    # uniform01 draws from (0, 1]: clamp the top value into range.
    rng_e = np.minimum((uniform01(21, np.arange(4096, dtype=np.uint64)) * N * N).astype(np.int64), N * N - 1)
    rng_p = np.minimum((uniform01(22, np.arange(4096, dtype=np.uint64)) * NP).astype(np.int64), NP - 1)
    nodes = (uniform01(23, np.arange(2 * 4096, dtype=np.uint64)).reshape(4096, 2) * N).astype(np.int64) + 1
    ni, nj = np.minimum(nodes[:, 0], N), np.minimum(nodes[:, 1], N)  # node rows 1..N (row 0 is clamped)
    # Elements around the picked nodes (column/row offsets -1, 0), clipped.
    aei = np.clip(ni[:, None, None] + np.array([-1, 0])[None, None, :], 0, N - 1)
    aej = np.clip(nj[:, None, None] + np.array([-1, 0])[None, :, None], 0, N - 1)
    aei, aej = np.broadcast_to(aei, (4096, 2, 2)), np.broadcast_to(aej, (4096, 2, 2))

    x = dirichlet_design_torch(N, N, NP, SEED, DEV)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    # Design fractions needed on the host, gathered before x is released.
    xs = x[:, t(rng_e // N), t(rng_e % N)].cpu().numpy()           # [NP, 4096]
    xa = x[:, t(aej.ravel()), t(aei.ravel())].cpu().numpy().reshape(NP, 4096, 2, 2)
    check = np.arange(512)
    np.testing.assert_allclose(xs[rng_p[check], check], host_fractions(rng_e[check], rng_p[check]),
                               rtol=2e-15, atol=0)
    f = torch.zeros((N + 1, N + 1, 2), dtype=torch.float64, device=DEV)
    f[N, :, 1] = -1.0
    mesh = mto.Mesh(N, N, n_coarsen=NC, precision="mixed", tol=TOL, max_it=1000)
    mesh.set_design(x, EP16, 3.0)
    del x
    torch.cuda.empty_cache()

    # Moduli (Eq. 5).
    E_gpu = mesh.moduli()[t(rng_e // N), t(rng_e % N)].cpu().numpy()
    E_ref = np.einsum("p,pk->k", np.asarray(EP16), xs ** 3)
    np.testing.assert_allclose(E_gpu, E_ref, rtol=1e-14, atol=0)

    u, st = mesh.solve(f)
    print(f"16384^2, 16 phases: {st['iters']} iterations, true residual {st['rel_res_true']:.3e}, "
          f"{st['ms_solve']:.0f} ms")
    assert st["converged"] == 1 and st["rel_res_true"] <= 1.1 * TOL

    # Sensitivities at (phase, element) picks, from each element's u_e.
    C, g = mesh.compliance_grad(f, u)
    g_pick = g[t(rng_p), t(rng_e // N), t(rng_e % N)].cpu().numpy()
    del g
    torch.cuda.empty_cache()
    ei, ej = rng_e % N, rng_e // N
    corners = [(ej, ei), (ej, ei + 1), (ej + 1, ei + 1), (ej + 1, ei)]  # BL, BR, TR, TL
    ue = np.concatenate([u[t(a), t(b)].cpu().numpy() for a, b in corners], axis=1)  # [4096, 8]
    de = ue - np.tile(ue[:, 0:2], (1, 4))
    w = np.einsum("ki,ij,kj->k", de, KE, de)
    ref = -3.0 * xs[rng_p, np.arange(4096)] ** 2 * np.asarray(EP16)[rng_p] * w
    np.testing.assert_allclose(g_pick, ref, rtol=1e-12, atol=1e-15 * np.abs(ref).max())

    # The float64 operator at picked nodes: sums of E_e KE u_e over the
    # node's elements (element (i-1+a, j-1+b) holds the node as corner
    # TR, TL, BR, BL for (a, b) = (0, 0), (1, 0), (0, 1), (1, 1)).
    y = mesh.apply_operator(NC, u)
    y_pick = y[t(nj), t(ni)].cpu().numpy()  # [4096, 2]
    fu = torch.dot(f.reshape(-1), u.reshape(-1)).item()
    uKu = torch.dot(u.reshape(-1), y.reshape(-1)).item()
    rnorm = torch.linalg.vector_norm((f - y).reshape(-1)).item()
    unorm = torch.linalg.vector_norm(u.reshape(-1)).item()
    del y
    Ea = np.einsum("p,pkba->kba", np.asarray(EP16), xa ** 3)  # [4096, b, a]
    yref, scale = np.zeros((4096, 2)), np.zeros((4096, 2))
    corner_of = {(0, 0): 2, (1, 0): 3, (0, 1): 1, (1, 1): 0}
    for b in (0, 1):
        for a in (0, 1):
            eI, eJ = ni - 1 + a, nj - 1 + b
            ok = (eI >= 0) & (eI < N) & (eJ >= 0) & (eJ < N)
            cs = [(eJ, eI), (eJ, eI + 1), (eJ + 1, eI + 1), (eJ + 1, eI)]
            uel = np.concatenate([u[t(np.clip(r, 0, N)), t(np.clip(c, 0, N))].cpu().numpy()
                                  for r, c in cs], axis=1)
            uel = uel - np.tile(uel[:, 0:2], (1, 4))
            k = corner_of[(a, b)]
            rows = KE[2 * k:2 * k + 2]  # the node's two rows of KE
            contrib = Ea[:, b, a][:, None] * (uel @ rows.T)
            absc = np.abs(Ea[:, b, a])[:, None] * (np.abs(uel) @ np.abs(rows).T)
            yref += np.where(ok[:, None], contrib, 0.0)
            scale += np.where(ok[:, None], absc, 0.0)
    assert np.all(np.abs(y_pick - yref) <= 1e-12 * scale), np.max(np.abs(y_pick - yref) / scale)

    # Compliance and the energy identity over all DOFs.
    assert abs(C.item() - fu) <= 1e-12 * abs(fu), (C.item(), fu)
    assert abs(fu - uKu) <= unorm * rnorm * (1 + 1e-6)
    mesh.close()
    del u, f
    torch.cuda.empty_cache()
