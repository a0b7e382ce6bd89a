"""Seeded synthetic steady-transport problems (upwind DG on triangle meshes).

The workloads follow the transport problems of Sec. 6.1 of the nAIR paper
(arXiv 1704.05001): a unit-square domain, constant, rotating or the paper's
non-constant flows b1-b3, element absorption sigma_t, source q = 1 and zero
inflow.  The paper's own domains
(*inset*, *block-source*) exist only in figures that are not available, so
these seeded inputs stand in for them.  Nothing in this package computes any
part of the multigrid method: it is shared input generation for the oracle,
the GPU library's tests and the benchmark.
"""
import numpy as np

from . import rng
from .dg import assemble, constant_flow, paper_flow, rotating_flow, RefElement, face_nodes  # noqa: F401

# name -> (N, p, flow, sigma kind, jitter, order, method parameters)
CONFIGS = {
    # P1, 32x32x2, constant b = (cos .3, sin .3), block lower triangular
    "C1": dict(N=32, p=1, flow=("const", 0.3), sigma="one", jitter=0.0,
               order="topological", neumann_degree=1),
    # P2, 256x256x2, rotating b, log-normal sigma_t (seed 2)
    "C2": dict(N=256, p=2, flow=("rot",), sigma="lognormal", jitter=0.0,
               order="natural", neumann_degree=2),
    # P6, 128x128x2 jittered (seed 1), constant b = (cos .7, sin .7)
    "C3": dict(N=128, p=6, flow=("const", 0.7), sigma="one", jitter=0.2,
               order="topological", neumann_degree=1),
    # adjoint workload: the C2 mesh and coefficients
    "C4": dict(N=256, p=2, flow=("rot",), sigma="lognormal", jitter=0.0,
               order="natural", neumann_degree=2),
    # P3, 512x512x2 jittered, rotating b, log-normal sigma_t; Neumann degree not
    # stated for this workload: 6, the fastest measured setup + solve of the
    # degrees 2 to 8 (with degree 1 GMRES(50) stalls near 1e-7)
    "C5": dict(N=512, p=3, flow=("rot",), sigma="lognormal", jitter=0.2,
               order="natural", neumann_degree=6),
    # second workload: the paper's non-constant flows b1, b2, b3 (Sec. 6.2) on a
    # P2, 256x256x2 jittered mesh, sigma_t = 1, Neumann degree 1 (paper default),
    # elements in flow order where the flow graph has none
    "F1": dict(N=256, p=2, flow=("b1",), sigma="one", jitter=0.2, order="auto", neumann_degree=1),
    "F2": dict(N=256, p=2, flow=("b2",), sigma="one", jitter=0.2, order="auto", neumann_degree=1),
    "F3": dict(N=256, p=2, flow=("b3",), sigma="one", jitter=0.2, order="auto", neumann_degree=1),
    # one direction of the angle sweep (Sec. 6.2): constant b = (cos theta, sin
    # theta), P2, 128x128x2 jittered; sweep_angles() gives the batch of theta
    "D": dict(N=128, p=2, flow=("const", 3 * np.pi / 16), sigma="one", jitter=0.2,
              order="topological", neumann_degree=1),
}


def sweep_angles(count=8):
    """Directions of the angle sweep: theta_k = (k + 1/2) (pi / 2) / count."""
    return [(k + 0.5) * 0.5 * np.pi / count for k in range(count)]

JITTER_SEED = 1
SIGMA_SEED = 2
WEIGHT_SEED = 3
COORD_SEED = 4


def make_problem(name="C1", N=None, p=None, theta=None, keep_parts=False, g=0.0):
    """Build a configuration by name, optionally on a smaller mesh (``N``)."""
    cfg = dict(CONFIGS[name])
    if N is not None:
        cfg["N"] = N
    if p is not None:
        cfg["p"] = p
    if cfg["flow"][0] == "const":
        flow = constant_flow(cfg["flow"][1] if theta is None else theta)
    elif cfg["flow"][0] == "rot":
        flow = rotating_flow
    else:
        flow = paper_flow(cfg["flow"][0])
    E = 2 * cfg["N"] * cfg["N"]
    if cfg["sigma"] == "one":
        sigma = 1.0
    else:
        sigma = np.exp(rng.normal(SIGMA_SEED, E))
    prob = assemble(cfg["N"], cfg["p"], flow, sigma, q=1.0, g=g, jitter=cfg["jitter"],
                    jitter_seed=JITTER_SEED, order=cfg["order"], keep_parts=keep_parts)
    prob["name"] = name
    prob["neumann_degree"] = cfg["neumann_degree"]
    return prob


def functional_weights(n, seed=WEIGHT_SEED):
    """w_i ~ U[0, 1] for the adjoint functional J = sum_i w_i x_i."""
    return rng.uniform(seed, n)


def fd_coordinates(n_dof, n_elem, count=8, seed=COORD_SEED):
    """Seeded coordinates for finite-difference gradient checks."""
    u = rng.uniform(seed, 2 * count)
    iq = np.minimum((u[:count] * n_dof).astype(np.int64), n_dof - 1)
    isg = np.minimum((u[count:] * n_elem).astype(np.int64), n_elem - 1)
    return iq, isg
