"""Upwind discontinuous Galerkin discretisation of steady 2D transport.

The model problem is the steady transport equation of Sec. 6.1 (Eq. transport),
    b(x, y) . grad u + sigma_t(x, y) u = q(x, y)   in the unit square,
    u = g                                          on the inflow boundary,
discretised with the fully upwinded DG method the paper uses (Sec. 6.1, after
Lesaint-Raviart and Reed-Hill): nodal Lagrange P_p elements on triangles,
each element one b x b block of the matrix, b = (p + 1)(p + 2) / 2.

Weak form used on each element K (strong form of the advection term):
    int_K (b . grad u_K) v + sigma u_K v
      - int_{dK} (b.n)^- (u_K - u_up) v  =  int_K q v,
with (b.n)^- = min(b.n, 0) evaluated pointwise, u_up the neighbour's trace
(or g on the domain boundary).  The element block A_KK collects the volume
terms and the inflow-face trace of u_K; the coupling block A_KK' collects the
upwind trace of the neighbour K'.  Only the p + 1 nodes on a face are nonzero
on that face, so a coupling block has exactly (p + 1)^2 nonzero entries.

This module is input generation only: it holds none of the multigrid method.
"""
import heapq
import numpy as np

from . import rng


# ----------------------------------------------------------------------------
# reference element
# ----------------------------------------------------------------------------

def _gauss_legendre01(m):
    x, w = np.polynomial.legendre.leggauss(m)
    return 0.5 * (x + 1.0), 0.5 * w


def ref_nodes(p):
    """Equispaced nodes (i/p, j/p), i + j <= p, ordered by j then i."""
    pts = [(i / p, j / p) for j in range(p + 1) for i in range(p + 1 - j)]
    return np.array(pts, dtype=np.float64)


def _node_index(p):
    idx = {}
    k = 0
    for j in range(p + 1):
        for i in range(p + 1 - j):
            idx[(i, j)] = k
            k += 1
    return idx


def face_nodes(p):
    """Node indices on each local face, in the order of the face parameter s = k/p.

    Face 0 runs v0 -> v1, face 1 v1 -> v2, face 2 v2 -> v0 (counter-clockwise).
    """
    idx = _node_index(p)
    f0 = [idx[(k, 0)] for k in range(p + 1)]
    f1 = [idx[(p - k, k)] for k in range(p + 1)]
    f2 = [idx[(0, p - k)] for k in range(p + 1)]
    return np.array([f0, f1, f2], dtype=np.int64)


def _monomials(p):
    return [(a, c) for a in range(p + 1) for c in range(p + 1 - a)]


def _vander(pts, p):
    mons = _monomials(p)
    x, y = pts[:, 0], pts[:, 1]
    V = np.empty((len(pts), len(mons)))
    Dx = np.zeros_like(V)
    Dy = np.zeros_like(V)
    for k, (a, c) in enumerate(mons):
        V[:, k] = x ** a * y ** c
        if a > 0:
            Dx[:, k] = a * x ** (a - 1) * y ** c
        if c > 0:
            Dy[:, k] = c * x ** a * y ** (c - 1)
    return V, Dx, Dy


def _lagrange1d(p, t):
    """1D Lagrange basis on s_k = k/p at points t: shape (len(t), p + 1)."""
    s = np.arange(p + 1) / p
    out = np.ones((len(t), p + 1))
    for k in range(p + 1):
        for m in range(p + 1):
            if m != k:
                out[:, k] *= (t - s[m]) / (s[k] - s[m])
    return out


class RefElement:
    """Basis values, gradients and quadrature on the reference triangle."""

    def __init__(self, p):
        self.p = p
        self.nb = (p + 1) * (p + 2) // 2
        nodes = ref_nodes(p)
        V, _, _ = _vander(nodes, p)
        coef = np.linalg.inv(V)
        # volume rule: collapsed (Duffy) Gauss-Legendre, exact to degree 2p + 2
        m = p + 2
        u, wu = _gauss_legendre01(m)
        uu, vv = np.meshgrid(u, u, indexing="ij")
        ww = np.outer(wu, wu) * (1.0 - vv)
        self.qpts = np.stack([(uu * (1.0 - vv)).ravel(), vv.ravel()], axis=1)
        self.qw = ww.ravel()
        Vq, Dxq, Dyq = _vander(self.qpts, p)
        self.phi = (Vq @ coef).T        # (nb, Q): phi_i at q
        self.dphi_x = (Dxq @ coef).T    # reference derivatives
        self.dphi_y = (Dyq @ coef).T
        # face rule: Gauss-Legendre on the face parameter
        self.ft, self.fw = _gauss_legendre01(m)
        self.fnodes = face_nodes(p)
        self.l1 = _lagrange1d(p, self.ft)            # (Qf, p+1) at t
        self.l1r = _lagrange1d(p, 1.0 - self.ft)     # at 1 - t (neighbour side)
        self.mass = (self.phi * self.qw) @ self.phi.T


# ----------------------------------------------------------------------------
# mesh
# ----------------------------------------------------------------------------

def square_mesh(N, jitter=0.0, seed=0):
    """N x N squares on the unit square, each split by its SW -> NE diagonal.

    Interior vertices move by U[-jitter*h, +jitter*h] in each coordinate
    (counter-based draws from ``seed``).  Returns vertices (NV, 2) and
    counter-clockwise triangles (2 N^2, 3).
    """
    h = 1.0 / N
    ii, jj = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="xy")
    X = (ii * h).ravel().astype(np.float64)
    Y = (jj * h).ravel().astype(np.float64)
    if jitter > 0.0:
        nv = (N + 1) * (N + 1)
        ux = rng.uniform(seed, nv, stream=0)
        uy = rng.uniform(seed, nv, stream=1)
        interior = ((ii > 0) & (ii < N) & (jj > 0) & (jj < N)).ravel()
        X = X + np.where(interior, (2.0 * ux - 1.0) * jitter * h, 0.0)
        Y = Y + np.where(interior, (2.0 * uy - 1.0) * jitter * h, 0.0)
    vid = lambda i, j: j * (N + 1) + i  # noqa: E731
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    sw, se, ne, nw = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
    t0 = np.stack([sw, se, ne], axis=1)
    t1 = np.stack([sw, ne, nw], axis=1)
    tri = np.empty((2 * N * N, 3), dtype=np.int64)
    tri[0::2] = t0
    tri[1::2] = t1
    return np.stack([X, Y], axis=1), tri


def _half_edges(tri, nv):
    E = tri.shape[0]
    a = np.concatenate([tri[:, 0], tri[:, 1], tri[:, 2]])
    b = np.concatenate([tri[:, 1], tri[:, 2], tri[:, 0]])
    elem = np.tile(np.arange(E), 3)
    face = np.repeat(np.arange(3), E)
    key = np.minimum(a, b) * nv + np.maximum(a, b)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    twin = np.full(3 * E, -1, dtype=np.int64)
    same = ks[1:] == ks[:-1]
    pos = np.nonzero(same)[0]
    twin[order[pos]] = order[pos + 1]
    twin[order[pos + 1]] = order[pos]
    return a, b, elem, face, twin


# ----------------------------------------------------------------------------
# flows and coefficients
# ----------------------------------------------------------------------------

def constant_flow(theta):
    c, s = np.cos(theta), np.sin(theta)

    def f(x, y):
        return np.full_like(x, c), np.full_like(y, s)
    return f


def paper_flow(kind):
    """The non-constant flows of the paper's flow study (Sec. 6.2):
    b1 = (cos^2(pi y), cos^2(pi x)), b2 = (sin^2(pi y), sin^2(pi x)),
    b3 = (y^4, cos^2(pi x / 2)).  Both components are nonnegative, so the
    flow has no closed streamlines."""
    def b1(x, y):
        return np.cos(np.pi * y) ** 2, np.cos(np.pi * x) ** 2

    def b2(x, y):
        return np.sin(np.pi * y) ** 2, np.sin(np.pi * x) ** 2

    def b3(x, y):
        return y ** 4, np.cos(0.5 * np.pi * x) ** 2
    return {"b1": b1, "b2": b2, "b3": b3}[kind]


def rotating_flow(x, y):
    """b = (0.5 - y, x - 0.5) / |.|, and b = 0 where |.| < 1e-14."""
    bx = 0.5 - y
    by = x - 0.5
    nrm = np.sqrt(bx * bx + by * by)
    small = nrm < 1e-14
    nrm = np.where(small, 1.0, nrm)
    return np.where(small, 0.0, bx / nrm), np.where(small, 0.0, by / nrm)


# ----------------------------------------------------------------------------
# assembly
# ----------------------------------------------------------------------------

def topological_order(E, rows, cols):
    """Kahn's algorithm on 'row depends on col' edges, smallest index first.

    Returns the new-to-old permutation, or None if the graph has a cycle.
    """
    indeg = np.zeros(E, dtype=np.int64)
    np.add.at(indeg, rows, 1)
    order = np.argsort(cols, kind="stable")
    cs = cols[order]
    rs = rows[order]
    start = np.searchsorted(cs, np.arange(E + 1))
    heap = [int(e) for e in np.nonzero(indeg == 0)[0]]
    heapq.heapify(heap)
    out = []
    indeg = indeg.tolist()
    while heap:
        e = heapq.heappop(heap)
        out.append(e)
        for k in range(start[e], start[e + 1]):
            r = int(rs[k])
            indeg[r] -= 1
            if indeg[r] == 0:
                heapq.heappush(heap, r)
    if len(out) != E:
        return None
    return np.array(out, dtype=np.int64)


def assemble(N, p, flow, sigma, q=1.0, g=0.0, jitter=0.0, jitter_seed=0,
             order="natural", keep_parts=False):
    """Assemble the upwind DG system on an N x N x 2 triangle mesh.

    ``flow(x, y) -> (bx, by)``; ``sigma`` is a scalar or one value per element
    (original numbering); ``q`` and ``g`` are constants; ``order`` is
    ``"natural"`` or ``"topological"`` (elements ordered along the flow so that
    A is block lower triangular; only valid for flows without cycles).
    """
    ref = RefElement(p)
    nb = ref.nb
    verts, tri = square_mesh(N, jitter, jitter_seed)
    E = tri.shape[0]
    nv = verts.shape[0]
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (E,)).copy()

    v0 = verts[tri[:, 0]]
    v1 = verts[tri[:, 1]]
    v2 = verts[tri[:, 2]]
    J00 = v1[:, 0] - v0[:, 0]
    J01 = v2[:, 0] - v0[:, 0]
    J10 = v1[:, 1] - v0[:, 1]
    J11 = v2[:, 1] - v0[:, 1]
    det = J00 * J11 - J01 * J10
    if np.any(det <= 0):
        raise ValueError("inverted element")

    # ---- volume terms: advection (strong form) and reaction
    xq = v0[:, 0:1] + J00[:, None] * ref.qpts[None, :, 0] + J01[:, None] * ref.qpts[None, :, 1]
    yq = v0[:, 1:2] + J10[:, None] * ref.qpts[None, :, 0] + J11[:, None] * ref.qpts[None, :, 1]
    bx, by = flow(xq, yq)
    # beta = J^{-1} b
    beta0 = (J11[:, None] * bx - J01[:, None] * by) / det[:, None]
    beta1 = (-J10[:, None] * bx + J00[:, None] * by) / det[:, None]
    Bx = np.einsum("iq,jq->qij", ref.phi, ref.dphi_x).reshape(len(ref.qw), nb * nb)
    By = np.einsum("iq,jq->qij", ref.phi, ref.dphi_y).reshape(len(ref.qw), nb * nb)
    cw = ref.qw[None, :] * det[:, None]
    adv = ((cw * beta0) @ Bx + (cw * beta1) @ By).reshape(E, nb, nb)
    mass = det[:, None, None] * ref.mass[None, :, :]

    # ---- face terms
    a, b_, helem, hface, twin = _half_edges(tri, nv)
    pa = verts[a]
    pb = verts[b_]
    d = pb - pa
    L = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2)
    nx = d[:, 1] / L
    ny = -d[:, 0] / L
    fx = pa[:, 0:1] + ref.ft[None, :] * d[:, 0:1]
    fy = pa[:, 1:2] + ref.ft[None, :] * d[:, 1:2]
    fbx, fby = flow(fx, fy)
    bn = fbx * nx[:, None] + fby * ny[:, None]
    bnm = np.minimum(bn, 0.0)                      # (H, Qf)
    cwf = (ref.fw[None, :] * L[:, None]) * bnm     # quadrature weight * (b.n)^-
    LL = np.einsum("qk,ql->qkl", ref.l1, ref.l1)
    LR = np.einsum("qk,ql->qkl", ref.l1, ref.l1r)
    S = -np.einsum("hq,qkl->hkl", cwf, LL)         # own inflow trace
    C = np.einsum("hq,qkl->hkl", cwf, LR)          # upwind neighbour trace

    diag0 = adv.copy()
    fn = ref.fnodes
    for f in range(3):
        hs = np.nonzero(hface == f)[0]
        e = helem[hs]
        diag0[e[:, None, None], fn[f][None, :, None], fn[f][None, None, :]] += S[hs]

    # ---- right-hand side: M q (q constant) plus the inflow trace of g
    rhs = (mass @ np.full(nb, float(q))).copy()
    if g != 0.0:
        bd = np.nonzero(twin < 0)[0]
        gi = -float(g) * (cwf[bd] @ ref.l1)        # (nbd, p+1)
        for f in range(3):
            sel = hface[bd] == f
            np.add.at(rhs, (helem[bd][sel][:, None], fn[f][None, :]), gi[sel])

    # ---- coupling blocks: row element helem[h] <- column element helem[twin[h]]
    inter = np.nonzero((twin >= 0) & np.any(bnm < 0.0, axis=1))[0]
    crow = helem[inter]
    ccol = helem[twin[inter]]
    cf_row = hface[inter]
    cf_col = hface[twin[inter]]

    # ---- ordering
    if order in ("topological", "auto"):
        perm = topological_order(E, crow, ccol)
        if perm is None:
            if order == "topological":
                raise ValueError("flow graph has a cycle: no topological order")
            perm = np.arange(E, dtype=np.int64)
    elif order == "natural":
        perm = np.arange(E, dtype=np.int64)
    else:
        raise ValueError(order)
    inv = np.empty(E, dtype=np.int64)
    inv[perm] = np.arange(E)

    # ---- block CSR in the new numbering
    R = np.concatenate([inv, inv[crow]])
    Cc = np.concatenate([inv, inv[ccol]])
    key = R * E + Cc
    srt = np.argsort(key, kind="stable")
    if np.any(np.diff(key[srt]) == 0):
        raise ValueError("duplicate block")
    nnzb = len(key)
    vals0 = np.zeros((nnzb, nb, nb))
    where = np.empty(nnzb, dtype=np.int64)
    where[srt] = np.arange(nnzb)
    dpos = where[:E]                  # position of diagonal block of old element e
    vals0[dpos] = diag0
    cpos = where[E:]
    for fr in range(3):
        for fc in range(3):
            sel = np.nonzero((cf_row == fr) & (cf_col == fc))[0]
            if len(sel):
                vals0[cpos[sel][:, None, None], fn[fr][None, :, None], fn[fc][None, None, :]] = C[inter[sel]]
    rows_sorted = R[srt]
    row_ptr = np.searchsorted(rows_sorted, np.arange(E + 1)).astype(np.int32)
    col = Cc[srt].astype(np.int32)
    # reorder per-element data into the new numbering
    mass_n = mass[perm]
    sig_n = sig[perm]
    rhs_n = rhs[perm].reshape(-1)
    diag_pos = where[perm].astype(np.int32)
    vals = vals0.copy()
    vals[diag_pos] = vals0[diag_pos] + sig_n[:, None, None] * mass_n
    out = dict(E=E, b=nb, p=p, n=E * nb, nnzb=nnzb, row_ptr=row_ptr, col=col,
               vals=vals, diag_pos=diag_pos, mass=mass_n, sigma=sig_n, rhs=rhs_n,
               q=np.full(E * nb, float(q)), perm=perm)
    if keep_parts:
        out["vals0"] = vals0
        out["verts"] = verts
        out["tri"] = tri[perm]
    return out
