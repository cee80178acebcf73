"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module only *generates* inputs: element node coordinates and face
connectivity of structured hexahedral/quadrilateral meshes, closed-form
initial and reference flow fields evaluated at caller-supplied coordinates,
seeded perturbations, and FW-H data-surface point sets.  It holds none of the
Flux Reconstruction arithmetic (no solution/flux points, no operators, no
metrics, no fluxes), so the oracle and the CUDA library each derive those on
their own from the same mesh description.

Mesh description (the layout ``fr_mesh_load`` takes):

* ``nodes``: float64 ``[E][(q+1)**dim][dim]`` with q the geometry order
  (1: bi/trilinear, 2: bi/triquadratic).  Nodes sit at the equispaced
  reference points {-1, (0,) 1} of each direction, local node index
  ``a + (q+1)*b (+ (q+1)**2 * c)`` with ``a`` along xi_1 (fastest).
* ``conn``: int32 ``[E][2*dim][3]``.  Face ``2*d`` is xi_d = -1, face
  ``2*d+1`` is xi_d = +1.  An interior face holds ``(neighbour element,
  neighbour face, orientation)``; a boundary face holds ``(-tag, 0, 0)`` with
  tag ``BC_WALL`` (no-slip adiabatic wall) or ``BC_FARFIELD``
  (characteristic far field).  The structured generators emit orientation 0
  (face points correspond one to one in the same order); ``reorient`` turns
  every element's local frame by a seeded rotation of the reference square or
  cube, which gives the faces every orientation code.

Workload recipes (paper Section 3.1 and Appendix C shapes):

* ``box_mesh``: uniform periodic box, optionally curved by a smooth periodic
  displacement and/or with walls on the y faces.
* ``ogrid_mesh``: spanwise-periodic O-grid of quadratic hexahedra around a
  NACA 4-digit section (Section 3.4 parametrisation; surface nodes uniform in
  arc length) or a circle; straight grid lines along the (smoothed) body
  normal to a circular far field centred at (0.5, 0); geometric radial
  stretching.
* ``isentropic_vortex``, ``taylor_green``: closed-form flow fields.
* ``perturbed_uniform``: free stream plus a seeded uniform velocity
  perturbation per solution point (PCG64).
* ``cylinder_surface`` / ``sphere_surface``: FW-H data surfaces (Section 3.1
  spacing 0.01c with the 0.005c offset from the periodic planes; Appendix C
  sphere with 30 polar rings and azimuthal spacing 2*pi/45).
* ``monopole_field`` / ``dipole_field``: Appendix C closed-form acoustic
  fields in a uniformly moving medium.
"""
from __future__ import annotations

import math

import numpy as np

BC_WALL = 1
BC_FARFIELD = 2

GAMMA = 1.4


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def _elem_nodes_from_grid(grid, q, dim, ne, shift=None):
    """Cut a structured node grid into per-element node blocks.

    grid: [n_0, .., n_{dim-1}, dim] node coordinates, q*ne[d] (+1 when not
    periodic) nodes along direction d.  A node index that wraps past the end
    of a periodic direction d takes the node at the wrapped index plus the
    period vector shift[d] (zero for a closed curve such as an O-grid ring).
    """
    shape = grid.shape[:dim]
    if shift is None:
        shift = np.zeros((dim, dim))
    shift = np.asarray(shift, float)
    loc = np.stack(np.meshgrid(*[np.arange(q + 1)] * dim, indexing="ij"), axis=-1)
    loc = loc.reshape(-1, dim)
    # local node index a + (q+1) b (+ (q+1)^2 c): a fastest
    order = np.lexsort(tuple(loc[:, d] for d in range(dim)))
    loc = loc[order]
    eidx = np.stack(np.meshgrid(*[np.arange(n) for n in ne], indexing="ij"), axis=-1)
    eidx = eidx.reshape(-1, dim)
    eorder = np.lexsort(tuple(eidx[:, d] for d in range(dim)))
    eidx = eidx[eorder]                                   # element e: e_0 fastest
    gi = q * eidx[:, None, :] + loc[None, :, :]          # [E, nloc, dim]
    wrap = gi // np.asarray(shape)
    gi = gi % np.asarray(shape)
    out = grid[tuple(gi[..., d] for d in range(dim))]
    out = out + np.einsum("end,dc->enc", wrap.astype(float), shift)
    return np.ascontiguousarray(out)


def _structured_conn(ne, periodic, bc_lo, bc_hi):
    """Face connectivity of a structured block of ne[0] x ne[1] (x ne[2]) elements.

    periodic[d]: wrap direction d.  bc_lo[d]/bc_hi[d]: boundary tag used on the
    xi_d = -1 / +1 block faces when direction d is not periodic.
    """
    dim = len(ne)
    E = int(np.prod(ne))
    conn = np.zeros((E, 2 * dim, 3), dtype=np.int32)
    strides = [1, ne[0], ne[0] * (ne[1] if dim > 1 else 1)]
    for e in range(E):
        idx = []
        r = e
        for d in range(dim):
            idx.append(r % ne[d])
            r //= ne[d]
        for d in range(dim):
            for side in (0, 1):
                f = 2 * d + side
                j = idx[d] + (1 if side else -1)
                if 0 <= j < ne[d] or periodic[d]:
                    j %= ne[d]
                    nb = e + (j - idx[d]) * strides[d]
                    conn[e, f] = (nb, 2 * d + (1 - side), 0)
                else:
                    tag = bc_hi[d] if side else bc_lo[d]
                    conn[e, f] = (-tag, 0, 0)
    return conn


def box_mesh(dim, n, lo, hi, q=1, periodic=None, walls_y=False, curve=0.0, seed=0, bc_tag=None):
    """Uniform box of n^dim (or n[0] x n[1] x n[2]) elements.

    curve > 0 displaces every node by a smooth field periodic on the box
    (amplitude ``curve`` times the element size, seeded phases), which makes
    elements curved (q=2) or skewed (q=1) while periodic faces still match.
    walls_y puts BC_WALL on both y faces (direction 1 not periodic).
    Non-periodic faces carry ``bc_tag`` (default BC_WALL).
    """
    ne = list(n) if np.ndim(n) else [int(n)] * dim
    lo = np.broadcast_to(np.asarray(lo, float), (dim,)).copy()
    hi = np.broadcast_to(np.asarray(hi, float), (dim,)).copy()
    if periodic is None:
        periodic = [True] * dim
    periodic = list(periodic)
    if walls_y:
        periodic[1] = False
    npts = [q * ne[d] + (0 if periodic[d] else 1) for d in range(dim)]
    axes = [lo[d] + (hi[d] - lo[d]) * np.arange(npts[d]) / (q * ne[d]) for d in range(dim)]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
    if curve > 0.0:
        rng = np.random.default_rng(seed)
        L = hi - lo
        h = np.min(L / np.asarray(ne))
        ph = rng.uniform(0, 2 * np.pi, size=(dim, dim))
        disp = np.zeros_like(grid)
        for c in range(dim):
            arg = np.zeros(grid.shape[:-1])
            for d in range(dim):
                arg = arg + 2 * np.pi * (grid[..., d] - lo[d]) / L[d] + ph[c, d]
            amp = curve * h
            field = amp * np.sin(arg)
            # keep wall planes flat so wall faces stay at y = lo/hi
            if walls_y:
                yy = (grid[..., 1] - lo[1]) / L[1]
                field = field * np.sin(np.pi * yy)
            disp[..., c] = field
        grid = grid + disp
    shift = np.diag(hi - lo)
    nodes = _elem_nodes_from_grid(grid, q, dim, ne, shift)
    bc = [BC_WALL if bc_tag is None else bc_tag] * dim
    conn = _structured_conn(ne, periodic, bc, bc)
    return nodes, conn


def proper_rotations(dim):
    """The proper rotations of the reference square (4) or cube (24), each as
    (perm, sign): old coordinate xi[perm[k]] = sign[k] * new coordinate xi'[k].
    Reflections are left out: they would make the element map left-handed
    (negative Jacobian)."""
    import itertools
    out = []
    for perm in itertools.permutations(range(dim)):
        # parity of the permutation
        inv = sum(1 for i in range(dim) for j in range(i + 1, dim) if perm[i] > perm[j])
        for sign in itertools.product((1, -1), repeat=dim):
            if (-1) ** inv * int(np.prod(sign)) == 1:
                out.append((tuple(perm), tuple(sign)))
    return out


def _old_index(new_idx, rot, n):
    """Old tensor multi-index of new multi-index new_idx (tuple over directions)
    of an n-point-per-direction tensor grid under rotation rot (symmetric
    points: reversal maps index i to n-1-i)."""
    perm, sign = rot
    old = [0] * len(perm)
    for k, (pk, sk) in enumerate(zip(perm, sign)):
        old[pk] = new_idx[k] if sk > 0 else n - 1 - new_idx[k]
    return tuple(old)


def _lin(idx, n):
    """Linear index i_0 + n i_1 (+ n^2 i_2): direction 0 fastest."""
    return sum(int(i) * n ** d for d, i in enumerate(idx))


def tensor_relabel(n, dim, rot):
    """Index array r with new_values[..., k] = old_values[..., r[k]] for the
    points of an n^dim tensor grid on the symmetric reference element."""
    out = np.empty(n ** dim, np.int64)
    for k in range(n ** dim):
        idx = tuple((k // n ** d) % n for d in range(dim))
        out[k] = _lin(_old_index(idx, rot, n), n)
    return out


def _face_point_index(dim, d, idx, n):
    """Face point index of tensor multi-index idx on a face normal to d: the
    remaining directions in increasing order, the lower one fastest."""
    rest = [idx[k] for k in range(dim) if k != d]
    return _lin(rest, n)


def _orientation_map(dim, n, o, fp):
    """Neighbour face point of face point fp for orientation code o (the
    mesh-description convention: dim 2 bit 0 reverses; dim 3 bit 2 swaps the
    two face indices, then bit 0 / bit 1 reverse the first / second)."""
    if dim == 2:
        return n - 1 - fp if o & 1 else fp
    a, b = fp % n, fp // n
    if o & 4:
        a, b = b, a
    if o & 1:
        a = n - 1 - a
    if o & 2:
        b = n - 1 - b
    return a + n * b


def reorient(nodes, conn, dim, seed=0, rots=None, nfp_check=3):
    """Turn every element's local frame by a proper rotation of the reference
    element (seeded choice, or rots[e] = (perm, sign)) and rebuild the face
    connectivity with the orientation codes that result.

    Returns (nodes', conn', rots).  The physical mesh is unchanged; only the
    labelling of each element's nodes, faces and face points changes, so any
    discretisation that is invariant under the symmetries of the reference
    element gives the same solution, relabelled point by point with
    ``tensor_relabel(p+1, dim, rots[e])``.  The base mesh must carry
    orientation 0.  ``nfp_check`` points per face direction are used to derive
    each code (any n >= 3 fixes it uniquely)."""
    nodes = np.asarray(nodes, float)
    conn = np.asarray(conn, np.int32)
    E, nn, _ = nodes.shape
    q = int(round(nn ** (1.0 / dim))) - 1
    if np.any(conn[:, :, 0] >= 0) and np.any(conn[conn[:, :, 0] >= 0][:, 2] != 0):
        raise ValueError("reorient needs a base mesh with orientation 0")
    allr = proper_rotations(dim)
    if rots is None:
        rng = np.random.default_rng(seed)
        rots = [allr[k] for k in rng.integers(0, len(allr), E)]
    rots = [(tuple(r[0]), tuple(r[1])) for r in rots]
    new_nodes = np.empty_like(nodes)
    for e in range(E):
        new_nodes[e] = nodes[e][tensor_relabel(q + 1, dim, rots[e])]
    n = nfp_check

    def new_face_of_old(e, f_old):
        perm, sign = rots[e]
        d_old, s_old = divmod(f_old, 2)
        k = perm.index(d_old)                       # new direction along old d
        s_new = s_old if sign[k] > 0 else 1 - s_old
        return 2 * k + s_new

    def old_fp_table(e, f_new):
        """old face point index (old face of e) of each new face point."""
        dn, sn = divmod(f_new, 2)
        out = []
        others = [k for k in range(dim) if k != dn]
        for fp in range(n ** (dim - 1)):
            idx = [0] * dim
            for j, k in enumerate(others):
                idx[k] = (fp // n ** j) % n
            idx[dn] = n - 1 if sn else 0
            old = _old_index(tuple(idx), rots[e], n)
            d_old = rots[e][0][dn]
            out.append(_face_point_index(dim, d_old, old, n))
        return out

    new_conn = np.zeros_like(conn)
    ncode = 2 if dim == 2 else 8
    for e in range(E):
        perm, sign = rots[e]
        for f_new in range(2 * dim):
            dn, sn = divmod(f_new, 2)
            d_old = perm[dn]
            s_old = sn if sign[dn] > 0 else 1 - sn
            f_old = 2 * d_old + s_old
            ne, nf_old, _ = conn[e, f_old]
            if ne < 0:
                new_conn[e, f_new] = conn[e, f_old]
                continue
            nf_new = new_face_of_old(ne, nf_old)
            mine = old_fp_table(e, f_new)            # my new fp -> old fp (shared, orientation 0)
            theirs = old_fp_table(ne, nf_new)        # their new fp -> old fp
            inv = {o: k for k, o in enumerate(theirs)}
            want = [inv[o] for o in mine]
            code = [o for o in range(ncode)
                    if all(_orientation_map(dim, n, o, k) == want[k] for k in range(len(want)))]
            if len(code) != 1:
                raise RuntimeError("no unique orientation code for a face")
            new_conn[e, f_new] = (ne, nf_new, code[0])
    return np.ascontiguousarray(new_nodes), new_conn, rots


def relabel_points(a, rots, n, dim):
    """Values a [E, ..., n^dim] at an element's tensor points in the base
    labelling -> the labelling of ``reorient``'s rotated elements."""
    out = np.empty_like(a)
    for e, r in enumerate(rots):
        out[e] = a[e][..., tensor_relabel(n, dim, r)]
    return out


def naca4_surface(m, pc, t, beta):
    """NACA 4-digit section point at curve parameter beta in [0, 2*pi).

    Chord from x=0 (leading edge) to x=1 (trailing edge), closed trailing
    edge.  beta runs clockwise from the trailing edge: lower surface for
    beta in [0, pi], upper surface for beta in [pi, 2*pi].
    """
    beta = np.asarray(beta, float)
    x = 0.5 * (1.0 + np.cos(beta))
    yt = 5.0 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2
                    + 0.2843 * x ** 3 - 0.1036 * x ** 4)
    if m != 0.0:
        fore = x < pc
        yc = np.where(fore, m / pc ** 2 * (2 * pc * x - x ** 2),
                      m / (1 - pc) ** 2 * ((1 - 2 * pc) + 2 * pc * x - x ** 2))
        dyc = np.where(fore, 2 * m / pc ** 2 * (pc - x), 2 * m / (1 - pc) ** 2 * (pc - x))
    else:
        yc = np.zeros_like(x)
        dyc = np.zeros_like(x)
    th = np.arctan(dyc)
    upper = np.sin(beta) < 0.0  # beta in (pi, 2pi)
    sgn = np.where(upper, 1.0, -1.0)
    xs = x - sgn * yt * np.sin(th)
    ys = yc + sgn * yt * np.cos(th)
    return xs, ys


def ogrid_mesh(n_theta, n_r, n_z, span, r_outer=10.0, first_cell=2e-3, body="naca",
               naca=(0.02, 0.4, 0.12), radius=0.5, center=(0.5, 0.0), q=2):
    """Spanwise-periodic O-grid of (q=2) quadratic hexahedra around a body.

    Element e = i_theta + n_theta*(i_r + n_r*i_z).  xi_1 runs clockwise around
    the body (periodic), xi_2 radially outward (face 2 = BC_WALL on the body,
    face 3 = BC_FARFIELD at r_outer), xi_3 along the span (periodic).
    body="naca" uses the NACA 4-digit (m, p, t) section, body="circle" a
    circle of the given radius about ``center``.
    """
    nt = q * n_theta
    beta = 2 * np.pi * np.arange(nt) / nt
    cx, cy = center
    if body == "naca":
        # surface nodes uniform in arc length (the cosine parameter alone
        # would make trailing-edge cells orders of magnitude smaller)
        fine = np.linspace(0.0, 2 * np.pi, 20001)
        fx, fy = naca4_surface(*naca, fine)
        arc = np.concatenate([[0.0], np.cumsum(np.hypot(np.diff(fx), np.diff(fy)))])
        bq = np.interp(arc[-1] * np.arange(nt) / nt, arc, fine)
        xs, ys = naca4_surface(*naca, bq)
    else:
        xs = cx + radius * np.cos(-beta)
        ys = cy + radius * np.sin(-beta)
    xo = cx + r_outer * np.cos(-beta)
    yo = cy + r_outer * np.sin(-beta)
    # geometric stretching: first element height ~ first_cell relative to r_outer
    D = r_outer
    target = first_cell / D

    def frac(ratio):
        return (ratio - 1.0) / (ratio ** n_r - 1.0)

    lo_r, hi_r = 1.0 + 1e-12, 2.0
    for _ in range(200):
        mid = 0.5 * (lo_r + hi_r)
        if frac(mid) > target:
            lo_r = mid
        else:
            hi_r = mid
    ratio = 0.5 * (lo_r + hi_r)
    jr = np.arange(q * n_r + 1) / q
    s = (ratio ** jr - 1.0) / (ratio ** n_r - 1.0)
    zz = span * np.arange(q * n_z) / (q * n_z)
    # straight grid lines along the body normal, smoothed along the surface
    # (the trailing-edge corner fans out over several nodes), each ending
    # where it meets the far-field circle; near the wall the cells are then
    # wall-normal, and lines of a convex body never cross
    tx = np.roll(xs, -1) - np.roll(xs, 1)
    ty = np.roll(ys, -1) - np.roll(ys, 1)
    ang = np.unwrap(np.arctan2(tx, -ty))        # outward normal (-ty, tx) of the clockwise traversal
    wdt = max(2, nt // 6)
    ker = np.exp(-0.5 * (np.arange(-3 * wdt, 3 * wdt + 1) / wdt) ** 2)
    ker /= ker.sum()
    turn = ang[-1] - ang[0] + (ang[1] - ang[0])  # one full turn (+-2 pi) over the closed curve
    ext = np.concatenate([ang[-3 * wdt:] - turn, ang, ang[:3 * wdt] + turn])
    angs = np.convolve(ext, ker, mode="valid")
    vx, vy = np.cos(angs), np.sin(angs)
    ddx, ddy = xs - cx, ys - cy
    dv = ddx * vx + ddy * vy
    tt = -dv + np.sqrt(dv * dv - (ddx * ddx + ddy * ddy) + r_outer ** 2)
    xo = xs + tt * vx
    yo = ys + tt * vy
    grid = np.empty((nt, q * n_r + 1, q * n_z, 3))
    for k, z in enumerate(zz):
        grid[:, :, k, 0] = (1 - s[None, :]) * xs[:, None] + s[None, :] * xo[:, None]
        grid[:, :, k, 1] = (1 - s[None, :]) * ys[:, None] + s[None, :] * yo[:, None]
        grid[:, :, k, 2] = z
    shift = np.zeros((3, 3))
    shift[2, 2] = span
    nodes = _elem_nodes_from_grid(grid, q, 3, [n_theta, n_r, n_z], shift)
    conn = _structured_conn([n_theta, n_r, n_z], [True, False, True],
                            [0, BC_WALL, 0], [0, BC_FARFIELD, 0])
    return nodes, conn


# --------------------------------------------------------------------------
# closed-form flow fields (conserved variables [rho, rho*V, rho*E])
# --------------------------------------------------------------------------

def sponge_orders(nodes, p, center=(0.5, 0.0), radii=(4.0, 6.0, 8.0)):
    """Per-element polynomial degree for the far-field sponge of Section 3.1:
    degree p inside radii[0] of ``center`` (element centroid in the x-y plane),
    then one degree less past each further radius, never below 0.  With the
    defaults and p = 3 on a 10c O-grid: p3 near the body, p2 from 4c, p1 from
    6c, p0 from 8c out to the far-field boundary."""
    X = np.asarray(nodes, float)
    r = np.hypot(X[:, :, 0].mean(axis=1) - center[0], X[:, :, 1].mean(axis=1) - center[1])
    drop = np.zeros(len(X), np.int32)
    for rr in radii:
        drop += (r >= rr).astype(np.int32)
    return np.maximum(p - drop, 0).astype(np.int32)


def primitive_to_conserved(rho, vel, p, gamma=GAMMA):
    vel = np.asarray(vel)
    ke = 0.5 * rho * np.sum(vel * vel, axis=0)
    return np.concatenate([rho[None], rho[None] * vel, (p / (gamma - 1.0) + ke)[None]], axis=0)


def isentropic_vortex(x, t=0.0, beta=5.0, mach=0.5, gamma=GAMMA, period=10.0, center=(0.0, 0.0)):
    """2D isentropic vortex advected at U = mach*sqrt(gamma) along +x.

    rho_inf = p_inf = T_inf = 1.  x: [..., 2] coordinates.  The displacement
    from the advected centre is wrapped into the periodic box [-5, 5)^2.
    Returns conserved variables with shape [4, ...].
    """
    U = mach * math.sqrt(gamma)
    dx = x[..., 0] - (center[0] + U * t)
    dy = x[..., 1] - center[1]
    dx = (dx + 0.5 * period) % period - 0.5 * period
    dy = (dy + 0.5 * period) % period - 0.5 * period
    r2 = dx * dx + dy * dy
    f = np.exp(0.5 * (1.0 - r2))
    du = -beta / (2 * np.pi) * dy * f
    dv = beta / (2 * np.pi) * dx * f
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return primitive_to_conserved(rho, np.stack([U + du, dv]), p, gamma)


def taylor_green(x, mach=0.1, gamma=GAMMA):
    """3D Taylor-Green vortex on [0, 2*pi]^3 (unit velocity, isothermal rho = p/p0)."""
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p0 = 1.0 / (gamma * mach ** 2)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    rho = p / p0
    return primitive_to_conserved(rho, np.stack([u, v, w]), p, gamma)


def freestream(mach, aoa_deg, dim=3, gamma=GAMMA):
    """Free-stream state: rho=1, |V|=1 at angle aoa in the x-y plane, p=1/(gamma M^2)."""
    a = math.radians(aoa_deg)
    vel = [math.cos(a), math.sin(a)] + ([0.0] if dim == 3 else [])
    return 1.0, np.array(vel), 1.0 / (gamma * mach ** 2)


def uniform_state(shape, rho, vel, p, gamma=GAMMA):
    """Conserved state [nvar, *shape] of a uniform flow."""
    vel = np.asarray(vel, float)
    r = np.full(shape, rho)
    V = np.stack([np.full(shape, v) for v in vel])
    P = np.full(shape, p)
    return primitive_to_conserved(r, V, P, gamma)


def perturbed_uniform(E, nsp, rho, vel, p, amplitude=0.01, seed=0, gamma=GAMMA):
    """Uniform flow plus U(-a, a)*|V| added to every velocity component at every
    solution point (PCG64 with the given seed).  Returns float64 [E][nvar][nsp].
    """
    vel = np.asarray(vel, float)
    dim = vel.size
    rng = np.random.Generator(np.random.PCG64(seed))
    dV = rng.uniform(-amplitude, amplitude, size=(dim, E, nsp)) * np.linalg.norm(vel)
    V = vel[:, None, None] + dV
    r = np.full((E, nsp), rho)
    P = np.full((E, nsp), p)
    u = primitive_to_conserved(r, V, P, gamma)  # [nvar, E, nsp]
    return np.ascontiguousarray(np.moveaxis(u, 0, 1))


def random_smooth_state(x, seed=0, gamma=GAMMA, amp=0.1, periods=None):
    """A smooth positive state from a few seeded Fourier modes of x ([..., dim])."""
    rng = np.random.default_rng(seed)
    dim = x.shape[-1]
    if periods is None:
        periods = np.ones(dim)
    periods = np.asarray(periods, float)

    def mode():
        k = rng.integers(1, 3, size=dim)
        ph = rng.uniform(0, 2 * np.pi)
        arg = sum(2 * np.pi * k[d] * x[..., d] / periods[d] for d in range(dim)) + ph
        return np.sin(arg)

    rho = 1.0 + amp * mode()
    vel = np.stack([0.3 + amp * mode() for _ in range(dim)])
    p = 1.0 + amp * mode()
    return primitive_to_conserved(rho, vel, p, gamma)


# --------------------------------------------------------------------------
# FW-H data surfaces
# --------------------------------------------------------------------------

def cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.01, span=0.2):
    """Closed cylindrical permeable surface about the spanwise axis.

    Panel centres every ``spacing`` in arc length and in z, the first and last
    spanwise rows spacing/2 from the periodic planes.  Returns (y [N,3],
    outward unit normal [N,3], panel area [N]).
    """
    n_az = int(round(2 * np.pi * radius / spacing))
    n_z = int(round(span / spacing))
    ang = 2 * np.pi * (np.arange(n_az) + 0.5) / n_az
    z = spacing * (np.arange(n_z) + 0.5) * (span / (n_z * spacing))
    A, Z = np.meshgrid(ang, z, indexing="xy")
    A = A.ravel()
    Z = Z.ravel()
    y = np.stack([center[0] + radius * np.cos(A), center[1] + radius * np.sin(A), Z], axis=1)
    nrm = np.stack([np.cos(A), np.sin(A), np.zeros_like(A)], axis=1)
    area = np.full(A.shape, (2 * np.pi * radius / n_az) * (span / n_z))
    return y, nrm, area


def sphere_surface(radius=1.0, n_polar=30, dphi=2 * np.pi / 45):
    """Sphere split into n_polar rings; ring i at theta_i=(i+1/2)pi/n_polar with
    max(1, round(2*pi*sin(theta_i)/dphi)) panels of equal area (exact band area
    divided evenly).  Returns (y [N,3], outward unit normal [N,3], area [N]).
    """
    ys, ns, As = [], [], []
    for i in range(n_polar):
        tlo = i * np.pi / n_polar
        thi = (i + 1) * np.pi / n_polar
        th = 0.5 * (tlo + thi)
        nphi = max(1, int(round(2 * np.pi * np.sin(th) / dphi)))
        band = 2 * np.pi * radius ** 2 * (np.cos(tlo) - np.cos(thi))
        phi = 2 * np.pi * (np.arange(nphi) + 0.5) / nphi
        n = np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi),
                      np.full(nphi, np.cos(th))], axis=1)
        ys.append(radius * n)
        ns.append(n)
        As.append(np.full(nphi, band / nphi))
    return np.concatenate(ys), np.concatenate(ns), np.concatenate(As)


# --------------------------------------------------------------------------
# Appendix C closed-form acoustic fields in a uniformly moving medium
# --------------------------------------------------------------------------

def _moving_medium_radii(r, M):
    """Amplitude radius R*, phase radius R and their x-gradients for r = x - y_s."""
    M = np.asarray(M, float)
    b2 = 1.0 / (1.0 - M @ M)
    Mr = r @ M
    rr = np.sum(r * r, axis=-1)
    Rs = np.sqrt(rr + b2 * Mr ** 2) / np.sqrt(b2)
    R = b2 * (Rs - Mr)
    dRs = (r + b2 * Mr[..., None] * M) / (b2 * Rs[..., None])
    dR = b2 * (dRs - M)
    return Rs, R, dRs, dR


def monopole_field(x, t, M, A=1.0, omega=10 * np.pi, c0=340.75, rho0=1.234, gamma=GAMMA):
    """Monopole of Appendix C.1 at the origin, medium moving at Mach vector M.

    phi = A/(4 pi R*) exp(i omega (t - R/c0)); u' = grad phi; p' = -rho0 (d/dt +
    c0 M.grad) phi; rho' = p'/c0^2 (real parts).  x: [..., 3], t: scalar or
    broadcastable.  Returns dict with rho, vel (total, [...,3]), p, and p'.
    """
    M = np.asarray(M, float)
    Rs, R, dRs, dR = _moving_medium_radii(x, M)
    ph = np.exp(1j * omega * (t - R / c0))
    phi = A / (4 * np.pi * Rs) * ph
    gphi = (A / (4 * np.pi)) * ph[..., None] * (-dRs / Rs[..., None] ** 2
                                               - 1j * omega / c0 * dR / Rs[..., None])
    return _acoustic_out(phi, gphi, M, omega, c0, rho0, gamma)


def dipole_field(x, t, M, A=1.0, omega=10 * np.pi, c0=340.75, rho0=1.234, gamma=GAMMA, h=1e-4):
    """Dipole of Appendix C.2: phi_d = d(phi_m)/d x_2, axis along x_2.

    The x_2 derivative and the gradient of phi_d are taken by 4th-order
    central differences of the closed-form monopole potential with step h.
    """
    M = np.asarray(M, float)

    def phim(xx):
        Rs, R, _, _ = _moving_medium_radii(xx, M)
        return A / (4 * np.pi * Rs) * np.exp(1j * omega * (t - R / c0))

    def d(f, xx, k):
        e = np.zeros(3)
        e[k] = h
        return (-f(xx + 2 * e) + 8 * f(xx + e) - 8 * f(xx - e) + f(xx - 2 * e)) / (12 * h)

    def phid(xx):
        return d(phim, xx, 1)

    phi = phid(x)
    gphi = np.stack([d(phid, x, k) for k in range(3)], axis=-1)
    return _acoustic_out(phi, gphi, M, omega, c0, rho0, gamma)


def _acoustic_out(phi, gphi, M, omega, c0, rho0, gamma):
    p0 = rho0 * c0 ** 2 / gamma
    pp = -rho0 * (1j * omega * phi + c0 * (gphi @ M))
    up = np.real(gphi)
    pr = np.real(pp)
    U = c0 * M
    return {"rho": rho0 + pr / c0 ** 2, "vel": U + up, "p": p0 + pr, "pprime": pr,
            "p0": p0, "rho0": rho0}
