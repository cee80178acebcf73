"""Pins of the oracle's boundary states, its BR2 lifting and its surface
sampling against facts that the mathematics fixes independently of the
oracle's own code:

* the characteristic far field (the Riemann-invariant boundary that
  Appendix D.1 names): the outgoing invariant comes from the interior, the
  incoming one from the free stream, and entropy and tangential velocity
  from the upwind side; supersonic normal flow takes one side whole;
* the inviscid slip wall: no mass or energy crosses it, its momentum flux is
  normal to it, and a closed channel keeps its mass, energy and
  wall-parallel momentum exactly;
* the BR2 lifting (Section 2.1, Eqs. 4-7, in the BR2 reading): on a
  piecewise-constant state the lifted face gradient is eta times face f's own
  correction alone, g'(+-1) (S_d / |J|) (u_c - u_f), with g'(+-1) the closed
  forms of the correction functions;
* data-surface sampling (Section 3.1): exact for every tensor polynomial of
  degree p in the element's reference coordinates, at points whose element
  map reproduces the requested position.
"""
import math

import numpy as np
import pytest

from oracle.basis import DG, HUYNH_G2
from oracle.fr import FRSolver
from oracle.mesh import Mesh
from oracle.physics import NavierStokes
from oracle.sampling import locate, sample
from paper_2501_05709_gb300 import workloads as W

G = 1.4


def _prim(u, dim):
    rho = u[0]
    V = u[1:1 + dim] / rho
    p = (G - 1.0) * (u[-1] - 0.5 * rho * np.sum(V * V, axis=0))
    return rho, V, p


def _cons(rho, V, p):
    return np.concatenate([rho[None], rho[None] * V, (p / (G - 1.0) + 0.5 * rho * np.sum(V * V, axis=0))[None]])


# ----------------------------------------------------------------- far field
def _farfield_case(seed, dim, vinf, K=400, amp=0.15):
    rng = np.random.default_rng(seed)
    rho_i, p_i = 1.0, 1.0 / G                       # c_inf = 1
    ph = NavierStokes(dim, freestream=(rho_i, np.asarray(vinf, float), p_i))
    n = rng.standard_normal((dim, K))
    n /= np.linalg.norm(n, axis=0)
    N = n * rng.uniform(0.5, 2.0, K)                 # area-weighted normals
    rho = rho_i * (1.0 + amp * rng.uniform(-1, 1, K))
    V = np.asarray(vinf, float)[:, None] + amp * rng.uniform(-1, 1, (dim, K))
    p = p_i * (1.0 + amp * rng.uniform(-1, 1, K))
    return ph, _cons(rho, V, p), N, n, (rho_i, np.asarray(vinf, float), p_i)


@pytest.mark.parametrize("dim", [2, 3])
def test_farfield_subsonic_characteristics(dim):
    vinf = [0.3, -0.2, 0.1][:dim]
    ph, uL, N, n, (rho_i, Vi, p_i) = _farfield_case(1, dim, vinf)
    ub = ph.farfield_state(uL, N)
    rL, VL, pL = _prim(uL, dim)
    rb, Vb, pb = _prim(ub, dim)
    cL, cb, ci = np.sqrt(G * pL / rL), np.sqrt(G * pb / rb), math.sqrt(G * p_i / rho_i)
    vnL, vnb, vni = np.sum(VL * n, 0), np.sum(Vb * n, 0), Vi @ n
    assert np.all(np.abs(vni) < ci)
    # outgoing invariant from the interior, incoming from the free stream
    assert np.allclose(vnb + 2 * cb / (G - 1), vnL + 2 * cL / (G - 1), rtol=0, atol=1e-13)
    assert np.allclose(vnb - 2 * cb / (G - 1), vni - 2 * ci / (G - 1), rtol=0, atol=1e-13)
    out = vnb > 0
    assert 40 < out.sum() < len(out) - 40          # both directions occur
    # entropy and tangential velocity from the upwind side
    s_b = pb / rb ** G
    assert np.allclose(s_b[out], (pL / rL ** G)[out], rtol=1e-13, atol=0)
    assert np.allclose(s_b[~out], p_i / rho_i ** G, rtol=1e-13, atol=0)
    tb = Vb - vnb * n
    assert np.allclose(tb[:, out], (VL - vnL * n)[:, out], rtol=0, atol=1e-13)
    assert np.allclose(tb[:, ~out], (Vi[:, None] - vni * n)[:, ~out], rtol=0, atol=1e-13)
    # the ghost used by the inviscid flux is the same state
    g, b = ph.bc_states(W.BC_FARFIELD, uL, N)
    assert np.array_equal(g, ub) and np.array_equal(b, ub)


@pytest.mark.parametrize("dim", [2, 3])
def test_farfield_supersonic_takes_one_side(dim):
    rng = np.random.default_rng(2)
    n = rng.standard_normal(dim)
    n /= np.linalg.norm(n)
    for sgn in (-1.0, 1.0):
        vinf = 1.6 * sgn * n                        # |V_inf.n| = 1.6 c_inf
        ph, uL, N, _, (rho_i, Vi, p_i) = _farfield_case(3, dim, vinf, K=50, amp=0.05)
        N = n[:, None] * np.ones((1, uL.shape[1]))
        ub = ph.farfield_state(uL, N)
        if sgn < 0:   # supersonic inflow: the free stream
            want = _cons(np.full(uL.shape[1], rho_i), np.repeat(Vi[:, None], uL.shape[1], 1),
                         np.full(uL.shape[1], p_i))
            assert np.allclose(ub, want, rtol=1e-15, atol=0)
        else:         # supersonic outflow: the interior state
            assert np.array_equal(ub, uL)


# ----------------------------------------------------------------- slip wall
@pytest.mark.parametrize("dim", [2, 3])
def test_slip_wall_flux_and_state(dim):
    rng = np.random.default_rng(4)
    K = 200
    ph = NavierStokes(dim, mu=0.0)
    rho = rng.uniform(0.8, 1.2, K)
    V = rng.uniform(-0.6, 0.6, (dim, K))
    p = rng.uniform(0.7, 1.3, K)
    uL = _cons(rho, V, p)
    N = rng.standard_normal((dim, K)) * rng.uniform(0.5, 2.0, K)
    n = N / np.linalg.norm(N, axis=0)
    ghost, ub = ph.bc_states(W.BC_WALL, uL, N)
    F = ph.rusanov(uL, ghost, N)
    scale = np.abs(F).max()
    assert np.abs(F[0]).max() <= 1e-15 * scale          # no mass through the wall
    assert np.abs(F[-1]).max() <= 1e-14 * scale         # no energy through the wall
    Fm = F[1:1 + dim]
    tang = Fm - np.sum(Fm * n, 0) * n
    assert np.abs(tang).max() <= 1e-14 * scale          # momentum flux normal to the wall
    # with no normal velocity, the momentum flux is the pressure force p N
    Vt = V - np.sum(V * n, 0) * n
    ut = _cons(rho, Vt, p)
    gt, _ = ph.bc_states(W.BC_WALL, ut, N)
    assert np.allclose(ph.rusanov(ut, gt, N)[1:1 + dim], p * N, rtol=0, atol=1e-14)
    # common solution: normal momentum removed, tangential kept, rho and p kept
    rb, Vb, pb = _prim(ub, dim)
    assert np.allclose(rb, rho, rtol=1e-15, atol=0)
    assert np.abs(np.sum(Vb * n, 0)).max() < 1e-15
    assert np.allclose(Vb, V - np.sum(V * n, 0) * n, rtol=0, atol=1e-15)
    assert np.allclose(pb, p, rtol=1e-14, atol=0)


def test_slip_channel_keeps_mass_energy_and_parallel_momentum():
    # a straight channel turned about (1, 2, 3), slip walls on both y faces,
    # periodic in x and z; any smooth state
    ax = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
    Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rt = np.eye(3) + math.sin(0.5) * Kx + (1 - math.cos(0.5)) * Kx @ Kx
    nodes, conn = W.box_mesh(3, [3, 4, 2], 0.0, [1.5, 1.0, 0.5], q=1, walls_y=True)
    nodes = np.asarray(nodes) @ Rt.T
    m = Mesh(nodes, conn, 2)
    u = np.ascontiguousarray(np.moveaxis(W.random_smooth_state(m.xsp @ Rt, seed=11, periods=[1.5, 1.0, 0.5]), 0, 1))
    R = FRSolver(m, NavierStokes(3, mu=0.0)).residual(u)
    tot = np.einsum("evs,es,s->v", R, m.J, m.sp_weights())
    scale = np.einsum("evs,es,s->v", np.abs(R), m.J, m.sp_weights()).max()
    mom = Rt.T @ tot[1:4]                                 # momentum rate in the channel frame
    assert abs(tot[0]) <= 1e-13 * scale and abs(tot[4]) <= 1e-13 * scale
    assert abs(mom[0]) <= 1e-13 * scale and abs(mom[2]) <= 1e-13 * scale
    assert abs(mom[1]) > 1e-6 * scale                     # the walls do push in y
    # a uniform flow parallel to the walls is steady
    V = Rt @ np.array([0.4, 0.0, -0.2])
    uu = np.ascontiguousarray(np.moveaxis(W.uniform_state((m.E, m.Nsp), 1.1, V, 0.9), 0, 1))
    R0 = FRSolver(m, NavierStokes(3, mu=0.0)).residual(uu)
    assert np.abs(R0).max() < 1e-12


# ------------------------------------------------------------------ BR2 lift
@pytest.mark.parametrize("kind,p", [(DG, 2), (DG, 3), (HUYNH_G2, 3)])
@pytest.mark.parametrize("eta", [1.0, 2.0])
def test_br2_lifting_is_the_single_face_correction(kind, p, eta):
    # affine periodic box turned about (1, 2, 3) and sheared: full metric
    # matrices; state constant in each element, so every gradient comes from
    # the lifting alone
    ax = np.array([1.0, 2.0, 3.0]) / math.sqrt(14.0)
    Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    A = (np.eye(3) + math.sin(0.5) * Kx + (1 - math.cos(0.5)) * Kx @ Kx) @ np.array(
        [[1.0, 0.3, 0.0], [0.0, 0.8, 0.2], [0.0, 0.0, 1.2]])
    nodes, conn = W.box_mesh(3, [3, 3, 3], 0.0, 1.0, q=1)
    nodes = np.ascontiguousarray(np.asarray(nodes) @ A.T)
    m = Mesh(nodes, conn, p, kind=kind)
    E = m.E
    rng = np.random.default_rng(7)
    c = _cons(rng.uniform(0.8, 1.2, E), rng.uniform(-0.3, 0.3, (3, E)), rng.uniform(0.8, 1.2, E))  # [5, E]
    u = np.repeat(c.T[:, :, None], m.Nsp, axis=2)
    ph = NavierStokes(3, mu=0.05, eta=eta)
    _, faces = FRSolver(m, ph).residual(u, want_faces=True)
    # element Jacobian matrix B = dx/dxi from the corner nodes (node a+2b+4c)
    X = np.asarray(nodes)
    B = np.stack([(X[:, 1] - X[:, 0]) / 2, (X[:, 2] - X[:, 0]) / 2, (X[:, 4] - X[:, 0]) / 2], axis=2)
    Binv = np.linalg.inv(B)                               # [E, d, i] = dxi_d/dx_i
    # g'(-1) of g_L and g'(+1) of g_R = -g_L'(-1): closed forms of the
    # correction functions (DG: right Radau of degree p+1; Huynh g2)
    gl = -(p + 1) ** 2 / 2.0 if kind == DG else -p * (p + 1) / 2.0
    for e in range(E):
        for f in range(6):
            d, s = divmod(f, 2)
            ne = conn[e, f, 0]
            jump = 0.5 * (c[:, ne] - c[:, e])             # u_c - u_f on this face
            gp = gl if s == 0 else -gl
            want = eta * gp * jump[:, None] * Binv[e, d][None, :]   # [v, i]
            got = faces["Gface"][e, f]                    # [v, i, fp]
            assert np.allclose(got, want[:, :, None], rtol=0, atol=1e-12 * max(1.0, np.abs(want).max()))
            # the common viscous flux: both sides carry the same lifted
            # gradient, so it is the mean viscous flux of the two states
            Nf = m.N[e, f]                                # [fp, i]
            Fv = 0.5 * (ph.flux_vis(c[:, e][:, None], want[:, :, None])[..., 0]
                        + ph.flux_vis(c[:, ne][:, None], want[:, :, None])[..., 0])   # [v, i]
            assert np.allclose(faces["Fv_common"][e, f], Fv @ Nf.T, rtol=0,
                               atol=1e-12 * max(1e-3, np.abs(Fv).max()))


# ------------------------------------------------------------------ sampling
@pytest.mark.parametrize("p", [2, 3])
def test_sampling_exact_for_degree_p_tensor_polynomials(p):
    nodes, conn = W.ogrid_mesh(24, 4, 2, 0.2, r_outer=3.0, first_cell=0.05)
    m = Mesh(nodes, conn, p)
    E = m.E
    rng = np.random.default_rng(9)
    # per element and variable: sum_{a,b,c <= p} C[a,b,c] xi^a eta^b zeta^c,
    # every coefficient of the top degree non-zero
    C = rng.uniform(-1.0, 1.0, (E, 5, p + 1, p + 1, p + 1)) * 0.05
    base = np.array([1.0, 0.3, -0.2, 0.1, 3.0])
    x1, _ = np.polynomial.legendre.leggauss(p + 1)        # GL solution points

    def poly(Ce, xi):                                     # Ce [5, a, b, c], xi [K, 3]
        P = [np.stack([xi[:, d] ** k for k in range(p + 1)], 1) for d in range(3)]   # [K, p+1]
        return base[:, None] + np.einsum("vabc,ka,kb,kc->vk", Ce, P[0], P[1], P[2])

    sp = np.array([[x1[i], x1[j], x1[k]] for k in range(p + 1) for j in range(p + 1) for i in range(p + 1)])
    u = np.stack([poly(C[e], sp) for e in range(E)])      # [E, 5, Nsp]
    y, _, _ = W.cylinder_surface(radius=1.5, center=(0.5, 0.0), spacing=0.1, span=0.2)
    el, xi = locate(m, y)
    # the element map (triquadratic on equispaced nodes) reproduces each point
    def lag3(t):
        return np.array([t * (t - 1) / 2, 1 - t * t, t * (t + 1) / 2])
    for k in range(len(y)):
        w = np.einsum("c,b,a->cba", lag3(xi[k, 2]), lag3(xi[k, 1]), lag3(xi[k, 0])).ravel()
        assert np.allclose(w @ np.asarray(nodes)[el[k]], y[k], rtol=0, atol=1e-12)
    got = sample(m, NavierStokes(3), u, el, xi)
    for k in range(len(y)):
        uk = poly(C[el[k]], xi[k][None])[:, 0]
        rho, V, pr = _prim(uk[:, None], 3)
        assert np.allclose(got[k], np.concatenate([rho, V[:, 0], pr]), rtol=0, atol=1e-12)
