"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a textbook
exact solution, a convergence order the paper states, an invariant of the
discrete scheme, or a special case that reduces to a textbook routine.
Together they are chosen so that a dropped term, a wrong sign or index, or a
transposed operand anywhere in the oracle fails at least one of them
(``test_oracle_mutants.py`` plants such mistakes to show it).
"""
import math
import os

import numpy as np
import pytest

from oracle import exact
from paper_0910_2854_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make_box(oracle_mod, w, **kw):
    ob = oracle_mod.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h, phi=w.phi, **kw)
    ob.set_state(w.state)
    return ob


def run_to(ob, T, cfl=0.5):
    t = 0.0
    n = 0
    while t < T - 1e-14:
        dt = min(ob.cfl(cfl), (T - t) / 2.0)
        ob.step(dt)
        t += 2.0 * dt
        n += 1
    return n


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


# ---------------------------------------------------------------------------
# the exact Riemann solver itself (used as the Sod reference)
# ---------------------------------------------------------------------------

def test_exact_riemann_reproduces_toro_table():
    g = read_golden("toro_sod_star_state.txt")
    ps, us = exact.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    assert abs(ps - g["p_star"]) < 1e-5
    assert abs(us - g["u_star"]) < 1e-5
    # star densities sampled just left / right of the contact
    r, u, p = exact.riemann_euler((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4,
                                  np.array([us - 1e-9, us + 1e-9]))
    assert abs(r[0] - g["rho_star_left"]) < 1e-5
    assert abs(r[1] - g["rho_star_right"]) < 1e-5


def test_exact_riemann_jump_conditions():
    """Rankine-Hugoniot across the right shock and isentropy across the left
    rarefaction of the exact solution (independent of any tabulated value)."""
    gam = 1.4
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = exact.star_state(L, R, gam)
    cr = math.sqrt(gam * R[2] / R[0])
    S = R[1] + cr * math.sqrt((gam + 1) / (2 * gam) * ps / R[2] + (gam - 1) / (2 * gam))
    r2, u2, p2 = exact.riemann_euler(L, R, gam, np.array([S - 1e-9]))
    r1, u1, p1 = R
    # mass and momentum flux continuity in the shock frame
    assert abs(r2[0] * (u2[0] - S) - r1 * (u1 - S)) < 1e-9
    assert abs(r2[0] * (u2[0] - S) ** 2 + p2[0] - (r1 * (u1 - S) ** 2 + p1)) < 1e-9
    # left rarefaction: p / rho^gamma constant and u + 2c/(gam-1) constant
    xi = np.linspace(-1.1, us - 0.1, 7)
    r, u, p = exact.riemann_euler(L, R, gam, xi)
    s = p / r ** gam
    assert np.allclose(s, 1.0, rtol=1e-12)
    riem = u + 2 * np.sqrt(gam * p / r) / (gam - 1)
    assert np.allclose(riem, 2 * math.sqrt(gam) / (gam - 1), rtol=1e-12)


# ---------------------------------------------------------------------------
# P-1: Sod shock tube against the exact Riemann solution
# ---------------------------------------------------------------------------

def test_sod_converges_to_exact_solution(oracle_mod):
    errs = []
    for n in (64, 128, 256):
        w = W.sod(n, axis=0, ntrans=1)
        ob = make_box(oracle_mod, w)
        run_to(ob, 0.2)
        assert ob.flags == 0
        r, u, p = exact.riemann_cell_averages((1, 0, 1), (0.125, 0, 0.1), 1.4,
                                              np.linspace(0, 1, n + 1), 0.5, 0.2)
        errs.append(np.mean(np.abs(ob.state[0, 0, 0] - r)))
    assert errs[0] / errs[1] > 1.6 and errs[1] / errs[2] > 1.6
    assert errs[2] < 4e-3


# ---------------------------------------------------------------------------
# P-2: circularly polarised Alfven wave (Sec. 4), second order
# ---------------------------------------------------------------------------

def _alfven_error(oracle_mod, w):
    ob = make_box(oracle_mod, w)
    run_to(ob, 1.0)
    assert ob.flags == 0
    # the paper's norm: mean over cells of |u^n - u^0|, summed over components
    return float(np.sum(np.mean(np.abs(ob.state - w.state), axis=(1, 2, 3)))), ob


def test_alfven_wave_x_second_order(oracle_mod):
    errs = [_alfven_error(oracle_mod, W.alfven_x(n, 1, 1))[0] for n in (32, 64, 128)]
    order = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert order[0] > 1.8 and order[1] > 1.9, (errs, order)
    assert errs[2] < 5e-4


def test_alfven_wave_oblique_second_order(oracle_mod):
    """The paper's own setup: 2-D at 30 degrees on [0,1/cos a] x [0,1/sin a]."""
    errs = []
    for n in (16, 32, 64):
        e, ob = _alfven_error(oracle_mod, W.alfven_oblique(n))
        errs.append(e)
    order = math.log2(errs[1] / errs[2])
    assert order > 1.8, (errs, order)


def test_linear_fast_wave_second_order(oracle_mod):
    """Textbook fast magnetosonic eigenmode (oblique field): after one period
    the perturbation returns, with error falling at second order.  Exercises
    the compressive MHD coupling (pressure, b.v energy flux, b_t advection)
    that a circularly polarised Alfven wave leaves untouched."""
    errs = []
    for n in (32, 64, 128):
        w = W.fast_wave(n)
        ob = make_box(oracle_mod, w)
        run_to(ob, w.meta["period"])
        errs.append(np.sum(np.mean(np.abs(ob.state - w.state), axis=(1, 2, 3))) / w.meta["eps"])
    assert math.log2(errs[1] / errs[2]) > 1.9, errs
    assert errs[2] < 1e-2


# ---------------------------------------------------------------------------
# P-3: smooth advection, second order along every axis, identical errors
# ---------------------------------------------------------------------------

def test_entropy_wave_order_all_axes(oracle_mod):
    res = {}
    for ax in (0, 1, 2):
        errs = []
        for n in (32, 64, 128):
            w = W.entropy_wave(n, axis=ax, ntrans=1)
            ob = make_box(oracle_mod, w)
            run_to(ob, 1.0)
            errs.append(np.mean(np.abs(ob.state[0] - w.state[0])))
        res[ax] = errs
        assert math.log2(errs[1] / errs[2]) > 1.9
    assert res[0] == res[1] == res[2]


# ---------------------------------------------------------------------------
# P-4 / P-5: conservation and div b = 0 to round-off (periodic, no gravity)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lim", [0, 1])
def test_conservation_and_divergence(oracle_mod, lim):
    w = W.random_smooth(12, 10, 8, seed=3, h=(0.1, 0.07, 0.13))
    ob = make_box(oracle_mod, w, limiter=lim)
    d0 = ob.diag()
    div0 = _divergence(ob)
    dt = ob.cfl(0.5)
    ob.step(dt, 4)
    assert ob.flags == 0
    d1 = ob.diag()
    vol = np.prod(ob.h)
    scale = np.array([np.sum(np.abs(ob.state[f])) * vol for f in range(8)])
    assert np.all(np.abs(d1[:8] - d0[:8]) <= 1e-13 * scale), (d1[:8] - d0[:8]) / scale
    div1 = _divergence(ob)
    bmax = np.max(np.abs(ob.state[5:8]))
    assert np.max(np.abs(div1 - div0)) * min(ob.h) / bmax < 1e-13


def _divergence(ob):
    bx, by, bz = ob.state[5], ob.state[6], ob.state[7]
    return ((bx - np.roll(bx, 1, 2)) / ob.h[0] + (by - np.roll(by, 1, 1)) / ob.h[1]
            + (bz - np.roll(bz, 1, 0)) / ob.h[2])


def test_divergence_kept_under_outflow(oracle_mod):
    """Outflow: every stored face is updated by CT with ghost fluxes, so the
    divergence of cells whose faces are all stored keeps its initial value."""
    w = W.random_smooth(10, 9, 8, seed=5, bc=W.BC_OUTFLOW)
    ob = make_box(oracle_mod, w)
    div0 = _divergence(ob)[1:, 1:, 1:]
    ob.step(ob.cfl(0.4), 3)
    div1 = _divergence(ob)[1:, 1:, 1:]
    bmax = np.max(np.abs(ob.state[5:8]))
    assert np.max(np.abs(div1 - div0)) * min(ob.h) / bmax < 1e-13


def test_ct_leaves_fluid_and_energy_untouched(oracle_mod):
    """During B_d every non-magnetic quantity, E included, is held constant."""
    w = W.random_smooth(8, 7, 6, seed=1)
    for d in range(3):
        ob = make_box(oracle_mod, w)
        before = ob.state.copy()
        ob.ct(d, 0.01)
        assert np.array_equal(ob.state[:5], before[:5])
        assert not np.array_equal(ob.state[5:], before[5:])


def test_fluid_leaves_field_untouched(oracle_mod):
    w = W.random_smooth(8, 7, 6, seed=2)
    for d in range(3):
        ob = make_box(oracle_mod, w)
        before = ob.state.copy()
        ob.fluid(d, 0.01)
        assert np.array_equal(ob.state[5:], before[5:])
        assert not np.array_equal(ob.state[:5], before[:5])


# ---------------------------------------------------------------------------
# P-6: special cases
# ---------------------------------------------------------------------------

def test_uniform_state_is_bitwise_fixed_point(oracle_mod):
    st = W.assemble(np.full((5, 6, 7), 1.3), (0.4, -0.2, 0.7), 0.9, (0.3, -0.5, 0.25), 5 / 3, 0)
    w = W.Workload("u", st, 5 / 3, (0.1, 0.2, 0.3))
    ob = make_box(oracle_mod, w)
    ob.step(0.01, 3)
    assert np.array_equal(ob.state, st)


def _euler_rusanov_pc(u, gam, dt, h):
    """Textbook (LeVeque) two-stage scheme with the local Lax-Friedrichs /
    Rusanov flux for the 1-D Euler equations on a periodic grid: half step
    with the first-order flux, full step with the first-order flux of the
    half-step state.  Independent numpy implementation."""
    def flux(u):
        rho, m, E = u
        v = m / rho
        p = (gam - 1) * (E - 0.5 * m * v)
        c = np.sqrt(gam * p / rho)
        return np.array([m, m * v + p, (E + p) * v]), np.abs(v) + c

    def llf(u):
        F, s = flux(u)
        Fr, sr = np.roll(F, -1, 1), np.roll(s, -1)
        ur = np.roll(u, -1, 1)
        return 0.5 * (F + Fr) - 0.5 * np.maximum(s, sr) * (ur - u)

    Fh = llf(u)
    uh = u - dt / (2 * h) * (Fh - np.roll(Fh, 1, 1))
    Ff = llf(uh)
    return u - dt / h * (Ff - np.roll(Ff, 1, 1))


def test_limiter_off_reduces_to_rusanov(oracle_mod):
    """Limiter identically zero: the TVD corrector flux collapses to the
    first-order Rusanov / LLF flux of the predicted state."""
    n, gam = 40, 1.4
    x = (np.arange(n) + 0.5) / n
    rho = 1 + 0.3 * np.sin(2 * np.pi * x)
    v = 0.5 * np.cos(2 * np.pi * x)
    p = 1 + 0.2 * np.sin(4 * np.pi * x)
    z = np.zeros(n)
    st = W.assemble(rho[None, None], (v[None, None], z[None, None], z[None, None]), p[None, None],
                    (z[None, None],) * 3, gam, 0)
    w = W.Workload("e", st, gam, (1.0 / n, 1.0, 1.0))
    ob = make_box(oracle_mod, w, limiter=oracle_mod.LIM_NONE)
    dt = 0.3 / n
    ob.fluid(0, dt)
    u = np.array([rho, rho * v, st[4, 0, 0]])
    ref = _euler_rusanov_pc(u, gam, dt, 1.0 / n)
    got = np.array([ob.state[0, 0, 0], ob.state[1, 0, 0], ob.state[4, 0, 0]])
    assert np.max(np.abs(got - ref)) < 1e-13


def _discrete_atmosphere(n, c0=1.0, gam=5 / 3, g=2.0):
    """Gas at rest with uniform sound speed c0 (p = c0^2 rho / gamma) in
    phi = g x, built so that the density difference of every interface equals
    the hydrostatic estimate of eq0321 exactly:
    rho_{j+1} - rho_j = -(rho_j + rho_{j+1}) (phi_{j+1} - phi_j) / (2 c0^2)."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    phi = g * x
    a = g * h / (2 * c0 * c0)
    rho = (1.0 * ((1 - a) / (1 + a)) ** np.arange(n))
    one = np.ones((1, 1, n))
    st = W.assemble(rho[None, None] * one, (0 * one,) * 3, (c0 * c0 / gam) * rho[None, None] * one,
                    (0 * one,) * 3, gam, W.BC_OUTFLOW)
    return W.Workload("atm", st, gam, (h, 1.0, 1.0), bc=W.BC_OUTFLOW, phi=phi[None, None] * one)


def test_hse_correction_removes_hydrostatic_dissipation(oracle_mod):
    """In a discrete hydrostatic atmosphere the HSE-corrected difference
    delta u of the density vanishes (eq0323), so the acoustic dissipation of
    the mass flux disappears: the density moves far less with the correction
    than with the plain relaxation flux (eq0140).  The limiter is switched off
    so that the first-order dissipation is not partly cancelled by the TVD
    slopes (on an exactly geometric profile the Van Leer slopes cancel it
    completely); what remains with the correction is the advective mass flux
    of the small momentum imbalance."""
    n = 32
    w = _discrete_atmosphere(n)
    drift = {}
    for hse in (False, True):
        ob = make_box(oracle_mod, w, hse=hse, limiter=oracle_mod.LIM_NONE)
        ob.fluid(0, 0.2 / n)
        inner = slice(4, n - 4)
        drift[hse] = np.max(np.abs(ob.state[0, 0, 0, inner] - w.state[0, 0, 0, inner]))
    assert drift[True] < 0.15 * drift[False], drift


def test_free_fall_in_linear_potential(oracle_mod):
    """Uniform gas at rest in phi = g x: interior cells follow the exact free
    fall of one operator step, m = -rho g dt and E gains rho g^2 dt^2 / 2
    (source of eq0254 with the sign of S_x)."""
    n, g, dt = 16, 0.7, 0.01
    x = (np.arange(n) + 0.5) / n
    one = np.ones((1, 1, n))
    st = W.assemble(one, (0 * one,) * 3, 1.0, (0 * one,) * 3, 5 / 3, W.BC_OUTFLOW)
    phi = (g * x)[None, None] * one
    w = W.Workload("ff", st, 5 / 3, (1.0 / n, 1.0, 1.0), bc=W.BC_OUTFLOW, phi=phi)
    ob = make_box(oracle_mod, w)
    ob.fluid(0, dt)
    inner = slice(4, n - 4)
    assert np.allclose(ob.state[1, 0, 0, inner], -g * dt, rtol=1e-13, atol=0)
    assert np.allclose(ob.state[4, 0, 0, inner], st[4, 0, 0, inner] + 0.5 * g * g * dt * dt,
                       rtol=1e-13, atol=0)
    assert np.allclose(ob.state[0, 0, 0, inner], 1.0, rtol=1e-14, atol=0)


def test_cfl_closed_form_fast_speed(oracle_mod):
    """Fast speed limits: along b it is max(a, v_A); across b it is
    sqrt(a^2 + v_A^2) (reading C-1); dt = k min_d h_d / (|v_d| + c_F,d)."""
    gam, rho, p, B = 5 / 3, 2.0, 0.6, 1.1
    a2 = gam * p / rho
    va2 = B * B / rho
    v = (0.3, -0.2, 0.1)
    h = (0.05, 0.07, 0.11)
    one = np.ones((3, 4, 5))
    st = W.assemble(rho * one, tuple(c * one for c in v), p, (B * one, 0 * one, 0 * one), gam, 0)
    w = W.Workload("c", st, gam, h)
    ob = make_box(oracle_mod, w)
    cf = [max(math.sqrt(a2), math.sqrt(va2)), math.sqrt(a2 + va2), math.sqrt(a2 + va2)]
    ref = 0.8 * min(h[d] / (abs(v[d]) + cf[d]) for d in range(3))
    assert abs(ob.cfl(0.8) - ref) < 1e-14 * ref


# ---------------------------------------------------------------------------
# P-7: axis permutation and mirror symmetry
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["sod", "brio_wu"])
def test_axis_permutation_bitwise(oracle_mod, kind):
    """A 1-D tube along x, y or z gives bitwise identical profiles with the
    components permuted.  For an MHD tube the constraint update of the
    transverse field comes from B_{d+1}, which sits between the two
    d-sweeps in the x-y-z-z-y-x order for d = x, y but outside them for
    d = z, so only x and y are compared there."""
    outs = []
    axes = range(3) if kind == "sod" else range(2)
    for ax in axes:
        w = W.sod(64, axis=ax, ntrans=1) if kind == "sod" else W.brio_wu(64, axis=ax, ntrans=1)
        ob = make_box(oracle_mod, w, limiter=1)
        for _ in range(10):
            ob.step(0.2 / 64)
        assert ob.flags == 0
        st = ob.state.reshape(8, -1)
        # rotate components back to the frame of the tube: (n, t1, t2)
        perm_m = [1 + ax, 1 + (ax + 1) % 3, 1 + (ax + 2) % 3]
        perm_b = [5 + ax, 5 + (ax + 1) % 3, 5 + (ax + 2) % 3]
        outs.append(st[[0] + perm_m + [4] + perm_b])
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


def test_mirror_symmetry_sod(oracle_mod):
    a = make_box(oracle_mod, W.sod(64, ntrans=1))
    b = make_box(oracle_mod, W.sod(64, ntrans=1, mirror=True))
    for _ in range(8):
        a.step(0.25 / 64)
        b.step(0.25 / 64)
    ra, rb = a.state[0, 0, 0], b.state[0, 0, 0][::-1]
    assert np.max(np.abs(ra - rb)) < 1e-13
    assert np.max(np.abs(a.state[1, 0, 0] + b.state[1, 0, 0][::-1])) < 1e-13


def test_three_rotations_identity(oracle_mod):
    """The paper's data rotation (2 pi/3 about (1,1,1), Sec. 3): the cyclic
    relabelling (x,y,z) -> (y,z,x) applied three times is the identity, and a
    y-sweep pair L_y B_y of a state equals the x-sweep pair L_x B_x of the
    rotated state, rotated back."""
    w = W.random_smooth(6, 6, 6, seed=7)
    st = w.state

    def rot(s):
        # new x = old y, new y = old z, new z = old x; numpy order (z, y, x)
        r = np.transpose(s, (0, 3, 1, 2))
        return r[[0, 2, 3, 1, 4, 6, 7, 5]]

    assert np.array_equal(rot(rot(rot(st))), st)
    a = make_box(oracle_mod, w)
    a.fluid(1, 0.01)
    a.ct(1, 0.01)
    b = make_box(oracle_mod, W.Workload("r", rot(st), w.gamma, w.h))
    b.fluid(0, 0.01)
    b.ct(0, 0.01)
    assert np.max(np.abs(rot(a.state) - b.state)) < 1e-14


# ---------------------------------------------------------------------------
# hybrid limiter (Van Leer subsonic, minmod supersonic; Sec. 2.2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("vel, twin", [(0.5, "vanleer"), (3.0, "minmod")])
def test_hybrid_limiter_limits(oracle_mod, vel, twin):
    """An entropy wave advected at |v| < c_s everywhere (c_s >= 1.17) is
    advanced exactly as with Van Leer; at |v| > c_s everywhere (c_s <= 1.44)
    exactly as with minmod."""
    w = W.entropy_wave(24, axis=0, ntrans=4, vel=vel)
    lim = oracle_mod.LIM_VANLEER if twin == "vanleer" else oracle_mod.LIM_MINMOD
    a = make_box(oracle_mod, w, limiter=oracle_mod.LIM_HYBRID)
    b = make_box(oracle_mod, w, limiter=lim)
    for _ in range(4):
        dt = a.cfl(0.5)
        a.step(dt)
        b.step(dt)
    assert np.array_equal(a.state, b.state)


def test_hybrid_limiter_mixed_flow(oracle_mod):
    """Gas at Mach 1.7 (left) driven into gas at rest (right): the flow has
    both sub- and supersonic interfaces, and the hybrid result differs from
    each pure limiter."""
    w = W.shock_tube(64, 0, 4, left=(1.0, 2.0, 1.0), right=(0.125, 0.0, 0.1), gamma=1.4)
    res = {}
    for lim in (oracle_mod.LIM_HYBRID, oracle_mod.LIM_VANLEER, oracle_mod.LIM_MINMOD):
        ob = make_box(oracle_mod, w, limiter=lim)
        for _ in range(6):
            ob.step(ob.cfl(0.4))
        res[lim] = ob.state[0]
    assert not np.array_equal(res[oracle_mod.LIM_HYBRID], res[oracle_mod.LIM_VANLEER])
    assert not np.array_equal(res[oracle_mod.LIM_HYBRID], res[oracle_mod.LIM_MINMOD])


# ---------------------------------------------------------------------------
# operator-split gravity G(dt/2) L G(dt/2) (eq025111-eq02513)
# ---------------------------------------------------------------------------

def test_split_gravity_free_fall(oracle_mod):
    """Uniform gas in a linear potential phi = g x: L_d leaves a uniform
    state unchanged and G is exact for constant rho, so after a double step
    of 2 dt the interior cells carry the momentum -rho g (2 dt) and their
    internal energy is unchanged (the split operator moves only momentum)."""
    n, g, rho, p, gam = 32, 0.7, 1.3, 2.0, 5.0 / 3.0
    shape = (4, 4, n)
    x = (np.arange(n) + 0.5) / n
    phi = np.broadcast_to(g * x, shape).copy()
    b = (0.3, 0.2, 0.1)
    zero = np.zeros(shape)
    st = W.assemble(rho + zero, (zero, zero, zero), p + zero, tuple(c + zero for c in b), gam, W.BC_OUTFLOW)
    ob = oracle_mod.OracleBox(n, 4, 4, gam, bc=W.BC_OUTFLOW, phi=phi, gravity_split=True)
    ob.set_state(st)
    dt = 0.3 * ob.cfl(1.0)
    ob.step(dt)
    inner = slice(10, 22)
    mx = ob.state[1][..., inner]
    assert np.allclose(mx, -rho * g * 2 * dt, rtol=1e-12, atol=0)
    eint = ob.state[4][..., inner] - 0.5 * ob.state[1][..., inner] ** 2 / rho - 0.5 * sum(c * c for c in b)
    assert np.allclose(eint, p / (gam - 1.0), rtol=1e-12, atol=0)
    assert np.all(ob.state[0][..., inner] == rho)
    # the unsplit form reaches the same momentum through its own source terms
    ou = oracle_mod.OracleBox(n, 4, 4, gam, bc=W.BC_OUTFLOW, phi=phi)
    ou.set_state(st)
    ou.step(dt)
    assert not np.array_equal(ou.state, ob.state)


# ---------------------------------------------------------------------------
# irregular Cartesian meshes (Sec. 2.5, eq037, eq0420; readings C-23 .. C-27)
# ---------------------------------------------------------------------------

def stretched(n, L=1.0, amp=0.3, phase=0.0):
    """Smoothly varying positive cell widths summing to L (periodic in i)."""
    x = (np.arange(n) + 0.5) / n
    w = 1.0 + amp * np.sin(2 * np.pi * x + phase)
    return L * w / w.sum()


def centres(w):
    return np.cumsum(w) - 0.5 * w


def nu_box(oracle_mod, w, widths, **kw):
    ob = oracle_mod.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h, phi=w.phi, widths=widths, **kw)
    ob.set_state(w.state)
    return ob


def nu_divergence(ob):
    b = ob.state[5:8]
    wx, wy, wz = (ob.widths[d] if ob.widths[d] is not None else np.full(ob.n[d], ob.h[d]) for d in range(3))
    return ((b[0] - np.roll(b[0], 1, 2)) / wx[None, None, :] + (b[1] - np.roll(b[1], 1, 1)) / wy[None, :, None]
            + (b[2] - np.roll(b[2], 1, 0)) / wz[:, None, None])


def test_irregular_mesh_with_uniform_widths_is_the_uniform_method(oracle_mod):
    """Width arrays that are all equal give the printed uniform-mesh method
    up to rounding (the per-length slopes times half a width reduce to
    eq0230, the centre span to 2h)."""
    w = W.random_smooth(10, 9, 8, seed=61, h=(0.1, 0.11, 0.125))
    phi = 0.3 * np.sin(2 * np.pi * np.arange(10) / 10)[None, None, :] * np.ones((8, 9, 10))
    w = W.Workload("r", w.state, w.gamma, w.h, w.bc, phi=phi)
    for lim in (0, 1, 3):
        a = make_box(oracle_mod, w, limiter=lim)
        b = nu_box(oracle_mod, w, [np.full(n, h) for n, h in zip(w.dims, w.h)], limiter=lim)
        dt = a.cfl(0.5)
        assert abs(b.cfl(0.5) - dt) <= 1e-15 * dt
        a.step(dt, 2)
        b.step(dt, 2)
        assert np.max(np.abs(a.state - b.state)) <= 1e-13 * np.max(np.abs(a.state))


@pytest.mark.parametrize("lim", [0, 1])
def test_irregular_mesh_conservation_and_divergence(oracle_mod, lim):
    """Periodic box stretched along every axis: the volume-weighted totals of
    all eight fields (sum u_ijk dx_i dy_j dz_k) and the discrete divergence
    with per-cell widths are kept to round-off (eq037 in flux form)."""
    w = W.random_smooth(12, 10, 9, seed=62)
    widths = [stretched(12, phase=0.3), stretched(10, amp=0.4, phase=1.1), stretched(9, amp=0.25, phase=2.0)]
    ob = nu_box(oracle_mod, w, widths, limiter=lim)
    d0 = ob.diag()
    div0 = nu_divergence(ob)
    ob.step(ob.cfl(0.5), 3)
    d1 = ob.diag()
    vol = widths[0][None, None, :] * widths[1][None, :, None] * widths[2][:, None, None]
    scale = np.array([np.sum(np.abs(ob.state[f]) * vol) for f in range(8)])
    assert np.all(np.abs(d1[:8] - d0[:8]) <= 1e-13 * scale)
    div1 = nu_divergence(ob)
    assert np.max(np.abs(div1 - div0)) * min(min(x) for x in widths) / np.max(np.abs(ob.state[5:8])) < 1e-13
    # the totals really are volume-weighted: plain sums are not conserved
    assert abs(np.sum(ob.state[0]) - np.sum(w.state[0])) > 1e-9


def test_irregular_mesh_uniform_state_is_fixed_point(oracle_mod):
    st = W.assemble(np.full((5, 6, 7), 1.3), (0.4, -0.2, 0.7), 0.9, (0.3, -0.5, 0.25), 5 / 3, 0)
    w = W.Workload("u", st, 5 / 3, (0.1, 0.2, 0.3))
    ob = nu_box(oracle_mod, w, [stretched(7, 0.7), stretched(6, 1.2, 0.4), stretched(5, 1.5, 0.2, 1.0)])
    ob.step(0.01, 2)
    assert np.max(np.abs(ob.state - st)) <= 1e-14 * np.max(np.abs(st))


@pytest.mark.parametrize("split", [False, True])
def test_irregular_mesh_free_fall(oracle_mod, split):
    """Uniform gas at rest in phi = g x on a stretched outflow mesh: the
    centred difference over the centre span (reading C-26) is exactly g, so
    interior cells gain -rho g dt of momentum in one L_x (unsplit source) or
    one G L G (split), with the internal energy unchanged."""
    n, g, rho, p, gam = 24, 0.7, 1.3, 2.0, 5.0 / 3.0
    wx = stretched(n, amp=0.5)
    x = centres(wx)
    shape = (1, 1, n)
    st = W.assemble(np.full(shape, rho), (0.0, 0.0, 0.0), p, (0.0, 0.0, 0.0), gam, W.BC_OUTFLOW)
    w = W.Workload("ff", st, gam, (1.0 / n, 1, 1), bc=W.BC_OUTFLOW, phi=np.broadcast_to(g * x, shape).copy())
    ob = nu_box(oracle_mod, w, [wx, None, None], gravity_split=split)
    dt = 0.004
    ob.fluid(0, dt)
    s = slice(4, n - 4)
    assert np.allclose(ob.state[1, 0, 0, s], -rho * g * dt, rtol=1e-12, atol=0)
    eint = ob.state[4, 0, 0, s] - 0.5 * ob.state[1, 0, 0, s] ** 2 / rho
    assert np.allclose(eint, p / (gam - 1), rtol=1e-12, atol=0)


def _mirror_x(st):
    """Reflection x -> -x of a state periodic in x: cells reversed, v_x and
    b_x change sign, b_x faces i+1/2 map to faces (n-2-i)+1/2."""
    out = st[..., ::-1].copy()
    out[1] = -out[1]
    out[5] = -np.roll(out[5], -1, axis=-1)
    return out


def test_irregular_mesh_mirror_symmetry(oracle_mod):
    """The method on a stretched mesh commutes with a reflection of state and
    mesh: catches a width taken from the wrong side of an interface."""
    w = W.random_smooth(16, 7, 6, seed=63)
    wx = stretched(16, amp=0.45, phase=0.7)
    wy, wz = stretched(7, amp=0.3), stretched(6, amp=0.2, phase=0.5)
    a = nu_box(oracle_mod, w, [wx, wy, wz])
    b = nu_box(oracle_mod, W.Workload("m", _mirror_x(w.state), w.gamma, w.h), [wx[::-1], wy, wz])
    dt = a.cfl(0.5)
    assert abs(b.cfl(0.5) - dt) <= 1e-15 * dt
    a.step(dt, 2)
    b.step(dt, 2)
    assert np.max(np.abs(_mirror_x(a.state) - b.state)) <= 1e-13 * np.max(np.abs(a.state))


def test_irregular_mesh_cfl_closed_form(oracle_mod):
    """eq0420: dt = k min over cells and axes of width / (|v_d| + c_F,d)."""
    gam, rho, p, B = 5 / 3, 2.0, 0.6, 1.1
    a2, va2 = gam * p / rho, B * B / rho
    v = (0.3, -0.2, 0.1)
    one = np.ones((3, 4, 5))
    st = W.assemble(rho * one, tuple(c * one for c in v), p, (B * one, 0 * one, 0 * one), gam, 0)
    widths = [stretched(5, 0.5, 0.4), stretched(4, 0.7, 0.3), stretched(3, 0.9, 0.2)]
    ob = nu_box(oracle_mod, W.Workload("c", st, gam, (0.1, 0.2, 0.3)), widths)
    cf = [max(math.sqrt(a2), math.sqrt(va2)), math.sqrt(a2 + va2), math.sqrt(a2 + va2)]
    ref = 0.8 * min(widths[d].min() / (abs(v[d]) + cf[d]) for d in range(3))
    assert abs(ob.cfl(0.8) - ref) < 1e-14 * ref


def face_velocity_case(oracle_mod, lib=None):
    """B_x on a shear flow v_x = U + s y (uniform in x) with b_y = b_y(x) on
    a mesh stretched along y: the face velocity interpolated linearly to
    the face y_{j+1/2} (reading C-27) is exactly U + s y_{j+1/2}, so each
    interior face pencil of b_y evolves as under the uniform velocity of its
    face.  True when every interior face matches to round-off."""
    nx, ny, U, s, dt = 16, 8, 0.3, 1.7, 0.01
    wy = stretched(ny, amp=0.5, phase=0.9)
    yc, yf = centres(wy), np.cumsum(wy)
    x = (np.arange(nx) + 0.5) / nx
    by = np.broadcast_to(0.2 + 0.1 * np.sin(2 * np.pi * x)[None, None, :], (1, ny, nx)).copy()
    zero = np.zeros((1, ny, nx))
    vx = np.broadcast_to((U + s * yc)[None, :, None], (1, ny, nx)).copy()

    def run(v):
        st = W.assemble(np.ones((1, ny, nx)), (v, zero, zero), 1.0, (zero, by, zero), 5 / 3, 0)
        ob = oracle_mod.OracleBox(nx, ny, 1, 5 / 3, lib=lib, widths=[None, wy, None])
        ob.set_state(st)
        ob.ct(0, dt)
        return ob.state[6, 0]

    got = run(vx)
    ok = True
    for j in range(ny - 1):
        ref = run(np.full((1, ny, nx), U + s * yf[j]))
        ok = ok and np.max(np.abs(got[j] - ref[j])) <= 1e-13
    return ok


def test_irregular_mesh_face_velocity_interpolation(oracle_mod):
    assert face_velocity_case(oracle_mod)


# ---------------------------------------------------------------------------
# constrained transport details (Sec. 2.4): closed forms of the linearised
# magnetic operator.  A face pencil of b_y along x, advanced by B_x with the
# limiter off (first-order corrector), is a linear recursion with constant
# coefficients when the velocity is uniform, so a single Fourier mode keeps
# its shape and is multiplied by an amplification factor G; and for a
# uniform b_y the response to a small velocity mode is linear in the mode,
# carrying the transfer function of the face-velocity smoothing.
# ---------------------------------------------------------------------------

def ct_upwind_mode_case(oracle_mod, lib=None):
    """Uniform velocity V > 0 (every edge velocity positive), b_y = A sin(theta i
    + phi), limiter off.  Upwind first-order predictor over half a step
    (eq0363 with the upwind cell of eq0364), then the corrector flux of the
    upwind predicted cell over a full step: with nu = V dt / h and
    z = 1 - exp(-i theta) the mode is multiplied by G = 1 - nu z + nu^2 z^2 / 2
    (the two-stage expansion of exp(-nu z)).  A downwind predictor gives
    1 - nu z - nu^2 z (exp(i theta) - 1) / 2 instead.  True when every face
    matches to 1e-14 of A."""
    n, m, A, phase, V, nu = 32, 3, 0.7, 0.4, 1.3, 0.4
    theta = 2 * np.pi * m / n
    i = np.arange(n)
    by = (A * np.sin(theta * i + phase))[None, None, :]
    one = np.ones((1, 1, n))
    st = W.assemble(one, (V * one, 0 * one, 0 * one), 1.0, (0 * one, by, 0 * one), 5 / 3, W.BC_PERIODIC)
    h = 1.0 / n
    ob = oracle_mod.OracleBox(n, 1, 1, 5 / 3, h=(h, 1.0, 1.0), limiter=2, lib=lib)
    ob.set_state(st)
    ob.ct(0, nu * h / V)
    z = 1 - np.exp(-1j * theta)
    G = 1 - nu * z + 0.5 * nu * nu * z * z
    ref = A * np.imag(G * np.exp(1j * (theta * i + phase)))
    return np.max(np.abs(ob.state[6, 0, 0] - ref)) <= 1e-14 * A


def ct_smoothing_case(oracle_mod, lib=None):
    """Uniform b_y = B, velocity V + eps sin(theta i) with eps << V (all edge
    velocities positive), limiter off.  To first order in eps the change of
    b_y is linear in the smoothed face velocity vh (eq0362), whose mode is
    the velocity mode times the [1,2,1]/4 transfer function cos^2(theta/2);
    with lambda = dt/h and z = 1 - exp(-i theta):
      (b_new - B) / eps = -lambda B cos^2(theta/2) Im[(z - V lambda z^2 / 2) e^{i theta i}].
    Without the smoothing the factor would be 1 (28 % off at this theta).
    True when the response matches to 1e-4 of its largest value (the
    remainder is of order eps)."""
    n, m, B, V, eps = 32, 5, 0.8, 1.1, 1e-6
    theta = 2 * np.pi * m / n
    i = np.arange(n)
    vx = (V + eps * np.sin(theta * i))[None, None, :]
    one = np.ones((1, 1, n))
    st = W.assemble(one, (vx, 0 * one, 0 * one), 1.0, (0 * one, B * one, 0 * one), 5 / 3, W.BC_PERIODIC)
    h = 1.0 / n
    lam = 0.45 / V
    ob = oracle_mod.OracleBox(n, 1, 1, 5 / 3, h=(h, 1.0, 1.0), limiter=2, lib=lib)
    ob.set_state(st)
    ob.ct(0, lam * h)
    got = (ob.state[6, 0, 0] - B) / eps
    z = 1 - np.exp(-1j * theta)
    ref = -lam * B * math.cos(theta / 2) ** 2 * np.imag((z - 0.5 * V * lam * z * z) * np.exp(1j * theta * i))
    return np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def ct_edge_velocity_case(oracle_mod, lib=None):
    """Irregular mesh along x (reading C-27): the edge velocity whose sign picks
    the upwind cell is the linear interpolation of the two smoothed face
    velocities to the interface, (w_b v_a + w_a v_b) / (w_a + w_b).  The cell
    velocities are linear in the cell index (the [1,2,1] smoothing leaves
    them unchanged away from the boundary) and change sign between cells 5
    and 6: v_5 = -0.3 a, v_6 = 0.7 a.  With widths (w_5, w_6) = (1, 4) the
    interpolated velocity at the interface is -0.1 a, so cell 6 is upwind;
    with (4, 1) it is +0.5 a and cell 5 is upwind.  b_y is 1 in cell 5 and
    0 elsewhere: when cell 6 is upwind of both its interfaces no flux reaches
    it and its b_y stays exactly 0; when cell 5 is upwind of the shared
    interface, b_y of cell 6 changes.  (Swapped weights, or the plain mean
    of the uniform mesh, pick cell 5 in both cases.)"""
    n, a, dt = 12, 0.1, 0.01
    i = np.arange(n)
    vx = (a * (i - 5.3))[None, None, :]
    by = np.zeros((1, 1, n))
    by[0, 0, 5] = 1.0
    one = np.ones((1, 1, n))
    st = W.assemble(one, (vx, 0 * one, 0 * one), 1.0, (0 * one, by, 0 * one), 5 / 3, W.BC_OUTFLOW)
    out = []
    for w5, w6 in ((1.0, 4.0), (4.0, 1.0)):
        wx = np.full(n, 1.0 / n)
        wx[5], wx[6] = w5 / n, w6 / n
        ob = oracle_mod.OracleBox(n, 1, 1, 5 / 3, bc=W.BC_OUTFLOW, h=(1.0 / n, 1.0, 1.0), limiter=2, lib=lib,
                                  widths=[wx, None, None])
        ob.set_state(st)
        ob.ct(0, dt)
        out.append(ob.state[6, 0, 0, 6])
    return out[0] == 0.0 and abs(out[1]) > 1e-4


def test_ct_upwind_predictor_mode_amplification(oracle_mod):
    assert ct_upwind_mode_case(oracle_mod)


def test_ct_face_velocity_smoothing_transfer_function(oracle_mod):
    assert ct_smoothing_case(oracle_mod)


def test_irregular_mesh_ct_edge_velocity_interpolation(oracle_mod):
    assert ct_edge_velocity_case(oracle_mod)
