"""Mutation test of the oracle pins: plant plausible mistakes (a wrong sign,
a dropped term, a wrong index, a transposed operand) in a copy of the oracle
source, compile it, and check that the pin battery rejects every mutant.
The unmodified oracle must pass the same battery.

The details of the constrained transport that no convergence order,
conservation law or divergence check tells apart -- the upwind (not
downwind) first-order predictor, the [1,2,1] smoothing of the face velocity
(eq0362) and, on an irregular mesh, the weights of the edge velocity
(reading C-27) -- are caught by closed forms of the linearised operator
(``test_oracle_pins.py``: mode amplification factor, smoothing transfer
function, upwind choice at a sign change of the interpolated velocity)."""
import math

import numpy as np
import pytest

from paper_0910_2854_gb300 import workloads as W

MUTANTS = {
    "ct_bz_sign_as_printed": ("nb[t2][idx] = q[5 + t2][idx] - dt", "nb[t2][idx] = q[5 + t2][idx] + dt"),
    "ct_constraint_index": ("(fa[s + 1] - fam[s + 1])", "(fa[s + 1] - fam[s])"),
    "ct_face_neighbour": ("cB[d] = s; cB[c] = fc + 1; cB[o] = fo;", "cB[d] = s; cB[c] = fc - 1; cB[o] = fo;"),
    "minus_slope_sign": ("slm = or_limit(lim, fm2 - fm1, fm3 - fm2);   /* eq0220 */",
                         "slm = or_limit(lim, fm1 - fm2, fm3 - fm2);   /* eq0220 */"),
    "hybrid_criterion_inverted": ("? OR_LIM_MINMOD : OR_LIM_VANLEER;", "? OR_LIM_VANLEER : OR_LIM_MINMOD;"),
    "split_gravity_sign": ("mn = mo - tau * rho * dphi;", "mn = mo + tau * rho * dphi;"),
    "nu_slope_width_other_side": ("        sp = dw[1];\n", "        sp = dw[2];\n"),
    "nu_update_neighbour_width": ("        const double he = nu ? dw[e] : hd;\n        for (k = 0; k < 5; ++k)\n            un[k]",
                                  "        const double he = nu ? dw[e + 1] : hd;\n        for (k = 0; k < 5; ++k)\n            un[k]"),
    "nu_centre_span_own_width": ("    return 0.5 * or_width(P, d, s - 1) + or_width(P, d, s) + 0.5 * or_width(P, d, s + 1);",
                                 "    return 2.0 * or_width(P, d, s);"),
    "nu_face_velocity_weights_swapped": ("vt[e] = (wB * (q[1 + d][iA] / q[0][iA]) + wA * (q[1 + d][iB] / q[0][iB])) / (wA + wB);",
                                         "vt[e] = (wA * (q[1 + d][iA] / q[0][iA]) + wB * (q[1 + d][iB] / q[0][iB])) / (wA + wB);"),
    "nu_constraint_width": ("ha = or_width(P, t1, a),", "ha = or_width(P, t1, a + 1),"),
    "nu_ct_corrector_width": ("f2[e] = wp[e] + 0.5 * dw[e] * or_limit", "f2[e] = wp[e] + 0.5 * dw[e + 1] * or_limit"),
    "split_gravity_energy_dropped": ("q[4][idx] = q[4][idx] + 0.5 * (mn * mn - mo * mo) / rho;", "(void)mo;"),
    "slopes_added": ("F[k] = fp1 + fm2 + 0.5 * (slp - slm);", "F[k] = fp1 + fm2 + 0.5 * (slp + slm);"),
    "freezing_speed_wrong_interface": ("double D = fmax(c1->d, c2->d);", "double D = fmax(c0->d, c1->d);"),
    "predictor_full_step": ("up[k] = u[k * m + e] - dt / (2.0 * he) *", "up[k] = u[k * m + e] - dt / he *"),
    "gravity_sign": ("up[1] = up[1] - 0.5 * dt * u[0 * m + e] * dphi;", "up[1] = up[1] + 0.5 * dt * u[0 * m + e] * dphi;"),
    "corrector_source_old_state": ("un[4] = un[4] - dt * S->up[1 * m + e] * dphi;", "un[4] = un[4] - dt * u[1 * m + e] * dphi;"),
    "pressure_drops_magnetic": ("p = (g - 1.0) * (u[4] - kin - mag);", "p = (g - 1.0) * (u[4] - kin);"),
    "flux_my_sign": ("c->F[2] = u[2] * v0 - bb[0] * bb[1];", "c->F[2] = u[2] * v0 + bb[0] * bb[1];"),
    "energy_flux_drops_bv": ("c->F[4] = (u[4] + ptot) * v0 - bb[0] * bv;", "c->F[4] = (u[4] + ptot) * v0;"),
    "fast_speed_wrong_component": ("disc = (a2 - B2) * (a2 - B2) + 4.0 * a2 * bt2;",
                                   "disc = (a2 - B2) * (a2 - B2) + 4.0 * a2 * bn2;"),
    "field_not_centred": ("bc3[ax] = 0.5 * (q[5 + ax][or_index(P, cm[0], cm[1], cm[2])] + q[5 + ax][idx]);",
                          "bc3[ax] = q[5 + ax][idx];"),
    "hse_sign": ("ddu[k] = or_minmod(du[k] - gk, du[k]);", "ddu[k] = or_minmod(du[k] + gk, du[k]);"),
    "ct_predictor_downwind": ("f1[e] = vbar > 0.0 ? w[e] : w[e + 1];", "f1[e] = vbar > 0.0 ? w[e + 1] : w[e];"),
    "ct_smoothing_dropped": ("vh[e] = 0.25 * (vt[e + 1] + 2.0 * vt[e] + vt[e - 1]);", "vh[e] = vt[e];"),
    "nu_edge_velocity_weights_swapped": ("return (wb * va + wa * vb) / (wa + wb);",
                                         "return (wa * va + wb * vb) / (wa + wb);"),
}


def _box(oracle_mod, lib, w, **kw):
    ob = oracle_mod.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h, phi=w.phi, lib=lib, **kw)
    ob.set_state(w.state)
    return ob


def _run(ob, T, cfl=0.5, max_steps=1500):
    t = 0.0
    n = 0
    while t < T - 1e-14:
        n += 1
        if n > max_steps:
            raise FloatingPointError("time step collapsed")
        dt = min(ob.cfl(cfl), (T - t) / 2)
        if not (dt > 0 and math.isfinite(dt)):
            raise FloatingPointError("bad dt")
        ob.step(dt)
        t += 2 * dt


def battery(oracle_mod, lib):
    """Names of the pin checks that fail for the oracle build ``lib``."""
    from test_oracle_pins import _discrete_atmosphere, _euler_rusanov_pc
    checks = {}

    def alfven():
        e = []
        for n in (32, 64):
            w = W.alfven_x(n, 1, 1)
            ob = _box(oracle_mod, lib, w)
            _run(ob, 1.0)
            e.append(np.sum(np.mean(np.abs(ob.state - w.state), axis=(1, 2, 3))))
        return math.log2(e[0] / e[1]) > 1.7 and e[1] < 2e-3

    def oblique():
        e = []
        for n in (16, 32):
            w = W.alfven_oblique(n)
            ob = _box(oracle_mod, lib, w)
            _run(ob, 1.0)
            e.append(np.sum(np.mean(np.abs(ob.state - w.state), axis=(1, 2, 3))))
        return math.log2(e[0] / e[1]) > 1.6 and e[1] < 1.5e-2

    def fastwave():
        e = []
        for n in (32, 64):
            w = W.fast_wave(n)
            ob = _box(oracle_mod, lib, w)
            _run(ob, w.meta["period"])
            e.append(np.sum(np.mean(np.abs(ob.state - w.state), axis=(1, 2, 3))) / w.meta["eps"])
        return math.log2(e[0] / e[1]) > 1.8 and e[1] < 5e-2

    def entropy():
        e = []
        for n in (32, 64):
            w = W.entropy_wave(n, 0, 1)
            ob = _box(oracle_mod, lib, w)
            _run(ob, 1.0)
            e.append(np.mean(np.abs(ob.state[0] - w.state[0])))
        return math.log2(e[0] / e[1]) > 1.8

    def sod():
        from oracle import exact
        w = W.sod(128, 0, 1)
        ob = _box(oracle_mod, lib, w)
        _run(ob, 0.2)
        r, _, _ = exact.riemann_cell_averages((1, 0, 1), (0.125, 0, 0.1), 1.4, np.linspace(0, 1, 129), 0.5, 0.2)
        return np.mean(np.abs(ob.state[0, 0, 0] - r)) < 7e-3

    def invariants():
        w = W.random_smooth(10, 9, 8, seed=3, h=(0.1, 0.07, 0.13))
        ob = _box(oracle_mod, lib, w)
        d0 = ob.diag()
        b = ob.state[5:8]
        div0 = ((b[0] - np.roll(b[0], 1, 2)) / ob.h[0] + (b[1] - np.roll(b[1], 1, 1)) / ob.h[1]
                + (b[2] - np.roll(b[2], 1, 0)) / ob.h[2])
        ob.step(ob.cfl(0.5), 2)
        d1 = ob.diag()
        vol = np.prod(ob.h)
        scale = np.array([np.sum(np.abs(ob.state[f])) * vol for f in range(8)])
        b = ob.state[5:8]
        div1 = ((b[0] - np.roll(b[0], 1, 2)) / ob.h[0] + (b[1] - np.roll(b[1], 1, 1)) / ob.h[1]
                + (b[2] - np.roll(b[2], 1, 0)) / ob.h[2])
        return (np.all(np.abs(d1[:8] - d0[:8]) <= 1e-13 * scale)
                and np.max(np.abs(div1 - div0)) * min(ob.h) / np.max(np.abs(b)) < 1e-13)

    def freefall():
        n, g, dt = 16, 0.7, 0.01
        x = (np.arange(n) + 0.5) / n
        one = np.ones((1, 1, n))
        st = W.assemble(one, (0 * one,) * 3, 1.0, (0 * one,) * 3, 5 / 3, W.BC_OUTFLOW)
        w = W.Workload("ff", st, 5 / 3, (1.0 / n, 1, 1), bc=W.BC_OUTFLOW, phi=(g * x)[None, None] * one)
        ob = _box(oracle_mod, lib, w)
        ob.fluid(0, dt)
        s = slice(4, n - 4)
        return (np.allclose(ob.state[1, 0, 0, s], -g * dt, rtol=1e-13, atol=0)
                and np.allclose(ob.state[4, 0, 0, s], st[4, 0, 0, s] + 0.5 * g * g * dt * dt, rtol=1e-13, atol=0))

    def cfl():
        gam, rho, p, B = 5 / 3, 2.0, 0.6, 1.1
        a2, va2 = gam * p / rho, B * B / rho
        v, h = (0.3, -0.2, 0.1), (0.05, 0.07, 0.11)
        one = np.ones((3, 4, 5))
        st = W.assemble(rho * one, tuple(c * one for c in v), p, (B * one, 0 * one, 0 * one), gam, 0)
        ob = _box(oracle_mod, lib, W.Workload("c", st, gam, h))
        cf = [max(math.sqrt(a2), math.sqrt(va2)), math.sqrt(a2 + va2), math.sqrt(a2 + va2)]
        ref = 0.8 * min(h[d] / (abs(v[d]) + cf[d]) for d in range(3))
        return abs(ob.cfl(0.8) - ref) < 1e-14 * ref

    def atmosphere():
        w = _discrete_atmosphere(32)
        dr = {}
        for hse in (False, True):
            ob = _box(oracle_mod, lib, w, hse=hse, limiter=2)
            ob.fluid(0, 0.2 / 32)
            dr[hse] = np.max(np.abs(ob.state[0, 0, 0, 4:-4] - w.state[0, 0, 0, 4:-4]))
        return dr[True] < 0.15 * dr[False]

    def rusanov():
        n, gam = 40, 1.4
        x = (np.arange(n) + 0.5) / n
        rho = 1 + 0.3 * np.sin(2 * np.pi * x)
        v = 0.5 * np.cos(2 * np.pi * x)
        p = 1 + 0.2 * np.sin(4 * np.pi * x)
        z = np.zeros(n)[None, None]
        st = W.assemble(rho[None, None], (v[None, None], z, z), p[None, None], (z,) * 3, gam, 0)
        ob = _box(oracle_mod, lib, W.Workload("e", st, gam, (1.0 / n, 1, 1)), limiter=2)
        dt = 0.3 / n
        ob.fluid(0, dt)
        ref = _euler_rusanov_pc(np.array([rho, rho * v, st[4, 0, 0]]), gam, dt, 1.0 / n)
        got = np.array([ob.state[0, 0, 0], ob.state[1, 0, 0], ob.state[4, 0, 0]])
        return np.max(np.abs(got - ref)) < 1e-13

    def uniform():
        st = W.assemble(np.full((5, 6, 7), 1.3), (0.4, -0.2, 0.7), 0.9, (0.3, -0.5, 0.25), 5 / 3, 0)
        ob = _box(oracle_mod, lib, W.Workload("u", st, 5 / 3, (0.1, 0.2, 0.3)))
        ob.step(0.01, 2)
        return np.array_equal(ob.state, st)

    def hybrid():
        ok = True
        for vel, lim in ((0.5, 0), (3.0, 1)):
            w = W.entropy_wave(24, axis=0, ntrans=4, vel=vel)
            a = _box(oracle_mod, lib, w, limiter=3)
            b = _box(oracle_mod, lib, w, limiter=lim)
            dt = a.cfl(0.5)
            a.step(dt)
            b.step(dt)
            ok = ok and np.array_equal(a.state, b.state)
        return ok

    def splitfall():
        n, g, rho, p = 16, 0.7, 1.3, 2.0
        shape = (1, 1, n)
        x = (np.arange(n) + 0.5) / n
        st = W.assemble(np.full(shape, rho), (0.0, 0.0, 0.0), p, (0.0, 0.0, 0.0), 5 / 3, W.BC_OUTFLOW)
        w = W.Workload("sf", st, 5 / 3, (1.0 / n, 1, 1), bc=W.BC_OUTFLOW, phi=np.broadcast_to(g * x, shape).copy())
        ob = _box(oracle_mod, lib, w, gravity_split=True)
        dt = 0.01
        ob.fluid(0, dt)
        s = slice(4, n - 4)
        return (np.allclose(ob.state[1, 0, 0, s], -rho * g * dt, rtol=1e-13, atol=0)
                and np.allclose(ob.state[4, 0, 0, s], p / (2 / 3) + 0.5 * (rho * g * dt) ** 2 / rho,
                                rtol=1e-13, atol=0))

    def nu_uniform():
        from test_oracle_pins import nu_box
        w = W.random_smooth(10, 9, 8, seed=61, h=(0.1, 0.11, 0.125))
        a = _box(oracle_mod, lib, w)
        b = oracle_mod.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h, lib=lib,
                                 widths=[np.full(n, h) for n, h in zip(w.dims, w.h)])
        b.set_state(w.state)
        dt = a.cfl(0.5)
        a.step(dt, 2)
        b.step(dt, 2)
        return np.max(np.abs(a.state - b.state)) <= 1e-13 * np.max(np.abs(a.state))

    def nu_conserve():
        from test_oracle_pins import stretched, nu_divergence
        w = W.random_smooth(12, 10, 9, seed=62)
        widths = [stretched(12, phase=0.3), stretched(10, amp=0.4, phase=1.1), stretched(9, amp=0.25, phase=2.0)]
        ob = oracle_mod.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h, lib=lib, widths=widths)
        ob.set_state(w.state)
        d0 = ob.diag()
        div0 = nu_divergence(ob)
        ob.step(ob.cfl(0.5), 2)
        d1 = ob.diag()
        vol = widths[0][None, None, :] * widths[1][None, :, None] * widths[2][:, None, None]
        scale = np.array([np.sum(np.abs(ob.state[f]) * vol) for f in range(8)])
        div1 = nu_divergence(ob)
        return (np.all(np.abs(d1[:8] - d0[:8]) <= 1e-13 * scale)
                and np.max(np.abs(div1 - div0)) * 0.05 / np.max(np.abs(ob.state[5:8])) < 1e-13)

    def nu_mirror():
        from test_oracle_pins import stretched, _mirror_x
        w = W.random_smooth(16, 7, 6, seed=63)
        wx = stretched(16, amp=0.45, phase=0.7)
        wy, wz = stretched(7, amp=0.3), stretched(6, amp=0.2, phase=0.5)
        a = oracle_mod.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h, lib=lib, widths=[wx, wy, wz])
        a.set_state(w.state)
        b = oracle_mod.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h, lib=lib, widths=[wx[::-1], wy, wz])
        b.set_state(_mirror_x(w.state))
        dt = a.cfl(0.5)
        a.step(dt, 2)
        b.step(dt, 2)
        return np.max(np.abs(_mirror_x(a.state) - b.state)) <= 1e-13 * np.max(np.abs(a.state))

    def nu_freefall():
        from test_oracle_pins import stretched, centres
        n, g, rho, p = 24, 0.7, 1.3, 2.0
        wx = stretched(n, amp=0.5)
        shape = (1, 1, n)
        st = W.assemble(np.full(shape, rho), (0.0, 0.0, 0.0), p, (0.0, 0.0, 0.0), 5 / 3, W.BC_OUTFLOW)
        phi = np.broadcast_to(g * centres(wx), shape).copy()
        ok = True
        for split in (False, True):
            ob = oracle_mod.OracleBox(n, 1, 1, 5 / 3, bc=W.BC_OUTFLOW, h=(1.0 / n, 1, 1), phi=phi, lib=lib,
                                      widths=[wx, None, None], gravity_split=split)
            ob.set_state(st)
            ob.fluid(0, 0.004)
            ok = ok and np.allclose(ob.state[1, 0, 0, 4:n - 4], -rho * g * 0.004, rtol=1e-12, atol=0)
        return ok

    def nu_face_velocity():
        from test_oracle_pins import face_velocity_case
        return face_velocity_case(oracle_mod, lib)

    def ct_mode():
        from test_oracle_pins import ct_upwind_mode_case
        return ct_upwind_mode_case(oracle_mod, lib)

    def ct_smoothing():
        from test_oracle_pins import ct_smoothing_case
        return ct_smoothing_case(oracle_mod, lib)

    def nu_ct_edge():
        from test_oracle_pins import ct_edge_velocity_case
        return ct_edge_velocity_case(oracle_mod, lib)

    for name, fn in [("alfven", alfven), ("oblique", oblique), ("fastwave", fastwave),
                     ("entropy", entropy), ("sod", sod),
                     ("invariants", invariants), ("freefall", freefall), ("cfl", cfl),
                     ("atmosphere", atmosphere), ("rusanov", rusanov), ("uniform", uniform),
                     ("hybrid", hybrid), ("splitfall", splitfall), ("nu_uniform", nu_uniform),
                     ("nu_conserve", nu_conserve), ("nu_mirror", nu_mirror), ("nu_freefall", nu_freefall),
                     ("nu_face_velocity", nu_face_velocity), ("ct_mode", ct_mode),
                     ("ct_smoothing", ct_smoothing), ("nu_ct_edge", nu_ct_edge)]:
        try:
            with np.errstate(all="ignore"):
                ok = bool(fn())
        except Exception:  # a blow-up counts as a caught mutant
            ok = False
        if not ok:
            checks[name] = False
    return sorted(checks)


def test_unmodified_oracle_passes_battery(oracle_mod):
    assert battery(oracle_mod, None) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(oracle_mod, name):
    old, new = MUTANTS[name]
    src = oracle_mod.source()
    assert src.count(old) == 1, name
    lib = oracle_mod.load_library(oracle_mod.build_variant(src.replace(old, new), name))
    failed = battery(oracle_mod, lib)
    assert failed, "planted mistake %s not caught by any pin" % name
