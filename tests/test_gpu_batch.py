"""GPU tests of the batched path (fish_batch_*): many FP32 boxes of uneven
sizes, boundary conditions and ratios of specific heats advanced by one graph
of persistent sweeps.

Every box must follow the single-box FP32 path (a fish_ctx stepped with
fish_step_cfl: same kernels, same per-box CFL time steps) to 1e-6 relative
per cell, the FP64 oracle to 1e-5 after two steps, and the scheduling options
chosen by the autotuner must not change a single bit."""
import numpy as np
import pytest

import oracle
from paper_0910_2854_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available()
    from paper_0910_2854_gb300 import build
    build.build()
    import paper_0910_2854_gb300 as mod
    mod.load()
    return mod


def rel_err(got, ref):
    """Largest cell error relative to the field's scale; the components of
    m and of b are scaled by the largest component of their vector (a
    component that is zero in exact arithmetic holds only round-off)."""
    mx = np.max(np.abs(ref), axis=(1, 2, 3))
    scale = mx.copy()
    scale[1:4] = np.max(mx[1:4])
    scale[5:8] = np.max(mx[5:8])
    scale = np.maximum(scale, 1e-300)[:, None, None, None]
    return float(np.max(np.abs(got - ref) / scale))


def small_boxes():
    """Four boxes: ragged sizes (several column groups, odd z, pencils
    shorter than the march unroll), both boundary conditions, three gammas.
    The blast sits off the box centre: a mirror-symmetric flow has
    stagnation edges whose velocity is zero only up to round-off, where the
    sign-selected upwind edge flux of eq0363 may pick the other cell in FP32
    than in FP64."""
    return [
        W.random_smooth(34, 20, 13, seed=41, h=(0.03, 0.05, 0.07)),
        W.sod(24, axis=1, ntrans=6),
        W.brio_wu(20, axis=0, ntrans=8),
        W.blast(16, 12, 7, radius_frac=0.25, centre=(0.41, 0.53, 0.37)),
    ]


def make_batch(F, ws, **kw):
    b = F.Batch([w.dims for w in ws], [w.gamma for w in ws], [w.bc for w in ws], hs=[w.h for w in ws], **kw)
    for i, w in enumerate(ws):
        b.set_state(i, w.state)
    return b


def test_batch_matches_single_box_path(F):
    ws = small_boxes()
    b = make_batch(F, ws)
    b.step(0.5, 3)
    dts = b.last_dt()
    for i, w in enumerate(ws):
        box = F.Box(*w.dims, w.gamma, bc=w.bc, precision="fp32", h=w.h)
        box.set_state(w.state)
        box.step_cfl(0.5, 3)
        assert abs(box.last_dt() - dts[i]) <= 1e-6 * dts[i]
        assert rel_err(b.get_state(i), box.get_state()) <= 1e-6, i
        box.close()
    b.close()


def test_batch_against_oracle(F):
    """Each box against the FP64 oracle stepped with the box's own time
    steps: the first dt (from the initial state) to 1e-5, later ones (from
    the FP32 state) to 1e-4, the states to 1e-5 after two steps."""
    ws = small_boxes()
    b = make_batch(F, ws)
    obs = []
    for w in ws:
        ob = oracle.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h)
        ob.set_state(w.state)
        obs.append(ob)
    for step in range(2):
        b.step(0.5, 1)
        dts = b.last_dt()
        for i, ob in enumerate(obs):
            ref = ob.cfl(0.5)
            assert abs(dts[i] - ref) <= (1e-5 if step == 0 else 1e-4) * ref, (i, step)
            ob.step(dts[i])
    for i, ob in enumerate(obs):
        assert rel_err(b.get_state(i), ob.state) <= 1e-5, i
    b.close()


def test_batch_tuning_options_do_not_change_results(F):
    ws = small_boxes()
    ref = make_batch(F, ws)
    ref.step(0.5, 2)
    want = [ref.get_state(i) for i in range(len(ws))]
    ref.close()
    for order, groups, grid, rows in ((1, 2, 1, 4), (2, 4, 2, 8), (0, 8, 4, 8), (0, 1, 1, 8)):
        b = make_batch(F, ws)
        b.set_option(F.FISH_BATCH_OPT_ORDER, order)
        b.set_option(F.FISH_BATCH_OPT_GROUPS, groups)
        b.set_option(F.FISH_BATCH_OPT_GRID, grid)
        b.set_option(F.FISH_BATCH_OPT_CTROWS, rows)
        b.step(0.5, 2)
        for i in range(len(ws)):
            assert np.array_equal(b.get_state(i), want[i]), (order, groups, grid, i)
        b.close()


def test_batch_rejects_odd_paired_extents(F):
    with pytest.raises(F.FishError) as ei:
        F.Batch([(9, 8, 8)], [1.4], [0])
    assert ei.value.code == F.FISH_ERR_ARG


def test_autotuner_picks_a_measured_choice(F, tmp_path, monkeypatch):
    from paper_0910_2854_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    ws = small_boxes()
    cands = [dict(order=0, groups=1, grid=1), dict(order=1, groups=2, grid=1)]
    c = autotune.tune([w.dims for w in ws], [w.gamma for w in ws], [w.bc for w in ws], [w.state for w in ws],
                      hs=[w.h for w in ws], candidates=cands)
    assert c["ms"] > 0 and len(c["tried"]) == 2
    assert c["ms"] == min(t["ms"] for t in c["tried"])
    again = autotune.tune([w.dims for w in ws], [w.gamma for w in ws], [w.bc for w in ws], [w.state for w in ws],
                          hs=[w.h for w in ws], candidates=cands)
    assert again == c  # served from the cache


def test_bench_size_batch_parity(F):
    """The 64 seeded boxes of the throughput batch (sizes 32..160 per axis,
    Sod / Brio-Wu / blast), two double steps: every box against the
    single-box FP32 path to 1e-6 (time steps and states), and the four
    smallest tube boxes against the FP64 oracle to 1e-5.  (The batch's
    blasts are centred: their mirror-symmetric stagnation edges carry edge
    velocities that are zero only up to round-off, where FP32 may take the
    other upwind cell than FP64 -- reading C-20 -- so the oracle comparison
    takes tube boxes.)"""
    specs = W.batch_specs()
    ws = [W.batch_box(*s) for s in specs]
    assert len(ws) == 64
    b = make_batch(F, ws)
    b.step(0.5, 2)
    dts = b.last_dt()
    for i, w in enumerate(ws):
        box = F.Box(*w.dims, w.gamma, bc=w.bc, precision="fp32", h=w.h)
        box.set_state(w.state)
        box.step_cfl(0.5, 2)
        assert abs(box.last_dt() - dts[i]) <= 1e-6 * dts[i], i
        assert rel_err(b.get_state(i), box.get_state()) <= 1e-6, i
        box.close()
    b.close()

    tubes = sorted((i for i, s in enumerate(specs) if s[0] != "blast"), key=lambda i: np.prod(ws[i].dims))[:4]
    sel = [ws[i] for i in tubes]
    b = make_batch(F, sel)
    obs = []
    for w in sel:
        ob = oracle.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h)
        ob.set_state(w.state)
        obs.append(ob)
    for step in range(2):
        b.step(0.5, 1)
        d = b.last_dt()
        for i, ob in enumerate(obs):
            ref = ob.cfl(0.5)
            assert abs(d[i] - ref) <= (1e-5 if step == 0 else 1e-4) * ref, (tubes[i], step)
            ob.step(d[i])
    for i, ob in enumerate(obs):
        assert rel_err(b.get_state(i), ob.state) <= 1e-5, tubes[i]
    b.close()
