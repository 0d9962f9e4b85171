"""The batched step (alelb_batch_*): several independent cases of different
sizes, motions and flows advanced by one launch per phase.

Per case the batch must give what the case's solver gives alone: against
the FP64 oracle to 1e-12 (FP64) or 2e-4 in rho, u, T (FP32 deviations);
against the same solver stepped alone with the same element choices (equal
walk counts) and values equal up to rounding, since the same per-node code
is compiled into other kernels, where the compiler may fuse multiply-adds
in another order (FP64 1e-11, FP32 2e-4 relative, element by element,
after 70 steps).
"""
import numpy as np
import pytest

import oracle as O
import parity_util
from paper_2002_04353_gb300 import alelb, inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-4


_rel = parity_util.rel


def _cases():
    """Four unlike cases: a deforming periodic box, a plunging and a
    pitching-plunging O-mesh of different sizes and Mach numbers, and a
    plunging O-mesh at Mach 0.6 on the lattice shifted by U = (0.3, 0)."""
    box = I.uniform_flow_case(n=12, L=24.0, period_steps=40.0)
    om1 = I.naca_omesh(48, 16, chord=200.0, R=4000.0, first=1.0)
    om2 = I.naca_omesh(64, 20, chord=200.0, thickness=0.15, R=4000.0, first=1.0)
    return [
        (box.mesh, box.motion, box.flow),
        (om1, I.Motion.make(I.MOTION_PLUNGE, 20.0, 0.002), I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)),
        (om2, I.Motion.make(I.MOTION_PITCH_PLUNGE, 0.05, 0.05, 0.003, 50.0, 0.0, 20.0, 0.003),
         I.flow_params(0.15, T_inf=0.3, Re=800.0, chord=200.0, angle_deg=2.0)),
        (om1, I.Motion.make(I.MOTION_PLUNGE, 20.0, 0.002),
         I.flow_params(0.6, T_inf=0.3, Re=500.0, chord=200.0, shift=(float(np.float32(0.3)), 0.0))),
    ]


def _solvers(cases, prec):
    out = []
    for mesh, motion, flow in cases:
        m = alelb.Mesh(mesh, motion)
        out.append(alelb.Solver(m, flow, prec))
    return out


@pytest.mark.parametrize("prec", [alelb.PREC_FP64, alelb.PREC_FP32_DEV])
def test_batch_matches_oracle_per_case(prec):
    cases = _cases()
    ss = _solvers(cases, prec)
    b = alelb.Batch(ss)
    b.step(5)
    b.sync()
    for c, ((mesh, motion, flow), s) in enumerate(zip(cases, ss)):
        o = O.Oracle(mesh, motion, flow)
        o.step(5)
        st = o.state()
        assert s.time() == (5.0, 5)
        mo = s.moments()
        if prec == alelb.PREC_FP64:
            f, g = s.get_pops()
            assert _rel(f, st["f"]) < TOL64 and _rel(g, st["g"]) < TOL64, f"case {c}"
            for k, e in parity_util.field_errors(mo, st).items():
                assert e < TOL64, f"case {c}: {k} {e:.2e}"
            if c > 0:
                fo, fg = o.forces(), s.forces()
                assert np.allclose(fg, fo, rtol=1e-10, atol=1e-12 * np.abs(fo).max())
        else:
            for k, err in parity_util.field_errors(mo, st).items():
                assert err < TOL32, f"case {c}: {k} err {err:.2e}"


@pytest.mark.parametrize("prec", [alelb.PREC_FP64, alelb.PREC_FP32_DEV])
def test_batch_equals_solvers_stepped_alone(prec):
    """70 steps cross the 64-step graph chunk; every case must equal the
    same solver stepped alone up to rounding, with the same walks.  The two
    differ only in the order of fused multiply-adds, which the flow
    amplifies over 70 steps like any rounding (most on the Mach 0.6 case):
    element by element 1e-11 in FP64; in FP32 the fields within the 2e-4
    budget, the populations within 1e-3."""
    tol = 1e-11 if prec == alelb.PREC_FP64 else 2e-4
    ptol = 1e-11 if prec == alelb.PREC_FP64 else 1e-3
    cases = _cases()
    alone = _solvers(cases, prec)
    for s in alone:
        s.lb_step(70)
    batched = _solvers(cases, prec)
    b = alelb.Batch(batched)
    b.step(40)
    b.step(30)
    b.sync()
    for c, (sa, sb) in enumerate(zip(alone, batched)):
        fa, ga = sa.get_pops()
        fb, gb = sb.get_pops()
        assert _rel(fb, fa) < ptol and _rel(gb, ga) < ptol, f"case {c}"
        ma, mb = sa.moments(), sb.moments()
        for k, e in parity_util.field_errors(mb, ma).items():
            assert e < tol, f"case {c}: {k} {e:.2e}"
        assert sa.info()["walks"] == sb.info()["walks"]


def test_tuning_changes_no_value():
    cases = _cases()
    plain = _solvers(cases, alelb.PREC_FP32_DEV)
    bp = alelb.Batch(plain)
    bp.step(6)
    tuned = _solvers(cases, alelb.PREC_FP32_DEV)
    bt = alelb.Batch(tuned)
    bt.step(2)
    choice = bt.tune(reps=2)  # one real step
    assert all(choice[k] in (64, 128, 256) for k in ("k_stream_fast", "k_stream_slow", "k_moments",
                                                     "k_deriv1", "k_collide"))
    assert choice["k_stream_slow_grid"] > 0
    assert choice["k_stream_fast_directions_per_thread"] in (1, 3, 9)
    bt.step(3)
    bp.sync()
    bt.sync()
    for sa, sb in zip(plain, tuned):
        assert sa.time() == sb.time() == (6.0, 6)
        fa, ga = sa.get_pops()
        fb, gb = sb.get_pops()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
        assert sa.info()["walks"] == sb.info()["walks"]


# every launch form of the FP32 batch (alelb_batch_tune's encoding): block
# sizes, directions per thread, the propagation fused with the moments
# (+256), staged derivative stencils (+16, +32), two or four case groups
# (+512, +1024), their propagations in turn (+4096, +8192)
FORMS = [[128, 128, 128, 256, 256, 128, 64, 9],
         [128, 64, 128, 256, 256, 128, 64, 1],
         [128, 256, 64, 128, 64, 256, 300, 3 | 16 | 32],
         [128, 64, 128, 64, 256, 128, 64, 3 | 256],
         [128, 128, 128, 256, 256, 128, 64, 3 | 256],
         [128, 256, 128, 256, 128, 128, 64, 3 | 256 | 16],
         [128, 64, 128, 256, 256, 128, 64, 9 | 256],
         [128, 128, 128, 256, 256, 128, 64, 9 | 256 | 32],
         [128, 256, 128, 256, 256, 128, 64, 9 | 256],
         [128, 256, 128, 256, 256, 128, 64, 9 | 256 | 512],
         [128, 256, 128, 256, 256, 128, 64, 9 | 256 | 512 | 4096],
         [128, 64, 128, 256, 256, 128, 64, 3 | 512 | 8192 | 32],
         [128, 64, 128, 256, 256, 128, 64, 1 | 512 | 4096],
         [128, 256, 128, 256, 256, 128, 64, 9 | 256 | 1024],
         [128, 128, 128, 256, 256, 128, 300, 3 | 256 | 1024 | 8192 | 16]]


def test_every_launch_form_gives_the_same_bits():
    """Each form of alelb_batch_set_choice, 6 steps (a wall node's missing
    populations, far-field cones and listed populations included): the
    same populations, fields and walk counts as the default form, bit for
    bit."""
    cases = _cases()
    ref = _solvers(cases, alelb.PREC_FP32_DEV)
    br = alelb.Batch(ref)
    br.step(6)
    br.sync()
    want = [(s.get_pops(), s.moments(), s.info()["walks"]) for s in ref]
    for choice in FORMS:
        ss = _solvers(cases, alelb.PREC_FP32_DEV)
        b = alelb.Batch(ss)
        b.set_choice(choice)
        b.step(6)
        b.sync()
        for c, s in enumerate(ss):
            (fr, gr), mr, wr = want[c]
            f, g = s.get_pops()
            assert np.array_equal(f, fr) and np.array_equal(g, gr), f"{choice} case {c}"
            mo = s.moments()
            assert all(np.array_equal(mo[k], mr[k]) for k in mr), f"{choice} case {c}"
            assert s.info()["walks"] == wr


@pytest.mark.parametrize("flags", [O.FLAG_PHI_OFF, O.FLAG_OFFWALL_VG | O.FLAG_SLIP_WALL])
def test_fused_form_with_run_options_gives_the_same_bits(flags):
    """The fused propagation with its pending-moments list under run options
    that change the step's kernel sequence (no derivative passes) or the
    wall condition: the same bits as the plain form over 6 steps."""
    import dataclasses
    cases = [(m, mo, dataclasses.replace(fl, flags=flags)) for m, mo, fl in _cases()]
    plain = _solvers(cases, alelb.PREC_FP32_DEV)
    bp = alelb.Batch(plain)
    bp.set_choice([128, 128, 128, 256, 256, 128, 64, 9])
    bp.step(6)
    bp.sync()
    fused = _solvers(cases, alelb.PREC_FP32_DEV)
    bf = alelb.Batch(fused)
    bf.set_choice([128, 256, 128, 256, 256, 128, 64, 9 | 256])
    bf.step(6)
    bf.sync()
    for c, (sa, sb) in enumerate(zip(plain, fused)):
        fa, ga = sa.get_pops()
        fb, gb = sb.get_pops()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), f"case {c}"
        assert sa.info()["walks"] == sb.info()["walks"]


def test_set_choice_refuses_unknown_forms():
    ss = _solvers(_cases()[:1], alelb.PREC_FP32_DEV)
    b = alelb.Batch(ss)
    good = [128, 128, 128, 256, 256, 128, 64, 3]
    bad = [dict(i=0, v=96), dict(i=6, v=0), dict(i=7, v=2), dict(i=7, v=1 | 256), dict(i=7, v=3 | 128),
           dict(i=7, v=3 | 512), dict(i=7, v=3 | 64)]
    for d in bad:
        c = list(good)
        c[d["i"]] = d["v"]
        with pytest.raises(alelb.AlelbError) as e:
            b.set_choice(c)
        assert e.value.status == -1
    b.set_choice(good)
    s64 = _solvers(_cases()[:1], alelb.PREC_FP64)
    b64 = alelb.Batch(s64)
    with pytest.raises(alelb.AlelbError):
        b64.set_choice([128, 128, 128, 256, 256, 128, 64, 3 | 256])
    b64.set_choice([128, 128, 128, 256, 256, 128, 64, 9])
    # case groups: the alternation needs two groups, and 3 x 4096 is no form
    s2 = _solvers(_cases()[:2], alelb.PREC_FP32_DEV)
    b2 = alelb.Batch(s2)
    for v in (3 | 4096, 3 | 8192, 3 | 512 | 3 * 4096, 3 | 512 | 16384, 3 | 512 | 1024, 3 | 1024):
        with pytest.raises(alelb.AlelbError):
            b2.set_choice(good[:7] + [v])
    b2.set_choice(good[:7] + [3 | 512 | 8192])


@pytest.mark.parametrize("prec", [alelb.PREC_FP64, alelb.PREC_FP32_DEV])
def test_case_groups_give_the_same_bits(prec):
    """Two and four case groups on their own streams, free and with their
    propagations in turn, over 40 + 30 steps (across the 64-step graph
    chunk): the same populations, fields and walk counts as one group, bit
    for bit."""
    base = [128, 128, 128, 256, 256, 128, 64, 9]
    cases = _cases()
    ref = _solvers(cases, prec)
    br = alelb.Batch(ref)
    br.set_choice(base)
    br.step(40)
    br.step(30)
    br.sync()
    want = [(s.get_pops(), s.moments(), s.info()["walks"]) for s in ref]
    for extra in (512, 512 | 4096, 512 | 8192, 1024, 1024 | 4096):
        ss = _solvers(cases, prec)
        b = alelb.Batch(ss)
        b.set_choice(base[:7] + [base[7] | extra])
        b.step(40)
        b.step(30)
        b.sync()
        for c, s in enumerate(ss):
            (fr, gr), mr, wr = want[c]
            f, g = s.get_pops()
            assert np.array_equal(f, fr) and np.array_equal(g, gr), f"{extra} case {c}"
            mo = s.moments()
            assert all(np.array_equal(mo[k], mr[k]) for k in mr), f"{extra} case {c}"
            assert s.info()["walks"] == wr
            assert s.time() == (70.0, 70)


def test_batched_host_exchange_matches_the_per_case_calls():
    """alelb_batch_set_pops / alelb_batch_get_pops move what the per-case
    calls move, bit for bit, and set the cases' times."""
    cases = _cases()
    for prec in (alelb.PREC_FP64, alelb.PREC_FP32_DEV):
        ss = _solvers(cases, prec)
        b = alelb.Batch(ss)
        b.step(4)
        b.sync()
        n = [s.nn for s in ss]
        hf = [np.empty((9, k)) for k in n]
        hg = [np.empty((9, k)) for k in n]
        b.get_pops(hf, hg)
        for s, f, g in zip(ss, hf, hg):
            fa, ga = s.get_pops()
            assert np.array_equal(f, fa) and np.array_equal(g, ga)
        # set every case back from perturbed arrays at new times, then read again
        rng = np.random.default_rng(3)
        pf = [f * (1 + 1e-6 * rng.standard_normal(f.shape)) for f in hf]
        pg = [g * (1 + 1e-6 * rng.standard_normal(g.shape)) for g in hg]
        t = np.arange(len(ss), dtype=np.float64) + 10.0
        b.set_pops(pf, pg, t=t)
        alone = _solvers(cases, prec)
        for s, f, g, tc in zip(alone, pf, pg, t):
            s.set_pops(f, g, t=tc)
        for sa, sb, tc in zip(alone, ss, t):
            assert sb.time()[0] == tc
            fa, ga = sa.get_pops()
            fb, gb = sb.get_pops()
            assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
        with pytest.raises(ValueError):
            b.get_pops(hf[:-1], hg[:-1])
        with pytest.raises(ValueError):
            b.set_pops([f.astype(np.float32) for f in pf], pg)


def test_batch_and_single_steps_interleave():
    cases = _cases()[:2]
    alone = _solvers(cases, alelb.PREC_FP64)
    for s in alone:
        s.lb_step(6)
    mixed = _solvers(cases, alelb.PREC_FP64)
    b = alelb.Batch(mixed)
    b.step(2)
    mixed[0].lb_step(2)
    mixed[1].lb_step(2)
    b.step(2)
    for sa, sb in zip(alone, mixed):
        fa, ga = sa.get_pops()
        fb, gb = sb.get_pops()
        assert _rel(fb, fa) < 1e-13 and _rel(gb, ga) < 1e-13


def test_batch_profile_counts_launches():
    ss = _solvers(_cases(), alelb.PREC_FP32_DEV)
    b = alelb.Batch(ss)
    b.profile(True)
    b.step(3)
    kt = b.kernel_times()
    for k in ("k_stream_fast", "k_stream_slow", "k_moments", "k_deriv1", "k_collide"):
        assert kt[k][1] == 3 and kt[k][0] > 0
    assert kt["k_stream"][1] == 0
    b.profile(False)


def test_batch_arguments_are_checked():
    cases = _cases()
    ss = _solvers(cases[:2], alelb.PREC_FP64)
    s32 = _solvers(cases[2:], alelb.PREC_FP32_DEV)
    for bad in ([], [ss[0], ss[0]], [ss[0], s32[0]]):
        with pytest.raises(alelb.AlelbError) as ex:
            alelb.Batch(bad)
        assert ex.value.status == -1
    with pytest.raises(alelb.AlelbError):
        alelb.Batch(ss).tune(reps=0)


def test_case_error_is_reported_with_its_index():
    """A non-finite state in one case (made on the host: NaN populations at
    one node) is reported by batch_sync, naming that case."""
    cases = _cases()
    ss = _solvers(cases, alelb.PREC_FP64)
    f, g = ss[1].get_pops()
    f[:, 7] = np.nan
    ss[1].set_pops(f, g)
    b = alelb.Batch(ss)
    b.step(1)
    with pytest.raises(alelb.AlelbError) as ex:
        b.sync()
    assert ex.value.status == -7 and "case 1" in str(ex.value)


# ---------------------------------------------------------------------------
# the persistent form: one cooperative launch per chunk, grid-wide barriers
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [alelb.PREC_FP64, alelb.PREC_FP32_DEV])
def test_persistent_batch_matches_oracle_and_the_graph_form(prec):
    """The persistent kernel runs the same per-node code as the phase
    kernels: per case it matches the oracle after 5 steps (1e-12 / 2e-4)
    and the graph form after 70 steps (across a 64-step chunk) up to
    rounding, with the same walks."""
    cases = _cases()
    ss = _solvers(cases, prec)
    b = alelb.Batch(ss)
    b.set_mode(alelb.BATCH_PERSISTENT)
    b.step(5)
    b.sync()
    for c, ((mesh, motion, flow), s) in enumerate(zip(cases, ss)):
        o = O.Oracle(mesh, motion, flow)
        o.step(5)
        st = o.state()
        tol = TOL64 if prec == alelb.PREC_FP64 else TOL32
        for k, e in parity_util.field_errors(s.moments(), st).items():
            assert e < tol, f"persistent case {c}: {k} {e:.2e}"
    b.step(65)
    b.sync()
    ref = _solvers(cases, prec)
    bg = alelb.Batch(ref)
    bg.step(70)
    bg.sync()
    tol = 1e-11 if prec == alelb.PREC_FP64 else 2e-4
    ptol = 1e-11 if prec == alelb.PREC_FP64 else 1e-3
    for c, (sp, sg) in enumerate(zip(ss, ref)):
        fp, gp = sp.get_pops()
        fg, gg = sg.get_pops()
        assert _rel(fp, fg) < ptol and _rel(gp, gg) < ptol, f"case {c}"
        for k, e in parity_util.field_errors(sp.moments(), sg.moments()).items():
            assert e < tol, f"case {c}: {k} {e:.2e}"
        assert sp.info()["walks"] == sg.info()["walks"]
        assert sp.time() == sg.time() == (70.0, 70)


def test_persistent_barrier_wait_runs_out_and_reports():
    """A barrier told to wait for one block more than the grid holds (a flag
    that nothing sets): every wait gives up after its limit, the kernel
    returns, every case reports ALELB_ERR_TIMEOUT, and the device stays
    usable for other work."""
    cases = _cases()
    ss = _solvers(cases, alelb.PREC_FP32_DEV)
    b = alelb.Batch(ss)
    b.set_mode(alelb.BATCH_PERSISTENT)
    b.set_wait(0.2, missing_arrivals=1)
    b.step(1)
    with pytest.raises(alelb.AlelbError) as e:
        b.sync()
    assert e.value.status == -8
    for s in ss:
        with pytest.raises(alelb.AlelbError) as e:
            s.sync()
        assert e.value.status == -8
    mesh, motion, flow = cases[1]
    other = alelb.Solver(alelb.Mesh(mesh, motion), flow, alelb.PREC_FP32_DEV)
    other.lb_step(3)
    other.sync()
    with pytest.raises(alelb.AlelbError) as e:
        b.set_wait(0.0)
    assert e.value.status == -1
