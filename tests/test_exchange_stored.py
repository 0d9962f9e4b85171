"""The host exchange in the FP32-deviation form's stored form
(alelb_get_pops_stored / alelb_set_pops_stored, their batched forms and
the pipelined host step), and the zero-copy exchange on device arrays
(alelb_get_pops_dev / alelb_set_pops_dev / alelb_moments_dev).

What it must give: the deviations exactly as the device stores them (a get,
then a set, restores the state bit for bit); the same fields as the FP64
exchange of the same state (both compute them from the full populations
d + f^eq in FP64); full FP64 populations that differ from the deviations by
one constant per direction (the reference equilibria); and refusals for the
FP64 form.
"""
import numpy as np
import pytest

from paper_2002_04353_gb300 import alelb
from test_batch import _cases, _solvers

pytestmark = pytest.mark.gpu


def test_round_trip_restores_the_stored_state_bit_for_bit():
    s = _solvers(_cases()[1:2], alelb.PREC_FP32_DEV)[0]
    s.lb_step(5)
    df, dg = s.get_pops_stored()
    s.lb_step(3)
    s.set_pops_stored(df, dg, t=5.0)
    assert s.time()[0] == 5.0
    ef, eg = s.get_pops_stored()
    assert np.array_equal(ef, df) and np.array_equal(eg, dg)
    assert all(np.isfinite(v).all() for v in s.moments().values())


def test_fields_equal_those_of_the_fp64_exchange():
    cases = _cases()[2:3]
    a, b = _solvers(cases, alelb.PREC_FP32_DEV), _solvers(cases, alelb.PREC_FP32_DEV)
    for s in a + b:
        s.lb_step(4)
    f, g = a[0].get_pops()
    df, dg = b[0].get_pops_stored()
    # full values minus stored deviations: the reference equilibria, one
    # constant per direction (to the FP64 rounding of the sum)
    for full, dev in ((f, df), (g, dg)):
        ref = full - dev.astype(np.float64)
        spread = ref.max(axis=1) - ref.min(axis=1)
        assert np.all(spread <= 4e-16 * np.abs(full).max()), spread
    a[0].set_pops(f, g, t=9.0)
    b[0].set_pops_stored(df, dg, t=9.0)
    ma, mb = a[0].moments(), b[0].moments()
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k


def test_batched_form_matches_the_per_case_calls():
    cases = _cases()
    ss = _solvers(cases, alelb.PREC_FP32_DEV)
    b = alelb.Batch(ss)
    b.step(4)
    b.sync()
    hf = [np.empty((9, s.nn), dtype=np.float32) for s in ss]
    hg = [np.empty((9, s.nn), dtype=np.float32) for s in ss]
    b.get_pops_stored(hf, hg)
    for s, f, g in zip(ss, hf, hg):
        ef, eg = s.get_pops_stored()
        assert np.array_equal(f, ef) and np.array_equal(g, eg)
    # perturbed deviations back in at new times, against the per-case call
    rng = np.random.default_rng(5)
    pf = [(f + 1e-6 * rng.standard_normal(f.shape)).astype(np.float32) for f in hf]
    pg = [(g + 1e-6 * rng.standard_normal(g.shape)).astype(np.float32) for g in hg]
    t = np.arange(len(ss), dtype=np.float64) + 20.0
    b.set_pops_stored(pf, pg, t=t)
    alone = _solvers(cases, alelb.PREC_FP32_DEV)
    for s, f, g, tc in zip(alone, pf, pg, t):
        s.set_pops_stored(f, g, t=tc)
    for sa, sb, f, g in zip(alone, ss, pf, pg):
        assert sa.time()[0] == sb.time()[0]
        fa, ga = sb.get_pops_stored()
        assert np.array_equal(fa, f) and np.array_equal(ga, g)
        ma, mb = sa.moments(), sb.moments()
        assert all(np.array_equal(ma[k], mb[k]) for k in ma)


def test_other_precisions_and_bad_arrays_are_refused():
    s64 = _solvers(_cases()[:1], alelb.PREC_FP64)[0]
    with pytest.raises(alelb.AlelbError) as e:
        s64.get_pops_stored()
    assert e.value.status == -1
    n = s64.nn
    with pytest.raises(alelb.AlelbError):
        s64.set_pops_stored(np.zeros((9, n), np.float32), np.zeros((9, n), np.float32))
    b64 = alelb.Batch([s64])
    with pytest.raises(alelb.AlelbError):
        b64.get_pops_stored([np.empty((9, n), np.float32)], [np.empty((9, n), np.float32)])
    planes = [np.zeros((9, n), np.float32)]
    with pytest.raises(alelb.AlelbError):
        b64.step_host(planes, planes, planes, planes)
    assert s64.time() == (0.0, 0)  # refused before anything ran
    s32 = _solvers(_cases()[:1], alelb.PREC_FP32_DEV)[0]
    with pytest.raises(ValueError):
        s32.get_pops_stored(np.empty((9, s32.nn)), None)  # float64 out array
    with pytest.raises(ValueError):
        s32.set_pops_stored(np.zeros((9, s32.nn - 1), np.float32), np.zeros((9, s32.nn), np.float32))
    b32 = alelb.Batch([s32])
    good = [np.zeros((9, s32.nn), np.float32)]
    with pytest.raises(ValueError):
        b32.step_host(good, good, [np.zeros((9, s32.nn))], good)  # float64 out array


@pytest.mark.parametrize("n_cases", [4, 2, 1])
def test_pipelined_host_step_equals_set_step_get(n_cases):
    """alelb_batch_step_host (uploads, the step and the read-back pipelined
    by case group) against the three calls it stands for, three steps in a
    row: the same stored deviations, times, fields and walk counts, bit for
    bit; in place (outputs = inputs) and into other arrays.  Four cases run
    as four groups, two as two, one as one."""
    cases = _cases()[:n_cases]
    ref, pip = _solvers(cases, alelb.PREC_FP32_DEV), _solvers(cases, alelb.PREC_FP32_DEV)
    br, bp = alelb.Batch(ref), alelb.Batch(pip)
    br.step(3)
    bp.step(3)
    hf = [np.empty((9, s.nn), dtype=np.float32) for s in ref]
    hg = [np.empty((9, s.nn), dtype=np.float32) for s in ref]
    br.get_pops_stored(hf, hg)
    pf, pg = [a.copy() for a in hf], [a.copy() for a in hg]
    of, og = [np.empty_like(a) for a in hf], [np.empty_like(a) for a in hg]
    for k in range(3):
        t = np.arange(len(cases), dtype=np.float64) + 3.0 + k
        br.set_pops_stored(hf, hg, t=t)
        br.step(1)
        br.get_pops_stored(hf, hg)
        if k == 1:  # into other arrays, then back
            bp.step_host(pf, pg, of, og, t=t)
            for a, b in zip(pf + pg, of + og):
                a[...] = b
        else:
            bp.step_host(pf, pg, pf, pg, t=t)
        for c in range(len(cases)):
            assert np.array_equal(pf[c], hf[c]) and np.array_equal(pg[c], hg[c]), f"step {k} case {c}"
            assert ref[c].time() == pip[c].time()
    for sa, sb in zip(ref, pip):
        ma, mb = sa.moments(), sb.moments()
        assert all(np.array_equal(ma[k], mb[k]) for k in ma)
        assert sa.info()["walks"] == sb.info()["walks"]


@pytest.mark.parametrize("prec", [alelb.PREC_FP64, alelb.PREC_FP32_DEV])
def test_zero_copy_device_exchange_equals_the_host_forms(prec):
    """alelb_get_pops_dev / alelb_set_pops_dev / alelb_moments_dev on CUDA
    tensors: the same values as the host forms, bit for bit."""
    import torch
    cases = _cases()[1:2]
    s = _solvers(cases, prec)[0]
    s.lb_step(4)
    f, g = s.get_pops()
    df = torch.empty((9, s.nn), dtype=torch.float64, device="cuda")
    dg = torch.empty_like(df)
    s.get_pops_dev(df, dg)
    assert np.array_equal(df.cpu().numpy(), f) and np.array_equal(dg.cpu().numpy(), g)
    m = s.moments()
    dm = {k: torch.empty(s.nn, dtype=torch.float64, device="cuda") for k in m}
    s.moments_dev(dm["rho"], dm["ux"], dm["uy"], dm["T"])
    assert all(np.array_equal(dm[k].cpu().numpy(), m[k]) for k in m)
    s.moments_dev(None, dm["ux"], None, None)  # any field may be left out
    # a perturbed state in, through the device and through the host
    rng = np.random.default_rng(7)
    pf = f * (1 + 1e-7 * rng.standard_normal(f.shape))
    pg = g * (1 + 1e-7 * rng.standard_normal(g.shape))
    a, b = _solvers(cases, prec)[0], _solvers(cases, prec)[0]
    a.set_pops(pf, pg, t=7.0)
    b.set_pops_dev(torch.from_numpy(pf).cuda(), torch.from_numpy(pg).cuda(), t=7.0)
    assert a.time()[0] == b.time()[0] == 7.0
    fa, ga = a.get_pops()
    fb, gb = b.get_pops()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    ma, mb = a.moments(), b.moments()
    assert all(np.array_equal(ma[k], mb[k]) for k in ma)


def test_zero_copy_refuses_host_addresses():
    """Host memory, pageable or pinned, is refused before any launch."""
    import torch
    s = _solvers(_cases()[:1], alelb.PREC_FP32_DEV)[0]
    L = alelb.load()
    host = np.zeros((9, s.nn))
    pinned = torch.zeros((9, s.nn), dtype=torch.float64).pin_memory()
    for addr in (host.ctypes.data, pinned.data_ptr()):
        assert L.alelb_get_pops_dev(s.h, addr, addr) == -1
        assert L.alelb_set_pops_dev(s.h, addr, addr, 0.0) == -1
        assert L.alelb_moments_dev(s.h, addr, None, None, None) == -1
    assert L.alelb_get_pops_dev(s.h, None, None) == -1
    with pytest.raises(ValueError):
        s.get_pops_dev(torch.empty((9, s.nn), dtype=torch.float32, device="cuda"),
                       torch.empty((9, s.nn), dtype=torch.float32, device="cuda"))
    s.lb_step(1)  # the solver is still usable
    s.sync()
