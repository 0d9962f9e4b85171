"""The kernels' element walk, compiled for the host (hostcheck.cu runs
the same per-node routine as the location kernel), against the oracle's
exhaustive point search: element choices must agree bit for bit.  Runs on
the CPU; the GPU parity tests repeat the comparison with the device build."""
import numpy as np
import pytest

import oracle as O
import hostcheck as H
from paper_2002_04353_gb300 import inputs as I

CASES = {
    "box_config_map": (lambda: I.uniform_flow_case().mesh,
                       lambda: I.uniform_flow_case().motion, [1, 25, 50, 99, 175]),
    "box_paper_map": (lambda: I.periodic_box(20, 40.0, 0.2, seed=2),
                      lambda: I.Motion.make(I.MOTION_SINE, 2.5, 40.0, 60.0, 1.0), [1, 15, 30]),
    "lattice": (lambda: I.lattice_box(12), lambda: I.Motion.make(I.MOTION_NONE), [1]),
    "plunge": (lambda: I.naca_omesh(96, 30, chord=1000.0, R=20000.0, first=1.0),
               lambda: I.Motion.make(I.MOTION_PLUNGE, 100.0, 2.6e-4), [1, 3000, 6000]),
    "pitch_plunge": (lambda: I.naca_omesh(96, 30, chord=1000.0, R=20000.0, first=1.0),
                     lambda: I.Motion.make(I.MOTION_PITCH_PLUNGE, 0.0, -0.05, 1e-4, 250.0, 0.0, 100.0, 1e-4),
                     [1, 5000, 12000]),
    "blended": (lambda: I.naca_omesh(96, 30, chord=1000.0, R=20000.0, first=1.0),
                lambda: I.Motion.make(I.MOTION_BLENDED_PITCH, -0.002, -0.0436, 7.8e-5, 250.0, 0.0, 2000.0, 10000.0),
                [1, 10000, 20000]),
    # flat walls along lattice directions: departure segments run along
    # boundary edges (inside the closed mesh)
    "channel_static": (lambda: I.wall_channel(first=1.0, growth=1.0), lambda: I.Motion.make(I.MOTION_NONE), [1]),
    "channel_plunge": (lambda: I.wall_channel(), lambda: I.Motion.make(I.MOTION_PLUNGE, 2.0, 0.02), [1, 40]),
}
# the same on meshes of the paper's 9-node quadrilaterals
CASES.update({
    "q2_box_config_map": (lambda: I.uniform_flow_case(elem="q2").mesh,
                          lambda: I.uniform_flow_case().motion, [1, 25, 50, 99, 175]),
    "q2_box_paper_map": (lambda: I.periodic_box(20, 40.0, 0.2, seed=2, elem="q2"),
                         lambda: I.Motion.make(I.MOTION_SINE, 2.5, 40.0, 60.0, 1.0), [1, 15, 30]),
    "q2_lattice": (lambda: I.lattice_box(12, elem="q2"), lambda: I.Motion.make(I.MOTION_NONE), [1]),
    "q2_plunge": (lambda: I.naca_omesh(96, 30, chord=1000.0, R=20000.0, first=1.0, elem="q2"),
                  lambda: I.Motion.make(I.MOTION_PLUNGE, 100.0, 2.6e-4), [1, 3000, 6000]),
    "q2_pitch_plunge": (lambda: I.naca_omesh(96, 30, chord=1000.0, R=20000.0, first=1.0, elem="q2"),
                        lambda: I.Motion.make(I.MOTION_PITCH_PLUNGE, 0.0, -0.05, 1e-4, 250.0, 0.0, 100.0, 1e-4),
                        [1, 5000, 12000]),
    "q2_blended": (lambda: I.naca_omesh(96, 30, chord=1000.0, R=20000.0, first=1.0, elem="q2"),
                   lambda: I.Motion.make(I.MOTION_BLENDED_PITCH, -0.002, -0.0436, 7.8e-5, 250.0, 0.0, 2000.0, 10000.0),
                   [1, 10000, 20000]),
    "q2_channel_static": (lambda: I.wall_channel(first=1.0, growth=1.0, elem="q2"),
                          lambda: I.Motion.make(I.MOTION_NONE), [1]),
    "q2_channel_plunge": (lambda: I.wall_channel(elem="q2"), lambda: I.Motion.make(I.MOTION_PLUNGE, 2.0, 0.02),
                          [1, 40]),
})


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_walk_matches_oracle(name):
    mk_mesh, mk_mot, times = CASES[name]
    mesh, mot = mk_mesh(), mk_mot()
    o = O.Oracle(mesh, mot, I.Flow())
    for t in times:
        st, e, k = H.locate(mesh, mot, float(t))
        assert st == 0
        eo, ko = o.locate(float(t))
        assert np.array_equal(e, eo), f"{name} t={t}: {np.sum(e != eo)} differ"
        assert np.array_equal(k, ko)


def test_host_walk_literal_form():
    mesh = I.naca_omesh(64, 20, chord=200.0, R=4000.0, first=1.0)
    mot = I.Motion.make(I.MOTION_PITCH, 0.05, 0.05, 0.003, 50.0, 0.0)
    o = O.Oracle(mesh, mot, I.Flow(flags=O.FLAG_LITERAL_VG))
    st, e, k = H.locate(mesh, mot, 11.0, literal=True)
    eo, ko = o.locate(11.0)
    assert st == 0 and np.array_equal(e, eo) and np.array_equal(k, ko)


def test_fp32_filter_never_accepts_a_point_that_is_not_strictly_inside():
    """The fast path's certified FP32 filter may decline, never err: against
    exact rationals, on points placed on, just inside and just outside the
    edges of elements of a graded O-mesh and a jittered box."""
    from fractions import Fraction as F
    rng = np.random.default_rng(3)
    for mesh in (I.naca_omesh(96, 30, chord=1000.0, R=20000.0, first=1.0), I.periodic_box(12, 24.0, 0.2, seed=4)):
        es, pxs, pys, exact, easy = [], [], [], [], []
        for e in rng.choice(mesh.n_elems, min(400, mesh.n_elems), replace=False):
            v = mesh.X[mesh.conn[e, :3]].copy()
            if mesh.period[0] > 0:  # unwrap the element around its first vertex
                L = mesh.period[0]
                v[1:] = v[0] + (v[1:] - v[0] + L / 2) % L - L / 2
                if np.any(v < 0) or np.any(v >= L):
                    continue
            for k in range(3):
                a, b, c = v[k], v[(k + 1) % 3], v[(k + 2) % 3]
                for s in (0.0, 1e-6, -1e-6, 1e-9, -1e-9, 1e-12, -1e-12, 0.3):
                    t = rng.uniform(0.05, 0.95)
                    p = a + t * (b - a) + s * (c - (a + b) / 2)
                    es.append(e)
                    pxs.append(p[0])
                    pys.append(p[1])
                    o = []
                    for kk in range(3):
                        A, B = v[kk], v[(kk + 1) % 3]
                        o.append((F(A[0]) - F(p[0])) * (F(B[1]) - F(p[1])) - (F(A[1]) - F(p[1])) * (F(B[0]) - F(p[0])))
                    exact.append(all(x > 0 for x in o))
                    easy.append(s == 0.3)
        got = H.inside_f32(mesh, np.array(es), np.array(pxs), np.array(pys))
        exact = np.array(exact)
        assert not np.any(got & ~exact), "filter accepted a point that is not strictly inside"
        easy = np.array(easy) & exact
        assert got[easy].sum() >= 0.99 * easy.sum()  # and it does decide the clear-cut ones


@pytest.mark.parametrize("name", sorted(CASES))
def test_fast_path_decisions_match_oracle(name):
    """The FP32-deviation propagation's decisions (previous-step element
    verified in FP32 with certified bounds, exact walk otherwise), run on the
    host, equal the oracle's element choices, and settle most populations."""
    mk_mesh, mk_mot, times = CASES[name]
    mesh, mot = mk_mesh(), mk_mot()
    o = O.Oracle(mesh, mot, I.Flow())
    for t in times[-2:]:
        st, e, k, fast = H.locate_fast(mesh, mot, float(t) - 1.0, float(t))
        assert st == 0
        eo, ko = o.locate(float(t))
        assert np.array_equal(e, eo), f"{name} t={t}: {np.sum(e != eo)} differ"
        assert np.array_equal(k, ko)
        # on the lattice every departure point is a node; the small channel
        # is mostly wall layers, where the exact path decides
        if name not in ("lattice", "q2_lattice") and "channel" not in name:
            assert fast.mean() > 0.8, f"{name}: only {fast.mean():.3f} settled by the fast path"


def _exact_sign(r):
    from fractions import Fraction as F
    ax, ay, bx, by, cx, cy = (F(float(v)) for v in r)
    d = (ax - cx) * (by - cy) - (ay - cy) * (bx - cx)
    return (d > 0) - (d < 0)


def test_library_orientation_is_exact():
    """The walk's orientation predicate (FP64 filter, integer stage, expansion
    stage) against rational arithmetic: exact ties (collinear points on
    quantised and unquantised lines), near ties one ulp off, far-apart
    exponents, and random points."""
    rng = np.random.default_rng(7)
    rows = []
    for _ in range(400):
        # a quantised segment and a point on its line or one ulp off it
        a = np.round(rng.uniform(-5e3, 5e3, 2) * 2**20) / 2**20
        d = np.round(rng.uniform(-8, 8, 2) * 2**20) / 2**20
        t = rng.choice([0.5, 0.25, 2.0, -1.0, 3.0])
        c = a + t * d
        b = a + d
        rows.append([*a, *b, *c])
        for s in (1, -1):
            rows.append([*a, *b, np.nextafter(c[0], c[0] + s), c[1]])
            rows.append([*a, *b, c[0], np.nextafter(c[1], c[1] - s)])
        # departure-like point: node plus a small FP64 offset along the edge
        off = rng.uniform(1e-3, 1.0)
        p = np.array([a[0] + off * d[0], a[1] + off * d[1]])
        rows.append([*a, *b, *p])
    for _ in range(200):
        # operands of very different magnitude (the expansion stage)
        big = rng.uniform(-1e6, 1e6, 2)
        small = rng.uniform(-1e-9, 1e-9, 4)
        rows.append([big[0], big[1], small[0], small[1], small[2], small[3]])
        rows.append([*rng.uniform(-1, 1, 6)])
    rows = np.array(rows)
    got, stage = H.orient(rows)
    want = np.array([_exact_sign(r) for r in rows])
    assert np.array_equal(got, want), f"{np.sum(got != want)} orientation signs differ"
    used = stage != 2
    assert used.sum() > 0.5 * len(rows)  # the integer stage decides the common cases
    assert np.array_equal(stage[used], want[used])
    assert (want == 0).sum() > 300  # exact ties are present
