"""The limiter pass (TVB-minmod in characteristic fields, then the positivity
scaling; Sec. 2.3 / Remark 2.2) on the GPU against the FP64 oracle, on a
state where both act (about a third of the cells troubled, the positivity
scaling changing about 2 % of them): periodic and outflow meshes, FP64 and
FP32, a ragged last tile of 128 columns (nx = 132 and 130), run through
crkdg_apply_limit (the pass as the default limit mode runs it before a step)
and through get_state (the pending limit applied on read).  The tall mesh
(130 x 2000, the box stretched to keep the cells' size) has 54 times the
cells of the short ones: where the positivity scaling acts on 4835 of its
cells, one FP32 pressure factor is a near-double root, the case the
positivity root band covers."""
import numpy as np
import pytest

import crkdg_inputs as inp
from oracle.limiter import positivity_limit, tvb_limit
from tests.pairing import from_planes, make_pair_2d, positivity_root_tie, rel_err, to_planes, tvb_margin

pytestmark = pytest.mark.gpu

BCS = {"periodic": {s: ("periodic",) for s in "WESN"},
       "outflow": {s: ("outflow",) for s in "WESN"}}
M_TVB, EPS = 5000.0, 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_06471_gb300 import build
    build.build()


def _state(nx, ny, prec):
    u = inp.random_modal_state(ny, nx, 2, "P", "euler", seed=31, amp=0.5)
    if prec == "f32":
        u = from_planes(to_planes(u).astype(np.float32).astype(np.float64))
    return u


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["periodic", "outflow"])
@pytest.mark.parametrize("nx,ny", [(132, 37), (130, 37), (130, 2000)])
def test_limit_pass_with_positivity_matches_the_oracle(prec, bc, nx, ny):
    box = (0, 1, 0, ny / 37.0)   # cells of 1/nx x 1/37: the same TVB thresholds
    u = _state(nx, ny, prec)
    got = []
    for apply_now in (True, False):
        gs, dg = make_pair_2d(nx, ny, box, 2, "P", "euler", "ssprk3", BCS[bc], prec)
        gs.set_state(to_planes(u), 0.0)
        gs.positivity(EPS)
        gs.limit(M_TVB)
        if apply_now:
            gs.apply_limit()
        got.append(from_planes(gs.get_state()))
        assert gs.sync() == (0, 0)
        gs.close()
    lim, flags = tvb_limit(dg, u, M_TVB, 0.0)
    want = positivity_limit(dg, lim, EPS)
    assert flags.any() and not flags.all()
    assert not np.allclose(want, lim)   # the positivity scaling acts
    ref = got[0]
    if prec == "f64":
        assert rel_err(ref, want) < 1e-13
    else:
        # FP32: a cell may differ from the FP64 oracle only where a
        # TVB-minmod decision sits within FP32 rounding of a tie, or where
        # the positivity scaling's pressure factor is a near-double root
        # (moved by FP32 rounding of its discriminant: the band of
        # positivity_root_tie)
        scale = np.max(np.abs(want), axis=(0, 1, 3))
        bad = np.argwhere(np.any(np.abs(ref - want) > 2e-6 * scale[None, None, :, None], axis=(2, 3)))
        for (cy, cx) in bad:
            c = (int(cy), int(cx))
            if tvb_margin(dg, u, 0.0, M_TVB, [c]) < 1e-4:
                continue
            assert not np.array_equal(want[c], lim[c]) and positivity_root_tie(dg, lim[c], ref[c], EPS), c
        assert len(bad) <= 3 + nx * ny // 20000
    # the pass and the limit applied on read are one kernel on one state
    assert np.array_equal(got[1], ref)


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_tvb_pass_on_a_tall_mesh_every_cell(bc):
    """FP32 TVB pass alone on 130 x 2000: every cell within the FP32 band
    of the oracle, except where a decision sits within FP32 rounding of a
    tie."""
    nx, ny = 130, 2000
    u = _state(nx, ny, "f32")
    gs, dg = make_pair_2d(nx, ny, (0, 1, 0, ny / 37.0), 2, "P", "euler", "ssprk3", BCS[bc], "f32")
    gs.set_state(to_planes(u), 0.0)
    gs.limit(M_TVB)
    gs.apply_limit()
    got = from_planes(gs.get_state())
    assert gs.sync() == (0, 0)
    gs.close()
    want, flags = tvb_limit(dg, u, M_TVB, 0.0)
    assert 0.2 < flags.mean() < 0.5
    scale = np.max(np.abs(want), axis=(0, 1, 3))
    bad = np.argwhere(np.any(np.abs(got - want) > 2e-6 * scale[None, None, :, None], axis=(2, 3)))
    for (cy, cx) in bad:
        assert tvb_margin(dg, u, 0.0, M_TVB, [(int(cy), int(cx))]) < 1e-4, (cy, cx)
    assert len(bad) <= 3
