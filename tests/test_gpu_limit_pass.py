"""The limiter pass (TVB-minmod in characteristic fields, then the positivity
scaling; Sec. 2.3 / Remark 2.2) on the GPU against the FP64 oracle, on a
state where both act (about a third of the cells troubled, the positivity
scaling changing about 2 % of them): periodic and outflow meshes, FP64 and
FP32, a ragged last tile of 128 columns (nx = 132 and 130), run through
crkdg_apply_limit (the pass as the default limit mode runs it before a step)
and through get_state (the pending limit applied on read)."""
import numpy as np
import pytest

import crkdg_inputs as inp
from oracle.limiter import positivity_limit, tvb_limit
from tests.pairing import from_planes, make_pair_2d, rel_err, to_planes, tvb_margin

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
@pytest.mark.parametrize("nx", [132, 130])
def test_limit_pass_with_positivity_matches_the_oracle(prec, bc, nx):
    ny = 37
    u = _state(nx, ny, prec)
    got = []
    for apply_now in (True, False):
        gs, dg = make_pair_2d(nx, ny, (0, 1, 0, 1), 2, "P", "euler", "ssprk3", BCS[bc], prec)
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
        # FP32 decisions: a cell may differ from the FP64 oracle only where a
        # TVB-minmod decision sits within FP32 rounding of a tie
        scale = np.max(np.abs(want), axis=(0, 1, 3))
        bad = np.argwhere(np.any(np.abs(ref - want) > 2e-6 * scale[None, None, :, None], axis=(2, 3)))
        for (cy, cx) in bad:
            assert tvb_margin(dg, u, 0.0, M_TVB, [(int(cy), int(cx))]) < 1e-4, (cy, cx)
        assert len(bad) <= 3
    # the pass and the limit applied on read are one kernel on one state
    assert np.array_equal(got[1], ref)
