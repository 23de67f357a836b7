"""gift_density (Eq. 5) against the oracle: the quantised integer bin sums
are bit-exact (the same FP64 geometry and rounding on both sides, integer
sums in any order), so densities and overflows are identical."""
import math

import numpy as np
import pytest

import oracle
from paper_2502_17632_gb300 import gift, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gift.gift_ctx_create(0)
    yield c
    gift.gift_ctx_destroy(c)


def placements():
    nl, _ = synth.workload("plain-10k")
    uni = synth.make_signals(nl, 3, 11)  # uniform over the die, 3 signals
    cen = synth.make_signals(nl, 1, 12, mode="centre")  # the paper's N(0, 1) around the die centre
    off = uni[:, :1] * 1.4 - 200.0  # a fifth of the cells off the die
    return {"uniform": uni, "clustered": np.ascontiguousarray(cen, dtype=np.float32),
            "off-die": np.ascontiguousarray(off, dtype=np.float32)}


PLACEMENTS = placements()


@pytest.mark.parametrize("name", sorted(PLACEMENTS))
@pytest.mark.parametrize("bins", [(1, 1), (7, 5), (32, 32), (128, 100)])  # the last exceeds the shared histogram
@pytest.mark.parametrize("sizes", ["unit", "per-cell"])
@pytest.mark.parametrize("device", [True, False])
def test_density_bit_exact(ctx, name, bins, sizes, device):
    xy = PLACEMENTS[name]
    N = xy.shape[0]
    kw = {"unit": (3.0, 2.5)}
    if sizes == "per-cell":
        u = synth.uniform(9, synth.T_MISC, np.arange(2 * N, dtype=np.uint64)).reshape(2, N)
        kw = {"cell_w": (1.0 + 9.0 * u[0]).astype(np.float32), "cell_h": (0.5 + 4.0 * u[1]).astype(np.float32)}
    die = (0.0, 0.0, 1000.0, 1000.0)
    _, want, want_ov = oracle.density(xy, die, bins[0], bins[1], 0.02, **kw)
    if device:
        kwd = dict(kw)
        if "cell_w" in kwd:
            kwd = {"cell_w": torch.from_numpy(kw["cell_w"]).cuda(), "cell_h": torch.from_numpy(kw["cell_h"]).cuda()}
        got, ov = gift.gift_density(ctx, torch.from_numpy(xy).cuda(), die, bins, 0.02, **kwd)
    else:
        got, ov = gift.gift_density(ctx, xy, die, bins, 0.02, **kw)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(ov, want_ov)


def test_density_invalid_arguments(ctx):
    xy = PLACEMENTS["uniform"]
    for die, bins in [((0, 0, 0, 10), (4, 4)), ((0, 0, 10, 10), (0, 4)), ((0, 0, 10, 10), (5000, 5000))]:
        with pytest.raises(gift.GiftError) as e:
            gift.gift_density(ctx, xy, die, bins)
        assert e.value.status == gift.GIFT_ERR_INVALID
    with pytest.raises(gift.GiftError):
        gift.gift_density(ctx, xy, target=-1.0)
    with pytest.raises(gift.GiftError):
        gift.gift_density(ctx, xy, cell_w=np.ones(xy.shape[0], np.float32))
    assert math.isfinite(gift.gift_density(ctx, xy)[1][0])
