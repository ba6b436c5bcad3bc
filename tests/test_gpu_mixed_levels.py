"""Mixed form against its exact model, entry by entry, at a known slice level.

Each case (tests/levels_case.py) is dense, so no product is skipped, and its
delta makes exactly one level L* the fewest whose charge fits in delta / 2. The
kernel must select L*, report a charge inside the bracket the CPU model gives for
it, and return the exact level-L* product (oracle/mixed_ref.py) up to the float64
rounding of its pass sums -- a bar that a level set off by one misses on nearly
every entry (checked on the CPU by tests/test_mixed_model.py). Levels 4, 5 and 6
cover one pass (2..4, 2..5) and two passes (6..6 added to 2..5), the plain
product, both SP2 branches with their mirrored blocks, and a ragged grid."""
import numpy as np
import pytest

import levels_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gctx():
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    if not ctx.supports("mixed", 64):
        pytest.fail("mixed-precision leaf products are not available on this device")
    return ctx


@pytest.mark.parametrize("case", levels_case.CASES, ids=lambda c: f"{c[0]}-n{c[1]}-L{c[3]}")
def test_level_product_matches_exact_model(gctx, case):
    c = levels_case.build(*case)
    G = gctx.from_dense(c.A, levels_case.BS)
    if c.kind == "plain":
        H = gctx.from_dense(c.B, levels_case.BS)
        C, rep = gctx.multiply(G, H, c.delta, prec="mixed")
        assert rep["kept"] == rep["candidates"]
    else:
        C, rep = gctx.sp2_step(G, 0 if c.kind == "sp2_0" else 1, delta=c.delta, prec="mixed")
    assert rep["lmax"] == c.level
    assert c.charge_lo * (1 - 1e-9) <= rep["bound_round"] <= c.charge_hi
    assert rep["bound_round"] <= rep["bound"] * (1 + 1e-12) and rep["bound"] < c.delta
    got = C.to_numpy()
    diff = np.abs(got - c.expected)
    bad = diff > c.tol
    assert not bad.any(), (int(bad.sum()), float((diff / c.tol).max()))
    if c.kind != "plain":
        np.testing.assert_array_equal(got, got.T)
