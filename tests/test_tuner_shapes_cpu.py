"""The launch shapes that `dslash_bench --sweep` pins one after another obey the rules the
library's shape setters enforce (hisq_tune_set, hisq_tune_set_block, hisq_tune_set_groups,
hisq_tune_set_block_groups in include/hisq.h), so a sweep never stops on a refused shape."""
import pytest

from paper_2306_01098_gb300 import dslash_bench


@pytest.mark.parametrize("prec", ["f64", "f64x", "f32", "f16"])
@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 8, 12, 16])
def test_sweep_shapes_are_accepted_shapes(prec, nrhs):
    shapes = dslash_bench.shapes(prec, nrhs)
    assert shapes, "every key has at least one shape"
    cap = 4 if prec in ("f64", "f64x") else 8
    seen = set()
    for nr, ds, order, bs, rg, wg in shapes:
        assert (nr, ds, order, bs, rg, wg) not in seen
        seen.add((nr, ds, order, bs, rg, wg))
        assert nr in (1, 2, 4, 8) and nr <= cap and nrhs % nr == 0
        assert ds in (1, 2, 4) and order in (0, 1) and bs in (64, 128, 256)
        assert rg in (1, 2, 4) and wg in (1, 2, 4)
        assert rg == 1 or wg == 1, "site groups and block groups are not combined"
        if rg > 1:
            assert ds == 1 and nr <= 4 and nrhs % (nr * rg) == 0
        if wg > 1:
            assert ds == 1 and nr <= 4 and nrhs % (nr * wg) == 0 and bs // wg >= 32
    # one thread per site with one right-hand side per thread is always among them
    assert any(s[:2] == (1, 1) and s[4:] == (1, 1) for s in shapes)


def test_sweep_includes_block_groups_where_they_apply():
    shapes = dslash_bench.shapes("f32", 8)
    assert (4, 1, 0, 128, 1, 2) in shapes and (2, 1, 1, 256, 1, 4) in shapes
    assert not any(s[5] == 4 and s[3] == 64 for s in shapes)      # 16 threads per slice
    assert not any(s[0] == 4 and s[5] == 4 for s in shapes)       # 16 right-hand sides > 8
