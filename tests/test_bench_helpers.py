"""Host helpers of bench.py (no GPU): the closed-form count check that makes a benchmark run
fail on a wrong eigenvalue count."""
import numpy as np
import pytest

import bench
from closed_form import count_in, lap_eigs


@pytest.mark.parametrize("dim,nx,a,b", [(2, 30, 0.5, 0.9), (3, 14, 1.0, 1.4), (3, 10, 0.0, 12.0)])
def test_laplacian_count_equals_the_closed_form(dim, nx, a, b):
    e = lap_eigs(dim, nx)
    for rc in (False, True):
        assert bench.laplacian_count(dim, nx, a, b, rc) == count_in(e, a, b, rc)


def test_check_counts_accepts_exact_and_rejects_wrong_counts():
    e = lap_eigs(3, 12)
    d = np.unique(np.round(e, 12))
    a, b = float(0.5 * (d[10] + d[11])), float(0.5 * (d[40] + d[41]))
    exact = count_in(e, a, b, False)
    recs = [{"slice": 0, "a": a, "b": b, "nev": exact}]
    bench.check_counts(recs, 3, 12, nslices=2)
    assert recs[0]["exact"] == exact
    with pytest.raises(RuntimeError):
        bench.check_counts([{"slice": 0, "a": a, "b": b, "nev": exact - 1}], 3, 12, nslices=2)
    # the last slice is closed: an eigenvalue at its right end counts
    top = float(d[41])
    last = [{"slice": 1, "a": a, "b": top, "nev": count_in(e, a, top, True)}]
    bench.check_counts(last, 3, 12, nslices=2)
