"""The seeded input generators: the direct patch-array form of the
Orszag-Tang input (used by the benchmark at 512^3, where the global 3-D
fields would take tens of GB) equals the global-field form cut into patches,
bit for bit."""
import numpy as np
import pytest

from paper_1705_10774_gb300 import ics


@pytest.mark.parametrize("patches,n", [(2, 8), (3, 8), (2, 32), (4, 16)])
def test_orszag_tang_patches_equal_the_global_fields_cut_into_patches(patches, n):
    lay, f = ics.config_orszag_tang(patches=patches, n=n)
    a = ics.to_patches(lay, f)
    lay2, b = ics.orszag_tang_patches(patches=patches, n=n)
    assert np.array_equal(lay.n, lay2.n) and np.array_equal(lay.lo, lay2.lo)
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and np.array_equal(x, y)
