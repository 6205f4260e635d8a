"""Quality side report: the SNR columns run end to end on the GPU."""
import math

import pytest

from paper_1212_2245_b300 import quality

pytestmark = pytest.mark.gpu


def test_quality_columns_run_and_restore(lib):
    cases = quality.default_cases()
    for c in (cases[0], cases[3]):
        row = quality.evaluate(c)
        assert all(math.isfinite(v) for v in row.values())
        # the iterations improve on their starting points: RRRL on the
        # blurred image, WR3L on the (periodic) Wiener filter
        assert row["RRRL 30 it."] > row["blurred"], row
        assert row["WR3L 5 it."] > row["Wiener (K=0.006)"], row
