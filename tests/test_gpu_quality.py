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


@pytest.mark.parametrize("index", [0, 3])
def test_quality_columns_equal_the_oracle_restorations(lib, index):
    """Every SNR column of the report (Sec. 3.1 definition, the paper's SNR
    table columns) against the same restoration computed by the FP64 oracle
    and scored by the oracle's SNR: box15 and the 30-degree line with
    salt-and-pepper noise, to 0.01 dB."""
    import dataclasses

    import oracle

    c = quality.default_cases()[index]
    p = c.params
    f0 = oracle.condition_input(c.f, p.pos_floor)
    rl = dataclasses.replace(p, phi_robust=0, alpha=0.0)
    ref = {"blurred": oracle.snr_db(c.f, c.g),
           f"Wiener (K={p.K})": oracle.snr_db(oracle.wr3l(c.f, c.h, p, 0)[0], c.g),
           "RL 30 it.": oracle.snr_db(oracle.rrrl(f0, f0, c.h, rl, 30), c.g)}
    for n in (5, 30, 100):
        ref[f"RRRL {n} it."] = oracle.snr_db(oracle.rrrl(f0, f0, c.h, p, n), c.g)
    ref["WR3L 5 it."] = oracle.snr_db(oracle.wr3l(c.f, c.h, p, 5)[1], c.g)
    row = quality.evaluate(c)
    assert set(row) == set(ref)
    for k, v in ref.items():
        assert abs(row[k] - v) <= 0.01, f"{c.name} {k}: report {row[k]:.4f} dB, oracle {v:.4f} dB"
