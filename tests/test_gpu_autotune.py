"""lpb_autotune: times candidate schedules on a batch, stores the winner in the handle and in a
table file; a fresh handle loads the entry instead of re-timing; solves that use the tuned
schedule keep parity with the oracle."""
import numpy as np
import pytest

import synth
from lp_helpers import compare, host, to_device

pytestmark = pytest.mark.gpu


def test_autotune_table_roundtrip_and_parity(tmp_path):
    from paper_1609_08114_gb300 import Solver
    sb = synth.mixed_sizes(400, seed=17, lo=8, hi=180)
    dev = to_device(sb)
    table = tmp_path / "tune.txt"
    s1 = Solver(0)
    ms = s1.autotune(dev, prec="fp32_refine", table_path=table)
    assert ms > 0
    lines = table.read_text().strip().splitlines()
    assert len(lines) == 1 and lines[0].startswith("lpb-tune ")
    got = host(s1.solve(dev, prec="fp32_refine"))
    compare(sb, got, obj_rtol=1e-8)
    s2 = Solver(0)
    assert s2.autotune(dev, prec="fp32_refine", table_path=table) == 0.0    # loaded, not timed
    assert len(table.read_text().strip().splitlines()) == 1
    got2 = host(s2.solve(dev, prec="fp32_refine"))
    assert np.array_equal(got2["status"], got["status"])
    np.testing.assert_allclose(got2["obj"], got["obj"], rtol=1e-12, atol=0)
