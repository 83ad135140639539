"""All three opt-in steps at the benchmark size: the 2M-row skewed LP with
30k planted parallel columns and 174k free singleton columns, presolved with
parallel columns, column singletons and dual fixing, every output compared
with the oracle (marked slow: about a minute of host time)."""
import numpy as np
import pytest

import oracle
from parity import compare
from paper_2609_16182_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2609_16182_gb300 import lpp  # noqa: E402


@pytest.mark.slow
def test_full_size_all_opt_in_steps():
    lp = synth.plant_col_singletons(synth.plant_parallel_cols(synth.skewed(0), 0), 0, frac=0.3, free_frac=1.0,
                                    cost_scale=0.0)
    kw = dict(parallel_cols=1, col_singletons=1, dual_fixing=1)
    g = lpp.presolve(lp, **kw)
    o = oracle.presolve(lp, oracle.default_opts(**kw))
    compare(g, o, lp)
    assert np.count_nonzero(g.col_kind == lpp.COL_PARALLEL) > 30_000
    assert np.count_nonzero(g.row_kind == lpp.ROW_SUBST) > 100_000
