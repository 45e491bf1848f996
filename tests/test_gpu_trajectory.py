"""Many GPU iterations in a row (deferred dual updates, activity bits,
worklists, graph replay) against the FP64 oracle run from the same initial
state: the residual history and the final iterate agree."""
import numpy as np
import pytest

import workloads
from oracle import twa

import _parity as par

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,n", [("square48_walls", 200), ("circle100", 60)])
def test_residual_history_follows_the_oracle(name, n):
    import paper_1311_4527_gb300 as pk
    inst = workloads.small_square(48, 8, seed=3) if name == "square48_walls" else workloads.circle100()
    prob = twa.Problem.from_instance(inst)
    L = par.scale_of(prob)
    st = twa.initial_state(prob)
    pl = pk.Planner.from_instance(inst)
    for k in range(n):
        st, info = twa.iterate(prob, st)
        r = pl.iterate(1, residual=True)
        assert abs(r - info.residual) <= 2e-3 * info.residual + 1e-5 * L, (k, r, info.residual)
    z = pl.trajectory().cpu().numpy()
    pl.close()
    assert np.abs(z - st.z).max() <= 1e-3 * L
