"""Batches of uneven problems: members imported at an oracle iterate match the
FP64 oracle's next iterate entry by entry; every member of a batch follows
exactly the iterates of the same problem solved alone (bit for bit: the
per-factor arithmetic is the same and the consensus sums are exact), whatever
launch shape the autotuner picks; and a batch solve stops each member where
its own solve stops."""
import numpy as np
import pytest

import workloads
from oracle import twa

import _parity as par

pytestmark = pytest.mark.gpu


def _members():
    insts = [m for m in workloads.batch_instances(40, seed=77) if m.p <= 96][:10]
    insts.append(workloads.small_square(40, 5, seed=12))              # walls
    insts.append(workloads.circle_swap(6, 1, 0.1, 0.01, 13))          # eta = 1
    insts.append(workloads.circle_swap(1, 4, 0.1, 0.0, 14))           # one agent
    return insts


def _alone(inst, iters):
    import paper_1311_4527_gb300 as pk
    with pk.Planner.from_instance(inst) as pl:
        pl.iterate(iters)
        return pl.trajectory().cpu().numpy()


def test_batch_members_match_single_planners_bit_for_bit():
    import paper_1311_4527_gb300 as pk
    insts = _members()
    with pk.PlannerBatch(insts) as B:
        B.iterate(37)
        zb = [B.trajectory(b).cpu().numpy() for b in range(len(insts))]
        choice = B.autotune(4)          # real iterations under other shapes
        assert choice["rows_per_warp"] in (4, 8, 16, 32)
        # the autotuner first aligns to an even iteration (37 -> 38), then per
        # candidate runs one graph's worth (2 or 8) plus the timed iterations
        # (4 rounded to whole graphs: 4 or 8): 4 x 3 shapes x (2 + 4 + 8 + 8)
        done = 38 + 12 * (2 + 4 + 8 + 8)
        B.iterate(11)
        zc = [B.trajectory(b).cpu().numpy() for b in range(len(insts))]
    for b, inst in enumerate(insts):
        assert np.array_equal(zb[b], _alone(inst, 37)), b
    # after autotuning the batch has advanced by a known, shape-independent count
    for b, inst in enumerate(insts[:4]):
        assert np.array_equal(zc[b], _alone(inst, done + 11)), b


def test_batch_solve_stops_members_where_their_own_solves_stop():
    import paper_1311_4527_gb300 as pk
    insts = [workloads.circle4()] + [m for m in workloads.batch_instances(30, seed=5) if m.p <= 40][:5]
    for m in insts:
        m.max_iter = 1200
    with pk.PlannerBatch(insts, check_every=10) as B:
        its, res, nconv = B.solve()
        zb = [B.trajectory(b).cpu().numpy() for b in range(len(insts))]
    assert nconv >= 1 and its[0] == 590 and res[0] < insts[0].tol
    for b, inst in enumerate(insts):
        with pk.Planner.from_instance(inst, check_every=10) as pl:
            conv, it, r = pl.solve()
            z = pl.trajectory().cpu().numpy()
        assert it == its[b], (b, it, its[b])
        assert np.array_equal(z, zb[b]), b


@pytest.mark.parametrize("rows", [4, 32])
def test_every_test_pass_shape_gives_the_same_iterates(rows):
    """The row-per-lane collision test (rows_per_warp = 32) and the
    rows-per-warp one take identical decisions and store identical state."""
    import paper_1311_4527_gb300 as pk
    insts = _members()
    with pk.PlannerBatch(insts) as B:
        B.set_shape(rows, 2, 2)
        B.iterate(24)
        zb = [B.trajectory(b).cpu().numpy() for b in range(len(insts))]
    for b, inst in enumerate(insts):
        assert np.array_equal(zb[b], _alone(inst, 24)), b


def test_batch_members_match_the_oracle_from_an_imported_iterate():
    """A mixed batch (walls, eta = 1, p = 1, the p = 100 circle and two
    uneven members): the walled member and the p = 100 member get the
    oracle's iterate 6, the batch takes one iteration (every member moves),
    and both are compared with the oracle's next iterate entry by entry.
    Back weights are those of the energy problem (rho0 inside, infinite at
    the fixed ends; batches run no other), so the oracle's are used."""
    import paper_1311_4527_gb300 as pk
    insts = [workloads.small_square(40, 5, seed=12), workloads.circle_swap(6, 1, 0.1, 0.01, 13),
             workloads.circle_swap(1, 4, 0.1, 0.0, 14), workloads.circle100()]
    insts += [m for m in workloads.batch_instances(20, seed=31) if m.p <= 64][:2]
    probs = [twa.Problem.from_instance(m) for m in insts]
    chosen = (0, 3)
    states = {b: par.oracle_state(probs[b], 6) for b in chosen}
    with pk.PlannerBatch(insts) as B:
        B.iterate(3)
        for b in chosen:
            st = states[b]
            B.import_state(b, st.z, st.u_coll, st.u_kin, st.u_wall)
        B.iterate(1)
        got = {b: {k: v.cpu().numpy() for k, v in B.export_state(b).items()} for b in chosen}
    for b in chosen:
        new, info = twa.iterate(probs[b], states[b], record_branches=True)
        gpu = dict(got[b], wback=new.wback)
        stats = par.compare(probs[b], new, info, gpu)
        assert stats["coll_active"] > 0 and stats["coll_compared_active"] > 0, (b, stats)

