"""Autotuner: selection logic on the host, and one tuning run on the GPU."""
import numpy as np
import pytest

from paper_1309_4018_b300 import autotune as AT


def test_pick_fastest_within_target_else_most_accurate():
    m = [({"a": 1}, 3.0, 1e-6), ({"a": 2}, 1.0, 5e-4), ({"a": 3}, 2.0, 4e-5), ({"a": 4}, 1.5, 6e-5)]
    assert AT.pick(m, 1e-4, safety=2.0)[0] == {"a": 3}        # 4e-5 <= 5e-5; 6e-5 is not
    assert AT.pick(m, 1e-4, safety=1.0)[0] == {"a": 4}
    assert AT.pick(m, 1e-7)[0] == {"a": 1}                    # nothing qualifies: most accurate


def test_size_classes_and_schedule_lookup():
    assert AT.size_class(8192) == 13 and AT.size_class(16383) == 13 and AT.size_class(16384) == 14
    s = AT.Schedule({13: AT.Choice(0.6, 4, 200, 0.0, 0.0), 15: AT.Choice(0.5, 6, 300, 0.0, 0.0)})
    mk = lambda n: {"surfaces": [{"tris": np.zeros((n, 3), np.int32)}]}
    assert s.params_for(mk(10000)) == dict(theta=0.6, P=4, ncrit=200, p2p_tile=64)
    assert s.params_for(mk(40000)) == dict(theta=0.5, P=6, ncrit=300, p2p_tile=64)
    assert s.params_for(mk(20000))["ncrit"] in (200, 300)     # nearest tuned class
    assert s.params_for(mk(300000)) == dict(theta=0.5, P=6, ncrit=300, p2p_tile=64)


@pytest.mark.gpu
def test_tuned_setting_meets_the_target():
    from gpu_util import ctx
    from paper_1309_4018_b300 import pbbem
    from synth.configs import fleet_ligand
    d = fleet_ligand(0, 600)
    cands = AT.candidates(((0.7, 3), (0.5, 6)), (100, 300))
    ref_pb = pbbem.Problem.from_dict(ctx(), d)
    ref_pb.setup(precision="mixed", **AT.REFERENCE)
    ref = ref_pb.solve().dG_solv
    ref_pb.close()
    c = AT.tune(ctx(), d, target=1e-4, cands=cands, reference=ref)
    assert c.rel_error <= 5e-5 and c.p2p_tile in AT.P2P_TILES
    pb = pbbem.Problem.from_dict(ctx(), d)
    pb.setup(precision="mixed", gmres_tol=1e-4, **c.params())
    assert abs(pb.solve().dG_solv - ref) <= 1e-4 * abs(ref)
    pb.close()


@pytest.mark.gpu
def test_p2p_tile_does_not_change_the_result():
    # every (target, leaf) record is the same sum whatever the number of targets per work item
    from gpu_util import problem
    from synth.configs import fleet_ligand
    d = fleet_ligand(1, 500)
    e = [problem(d, precision="mixed", gmres_tol=1e-5, p2p_tile=t).solve().dG_solv for t in (64, 48, 32, 16, 8, 5)]
    assert e[1:] == e[:-1]
