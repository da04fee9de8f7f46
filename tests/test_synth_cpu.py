"""The porous-medium generators of synth/: which pore clusters carry flow."""
import numpy as np

import synth


def _box(n=8):
    return np.zeros((n, n, n), dtype=bool)      # [z, y, x]


def test_straight_tube_percolates_in_both_senses():
    pore = _box()
    pore[3, 4, :] = True
    for fn in (synth.percolating_pores, synth.periodic_percolating_pores):
        kept, ok = fn(pore)
        assert ok and np.array_equal(kept, pore)


def test_tube_that_does_not_meet_its_periodic_image():
    # enters at y = 1, leaves at y = 5: it touches both x faces, but across the periodic
    # boundary (x = 7 -> x = 0, same y, z) it meets solid, so no flow passes through the box
    pore = _box()
    pore[3, 1, :4] = True
    pore[3, 1:6, 3] = True
    pore[3, 5, 3:] = True
    kept, ok = synth.percolating_pores(pore)
    assert ok and np.array_equal(kept, pore)
    kept, ok = synth.periodic_percolating_pores(pore)
    assert not ok and not kept.any()


def test_blocked_tube_and_isolated_pocket():
    pore = _box()
    pore[3, 4, :] = True
    pore[3, 4, 5] = False                        # one solid voxel blocks the tube
    assert not synth.periodic_percolating_pores(pore)[1]
    pore[3, 4, 5] = True
    pore[6, 1, 2:4] = True                       # a pocket that touches no face
    pore[1, 1, 0] = True                         # a pore on the x = 0 face, on its own
    kept, ok = synth.periodic_percolating_pores(pore)
    assert ok
    expected = _box()
    expected[3, 4, :] = True
    assert np.array_equal(kept, expected)


def test_winding_path_through_the_periodic_boundary():
    # the path leaves through x = 7 at y = 2, re-enters at x = 0 and returns to y = 2
    # by a detour through y = 4
    pore = _box()
    pore[2, 2, 5:] = True
    pore[2, 2, :3] = True
    pore[2, 2:5, 2] = True
    pore[2, 4, 2:6] = True
    pore[2, 2:5, 5] = True
    kept, ok = synth.periodic_percolating_pores(pore)
    assert ok and np.array_equal(kept, pore)


def test_warm_start_samples_percolate_periodically():
    from paper_2506_17713_gb300.warmstart import sample_solid
    for seed, phi in ((5009, 0.11), (5012, 0.12), (5000, 0.3)):
        solid = sample_solid(24, seed, phi)
        pore = solid == 0
        kept, ok = synth.periodic_percolating_pores(pore)
        assert ok and np.array_equal(kept, pore)


def test_workload_wetting_parameters_are_the_calibrated_ones():
    # the virtual-density factors the porous and sphere-pack workloads use are the ones
    # tests/golden/make_wetting_calibration.py found with the oracle for 45 and 30 degrees
    import json
    import os
    from synth import cases
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "wetting_calibration.json")) as fh:
        cal = json.load(fh)
    assert cal["two_component"]["theta_set"] == 45.0 and cal["pr08"]["theta_set"] == 30.0
    assert abs(cases.WET_PHI_45 - cal["two_component"]["phi"]) < 1e-9
    assert abs(cases.WET_PHI_30_PR08 - cal["pr08"]["phi"]) < 1e-9
    c = cases.porous_two_component(shape=(24, 12, 10), buffer=3, porosity=0.7)[0]
    assert c["wet_phi"][0] == cases.WET_PHI_45
    b = cases.sphere_pack_batch(count=1, edge_lo=24, edge_hi=24)[0][0]
    assert b["wet_phi"][0] == cases.WET_PHI_30_PR08
