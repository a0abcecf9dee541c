"""The seeded input generators shared by the oracle, the tests and the bench."""
import numpy as np

import sfac_inputs as I


def test_splitmix64_published_outputs():
    # First outputs of SplitMix64 for seeds 0 and 1234567 as printed with the
    # published reference generator (Steele-Lea-Flood 2014, variant-13 mixer).
    assert [int(x) for x in I.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x) for x in I.splitmix64(1234567, 2)] == [
        6457827717110365317, 3203168211198807973]


def test_uniform_range_offsets_and_determinism():
    u = I.uniform01(5, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    np.testing.assert_array_equal(I.uniform01(5, 10, start=7), u[7:17])
    v = I.uniform(9, 1000, -0.9, 0.9)
    assert v.min() >= -0.9 and v.max() <= 0.9


def test_problem_grid_and_layout():
    p = I.Problem(n=(4, 3), alpha=(1.5, 1.5), eps=0.1, tau=0.1, a=0.0, b=2.0)
    assert p.shape == (3, 4) and p.points == 12
    np.testing.assert_allclose(p.nodes(0), 0.4 * np.arange(1, 5))
    x1, x2 = p.mesh()
    assert x1[0, 1] > x1[0, 0] and x2[1, 0] > x2[0, 0]      # axis 1 fastest


def test_config_fields():
    u = I.config1_u0()
    assert u.shape == (64, 64) and np.abs(u).max() <= 0.9
    p = I.Problem(n=(32, 32), alpha=(1.3, 1.7), eps=0.05, tau=1e-3)
    u2 = I.config2_u0(p)
    assert np.abs(u2).max() <= 0.95 + 1e-12
    inst = I.batched_instances(16)
    assert all(pp.n[0] in I.BATCH_SIZES and 50 <= pp.steps <= 500 for _, pp in inst)
    reqs = I.serving_stream(50)
    assert all(r.arrival_s > 0 for r in reqs)
    assert np.all(np.diff([r.arrival_s for r in reqs]) > 0)
